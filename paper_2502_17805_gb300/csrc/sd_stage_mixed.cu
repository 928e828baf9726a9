// Instantiations of the fused element kernels for the FP32-mixed policy, N = 2..8.
#include "sd_stage.cuh"

namespace sd {

cudaError_t launch_stage_mixed(const sd_mesh* m, const StageParams& P, bool traces_only, cudaStream_t s) {
  switch (m->N) {
    case 2: return launch_stage_t<2, PolMixed>(P, m->ops32, traces_only, s);
    case 3: return launch_stage_t<3, PolMixed>(P, m->ops32, traces_only, s);
    case 4: return launch_stage_t<4, PolMixed>(P, m->ops32, traces_only, s);
    case 5: return launch_stage_t<5, PolMixed>(P, m->ops32, traces_only, s);
    case 6: return launch_stage_t<6, PolMixed>(P, m->ops32, traces_only, s);
    case 7: return launch_stage_t<7, PolMixed>(P, m->ops32, traces_only, s);
    case 8: return launch_stage_t<8, PolMixed>(P, m->ops32, traces_only, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace sd
