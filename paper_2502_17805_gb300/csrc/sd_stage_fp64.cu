// Instantiations of the fused element kernels for the FP64 policy, N = 2..8.
#include "sd_stage.cuh"

namespace sd {

cudaError_t launch_stage_fp64(const sd_mesh* m, const StageParams& P, bool traces_only, cudaStream_t s) {
  switch (m->N) {
    case 2: return launch_stage_t<2, PolFP64>(P, m->ops64, traces_only, s);
    case 3: return launch_stage_t<3, PolFP64>(P, m->ops64, traces_only, s);
    case 4: return launch_stage_t<4, PolFP64>(P, m->ops64, traces_only, s);
    case 5: return launch_stage_t<5, PolFP64>(P, m->ops64, traces_only, s);
    case 6: return launch_stage_t<6, PolFP64>(P, m->ops64, traces_only, s);
    case 7: return launch_stage_t<7, PolFP64>(P, m->ops64, traces_only, s);
    case 8: return launch_stage_t<8, PolFP64>(P, m->ops64, traces_only, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace sd
