// Instantiations of the viscous FP32-mixed kernels (sd_mixed_visc.cuh), N = 2..8.
#include "sd_mixed_visc.cuh"

namespace sd {

cudaError_t launch_mixed_visc(const sd_mesh* m, const StageParams& Pg, const StageParams& Pv, cudaStream_t s) {
  switch (m->N) {
    case 2: return launch_mixed_visc_t<2>(Pg, Pv, m->ops32, m->ops2, s);
    case 3: return launch_mixed_visc_t<3>(Pg, Pv, m->ops32, m->ops2, s);
    case 4: return launch_mixed_visc_t<4>(Pg, Pv, m->ops32, m->ops2, s);
    case 5: return launch_mixed_visc_t<5>(Pg, Pv, m->ops32, m->ops2, s);
    case 6: return launch_mixed_visc_t<6>(Pg, Pv, m->ops32, m->ops2, s);
    case 7: return launch_mixed_visc_t<7>(Pg, Pv, m->ops32, m->ops2, s);
    case 8: return launch_mixed_visc_t<8>(Pg, Pv, m->ops32, m->ops2, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace sd
