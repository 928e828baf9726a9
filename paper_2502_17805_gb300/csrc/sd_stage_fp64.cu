// Instantiations of the FP64 kernels, N = 2..8: the face-flux and line-blocked
// element kernels of the stages, the trace kernel, and the viscous kernel (BR1
// gradient record, its face traces, the interior viscous divergence).
#include "sd_stage.cuh"
#include "sd_stage_f64.cuh"
#include "sd_viscous.cuh"

namespace sd {

template <int N>
static cudaError_t launch_fp64_n(const sd_mesh* m, const StageParams& P, bool traces_only, cudaStream_t s) {
  if (traces_only) return launch_traces_t<N, PolFP64>(P, m->ops64, s);
  return launch_stage_f64_t<N>(P, m->ops64, s);
}

cudaError_t launch_stage_fp64(const sd_mesh* m, const StageParams& P, bool traces_only, cudaStream_t s) {
  switch (m->N) {
    case 2: return launch_fp64_n<2>(m, P, traces_only, s);
    case 3: return launch_fp64_n<3>(m, P, traces_only, s);
    case 4: return launch_fp64_n<4>(m, P, traces_only, s);
    case 5: return launch_fp64_n<5>(m, P, traces_only, s);
    case 6: return launch_fp64_n<6>(m, P, traces_only, s);
    case 7: return launch_fp64_n<7>(m, P, traces_only, s);
    case 8: return launch_fp64_n<8>(m, P, traces_only, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_grad(const sd_mesh* m, const StageParams& P, cudaStream_t s) {
  switch (m->N) {
    case 2: return launch_visc_f64_t<2>(P, m->ops64, s);
    case 3: return launch_visc_f64_t<3>(P, m->ops64, s);
    case 4: return launch_visc_f64_t<4>(P, m->ops64, s);
    case 5: return launch_visc_f64_t<5>(P, m->ops64, s);
    case 6: return launch_visc_f64_t<6>(P, m->ops64, s);
    case 7: return launch_visc_f64_t<7>(P, m->ops64, s);
    case 8: return launch_visc_f64_t<8>(P, m->ops64, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace sd
