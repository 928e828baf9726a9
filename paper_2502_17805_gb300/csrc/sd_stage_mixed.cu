// Instantiations of the fused element kernels for the FP32-mixed policy, N = 2..8:
// the line-blocked stage kernel (sd_stage_v2.cuh) and the trace kernel.
#include "sd_stage.cuh"
#include "sd_stage_v2.cuh"

namespace sd {

template <int N>
static cudaError_t launch_mixed_n(const sd_mesh* m, const StageParams& P, bool traces_only, cudaStream_t s) {
  if (traces_only) return launch_traces_t<N, PolMixed>(P, m->ops32, s);
  return launch_stage_v2_t<N>(P, m->ops2, s);
}

cudaError_t launch_stage_mixed(const sd_mesh* m, const StageParams& P, bool traces_only, cudaStream_t s) {
  switch (m->N) {
    case 2: return launch_mixed_n<2>(m, P, traces_only, s);
    case 3: return launch_mixed_n<3>(m, P, traces_only, s);
    case 4: return launch_mixed_n<4>(m, P, traces_only, s);
    case 5: return launch_mixed_n<5>(m, P, traces_only, s);
    case 6: return launch_mixed_n<6>(m, P, traces_only, s);
    case 7: return launch_mixed_n<7>(m, P, traces_only, s);
    case 8: return launch_mixed_n<8>(m, P, traces_only, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_packed_mixed(int N, int kind, const StageParams* tab, const int64_t* off, int n_req,
                                int64_t blocks, const Ops<float>& ops, const Ops2& o2, cudaStream_t s) {
  switch (N) {
    case 2: return launch_packed_t<2>(kind, tab, off, n_req, blocks, ops, o2, s);
    case 3: return launch_packed_t<3>(kind, tab, off, n_req, blocks, ops, o2, s);
    case 4: return launch_packed_t<4>(kind, tab, off, n_req, blocks, ops, o2, s);
    case 5: return launch_packed_t<5>(kind, tab, off, n_req, blocks, ops, o2, s);
    case 6: return launch_packed_t<6>(kind, tab, off, n_req, blocks, ops, o2, s);
    case 7: return launch_packed_t<7>(kind, tab, off, n_req, blocks, ops, o2, s);
    case 8: return launch_packed_t<8>(kind, tab, off, n_req, blocks, ops, o2, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace sd
