// sd_noalloc.cu -- sd_residual_noalloc: the FP64 residual with its scratch in a
// fixed device array instead of the mesh's trace buffers.
//
// Some callers cannot call cudaMalloc when they need a residual: an application
// whose memory pool has already reserved the device memory it is allowed to
// use, or a latency-bound loop that must not risk the device-wide
// synchronisation an allocation can cause.  This entry point performs no
// allocation of any kind.  Its only scratch is the buffer below (the face
// traces of q, then the common face fluxes), a file-scope device array of
// kNoAllocScratchBytes that every GPU loading this library holds until the
// process exits.
#include <string.h>

#include <mutex>
#include <string>

#include "sd_internal.h"

namespace {

constexpr size_t kNoAllocScratchBytes = 8u << 20;  // 8 MiB per device
constexpr size_t kNoAllocScratchDoubles = kNoAllocScratchBytes / sizeof(double);
constexpr int kMaxDevices = 64;

// Face traces of the input state, [element][face][variable][N^2] doubles, then
// the common face fluxes [owned face][10][N^2].
static __device__ __align__(256) double g_noalloc_traces[kNoAllocScratchDoubles];

// Device address of g_noalloc_traces on each device, looked up once per device
// (with that device current) by the first call made on it.
void* g_scratch_addr[kMaxDevices];
bool g_scratch_ready[kMaxDevices];
std::mutex g_scratch_mutex;

}  // namespace

namespace sd {
cudaError_t launch_stage_fp64(const sd_mesh* m, const StageParams& P, bool traces_only, cudaStream_t s);
void set_last_error(const std::string& msg);
}  // namespace sd

namespace {
sd_status noalloc_fail(sd_status st, const std::string& msg) {
  sd::set_last_error(msg);
  return st;
}
}  // namespace

extern "C" {

sd_status sd_residual_noalloc(const sd_mesh* m, const sd_phys* ph, const double* q, double* dqdt, void* stream) {
  if (!m || !ph || !q || !dqdt) return noalloc_fail(SD_ERR_INVALID_ARGUMENT, "null argument");
  if ((((uintptr_t)q) & 15) != 0 || (((uintptr_t)dqdt) & 15) != 0)
    return noalloc_fail(SD_ERR_INVALID_ARGUMENT, "q and dqdt must be 16-byte aligned");
  if (q == dqdt) return noalloc_fail(SD_ERR_INVALID_ARGUMENT, "dqdt must not alias q");
  if (!(ph->gamma > 1.0)) return noalloc_fail(SD_ERR_INVALID_ARGUMENT, "gamma must exceed 1");
  if (ph->viscous)
    return noalloc_fail(SD_ERR_UNSUPPORTED, "viscous fluxes need gradient buffers: use sd_residual");
  const size_t N2 = (size_t)m->N * m->N;
  const size_t n_tr = ((size_t)m->n_e * 6 * 9 * N2 + 31) / 32 * 32;  // traces, then the face fluxes
  const size_t need = n_tr + (size_t)m->n_own * 10 * N2;
  if (need > kNoAllocScratchDoubles)
    return noalloc_fail(SD_ERR_INVALID_ARGUMENT,
                        "mesh too large for sd_residual_noalloc: its face traces and face fluxes need " +
                            std::to_string(need * sizeof(double)) + " bytes, the fixed scratch holds " +
                            std::to_string(kNoAllocScratchBytes) +
                            " ((n_elements * 54 + n_owned_faces * 10) * N^2 * 8 bytes)");
  cudaGetLastError();  // a pending error of an earlier, unrelated call is not this call's
  int dev = -1;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return noalloc_fail(SD_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(err));
  if (dev != m->device)
    return noalloc_fail(SD_ERR_INVALID_ARGUMENT, "the current device is not the device the mesh was built on");
  if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(SD_ERR_UNSUPPORTED, "device index out of range");
  {
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_ready[dev]) {
      void* ptr = nullptr;
      err = cudaGetSymbolAddress(&ptr, g_noalloc_traces);
      if (err != cudaSuccess || !ptr)
        return noalloc_fail(SD_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(err));
      g_scratch_addr[dev] = ptr;
      g_scratch_ready[dev] = true;
    }
  }
  double* tr = static_cast<double*>(g_scratch_addr[dev]);
  cudaStream_t s = (cudaStream_t)stream;

  sd::StageParams P;
  memset(&P, 0, sizeof(P));
  P.n_e = m->n_e;
  P.stride = m->stride;
  P.plane = m->n_e * m->stride;
  P.gamma = ph->gamma;
  P.GM = ph->GM;
  P.omega = ph->omega;
  P.alpha = ph->glm_alpha;
  P.inv_gm1 = 1.0 / (ph->gamma - 1.0);
  P.c_h = ph->c_h;
  P.powell = ph->powell;
  P.gravity = ph->gravity;
  P.coriolis = ph->coriolis;
  for (int v = 0; v < 9; ++v) P.farfield[v] = ph->farfield[v];
  P.Sfam = m->Sfam64;
  P.invJ = m->invJ64;
  P.X = m->X64;
  P.nbr = m->nbr;
  P.meta = m->meta;
  P.err = m->err;
  P.wait_spins = m->wait_spins;
  P.n_own = m->n_own;
  P.own_faces = m->own_faces;
  P.face_k = m->face_k;
  P.gface = tr + n_tr;
  // every trace and face-flux entry a kernel reads is written earlier in the
  // same call, so the scratch needs no clearing between calls
  P.q_in = q;
  P.tr_out = tr;
  err = sd::launch_stage_fp64(m, P, true, s);
  if (err != cudaSuccess) return noalloc_fail(SD_ERR_CUDA, std::string("trace kernel: ") + cudaGetErrorString(err));
  P.tr_out = nullptr;
  P.tr_in = tr;
  P.mode = sd::MODE_RESIDUAL;
  P.out = dqdt;
  err = sd::launch_stage_fp64(m, P, false, s);
  if (err != cudaSuccess)
    return noalloc_fail(SD_ERR_CUDA, std::string("residual kernel: ") + cudaGetErrorString(err));
  return SD_OK;
}

}  // extern "C"
