// sd_packed.cu -- sd_step_packed: one SSP-RK3 step of many independent solves
// with shared launches (the serving path).
//
// Requests are grouped by order N.  Per call the packer writes, for every
// request, the parameters of its trace (+lambda) launch and of its three stage
// launches into pinned host tables, copies them to the device in one transfer,
// and launches: lambda reset, one packed trace kernel per N, one step-control
// kernel (all requests), then for each stage one packed stage kernel per N (the
// last one in the exact form).  A CTA of a packed kernel finds its request by
// binary search in the element offsets of its group and copies its parameters
// to shared memory; an order with a single request takes the plain kernels
// instead, with the parameters passed by value (the same arithmetic and bits).
//
// A request's `traces` scratch holds three trace buffers A, B, C and its 16
// partial maxima of lambda.  The trace pass writes A; stage 0 reads A and writes
// B, stage 1 reads B and writes C, stage 2 reads C and, with
// SD_REQ_KEEP_TRACES, writes A and the maxima again for the next call, which
// with SD_REQ_TRACES_READY then skips its trace pass (its CTAs return at once).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "sd_internal.h"

namespace sd {
cudaError_t launch_packed_mixed(int N, int kind, const StageParams* tab, const int64_t* off, int n_req,
                                int64_t blocks, const Ops<float>& ops, const Ops2& o2, cudaStream_t s);
cudaError_t launch_stage_mixed(const sd_mesh* m, const StageParams& P, bool traces_only, cudaStream_t s);
void set_last_error(const std::string& msg);

// partial maxima of lambda per request (at the end of the request's traces scratch)
constexpr int PK_SLOTS = 16;

struct StepCtl {
  double* dyn;
  unsigned long long* slots;  // [PK_SLOTS]
  double cfl, dx_min, ch_fixed;
  int reset;  // the maxima are cleared before the trace pass (not for SD_REQ_TRACES_READY)
  int pad_;
};

__global__ void packed_reset_kernel(const StepCtl* __restrict__ ctl, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n * PK_SLOTS && ctl[i / PK_SLOTS].reset) ctl[i / PK_SLOTS].slots[i % PK_SLOTS] = 0ull;
}

// dt, c_h and lambda_max from the maxima, which are then cleared for the exact
// last stage to fill
__global__ void packed_control_kernel(const StepCtl* __restrict__ ctl, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double* dyn = ctl[i].dyn;
  unsigned long long b = 0ull;
  for (int k = 0; k < PK_SLOTS; ++k) {
    b = ctl[i].slots[k] > b ? ctl[i].slots[k] : b;
    ctl[i].slots[k] = 0ull;
  }
  const double lam = __longlong_as_double((long long)b);
  dyn[0] = ctl[i].cfl * ctl[i].dx_min / lam;
  dyn[1] = ctl[i].ch_fixed > 0.0 ? ctl[i].ch_fixed : lam;
  dyn[2] = lam;
}
}  // namespace sd

struct sd_packer {
  int cap;
  int parity;
  // double-buffered tables: [4][cap] stage parameters (trace, stage 0, 1, 2),
  // element offsets (cap + 8 groups), step-control records
  sd::StageParams* h_tab[2];
  sd::StageParams* d_tab[2];
  int64_t* h_off[2];
  int64_t* d_off[2];
  sd::StepCtl* h_ctl[2];
  sd::StepCtl* d_ctl[2];
  // copied[b]: the host tables of buffer b have reached the device (the host may
  // refill them); read[b]: the kernels of the last call on buffer b have run (the
  // device tables may be overwritten, on whichever stream the next call uses)
  cudaEvent_t copied[2];
  cudaEvent_t read[2];
  bool used[2];
  int device;
};

namespace {

sd_status pk_fail(sd_status st, const std::string& msg) {
  sd::set_last_error(msg);
  return st;
}

void free_packer(sd_packer* p) {
  for (int b = 0; b < 2; ++b) {
    if (p->h_tab[b]) cudaFreeHost(p->h_tab[b]);
    if (p->h_off[b]) cudaFreeHost(p->h_off[b]);
    if (p->h_ctl[b]) cudaFreeHost(p->h_ctl[b]);
    if (p->d_tab[b]) cudaFree(p->d_tab[b]);
    if (p->d_off[b]) cudaFree(p->d_off[b]);
    if (p->d_ctl[b]) cudaFree(p->d_ctl[b]);
    if (p->copied[b]) cudaEventDestroy(p->copied[b]);
    if (p->read[b]) cudaEventDestroy(p->read[b]);
  }
  delete p;
}

bool aligned16(const void* p) { return p && (((uintptr_t)p) & 15) == 0; }

}  // namespace

extern "C" {

sd_status sd_packer_create(int32_t max_requests, sd_packer** out) {
  if (!out) return pk_fail(SD_ERR_INVALID_ARGUMENT, "out is NULL");
  *out = nullptr;
  if (max_requests <= 0 || max_requests > (1 << 20)) return pk_fail(SD_ERR_INVALID_ARGUMENT, "max_requests out of range");
  sd_packer* p = new sd_packer();
  p->cap = max_requests;
  cudaError_t err = cudaGetDevice(&p->device);
  const size_t ntab = 4 * (size_t)max_requests, noff = (size_t)max_requests + 16;
  for (int b = 0; b < 2 && err == cudaSuccess; ++b) {
    err = cudaMallocHost((void**)&p->h_tab[b], ntab * sizeof(sd::StageParams));
    if (err == cudaSuccess) err = cudaMallocHost((void**)&p->h_off[b], noff * sizeof(int64_t));
    if (err == cudaSuccess) err = cudaMallocHost((void**)&p->h_ctl[b], max_requests * sizeof(sd::StepCtl));
    if (err == cudaSuccess) err = cudaMalloc((void**)&p->d_tab[b], ntab * sizeof(sd::StageParams));
    if (err == cudaSuccess) err = cudaMalloc((void**)&p->d_off[b], noff * sizeof(int64_t));
    if (err == cudaSuccess) err = cudaMalloc((void**)&p->d_ctl[b], max_requests * sizeof(sd::StepCtl));
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&p->copied[b], cudaEventDisableTiming);
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&p->read[b], cudaEventDisableTiming);
  }
  if (err != cudaSuccess) {
    free_packer(p);
    cudaGetLastError();
    return pk_fail(err == cudaErrorMemoryAllocation ? SD_ERR_OUT_OF_MEMORY : SD_ERR_CUDA,
                   std::string("packer allocation: ") + cudaGetErrorString(err));
  }
  *out = p;
  return SD_OK;
}

sd_status sd_packer_destroy(sd_packer* p) {
  if (!p) return SD_OK;
  for (int b = 0; b < 2; ++b)
    if (p->used[b]) {
      cudaEventSynchronize(p->copied[b]);
      cudaEventSynchronize(p->read[b]);
    }
  free_packer(p);
  return SD_OK;
}

sd_status sd_step_packed(sd_packer* pk, int32_t n, const sd_step_req* reqs, void* stream) {
  if (!pk) return pk_fail(SD_ERR_INVALID_ARGUMENT, "packer is NULL");
  if (n < 0 || n > pk->cap) return pk_fail(SD_ERR_INVALID_ARGUMENT, "request count exceeds the packer's capacity");
  if (n == 0) return SD_OK;
  if (!reqs) return pk_fail(SD_ERR_INVALID_ARGUMENT, "reqs is NULL");
  cudaGetLastError();  // a pending error of an earlier, unrelated call is not this call's
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != pk->device)
    return pk_fail(SD_ERR_INVALID_ARGUMENT, "the current device is not the packer's device");
  for (int i = 0; i < n; ++i) {
    const sd_step_req& r = reqs[i];
    const std::string where = "request " + std::to_string(i) + ": ";
    if (!r.mesh || !r.bg) return pk_fail(SD_ERR_INVALID_ARGUMENT, where + "mesh and background are required");
    if (r.bg->mesh != r.mesh) return pk_fail(SD_ERR_INVALID_ARGUMENT, where + "background belongs to another mesh");
    if (r.mesh->device != dev) return pk_fail(SD_ERR_INVALID_ARGUMENT, where + "mesh is on another device");
    if (!(r.phys.gamma > 1.0) || r.bg->gamma != r.phys.gamma)
      return pk_fail(SD_ERR_INVALID_ARGUMENT, where + "gamma must exceed 1 and match the background");
    if (!aligned16(r.q) || !aligned16(r.work) || !aligned16(r.traces) || !r.dyn || r.q == r.work)
      return pk_fail(SD_ERR_INVALID_ARGUMENT, where + "q, work, traces must be distinct 16-byte aligned buffers, dyn non-NULL");
    if (!(r.cfl > 0.0)) return pk_fail(SD_ERR_INVALID_ARGUMENT, where + "cfl must be positive");
    if (r.phys.viscous) return pk_fail(SD_ERR_UNSUPPORTED, where + "sd_step_packed takes no viscous fluxes (sd_step runs them)");
    if (r.phys.rk_scheme != SD_RK_SSP33)
      return pk_fail(SD_ERR_UNSUPPORTED, where + "sd_step_packed runs the three-stage method (rk_scheme SD_RK_SSP33)");
    if (r.flags & ~(SD_REQ_KEEP_TRACES | SD_REQ_TRACES_READY))
      return pk_fail(SD_ERR_INVALID_ARGUMENT, where + "unknown flags");
  }
  {  // the background holds the step's FP32 scratch: one request per background
    std::vector<const sd_background*> bgs(n);
    for (int i = 0; i < n; ++i) bgs[i] = reqs[i].bg;
    std::sort(bgs.begin(), bgs.end());
    if (std::adjacent_find(bgs.begin(), bgs.end()) != bgs.end())
      return pk_fail(SD_ERR_INVALID_ARGUMENT, "two requests share a background");
  }
  // group by order
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return reqs[a].mesh->N < reqs[b].mesh->N; });

  const int b = pk->parity;
  if (pk->used[b]) {
    cudaError_t err = cudaEventSynchronize(pk->copied[b]);
    if (err != cudaSuccess) return pk_fail(SD_ERR_CUDA, std::string("packer event: ") + cudaGetErrorString(err));
  }
  sd::StageParams* T = pk->h_tab[b];
  int64_t* OFF = pk->h_off[b];
  sd::StepCtl* CTL = pk->h_ctl[b];
  static const double A[3] = {0.0, 0.75, 1.0 / 3.0};
  static const double Bc[3] = {1.0, 0.25, 2.0 / 3.0};
  struct Group {
    int N, k0, k1;
    int64_t off0;  // index of the group's offsets in OFF
  };
  std::vector<Group> groups;
  int64_t off_pos = 0;
  for (int k = 0; k < n; ++k) {
    const sd_step_req& r = reqs[order[k]];
    const sd_mesh* m = r.mesh;
    if (groups.empty() || groups.back().N != m->N) {
      if (!groups.empty()) {
        Group& g = groups.back();
        g.k1 = k;
        off_pos += (g.k1 - g.k0) + 1;
      }
      groups.push_back({m->N, k, n, off_pos});
      OFF[off_pos] = 0;
    }
    Group& g = groups.back();
    OFF[g.off0 + (k - g.k0) + 1] = OFF[g.off0 + (k - g.k0)] + m->n_e;
    const int64_t trace_elems = m->n_e * 6 * 9 * (int64_t)m->N * m->N;
    float* trA = static_cast<float*>(r.traces);
    float* trB = trA + trace_elems;
    float* trC = trB + trace_elems;
    unsigned long long* slots = reinterpret_cast<unsigned long long*>(trC + trace_elems);
    const bool ready = (r.flags & SD_REQ_TRACES_READY) != 0, keep = (r.flags & SD_REQ_KEEP_TRACES) != 0;
    sd::StageParams P;
    memset(&P, 0, sizeof(P));
    P.n_e = m->n_e;
    P.stride = m->stride;
    P.plane = m->n_e * m->stride;
    P.gamma = r.phys.gamma;
    P.GM = r.phys.GM;
    P.omega = r.phys.omega;
    P.alpha = r.phys.glm_alpha;
    P.inv_gm1 = 1.0 / (r.phys.gamma - 1.0);
    P.c_h = r.phys.c_h;
    P.powell = r.phys.powell;
    P.gravity = r.phys.gravity;
    P.coriolis = r.phys.coriolis;
    for (int v = 0; v < 9; ++v) P.farfield[v] = r.phys.farfield[v];
    P.Sfam = m->Sfam32;
    P.invJ = m->invJ32;
    P.X = m->X32;
    P.nbr = m->nbr;
    P.meta = m->meta;
    P.bg = r.bg->rec;
    P.bg_jump = r.bg->jump;
    P.dyn = r.dyn;
    P.err = m->err;
    P.wait_spins = m->wait_spins;
    // trace (+lambda) of q into A (skipped when the previous call left them there)
    sd::StageParams Pt = P;
    Pt.q_in = r.q;
    Pt.tr_out = trA;
    Pt.lam_max = slots;
    Pt.lam_nslot = sd::PK_SLOTS;
    Pt.qp_out = r.bg->qp;  // q' of q for the stages
    Pt.dstride = r.bg->dstride;
    Pt.skip = ready ? 1 : 0;
    T[0 * n + k] = Pt;
    // increment form (as sd_step): every stage reads q^n and the FP32 register D
    // carries the stage states.  Stage 0: D = t, traces A -> B; stage 1: D += t,
    // B -> C; stage 2: q = q + D + t, reads C (work is not written) and, to keep
    // them, writes the traces of the new q into A
    const double* qin[3] = {r.q, r.q, r.q};
    double* qout[3] = {r.work, r.work, r.q};
    void* tin[3] = {trA, trB, trC};
    void* tout[3] = {trB, trC, keep ? trA : nullptr};
    for (int s = 0; s < 3; ++s) {
      sd::StageParams Ps = P;
      Ps.mode = sd::MODE_RK;
      Ps.rk_a = A[s];
      Ps.rk_b = Bc[s];
      Ps.q_n = r.q;
      Ps.q_in = qin[s];
      Ps.out = qout[s];
      Ps.tr_in = tin[s];
      Ps.tr_out = tout[s];
      // low-storage form (as sd_step): D = q^(s) - q^n in the background's FP32 register
      Ps.dreg = r.bg->dreg;
      Ps.dstride = r.bg->dstride;
      Ps.lsr_read = s > 0 ? 1 : 0;
      Ps.lsr_write = s == 0 ? 1 : (s == 1 ? 2 : 0);
      Ps.incr = 1;
      Ps.qp_in = r.bg->qp;
      if (s == 2 && keep) {  // lambda_max and q' of the new q for the next call
        Ps.lam_max = slots;
        Ps.lam_nslot = sd::PK_SLOTS;
        Ps.qp_out = r.bg->qp;
      }
      T[(1 + s) * n + k] = Ps;
    }
    CTL[k] = {r.dyn, slots, r.cfl, m->h_min * (m->ops64.xs[1] - m->ops64.xs[0]), r.phys.c_h, ready ? 0 : 1, 0};
  }
  off_pos += (groups.back().k1 - groups.back().k0) + 1;

  cudaStream_t s = (cudaStream_t)stream;
  // the device tables of buffer b may still be read by the kernels of the call
  // before last, which may have run on another stream
  cudaError_t err = pk->used[b] ? cudaStreamWaitEvent(s, pk->read[b], 0) : cudaSuccess;
  if (err == cudaSuccess) err = cudaMemcpyAsync(pk->d_tab[b], T, 4 * (size_t)n * sizeof(sd::StageParams), cudaMemcpyHostToDevice, s);
  if (err == cudaSuccess) err = cudaMemcpyAsync(pk->d_off[b], OFF, off_pos * sizeof(int64_t), cudaMemcpyHostToDevice, s);
  if (err == cudaSuccess) err = cudaMemcpyAsync(pk->d_ctl[b], CTL, n * sizeof(sd::StepCtl), cudaMemcpyHostToDevice, s);
  if (err == cudaSuccess) err = cudaEventRecord(pk->copied[b], s);
  if (err != cudaSuccess) return pk_fail(SD_ERR_CUDA, std::string("packer copy: ") + cudaGetErrorString(err));
  pk->used[b] = true;
  pk->parity ^= 1;

  const unsigned cblocks = (unsigned)((n + 127) / 128);
  sd::packed_reset_kernel<<<(unsigned)(((int64_t)n * sd::PK_SLOTS + 127) / 128), 128, 0, s>>>(pk->d_ctl[b], n);
  err = cudaGetLastError();
  for (size_t gi = 0; gi < groups.size() && err == cudaSuccess; ++gi) {
    const Group& g = groups[gi];
    const int ng = g.k1 - g.k0;
    bool any = false;  // a request of the group needs its trace pass
    for (int k = g.k0; k < g.k1 && !any; ++k) any = !(reqs[order[k]].flags & SD_REQ_TRACES_READY);
    if (!any) continue;
    if (ng == 1) {  // a lone request of its order: the plain kernel, parameters by value
      err = sd::launch_stage_mixed(reqs[order[g.k0]].mesh, T[0 * n + g.k0], true, s);
      continue;
    }
    const int64_t blocks = OFF[g.off0 + ng];
    err = sd::launch_packed_mixed(g.N, 0, pk->d_tab[b] + 0 * n + g.k0, pk->d_off[b] + g.off0, ng, blocks,
                                  reqs[order[g.k0]].mesh->ops32, reqs[order[g.k0]].mesh->ops2, s);
  }
  if (err == cudaSuccess) {
    sd::packed_control_kernel<<<cblocks, 128, 0, s>>>(pk->d_ctl[b], n);
    err = cudaGetLastError();
  }
  for (int st = 0; st < 3 && err == cudaSuccess; ++st)
    for (size_t gi = 0; gi < groups.size() && err == cudaSuccess; ++gi) {
      const Group& g = groups[gi];
      const int ng = g.k1 - g.k0;
      if (ng == 1) {  // the plain stage kernel: the same arithmetic, without the per-block table look-up
        err = sd::launch_stage_mixed(reqs[order[g.k0]].mesh, T[(1 + st) * n + g.k0], false, s);
        continue;
      }
      const int64_t blocks = OFF[g.off0 + ng];
      err = sd::launch_packed_mixed(g.N, st == 2 ? 2 : 1, pk->d_tab[b] + (1 + st) * n + g.k0, pk->d_off[b] + g.off0, ng,
                                    blocks, reqs[order[g.k0]].mesh->ops32, reqs[order[g.k0]].mesh->ops2, s);
    }
  if (err == cudaSuccess) err = cudaEventRecord(pk->read[b], s);
  if (err != cudaSuccess) return pk_fail(SD_ERR_CUDA, std::string("packed launch: ") + cudaGetErrorString(err));
  return SD_OK;
}

}  // extern "C"
