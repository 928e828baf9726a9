// sd_stage.cuh -- pieces shared by the stage kernels of both policies: the line
// and solution-point indexing of an element, the bound of the wave speeds and its
// reduction, the element load (FP64 state, or the FP32 perturbation about the
// background), the face-trace kernel (+lambda_max), and the sources M of the
// governing equations (Sec. MHD Governing Equations).
#pragma once

#include "sd_internal.h"
#include "sd_physics.cuh"

namespace sd {

template <int N>
struct Dims {
  static constexpr int N2 = N * N, N3 = N2 * N, NF = N + 1;
  static constexpr int NFACE = 6 * N2;
  static constexpr int MAXW = NFACE > N3 ? NFACE : N3;
  static constexpr int BLK = ((MAXW + 31) / 32) * 32;
};

// shared memory of the trace kernel: the state, then the extrapolation table
template <int N, class Pol>
struct Smem {
  using R = typename Pol::R;
  static constexpr int N2 = N * N, N3 = N2 * N, NF = N + 1, NV = Pol::NV;
  static constexpr int oQ = 0;
  static constexpr int oTE = NV * N3;
  static constexpr size_t trace_bytes = ((oTE + NF * N) * sizeof(R) + 15) / 16 * 16;
};

// index of solution point (i along d; a, b the other two directions in increasing order)
template <int N>
__device__ __forceinline__ int sol_index(int d, int i, int a, int b) {
  return d == 0 ? i + N * (a + N * b) : (d == 1 ? a + N * (i + N * b) : a + N * (b + N * i));
}

// solution-point index of position i along the line (d, L), L = a + N b over the
// other two directions in increasing order: base + i * stride
template <int N>
__device__ __forceinline__ void line_geom(int d, int L, int& base, int& stride) {
  const int a = L % N, b = L / N;
  if (d == 0) {
    base = N * L;
    stride = 1;
  } else if (d == 1) {
    base = a + N * N * b;
    stride = N;
  } else {
    base = L;
    stride = N * N;
  }
}

// Lines whose N values a thread reads with each pair of neighbours (i, i^1)
// swapped: the lines along xi with (L mod 32) >= 16 (rows N floats apart, which
// otherwise meet lines 16 further on in the same bank) and the lines along eta in
// odd rows.  Modelled on [v][N^3] shared-memory planes, this removes about a sixth of the
// bank conflicts of the line reads; the values reach the same registers.
template <int N>
__device__ __forceinline__ bool line_flip(int d, int L) {
  return (d == 0 && (L & 31) >= 16) || (d == 1 && ((L / N) & 1));
}

// The N values of variables a (lane x) and b (lane y) along a line, read in the
// order of line_flip and put back in order.
template <int N>
__device__ __forceinline__ void load_line(const float* a, const float* b, int base, int stride, bool flip,
                                          float2* out) {
  const int be = base + (flip ? stride : 0), bo = base - (flip ? stride : 0);
  float2 x[N];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const int o = ((i ^ 1) < N ? ((i & 1) ? bo : be) : base) + i * stride;
    x[i] = make_float2(a[o], b[o]);
  }
#pragma unroll
  for (int i = 0; i < N; ++i) out[i] = ((i ^ 1) < N && flip) ? x[i ^ 1] : x[i];
}

// Upper bound of the wave speeds at one point, |U| + sqrt(gamma p / rho + |B|^2 / rho)
// (>= |u_n| + c_f along every direction), from the full conserved state.  The
// trace kernel and the stage kernels that also return lambda_max of their output
// use these same functions, so both give the same bits for the same state.
__device__ __forceinline__ double point_speed_fp64(const double* qv, double gamma) {
  const double ir = 1.0 / qv[0];
  const double m2 = qv[1] * qv[1] + qv[2] * qv[2] + qv[3] * qv[3];
  const double B2 = qv[5] * qv[5] + qv[6] * qv[6] + qv[7] * qv[7];
  const double p = (gamma - 1.0) * (qv[4] - 0.5 * (m2 * ir + B2 + qv[8] * qv[8]));
  return sqrt(m2) * ir + sqrt(gamma * p * ir + B2 * ir);
}

// The same bound in FP32 from the FP32 rounding of the full state (mixed policy).
__device__ __forceinline__ float point_speed_mixed(const float* qf, float g) {
  const float ir = 1.0f / qf[0];
  const float m2 = qf[1] * qf[1] + qf[2] * qf[2] + qf[3] * qf[3];
  const float B2 = qf[5] * qf[5] + qf[6] * qf[6] + qf[7] * qf[7];
  const float p = (g - 1.0f) * (qf[4] - 0.5f * (m2 * ir + B2 + qf[8] * qf[8]));
  return sqrtf(m2) * ir + sqrtf(g * p * ir + B2 * ir);
}

// Running maximum that keeps a NaN (a non-physical state must not pass unseen).
__device__ __forceinline__ double speed_max(double lam, double l) { return (l > lam || l != l) ? l : lam; }
__device__ __forceinline__ float speed_max(float lam, float l) { return (l > lam || l != l) ? l : lam; }

// Maximum over the warp, then one atomic per warp into one of nslot (a power of
// two) partial maxima, so that the atomics of a launch spread over several
// addresses instead of queueing on one; the step-control kernel reduces the
// slots.  Positive doubles order like their bit patterns, and a NaN (all
// exponent bits set) is above every finite value.
template <typename R>
__device__ __forceinline__ void speed_reduce(R lam, unsigned long long* dst, int nslot) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) lam = speed_max(lam, __shfl_xor_sync(0xffffffffu, lam, o));
  if ((threadIdx.x & 31) == 0) {
    const unsigned warp = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const unsigned slot = nslot > 1 ? warp & (unsigned)(nslot - 1) : 0u;
    atomicMax(dst + slot, (unsigned long long)__double_as_longlong((double)lam));
  }
}

// Load one element's state into shared memory.  Mixed policy: q' = q - Q0 with
// the subtraction in FP64 (rho0 and E0 = p0 / (gamma - 1) from the FP32
// background record), rounded to FP32, plus rho0 and p0.  lam_out receives the
// largest |U| + sqrt(gamma p / rho + |B|^2 / rho) of the points this thread loaded
// (FP64 policy in FP64, mixed policy in FP32).
template <int N, class Pol>
__device__ __forceinline__ void load_element(const StageParams& P, const double* q, int64_t e,
                                             typename Pol::R* sQ, double* lam_out) {
  constexpr int N3 = N * N * N, BLK = Dims<N>::BLK;
  double lam = 0.0;
  float lamf = 0.0f;  // mixed policy: the maximum of FP32 speeds, taken in FP32 (the same value)
  for (int n = threadIdx.x; n < N3; n += BLK) {
    const int64_t g = e * P.stride + n;
    double qv[9];
#pragma unroll
    for (int v = 0; v < 9; ++v) qv[v] = __ldg(q + v * P.plane + g);
    if constexpr (!Pol::mixed) {
      if (lam_out) lam = speed_max(lam, point_speed_fp64(qv, P.gamma));
#pragma unroll
      for (int v = 0; v < 9; ++v) sQ[v * N3 + n] = qv[v];
    } else {
      const int64_t gb = e * N3 + n;
      const float r0 = __ldg(P.bg + gb), p0 = __ldg(P.bg + P.n_e * N3 + gb);
      float qf[9];
#pragma unroll
      for (int v = 0; v < 9; ++v) qf[v] = f64_to_f32(qv[v]);
      if (lam_out) lamf = speed_max(lamf, point_speed_mixed(qf, (float)P.gamma));
      qf[0] = f64_to_f32(qv[0] - f32_to_f64(r0));
      qf[4] = f64_to_f32(fma(-f32_to_f64(p0), P.inv_gm1, qv[4]));
#pragma unroll
      for (int v = 0; v < 9; ++v) sQ[v * N3 + n] = qf[v];
      if (P.qp_out) {
        const int64_t qplane = P.n_e * P.dstride;
#pragma unroll
        for (int v = 0; v < 9; ++v) P.qp_out[v * qplane + e * P.dstride + n] = qf[v];
      }
      sQ[9 * N3 + n] = r0;
      sQ[10 * N3 + n] = p0;
    }
  }
  if (lam_out) *lam_out = Pol::mixed ? (double)lamf : lam;
}

// Extrapolate the element state in shared memory to its 6 N^2 face points and
// write the trace block [F][v][N^2] of element e.
template <int N, class Pol>
__device__ __forceinline__ void write_traces(const typename Pol::R* sQ, const typename Pol::R* sE,
                                             typename Pol::R* tr, int64_t e) {
  using R = typename Pol::R;
  constexpr int N2 = N * N, N3 = N2 * N, BLK = Dims<N>::BLK;
  for (int t = threadIdx.x; t < 6 * N2; t += BLK) {
    const int F = t / N2, pt = t - F * N2, a = pt % N, b = pt / N;
    const int d = F >> 1, f = (F & 1) ? N : 0;
    R* T = tr + (e * 6 + F) * 9 * N2 + pt;
#pragma unroll
    for (int v = 0; v < 9; ++v) {
      R s = R(0);
#pragma unroll
      for (int i = 0; i < N; ++i) s += sE[f * N + i] * sQ[v * N3 + sol_index<N>(d, i, a, b)];
      T[v * N2] = s;
    }
  }
}

// Face traces of element e (and, with P.lam_max, its lambda_max contribution).
template <int N, class Pol>
__device__ __forceinline__ void trace_body(const StageParams& P, const Ops<typename Pol::R>& ops, int64_t e,
                                           unsigned char* smem) {
  using R = typename Pol::R;
  constexpr int NF = N + 1, BLK = Dims<N>::BLK;
  using S = Smem<N, Pol>;
  R* sQ = reinterpret_cast<R*>(smem) + S::oQ;
  R* sE = reinterpret_cast<R*>(smem) + S::oTE;
  for (int i = threadIdx.x; i < NF * N; i += BLK) sE[i] = ops.E[i];
  double lam = 0.0;
  load_element<N, Pol>(P, P.q_in, e, sQ, P.lam_max ? &lam : nullptr);
  if (P.lam_max) {
    if constexpr (Pol::mixed)
      speed_reduce((float)lam, P.lam_max, P.lam_nslot);  // exact: lam holds an FP32 value
    else
      speed_reduce(lam, P.lam_max, P.lam_nslot);
  }
  __syncthreads();
  write_traces<N, Pol>(sQ, sE, reinterpret_cast<R*>(P.tr_out), e);
}

template <int N, class Pol>
__global__ void __launch_bounds__(Dims<N>::BLK) trace_kernel(const StageParams P, const Ops<typename Pol::R> ops) {
  extern __shared__ __align__(16) unsigned char smem[];
  trace_body<N, Pol>(P, ops, (int64_t)blockIdx.x, smem);
}

// Packed launches: CTA b works on element b - off[r] of request r, off[r] <= b < off[r+1];
// the request's parameters are copied to shared memory first.
__device__ __forceinline__ int packed_request(const int64_t* __restrict__ off, int n_req, int64_t b) {
  int lo = 0, hi = n_req - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(off + mid) <= b) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ void copy_params(const StageParams* __restrict__ src, StageParams* dst) {
  const int* s = reinterpret_cast<const int*>(src);
  int* d = reinterpret_cast<int*>(dst);
  for (int i = threadIdx.x; i < (int)(sizeof(StageParams) / sizeof(int)); i += blockDim.x) d[i] = __ldg(s + i);
  __syncthreads();
}

template <int N>
__global__ void __launch_bounds__(Dims<N>::BLK) trace_kernel_packed(const StageParams* __restrict__ tab,
                                                                    const int64_t* __restrict__ off, int n_req,
                                                                    const Ops<float> ops) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ StageParams sP;
  const int r = packed_request(off, n_req, (int64_t)blockIdx.x);
  copy_params(tab + r, &sP);
  if (sP.skip) return;  // uniform over the CTA
  trace_body<N, PolMixed>(sP, ops, (int64_t)blockIdx.x - __ldg(off + r), smem);
}

// Sources M (Sec. MHD Governing Equations) for the full FP64 state.
__device__ __forceinline__ void sources_fp64(const StageParams& P, const double* q, double divB, double x0, double x1,
                                             double x2, double* M) {
  const double ir = 1.0 / q[0];
  const double ux = q[1] * ir, uy = q[2] * ir, uz = q[3] * ir;
#pragma unroll
  for (int v = 0; v < 9; ++v) M[v] = 0.0;
  if (P.gravity) {
    const double r2 = x0 * x0 + x1 * x1 + x2 * x2;
    const double ir3 = 1.0 / (r2 * sqrt(r2));
    const double gx = -P.GM * x0 * ir3, gy = -P.GM * x1 * ir3, gz = -P.GM * x2 * ir3;
    M[1] += q[0] * gx;
    M[2] += q[0] * gy;
    M[3] += q[0] * gz;
    M[4] += q[1] * gx + q[2] * gy + q[3] * gz;
  }
  if (P.coriolis) {
    M[1] += 2.0 * P.omega * q[2];
    M[2] -= 2.0 * P.omega * q[1];
  }
  if (P.powell) {
    const double uB = ux * q[5] + uy * q[6] + uz * q[7];
    M[1] -= divB * q[5];
    M[2] -= divB * q[6];
    M[3] -= divB * q[7];
    M[4] -= divB * uB;
    M[5] -= divB * ux;
    M[6] -= divB * uy;
    M[7] -= divB * uz;
  }
  M[8] -= P.alpha * q[8];
}

// Uniform FP32 constants of the mixed sources (GM, 2 Omega, the GLM damping).
struct MixedConsts {
  float GM, om2, alpha;
  int gravity, coriolis, powell;
};

// Sources of the perturbation (rho0 g lives in the FP64 background residual).
__device__ __forceinline__ void sources_mixed(const MixedConsts& C, const float* q, float divB, float x0, float x1,
                                              float x2, float* M) {
  const float rho = q[9] + q[0];
  const float ir = 1.0f / rho;
  const float ux = q[1] * ir, uy = q[2] * ir, uz = q[3] * ir;
#pragma unroll
  for (int v = 0; v < 9; ++v) M[v] = 0.0f;
  if (C.gravity) {
    const float r2 = x0 * x0 + x1 * x1 + x2 * x2;
    const float rr = rsqrtf(r2);
    const float ir3 = rr * rr * rr;
    const float gx = -C.GM * x0 * ir3, gy = -C.GM * x1 * ir3, gz = -C.GM * x2 * ir3;
    M[1] += q[0] * gx;
    M[2] += q[0] * gy;
    M[3] += q[0] * gz;
    M[4] += q[1] * gx + q[2] * gy + q[3] * gz;
  }
  if (C.coriolis) {
    M[1] += C.om2 * q[2];
    M[2] -= C.om2 * q[1];
  }
  if (C.powell) {
    const float uB = ux * q[5] + uy * q[6] + uz * q[7];
    M[1] -= divB * q[5];
    M[2] -= divB * q[6];
    M[3] -= divB * q[7];
    M[4] -= divB * uB;
    M[5] -= divB * ux;
    M[6] -= divB * uy;
    M[7] -= divB * uz;
  }
  M[8] -= C.alpha * q[8];
}

// The trace (+lambda_max) kernel of either policy.
template <int N, class Pol>
cudaError_t launch_traces_t(const StageParams& P, const Ops<typename Pol::R>& ops, cudaStream_t s) {
  const size_t bytes = Smem<N, Pol>::trace_bytes;
  if (bytes > 48 * 1024) {
    cudaError_t err = cudaFuncSetAttribute(trace_kernel<N, Pol>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (err != cudaSuccess) return err;
  }
  if (P.n_e == 0) return cudaSuccess;
  trace_kernel<N, Pol><<<(unsigned)P.n_e, Dims<N>::BLK, bytes, s>>>(P, ops);
  return cudaGetLastError();
}

}  // namespace sd
