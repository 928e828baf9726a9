// sd_physics.cuh -- pointwise physics of ideal MHD with GLM cleaning on the
// device (arXiv 2502.17805, Sec. MHD Governing Equations):
//   Q = (rho, m = rho U, E, B, psi),  E = p/(gamma-1) + rho|U|^2/2 + |B|^2/2 + psi^2/2  (Eq. 2-3)
//   inviscid flux through a surface of normal n (Eq. invF):
//     rho: rho U.n
//     m  : m U.n + (p + |B|^2/2) n - B (B.n)
//     E  : U.n (e + p + |B|^2/2) - (B.n)(U.B) + c_h psi (B.n),   e = E - psi^2/2
//     B  : (U.n) B - (B.n) U + c_h psi n
//     psi: c_h (B.n)
// Two precision policies share the SD kernels:
//   PolFP64  -- every value is the full state in FP64.
//   PolMixed -- the state is carried as the FP32 perturbation q' about a
//               hydrostatic background (rho0, p0; U = B = psi = 0), whose
//               pressure-gradient flux lives in an FP64 background residual.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

namespace sd {

struct PolFP64 {
  using R = double;
  static constexpr int NV = 9;  // values carried per point
  static constexpr bool mixed = false;
};

struct PolMixed {
  using R = float;
  static constexpr int NV = 11;  // q'(9), rho0, p0
  static constexpr bool mixed = true;
};

template <typename R>
__device__ __forceinline__ R rcp_(R x) {
  return R(1) / x;
}

// FP64 <-> FP32 conversions done with integer operations on the IEEE-754 bit
// fields (binary64: 1 sign, 11 exponent (bias 1023), 52 fraction bits;
// binary32: 1, 8 (bias 127), 23).  They keep these conversions off the FP64
// pipe, which issues only two operations per SM and clock on this GPU.
// Narrowing rounds half up on the 24th significant bit; values below the
// binary32 normal range become signed zero; overflow, inf and NaN map to inf / NaN.
__device__ __forceinline__ float f64_to_f32(double x) {
  const unsigned hi = (unsigned)__double2hiint(x);
  const unsigned lo = (unsigned)__double2loint(x);
  const unsigned sign = hi & 0x80000000u;
  const int ef = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;
  const unsigned frac = ((hi & 0xfffffu) << 3) | (lo >> 29);
  unsigned bits = (sign | ((unsigned)ef << 23) | frac) + ((lo >> 28) & 1u);
  bits = ef > 0 ? bits : sign;
  bits = ef < 255 ? bits : (sign | 0x7f800000u | (frac ? 0x400000u : 0u));
  return __uint_as_float(bits);
}

__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned sign = b & 0x80000000u;
  const unsigned e = (b >> 23) & 0xffu;
  const unsigned frac = b & 0x7fffffu;
  unsigned hi = sign | ((e + (1023u - 127u)) << 20) | (frac >> 3);
  unsigned lo = frac << 29;
  hi = e ? hi : sign;  // zero and subnormal inputs give signed zero
  lo = e ? lo : 0u;
  hi = e == 255u ? (sign | 0x7ff00000u | (frac >> 3) | (frac ? 0x80000u : 0u)) : hi;
  return __hiloint2double((int)hi, (int)lo);
}

// Full-state flux through the (not necessarily unit) normal n.
template <typename R>
__device__ __forceinline__ void flux_full(const R* q, R nx, R ny, R nz, R gm1, R ch, R* F) {
  const R ir = rcp_(q[0]);
  const R ux = q[1] * ir, uy = q[2] * ir, uz = q[3] * ir;
  const R Bx = q[5], By = q[6], Bz = q[7], psi = q[8];
  const R B2 = Bx * Bx + By * By + Bz * Bz;
  const R mu = q[1] * ux + q[2] * uy + q[3] * uz;
  const R p = gm1 * (q[4] - R(0.5) * (mu + B2 + psi * psi));
  const R e = q[4] - R(0.5) * psi * psi;
  const R un = ux * nx + uy * ny + uz * nz;
  const R Bn = Bx * nx + By * ny + Bz * nz;
  const R uB = ux * Bx + uy * By + uz * Bz;
  const R pt = p + R(0.5) * B2;
  const R chpsi = ch * psi;
  F[0] = q[0] * un;
  F[1] = q[1] * un + pt * nx - Bx * Bn;
  F[2] = q[2] * un + pt * ny - By * Bn;
  F[3] = q[3] * un + pt * nz - Bz * Bn;
  F[4] = un * (e + pt) - Bn * uB + chpsi * Bn;
  F[5] = un * Bx - Bn * ux + chpsi * nx;
  F[6] = un * By - Bn * uy + chpsi * ny;
  F[7] = un * Bz - Bn * uz + chpsi * nz;
  F[8] = ch * Bn;
}

// Perturbation flux F(Q0 + q') - F(Q0) with Q0 = (rho0, 0, p0/(gamma-1), 0, 0):
// the background carries only the pressure flux p0 n, which is left out here.
// q holds q'(9), rho0, p0.  gg1 = gamma/(gamma-1).
__device__ __forceinline__ void flux_pert(const float* q, float nx, float ny, float nz, float gm1, float gg1, float ch,
                                          float* F) {
  const float rho = q[9] + q[0];
  const float ir = 1.0f / rho;
  const float ux = q[1] * ir, uy = q[2] * ir, uz = q[3] * ir;
  const float Bx = q[5], By = q[6], Bz = q[7], psi = q[8];
  const float B2 = Bx * Bx + By * By + Bz * Bz;
  const float mu = q[1] * ux + q[2] * uy + q[3] * uz;
  const float pp = gm1 * (q[4] - 0.5f * (mu + B2 + psi * psi));  // p' = p - p0
  const float un = ux * nx + uy * ny + uz * nz;
  const float Bn = Bx * nx + By * ny + Bz * nz;
  const float uB = ux * Bx + uy * By + uz * Bz;
  const float ptp = pp + 0.5f * B2;
  const float chpsi = ch * psi;
  F[0] = q[1] * nx + q[2] * ny + q[3] * nz;
  F[1] = q[1] * un + ptp * nx - Bx * Bn;
  F[2] = q[2] * un + ptp * ny - By * Bn;
  F[3] = q[3] * un + ptp * nz - Bz * Bn;
  F[4] = un * (gg1 * q[10] + q[4] + ptp - 0.5f * psi * psi) - Bn * uB + chpsi * Bn;
  F[5] = un * Bx - Bn * ux + chpsi * nx;
  F[6] = un * By - Bn * uy + chpsi * ny;
  F[7] = un * Bz - Bn * uz + chpsi * nz;
  F[8] = ch * Bn;
}

// Wall ghost state: rho, p and E copied, U reflected.  Conducting walls reflect
// B (B_n = 0) and copy psi; radial walls reverse the tangential part of B and
// leave B_n free, so the GLM pair (B_n, psi) takes its one wall condition on
// psi = 0 (psi reversed).  For the mixed policy the same rule applies to the
// perturbation (the background is symmetric and has no psi).
template <typename R>
__device__ __forceinline__ void wall_ghost(const R* q, R nx, R ny, R nz, int bc, R* g) {
  const R mn = q[1] * nx + q[2] * ny + q[3] * nz;
  const R Bn = q[5] * nx + q[6] * ny + q[7] * nz;
  g[0] = q[0];
  g[1] = q[1] - R(2) * mn * nx;
  g[2] = q[2] - R(2) * mn * ny;
  g[3] = q[3] - R(2) * mn * nz;
  g[4] = q[4];
  if (bc == SD_BC_WALL_CONDUCTING) {
    g[5] = q[5] - R(2) * Bn * nx;
    g[6] = q[6] - R(2) * Bn * ny;
    g[7] = q[7] - R(2) * Bn * nz;
    g[8] = q[8];
  } else {
    g[5] = R(2) * Bn * nx - q[5];
    g[6] = R(2) * Bn * ny - q[6];
    g[7] = R(2) * Bn * nz - q[7];
    g[8] = -q[8];
  }
}

// One side of the FP64 Rusanov flux: the flux of q along the unit normal n and,
// with `speed`, |U.n| + c_f (else 0); 1/rho, the velocity, |B|^2, B.n and p
// serve both.
__device__ __forceinline__ double side_fp64(const double* q, double nx, double ny, double nz, double gamma,
                                            double gm1, double ch, bool speed, double* F) {
  const double ir = 1.0 / q[0];
  const double ux = q[1] * ir, uy = q[2] * ir, uz = q[3] * ir;
  const double Bx = q[5], By = q[6], Bz = q[7], psi = q[8];
  const double B2 = Bx * Bx + By * By + Bz * Bz;
  const double mu = q[1] * ux + q[2] * uy + q[3] * uz;
  const double p = gm1 * (q[4] - 0.5 * (mu + B2 + psi * psi));
  const double e = q[4] - 0.5 * psi * psi;
  const double un = ux * nx + uy * ny + uz * nz;
  const double Bn = Bx * nx + By * ny + Bz * nz;
  const double uB = ux * Bx + uy * By + uz * Bz;
  const double pt = p + 0.5 * B2;
  const double chpsi = ch * psi;
  F[0] = q[0] * un;
  F[1] = q[1] * un + pt * nx - Bx * Bn;
  F[2] = q[2] * un + pt * ny - By * Bn;
  F[3] = q[3] * un + pt * nz - Bz * Bn;
  F[4] = un * (e + pt) - Bn * uB + chpsi * Bn;
  F[5] = un * Bx - Bn * ux + chpsi * nx;
  F[6] = un * By - Bn * uy + chpsi * ny;
  F[7] = un * Bz - Bn * uz + chpsi * nz;
  F[8] = ch * Bn;
  if (!speed) return 0.0;
  const double a2 = gamma * p * ir;
  const double b2 = B2 * ir;
  const double s = a2 + b2;
  double disc = s * s - 4.0 * a2 * (Bn * Bn * ir);
  disc = disc > 0.0 ? disc : 0.0;
  return fabs(un) + sqrt(0.5 * (s + sqrt(disc)));
}

// Rusanov common flux along the unit outward normal n of this side:
//   F* = (F(qo) + F(qn))/2 - lambda/2 (qn - qo),  lambda = max(|u_n|+c_f both sides, c_h).
// The same instruction sequence runs on both sides of a face with n negated and
// the states swapped, which makes the two results exact negatives.
__device__ __forceinline__ void riemann_fp64(const double* qo, const double* qn, double nx, double ny, double nz,
                                             double gamma, double ch, int central, double* Fs) {
  const double gm1 = gamma - 1.0;
  double FL[9], FR[9];
  const double lo = side_fp64(qo, nx, ny, nz, gamma, gm1, ch, !central, FL);
  const double ln = side_fp64(qn, nx, ny, nz, gamma, gm1, ch, !central, FR);
  if (central) {
#pragma unroll
    for (int v = 0; v < 9; ++v) Fs[v] = 0.5 * (FL[v] + FR[v]);
    return;
  }
  double lam = fmax(lo, ln);
  lam = fmax(lam, ch);
  const double hl = 0.5 * lam;
#pragma unroll
  for (int v = 0; v < 9; ++v) Fs[v] = 0.5 * (FL[v] + FR[v]) - hl * (qn[v] - qo[v]);
}

// One side of the mixed-policy Rusanov flux: the perturbation flux of q (q'(9);
// background rho0 = r0, p0 = p0) along the unit normal n, and |U.n| + c_f.  The
// velocity, 1/rho, |B|^2, B.n and p' serve both.
__device__ __forceinline__ float side_mixed(const float* q, float r0, float p0, float nx, float ny, float nz,
                                            float gamma, float gm1, float gg1, float ch, float* F) {
  const float rho = r0 + q[0];
  const float ir = 1.0f / rho;
  const float ux = q[1] * ir, uy = q[2] * ir, uz = q[3] * ir;
  const float Bx = q[5], By = q[6], Bz = q[7], psi = q[8];
  const float B2 = Bx * Bx + By * By + Bz * Bz;
  const float mu = q[1] * ux + q[2] * uy + q[3] * uz;
  const float pp = gm1 * (q[4] - 0.5f * (mu + B2 + psi * psi));  // p' = p - p0
  const float un = ux * nx + uy * ny + uz * nz;
  const float Bn = Bx * nx + By * ny + Bz * nz;
  const float uB = ux * Bx + uy * By + uz * Bz;
  const float ptp = pp + 0.5f * B2;
  const float chpsi = ch * psi;
  F[0] = q[1] * nx + q[2] * ny + q[3] * nz;
  F[1] = q[1] * un + ptp * nx - Bx * Bn;
  F[2] = q[2] * un + ptp * ny - By * Bn;
  F[3] = q[3] * un + ptp * nz - Bz * Bn;
  F[4] = un * (gg1 * p0 + q[4] + ptp - 0.5f * psi * psi) - Bn * uB + chpsi * Bn;
  F[5] = un * Bx - Bn * ux + chpsi * nx;
  F[6] = un * By - Bn * uy + chpsi * ny;
  F[7] = un * Bz - Bn * uz + chpsi * nz;
  F[8] = ch * Bn;
  // fast magnetosonic speed along n
  const float a2 = gamma * (p0 + pp) * ir;
  const float b2 = B2 * ir;
  const float s = a2 + b2;
  float disc = s * s - 4.0f * a2 * (Bn * Bn * ir);
  disc = disc > 0.0f ? disc : 0.0f;
  return fabsf(un) + sqrtf(0.5f * (s + sqrtf(disc)));
}

// Mixed-policy Rusanov flux of the perturbation.  qo: own q'(9), rho0, p0;
// qn: neighbour q'(9); jr, jp: FP64-accurate background jumps (neighbour minus
// own) of rho0 and p0 at the face point.  Each side's perturbation flux and
// wave speed are taken about its own background (the neighbour's is this side's
// plus the jumps), so that with the background's central face flux (in R0) the
// average is that of the full-state fluxes: F(Q0 + q') - F(Q0) depends on Q0,
// and the extrapolated background of the two sides differs at a face.
__device__ __forceinline__ void riemann_mixed(const float* qo, const float* qn, float nx, float ny, float nz,
                                              float gamma, float ch, float jr, float jp, float* Fs) {
  const float gm1 = gamma - 1.0f, gg1 = gamma / (gamma - 1.0f);
  float FL[9], FR[9];
  const float lo = side_mixed(qo, qo[9], qo[10], nx, ny, nz, gamma, gm1, gg1, ch, FL);
  const float ln = side_mixed(qn, qo[9] + jr, qo[10] + jp, nx, ny, nz, gamma, gm1, gg1, ch, FR);
  const float lam = fmaxf(fmaxf(lo, ln), ch);
  const float hl = 0.5f * lam;
#pragma unroll
  for (int v = 0; v < 9; ++v) {
    float dq = qn[v] - qo[v];
    if (v == 0) dq += jr;
    if (v == 4) dq += jp / gm1;
    Fs[v] = 0.5f * (FL[v] + FR[v]) - hl * dq;
  }
}

}  // namespace sd

namespace sd {

// ---- TMA bulk copies (cp.async.bulk) into shared memory, completed on an
// mbarrier.  Sources, destinations and sizes must be multiples of 16 bytes.
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// Hint to fetch global memory [p, p + bytes) into L2 (cp.async.bulk.prefetch).
// The range is first shrunk to the 16-byte boundaries inside it, so nothing
// outside it is touched.
__device__ __forceinline__ void l2_prefetch(const void* p, size_t bytes) {
  const unsigned long long a = reinterpret_cast<unsigned long long>(p);
  const unsigned long long lo = (a + 15ull) & ~15ull, hi = (a + bytes) & ~15ull;
  if (hi > lo)
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(lo), "r"((unsigned)(hi - lo)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned phase) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}

// Bounded wait on phase `phase` of the barrier: at most `spins` polls.  On
// time-out (or once another CTA has reported one in the kernel's error word)
// the error word is set and the wait continues, again bounded, so that no copy
// is still writing this CTA's shared memory when it exits.  Returns false on
// time-out.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned phase, int* err, int spins) {
  for (int it = 0; it < spins; ++it) {
    if (mbar_try_wait(bar, phase)) return true;
    if ((it & 255) == 255 && err && *reinterpret_cast<volatile int*>(err)) break;
  }
  if (err) atomicExch(err, 1);
  for (int it = 0; it < (1 << 18); ++it)
    if (mbar_try_wait(bar, phase)) break;
  return false;
}

}  // namespace sd
