// sd_physics2.cuh -- the mixed-policy pointwise physics of sd_physics.cuh for two
// points at once, in Blackwell's paired FP32 arithmetic (add / mul / fma on
// .f32x2: one instruction computes both lanes, each lane rounded as the scalar
// operation would round it).  Lane x is one flux point, lane y another; the
// formulas are those of flux_pert, side_mixed and riemann_mixed (Eq. invF with
// the background's pressure flux left out, the Rusanov flux of Sec. SD Method).
// Reciprocals and square roots stay scalar per lane.
#pragma once

#include <cuda_runtime.h>

namespace sd {

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// a - b as a + (-1) b: one fused operation, exact product, one rounding
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, f2(-1.0f), a); }
__device__ __forceinline__ float2 rcp2(float2 a) { return make_float2(1.0f / a.x, 1.0f / a.y); }
__device__ __forceinline__ float2 sqrt2(float2 a) { return make_float2(sqrtf(a.x), sqrtf(a.y)); }
__device__ __forceinline__ float2 abs2(float2 a) { return make_float2(fabsf(a.x), fabsf(a.y)); }
__device__ __forceinline__ float2 max2(float2 a, float2 b) { return make_float2(fmaxf(a.x, b.x), fmaxf(a.y, b.y)); }
// a.b over three components: ((a0 b0) + a1 b1) + a2 b2
__device__ __forceinline__ float2 dot3(float2 a0, float2 a1, float2 a2, float2 b0, float2 b1, float2 b2) {
  return fma2(a2, b2, fma2(a1, b1, mul2(a0, b0)));
}

// Uniform FP32 constants of the paired physics, each held in both lanes.
struct Mixed2 {
  float2 gamma, gm1, gg1, ch, half;
};

// flux_pert for two points: q[11] = q'(9), rho0, p0; S the (not unit) normal.
__device__ __forceinline__ void flux_pert2(const float2* q, float2 nx, float2 ny, float2 nz, const Mixed2& C,
                                           float2* F) {
  const float2 rho = add2(q[9], q[0]);
  const float2 ir = rcp2(rho);
  const float2 ux = mul2(q[1], ir), uy = mul2(q[2], ir), uz = mul2(q[3], ir);
  const float2 Bx = q[5], By = q[6], Bz = q[7], psi = q[8];
  const float2 B2 = dot3(Bx, By, Bz, Bx, By, Bz);
  const float2 mu = dot3(q[1], q[2], q[3], ux, uy, uz);
  const float2 pp = mul2(C.gm1, sub2(q[4], mul2(C.half, add2(add2(mu, B2), mul2(psi, psi)))));
  const float2 un = dot3(ux, uy, uz, nx, ny, nz);
  const float2 Bn = dot3(Bx, By, Bz, nx, ny, nz);
  const float2 uB = dot3(ux, uy, uz, Bx, By, Bz);
  const float2 ptp = fma2(C.half, B2, pp);
  const float2 chpsi = mul2(C.ch, psi);
  F[0] = dot3(q[1], q[2], q[3], nx, ny, nz);
  F[1] = sub2(fma2(ptp, nx, mul2(q[1], un)), mul2(Bx, Bn));
  F[2] = sub2(fma2(ptp, ny, mul2(q[2], un)), mul2(By, Bn));
  F[3] = sub2(fma2(ptp, nz, mul2(q[3], un)), mul2(Bz, Bn));
  const float2 h = sub2(add2(fma2(C.gg1, q[10], q[4]), ptp), mul2(C.half, mul2(psi, psi)));
  F[4] = fma2(chpsi, Bn, sub2(mul2(un, h), mul2(Bn, uB)));
  F[5] = fma2(chpsi, nx, sub2(mul2(un, Bx), mul2(Bn, ux)));
  F[6] = fma2(chpsi, ny, sub2(mul2(un, By), mul2(Bn, uy)));
  F[7] = fma2(chpsi, nz, sub2(mul2(un, Bz), mul2(Bn, uz)));
  F[8] = mul2(C.ch, Bn);
}

// side_mixed for two points: the perturbation flux of q'(9) about the background
// (r0, p0) along the unit normal n, and |U.n| + c_f.
__device__ __forceinline__ float2 side_mixed2(const float2* q, float2 r0, float2 p0, float2 nx, float2 ny, float2 nz,
                                              const Mixed2& C, float2* F) {
  const float2 rho = add2(r0, q[0]);
  const float2 ir = rcp2(rho);
  const float2 ux = mul2(q[1], ir), uy = mul2(q[2], ir), uz = mul2(q[3], ir);
  const float2 Bx = q[5], By = q[6], Bz = q[7], psi = q[8];
  const float2 B2 = dot3(Bx, By, Bz, Bx, By, Bz);
  const float2 mu = dot3(q[1], q[2], q[3], ux, uy, uz);
  const float2 pp = mul2(C.gm1, sub2(q[4], mul2(C.half, add2(add2(mu, B2), mul2(psi, psi)))));
  const float2 un = dot3(ux, uy, uz, nx, ny, nz);
  const float2 Bn = dot3(Bx, By, Bz, nx, ny, nz);
  const float2 uB = dot3(ux, uy, uz, Bx, By, Bz);
  const float2 ptp = fma2(C.half, B2, pp);
  const float2 chpsi = mul2(C.ch, psi);
  F[0] = dot3(q[1], q[2], q[3], nx, ny, nz);
  F[1] = sub2(fma2(ptp, nx, mul2(q[1], un)), mul2(Bx, Bn));
  F[2] = sub2(fma2(ptp, ny, mul2(q[2], un)), mul2(By, Bn));
  F[3] = sub2(fma2(ptp, nz, mul2(q[3], un)), mul2(Bz, Bn));
  const float2 h = sub2(add2(fma2(C.gg1, p0, q[4]), ptp), mul2(C.half, mul2(psi, psi)));
  F[4] = fma2(chpsi, Bn, sub2(mul2(un, h), mul2(Bn, uB)));
  F[5] = fma2(chpsi, nx, sub2(mul2(un, Bx), mul2(Bn, ux)));
  F[6] = fma2(chpsi, ny, sub2(mul2(un, By), mul2(Bn, uy)));
  F[7] = fma2(chpsi, nz, sub2(mul2(un, Bz), mul2(Bn, uz)));
  F[8] = mul2(C.ch, Bn);
  // fast magnetosonic speed along n
  const float2 a2 = mul2(mul2(C.gamma, add2(p0, pp)), ir);
  const float2 b2 = mul2(B2, ir);
  const float2 s = add2(a2, b2);
  const float2 disc = max2(sub2(mul2(s, s), mul2(f2(4.0f), mul2(a2, mul2(mul2(Bn, Bn), ir)))), f2(0.0f));
  return add2(abs2(un), sqrt2(mul2(C.half, add2(s, sqrt2(disc)))));
}

// riemann_mixed for two points: qo own q'(9), rho0, p0; qn the other side's q'(9);
// jr, jp the background jumps (other minus own).
__device__ __forceinline__ void riemann_mixed2(const float2* qo, const float2* qn, float2 nx, float2 ny, float2 nz,
                                               float2 jr, float2 jp, const Mixed2& C, float2* Fs) {
  float2 FL[9], FR[9];
  const float2 lo = side_mixed2(qo, qo[9], qo[10], nx, ny, nz, C, FL);
  const float2 ln = side_mixed2(qn, add2(qo[9], jr), add2(qo[10], jp), nx, ny, nz, C, FR);
  const float2 hl = mul2(C.half, max2(max2(lo, ln), C.ch));
  const float2 igm1 = rcp2(C.gm1);
#pragma unroll
  for (int v = 0; v < 9; ++v) {
    float2 dq = sub2(qn[v], qo[v]);
    if (v == 0) dq = add2(dq, jr);
    if (v == 4) dq = fma2(jp, igm1, dq);
    Fs[v] = sub2(mul2(C.half, add2(FL[v], FR[v])), mul2(hl, dq));
  }
}

}  // namespace sd
