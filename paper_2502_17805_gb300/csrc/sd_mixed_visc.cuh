// sd_mixed_visc.cuh -- viscous, resistive and thermal fluxes on the FP32-mixed
// path, as perturbations about the hydrostatic background.
//
// F = F_inv - F_vis (Sec. MHD Governing Equations), F_vis . n = (0, tau n,
// (U . tau - q + eta B x J) . n, eta J x n, 0), q = -kappa rho T grad S -
// kappa_r rho C_p grad T, from the BR1 gradients (Sec. SD Method) of
// w = (U, T, S, B).  The background Q0 (U = B = 0) carries only a heat flux q0;
// its viscous residual is computed once in FP64 with the background (the
// energy component; the others vanish) together with grad T0 and grad S0.
// Each stage then takes in FP32:
//   w' = w(Q0 + q') - w(Q0) = (U, T', S', B), with
//     T' = (p' rho0 - p0 rho') / (rho rho0 R),
//     S' = C_p (log1p(p'/p0) / gamma - log1p(rho'/rho0))
//   (no cancellation between background and perturbation), its BR1 gradient
//   (face value the average of both sides' w', each about its own background,
//   so that with the background's own BR1 average the two add up to the full
//   one), and
//   F_vis(Q0 + q') - F_vis(Q0): tau, J and U . tau, eta B x J are perturbation
//   quantities alone; q - q0 = -kappa (rho T grad S' + (p'/R) grad S0)
//                              - kappa_r C_p (rho grad T' + rho' grad T0),
//   exactly, since rho T - rho0 T0 = p'/R.
// Of grad w' the fluxes need only the viscous stress tau (mu constant, so tau is
// linear in grad U and may be formed at the solution points and extrapolated like
// the gradients themselves), the current J = curl B, grad T' and grad S': the
// gradient record, MV_REC = 15 values per point.
// mgrad_kernel writes the record [e][15][N^3] and, at every face point of the
// element, its own F_vis . n along its outward unit normal [e][F][7][N^2] (the
// record extrapolated there, its face trace of q', the background's values);
// mvisc_kernel writes the viscous residual of the stage state (background's
// included) [7][n_e N^3] (components rho U, E, B), which the stage kernel adds:
// at a face it averages its own F_vis . n with the neighbour's, whose outward
// normal is exactly the opposite (the two sides share the owner's metric there).
// The radiative diffusivity kappa_r(r) of a face point is taken at the owner's
// face point by both sides.
// Both are line-blocked like the inviscid stage kernel: the 1D extrapolation and
// derivative operators run along the lines of the element from registers, two
// variables at a time in paired FP32 arithmetic, in the even-odd form.
// Walls pass this side's own viscous flux (no wall conditions of the viscous
// path); meshes with far-field faces are not taken.
#pragma once

#include "sd_internal.h"
#include "sd_physics.cuh"
#include "sd_physics2.cuh"
#include "sd_stage.cuh"

namespace sd {

struct MViscCoef {
  float gm1, mu, lam, eta, kappa, kappa_r, kappa_r1, kappa_r2, R, cp, inv_gamma, inv_R;
  bool kr_varies;
};

// The FP32 coefficients, converted once on the host (the FP64 pipe of an SM is
// narrow: per-thread FP64 divisions cost more than a phase's point work).
inline MViscCoef mvisc_coef(const StageParams& P) {
  MViscCoef c;
  c.gm1 = (float)(P.gamma - 1.0);
  c.mu = (float)P.mu;
  c.lam = (float)(-2.0 / 3.0 * P.mu);
  c.eta = (float)P.eta;
  c.kappa = (float)P.kappa;
  c.kappa_r = (float)P.kappa_r;
  c.kappa_r1 = (float)P.kappa_r1;
  c.kappa_r2 = (float)P.kappa_r2;
  c.kr_varies = P.kappa_r1 != 0.0 || P.kappa_r2 != 0.0;
  c.R = (float)P.R_gas;
  c.inv_R = (float)(1.0 / P.R_gas);
  c.cp = (float)(P.gamma * P.R_gas / (P.gamma - 1.0));
  c.inv_gamma = (float)(1.0 / P.gamma);
  return c;
}

// log(1 + x) for x > -1.  For |x| <= 1/32 (the perturbation ratios p'/p0 and
// rho'/rho0 of the mixed path, as a rule) from log(1 + x) = 2 atanh(z),
// z = x / (2 + x), by the Taylor series of atanh through z^7 (|z| <= 1/63: the
// next term is below 1e-15 of the sum); elsewhere the library's log1pf.
__device__ __forceinline__ float mv_log1p(float x) {
  if (fabsf(x) > 0.03125f) return log1pf(x);
  const float z = x / (2.0f + x), z2 = z * z;
  const float s = fmaf(z2, fmaf(z2, fmaf(z2, 1.0f / 7.0f, 0.2f), 1.0f / 3.0f), 1.0f);
  return 2.0f * z * s;
}

// p' of a perturbation q'(9) about (rho0, p0): the pressure minus p0, given
// ir = 1 / (rho0 + rho')
__device__ __forceinline__ float mv_pprime(const float* q, float ir, const MViscCoef& c) {
  const float m2 = q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
  const float B2 = q[5] * q[5] + q[6] * q[6] + q[7] * q[7];
  return c.gm1 * (q[4] - 0.5f * (m2 * ir + B2 + q[8] * q[8]));
}

// w' = (u, v, w, T', S', Bx, By, Bz) of the perturbation q'(9) about (r0, p0)
__device__ __forceinline__ void mv_prim(const float* q, float r0, float p0, const MViscCoef& c, float* w) {
  const float rho = r0 + q[0];
  const float ir = 1.0f / rho;
  w[0] = q[1] * ir;
  w[1] = q[2] * ir;
  w[2] = q[3] * ir;
  const float pp = mv_pprime(q, ir, c);
  w[3] = (pp * r0 - p0 * q[0]) * ir * (1.0f / (r0 * c.R));
  w[4] = c.cp * (mv_log1p(pp * (1.0f / p0)) * c.inv_gamma - mv_log1p(q[0] * (1.0f / r0)));
  w[5] = q[5];
  w[6] = q[6];
  w[7] = q[7];
}

// mv_prim for two points at once (paired FP32; reciprocals and log1p per lane)
__device__ __forceinline__ void mv_prim2(const float2* q, float2 r0, float2 p0, const MViscCoef& c, float2* w) {
  const float2 half = f2(0.5f);
  const float2 rho = add2(r0, q[0]);
  const float2 ir = rcp2(rho);
  w[0] = mul2(q[1], ir);
  w[1] = mul2(q[2], ir);
  w[2] = mul2(q[3], ir);
  const float2 m2 = dot3(q[1], q[2], q[3], q[1], q[2], q[3]);
  const float2 B2 = dot3(q[5], q[6], q[7], q[5], q[6], q[7]);
  const float2 pp = mul2(f2(c.gm1), sub2(q[4], mul2(half, fma2(q[8], q[8], add2(mul2(m2, ir), B2)))));
  w[3] = mul2(mul2(sub2(mul2(pp, r0), mul2(p0, q[0])), ir), rcp2(mul2(r0, f2(c.R))));
  const float2 a = mul2(pp, rcp2(p0)), b = mul2(q[0], rcp2(r0));
  w[4] = mul2(f2(c.cp), make_float2(mv_log1p(a.x) * c.inv_gamma - mv_log1p(b.x), mv_log1p(a.y) * c.inv_gamma - mv_log1p(b.y)));
  w[5] = q[5];
  w[6] = q[6];
  w[7] = q[7];
}

// The gradient record: tau (xx, yy, zz, xy, xz, yz), J (x, y, z), grad T',
// grad S' at a point.
enum { MV_TAU = 0, MV_J = 6, MV_GT = 9, MV_GS = 12 };
static_assert(MV_GS + 3 == MV_REC, "record layout");

// (F_vis(Q0 + q') - F_vis(Q0)) . n from q'(9), the background (r0, p0), the
// gradient record rec[MV_REC] and the background's gT0 = grad T0, gS0 = grad S0,
// with the radiative diffusivity kr at the point: F[0..6] = components rho U (3),
// E, B (3).  n need not be a unit vector (F_vis . n is linear in n).
__device__ __forceinline__ void mv_flux(const float* q, float r0, float p0, const float* rec, const float* gT0,
                                        const float* gS0, float nx, float ny, float nz, const MViscCoef& c, float kr,
                                        float* F) {
  const float rho = r0 + q[0];
  const float ir = 1.0f / rho;
  const float Ux = q[1] * ir, Uy = q[2] * ir, Uz = q[3] * ir;
  const float pp = mv_pprime(q, ir, c);
  const float txx = rec[0], tyy = rec[1], tzz = rec[2], txy = rec[3], txz = rec[4], tyz = rec[5];
  const float Jx = rec[MV_J], Jy = rec[MV_J + 1], Jz = rec[MV_J + 2];
  F[0] = txx * nx + txy * ny + txz * nz;
  F[1] = txy * nx + tyy * ny + tyz * nz;
  F[2] = txz * nx + tyz * ny + tzz * nz;
  const float uTx = Ux * txx + Uy * txy + Uz * txz;
  const float uTy = Ux * txy + Uy * tyy + Uz * tyz;
  const float uTz = Ux * txz + Uy * tyz + Uz * tzz;
  const float Bx = q[5], By = q[6], Bz = q[7];
  const float BJx = By * Jz - Bz * Jy, BJy = Bz * Jx - Bx * Jz, BJz = Bx * Jy - By * Jx;
  const float rT = (p0 + pp) * c.inv_R;  // rho T of the full state
  const float dRT = pp * c.inv_R;        // rho T - rho0 T0
  const float krc = kr * c.cp;
  const float n3[3] = {nx, ny, nz}, uT[3] = {uTx, uTy, uTz}, BJ[3] = {BJx, BJy, BJz};
  float e = 0.0f;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const float qh = -c.kappa * (rT * rec[MV_GS + j] + dRT * gS0[j]) - krc * (rho * rec[MV_GT + j] + q[0] * gT0[j]);
    e += (uT[j] - qh + c.eta * BJ[j]) * n3[j];
  }
  F[3] = e;
  F[4] = c.eta * (Jy * nz - Jz * ny);
  F[5] = c.eta * (Jz * nx - Jx * nz);
  F[6] = c.eta * (Jx * ny - Jy * nx);
}

__device__ __forceinline__ float mv_kappa_r(const MViscCoef& c, float x, float y, float z) {
  if (!c.kr_varies) return c.kappa_r;
  const float r = sqrtf(x * x + y * y + z * z);
  return c.kappa_r + c.kappa_r1 * r + c.kappa_r2 * r * r;
}

// The stage state of the FP32-mixed path as q'(9), rho0, p0 at the solution
// points, [11][QS] (planes QS >= N^3 floats apart): the increment form's stored
// q' of q^n plus the register D (stages that read it), or the FP64 state q_in
// less the background.
template <int N>
__device__ __forceinline__ void mv_load_state(const StageParams& P, int64_t e, float* sQ, int T, int QS) {
  constexpr int N3 = N * N * N;
  const int64_t n_e = P.n_e;
  for (int n = threadIdx.x; n < N3; n += T) {
    const int64_t gb = e * N3 + n;
    const float r0 = __ldg(P.bg + gb), p0 = __ldg(P.bg + n_e * N3 + gb);
    if (P.incr) {
      const int64_t qplane = n_e * P.dstride, gd = e * P.dstride + n;
#pragma unroll
      for (int v = 0; v < 9; ++v) {
        float x = __ldg(P.qp_in + v * qplane + gd);
        if (P.lsr_read) x += __ldg(P.dreg + v * qplane + gd);
        sQ[v * QS + n] = x;
      }
    } else {
      const int64_t g = e * P.stride + n;
      double qv[9];
#pragma unroll
      for (int v = 0; v < 9; ++v) qv[v] = __ldg(P.q_in + v * P.plane + g);
      sQ[0 * QS + n] = f64_to_f32(qv[0] - f32_to_f64(r0));
#pragma unroll
      for (int v = 1; v < 9; ++v) sQ[v * QS + n] = f64_to_f32(qv[v]);
      sQ[4 * QS + n] = f64_to_f32(fma(-f32_to_f64(p0), P.inv_gm1, qv[4]));
    }
    sQ[9 * QS + n] = r0;
    sQ[10 * QS + n] = p0;
  }
}

// Extrapolate NV variables (planes of `in` VS floats apart, solution point n at
// n) along every line of the directions D0 <= d < D1 to the flux points
// F0 <= f <= N - F0 of the line's family (F0 = 0: all N + 1; F0 = 1: the
// interior ones), two variables at a time in paired FP32 arithmetic, in the
// even-odd form (E[N-f][N-1-i] = E[f][i]): variable v at flux point f of line L
// of direction d goes to out[f OF + v OV + (d - D0) OD + L].  The tasks
// (variable pair, line), lines innermost, are spread over the T threads; the
// lines of line_flip read their points in swapped pairs (fewer bank conflicts).
template <int N, int T, int NV, int D0, int D1, int F0 = 0>
__device__ __forceinline__ void mv_extrap(const float* in, int VS, float* out, int OF, int OV, int OD,
                                          const Ops2& o2) {
  constexpr int N2 = N * N, HP = N / 2, NL = (D1 - D0) * N2, NP = (NV + 1) / 2;
#pragma unroll 1
  for (int t = threadIdx.x; t < NL * NP; t += T) {
    const int pr = t / NL, l = t - pr * NL;
    const int d = D1 - D0 == 1 ? D0 : D0 + l / N2, L = D1 - D0 == 1 ? l : l - (l / N2) * N2;
    int base, stride;
    line_geom<N>(d, L, base, stride);
    const int v0 = 2 * pr, v1 = v0 + 1 < NV ? v0 + 1 : v0;
    float2 ql[N];
    load_line<N>(in + v0 * VS, in + v1 * VS, base, stride, line_flip<N>(d, L), ql);
    float2 sv[HP > 0 ? HP : 1], dv[HP > 0 ? HP : 1];
#pragma unroll
    for (int i = 0; i < HP; ++i) {
      sv[i] = add2(ql[i], ql[N - 1 - i]);
      dv[i] = sub2(ql[i], ql[N - 1 - i]);
    }
    float* X = out + (d - D0) * OD + L;
#pragma unroll
    for (int f = F0; 2 * f <= N; ++f) {
      float2 s = (N & 1) ? mul2(o2.Es[f * N + HP], ql[HP]) : make_float2(0.0f, 0.0f);
      float2 r = make_float2(0.0f, 0.0f);
#pragma unroll
      for (int i = 0; i < HP; ++i) {
        s = fma2(o2.Es[f * N + i], sv[i], s);
        r = fma2(o2.Ed[f * N + i], dv[i], r);
      }
      if (2 * f == N) {
        X[f * OF + v0 * OV] = s.x;
        X[f * OF + v1 * OV] = s.y;
      } else {
        const float2 lo = add2(s, r), hi = sub2(s, r);
        X[f * OF + v0 * OV] = lo.x;
        X[f * OF + v1 * OV] = lo.y;
        X[(N - f) * OF + v0 * OV] = hi.x;
        X[(N - f) * OF + v1 * OV] = hi.y;
      }
    }
  }
}

// Differentiate NV flux variables given at the N+1 flux points of every line of
// direction D (variable v at flux point f of line L at in[f IF + v IV + L]) back
// to the line's N solution points (even-odd form, D[N-1-i][f] = -D[i][N-f]) and
// store (ADD false) or add (ADD true) the result into acc[v AS + n].  For one
// direction the lines partition the solution points, so no two tasks touch the
// same word.
template <int N, int T, int NV, int D, bool ADD>
__device__ __forceinline__ void mv_deriv(const float* in, int IF, int IV, float* acc, int AS, const Ops2& o2) {
  constexpr int N2 = N * N, NF = N + 1, HF = NF / 2, NP = (NV + 1) / 2;
#pragma unroll 1
  for (int t = threadIdx.x; t < N2 * NP; t += T) {
    const int pr = t / N2, L = t - pr * N2;
    int base, stride;
    line_geom<N>(D, L, base, stride);
    const int v0 = 2 * pr, v1 = v0 + 1 < NV ? v0 + 1 : v0;
    float2 fv[NF];
#pragma unroll
    for (int f = 0; f <= N; ++f) fv[f] = make_float2(in[f * IF + v0 * IV + L], in[f * IF + v1 * IV + L]);
    float2 sf[HF], df[HF];
#pragma unroll
    for (int f = 0; f < HF; ++f) {
      sf[f] = add2(fv[f], fv[N - f]);
      df[f] = sub2(fv[f], fv[N - f]);
    }
    float2 o[N];
#pragma unroll
    for (int i = 0; 2 * i <= N - 1; ++i) {
      float2 p = (NF & 1) ? mul2(o2.Ds[i * NF + HF], fv[HF]) : make_float2(0.0f, 0.0f);
      float2 r = make_float2(0.0f, 0.0f);
#pragma unroll
      for (int f = 0; f < HF; ++f) {
        p = fma2(o2.Ds[i * NF + f], sf[f], p);
        r = fma2(o2.Dd[i * NF + f], df[f], r);
      }
      if (2 * i == N - 1) {
        o[i] = r;
      } else {
        o[i] = add2(p, r);
        o[N - 1 - i] = sub2(r, p);
      }
    }
    float* a = acc + v0 * AS + base;
    float* b = acc + v1 * AS + base;
    const bool two = v1 != v0, flip = line_flip<N>(D, L);
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const int k = ((i ^ 1) < N && flip) ? (i ^ 1) : i;
      if (ADD) {
        a[k * stride] += o[k].x;
        if (two) b[k * stride] += o[k].y;
      } else {
        a[k * stride] = o[k].x;
        if (two) b[k * stride] = o[k].y;
      }
    }
  }
}

// The neighbour's side of point pt of a face with neighbour nb >= 0 and
// metadata mt: its face nf = nb * 6 + (its face number) and the point p2 there.
template <int N>
__device__ __forceinline__ void mv_partner(int nb, int mt, int pt, int64_t& nf, int& p2) {
  const int code = meta_code(mt), a = pt % N, b = pt / N;
  const int u = (code & 4) ? b : a, w = (code & 4) ? a : b;
  const int a2 = (code & 2) ? N - 1 - u : u, b2 = (code & 1) ? N - 1 - w : w;
  nf = (int64_t)nb * 6 + meta_nbF(mt);
  p2 = a2 + N * b2;
}

// Position of point pt of face F of element e at the face's owner (the neighbour
// nb >= 0 when this side does not own the face; the same point but for periodic
// images): the map is a polynomial of degree floor(N/2) < N, so the end rows of E
// give it exactly from the owner's solution points.
template <int N>
__device__ __forceinline__ void mv_face_position(const StageParams& P, const Ops2& o2, int64_t e, int F, int pt, int nb,
                                                 int mt, float* x) {
  constexpr int N3 = N * N * N;
  int64_t eo = e;
  int Fo = F, po = pt;
  if (nb >= 0 && !meta_owner(mt)) {
    int64_t nf;
    mv_partner<N>(nb, mt, pt, nf, po);
    eo = nb;
    Fo = meta_nbF(mt);
  }
  const int d = Fo >> 1, a = po % N, b = po / N;
  const float* X = reinterpret_cast<const float*>(P.X) + eo * 3 * N3;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < N; ++i)
      s = fmaf((Fo & 1) ? o2.EN[i].x : o2.E0[i].x, __ldg(X + k * N3 + sol_index<N>(d, i, a, b)), s);
    x[k] = s;
  }
}

template <int N>
struct MVDims {
  static constexpr int N2 = N * N, N3 = N2 * N, NF = N + 1;
  // threads: mgrad_kernel T; mvisc_kernel TV, at N = 6 288 so that its line
  // tasks (36 lines x 16 variable pairs per family) take two full rounds
  static constexpr int T = N >= 6 ? 256 : 128;
  static constexpr int TV = N == 6 ? 288 : T;
  // Plane stride of the solution-point arrays in shared memory: the least
  // QS >= N^3 with QS = 2 (mod 16), so that the warps' line reads meet fewer
  // bank conflicts where their lanes span two variable planes (modelled at N = 6:
  // with line_flip, 1,680 -> 1,104 wavefronts for mvisc_kernel's line reads).
  static constexpr int QS = N3 + ((18 - N3 % 16) % 16);
  // mgrad_kernel: the record [MV_REC][QS] (first the state [11][QS]), then the
  // flux points of all three families [NF][11][3][N2] (the inviscid kernel's layout);
  // the record at the six faces [6][MV_REC][N2] over the interior flux points'
  // slots where it fits between the two face blocks (N >= 4), else after them
  static constexpr int gO = 0, gX = (MV_REC * QS + 3) / 4 * 4;
  static constexpr int XD = N2, XV = 3 * N2, XF = 11 * 3 * N2;
  static constexpr int RF = 6 * MV_REC * N2;
  static constexpr int gRF = XF + RF <= N * XF ? gX + XF : gX + NF * XF;
  static constexpr size_t gbytes = (size_t)(gRF + RF > gX + NF * XF ? gRF + RF : gX + NF * XF) * sizeof(float);
  // mvisc_kernel: NQ values at the solution points [NQ][QS], one family's flux
  // points [NF][NQ][N2], the residual [7][QS]
  template <bool KR>
  struct V {
    static constexpr int NQ = 11 + MV_REC + 6 + (KR ? 3 : 0);
    static constexpr int oQ = 0, oX = (NQ * QS + 3) / 4 * 4, oR = oX + (NF * NQ * N2 + 3) / 4 * 4;
    static constexpr size_t bytes = (size_t)(oR + 7 * QS) * sizeof(float);
  };
  static constexpr int minb(size_t bytes, int threads) {
    const int s = (int)(233472 / (bytes + 1024 + 64)), r = 65536 / (threads * 64);
    const int m = s < r ? s : r;
    return m < 1 ? 1 : m;
  }
};

// BR1 gradients of w' and the record formed from them, with its face traces.
template <int N>
__global__ void __launch_bounds__(MVDims<N>::T, MVDims<N>::minb(MVDims<N>::gbytes, MVDims<N>::T))
    mgrad_kernel(const StageParams P, const Ops<float> ops, const Ops2 o2, const MViscCoef c) {
  using MD = MVDims<N>;
  constexpr int N2 = MD::N2, N3 = MD::N3, NF = MD::NF, T = MD::T, XD = MD::XD, XV = MD::XV, XF = MD::XF;
  constexpr int QS = MD::QS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sO = reinterpret_cast<float*>(smem_raw) + MD::gO;  // the state, then the record
  float* sX = reinterpret_cast<float*>(smem_raw) + MD::gX;
  __shared__ int sNb[6], sMt[6];
  const int tid = threadIdx.x;
  const int64_t e = blockIdx.x;
  const float* Sfam = reinterpret_cast<const float*>(P.Sfam) + e * (9 * N2 * NF);
  if (tid < 6) {
    sNb[tid] = __ldg(P.nbr + e * 6 + tid);
    sMt[tid] = __ldg(P.meta + e * 6 + tid);
  } else if (tid >= 32 && tid < 32 + 8) {
    // L2 prefetch of the neighbours' traces that the face points read, and of the
    // element's own traces of q' and of grad T0, grad S0 (the face fluxes at the end)
    const int k = tid - 32;
    if (k < 6) {
      const int nb = __ldg(P.nbr + e * 6 + k), mt = __ldg(P.meta + e * 6 + k);
      if (nb >= 0)
        l2_prefetch(reinterpret_cast<const float*>(P.tr_in) + ((int64_t)nb * 6 + meta_nbF(mt)) * 9 * N2,
                    9 * N2 * sizeof(float));
    } else if (k == 6) {
      l2_prefetch(reinterpret_cast<const float*>(P.tr_in) + e * 6 * 9 * N2, 6 * 9 * N2 * sizeof(float));
    } else {
      l2_prefetch(P.bg_vtr + e * 6 * 6 * N2, 6 * 6 * N2 * sizeof(float));
    }
  }
  mv_load_state<N>(P, e, sO, T, QS);
  __syncthreads();
  // extrapolate q'(9), rho0, p0 along every line to its family's flux points
  mv_extrap<N, T, 11, 0, 3>(sO, QS, sX, XF, XV, XD, o2);
  __syncthreads();
  // w' at every flux point: pairs of interior points (r, r + NINT/2) in the lanes
  // of one paired evaluation, then the element faces one point at a time, with
  // the BR1 average of this side's w' and the other side's (the neighbour's trace
  // about its own background, or the wall ghost)
  constexpr int NINT = 3 * (N - 1) * N2, NIP = NINT / 2, NIP_W = (NIP + 31) / 32 * 32;
#pragma unroll 1
  for (int t = tid; t < NIP_W + 6 * N2; t += T) {
    if (t < NIP_W) {
      if (t >= NIP) continue;
      float* Xp[2];
      float2 q[11], w[8];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int r0 = t + h * NIP;
        const int d = r0 / ((N - 1) * N2), r = r0 - d * ((N - 1) * N2);
        const int f = 1 + r / N2, L = r - (f - 1) * N2;
        Xp[h] = sX + f * XF + d * XD + L;
#pragma unroll
        for (int v = 0; v < 11; ++v) (h ? q[v].y : q[v].x) = Xp[h][v * XV];
      }
      mv_prim2(q, q[9], q[10], c, w);
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        Xp[0][k * XV] = w[k].x;
        Xp[1][k * XV] = w[k].y;
      }
      continue;
    }
    const int u = t - NIP_W, F = u / N2, L = u - F * N2, d = F >> 1, f = (F & 1) ? N : 0;
    float* X = sX + f * XF + d * XD + L;
    float q[11], w[8];
#pragma unroll
    for (int v = 0; v < 11; ++v) q[v] = X[v * XV];
    mv_prim(q, q[9], q[10], c, w);
    const int nb = sNb[F], mt = sMt[F];
    float q2[9], r2 = q[9], p2 = q[10];
    if (nb >= 0) {
      int64_t nf;
      int pn;
      mv_partner<N>(nb, mt, L, nf, pn);
      const float* Tn = reinterpret_cast<const float*>(P.tr_in) + nf * 9 * N2 + pn;
#pragma unroll
      for (int v = 0; v < 9; ++v) q2[v] = Tn[v * N2];
      const int64_t gidx = e * 6 + F;
      r2 += __ldg(P.bg_jump + (gidx * 2 + 0) * N2 + L);
      p2 += __ldg(P.bg_jump + (gidx * 2 + 1) * N2 + L);
    } else {
      const float* Sp = Sfam + s32_index(N, d, f, 0, L);
      const float Sx = __ldg(Sp), Sy = __ldg(Sp + N2), Sz = __ldg(Sp + 2 * N2);
      const float im = rsqrtf(Sx * Sx + Sy * Sy + Sz * Sz), sg = (f == N) ? 1.0f : -1.0f;
      wall_ghost<float>(q, sg * Sx * im, sg * Sy * im, sg * Sz * im, meta_bc(mt), q2);
    }
    float w2[8];
    mv_prim(q2, r2, p2, c, w2);
#pragma unroll
    for (int k = 0; k < 8; ++k) X[k * XV] = 0.5f * (w[k] + w2[k]);
  }
  __syncthreads();
  // |J| d w'_c / d x_j = sum_d D_d (S^d_j w'_c) at this thread's solution points,
  // two components c at a time; then the record tau, J, grad T', grad S'
#pragma unroll 1
  for (int n = tid; n < N3; n += T) {
    const int i0 = n % N, j0 = (n / N) % N, k0 = n / N2;
    float2 acc[12];  // acc[4 j + p]: components (2p, j) and (2p + 1, j)
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int id = d == 0 ? i0 : (d == 1 ? j0 : k0);
      const int L = d == 0 ? j0 + N * k0 : (d == 1 ? i0 + N * k0 : i0 + N * j0);
#pragma unroll
      for (int f = 0; f <= N; ++f) {
        const float Df = ops.D[id * NF + f];
        const float* Sp = Sfam + s32_index(N, d, f, 0, L);
        const float2 DS[3] = {f2(Df * __ldg(Sp)), f2(Df * __ldg(Sp + N2)), f2(Df * __ldg(Sp + 2 * N2))};
        const float* W = sX + f * XF + d * XD + L;
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          const float2 wp = make_float2(W[(2 * p) * XV], W[(2 * p + 1) * XV]);
#pragma unroll
          for (int j = 0; j < 3; ++j) acc[4 * j + p] = fma2(DS[j], wp, acc[4 * j + p]);
        }
      }
    }
    const float iJ = __ldg(reinterpret_cast<const float*>(P.invJ) + e * N3 + n);
    float g[24];  // g[3 c + j] = d w'_c / d x_j
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        g[3 * (2 * p) + j] = acc[4 * j + p].x * iJ;
        g[3 * (2 * p + 1) + j] = acc[4 * j + p].y * iJ;
      }
    const float divu = g[0] + g[4] + g[8];
    float rec[MV_REC];
    rec[0] = c.mu * (g[0] + g[0]) + c.lam * divu;
    rec[1] = c.mu * (g[4] + g[4]) + c.lam * divu;
    rec[2] = c.mu * (g[8] + g[8]) + c.lam * divu;
    rec[3] = c.mu * (g[1] + g[3]);
    rec[4] = c.mu * (g[2] + g[6]);
    rec[5] = c.mu * (g[5] + g[7]);
    rec[MV_J + 0] = g[3 * 7 + 1] - g[3 * 6 + 2];
    rec[MV_J + 1] = g[3 * 5 + 2] - g[3 * 7 + 0];
    rec[MV_J + 2] = g[3 * 6 + 0] - g[3 * 5 + 1];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      rec[MV_GT + j] = g[3 * 3 + j];
      rec[MV_GS + j] = g[3 * 4 + j];
    }
    float* Ge = P.mgrad_out + e * MV_REC * N3 + n;
#pragma unroll
    for (int k = 0; k < MV_REC; ++k) {
      sO[k * QS + n] = rec[k];
      Ge[k * N3] = rec[k];
    }
  }
  __syncthreads();
  // the record at both ends of every line, two values at a time -> sRF[F][k][L]
  float* sRF = reinterpret_cast<float*>(smem_raw) + MD::gRF;
  constexpr int NL = 3 * N2, NP = (MV_REC + 1) / 2;
#pragma unroll 1
  for (int t = tid; t < NL * NP; t += T) {
    const int pr = t / NL, l = t - pr * NL, d = l / N2, L = l - d * N2;
    int base, stride;
    line_geom<N>(d, L, base, stride);
    const int v0 = 2 * pr, v1 = v0 + 1 < MV_REC ? v0 + 1 : v0;
    float2 x[N];
    load_line<N>(sO + v0 * QS, sO + v1 * QS, base, stride, line_flip<N>(d, L), x);
    float2 s0 = make_float2(0.0f, 0.0f), s1 = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int i = 0; i < N; ++i) {
      s0 = fma2(o2.E0[i], x[i], s0);
      s1 = fma2(o2.EN[i], x[i], s1);
    }
    float* Tr = sRF + (2 * d) * MV_REC * N2 + L;
    Tr[v0 * N2] = s0.x;
    Tr[MV_REC * N2 + v0 * N2] = s1.x;
    if (v1 != v0) {
      Tr[v1 * N2] = s0.y;
      Tr[MV_REC * N2 + v1 * N2] = s1.y;
    }
  }
  __syncthreads();
  // this side's F_vis . n at every face point, n its outward unit normal: its face
  // trace of q', rho0 and p0 at the face flux point (sX slots 9 and 10, which the
  // w' phase leaves), the record there, the background's grad T0 and grad S0
#pragma unroll 1
  for (int t = tid; t < 6 * N2; t += T) {
    const int F = t / N2, L = t - F * N2, d = F >> 1, f = (F & 1) ? N : 0;
    float q[9], rec[MV_REC], gT0[3], gS0[3], Fv[7];
    const float* To = reinterpret_cast<const float*>(P.tr_in) + (e * 6 + F) * 9 * N2 + L;
#pragma unroll
    for (int v = 0; v < 9; ++v) q[v] = __ldg(To + v * N2);
    const float* Xf = sX + f * XF + d * XD + L;
    const float r0 = Xf[9 * XV], p0 = Xf[10 * XV];
#pragma unroll
    for (int k = 0; k < MV_REC; ++k) rec[k] = sRF[(F * MV_REC + k) * N2 + L];
    const float* Bv = P.bg_vtr + (e * 6 + F) * 6 * N2 + L;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      gT0[k] = __ldg(Bv + k * N2);
      gS0[k] = __ldg(Bv + (3 + k) * N2);
    }
    const float* Sp = Sfam + s32_index(N, d, f, 0, L);
    const float Sx = __ldg(Sp), Sy = __ldg(Sp + N2), Sz = __ldg(Sp + 2 * N2);
    const float im = 1.0f / sqrtf(Sx * Sx + Sy * Sy + Sz * Sz), sg = (f == N) ? 1.0f : -1.0f;
    float kr = c.kappa_r;
    if (c.kr_varies) {
      float xo[3];
      mv_face_position<N>(P, o2, e, F, L, sNb[F], sMt[F], xo);
      kr = mv_kappa_r(c, xo[0], xo[1], xo[2]);
    }
    mv_flux(q, r0, p0, rec, gT0, gS0, sg * Sx * im, sg * Sy * im, sg * Sz * im, c, kr, Fv);
    float* Out = P.mvf_out + (e * 6 + F) * 7 * N2 + L;
#pragma unroll
    for (int v = 0; v < 7; ++v) Out[v * N2] = Fv[v];
  }
}

// One family of the viscous flux: S^d . F_vis at the flux points of family D
// (values at flux point (f, L) read from X[f NQ N^2 + v N^2 + L], the flux
// written over its first seven values; the state is not extrapolated to the two
// faces).  At the element faces the common flux is the average of both sides'
// F_vis . n as their gradient kernels wrote them (each about its own
// background), at a wall this side's alone.
template <int N, bool KR, int D>
__device__ __forceinline__ void mv_family_flux(const StageParams& P, const MViscCoef& c, int64_t e, const float* Sfam,
                                               float* X, const int* sNb, const int* sMt) {
  constexpr int N2 = N * N, NF = N + 1, T = MVDims<N>::TV, NQ = MVDims<N>::template V<KR>::NQ;
  constexpr int Q_R0 = 9, Q_P0 = 10, Q_REC = 11, Q_GT0 = Q_REC + MV_REC, Q_GS0 = Q_GT0 + 3, Q_X = Q_GS0 + 3;
#pragma unroll 1
  for (int t = threadIdx.x; t < NF * N2; t += T) {
    const int f = t / N2, L = t - f * N2;
    float* Xp = X + f * NQ * N2 + L;
    const float* Sp = Sfam + s32_index(N, D, f, 0, L);
    const float Sx = __ldg(Sp), Sy = __ldg(Sp + N2), Sz = __ldg(Sp + 2 * N2);
    float Fv[7];
    if (f > 0 && f < N) {
      float x[NQ];
#pragma unroll
      for (int v = 0; v < NQ; ++v) x[v] = Xp[v * N2];
      const float kr = KR ? mv_kappa_r(c, x[Q_X], x[Q_X + 1], x[Q_X + 2]) : c.kappa_r;
      mv_flux(x, x[Q_R0], x[Q_P0], x + Q_REC, x + Q_GT0, x + Q_GS0, Sx, Sy, Sz, c, kr, Fv);
    } else {
      // this side's F_vis . n and the neighbour's F_vis . n_nb (n_nb = -n exactly), both as
      // the gradient kernels wrote them; scaled to S^d along this side's direction
      const int F = 2 * D + (f == N);
      const int nb = sNb[F], mt = sMt[F];
      const float* Fo = P.mvf_in + (e * 6 + F) * 7 * N2 + L;
#pragma unroll
      for (int v = 0; v < 7; ++v) Fv[v] = Fo[v * N2];
      if (nb >= 0) {
        int64_t nf;
        int pn;
        mv_partner<N>(nb, mt, L, nf, pn);
        const float* Fn = P.mvf_in + nf * 7 * N2 + pn;
#pragma unroll
        for (int v = 0; v < 7; ++v) Fv[v] = 0.5f * (Fv[v] - Fn[v * N2]);
      }
      const float sm = ((f == N) ? 1.0f : -1.0f) * sqrtf(Sx * Sx + Sy * Sy + Sz * Sz);
#pragma unroll
      for (int v = 0; v < 7; ++v) Fv[v] *= sm;
    }
#pragma unroll
    for (int v = 0; v < 7; ++v) Xp[v * N2] = Fv[v];
  }
}


// The viscous residual of the stage state, R_vis = div(S^d . F_vis)/|J|, the
// background's included: out [7][n_e N^3] (components rho U, E, B).  Family by
// family: extrapolate the NQ values (q'(9), rho0, p0, the record, grad T0,
// grad S0 and, with KR, x for kappa_r(r)) along the lines of direction d, the flux
// at the family's points, its derivative along the lines added to the residual.
template <int N, bool KR>
__global__ void __launch_bounds__(MVDims<N>::TV, MVDims<N>::minb(MVDims<N>::template V<KR>::bytes, MVDims<N>::TV))
    mvisc_kernel(const StageParams P, const Ops2 o2, const MViscCoef c) {
  using MD = MVDims<N>;
  using MV = typename MD::template V<KR>;
  constexpr int N2 = MD::N2, N3 = MD::N3, T = MD::TV, NQ = MV::NQ, QS = MD::QS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sQ = reinterpret_cast<float*>(smem_raw) + MV::oQ;
  float* sX = reinterpret_cast<float*>(smem_raw) + MV::oX;
  float* sR = reinterpret_cast<float*>(smem_raw) + MV::oR;
  __shared__ int sNb[6], sMt[6];
  const int tid = threadIdx.x;
  const int64_t e = blockIdx.x;
  const int64_t n_e = P.n_e;
  const float* Sfam = reinterpret_cast<const float*>(P.Sfam) + e * (9 * N2 * (N + 1));
  if (tid < 6) {
    sNb[tid] = __ldg(P.nbr + e * 6 + tid);
    sMt[tid] = __ldg(P.meta + e * 6 + tid);
  } else if (tid >= 32 && tid < 32 + 7) {
    // L2 prefetch of what the face fluxes read: the neighbours' own F_vis . n at
    // the shared faces, and this element's
    const int k = tid - 32;
    if (k < 6) {
      const int nb = __ldg(P.nbr + e * 6 + k), mt = __ldg(P.meta + e * 6 + k);
      if (nb >= 0) l2_prefetch(P.mvf_in + ((int64_t)nb * 6 + meta_nbF(mt)) * 7 * N2, 7 * N2 * sizeof(float));
    } else {
      l2_prefetch(P.mvf_in + e * 6 * 7 * N2, 6 * 7 * N2 * sizeof(float));
    }
  }
  mv_load_state<N>(P, e, sQ, T, QS);
  for (int n = tid; n < N3; n += T) {
    const float* G = P.mgrad + e * MV_REC * N3 + n;
#pragma unroll
    for (int k = 0; k < MV_REC; ++k) sQ[(11 + k) * QS + n] = __ldg(G + k * N3);
#pragma unroll
    for (int k = 0; k < 6; ++k) sQ[(11 + MV_REC + k) * QS + n] = __ldg(P.bg_visc + (1 + k) * n_e * N3 + e * N3 + n);
    if (KR) {
#pragma unroll
      for (int k = 0; k < 3; ++k)
        sQ[(11 + MV_REC + 6 + k) * QS + n] = __ldg(reinterpret_cast<const float*>(P.X) + (e * 3 + k) * N3 + n);
    }
  }
  constexpr int OF = NQ * N2;
  __syncthreads();
  mv_extrap<N, T, NQ, 0, 1, 1>(sQ, QS, sX, OF, N2, 0, o2);
  __syncthreads();
  mv_family_flux<N, KR, 0>(P, c, e, Sfam, sX, sNb, sMt);
  __syncthreads();
  mv_deriv<N, T, 7, 0, false>(sX, OF, N2, sR, QS, o2);
  __syncthreads();
  mv_extrap<N, T, NQ, 1, 2, 1>(sQ, QS, sX, OF, N2, 0, o2);
  __syncthreads();
  mv_family_flux<N, KR, 1>(P, c, e, Sfam, sX, sNb, sMt);
  __syncthreads();
  mv_deriv<N, T, 7, 1, true>(sX, OF, N2, sR, QS, o2);
  __syncthreads();
  mv_extrap<N, T, NQ, 2, 3, 1>(sQ, QS, sX, OF, N2, 0, o2);
  __syncthreads();
  mv_family_flux<N, KR, 2>(P, c, e, Sfam, sX, sNb, sMt);
  __syncthreads();
  mv_deriv<N, T, 7, 2, true>(sX, OF, N2, sR, QS, o2);
  __syncthreads();
  const int64_t pl = n_e * N3;
  for (int n = tid; n < N3; n += T) {
    const int64_t g = e * N3 + n;
    const float iJ = __ldg(reinterpret_cast<const float*>(P.invJ) + g);
#pragma unroll
    for (int v = 0; v < 7; ++v) {
      float r = sR[v * QS + n] * iJ;            // + div(S F_vis)/|J|
      if (v == 3) r += __ldg(P.bg_visc + g);  // the background's viscous residual (energy)
      P.rvis_out[v * pl + g] = r;
    }
  }
}

template <int N>
cudaError_t launch_mixed_visc_t(const StageParams& Pg, const StageParams& Pv, const Ops<float>& ops, const Ops2& o2,
                                cudaStream_t s) {
  using MD = MVDims<N>;
  if (Pg.n_e == 0) return cudaSuccess;
  // every buffer the two kernels address (a missing one is a caller's error, not a fault)
  if (!Pg.tr_in || !Pg.bg || !Pg.bg_jump || !Pg.bg_vtr || !Pg.mgrad_out || !Pg.mvf_out || !Pv.mgrad || !Pv.mvf_in ||
      !Pv.bg_visc || !Pv.rvis_out)
    return cudaErrorInvalidValue;
  const bool kr = Pv.kappa_r1 != 0.0 || Pv.kappa_r2 != 0.0;
  auto kv = kr ? mvisc_kernel<N, true> : mvisc_kernel<N, false>;
  const size_t vbytes = kr ? MD::template V<true>::bytes : MD::template V<false>::bytes;
  cudaError_t err = cudaSuccess;
  if (MD::gbytes > 48 * 1024)
    err = cudaFuncSetAttribute(mgrad_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MD::gbytes);
  if (err == cudaSuccess && vbytes > 48 * 1024)
    err = cudaFuncSetAttribute(kv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vbytes);
  if (err != cudaSuccess) return err;
  const MViscCoef c = mvisc_coef(Pv);
  mgrad_kernel<N><<<(unsigned)Pg.n_e, MD::T, MD::gbytes, s>>>(Pg, ops, o2, c);
  err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  kv<<<(unsigned)Pv.n_e, MD::TV, vbytes, s>>>(Pv, o2, c);
  return cudaGetLastError();
}

}  // namespace sd
