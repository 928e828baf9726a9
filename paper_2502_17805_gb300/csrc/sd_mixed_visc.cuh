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
// mgrad_kernel writes grad w' [e][24][N^3] and its face traces [e][F][24][N^2];
// mvisc_kernel writes the viscous residual of the stage state (background's
// included) [7][n_e N^3] (components rho U, E, B), which the stage kernel adds.
// Walls pass this side's own viscous flux (no wall conditions of the viscous
// path); meshes with far-field faces are not taken.
#pragma once

#include "sd_internal.h"
#include "sd_physics.cuh"
#include "sd_stage.cuh"

namespace sd {

struct MViscCoef {
  float gm1, mu, lam, eta, kappa, kappa_r, kappa_r1, kappa_r2, R, cp, inv_gamma, inv_R;
  bool kr_varies;
};

__device__ __forceinline__ MViscCoef mvisc_coef(const StageParams& P) {
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

// p' of a perturbation q'(9) about (rho0, p0): the pressure minus p0
__device__ __forceinline__ float mv_pprime(const float* q, float r0, const MViscCoef& c) {
  const float rho = r0 + q[0];
  const float m2 = q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
  const float B2 = q[5] * q[5] + q[6] * q[6] + q[7] * q[7];
  return c.gm1 * (q[4] - 0.5f * (m2 / rho + B2 + q[8] * q[8]));
}

// w' = (u, v, w, T', S', Bx, By, Bz) of the perturbation q'(9) about (r0, p0)
__device__ __forceinline__ void mv_prim(const float* q, float r0, float p0, const MViscCoef& c, float* w) {
  const float rho = r0 + q[0];
  const float ir = 1.0f / rho;
  w[0] = q[1] * ir;
  w[1] = q[2] * ir;
  w[2] = q[3] * ir;
  const float pp = mv_pprime(q, r0, c);
  w[3] = (pp * r0 - p0 * q[0]) * ir / (r0 * c.R);
  w[4] = c.cp * (log1pf(pp / p0) * c.inv_gamma - log1pf(q[0] / r0));
  w[5] = q[5];
  w[6] = q[6];
  w[7] = q[7];
}

// (F_vis(Q0 + q') - F_vis(Q0)) . n from q'(9), the background (r0, p0), the
// perturbation gradients g[3 c + j] = d w'_c / d x_j and the background's
// gT0 = grad T0, gS0 = grad S0, with the radiative diffusivity kr at the point.
// F[0..6] = components rho U (3), E, B (3).
__device__ __forceinline__ void mv_flux(const float* q, float r0, float p0, const float* g, const float* gT0,
                                        const float* gS0, float nx, float ny, float nz, const MViscCoef& c, float kr,
                                        float* F) {
  const float rho = r0 + q[0];
  const float ir = 1.0f / rho;
  const float U[3] = {q[1] * ir, q[2] * ir, q[3] * ir};
  const float pp = mv_pprime(q, r0, c);
  const float n[3] = {nx, ny, nz};
  const float divu = g[0] + g[4] + g[8];
  float tn[3] = {0.0f, 0.0f, 0.0f}, uT[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const float t = c.mu * (g[3 * i + j] + g[3 * j + i]) + (i == j ? c.lam * divu : 0.0f);
      tn[i] += t * n[j];
      uT[j] += U[i] * t;
    }
  const float Jx = g[3 * 7 + 1] - g[3 * 6 + 2], Jy = g[3 * 5 + 2] - g[3 * 7 + 0], Jz = g[3 * 6 + 0] - g[3 * 5 + 1];
  const float Bx = q[5], By = q[6], Bz = q[7];
  const float BJ[3] = {By * Jz - Bz * Jy, Bz * Jx - Bx * Jz, Bx * Jy - By * Jx};
  const float rT = (p0 + pp) * c.inv_R;  // rho T of the full state
  const float dRT = pp * c.inv_R;        // rho T - rho0 T0
  float e = 0.0f;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const float qh = -c.kappa * (rT * g[3 * 4 + j] + dRT * gS0[j]) - kr * c.cp * (rho * g[3 * 3 + j] + q[0] * gT0[j]);
    e += (uT[j] - qh + c.eta * BJ[j]) * n[j];
  }
  F[0] = tn[0];
  F[1] = tn[1];
  F[2] = tn[2];
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
// points, [11][N^3]: the increment form's stored q' of q^n plus the register D
// (stages that read it), or the FP64 state q_in less the background.
template <int N>
__device__ __forceinline__ void mv_load_state(const StageParams& P, int64_t e, float* sQ, int T) {
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
        sQ[v * N3 + n] = x;
      }
    } else {
      const int64_t g = e * P.stride + n;
      double qv[9];
#pragma unroll
      for (int v = 0; v < 9; ++v) qv[v] = __ldg(P.q_in + v * P.plane + g);
      sQ[0 * N3 + n] = f64_to_f32(qv[0] - f32_to_f64(r0));
#pragma unroll
      for (int v = 1; v < 9; ++v) sQ[v * N3 + n] = f64_to_f32(qv[v]);
      sQ[4 * N3 + n] = f64_to_f32(fma(-f32_to_f64(p0), P.inv_gm1, qv[4]));
    }
    sQ[9 * N3 + n] = r0;
    sQ[10 * N3 + n] = p0;
  }
}

template <int N>
struct MVDims {
  static constexpr int N2 = N * N, N3 = N2 * N, NF = N + 1;
  static constexpr int MAXW = 6 * N2 > N3 ? 6 * N2 : N3;
  static constexpr int T = ((MAXW + 31) / 32) * 32;
};

// BR1 gradients of w' and their face traces.
template <int N>
__global__ void __launch_bounds__(MVDims<N>::T) mgrad_kernel(const StageParams P, const Ops<float> ops) {
  using MD = MVDims<N>;
  constexpr int N2 = MD::N2, N3 = MD::N3, NF = MD::NF, T = MD::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sQ = reinterpret_cast<float*>(smem_raw);  // [11][N3]
  float* sW = sQ + 11 * N3;                          // [8][NF][N2] one family
  float* sG = sW + 8 * NF * N2;                      // [24][N3]
  const int tid = threadIdx.x;
  const int64_t e = blockIdx.x;
  const float* Sfam = reinterpret_cast<const float*>(P.Sfam) + e * (9 * N2 * NF);
  const MViscCoef c = mvisc_coef(P);
  mv_load_state<N>(P, e, sQ, T);
  const int n = tid;
  const int i0 = n % N, j0 = (n / N) % N, k0 = n / N2;
  float acc[NGRAD];
#pragma unroll
  for (int k = 0; k < NGRAD; ++k) acc[k] = 0.0f;
#pragma unroll 1
  for (int d = 0; d < 3; ++d) {
    __syncthreads();
    // w' at the flux points of family d, the BR1 common value at the two faces
    for (int t = tid; t < NF * N2; t += T) {
      const int f = t % NF, line = t / NF, a = line % N, b = line / N;
      float Qf[11], w[8];
#pragma unroll
      for (int v = 0; v < 11; ++v) {
        float s = 0.0f;
#pragma unroll
        for (int i = 0; i < N; ++i) s = fmaf(ops.E[f * N + i], sQ[v * N3 + sol_index<N>(d, i, a, b)], s);
        Qf[v] = s;
      }
      mv_prim(Qf, Qf[9], Qf[10], c, w);
      if (f == 0 || f == N) {
        const int side = f == N, F = 2 * d + side;
        const int64_t gidx = e * 6 + F;
        const int nb = __ldg(P.nbr + gidx), mt = __ldg(P.meta + gidx);
        float q2[9], w2[8], r2 = Qf[9], p2 = Qf[10];
        if (nb >= 0) {
          const int code = meta_code(mt);
          const int u = (code & 4) ? b : a, ww = (code & 4) ? a : b;
          const int a2 = (code & 2) ? N - 1 - u : u, b2 = (code & 1) ? N - 1 - ww : ww;
          const float* Tn =
              reinterpret_cast<const float*>(P.tr_in) + ((int64_t)nb * 6 + meta_nbF(mt)) * 9 * N2 + a2 + N * b2;
#pragma unroll
          for (int v = 0; v < 9; ++v) q2[v] = Tn[v * N2];
          const int pt = a + N * b;
          r2 += __ldg(P.bg_jump + (gidx * 2 + 0) * N2 + pt);
          p2 += __ldg(P.bg_jump + (gidx * 2 + 1) * N2 + pt);
        } else {
          const float* Sp = Sfam + s32_index(N, d, f, 0, line);
          const float Sx = Sp[0], Sy = Sp[N2], Sz = Sp[2 * N2];
          const float im = rsqrtf(Sx * Sx + Sy * Sy + Sz * Sz), sg = side ? 1.0f : -1.0f;
          wall_ghost<float>(Qf, sg * Sx * im, sg * Sy * im, sg * Sz * im, meta_bc(mt), q2);
        }
        mv_prim(q2, r2, p2, c, w2);
#pragma unroll
        for (int k = 0; k < 8; ++k) w[k] = 0.5f * (w[k] + w2[k]);
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) sW[(k * NF + f) * N2 + line] = w[k];
    }
    __syncthreads();
    // sum_f D[i][f] S^d_j w'_f at this thread's solution point
    if (n < N3) {
      const int id = d == 0 ? i0 : (d == 1 ? j0 : k0);
      const int line = d == 0 ? j0 + N * k0 : (d == 1 ? i0 + N * k0 : i0 + N * j0);
#pragma unroll 1
      for (int f = 0; f <= N; ++f) {
        const float* Sp = Sfam + s32_index(N, d, f, 0, line);
        const float Df = ops.D[id * NF + f];
        const float DS0 = Df * Sp[0], DS1 = Df * Sp[N2], DS2 = Df * Sp[2 * N2];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const float wv = sW[(k * NF + f) * N2 + line];
          acc[3 * k + 0] = fmaf(DS0, wv, acc[3 * k + 0]);
          acc[3 * k + 1] = fmaf(DS1, wv, acc[3 * k + 1]);
          acc[3 * k + 2] = fmaf(DS2, wv, acc[3 * k + 2]);
        }
      }
    }
  }
  if (n < N3) {
    const float iJ = __ldg(reinterpret_cast<const float*>(P.invJ) + e * N3 + n);
    float* Ge = P.mgrad_out + e * NGRAD * N3;
#pragma unroll
    for (int k = 0; k < NGRAD; ++k) {
      const float gk = acc[k] * iJ;
      sG[k * N3 + n] = gk;
      Ge[k * N3 + n] = gk;
    }
  }
  __syncthreads();
  // face traces of the gradients
  for (int t = tid; t < 6 * N2; t += T) {
    const int F = t / N2, pt = t - F * N2, a = pt % N, b = pt / N;
    const int d = F >> 1, f = (F & 1) ? N : 0;
    float* Tr = P.mgtr_out + (e * 6 + F) * NGRAD * N2 + pt;
#pragma unroll 4
    for (int k = 0; k < NGRAD; ++k) {
      float s = 0.0f;
#pragma unroll
      for (int i = 0; i < N; ++i) s = fmaf(ops.E[f * N + i], sG[k * N3 + sol_index<N>(d, i, a, b)], s);
      Tr[k * N2] = s;
    }
  }
}

// The viscous residual of the stage state, R_vis = div(S^d . F_vis)/|J| with
// the face flux the average of both sides' (F_vis . n), background included:
// out [7][n_e N^3] (components rho U, E, B).
template <int N>
__global__ void __launch_bounds__(MVDims<N>::T) mvisc_kernel(const StageParams P, const Ops<float> ops) {
  using MD = MVDims<N>;
  constexpr int N2 = MD::N2, N3 = MD::N3, NF = MD::NF, T = MD::T;
  constexpr int NQ = 11 + NGRAD + 6 + 3;  // q', rho0, p0, grad w', grad T0, grad S0, x
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sQ = reinterpret_cast<float*>(smem_raw);  // [NQ][N3]
  float* sF = sQ + NQ * N3;                          // [7][NF][N2] one family
  const int tid = threadIdx.x;
  const int64_t e = blockIdx.x;
  const int64_t n_e = P.n_e;
  const float* Sfam = reinterpret_cast<const float*>(P.Sfam) + e * (9 * N2 * NF);
  const MViscCoef c = mvisc_coef(P);
  mv_load_state<N>(P, e, sQ, T);
  for (int n = tid; n < N3; n += T) {
#pragma unroll 4
    for (int k = 0; k < NGRAD; ++k) sQ[(11 + k) * N3 + n] = __ldg(P.mgrad + (e * NGRAD + k) * N3 + n);
#pragma unroll
    for (int k = 0; k < 6; ++k) sQ[(11 + NGRAD + k) * N3 + n] = __ldg(P.bg_visc + (1 + k) * n_e * N3 + e * N3 + n);
#pragma unroll
    for (int k = 0; k < 3; ++k)
      sQ[(11 + NGRAD + 6 + k) * N3 + n] = __ldg(reinterpret_cast<const float*>(P.X) + (e * 3 + k) * N3 + n);
  }
  const int n = tid;
  const int i0 = n % N, j0 = (n / N) % N, k0 = n / N2;
  float acc[7];
#pragma unroll
  for (int v = 0; v < 7; ++v) acc[v] = 0.0f;
#pragma unroll 1
  for (int d = 0; d < 3; ++d) {
    __syncthreads();
    for (int t = tid; t < NF * N2; t += T) {
      const int f = t % NF, line = t / NF, a = line % N, b = line / N;
      float x[NQ];
#pragma unroll
      for (int v = 0; v < NQ; ++v) {
        float s = 0.0f;
#pragma unroll
        for (int i = 0; i < N; ++i) s = fmaf(ops.E[f * N + i], sQ[v * N3 + sol_index<N>(d, i, a, b)], s);
        x[v] = s;
      }
      const float* Sp = Sfam + s32_index(N, d, f, 0, line);
      const float Sx = Sp[0], Sy = Sp[N2], Sz = Sp[2 * N2];
      const float kr = mv_kappa_r(c, x[NQ - 3], x[NQ - 2], x[NQ - 1]);
      float Fv[7];
      if (f > 0 && f < N) {
        mv_flux(x, x[9], x[10], x + 11, x + 11 + NGRAD, x + 11 + NGRAD + 3, Sx, Sy, Sz, c, kr, Fv);
      } else {
        // the average of both sides' F_vis . n along this side's outward unit normal, times |S|
        const int side = f == N, F = 2 * d + side;
        const float mag = sqrtf(Sx * Sx + Sy * Sy + Sz * Sz), im = 1.0f / mag, sg = side ? 1.0f : -1.0f;
        const float nx = sg * Sx * im, ny = sg * Sy * im, nz = sg * Sz * im;
        mv_flux(x, x[9], x[10], x + 11, x + 11 + NGRAD, x + 11 + NGRAD + 3, nx, ny, nz, c, kr, Fv);
        const int64_t gidx = e * 6 + F;
        const int nb = __ldg(P.nbr + gidx), mt = __ldg(P.meta + gidx);
        if (nb >= 0) {
          const int code = meta_code(mt);
          const int u = (code & 4) ? b : a, ww = (code & 4) ? a : b;
          const int a2 = (code & 2) ? N - 1 - u : u, b2 = (code & 1) ? N - 1 - ww : ww;
          const int64_t nf = (int64_t)nb * 6 + meta_nbF(mt);
          float q2[9], g2[NGRAD], gT2[3], gS2[3], F2[7];
          const float* Tn = reinterpret_cast<const float*>(P.tr_in) + nf * 9 * N2 + a2 + N * b2;
#pragma unroll
          for (int v = 0; v < 9; ++v) q2[v] = Tn[v * N2];
          const float* Gn = P.mgtr_in + nf * NGRAD * N2 + a2 + N * b2;
#pragma unroll
          for (int k = 0; k < NGRAD; ++k) g2[k] = Gn[k * N2];
          const float* Bn = P.bg_vtr + nf * 6 * N2 + a2 + N * b2;
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            gT2[k] = __ldg(Bn + k * N2);
            gS2[k] = __ldg(Bn + (3 + k) * N2);
          }
          const int pt = a + N * b;
          const float r2 = x[9] + __ldg(P.bg_jump + (gidx * 2 + 0) * N2 + pt);
          const float p2 = x[10] + __ldg(P.bg_jump + (gidx * 2 + 1) * N2 + pt);
          mv_flux(q2, r2, p2, g2, gT2, gS2, nx, ny, nz, c, kr, F2);
#pragma unroll
          for (int v = 0; v < 7; ++v) Fv[v] = 0.5f * (Fv[v] + F2[v]);
        }
        const float sm = sg * mag;
#pragma unroll
        for (int v = 0; v < 7; ++v) Fv[v] *= sm;
      }
#pragma unroll
      for (int v = 0; v < 7; ++v) sF[(v * NF + f) * N2 + line] = Fv[v];
    }
    __syncthreads();
    if (n < N3) {
      const int id = d == 0 ? i0 : (d == 1 ? j0 : k0);
      const int line = d == 0 ? j0 + N * k0 : (d == 1 ? i0 + N * k0 : i0 + N * j0);
#pragma unroll
      for (int f = 0; f <= N; ++f) {
        const float Df = ops.D[id * NF + f];
#pragma unroll
        for (int v = 0; v < 7; ++v) acc[v] = fmaf(Df, sF[(v * NF + f) * N2 + line], acc[v]);
      }
    }
  }
  if (n < N3) {
    const float iJ = __ldg(reinterpret_cast<const float*>(P.invJ) + e * N3 + n);
    const int64_t pl = n_e * N3, g = e * N3 + n;
#pragma unroll
    for (int v = 0; v < 7; ++v) {
      float r = acc[v] * iJ;                                  // + div(S F_vis)/|J|
      if (v == 3) r += __ldg(P.bg_visc + g);                  // the background's viscous residual (energy)
      P.rvis_out[v * pl + g] = r;
    }
  }
}

template <int N>
cudaError_t launch_mixed_visc_t(const StageParams& Pg, const StageParams& Pv, const Ops<float>& ops, cudaStream_t s) {
  using MD = MVDims<N>;
  constexpr size_t gbytes = (size_t)(11 * MD::N3 + 8 * MD::NF * MD::N2 + NGRAD * MD::N3) * sizeof(float);
  constexpr size_t vbytes = (size_t)((11 + NGRAD + 6 + 3) * MD::N3 + 7 * MD::NF * MD::N2) * sizeof(float);
  if (Pg.n_e == 0) return cudaSuccess;
  cudaError_t err = cudaSuccess;
  if (gbytes > 48 * 1024) err = cudaFuncSetAttribute(mgrad_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gbytes);
  if (err == cudaSuccess && vbytes > 48 * 1024)
    err = cudaFuncSetAttribute(mvisc_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vbytes);
  if (err != cudaSuccess) return err;
  mgrad_kernel<N><<<(unsigned)Pg.n_e, MD::T, gbytes, s>>>(Pg, ops);
  err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  mvisc_kernel<N><<<(unsigned)Pv.n_e, MD::T, vbytes, s>>>(Pv, ops);
  return cudaGetLastError();
}

}  // namespace sd
