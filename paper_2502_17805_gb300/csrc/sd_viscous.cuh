// sd_viscous.cuh -- viscous, resistive and thermal fluxes of the FP64 path.
//
// F = F_inv - F_vis (Sec. MHD Governing Equations) with
//   F_vis . n = (0, tau n, (U . tau - q + eta B x J) . n, eta J x n, 0),
//   tau = mu (grad U + grad U^T) - 2/3 mu (div U) I,
//   q   = -kappa rho T grad S - kappa_r rho C_p grad T,   J = curl B,
// from the gradients of the primitive variables w = (U, T, S, B),
// T = p / (rho R), S = C_p ln(p^(1/gamma) / rho).  BR1 (Sec. SD Method): w is
// evaluated from the conserved state at the flux points of each family, its
// common value at an element face is the average of the two sides (the far
// side being the neighbour's face trace or the wall / far-field ghost state),
// and |J| dw/dx_j = sum_d D_d (S^d_j w) at the solution points.  The gradients
// are extrapolated to the flux points like the state; at an element face the
// viscous flux is the average of the two sides' F_vis . n (a wall or far-field
// face takes this side's alone).
//
// F_vis is linear in the gradients through 15 values per point, the record:
// tau (xx, yy, zz, xy, xz, yz), J (x, y, z), grad T, grad S.  Extrapolation is
// linear too, so the record is formed once at the solution points and
// extrapolated in place of the 24 gradient components.
//
// visc_f64_kernel (one element per CTA, before every stage) writes the record's
// face traces [e][F][15][N^2] (the face-flux kernel's input: it adds the common
// viscous flux to the Rusanov flux, once per face point, by the owner) and the
// interior part of the viscous divergence, sum_d D_d (S^d . F_vis) over the
// interior flux points [e][7][N^3] (components rho U, E, B: the element kernel
// subtracts it from its flux divergence).  Its phases run along the lines of
// one family at a time in the even-odd form of the 1D operators, like the
// element kernel:
//   A  load the state
//   for each family d:
//     B1 extrapolate the state to the interior flux points of every line (the
//        element's own face traces give the two faces)
//     B2 w at every flux point, the BR1 average at the two faces
//     B3 sum_f D[i][f] S^d_j(f) w_k(f) along every line, for the 21 (k, j) the
//        record takes
//   C  gradients -> the record at the solution points
//   D  the record's face traces (both ends of every line)
//   for each family d:
//     E1 extrapolate the state and the record to the interior flux points
//     E2 S^d . F_vis at every interior flux point
//     E3 derivative along every line of the interior values
//   F  write the interior divergence.
// GB300 issues two FP64 FMA per SM and clock: the kernel is bound by its FP64
// operations, of which the two logarithms of S at every flux point and the 24
// gradient components' derivatives are the largest share.
#pragma once

#include "sd_internal.h"
#include "sd_physics.cuh"
#include "sd_stage.cuh"

namespace sd {

struct ViscCoef {
  double gamma, mu, lam, eta, kappa, kappa_r, kappa_r1, kappa_r2, R, cp, inv_gamma;
  bool kr_varies;  // kappa_r depends on the radius
};

// radiative diffusivity at position (x, y, z): kappa_r + kappa_r1 r + kappa_r2 r^2
__device__ __forceinline__ double kappa_r_at(const ViscCoef& c, double x, double y, double z) {
  const double r = sqrt(x * x + y * y + z * z);
  return c.kappa_r + c.kappa_r1 * r + c.kappa_r2 * r * r;
}

__host__ __device__ inline ViscCoef visc_coef(const StageParams& P) {
  ViscCoef c;
  c.gamma = P.gamma;
  c.mu = P.mu;
  c.lam = -2.0 / 3.0 * P.mu;
  c.eta = P.eta;
  c.kappa = P.kappa;
  c.kappa_r = P.kappa_r;
  c.kappa_r1 = P.kappa_r1;
  c.kappa_r2 = P.kappa_r2;
  c.kr_varies = P.kappa_r1 != 0.0 || P.kappa_r2 != 0.0;
  c.R = P.R_gas;
  c.cp = P.gamma * P.R_gas / (P.gamma - 1.0);
  c.inv_gamma = 1.0 / P.gamma;
  return c;
}

// (u, v, w, T, S, Bx, By, Bz) of a conserved state
__device__ __forceinline__ void prim_w(const double* Q, const ViscCoef& c, double* w) {
  const double ir = 1.0 / Q[0];
  w[0] = Q[1] * ir;
  w[1] = Q[2] * ir;
  w[2] = Q[3] * ir;
  const double p = (c.gamma - 1.0) * (Q[4] - 0.5 * (Q[1] * w[0] + Q[2] * w[1] + Q[3] * w[2]) -
                                      0.5 * (Q[5] * Q[5] + Q[6] * Q[6] + Q[7] * Q[7]) - 0.5 * Q[8] * Q[8]);
  w[3] = p * ir / c.R;
  w[4] = c.cp * (log(p) * c.inv_gamma - log(Q[0]));
  w[5] = Q[5];
  w[6] = Q[6];
  w[7] = Q[7];
}

// The record from the gradients g[3 c + j] = d w_c / d x_j.
__device__ __forceinline__ void visc_record(const double* g, const ViscCoef& c, double* rec) {
  const double ld = c.lam * (g[0] + g[4] + g[8]);
  rec[0] = 2.0 * c.mu * g[0] + ld;
  rec[1] = 2.0 * c.mu * g[4] + ld;
  rec[2] = 2.0 * c.mu * g[8] + ld;
  rec[3] = c.mu * (g[1] + g[3]);
  rec[4] = c.mu * (g[2] + g[6]);
  rec[5] = c.mu * (g[5] + g[7]);
  rec[6] = g[3 * 7 + 1] - g[3 * 6 + 2];
  rec[7] = g[3 * 5 + 2] - g[3 * 7 + 0];
  rec[8] = g[3 * 6 + 0] - g[3 * 5 + 1];
#pragma unroll
  for (int k = 0; k < 6; ++k) rec[9 + k] = g[9 + k];
}

// velocity and temperature of a conserved state
__device__ __forceinline__ void visc_prim(const double* Q, const ViscCoef& c, double* u, double& T) {
  const double ir = 1.0 / Q[0];
  u[0] = Q[1] * ir;
  u[1] = Q[2] * ir;
  u[2] = Q[3] * ir;
  const double p = (c.gamma - 1.0) * (Q[4] - 0.5 * (Q[1] * u[0] + Q[2] * u[1] + Q[3] * u[2]) -
                                      0.5 * (Q[5] * Q[5] + Q[6] * Q[6] + Q[7] * Q[7]) - 0.5 * Q[8] * Q[8]);
  T = p * ir / c.R;
}

// F_vis contracted with the vector (nx, ny, nz) (not necessarily a unit vector), from the
// state Q and the record: Fv[0..6] = components rho U (3), E, B (3); rho and psi carry none.
__device__ __forceinline__ void visc_flux_rec(const double* Q, const double* rec, double nx, double ny, double nz,
                                              const ViscCoef& c, double kr, double* Fv) {
  double u[3], T;
  visc_prim(Q, c, u, T);
  const double tx = rec[0] * nx + rec[3] * ny + rec[4] * nz;
  const double ty = rec[3] * nx + rec[1] * ny + rec[5] * nz;
  const double tz = rec[4] * nx + rec[5] * ny + rec[2] * nz;
  const double Jx = rec[6], Jy = rec[7], Jz = rec[8];
  const double Bx = Q[5], By = Q[6], Bz = Q[7];
  const double rT = Q[0] * T, rc = kr * Q[0] * c.cp;
  // -q . n, q = -kappa rho T grad S - kappa_r rho C_p grad T
  const double mq = (c.kappa * rT * rec[12] + rc * rec[9]) * nx + (c.kappa * rT * rec[13] + rc * rec[10]) * ny +
                    (c.kappa * rT * rec[14] + rc * rec[11]) * nz;
  const double bj = (By * Jz - Bz * Jy) * nx + (Bz * Jx - Bx * Jz) * ny + (Bx * Jy - By * Jx) * nz;
  Fv[0] = tx;
  Fv[1] = ty;
  Fv[2] = tz;
  Fv[3] = u[0] * tx + u[1] * ty + u[2] * tz + mq + c.eta * bj;
  Fv[4] = c.eta * (Jy * nz - Jz * ny);
  Fv[5] = c.eta * (Jz * nx - Jx * nz);
  Fv[6] = c.eta * (Jx * ny - Jy * nx);
}

// Viscous flux through a wall face along its unit outward normal n (visc_walls):
// stress-free and impenetrable, only the normal stress n.tau.n acts, on the face
// state qf = (own + ghost) / 2 (whose normal velocity vanishes); the heat flux is
// q_bottom into the shell on the inner sphere (q = q_bottom r^, n = -r^) and the
// conducted one on the outer; the resistive terms take this side's current, of
// which a perfectly conducting wall keeps only the normal part (J = J_r r^).
// Fv as for visc_flux_rec.
__device__ __forceinline__ void wall_visc_flux_rec(const double* qo, const double* qn, const double* rec, double nx,
                                                   double ny, double nz, bool outer, bool conducting,
                                                   double q_bottom, const ViscCoef& c, double kr, double* Fv) {
  double qf[9], u[3], T;
#pragma unroll
  for (int v = 0; v < 9; ++v) qf[v] = 0.5 * (qo[v] + qn[v]);
  visc_prim(qf, c, u, T);
  const double tnn = rec[0] * nx * nx + rec[1] * ny * ny + rec[2] * nz * nz +
                     2.0 * (rec[3] * nx * ny + rec[4] * nx * nz + rec[5] * ny * nz);
  double Jx = rec[6], Jy = rec[7], Jz = rec[8];
  if (conducting) {  // a perfectly conducting wall: J = J_r r^, the normal part only
    const double jn = Jx * nx + Jy * ny + Jz * nz;
    Jx = jn * nx;
    Jy = jn * ny;
    Jz = jn * nz;
  }
  const double Bx = qf[5], By = qf[6], Bz = qf[7];
  const double bj = c.eta * ((By * Jz - Bz * Jy) * nx + (Bz * Jx - Bx * Jz) * ny + (Bx * Jy - By * Jx) * nz);
  double qdn;
  if (outer) {
    const double rT = qf[0] * T, rc = kr * qf[0] * c.cp;
    qdn = -((c.kappa * rT * rec[12] + rc * rec[9]) * nx + (c.kappa * rT * rec[13] + rc * rec[10]) * ny +
            (c.kappa * rT * rec[14] + rc * rec[11]) * nz);
  } else {
    qdn = -q_bottom;
  }
  const double un = u[0] * nx + u[1] * ny + u[2] * nz;
  Fv[0] = tnn * nx;
  Fv[1] = tnn * ny;
  Fv[2] = tnn * nz;
  Fv[3] = un * tnn - qdn + bj;
  Fv[4] = c.eta * (Jy * nz - Jz * ny);
  Fv[5] = c.eta * (Jz * nx - Jx * nz);
  Fv[6] = c.eta * (Jx * ny - Jy * nx);
}

// position of flux point (d, f, a, b) of element e: the map is a polynomial of
// degree floor(N/2) < N, so E gives it exactly from the solution points
template <int N>
__device__ __forceinline__ double visc_kr(const ViscCoef& c, const Ops<double>& ops, const double* X, int64_t e, int d,
                                          int f, int a, int b) {
  if (!c.kr_varies) return c.kappa_r;
  constexpr int N3 = N * N * N;
  const double* Xe = X + e * 3 * N3;
  double x[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < N; ++i) s = fma(ops.E[f * N + i], __ldg(Xe + k * N3 + sol_index<N>(d, i, a, b)), s);
    x[k] = s;
  }
  return kappa_r_at(c, x[0], x[1], x[2]);
}

// ---- 1D operators along a line in the even-odd form (E[N-f][N-1-i] = E[f][i],
// D[N-1-i][f] = -D[i][N-f]); x: the N values of a line at its solution points

// the flux points F0 <= f <= N - F0 (F0 = 0: all N + 1; F0 = 1: the interior ones)
template <int N, int F0 = 0>
__device__ __forceinline__ void eo_extrap(const double* x, const Ops<double>& ops, double* y) {
  constexpr int HP = N / 2;
  double sv[HP], dv[HP];
#pragma unroll
  for (int i = 0; i < HP; ++i) {
    sv[i] = x[i] + x[N - 1 - i];
    dv[i] = x[i] - x[N - 1 - i];
  }
#pragma unroll
  for (int f = F0; 2 * f <= N; ++f) {
    double a = (N & 1) ? ops.Es[f * N + HP] * x[HP] : 0.0;
    double b = 0.0;
#pragma unroll
    for (int i = 0; i < HP; ++i) {
      a = fma(ops.Es[f * N + i], sv[i], a);
      b = fma(ops.Ed[f * N + i], dv[i], b);
    }
    if (2 * f == N) {
      y[f] = a;
    } else {
      y[f] = a + b;
      y[N - f] = a - b;
    }
  }
}

// derivative at the N solution points of the flux polynomial through y[0..N]
template <int N>
__device__ __forceinline__ void eo_deriv(const double* y, const Ops<double>& ops, double* o) {
  constexpr int NF = N + 1, HF = NF / 2;
  double sf[HF], df[HF];
#pragma unroll
  for (int f = 0; f < HF; ++f) {
    sf[f] = y[f] + y[N - f];
    df[f] = y[f] - y[N - f];
  }
#pragma unroll
  for (int i = 0; 2 * i <= N - 1; ++i) {
    double p = (NF & 1) ? ops.Ds[i * NF + HF] * y[HF] : 0.0;
    double r = 0.0;
#pragma unroll
    for (int f = 0; f < HF; ++f) {
      p = fma(ops.Ds[i * NF + f], sf[f], p);
      r = fma(ops.Dd[i * NF + f], df[f], r);
    }
    if (2 * i == N - 1) {
      o[i] = r;
    } else {
      o[i] = p + r;
      o[N - 1 - i] = r - p;
    }
  }
}

// The gradient components the record takes: all of U, T and S (m < 15: k = m / 3,
// j = m % 3) and the off-diagonal ones of B (m >= 15: d B_k / d x_j with j != k - 5).
constexpr int NGRAD_REC = 21;
__device__ __forceinline__ void grad_component(int m, int& k, int& j) {
  if (m < 15) {
    k = m / 3;
    j = m - 3 * k;
  } else {
    const int r = m - 15, kb = r >> 1;  // B component 0..2
    k = 5 + kb;
    j = (r & 1) ? (kb == 2 ? 1 : 2) : (kb == 0 ? 1 : 0);
  }
}

template <int N>
struct DimsVisc {
  static constexpr int N2 = N * N, N3 = N2 * N, NF = N + 1, NI = N - 1;
  static constexpr int T = N >= 6 ? 256 : 128;
  static constexpr int oQ = 0;                       // [9][N3] the state
  static constexpr int oB = 9 * N3;                  // [24][N3] gradient sums, then [24][NI][N2]
  static constexpr int oC = oB + NGRAD * N3;         // [9][NF][N2] one family's flux points, then [15][N3]
  static constexpr int nC = 9 * NF * N2 > MV_REC * N3 ? 9 * NF * N2 : MV_REC * N3;
  static constexpr int oR = oC + nC;                 // [7][N3] interior viscous divergence
  static constexpr size_t bytes = (size_t)(oR + 7 * N3) * sizeof(double);
  static constexpr int minb = bytes <= 113 * 1024 ? 2 : 1;
  static_assert((9 + MV_REC) * NI * N2 <= NGRAD * N3, "interior values fit the gradient sums' space");
};

// The record's face traces and the interior viscous divergence of P.q_in (whose face
// traces are P.tr_in) into P.gtr_out and P.rvis64_out; the record at the solution
// points into P.grad_out when that is set.
template <int N>
__global__ void __launch_bounds__(DimsVisc<N>::T, DimsVisc<N>::minb)
    visc_f64_kernel(const StageParams P, const Ops<double> ops) {
  using DV = DimsVisc<N>;
  constexpr int N2 = DV::N2, N3 = DV::N3, NF = DV::NF, NI = DV::NI, T = DV::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sQ = reinterpret_cast<double*>(smem_raw) + DV::oQ;
  double* sB = reinterpret_cast<double*>(smem_raw) + DV::oB;
  double* sC = reinterpret_cast<double*>(smem_raw) + DV::oC;
  double* sR = reinterpret_cast<double*>(smem_raw) + DV::oR;
  const int tid = threadIdx.x;
  const int64_t e = blockIdx.x;
  const double* Sfam = reinterpret_cast<const double*>(P.Sfam) + e * (9 * N2 * NF);
  const ViscCoef c = visc_coef(P);

  // ---- A: load
  for (int n = tid; n < N3; n += T) {
#pragma unroll
    for (int v = 0; v < 9; ++v) sQ[v * N3 + n] = __ldg(P.q_in + v * P.plane + e * P.stride + n);
  }
  __syncthreads();

#pragma unroll 1
  for (int d = 0; d < 3; ++d) {
    // ---- B1: the state at the interior flux points of the family's lines (at the two
    // faces it is the element's own face trace, which B2 reads)
    for (int t = tid; t < 9 * N2; t += T) {
      const int v = t / N2, L = t - v * N2;
      int base, str;
      line_geom<N>(d, L, base, str);
      double x[N], y[NF];
#pragma unroll
      for (int i = 0; i < N; ++i) x[i] = sQ[v * N3 + base + i * str];
      eo_extrap<N, 1>(x, ops, y);
#pragma unroll
      for (int f = 1; f < N; ++f) sC[(v * NF + f) * N2 + L] = y[f];
    }
    __syncthreads();
    // ---- B2: w at every flux point; at the faces the BR1 average with the far side
    for (int t = tid; t < NF * N2; t += T) {
      const int f = t / N2, L = t - f * N2, a = L % N, b = L / N;
      double Qf[9], w[8];
      if (f == 0 || f == N) {
        const double* To = reinterpret_cast<const double*>(P.tr_in) + (e * 6 + 2 * d + (f == N)) * 9 * N2 + L;
#pragma unroll
        for (int v = 0; v < 9; ++v) Qf[v] = __ldg(To + v * N2);
      } else {
#pragma unroll
        for (int v = 0; v < 9; ++v) Qf[v] = sC[(v * NF + f) * N2 + L];
      }
      prim_w(Qf, c, w);
      if (f == 0 || f == N) {
        const int side = f == N, F = 2 * d + side;
        const int nb = __ldg(P.nbr + e * 6 + F), mt = __ldg(P.meta + e * 6 + F);
        double Q2[9], w2[8];
        if (nb >= 0) {
          const int code = meta_code(mt);
          const int u = (code & 4) ? b : a, ww = (code & 4) ? a : b;
          const int a2 = (code & 2) ? N - 1 - u : u, b2 = (code & 1) ? N - 1 - ww : ww;
          const double* Tn =
              reinterpret_cast<const double*>(P.tr_in) + ((int64_t)nb * 6 + meta_nbF(mt)) * 9 * N2 + a2 + N * b2;
#pragma unroll
          for (int v = 0; v < 9; ++v) Q2[v] = __ldg(Tn + v * N2);
        } else if (meta_bc(mt) == SD_BC_FARFIELD) {
#pragma unroll
          for (int v = 0; v < 9; ++v) Q2[v] = P.farfield[v];
        } else {
          const double* Sp = Sfam + (d * 3 * N2 + L) * NF + f;
          const double Sx = __ldg(Sp), Sy = __ldg(Sp + N2 * NF), Sz = __ldg(Sp + 2 * N2 * NF);
          const double im = 1.0 / sqrt(Sx * Sx + Sy * Sy + Sz * Sz), sg = side ? 1.0 : -1.0;
          wall_ghost<double>(Qf, sg * Sx * im, sg * Sy * im, sg * Sz * im, meta_bc(mt), Q2);
        }
        prim_w(Q2, c, w2);
        if (nb < 0 && P.visc_walls && meta_outer(mt)) w2[3] = 2.0 * P.T_top - w[3];  // T held on the outer wall
#pragma unroll
        for (int k = 0; k < 8; ++k) w[k] = 0.5 * (w[k] + w2[k]);
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) sC[(k * NF + f) * N2 + L] = w[k];
    }
    __syncthreads();
    // ---- B3: sum_f D[i][f] S^d_j(f) w_k(f) along every line, component 3 k + j, for the
    // 21 components the record takes (not the diagonal of grad B)
    for (int t = tid; t < NGRAD_REC * N2; t += T) {
      const int m = t / N2, L = t - m * N2;
      int k, j;
      grad_component(m, k, j);
      const int kj = 3 * k + j;
      int base, str;
      line_geom<N>(d, L, base, str);
      const double* Sp = Sfam + ((d * 3 + j) * N2 + L) * NF;
      double y[NF], o[N];
#pragma unroll
      for (int f = 0; f <= N; ++f) y[f] = __ldg(Sp + f) * sC[(k * NF + f) * N2 + L];
      eo_deriv<N>(y, ops, o);
      double* G = sB + kj * N3 + base;
      if (d == 0) {
#pragma unroll
        for (int i = 0; i < N; ++i) G[i * str] = o[i];
      } else {
#pragma unroll
        for (int i = 0; i < N; ++i) G[i * str] += o[i];
      }
    }
    __syncthreads();
  }

  // ---- C: the gradients, then the record, at the solution points
  for (int n = tid; n < N3; n += T) {
    const double iJ = __ldg(reinterpret_cast<const double*>(P.invJ) + e * N3 + n);  // 1 / |J|
    double g[NGRAD], rec[MV_REC];
#pragma unroll
    for (int m = 0; m < NGRAD_REC; ++m) {
      int k, j;
      grad_component(m, k, j);
      g[3 * k + j] = sB[(3 * k + j) * N3 + n] * iJ;
    }
    visc_record(g, c, rec);  // reads no diagonal component of grad B
#pragma unroll
    for (int k = 0; k < MV_REC; ++k) sC[k * N3 + n] = rec[k];
    if (P.grad_out) {
#pragma unroll
      for (int k = 0; k < MV_REC; ++k) P.grad_out[(e * MV_REC + k) * N3 + n] = rec[k];
    }
  }
  __syncthreads();

  // ---- D: the record's face traces, both ends of every line (E[N][i] = E[0][N-1-i])
  for (int t = tid; t < 3 * MV_REC * N2; t += T) {
    const int d = t / (MV_REC * N2), r = t - d * (MV_REC * N2), k = r / N2, L = r - k * N2;
    int base, str;
    line_geom<N>(d, L, base, str);
    constexpr int HP = N / 2;
    double x[N];
#pragma unroll
    for (int i = 0; i < N; ++i) x[i] = sC[k * N3 + base + i * str];
    double a = (N & 1) ? ops.Es[HP] * x[HP] : 0.0, bb = 0.0;
#pragma unroll
    for (int i = 0; i < HP; ++i) {
      a = fma(ops.Es[i], x[i] + x[N - 1 - i], a);
      bb = fma(ops.Ed[i], x[i] - x[N - 1 - i], bb);
    }
    double* Tr = P.gtr_out + ((e * 6 + 2 * d) * MV_REC + k) * N2 + L;
    Tr[0] = a + bb;
    Tr[MV_REC * N2] = a - bb;
  }

  // ---- E: the interior part of the viscous divergence, family by family
#pragma unroll 1
  for (int d = 0; d < 3; ++d) {
    __syncthreads();
    // E1: state (c < 9) and record (c >= 9) at the interior flux points -> sB[(c NI + f - 1) N2 + L]
    for (int t = tid; t < (9 + MV_REC) * N2; t += T) {
      const int cc = t / N2, L = t - cc * N2;
      int base, str;
      line_geom<N>(d, L, base, str);
      const double* src = cc < 9 ? sQ + cc * N3 : sC + (cc - 9) * N3;
      double x[N], y[NF];
#pragma unroll
      for (int i = 0; i < N; ++i) x[i] = src[base + i * str];
      eo_extrap<N, 1>(x, ops, y);
#pragma unroll
      for (int f = 1; f < N; ++f) sB[(cc * NI + f - 1) * N2 + L] = y[f];
    }
    __syncthreads();
    // E2: S^d . F_vis at every interior flux point, into the point's first 7 slots
    for (int t = tid; t < NI * N2; t += T) {
      const int fm = t / N2, L = t - fm * N2, f = fm + 1;
      double* X = sB + fm * N2 + L;
      double q[9], rec[MV_REC], Fv[7];
#pragma unroll
      for (int v = 0; v < 9; ++v) q[v] = X[v * NI * N2];
#pragma unroll
      for (int k = 0; k < MV_REC; ++k) rec[k] = X[(9 + k) * NI * N2];
      const double* Sp = Sfam + (d * 3 * N2 + L) * NF + f;
      const double Sx = __ldg(Sp), Sy = __ldg(Sp + N2 * NF), Sz = __ldg(Sp + 2 * N2 * NF);
      const double kr = visc_kr<N>(c, ops, reinterpret_cast<const double*>(P.X), e, d, f, L % N, L / N);
      visc_flux_rec(q, rec, Sx, Sy, Sz, c, kr, Fv);
#pragma unroll
      for (int k = 0; k < 7; ++k) X[k * NI * N2] = Fv[k];
    }
    __syncthreads();
    // E3: derivative along every line of the interior values (the face values are the
    // face kernel's) -> sR
    for (int t = tid; t < 7 * N2; t += T) {
      const int k = t / N2, L = t - k * N2;
      int base, str;
      line_geom<N>(d, L, base, str);
      double y[NF], o[N];
      y[0] = 0.0;
      y[N] = 0.0;
#pragma unroll
      for (int f = 1; f < N; ++f) y[f] = sB[(k * NI + f - 1) * N2 + L];
      eo_deriv<N>(y, ops, o);
      double* R = sR + k * N3 + base;
      if (d == 0) {
#pragma unroll
        for (int i = 0; i < N; ++i) R[i * str] = o[i];
      } else {
#pragma unroll
        for (int i = 0; i < N; ++i) R[i * str] += o[i];
      }
    }
  }
  __syncthreads();
  // ---- F: write the interior divergence
  double* Ro = P.rvis64_out + e * 7 * N3;
  for (int t = tid; t < 7 * N3; t += T) Ro[t] = sR[t];
}

template <int N>
cudaError_t launch_visc_f64_t(const StageParams& P, const Ops<double>& ops, cudaStream_t s) {
  using DV = DimsVisc<N>;
  if (DV::bytes > 48 * 1024) {
    cudaError_t err =
        cudaFuncSetAttribute(visc_f64_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DV::bytes);
    if (err != cudaSuccess) return err;
  }
  if (P.n_e == 0) return cudaSuccess;
  visc_f64_kernel<N><<<(unsigned)P.n_e, DV::T, DV::bytes, s>>>(P, ops);
  return cudaGetLastError();
}

}  // namespace sd
