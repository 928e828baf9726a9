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
// grad_kernel writes the gradients of every element [e][24][N^3] and their
// face traces [e][F][24][N^2] (the neighbours' input of the next stage kernel).
#pragma once

#include "sd_internal.h"
#include "sd_physics.cuh"

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

// F_vis contracted with the vector (nx, ny, nz), from the state Q and the
// gradients g[3 c + j] = d w_c / d x_j
__device__ __forceinline__ void visc_flux(const double* Q, const double* g, double nx, double ny, double nz,
                                          const ViscCoef& c, double kr, double* F) {
  double w[8];
  prim_w(Q, c, w);
  const double n[3] = {nx, ny, nz};
  const double divu = g[0] + g[4] + g[8];
  double tn[3], uT[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) tn[i] = 0.0;
#pragma unroll
  for (int j = 0; j < 3; ++j) uT[j] = 0.0;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const double t = c.mu * (g[3 * i + j] + g[3 * j + i]) + (i == j ? c.lam * divu : 0.0);
      tn[i] += t * n[j];
      uT[j] += w[i] * t;
    }
  // J = curl B from the gradients of Bx (c = 5), By (6), Bz (7)
  const double Jx = g[3 * 7 + 1] - g[3 * 6 + 2], Jy = g[3 * 5 + 2] - g[3 * 7 + 0], Jz = g[3 * 6 + 0] - g[3 * 5 + 1];
  const double Bx = w[5], By = w[6], Bz = w[7];
  const double BJ[3] = {By * Jz - Bz * Jy, Bz * Jx - Bx * Jz, Bx * Jy - By * Jx};
  const double rT = Q[0] * w[3];
  double e = 0.0;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const double qh = -c.kappa * rT * g[3 * 4 + j] - kr * Q[0] * c.cp * g[3 * 3 + j];
    e += (uT[j] - qh + c.eta * BJ[j]) * n[j];
  }
  F[0] = 0.0;
  F[1] = tn[0];
  F[2] = tn[1];
  F[3] = tn[2];
  F[4] = e;
  F[5] = c.eta * (Jy * nz - Jz * ny);
  F[6] = c.eta * (Jz * nx - Jx * nz);
  F[7] = c.eta * (Jx * ny - Jy * nx);
  F[8] = 0.0;
}

// Viscous flux through a wall face along its unit outward normal n (visc_walls):
// stress-free and impenetrable, only the normal stress n.tau.n acts, on the face
// state qf = (own + ghost) / 2 (whose normal velocity vanishes); the heat flux is
// q_bottom into the shell on the inner sphere (q = q_bottom r^, n = -r^) and the
// conducted one on the outer; the resistive terms take this side's current, of
// which a perfectly conducting wall keeps only the normal part (J = J_r r^).
__device__ __forceinline__ void wall_visc_flux(const double* qo, const double* qn, const double* g, double nx,
                                               double ny, double nz, bool outer, bool conducting, double q_bottom,
                                               const ViscCoef& c, double kr, double* F) {
  double qf[9], w[8];
#pragma unroll
  for (int v = 0; v < 9; ++v) qf[v] = 0.5 * (qo[v] + qn[v]);
  prim_w(qf, c, w);
  const double n[3] = {nx, ny, nz};
  const double divu = g[0] + g[4] + g[8];
  double tnn = 0.0;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      tnn += n[i] * (c.mu * (g[3 * i + j] + g[3 * j + i]) + (i == j ? c.lam * divu : 0.0)) * n[j];
  double Jx = g[3 * 7 + 1] - g[3 * 6 + 2], Jy = g[3 * 5 + 2] - g[3 * 7 + 0], Jz = g[3 * 6 + 0] - g[3 * 5 + 1];
  if (conducting) {  // a perfectly conducting wall: J = J_r r^, the normal part only
    const double jn = Jx * nx + Jy * ny + Jz * nz;
    Jx = jn * nx;
    Jy = jn * ny;
    Jz = jn * nz;
  }
  const double Bx = w[5], By = w[6], Bz = w[7];
  const double bj = c.eta * ((By * Jz - Bz * Jy) * nx + (Bz * Jx - Bx * Jz) * ny + (Bx * Jy - By * Jx) * nz);
  double qdn;
  if (outer) {
    const double rT = qf[0] * w[3];
    qdn = 0.0;
#pragma unroll
    for (int j = 0; j < 3; ++j) qdn += (-c.kappa * rT * g[3 * 4 + j] - kr * qf[0] * c.cp * g[3 * 3 + j]) * n[j];
  } else {
    qdn = -q_bottom;
  }
  const double un = w[0] * nx + w[1] * ny + w[2] * nz;
  F[0] = 0.0;
  F[1] = tnn * nx;
  F[2] = tnn * ny;
  F[3] = tnn * nz;
  F[4] = un * tnn - qdn + bj;
  F[5] = c.eta * (Jy * nz - Jz * ny);
  F[6] = c.eta * (Jz * nx - Jx * nz);
  F[7] = c.eta * (Jx * ny - Jy * nx);
  F[8] = 0.0;
}

// gradients of element e's solution extrapolated to point (a, b) of its face F
// (sG: [24][N^3] in shared memory); the stage kernel and the face traces below
// use this same sum, so both sides of a face see the same bits
template <int N>
__device__ __forceinline__ void grad_face(const double* sG, const double* sE, int F, int a, int b, double* g) {
  constexpr int N3 = N * N * N;
  const int d = F >> 1, f = (F & 1) ? N : 0;
#pragma unroll
  for (int k = 0; k < NGRAD; ++k) {
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < N; ++i) s += sE[f * N + i] * sG[k * N3 + sol_index<N>(d, i, a, b)];
    g[k] = s;
  }
}

template <int N>
struct GradSmem {
  static constexpr int N2 = N * N, N3 = N2 * N, NF = N + 1;
  static constexpr int oQ = 0;                  // [9][N3]
  static constexpr int oW = oQ + 9 * N3;        // [8][NF][N2] (one family at a time)
  static constexpr int oG = oW + 8 * NF * N2;   // [24][N3]
  static constexpr int oE = oG + NGRAD * N3;    // [NF][N]
  static constexpr int oD = oE + NF * N;        // [N][NF]
  static constexpr size_t bytes = (oD + N * NF) * sizeof(double);
};

// BR1 gradients of one element and their face traces.
template <int N>
__global__ void __launch_bounds__(Dims<N>::BLK) grad_kernel(const StageParams P, const Ops<double> ops) {
  using GS = GradSmem<N>;
  constexpr int N2 = N * N, N3 = N2 * N, NF = N + 1, BLK = Dims<N>::BLK;
  extern __shared__ __align__(16) unsigned char smem[];
  double* sQ = reinterpret_cast<double*>(smem) + GS::oQ;
  double* sW = reinterpret_cast<double*>(smem) + GS::oW;
  double* sG = reinterpret_cast<double*>(smem) + GS::oG;
  double* sE = reinterpret_cast<double*>(smem) + GS::oE;
  double* sD = reinterpret_cast<double*>(smem) + GS::oD;
  const int tid = threadIdx.x;
  for (int i = tid; i < NF * N; i += BLK) {
    sE[i] = ops.E[i];
    sD[i] = ops.D[i];
  }
  const int64_t e = blockIdx.x;
  const double* Sfam = reinterpret_cast<const double*>(P.Sfam) + e * (9 * N2 * NF);
  const ViscCoef c = visc_coef(P);
  load_element<N, PolFP64>(P, P.q_in, e, sQ, nullptr);

  const int n = tid;
  const int i0 = n % N, j0 = (n / N) % N, k0 = n / N2;
  double acc[NGRAD];
#pragma unroll
  for (int k = 0; k < NGRAD; ++k) acc[k] = 0.0;
#pragma unroll 1
  for (int d = 0; d < 3; ++d) {
    __syncthreads();
    // w at the flux points of family d, BR1 common value at the two faces
    for (int t = tid; t < NF * N2; t += BLK) {
      const int f = t % NF, line = t / NF, a = line % N, b = line / N;
      double Qf[9], w[8];
#pragma unroll
      for (int v = 0; v < 9; ++v) {
        double s = 0.0;
#pragma unroll
        for (int i = 0; i < N; ++i) s += sE[f * N + i] * sQ[v * N3 + sol_index<N>(d, i, a, b)];
        Qf[v] = s;
      }
      prim_w(Qf, c, w);
      if (f == 0 || f == N) {
        const int side = f == N, F = 2 * d + side;
        const int64_t gidx = e * 6 + F;
        const int nb = P.nbr[gidx], mt = P.meta[gidx];
        double Q2[9], w2[8];
        if (nb >= 0) {
          const int code = meta_code(mt);
          const int u = (code & 4) ? b : a, ww = (code & 4) ? a : b;
          const int a2 = (code & 2) ? N - 1 - u : u, b2 = (code & 1) ? N - 1 - ww : ww;
          const double* Tn =
              reinterpret_cast<const double*>(P.tr_in) + ((int64_t)nb * 6 + meta_nbF(mt)) * 9 * N2 + a2 + N * b2;
#pragma unroll
          for (int v = 0; v < 9; ++v) Q2[v] = Tn[v * N2];
        } else {
          const int bc = meta_bc(mt);
          if (bc == SD_BC_FARFIELD) {
#pragma unroll
            for (int v = 0; v < 9; ++v) Q2[v] = P.farfield[v];
          } else {
            const double* Sp = Sfam + (d * 3 * N2 + line) * NF + f;
            const double Sx = Sp[0], Sy = Sp[N2 * NF], Sz = Sp[2 * N2 * NF];
            const double im = 1.0 / sqrt(Sx * Sx + Sy * Sy + Sz * Sz), sg = side ? 1.0 : -1.0;
            wall_ghost<double>(Qf, sg * Sx * im, sg * Sy * im, sg * Sz * im, bc, Q2);
          }
        }
        prim_w(Q2, c, w2);
        if (nb < 0 && P.visc_walls && meta_outer(mt)) w2[3] = 2.0 * P.T_top - w[3];  // T held on the outer wall
#pragma unroll
        for (int k = 0; k < 8; ++k) w[k] = 0.5 * (w[k] + w2[k]);
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) sW[(k * NF + f) * N2 + line] = w[k];
    }
    __syncthreads();
    // sum_f D[i][f] S^d_j w_f at this thread's solution point
    if (n < N3) {
      const int id = d == 0 ? i0 : (d == 1 ? j0 : k0);
      const int line = d == 0 ? j0 + N * k0 : (d == 1 ? i0 + N * k0 : i0 + N * j0);
      const double* Dr = sD + id * NF;
#pragma unroll 1
      for (int f = 0; f <= N; ++f) {
        const double* Sp = Sfam + (d * 3 * N2 + line) * NF + f;
        const double DS0 = Dr[f] * Sp[0], DS1 = Dr[f] * Sp[N2 * NF], DS2 = Dr[f] * Sp[2 * N2 * NF];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const double wv = sW[(k * NF + f) * N2 + line];
          acc[3 * k + 0] += DS0 * wv;
          acc[3 * k + 1] += DS1 * wv;
          acc[3 * k + 2] += DS2 * wv;
        }
      }
    }
  }
  if (n < N3) {
    const double iJ = reinterpret_cast<const double*>(P.invJ)[e * N3 + n];  // 1 / |J|
    double* Ge = P.grad_out + e * NGRAD * N3;
#pragma unroll
    for (int k = 0; k < NGRAD; ++k) {
      const double gk = acc[k] * iJ;
      sG[k * N3 + n] = gk;
      Ge[k * N3 + n] = gk;
    }
  }
  __syncthreads();
  // face traces of the gradients
  for (int t = tid; t < 6 * N2; t += BLK) {
    const int F = t / N2, pt = t - F * N2, a = pt % N, b = pt / N;
    double g[NGRAD];
    grad_face<N>(sG, sE, F, a, b, g);
    double* T = P.gtr_out + (e * 6 + F) * NGRAD * N2 + pt;
#pragma unroll
    for (int k = 0; k < NGRAD; ++k) T[k * N2] = g[k];
  }
}

template <int N>
cudaError_t launch_grad_t(const StageParams& P, const Ops<double>& ops, cudaStream_t s) {
  constexpr size_t bytes = GradSmem<N>::bytes;
  if (bytes > 48 * 1024) {
    cudaError_t err = cudaFuncSetAttribute(grad_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (err != cudaSuccess) return err;
  }
  if (P.n_e == 0) return cudaSuccess;
  grad_kernel<N><<<(unsigned)P.n_e, Dims<N>::BLK, bytes, s>>>(P, ops);
  return cudaGetLastError();
}

}  // namespace sd
