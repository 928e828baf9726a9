// sd_stage_f64.cuh -- FP64 SD residual + SSP-RK stage: a face-flux kernel and a
// line-blocked element kernel.
//
// GB300 issues two FP64 FMA per SM and clock, so the FP64 path is bound by the
// number of FP64 operations, not by memory.  Two changes cut that number:
//  * the common face flux (Rusanov, Sec. SD Method) and the BR1 normal field are
//    computed once per face point, by the side that owns the face (the first of
//    the pair when faces are matched, or the element of a boundary face), in a
//    separate kernel; both elements read the result, the other side negated,
//    which also makes the two sides' face fluxes exact negatives;
//  * the element kernel applies the 1D extrapolation and derivative along
//    every line in the even-odd form (the solution and flux points are
//    symmetric about the element centre), about a fifth fewer operations.
// Per element (one CTA):
//   A  load     q at the N^3 solution points -> sQ
//   B  lines    extrapolate every line to its N-1 interior flux points -> sX
//   C  points   interior flux points: contravariant flux S^d . F(q) and S^d . B;
//               face points: the face kernel's values, signed for this side
//   D  lines    derivative of the flux polynomial along every line, over the
//               line's own slots in sX
//   E  points   R = -sum_d div_d / |J| + M, the SSP-RK combination, new state -> sQ
//   F  lines    face traces of the new state (the two ends of every line).
#pragma once

#include "sd_internal.h"
#include "sd_physics.cuh"
#include "sd_stage.cuh"
#include "sd_viscous.cuh"

namespace sd {

template <int N>
struct DimsF64 {
  static constexpr int N2 = N * N, N3 = N2 * N, NF = N + 1, NLINE = 3 * N2;
  static constexpr int T = N >= 6 ? 256 : 128;
  static_assert(NLINE <= T, "one thread per line at least");
  static constexpr int G = T / NLINE;  // threads that share a line in B, D, F
  static constexpr int oQ = 0;          // [9][N3]
  static constexpr int oX = 9 * N3;     // [3][NF][10][N2]
  static constexpr size_t bytes = (size_t)(oX + 3 * NF * 10 * N2) * sizeof(double);
};

// Common flux of one face point, computed by the face's owner: G[k][v][pt] =
// |S| F*(q_own, q_other, n) for v < 9 and |S| (B_own + B_other) / 2 . n for v = 9,
// n the owner's outward unit normal.  q_other is the neighbour's trace, the wall
// ghost state or the far-field state.  VISC: less the common viscous flux, the
// average of both sides' F_vis . n from their states and gradient records (this
// side's alone at a boundary face; the wall conditions of visc_walls at a wall).
template <int N, bool VISC>
__global__ void __launch_bounds__(256, 2) face_flux_kernel(const StageParams P, const Ops<double> ops) {
  constexpr int N2 = N * N, NF = N + 1;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= P.n_own * N2) return;
  const int64_t k = t / N2;
  const int pt = (int)(t - k * N2), a = pt % N, b = pt / N;
  const int ef = __ldg(P.own_faces + k);
  const int64_t e = ef / 6;
  const int F = ef - (int)(6 * e);
  const int d = F >> 1, side = F & 1, f = side ? N : 0;
  const double* tr = reinterpret_cast<const double*>(P.tr_in);
  double qo[9];
#pragma unroll
  for (int v = 0; v < 9; ++v) qo[v] = tr[((e * 6 + F) * 9 + v) * N2 + pt];
  const double* Sp = reinterpret_cast<const double*>(P.Sfam) + e * (9 * N2 * NF) + (d * 3 * N2 + pt) * NF + f;
  const double Sx = Sp[0], Sy = Sp[N2 * NF], Sz = Sp[2 * N2 * NF];
  const double mag = sqrt(Sx * Sx + Sy * Sy + Sz * Sz);
  const double im = 1.0 / mag;
  const double sg = side ? 1.0 : -1.0;
  const double nx = sg * Sx * im, ny = sg * Sy * im, nz = sg * Sz * im;
  const int nb = __ldg(P.nbr + e * 6 + F);
  const int mt = __ldg(P.meta + e * 6 + F);
  double qn[9];
  if (nb >= 0) {
    const int code = meta_code(mt);
    const int u = (code & 4) ? b : a, w = (code & 4) ? a : b;
    const int a2 = (code & 2) ? N - 1 - u : u, b2 = (code & 1) ? N - 1 - w : w;
    const double* T = tr + ((int64_t)nb * 6 + meta_nbF(mt)) * 9 * N2 + a2 + N * b2;
#pragma unroll
    for (int v = 0; v < 9; ++v) qn[v] = T[v * N2];
  } else {
    const int bc = meta_bc(mt);
    if (bc == SD_BC_FARFIELD) {
#pragma unroll
      for (int v = 0; v < 9; ++v) qn[v] = P.ff_own ? qo[v] : P.farfield[v];
    } else {
      wall_ghost<double>(qo, nx, ny, nz, bc, qn);
    }
  }
  const double ch = P.dyn ? P.dyn[1] : P.c_h;
  double Fs[9];
  riemann_fp64(qo, qn, nx, ny, nz, P.gamma, ch, P.central, Fs);
  if constexpr (VISC) {
    const ViscCoef c = visc_coef(P);
    const double kr = visc_kr<N>(c, ops, reinterpret_cast<const double*>(P.X), e, d, f, a, b);
    double rec[MV_REC], Fv[7];
    const double* Ro = P.gtr_in + (e * 6 + F) * MV_REC * N2 + pt;
#pragma unroll
    for (int k = 0; k < MV_REC; ++k) rec[k] = Ro[k * N2];
    if (nb < 0 && P.visc_walls) {
      wall_visc_flux_rec(qo, qn, rec, nx, ny, nz, meta_outer(mt) != 0, meta_bc(mt) == SD_BC_WALL_CONDUCTING,
                         P.q_bottom, c, kr, Fv);
    } else {
      visc_flux_rec(qo, rec, nx, ny, nz, c, kr, Fv);
      if (nb >= 0) {
        const int code = meta_code(mt);
        const int u = (code & 4) ? b : a, w = (code & 4) ? a : b;
        const int a2 = (code & 2) ? N - 1 - u : u, b2 = (code & 1) ? N - 1 - w : w;
        const double* Rn = P.gtr_in + ((int64_t)nb * 6 + meta_nbF(mt)) * MV_REC * N2 + a2 + N * b2;
#pragma unroll
        for (int k = 0; k < MV_REC; ++k) rec[k] = Rn[k * N2];
        double Fn[7];
        visc_flux_rec(qn, rec, nx, ny, nz, c, kr, Fn);
#pragma unroll
        for (int k = 0; k < 7; ++k) Fv[k] = 0.5 * (Fv[k] + Fn[k]);
      }
    }
#pragma unroll
    for (int k = 0; k < 7; ++k) Fs[1 + k] -= Fv[k];
  }
  const double Bn = 0.5 * ((qo[5] + qn[5]) * nx + (qo[6] + qn[6]) * ny + (qo[7] + qn[7]) * nz);
  double* G = reinterpret_cast<double*>(P.gface) + k * 10 * N2 + pt;
#pragma unroll
  for (int v = 0; v < 9; ++v) G[v * N2] = mag * Fs[v];
  G[9 * N2] = mag * Bn;
}

template <int N>
__global__ void __launch_bounds__(DimsF64<N>::T) stage_kernel_f64(const StageParams P, const Ops<double> ops) {
  using DV = DimsF64<N>;
  constexpr int N2 = DV::N2, N3 = DV::N3, NF = DV::NF, T = DV::T, NL = DV::NLINE, G = DV::G;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sQ = reinterpret_cast<double*>(smem_raw) + DV::oQ;
  double* sX = reinterpret_cast<double*>(smem_raw) + DV::oX;
  const int tid = threadIdx.x;
  const int64_t e = blockIdx.x;
  const int64_t stride = P.stride, plane = P.plane;
  const double* Sfam = reinterpret_cast<const double*>(P.Sfam) + e * (9 * N2 * NF);

  // line role (B, D, F): G threads per line, thread g of a line takes the variables g, g + G, ...
  const bool is_line = tid < G * NL;
  const int lg = is_line ? tid / NL : 0;
  const int lline = tid - lg * NL;
  const int ld = is_line ? lline / N2 : 0;
  const int lL = is_line ? lline % N2 : 0;
  int lbase = 0, lstride = 1;
  line_geom<N>(ld, lL, lbase, lstride);

  // ---- A: load
  for (int n = tid; n < N3; n += T) {
#pragma unroll
    for (int v = 0; v < 9; ++v) sQ[v * N3 + n] = __ldg(P.q_in + v * plane + e * stride + n);
  }
  __syncthreads();

  // ---- B: extrapolate every line to its interior flux points 1..N-1 (even-odd form)
  if (is_line) {
    double* X = sX + (ld * NF * 10) * N2 + lL;
#pragma unroll 1
    for (int v = lg; v < 9; v += G) {
      double ql[N];
#pragma unroll
      for (int i = 0; i < N; ++i) ql[i] = sQ[v * N3 + lbase + i * lstride];
      constexpr int HP = N / 2;
      double sv[HP], dv[HP];
#pragma unroll
      for (int i = 0; i < HP; ++i) {
        sv[i] = ql[i] + ql[N - 1 - i];
        dv[i] = ql[i] - ql[N - 1 - i];
      }
#pragma unroll
      for (int f = 1; 2 * f <= N; ++f) {
        double a = (N & 1) ? ops.Es[f * N + HP] * ql[HP] : 0.0;
        double b = 0.0;
#pragma unroll
        for (int i = 0; i < HP; ++i) {
          a = fma(ops.Es[f * N + i], sv[i], a);
          b = fma(ops.Ed[f * N + i], dv[i], b);
        }
        if (2 * f == N) {
          X[(f * 10 + v) * N2] = a;
        } else {
          X[(f * 10 + v) * N2] = a + b;
          X[((N - f) * 10 + v) * N2] = a - b;
        }
      }
    }
  }
  __syncthreads();

  // ---- C: interior fluxes (in place) and the face kernel's values at the face slots
  const double gm1 = P.gamma - 1.0;
  const double ch = P.dyn ? P.dyn[1] : P.c_h;
  constexpr int NINT = 3 * (N - 1) * N2;
  for (int t = tid; t < NINT + 6 * N2; t += T) {
    if (t < NINT) {
      const int d = t / ((N - 1) * N2), r = t - d * ((N - 1) * N2);
      const int f = 1 + r / N2, L = r - (f - 1) * N2;
      double* X = sX + ((d * NF + f) * 10) * N2 + L;
      double qf[9];
#pragma unroll
      for (int v = 0; v < 9; ++v) qf[v] = X[v * N2];
      const double* Sp = Sfam + (d * 3 * N2 + L) * NF + f;
      const double Sx = __ldg(Sp), Sy = __ldg(Sp + N2 * NF), Sz = __ldg(Sp + 2 * N2 * NF);
      double Fv[9];
      flux_full<double>(qf, Sx, Sy, Sz, gm1, ch, Fv);
#pragma unroll
      for (int v = 0; v < 9; ++v) X[v * N2] = Fv[v];
      X[9 * N2] = Sx * qf[5] + Sy * qf[6] + Sz * qf[7];
    } else {
      const int u = t - NINT;
      const int F = u / N2, pt = u - F * N2, a = pt % N, b = pt / N;
      const int d = F >> 1, side = F & 1, f = side ? N : 0;
      const int mt = __ldg(P.meta + e * 6 + F);
      const int nb = __ldg(P.nbr + e * 6 + F);
      const int k = __ldg(P.face_k + e * 6 + F);
      double sgn = side ? 1.0 : -1.0;
      int idx = pt;
      if (nb >= 0 && !meta_owner(mt)) {
        // the neighbour owns the face: its value along its own outward normal, negated
        const int code = meta_code(mt);
        const int uu = (code & 4) ? b : a, w = (code & 4) ? a : b;
        const int a2 = (code & 2) ? N - 1 - uu : uu, b2 = (code & 1) ? N - 1 - w : w;
        idx = a2 + N * b2;
        sgn = -sgn;
      }
      const double* Gk = reinterpret_cast<const double*>(P.gface) + (int64_t)k * 10 * N2 + idx;
      double* X = sX + ((d * NF + f) * 10) * N2 + pt;
#pragma unroll
      for (int v = 0; v < 10; ++v) X[v * N2] = sgn * __ldg(Gk + v * N2);
    }
  }
  __syncthreads();

  // ---- D: derivative along every line (even-odd form), value i of variable v to slot (i, v)
  if (is_line) {
    double* X = sX + (ld * NF * 10) * N2 + lL;
#pragma unroll 1
    for (int v = lg; v < 10; v += G) {
      double fv[NF];
#pragma unroll
      for (int f = 0; f <= N; ++f) fv[f] = X[(f * 10 + v) * N2];
      constexpr int HF = NF / 2;
      double sf[HF], df[HF];
#pragma unroll
      for (int f = 0; f < HF; ++f) {
        sf[f] = fv[f] + fv[N - f];
        df[f] = fv[f] - fv[N - f];
      }
#pragma unroll
      for (int i = 0; 2 * i <= N - 1; ++i) {
        double p = (NF & 1) ? ops.Ds[i * NF + HF] * fv[HF] : 0.0;
        double r = 0.0;
#pragma unroll
        for (int f = 0; f < HF; ++f) {
          p = fma(ops.Ds[i * NF + f], sf[f], p);
          r = fma(ops.Dd[i * NF + f], df[f], r);
        }
        if (2 * i == N - 1) {
          X[(i * 10 + v) * N2] = r;
        } else {
          X[(i * 10 + v) * N2] = p + r;
          X[((N - 1 - i) * 10 + v) * N2] = r - p;
        }
      }
    }
  }
  __syncthreads();

  // ---- E: residual, sources, RK combination q_out = a q_n + b (q_in + dt R)
  const double dt = P.dyn ? P.dyn[0] : P.dt;
  double lam = 0.0;  // lambda_max of the new state (MODE_RK with P.lam_max)
  for (int n = tid; n < N3; n += T) {
    const int i0 = n % N, j0 = (n / N) % N, k0 = n / N2;
    const double* D0 = sX + ((0 * NF + i0) * 10) * N2 + (j0 + N * k0);
    const double* D1 = sX + ((1 * NF + j0) * 10) * N2 + (i0 + N * k0);
    const double* D2 = sX + ((2 * NF + k0) * 10) * N2 + (i0 + N * j0);
    double acc[10];
#pragma unroll
    for (int v = 0; v < 10; ++v) acc[v] = (D0[v * N2] + D1[v * N2]) + D2[v * N2];
    if (P.rvis64) {  // the viscous fluxes' divergence over the interior flux points (the faces' is in D)
      const double* Rv = P.rvis64 + e * 7 * N3 + n;
#pragma unroll
      for (int k = 0; k < 7; ++k) acc[1 + k] -= __ldg(Rv + k * N3);
    }
    const double iJ = __ldg(reinterpret_cast<const double*>(P.invJ) + e * N3 + n);
    const double* Xe = reinterpret_cast<const double*>(P.X) + e * 3 * N3;
    const double divB = acc[9] * iJ;
    const int64_t g = e * stride + n;
    double q[9], M[9], Rv[9];
#pragma unroll
    for (int v = 0; v < 9; ++v) q[v] = sQ[v * N3 + n];
    sources_fp64(P, q, divB, __ldg(Xe + n), __ldg(Xe + N3 + n), __ldg(Xe + 2 * N3 + n), M);
#pragma unroll
    for (int v = 0; v < 9; ++v) Rv[v] = -acc[v] * iJ + M[v];
    if (P.mode == MODE_RESIDUAL) {
#pragma unroll
      for (int v = 0; v < 9; ++v) P.out[v * plane + g] = Rv[v];
    } else if (P.mode == MODE_DIVB) {
      P.divb[e * N3 + n] = divB;
    } else {
      double qout[9];
      if (P.rk_a != 0.0) {
#pragma unroll
        for (int v = 0; v < 9; ++v) qout[v] = P.rk_a * __ldg(P.q_n + v * plane + g) + P.rk_b * (q[v] + dt * Rv[v]);
      } else {
#pragma unroll
        for (int v = 0; v < 9; ++v) qout[v] = P.rk_b * (q[v] + dt * Rv[v]);
      }
#pragma unroll
      for (int v = 0; v < 9; ++v) P.out[v * plane + g] = qout[v];
      if (P.lam_max) lam = speed_max(lam, point_speed_fp64(qout, P.gamma));
      if (P.tr_out) {
#pragma unroll
        for (int v = 0; v < 9; ++v) sQ[v * N3 + n] = qout[v];  // each thread rewrites only its own points
      }
    }
  }
  if (P.mode == MODE_RK && P.lam_max) speed_reduce(lam, P.lam_max, P.lam_nslot);

  // ---- F: face traces of the new state, in the order of the trace kernel's sums
  if (P.mode == MODE_RK && P.tr_out) {
    __syncthreads();
    if (is_line) {
      double* Tr = reinterpret_cast<double*>(P.tr_out) + (e * 6 + 2 * ld) * 9 * N2 + lL;
#pragma unroll 1
      for (int v = lg; v < 9; v += G) {
        double s0 = 0.0, s1 = 0.0;
#pragma unroll
        for (int i = 0; i < N; ++i) {
          const double x = sQ[v * N3 + lbase + i * lstride];
          s0 = fma(ops.E[i], x, s0);
          s1 = fma(ops.E[N * N + i], x, s1);
        }
        Tr[v * N2] = s0;
        Tr[9 * N2 + v * N2] = s1;
      }
    }
  }
}

// The face-flux kernel (with the common viscous flux when P.visc and the viscous
// kernel has run: P.gtr_in set), then the element kernel.
template <int N>
cudaError_t launch_stage_f64_t(const StageParams& P, const Ops<double>& ops, cudaStream_t s) {
  using DV = DimsF64<N>;
  if (P.n_e == 0) return cudaSuccess;
  const int64_t pts = P.n_own * (int64_t)N * N;
  if (pts > 0) {
    const unsigned blocks = (unsigned)((pts + 255) / 256);
    if (P.visc && P.gtr_in)
      face_flux_kernel<N, true><<<blocks, 256, 0, s>>>(P, ops);
    else
      face_flux_kernel<N, false><<<blocks, 256, 0, s>>>(P, ops);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
  }
  auto kern = stage_kernel_f64<N>;
  if (DV::bytes > 48 * 1024) {
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DV::bytes);
    if (err != cudaSuccess) return err;
  }
  kern<<<(unsigned)P.n_e, DV::T, DV::bytes, s>>>(P, ops);
  return cudaGetLastError();
}

}  // namespace sd
