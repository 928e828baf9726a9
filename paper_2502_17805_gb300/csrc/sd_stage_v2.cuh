// sd_stage_v2.cuh -- FP32-mixed fused SD residual + SSP-RK stage, line-blocked.
//
// The SD residual of the perturbation q' = q - Q0 in FP32 (arXiv 2502.17805,
// Sec. Spectral Difference Method; the background Q0 and its FP64 residual R0
// come from sd_background_create), organised so that the 1D operators run from
// registers.  Per element (one CTA):
//   A  load     q' (FP32 perturbation), rho0, p0 at the N^3 points -> sQ
//   B  lines    G threads per line of each direction (3 N^2 lines) take the
//               line's values of one variable at a time into registers and write
//               their extrapolation to all N+1 flux points of its family -> sX
//   C  points   interior flux points: contravariant flux; face points: Rusanov
//               and BR1 against the neighbour trace; results overwrite sX in place
//   D  lines    the line threads differentiate the 10 x (N+1) fluxes and write
//               the N derivative values over its own flux slots in sX
//   E  points   R = -sum_d div_d / |J| + M + R0, FP64 RK sum, q' of the new state -> sQ
//   F  lines    face traces of the new state (the two ends of every line).
// Thread count T = 256 (N >= 6), 96 (N = 4) or 128; G = T / (3 N^2) threads
// share a line in B, D and F.  The line phases work on two variables at a time
// and phase C on two interior flux points at a time, in Blackwell's paired FP32
// arithmetic (one instruction for both lanes, each lane rounded as the scalar
// operation rounds it).
#pragma once

#include "sd_internal.h"
#include "sd_physics.cuh"
#include "sd_physics2.cuh"
#include "sd_stage.cuh"

namespace sd {

template <int N>
struct DimsV2 {
  static constexpr int N2 = N * N, N3 = N2 * N, NF = N + 1, NV = 11;
  static constexpr int NLINE = 3 * N2;
  // 256 threads from N = 6 up; below, where an element has at most 125 points,
  // 96 at N = 4 (two per line) and 128 otherwise (measured on 24,576-element
  // shells: N = 4 128 -> 96 threads 0.53 -> 0.48 ms per step, N = 5 160 threads
  // no faster than 128).  Up to G = T / (3 N^2) threads share a line in the line
  // phases, each taking every G-th variable.
  static constexpr int T = N >= 6 ? 256 : (N == 4 ? 96 : 128);
  static_assert(NLINE <= T, "one thread per line at least");
  static constexpr int G = T / NLINE;
  // shared memory in floats
  static constexpr int oQ = 0;                       // [11][N3]
  // [NF][11][3][N2]: for flux point f and value v the three directions' planes of
  // N^2 line points follow each other, so that the lines of different directions
  // that one warp handles fall into different shared-memory banks
  static constexpr int oX = oQ + NV * N3;
  static constexpr int XD = N2, XV = 3 * N2, XF = 11 * 3 * N2;  // strides of d, v, f
  static constexpr int nX = 3 * NF * NV * N2;
  static constexpr int DSTRIDE = (N3 + 3) / 4 * 4;   // element stride of the FP32 difference register
  static constexpr int oDs = (oX + nX + 3) / 4 * 4;  // [9][DSTRIDE]: D staged by a TMA bulk copy
  // With N^3 a multiple of 4 every per-element block of the FP32 geometry and
  // background planes starts on a 16-byte boundary: 1/|J|, x, y, z and the three
  // components of R0 are then staged by TMA too, [7][N3].
  static constexpr bool STAGE_G = N3 % 4 == 0;
  static constexpr int oG = oDs + 9 * DSTRIDE;
  static constexpr int nF = oG + (STAGE_G ? 7 * N3 : 0);
  static constexpr size_t bytes = ((nF * 4) + 15) / 16 * 16;
  // CTAs per SM that the shared memory admits (228 KB per SM, 1 KB reserved per
  // CTA); with the register bound below it sets __launch_bounds__.
  static constexpr int SMEM_CTAS = (int)(233472 / (bytes + 1024 + 64));
  // CTAs per SM that 64 registers per thread admit
  static constexpr int REG_CTAS = 65536 / (T * 64);
  static constexpr int MIN_CTAS = SMEM_CTAS < REG_CTAS ? SMEM_CTAS : REG_CTAS;
  static constexpr int MINB = MIN_CTAS < 1 ? 1 : MIN_CTAS;
};

// q' of variable v at a point of the new state qo (FP64), rounded as load_element
// rounds a stored state: rho and E lose their background in FP64 first.
__device__ __forceinline__ float new_qprime(int v, double qo, float qo32, float r0, float p0, double inv_gm1) {
  if (v == 0) return f64_to_f32(qo - f32_to_f64(r0));
  if (v == 4) return f64_to_f32(fma(-f32_to_f64(p0), inv_gm1, qo));
  return qo32;
}

template <int N, bool EXACT, bool INCR>
__device__ __forceinline__ void stage_body_v2(const StageParams& P, const Ops2& o2, const int64_t e,
                                              unsigned char* smem_raw) {
  using DV = DimsV2<N>;
  constexpr int N2 = DV::N2, N3 = DV::N3, NF = DV::NF, T = DV::T, NL = DV::NLINE;
  float* smem = reinterpret_cast<float*>(smem_raw);
  float* sQ = smem + DV::oQ;
  float* sX = smem + DV::oX;
  const int tid = threadIdx.x;
  const float* Sfam = reinterpret_cast<const float*>(P.Sfam) + e * (9 * N2 * NF);
  // FP32 copies of the uniform FP64 parameters, converted once per CTA by thread 0
  // (the FP64 pipe of an SM is narrow: per-thread conversions cost more than the
  // point work of some phases) and read after the first barrier
  __shared__ float sConst[9];
  if (tid == 0) {
    double dt = P.dt, chd = P.c_h;
    if (P.dyn) {
      dt = P.dyn[0];
      chd = P.dyn[1];
    }
    const float g = (float)P.gamma;
    sConst[0] = g;
    sConst[1] = g - 1.0f;
    sConst[2] = g / (g - 1.0f);
    sConst[3] = (float)chd;
    sConst[4] = (float)(P.rk_b * dt);
    sConst[5] = (float)P.rk_a;
    sConst[6] = (float)P.GM;
    sConst[7] = 2.0f * (float)P.omega;
    sConst[8] = (float)P.alpha;
  }
  const int mode = P.mode, lsr_read = P.lsr_read, lsr_write = P.lsr_write;
  constexpr bool incr = INCR;
  const int64_t n_e = P.n_e, stride = P.stride, plane = P.plane;

  // Per-element inputs copied to shared memory by TMA at kernel start: the
  // difference register D of the low-storage RK form (mbarrier dbar; read by the
  // epilogue, and by phase A in the increment form) and, with STAGE_G, 1/|J|, x
  // and R0 for the epilogue (mbarrier gbar).
  // In the increment form the stage state q^n + D starts from the stored FP32 q'
  // of q^n (P.qp_in): with STAGE_G it is copied, with rho0 and p0, straight into
  // sQ by TMA as well (mbarrier qbar).
  __shared__ __align__(8) unsigned long long dbar, gbar, qbar;
  float* sDs = smem + DV::oDs;
  float* sG = smem + DV::oG;
  const bool lsr = P.lsr_read != 0;
  constexpr bool qtma = INCR && DV::STAGE_G;
  if (tid == 0) {
    constexpr unsigned plane_bytes = DV::DSTRIDE * 4, blk = N3 * 4;
    if constexpr (qtma) {
      mbar_init(&qbar, 1);
      mbar_expect_tx(&qbar, 11 * blk);
      const int64_t qplane = P.n_e * DV::DSTRIDE;
#pragma unroll 1
      for (int v = 0; v < 9; ++v) tma_load_1d(sQ + v * N3, P.qp_in + v * qplane + e * DV::DSTRIDE, blk, &qbar);
      tma_load_1d(sQ + 9 * N3, P.bg + e * N3, blk, &qbar);
      tma_load_1d(sQ + 10 * N3, P.bg + P.n_e * N3 + e * N3, blk, &qbar);
    }
    if (lsr) {
      mbar_init(&dbar, 1);
      mbar_expect_tx(&dbar, 9 * plane_bytes);
      const float* src = P.dreg + e * DV::DSTRIDE;
      const int64_t dplane = P.n_e * DV::DSTRIDE;
#pragma unroll 1
      for (int v = 0; v < 9; ++v) tma_load_1d(sDs + v * DV::DSTRIDE, src + v * dplane, plane_bytes, &dbar);
    }
    if constexpr (DV::STAGE_G) {
      mbar_init(&gbar, 1);
      mbar_expect_tx(&gbar, 7 * blk);
      tma_load_1d(sG, reinterpret_cast<const float*>(P.invJ) + e * N3, blk, &gbar);
      tma_load_1d(sG + N3, reinterpret_cast<const float*>(P.X) + e * 3 * N3, 3 * blk, &gbar);
#pragma unroll 1
      for (int c = 0; c < 3; ++c) tma_load_1d(sG + (4 + c) * N3, P.bg + (2 + c) * P.n_e * N3 + e * N3, blk, &gbar);
    }
  }
  // L2 prefetch, at kernel start, of what the element reads from global memory
  // later: the neighbours' face traces, S^d and the background jumps (phase C)
  // and, in the last stage of the increment form, q^n (epilogue).  One thread of
  // the second warp per block, so that the TMA issue above is not delayed.
  __shared__ int sNb[6], sMt[6];
  if (tid >= 32 && tid < 32 + 17) {
    const int k = tid - 32;
    if (k < 6) {
      const int nb = __ldg(P.nbr + e * 6 + k);
      const int mt = __ldg(P.meta + e * 6 + k);
      sNb[k] = nb;
      sMt[k] = mt;
      if (nb >= 0 && P.tr_in) {
        l2_prefetch(reinterpret_cast<const float*>(P.tr_in) + ((int64_t)nb * 6 + meta_nbF(mt)) * 9 * N2,
                    9 * N2 * sizeof(float));
      }
    } else if (k == 6) {
      l2_prefetch(Sfam, 9 * N2 * NF * sizeof(float));
    } else if (k == 7) {
      if (P.bg_jump) l2_prefetch(P.bg_jump + e * 6 * 2 * N2, 6 * 2 * N2 * sizeof(float));
    } else if (INCR && mode == MODE_RK && lsr_write == 0) {
      l2_prefetch(P.q_in + (k - 8) * plane + e * stride, N3 * sizeof(double));
    }
  }

  // increment form: the stage's state is q' + D, so phase A needs D (and, with
  // qtma, the copied q')
  if (incr && (lsr || qtma)) __syncthreads();  // barriers initialised before anyone polls them

  // line role of this thread (B, D, F): G threads per line, thread g of a line
  // takes the variables g, g + G, ...
  constexpr int G = DV::G;
  const bool is_line = tid < G * NL;
  const int lg = is_line ? tid / NL : 0;
  const int lline = tid - lg * NL;
  const int ld = is_line ? lline / N2 : 0;
  const int lL = is_line ? lline % N2 : 0;
  int lbase = 0, lstride = 1;
  line_geom<N>(ld, lL, lbase, lstride);
  const bool lflip = line_flip<N>(ld, lL);

  // ---- A: load (every round's loads issued before the first conversion)
  const double inv_gm1 = P.inv_gm1;
  if constexpr (qtma) {
    // q', rho0, p0 are in sQ once qbar completes; add D
    mbar_wait_bounded(&qbar, 0u, P.err, P.wait_spins);
    if (lsr) {
      mbar_wait_bounded(&dbar, 0u, P.err, P.wait_spins);
      for (int n = tid; n < N3; n += T) {
#pragma unroll
        for (int v = 0; v < 9; ++v) sQ[v * N3 + n] += sDs[v * DV::DSTRIDE + n];
      }
    }
  } else if constexpr (INCR) {
    // stored q' (element blocks not 16-byte aligned: plain loads)
    constexpr int NRA = (N3 + T - 1) / T;
    float qv[NRA][11];
    const int64_t qplane = n_e * DV::DSTRIDE;
#pragma unroll
    for (int r = 0; r < NRA; ++r) {
      const int n = tid + r * T;
      if (n < N3) {
        const int64_t gb = e * N3 + n;
#pragma unroll
        for (int v = 0; v < 9; ++v) qv[r][v] = __ldg(P.qp_in + v * qplane + e * DV::DSTRIDE + n);
        qv[r][9] = __ldg(P.bg + gb);
        qv[r][10] = __ldg(P.bg + n_e * N3 + gb);
      }
    }
    if (lsr) mbar_wait_bounded(&dbar, 0u, P.err, P.wait_spins);
#pragma unroll
    for (int r = 0; r < NRA; ++r) {
      const int n = tid + r * T;
      if (n < N3) {
        if (lsr) {
#pragma unroll
          for (int v = 0; v < 9; ++v) qv[r][v] += sDs[v * DV::DSTRIDE + n];
        }
#pragma unroll
        for (int v = 0; v < 11; ++v) sQ[v * N3 + n] = qv[r][v];
      }
    }
  } else {
    constexpr int NRA = (N3 + T - 1) / T;
    double qv[NRA][9];
    float r0[NRA], p0[NRA];
#pragma unroll
    for (int r = 0; r < NRA; ++r) {
      const int n = tid + r * T;
      if (n < N3) {
        const int64_t g = e * stride + n, gb = e * N3 + n;
        r0[r] = __ldg(P.bg + gb);
        p0[r] = __ldg(P.bg + n_e * N3 + gb);
#pragma unroll
        for (int v = 0; v < 9; ++v) qv[r][v] = __ldg(P.q_in + v * plane + g);
      }
    }
#pragma unroll
    for (int r = 0; r < NRA; ++r) {
      const int n = tid + r * T;
      if (n < N3) {
        float qp[9];
        qp[0] = f64_to_f32(qv[r][0] - f32_to_f64(r0[r]));
#pragma unroll
        for (int v = 1; v < 9; ++v) qp[v] = f64_to_f32(qv[r][v]);
        qp[4] = f64_to_f32(fma(-f32_to_f64(p0[r]), inv_gm1, qv[r][4]));
#pragma unroll
        for (int v = 0; v < 9; ++v) sQ[v * N3 + n] = qp[v];
        sQ[9 * N3 + n] = r0[r];
        sQ[10 * N3 + n] = p0[r];
      }
    }
  }
  __syncthreads();
  const float gamma = sConst[0], gm1 = sConst[1], gg1 = sConst[2], ch = sConst[3];
  const float bdt = sConst[4], rka = sConst[5];
  const bool classic_qn = rka != 0.0f;
  const MixedConsts MC{sConst[6], sConst[7], sConst[8], P.gravity, P.coriolis, P.powell};

  // ---- B: extrapolate every line to its N+1 flux points, two variables at a time
  //      (variable pairs (0,1) ... (10,10): N values of each in the lanes of a
  //      register pair, N+1 outputs)
  if (is_line) {
    float* X = sX + ld * DV::XD + lL;
#pragma unroll 1
    for (int pr = lg; pr < 6; pr += G) {
      const int v0 = 2 * pr, v1 = v0 + 1 < 11 ? v0 + 1 : v0;
      float2 ql[N];
      load_line<N>(sQ + v0 * N3, sQ + v1 * N3, lbase, lstride, lflip, ql);
      // even-odd form: the pair (f, N-f) of outputs from the sums and differences
      // of the pairs (i, N-1-i) of inputs
      constexpr int HP = N / 2;
      float2 sv[HP], dv[HP];
#pragma unroll
      for (int i = 0; i < HP; ++i) {
        sv[i] = add2(ql[i], ql[N - 1 - i]);
        dv[i] = sub2(ql[i], ql[N - 1 - i]);
      }
#pragma unroll
      for (int f = 0; 2 * f <= N; ++f) {
        float2 a = (N & 1) ? mul2(o2.Es[f * N + HP], ql[HP]) : make_float2(0.0f, 0.0f);
        float2 b = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int i = 0; i < HP; ++i) {
          a = fma2(o2.Es[f * N + i], sv[i], a);
          b = fma2(o2.Ed[f * N + i], dv[i], b);
        }
        if (2 * f == N) {
          X[f * DV::XF + v0 * DV::XV] = a.x;
          X[f * DV::XF + v1 * DV::XV] = a.y;
        } else {
          const float2 pa = add2(a, b), ma = sub2(a, b);
          X[f * DV::XF + v0 * DV::XV] = pa.x;
          X[f * DV::XF + v1 * DV::XV] = pa.y;
          X[(N - f) * DV::XF + v0 * DV::XV] = ma.x;
          X[(N - f) * DV::XF + v1 * DV::XV] = ma.y;
        }
      }
    }
  }
  __syncthreads();

  // ---- C: fluxes at the flux points: pairs of interior points first (point r and
  //      point r + NINT/2 in the lanes of one paired evaluation), their count
  //      padded to whole warps so that no warp mixes the two kinds of work, then
  //      the element faces one point at a time
  constexpr int NINT = 3 * (N - 1) * N2, NIP = NINT / 2, NIP_W = (NIP + 31) / 32 * 32;
  static_assert(NINT % 2 == 0, "interior flux points pair up");
  const Mixed2 C2{f2(gamma), f2(gm1), f2(gg1), f2(ch), f2(0.5f)};
  for (int t = tid; t < NIP_W + 6 * N2; t += T) {
    if (t < NIP_W) {
      if (t >= NIP) continue;
      float* Xp[2];
      float2 qf[11], S[3];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int r0 = t + h * NIP;
        const int d = r0 / ((N - 1) * N2), r = r0 - d * ((N - 1) * N2);
        const int f = 1 + r / N2, L = r - (f - 1) * N2;
        Xp[h] = sX + f * DV::XF + d * DV::XD + L;
        const float* Sp = Sfam + s32_index(N, d, f, 0, L);
#pragma unroll
        for (int c = 0; c < 3; ++c) (h ? S[c].y : S[c].x) = __ldg(Sp + c * N2);
#pragma unroll
        for (int v = 0; v < 11; ++v) (h ? qf[v].y : qf[v].x) = Xp[h][v * DV::XV];
      }
      float2 Fv[9];
      flux_pert2(qf, S[0], S[1], S[2], C2, Fv);
      const float2 SB = dot3(S[0], S[1], S[2], qf[5], qf[6], qf[7]);
#pragma unroll
      for (int v = 0; v < 9; ++v) {
        Xp[0][v * DV::XV] = Fv[v].x;
        Xp[1][v * DV::XV] = Fv[v].y;
      }
      Xp[0][9 * DV::XV] = SB.x;
      Xp[1][9 * DV::XV] = SB.y;
    } else {
      const int u = t - NIP_W;
      const int F = u / N2, pt = u - F * N2, a = pt % N, b = pt / N;
      const int d = F >> 1, side = F & 1, f = side ? N : 0;
      float* X = sX + f * DV::XF + d * DV::XD + pt;
      float qo[11];
#pragma unroll
      for (int v = 0; v < 11; ++v) qo[v] = X[v * DV::XV];
      const float* Sp = Sfam + s32_index(N, d, f, 0, pt);
      const float Sx = __ldg(Sp), Sy = __ldg(Sp + N2), Sz = __ldg(Sp + 2 * N2);
      const float mag = sqrtf(Sx * Sx + Sy * Sy + Sz * Sz);
      const float im = 1.0f / mag;
      const float sg = side ? 1.0f : -1.0f;
      const float nx = sg * Sx * im, ny = sg * Sy * im, nz = sg * Sz * im;
      const int64_t gidx = e * 6 + F;
      const int nb = sNb[F];
      const int mt = sMt[F];
      float qn[9];
      float jr = 0.0f, jp = 0.0f;
      if (nb >= 0) {
        const int code = meta_code(mt);
        const int uu = (code & 4) ? b : a, w = (code & 4) ? a : b;
        const int a2 = (code & 2) ? N - 1 - uu : uu, b2 = (code & 1) ? N - 1 - w : w;
        const float* Tn = reinterpret_cast<const float*>(P.tr_in) + ((int64_t)nb * 6 + meta_nbF(mt)) * 9 * N2 + a2 + N * b2;
#pragma unroll
        for (int v = 0; v < 9; ++v) qn[v] = Tn[v * N2];
        jr = __ldg(P.bg_jump + (gidx * 2 + 0) * N2 + pt);
        jp = __ldg(P.bg_jump + (gidx * 2 + 1) * N2 + pt);
      } else {
        const int bc = meta_bc(mt);
        if (bc == SD_BC_FARFIELD) {
#pragma unroll
          for (int v = 0; v < 9; ++v) qn[v] = (float)P.farfield[v];
          qn[0] -= qo[9];
          qn[4] -= qo[10] / gm1;
        } else {
          wall_ghost<float>(qo, nx, ny, nz, bc, qn);
        }
      }
      float Fs[9];
      riemann_mixed(qo, qn, nx, ny, nz, gamma, ch, jr, jp, Fs);
      const float Bn = 0.5f * ((qo[5] + qn[5]) * nx + (qo[6] + qn[6]) * ny + (qo[7] + qn[7]) * nz);
      const float sm = sg * mag;
#pragma unroll
      for (int v = 0; v < 9; ++v) X[v * DV::XV] = sm * Fs[v];
      X[9 * DV::XV] = sm * Bn;
    }
  }
  __syncthreads();

  // ---- D: derivative of the flux polynomial along every line, written over the
  //      line's own flux slots (value i of variable v goes to slot (f = i, v)):
  //      each thread reads and writes only its own line, two variables at a time.
  if (is_line) {
    float* X = sX + ld * DV::XD + lL;
#pragma unroll 1
    for (int pr = lg; pr < 5; pr += G) {
      const int v0 = 2 * pr, v1 = v0 + 1;
      float2 fv[NF];
#pragma unroll
      for (int f = 0; f <= N; ++f) fv[f] = make_float2(X[f * DV::XF + v0 * DV::XV], X[f * DV::XF + v1 * DV::XV]);
      // even-odd form: D[N-1-i][f] = -D[i][N-f] gives the pair (i, N-1-i) from the
      // sums and differences of the flux pairs (f, N-f)
      constexpr int HF = NF / 2;
      float2 sf[HF], df[HF];
#pragma unroll
      for (int f = 0; f < HF; ++f) {
        sf[f] = add2(fv[f], fv[N - f]);
        df[f] = sub2(fv[f], fv[N - f]);
      }
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
          X[i * DV::XF + v0 * DV::XV] = r.x;
          X[i * DV::XF + v1 * DV::XV] = r.y;
        } else {
          const float2 pr_ = add2(p, r), mr = sub2(r, p);
          X[i * DV::XF + v0 * DV::XV] = pr_.x;
          X[i * DV::XF + v1 * DV::XV] = pr_.y;
          X[(N - 1 - i) * DV::XF + v0 * DV::XV] = mr.x;
          X[(N - 1 - i) * DV::XF + v1 * DV::XV] = mr.y;
        }
      }
    }
  }
  __syncthreads();

  // ---- E: residual, sources, RK sum
  // With P.lam_max (MODE_RK) the stage also returns lambda_max of its output, and
  // the q' it leaves for the traces is rounded from the stored FP64 state exactly
  // as a fresh load would round it: the traces and lambda_max equal those of a
  // separate trace pass over the output, bit for bit.
  constexpr bool exact = EXACT;
  float lam = 0.0f;  // maximum of FP32 speeds (taken in FP32, converted once when reduced)
  if (lsr && !incr) mbar_wait_bounded(&dbar, 0u, P.err, P.wait_spins);
  if (DV::STAGE_G) mbar_wait_bounded(&gbar, 0u, P.err, P.wait_spins);
  for (int n = tid; n < N3; n += T) {
    const int i0 = n % N, j0 = (n / N) % N, k0 = n / N2;
    const float* D0 = sX + i0 * DV::XF + 0 * DV::XD + (j0 + N * k0);
    const float* D1 = sX + j0 * DV::XF + 1 * DV::XD + (i0 + N * k0);
    const float* D2 = sX + k0 * DV::XF + 2 * DV::XD + (i0 + N * j0);
    // q_in of the RK sum (FP64; in the increment form only the last stage reads it),
    // all nine loads issued before the direction sums: q_out may be q_in itself, so
    // the compiler cannot move a load of the loop below past its stores, and each
    // point would wait for nine L2 round trips in turn (a thread reads its own
    // point's values before it overwrites them; 2.45 -> 2.31 ms per step on the
    // 41,472-element shell)
    double qin9[9];
    if (mode == MODE_RK && (!incr || !lsr_write)) {
#pragma unroll
      for (int v = 0; v < 9; ++v) qin9[v] = __ldg(P.q_in + v * plane + e * stride + n);
    }
    float acc[10];
#pragma unroll
    for (int v = 0; v < 10; ++v) acc[v] = D0[v * DV::XV] + D1[v * DV::XV] + D2[v * DV::XV];
    float G[7];  // 1/|J|, x, y, z, R0 (momentum components)
    if constexpr (DV::STAGE_G) {
#pragma unroll
      for (int c = 0; c < 7; ++c) G[c] = sG[c * N3 + n];
    } else {
      const int64_t gb = e * N3 + n, bp = n_e * N3;
      const float* Xe = reinterpret_cast<const float*>(P.X) + e * 3 * N3;
      G[0] = __ldg(reinterpret_cast<const float*>(P.invJ) + gb);
#pragma unroll
      for (int c = 0; c < 3; ++c) G[1 + c] = __ldg(Xe + c * N3 + n);
#pragma unroll
      for (int c = 0; c < 3; ++c) G[4 + c] = __ldg(P.bg + (2 + c) * bp + gb);
    }
    const float iJ = G[0];
    const float divB = acc[9] * iJ;
    float q[11], M[9], Rv[9];
#pragma unroll
    for (int v = 0; v < 11; ++v) q[v] = sQ[v * N3 + n];
    sources_mixed(MC, q, divB, G[1], G[2], G[3], M);
#pragma unroll
    for (int v = 0; v < 9; ++v) Rv[v] = -acc[v] * iJ + M[v];
    Rv[1] += G[4];
    Rv[2] += G[5];
    Rv[3] += G[6];
    if (P.rvis) {  // viscous fluxes: the residual the viscous kernels computed for this stage state
      const float* rv = P.rvis + e * N3 + n;
#pragma unroll
      for (int v = 0; v < 7; ++v) Rv[1 + v] += __ldg(rv + v * n_e * N3);
    }
    const int64_t g = e * stride + n;
    if (mode == MODE_RESIDUAL) {
#pragma unroll
      for (int v = 0; v < 9; ++v) P.out[v * plane + g] = f32_to_f64(Rv[v]);
    } else if (mode == MODE_DIVB) {
      P.divb[e * N3 + n] = f32_to_f64(divB);
    } else if (incr) {
      // increment form: the stage's state is q^n + D (q_in = q^n, D = 0 at stage 0);
      // t = -a D + b dt R; intermediate stages only advance D <- D + t (FP32),
      // the last writes q^n + (D + t) in FP64
      const int64_t gd = e * DV::DSTRIDE + n, dplane = n_e * DV::DSTRIDE;
      float* const wreg = P.wreg;  // five-stage method: W = w_old D + w_new (D + t) beside D
      float qe[9];
#pragma unroll
      for (int v = 0; v < 9; ++v) {
        const float Dv = lsr_read ? sDs[v * DV::DSTRIDE + n] : 0.0f;
        const float t = fmaf(-rka, Dv, bdt * Rv[v]);
        if (lsr_write) {
          P.dreg[v * dplane + gd] = Dv + t;
          if (wreg) wreg[v * dplane + gd] = fmaf(P.w_old, Dv, P.w_new * (Dv + t));
          sQ[v * N3 + n] = q[v] + t;
        } else {
          const double qo = qin9[v] + f32_to_f64(Dv + t);
          P.out[v * plane + g] = qo;
          if (exact) {
            qe[v] = f64_to_f32(qo);
            const float qpn = new_qprime(v, qo, qe[v], q[9], q[10], inv_gm1);
            sQ[v * N3 + n] = qpn;
            if (P.qp_out) P.qp_out[v * dplane + gd] = qpn;  // q' of the new state for the next step
          } else {
            sQ[v * N3 + n] = q[v] + t;
          }
        }
      }
      if (exact) lam = speed_max(lam, point_speed_mixed(qe, gamma));
    } else if (lsr_read || lsr_write) {
      // low-storage form: t = -a D + b dt R, q_out = q_in + t, D <- D + t, with D = q_in - q_n
      const int64_t gd = e * DV::DSTRIDE + n, dplane = n_e * DV::DSTRIDE;
      float qe[9];
#pragma unroll
      for (int v = 0; v < 9; ++v) {
        const double qin = qin9[v];
        const float Dv = lsr_read ? sDs[v * DV::DSTRIDE + n] : 0.0f;
        const float t = fmaf(-rka, Dv, bdt * Rv[v]);
        const double qo = qin + f32_to_f64(t);
        P.out[v * plane + g] = qo;
        if (lsr_write) P.dreg[v * dplane + gd] = (lsr_write == 1) ? t : Dv + t;
        if (exact) qe[v] = f64_to_f32(qo);
        sQ[v * N3 + n] = exact ? new_qprime(v, qo, qe[v], q[9], q[10], inv_gm1) : q[v] + t;
      }
      if (exact) lam = speed_max(lam, point_speed_mixed(qe, gamma));
    } else {
      float qe[9];
#pragma unroll
      for (int v = 0; v < 9; ++v) {
        const double qin = qin9[v];
        float t = bdt * Rv[v];
        if (classic_qn) t = fmaf(rka, f64_to_f32(__ldg(P.q_n + v * plane + g) - qin), t);
        const double qo = qin + f32_to_f64(t);
        P.out[v * plane + g] = qo;
        if (exact) qe[v] = f64_to_f32(qo);
        sQ[v * N3 + n] = exact ? new_qprime(v, qo, qe[v], q[9], q[10], inv_gm1) : q[v] + t;
      }
      if (exact) lam = speed_max(lam, point_speed_mixed(qe, gamma));
    }
  }
  if (exact && P.lam_max) speed_reduce(lam, P.lam_max, P.lam_nslot);

  // ---- F: face traces of the new state, two variables at a time (each lane the
  //      trace kernel's sum in its order)
  if (mode == MODE_RK && P.tr_out) {
    __syncthreads();
    if (is_line) {
      float* Tr = reinterpret_cast<float*>(P.tr_out) + (e * 6 + 2 * ld) * 9 * N2 + lL;
#pragma unroll 1
      for (int pr = lg; pr < 5; pr += G) {
        const int v0 = 2 * pr, v1 = v0 + 1 < 9 ? v0 + 1 : v0;
        float2 s0 = make_float2(0.0f, 0.0f), s1 = make_float2(0.0f, 0.0f);
        float2 x[N];
        load_line<N>(sQ + v0 * N3, sQ + v1 * N3, lbase, lstride, lflip, x);
#pragma unroll
        for (int i = 0; i < N; ++i) {
          s0 = fma2(o2.E0[i], x[i], s0);
          s1 = fma2(o2.EN[i], x[i], s1);
        }
        Tr[v0 * N2] = s0.x;
        Tr[9 * N2 + v0 * N2] = s1.x;
        Tr[v1 * N2] = s0.y;
        Tr[9 * N2 + v1 * N2] = s1.y;
      }
    }
  }
}

template <int N, bool EXACT, bool INCR>
__global__ void __launch_bounds__(DimsV2<N>::T, DimsV2<N>::MINB) stage_kernel_v2(const StageParams P, const Ops2 o2) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  stage_body_v2<N, EXACT, INCR>(P, o2, (int64_t)blockIdx.x, smem_raw);
}

// Packed launch over several requests (see packed_request in sd_stage.cuh); the
// packed stages always run the increment form.  The last stage runs the exact
// form (EXACT): a request whose row has tr_out, lam_max and qp_out set leaves
// the traces, lambda_max and q' of its new state for its next step; with them
// unset it gets what the plain last stage gives (the state is the same bits).
template <int N, bool EXACT>
__global__ void __launch_bounds__(DimsV2<N>::T, DimsV2<N>::MINB) stage_kernel_v2_packed(const StageParams* __restrict__ tab,
                                                                         const int64_t* __restrict__ off, int n_req,
                                                                         const Ops2 o2) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ StageParams sP;
  const int r = packed_request(off, n_req, (int64_t)blockIdx.x);
  copy_params(tab + r, &sP);
  stage_body_v2<N, EXACT, true>(sP, o2, (int64_t)blockIdx.x - __ldg(off + r), smem_raw);
}

template <int N, bool EXACT, bool INCR>
cudaError_t launch_stage_v2_e(const StageParams& P, const Ops2& o2, cudaStream_t s) {
  using DV = DimsV2<N>;
  auto kern = stage_kernel_v2<N, EXACT, INCR>;
  cudaError_t err =
      cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
  if (err != cudaSuccess) return err;
  if (DV::bytes > 48 * 1024) {
    err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DV::bytes);
    if (err != cudaSuccess) return err;
  }
  if (P.n_e == 0) return cudaSuccess;
  kern<<<(unsigned)P.n_e, DV::T, DV::bytes, s>>>(P, o2);
  return cudaGetLastError();
}

// The exact form (traces and lambda_max of the output as a fresh load of it
// gives them) and the increment form are separate instantiations, so each
// stage carries only the code it runs.
template <int N>
cudaError_t launch_stage_v2_t(const StageParams& P, const Ops2& o2, cudaStream_t s) {
  const bool exact = P.mode == MODE_RK && P.lam_max;
  if (P.incr) return exact ? launch_stage_v2_e<N, true, true>(P, o2, s) : launch_stage_v2_e<N, false, true>(P, o2, s);
  return exact ? launch_stage_v2_e<N, true, false>(P, o2, s) : launch_stage_v2_e<N, false, false>(P, o2, s);
}

// Packed launches of one order N over `blocks` elements of n_req requests: the
// trace (+lambda) kernel (kind 0), a stage (kind 1) or the last stage in the
// exact form (kind 2).
template <int N, bool EXACT>
cudaError_t launch_packed_stage(const StageParams* tab, const int64_t* off, int n_req, int64_t blocks,
                                const Ops2& o2, cudaStream_t s) {
  using DV = DimsV2<N>;
  auto kern = stage_kernel_v2_packed<N, EXACT>;
  cudaError_t err =
      cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
  if (err != cudaSuccess) return err;
  if (DV::bytes > 40 * 1024) {
    err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DV::bytes);
    if (err != cudaSuccess) return err;
  }
  kern<<<(unsigned)blocks, DV::T, DV::bytes, s>>>(tab, off, n_req, o2);
  return cudaGetLastError();
}

template <int N>
cudaError_t launch_packed_t(int kind, const StageParams* tab, const int64_t* off, int n_req, int64_t blocks,
                            const Ops<float>& ops, const Ops2& o2, cudaStream_t s) {
  if (blocks == 0) return cudaSuccess;
  if (kind == 0) {
    const size_t bytes = Smem<N, PolMixed>::trace_bytes;
    if (bytes > 40 * 1024) {
      cudaError_t err = cudaFuncSetAttribute(trace_kernel_packed<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)bytes);
      if (err != cudaSuccess) return err;
    }
    trace_kernel_packed<N><<<(unsigned)blocks, Dims<N>::BLK, bytes, s>>>(tab, off, n_req, ops);
    return cudaGetLastError();
  }
  return kind == 2 ? launch_packed_stage<N, true>(tab, off, n_req, blocks, o2, s)
                   : launch_packed_stage<N, false>(tab, off, n_req, blocks, o2, s);
}

}  // namespace sd
