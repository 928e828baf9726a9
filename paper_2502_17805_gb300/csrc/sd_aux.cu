// sd_aux.cu -- geometry, initial state, diagnostics, background and step-control
// kernels of the SD MHD+GLM library.
#include <algorithm>
#include <limits.h>
#include <math.h>

#include "sd_internal.h"

namespace sd {

cudaError_t launch_stage_fp64(const sd_mesh* m, const StageParams& P, bool traces_only, cudaStream_t s);
cudaError_t launch_stage_mixed(const sd_mesh* m, const StageParams& P, bool traces_only, cudaStream_t s);

cudaError_t launch_stage(const sd_mesh* m, int prec, const StageParams& P, cudaStream_t s) {
  return prec == SD_FP64 ? launch_stage_fp64(m, P, false, s) : launch_stage_mixed(m, P, false, s);
}
cudaError_t launch_traces(const sd_mesh* m, int prec, const StageParams& P, cudaStream_t s) {
  return prec == SD_FP64 ? launch_stage_fp64(m, P, true, s) : launch_stage_mixed(m, P, true, s);
}

// ---------------------------------------------------------------------------
// Geometry (Sec. SD Method): transfinite map from the 12 element edges
// (constant-radius edges are great-circle arcs in the shell), sampled at
// (p+1)^3 Chebyshev-Lobatto nodes; the tensor Lagrange interpolant of those
// samples is the element map.  S^xi = x_eta x x_zeta, S^eta = x_zeta x x_xi,
// S^zeta = x_xi x x_eta at the flux points of each family; |J| and x at the
// solution points.
// ---------------------------------------------------------------------------

__device__ void edge_point_d(const double* A, const double* B, double t, int geom, double* out) {
  if (geom == 0) {
    for (int d = 0; d < 3; ++d) out[d] = A[d] + t * (B[d] - A[d]);
    return;
  }
  const double ra = sqrt(A[0] * A[0] + A[1] * A[1] + A[2] * A[2]);
  const double rb = sqrt(B[0] * B[0] + B[1] * B[1] + B[2] * B[2]);
  double ua[3], ub[3];
  for (int d = 0; d < 3; ++d) {
    ua[d] = A[d] / ra;
    ub[d] = B[d] / rb;
  }
  const double cx = ua[1] * ub[2] - ua[2] * ub[1], cy = ua[2] * ub[0] - ua[0] * ub[2], cz = ua[0] * ub[1] - ua[1] * ub[0];
  const double ang = atan2(sqrt(cx * cx + cy * cy + cz * cz), ua[0] * ub[0] + ua[1] * ub[1] + ua[2] * ub[2]);
  const double r = ra + t * (rb - ra);
  double dir[3];
  if (ang < 1e-12) {
    double nn = 0.0;
    for (int d = 0; d < 3; ++d) {
      dir[d] = (1.0 - t) * ua[d] + t * ub[d];
      nn += dir[d] * dir[d];
    }
    nn = sqrt(nn);
    for (int d = 0; d < 3; ++d) dir[d] /= nn;
  } else {
    const double s = sin(ang);
    const double wa = sin((1.0 - t) * ang) / s, wb = sin(t * ang) / s;
    for (int d = 0; d < 3; ++d) dir[d] = wa * ua[d] + wb * ub[d];
  }
  for (int d = 0; d < 3; ++d) out[d] = r * dir[d];
}

// edge-based blend: bilinear projectors of the 12 edges minus twice the trilinear corner projector
__device__ void tfi_d(const double* V, int geom, double u, double v, double w, double* X) {
  const double bu[2] = {1.0 - u, u}, bv[2] = {1.0 - v, v}, bw[2] = {1.0 - w, w};
  double P[3];
  X[0] = X[1] = X[2] = 0.0;
  for (int j = 0; j < 2; ++j)
    for (int k = 0; k < 2; ++k) {
      edge_point_d(V + 3 * (2 * j + 4 * k), V + 3 * (1 + 2 * j + 4 * k), u, geom, P);
      for (int d = 0; d < 3; ++d) X[d] += bv[j] * bw[k] * P[d];
    }
  for (int i = 0; i < 2; ++i)
    for (int k = 0; k < 2; ++k) {
      edge_point_d(V + 3 * (i + 4 * k), V + 3 * (i + 2 + 4 * k), v, geom, P);
      for (int d = 0; d < 3; ++d) X[d] += bu[i] * bw[k] * P[d];
    }
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      edge_point_d(V + 3 * (i + 2 * j), V + 3 * (i + 2 * j + 4), w, geom, P);
      for (int d = 0; d < 3; ++d) X[d] += bu[i] * bv[j] * P[d];
    }
  for (int c = 0; c < 8; ++c) {
    const double wc = bu[c & 1] * bv[(c >> 1) & 1] * bw[(c >> 2) & 1];
    for (int d = 0; d < 3; ++d) X[d] -= 2.0 * wc * V[3 * c + d];
  }
}

// The 1D Lagrange bases of the map's p+1 nodes y (Chebyshev-Lobatto), tabulated
// on the host: values A and derivatives B at the solution points (s) and the
// flux points (f), row [point][node].
struct GeoTab {
  double y[kMaxGeoP1];
  double As[kMaxN * kMaxGeoP1], Bs[kMaxN * kMaxGeoP1];
  double Af[(kMaxN + 1) * kMaxGeoP1], Bf[(kMaxN + 1) * kMaxGeoP1];
};

// One tensor contraction of the map nodes, block-wide, its first two passes:
//   out[c][k][j][i] = sum_{a,b,g} P[i][a] Q[j][b] R[k][g] X[c][g][b][a]
// (c the coordinate; P, Q, R one 1D operator per direction, rows of p1 values).
// Pass 1 T1[c][g][b][i] = sum_a P[i][a] X[c][g][b][a]; pass 2 T2[c][g][j][i] =
// sum_b Q[j][b] T1[c][g][b][i].  The third pass (over g) is taken point by point
// by geo_pass3 where the contraction is used.
__device__ void geo_pass1(const double* X, const double* P, int ni, int p1, double* T1) {
  const int n = 3 * p1 * p1 * ni;
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    const int i = t % ni, r = t / ni;  // r = (c p1 + g) p1 + b
    const double* x = X + r * p1;
    const double* w = P + i * p1;
    double s = 0.0;
    for (int a = 0; a < p1; ++a) s += w[a] * x[a];
    T1[t] = s;
  }
}

__device__ void geo_pass2(const double* T1, const double* Q, int ni, int nj, int p1, double* T2) {
  const int n = 3 * p1 * nj * ni;
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    const int i = t % ni, j = (t / ni) % nj, cg = t / (ni * nj);  // cg = c p1 + g
    const double* w = Q + j * p1;
    const double* x = T1 + cg * p1 * ni + i;
    double s = 0.0;
    for (int b = 0; b < p1; ++b) s += w[b] * x[b * ni];
    T2[t] = s;
  }
}

// the three coordinates of a contraction at point (i, j, k) from its T2
__device__ __forceinline__ void geo_pass3(const double* T2, const double* R, int ni, int nj, int p1, int i, int j,
                                          int k, double* out) {
  const double* w = R + k * p1;
  for (int c = 0; c < 3; ++c) {
    const double* x = T2 + (c * p1 * nj + j) * ni + i;
    double s = 0.0;
    for (int g = 0; g < p1; ++g) s += w[g] * x[g * nj * ni];
    out[c] = s;
  }
}

// Shared memory of geometry_kernel, in doubles: the map nodes [3][p1^3], then
// four (T1, T2) pairs of contraction buffers.
__host__ __device__ inline int geo_t1_size(int N, int p1) { return 3 * p1 * p1 * (N + 1); }
__host__ __device__ inline int geo_t2_size(int N, int p1) { return 3 * p1 * (N + 1) * (N + 1); }
__host__ __device__ inline int geo_smem_doubles(int N, int p1) {
  return 24 + 3 * p1 * p1 * p1 + 4 * (geo_t1_size(N, p1) + geo_t2_size(N, p1));
}

// Sum-factorised geometry of one element per CTA: the map nodes from the
// transfinite map, then each derivative or value of the degree-p map at a
// point set as three 1D contractions.  S^d = x_(d+1) x x_(d+2) at the flux points
// of family d (flux points along d, solution points along the other two);
// |J| = x_xi . (x_eta x x_zeta) and x at the solution points.
__global__ void geometry_kernel(int N, int p, int geom, const double* __restrict__ corners, const GeoTab tab,
                                double* Sfam64, double* invJ64, double* X64, float* Sfam32, float* invJ32, float* X32,
                                int* flag) {
  extern __shared__ double gsm[];
  const int p1 = p + 1, N2 = N * N, N3 = N2 * N, NF = N + 1;
  double* sV = gsm;
  double* sX = sV + 24;  // [c][g][b][a]
  double* T1 = sX + 3 * p1 * p1 * p1;
  const int t1 = geo_t1_size(N, p1), t2 = geo_t2_size(N, p1);
  double* T2 = T1 + 4 * t1;
  const int64_t e = blockIdx.x;
  for (int i = threadIdx.x; i < 24; i += blockDim.x) sV[i] = corners[e * 24 + i];
  __syncthreads();
  for (int t = threadIdx.x; t < p1 * p1 * p1; t += blockDim.x) {
    const int a = t % p1, b = (t / p1) % p1, g = t / (p1 * p1);
    double X[3];
    tfi_d(sV, geom, tab.y[a], tab.y[b], tab.y[g], X);
    for (int c = 0; c < 3; ++c) sX[c * p1 * p1 * p1 + t] = X[c];
  }
  __syncthreads();
  // family d: x_(d+1) and x_(d+2) at its points; operator per direction: the
  // flux-point value along d, the solution-point derivative along the
  // differentiated direction, the solution-point value along the third
  for (int d = 0; d < 3; ++d) {
    const int d1 = (d + 1) % 3, d2 = (d + 2) % 3;
    const double* op[2][3];
    int n[3];
    for (int q = 0; q < 3; ++q) n[q] = q == d ? NF : N;
    for (int h = 0; h < 2; ++h) {
      const int dd = h == 0 ? d1 : d2;  // the direction differentiated
      for (int q = 0; q < 3; ++q) op[h][q] = q == d ? tab.Af : (q == dd ? tab.Bs : tab.As);
    }
    for (int h = 0; h < 2; ++h) geo_pass1(sX, op[h][0], n[0], p1, T1 + h * t1);
    __syncthreads();
    for (int h = 0; h < 2; ++h) geo_pass2(T1 + h * t1, op[h][1], n[0], n[1], p1, T2 + h * t2);
    __syncthreads();
    for (int t = threadIdx.x; t < NF * N2; t += blockDim.x) {
      const int f = t % NF, line = t / NF, la = line % N, lb = line / N;
      int ijk[3];
      ijk[d] = f;
      ijk[d == 0 ? 1 : 0] = la;
      ijk[d == 2 ? 1 : 2] = lb;
      double xa[3], xb[3];  // x_(d+1), x_(d+2)
      geo_pass3(T2, op[0][2], n[0], n[1], p1, ijk[0], ijk[1], ijk[2], xa);
      geo_pass3(T2 + t2, op[1][2], n[0], n[1], p1, ijk[0], ijk[1], ijk[2], xb);
      const double S[3] = {xa[1] * xb[2] - xa[2] * xb[1], xa[2] * xb[0] - xa[0] * xb[2], xa[0] * xb[1] - xa[1] * xb[0]};
      for (int c = 0; c < 3; ++c) {
        const int64_t idx = (((e * 3 + d) * 3 + c) * N2 + line) * NF + f;
        Sfam64[idx] = S[c];
        Sfam32[e * 9 * N2 * NF + s32_index(N, d, f, c, line)] = (float)S[c];
      }
    }
    __syncthreads();
  }
  // solution points: x_xi, x_eta, x_zeta and x
  {
    for (int h = 0; h < 4; ++h) geo_pass1(sX, h == 0 ? tab.Bs : tab.As, N, p1, T1 + h * t1);
    __syncthreads();
    for (int h = 0; h < 4; ++h) geo_pass2(T1 + h * t1, h == 1 ? tab.Bs : tab.As, N, N, p1, T2 + h * t2);
    __syncthreads();
    for (int t = threadIdx.x; t < N3; t += blockDim.x) {
      const int i = t % N, j = (t / N) % N, k = t / N2;
      double J9[9], X[3];
      for (int h = 0; h < 3; ++h) geo_pass3(T2 + h * t2, h == 2 ? tab.Bs : tab.As, N, N, p1, i, j, k, J9 + 3 * h);
      geo_pass3(T2 + 3 * t2, tab.As, N, N, p1, i, j, k, X);
      const double* xa = J9;
      const double* xb = J9 + 3;
      const double* xc = J9 + 6;
      const double det = xa[0] * (xb[1] * xc[2] - xb[2] * xc[1]) + xa[1] * (xb[2] * xc[0] - xb[0] * xc[2]) +
                         xa[2] * (xb[0] * xc[1] - xb[1] * xc[0]);
      if (!(det > 0.0)) atomicExch(flag, 1);
      invJ64[e * N3 + t] = 1.0 / det;
      invJ32[e * N3 + t] = (float)(1.0 / det);
      for (int c = 0; c < 3; ++c) {
        X64[(e * 3 + c) * N3 + t] = X[c];
        X32[(e * 3 + c) * N3 + t] = (float)X[c];
      }
    }
  }
}

// The side of an interior face that does not own it takes the owner's metric at
// the coincident point, negated to its own orientation, so the two sides use
// exactly opposite normals and equal areas.
__global__ void canonical_faces_kernel(int N, int64_t n_e, const int* __restrict__ nbr, const int* __restrict__ meta,
                                       double* Sfam64, float* Sfam32) {
  const int N2 = N * N, NF = N + 1;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_e * 6 * N2) return;
  const int64_t e = t / (6 * N2);
  const int F = (int)((t / N2) % 6), pt = (int)(t % N2), a = pt % N, b = pt / N;
  const int mt = meta[e * 6 + F];
  const int nb = nbr[e * 6 + F];
  if (nb < 0 || meta_owner(mt)) return;
  const int code = meta_code(mt), nbF = meta_nbF(mt);
  const int u = (code & 4) ? b : a, w = (code & 4) ? a : b;
  const int a2 = (code & 2) ? N - 1 - u : u, b2 = (code & 1) ? N - 1 - w : w;
  const int d = F >> 1, f = (F & 1) ? N : 0, d2 = nbF >> 1, f2 = (nbF & 1) ? N : 0;
  const double sgn = ((F & 1) ? 1.0 : -1.0) * ((nbF & 1) ? 1.0 : -1.0);
  for (int c = 0; c < 3; ++c) {
    const double Sn = Sfam64[((((int64_t)nb * 3 + d2) * 3 + c) * N2 + a2 + N * b2) * NF + f2];
    const int64_t idx = (((e * 3 + d) * 3 + c) * N2 + pt) * NF + f;
    Sfam64[idx] = -sgn * Sn;
    Sfam32[e * 9 * N2 * NF + s32_index(N, d, f, c, pt)] = (float)(-sgn * Sn);
  }
}

// Lagrange basis l_a over nodes y (p1 of them) and its derivative, at t
static void host_lagrange(const double* y, int p1, double t, double* L, double* dL) {
  for (int a = 0; a < p1; ++a) {
    double v = 1.0, dv = 0.0;
    for (int m = 0; m < p1; ++m) {
      if (m == a) continue;
      double prod = 1.0 / (y[a] - y[m]);
      for (int q = 0; q < p1; ++q)
        if (q != a && q != m) prod *= (t - y[q]) / (y[a] - y[q]);
      dv += prod;
      v *= (t - y[m]) / (y[a] - y[m]);
    }
    L[a] = v;
    dL[a] = dv;
  }
}

cudaError_t launch_geometry(sd_mesh* m, const double* d_corners, int* d_flag, cudaStream_t s) {
  if (m->n_e == 0) return cudaSuccess;
  const int N = m->N, p = m->p, p1 = p + 1;
  if (p1 > kMaxGeoP1) return cudaErrorInvalidValue;
  GeoTab tab;
  for (int a = 0; a < p1; ++a) tab.y[a] = 0.5 * (1.0 - cos(M_PI * a / p));
  for (int i = 0; i < N; ++i) host_lagrange(tab.y, p1, m->ops64.xs[i], tab.As + i * p1, tab.Bs + i * p1);
  for (int f = 0; f <= N; ++f) host_lagrange(tab.y, p1, m->ops64.xf[f], tab.Af + f * p1, tab.Bf + f * p1);
  const size_t bytes = (size_t)geo_smem_doubles(N, p1) * sizeof(double);
  if (bytes > 48 * 1024) {
    cudaError_t err = cudaFuncSetAttribute(geometry_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (err != cudaSuccess) return err;
  }
  geometry_kernel<<<(unsigned)m->n_e, 128, bytes, s>>>(N, p, m->geom, d_corners, tab, m->Sfam64, m->invJ64, m->X64,
                                                      m->Sfam32, m->invJ32, m->X32, d_flag);
  return cudaGetLastError();
}

cudaError_t launch_canonical_faces(sd_mesh* m, cudaStream_t s) {
  const int64_t tot = m->n_e * 6 * m->N * m->N;
  if (tot == 0) return cudaSuccess;
  canonical_faces_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(m->N, m->n_e, m->nbr, m->meta, m->Sfam64,
                                                                       m->Sfam32);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Initial states (Sec. Initial Conditions)
// ---------------------------------------------------------------------------

// SplitMix64 (Steele, Lea and Flood; Vigna's reference generator): the
// (index+1)-th output of the generator whose state starts at seed.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long seed, unsigned long long index) {
  unsigned long long z = seed + (index + 1ULL) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

__device__ void cons_from_prim(double rho, const double* u, double p, const double* B, double psi, double gamma,
                               double* Q) {
  Q[0] = rho;
  for (int d = 0; d < 3; ++d) Q[1 + d] = rho * u[d];
  Q[4] = p / (gamma - 1.0) + 0.5 * rho * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]) +
         0.5 * (B[0] * B[0] + B[1] * B[1] + B[2] * B[2]) + 0.5 * psi * psi;
  for (int d = 0; d < 3; ++d) Q[5 + d] = B[d];
  Q[8] = psi;
}

struct InitArgs {
  int kind;
  int N;
  int64_t n_e, stride, plane;
  double P[16];
  unsigned long long seed;
  double gamma, GM, B0dip;
  ProfileTable tab;
};

// rho and p of the flux-balanced profile at radius r: cubic Hermite interpolation of rho and S
// between the table's nodes, p = (rho exp(S / C_p))^gamma
__device__ __forceinline__ void profile_at(const ProfileTable& T, double gamma, double r, double& rho, double& p) {
  const double u = (r - T.rb) / T.h;
  int k = (int)floor(u);
  k = k < 0 ? 0 : (k >= T.n ? T.n - 1 : k);
  const double t = u - k, h = T.h;
  const int n1 = T.n + 1;
  const double* R = T.tab;
  const double a = (1 + 2 * t) * (1 - t) * (1 - t), b = t * (1 - t) * (1 - t), c = t * t * (3 - 2 * t),
               d = t * t * (t - 1);
  rho = a * R[k] + b * h * R[2 * n1 + k] + c * R[k + 1] + d * h * R[2 * n1 + k + 1];
  const double S = a * R[n1 + k] + b * h * R[3 * n1 + k] + c * R[n1 + k + 1] + d * h * R[3 * n1 + k + 1];
  p = pow(rho * exp(S / T.Cp), gamma);
}

__global__ void state_init_kernel(const InitArgs A, const double* __restrict__ X64, double* q, double* qbg) {
  const int N3 = A.N * A.N * A.N;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= A.n_e * A.stride) return;
  const int64_t e = t / A.stride;
  const int n = (int)(t % A.stride);
  double Q[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, Qb[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  if (n < N3) {
    const double x[3] = {X64[(e * 3 + 0) * N3 + n], X64[(e * 3 + 1) * N3 + n], X64[(e * 3 + 2) * N3 + n]};
    const double zero[3] = {0.0, 0.0, 0.0};
    const double* P = A.P;
    if (A.kind == SD_INIT_UNIFORM) {
      const double u[3] = {P[1], P[2], P[3]}, B[3] = {P[5], P[6], P[7]};
      cons_from_prim(P[0], u, P[4], B, P[8], A.gamma, Q);
    } else if (A.kind == SD_INIT_ALFVEN) {
      const double rho = P[0], p = P[1], B0 = P[2], amp = P[3], tt = P[7];
      const double k[3] = {P[4], P[5], P[6]};
      const double kn = sqrt(k[0] * k[0] + k[1] * k[1] + k[2] * k[2]);
      const double kh[3] = {k[0] / kn, k[1] / kn, k[2] / kn};
      // e1 = unit(khat x z) (or unit(x x khat) when k is along z); e2 = khat x e1
      double e1[3] = {kh[1], -kh[0], 0.0};
      double n1 = sqrt(e1[0] * e1[0] + e1[1] * e1[1]);
      if (n1 < 1e-8) {
        e1[0] = 0.0;
        e1[1] = -kh[2];
        e1[2] = kh[1];
        n1 = sqrt(e1[1] * e1[1] + e1[2] * e1[2]);
      }
      for (int d = 0; d < 3; ++d) e1[d] /= n1;
      const double e2[3] = {kh[1] * e1[2] - kh[2] * e1[1], kh[2] * e1[0] - kh[0] * e1[2], kh[0] * e1[1] - kh[1] * e1[0]};
      const double om = kn * B0 / sqrt(rho);
      const double ph = k[0] * x[0] + k[1] * x[1] + k[2] * x[2] - om * tt;
      const double cp = cos(ph), sp = sin(ph);
      double B[3], u[3];
      for (int d = 0; d < 3; ++d) {
        const double dB = amp * (cp * e1[d] + sp * e2[d]);
        B[d] = B0 * kh[d] + dB;
        u[d] = -dB / sqrt(rho);
      }
      cons_from_prim(rho, u, p, B, 0.0, A.gamma, Q);
    } else if (A.kind == SD_INIT_SHELL_POLYTROPE || A.kind == SD_INIT_SHELL_FLUX_BALANCED) {
      // Eq. (polytrop eqns) with T_b from N_rho; R_gas = P[4], C_p = gamma R/(gamma-1); or the
      // flux-balanced profile's table
      const double Nr = P[0], rb = P[1], rt = P[2], rhob = P[3], Rg = P[4], amp = P[5];
      const double g = A.gamma;
      const double Cp = g * Rg / (g - 1.0);
      const double r = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
      double rho0, p0;
      if (A.kind == SD_INIT_SHELL_POLYTROPE) {
        const double Tb = (-A.GM / rt + A.GM / rb) / (Cp * (1.0 - exp(-(g - 1.0) * Nr)));
        const double pb = rhob * Rg * Tb;
        const double zeta = 1.0 - (-A.GM / r + A.GM / rb) / (Cp * Tb);
        rho0 = rhob * pow(zeta, 1.0 / (g - 1.0));
        p0 = pb * pow(zeta, g / (g - 1.0));
      } else {
        profile_at(A.tab, g, r, rho0, p0);
      }
      const unsigned long long z = splitmix64(A.seed, (unsigned long long)(e * N3 + n));
      const double xi = 2.0 * ((double)(z >> 11) * 0x1.0p-53) - 1.0;
      const double rho = rho0 * (1.0 - amp * xi * sin(M_PI * (r - rb) / (rt - rb)));
      const double rh[3] = {x[0] / r, x[1] / r, x[2] / r};
      const double r3 = r * r * r;
      const double B[3] = {A.B0dip * (3.0 * rh[2] * rh[0]) / r3, A.B0dip * (3.0 * rh[2] * rh[1]) / r3,
                           A.B0dip * (3.0 * rh[2] * rh[2] - 1.0) / r3};
      cons_from_prim(rho, zero, p0, B, 0.0, g, Q);
      cons_from_prim(rho0, zero, p0, zero, 0.0, g, Qb);
    } else if (A.kind == SD_INIT_DIVB_PULSE) {
      const double dx = x[0] - P[3], dy = x[1] - P[4], dz = x[2] - P[5];
      const double B[3] = {P[2] * exp(-(dx * dx + dy * dy + dz * dz) / (2.0 * P[6] * P[6])), 0.0, 0.0};
      cons_from_prim(P[0], zero, P[1], B, 0.0, A.gamma, Q);
    }
  }
  for (int v = 0; v < 9; ++v) {
    q[v * A.plane + e * A.stride + n] = Q[v];
    if (qbg) qbg[v * A.plane + e * A.stride + n] = Qb[v];
  }
}

cudaError_t launch_state_init(const sd_mesh* m, const sd_phys* ph, const sd_init* in, double B0dip,
                              const ProfileTable& tab, double* q,
                              double* qbg, cudaStream_t s) {
  InitArgs A;
  A.kind = in->kind;
  A.N = m->N;
  A.n_e = m->n_e;
  A.stride = m->stride;
  A.plane = m->n_e * m->stride;
  for (int i = 0; i < 16; ++i) A.P[i] = in->params[i];
  A.seed = in->seed;
  A.gamma = ph->gamma;
  A.GM = ph->GM;
  A.B0dip = B0dip;
  A.tab = tab;
  if (in->kind == SD_INIT_SHELL_FLUX_BALANCED && !tab.tab) return cudaErrorInvalidValue;
  const int64_t tot = m->n_e * m->stride;
  if (tot == 0) return cudaSuccess;
  state_init_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(A, m->X64, q, qbg);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Diagnostics (Sec. Results): per-element partial sums, then one block sums
// the partials in element order -- a fixed order, so results are reproducible.
// slot: 0 ke, 1 eb, 2 mass, 3 energy, 4 volume, 5 max|divB|, 6 lambda_max,
//       7 min rho, 8 min p, 9 nonphysical count
// ---------------------------------------------------------------------------

constexpr int kDiag = 12;
constexpr int kDiagThreads = 256;

__device__ __forceinline__ double dmax_nan(double a, double b) { return (b > a || b != b) ? b : a; }
__device__ __forceinline__ double dmin_nan(double a, double b) { return (b < a || b != b) ? b : a; }

__device__ void block_reduce_diag(double* vals, double (*sm)[kDiagThreads]) {
  const int t = threadIdx.x;
  for (int k = 0; k < 10; ++k) sm[k][t] = vals[k];
  __syncthreads();
  for (int off = kDiagThreads / 2; off > 0; off >>= 1) {
    if (t < off) {
      for (int k = 0; k < 5; ++k) sm[k][t] += sm[k][t + off];
      sm[5][t] = dmax_nan(sm[5][t], sm[5][t + off]);
      sm[6][t] = dmax_nan(sm[6][t], sm[6][t + off]);
      sm[7][t] = dmin_nan(sm[7][t], sm[7][t + off]);
      sm[8][t] = dmin_nan(sm[8][t], sm[8][t + off]);
      sm[9][t] += sm[9][t + off];
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kDiagThreads) diag_partial_kernel(int N, int64_t stride, int64_t plane, double gamma,
                                                                    const Ops<double> ops, const double* __restrict__ q,
                                                                    const double* __restrict__ invJ,
                                                                    const double* __restrict__ divb, double* part) {
  __shared__ double sm[10][kDiagThreads];
  const int64_t e = blockIdx.x;
  const int N3 = N * N * N;
  double v[10] = {0, 0, 0, 0, 0, 0, 0, INFINITY, INFINITY, 0};
  for (int n = threadIdx.x; n < N3; n += kDiagThreads) {
    const int i = n % N, j = (n / N) % N, k = n / (N * N);
    double Q[9];
    for (int c = 0; c < 9; ++c) Q[c] = q[c * plane + e * stride + n];
    const double wq = ops.w[i] * ops.w[j] * ops.w[k] / invJ[e * N3 + n];
    const double rho = Q[0];
    const double m2 = Q[1] * Q[1] + Q[2] * Q[2] + Q[3] * Q[3];
    const double B2 = Q[5] * Q[5] + Q[6] * Q[6] + Q[7] * Q[7];
    const double p = (gamma - 1.0) * (Q[4] - 0.5 * (m2 / rho + B2 + Q[8] * Q[8]));
    v[0] += wq * 0.5 * m2 / rho;
    v[1] += wq * 0.5 * B2;
    v[2] += wq * rho;
    v[3] += wq * Q[4];
    v[4] += wq;
    v[5] = dmax_nan(v[5], fabs(divb[e * N3 + n]));
    v[6] = dmax_nan(v[6], sqrt(m2) / rho + sqrt(gamma * p / rho + B2 / rho));
    v[7] = dmin_nan(v[7], rho);
    v[8] = dmin_nan(v[8], p);
    if (!(rho > 0.0) || !(p > 0.0)) v[9] += 1.0;
  }
  block_reduce_diag(v, sm);
  if (threadIdx.x == 0)
    for (int k = 0; k < 10; ++k) part[e * kDiag + k] = sm[k][0];
}

__global__ void __launch_bounds__(kDiagThreads) diag_final_kernel(int64_t n_e, const double* __restrict__ part,
                                                                  double* out) {
  __shared__ double sm[10][kDiagThreads];
  double v[10] = {0, 0, 0, 0, 0, 0, 0, INFINITY, INFINITY, 0};
  for (int64_t e = threadIdx.x; e < n_e; e += kDiagThreads) {
    const double* p = part + e * kDiag;
    for (int k = 0; k < 5; ++k) v[k] += p[k];
    v[5] = dmax_nan(v[5], p[5]);
    v[6] = dmax_nan(v[6], p[6]);
    v[7] = dmin_nan(v[7], p[7]);
    v[8] = dmin_nan(v[8], p[8]);
    v[9] += p[9];
  }
  block_reduce_diag(v, sm);
  if (threadIdx.x == 0)
    for (int k = 0; k < 10; ++k) out[k] = sm[k][0];
}

cudaError_t launch_diag(const sd_mesh* m, const sd_phys* ph, const double* q, cudaStream_t s) {
  if (m->n_e == 0) return cudaSuccess;
  diag_partial_kernel<<<(unsigned)m->n_e, kDiagThreads, 0, s>>>(m->N, m->stride, m->n_e * m->stride, ph->gamma,
                                                                 m->ops64, q, m->invJ64, m->divb, m->diag_part);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  diag_final_kernel<<<1, kDiagThreads, 0, s>>>(m->n_e, m->diag_part, m->diag_out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Longitude averages on the shell (Sec. Results): volume sums over bins of
// radius x colatitude of (1, V_r, V_theta, V_phi, (B_r^2 + B_theta^2)/2,
// B_phi^2/2, rho, rho |U|^2 / 2), each weighted by w |J|.
//
// The sums do not depend on the order of the points: each quantity c is scaled
// by 2^s_c, with s_c chosen from the largest |term| of c over the mesh so that
// every scaled term is below 2^126, and split exactly into four signed 32-bit
// limbs of weights 2^0, 2^32, 2^64, 2^96 (the last one rounded to an integer).
// Integer additions of the limbs are exact and associative, so atomic additions
// give the same bits in any order; below 2^31 points per mesh no limb sum can
// overflow 64 bits.  The finish kernel propagates the carries and converts the
// four limbs to one double (within about one unit in its last place of the
// exact sum of the scaled terms).  Kernels: the maxima (one CTA per element, a
// block reduction, one atomicMax per quantity on the bits of a non-negative
// double, whose order is the integers'), the limb sums (one CTA per element:
// its points touch a small window of bins, summed in shared memory before one
// atomic per touched limb; a window too large for shared memory adds point by
// point), the finish (one thread per bin and quantity).
// ---------------------------------------------------------------------------

constexpr int kSphThreads = 256;
constexpr int kSphVals = 8;
constexpr int kSphLimbs = 4;
constexpr int kSphWindow = 64;  // bins per element window in shared memory

__device__ __forceinline__ void sph_point(const double* Q, const double* x, double wq, double r_min, double r_max,
                                          int n_r, int n_t, int& bin, double* val) {
  const double r = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  const double s = sqrt(x[0] * x[0] + x[1] * x[1]);
  const double th = atan2(s, x[2]);
  const double cp = s > 0.0 ? x[0] / s : 1.0, sp = s > 0.0 ? x[1] / s : 0.0;
  const double ct = cos(th), st = sin(th);
  const double ir = 1.0 / Q[0];
  const double U[3] = {Q[1] * ir, Q[2] * ir, Q[3] * ir};
  const double Vr = (U[0] * cp + U[1] * sp) * st + U[2] * ct;
  const double Vt = (U[0] * cp + U[1] * sp) * ct - U[2] * st;
  const double Vp = -U[0] * sp + U[1] * cp;
  const double Br = (Q[5] * cp + Q[6] * sp) * st + Q[7] * ct;
  const double Bt = (Q[5] * cp + Q[6] * sp) * ct - Q[7] * st;
  const double Bp = -Q[5] * sp + Q[6] * cp;
  int kr = (int)floor((r - r_min) / (r_max - r_min) * n_r);
  int kt = (int)floor(th / M_PI * n_t);
  kr = kr < 0 ? 0 : (kr >= n_r ? n_r - 1 : kr);
  kt = kt < 0 ? 0 : (kt >= n_t ? n_t - 1 : kt);
  bin = kr * n_t + kt;
  val[0] = wq;
  val[1] = wq * Vr;
  val[2] = wq * Vt;
  val[3] = wq * Vp;
  val[4] = wq * 0.5 * (Br * Br + Bt * Bt);
  val[5] = wq * 0.5 * Bp * Bp;
  val[6] = wq * Q[0];
  val[7] = wq * 0.5 * Q[0] * (U[0] * U[0] + U[1] * U[1] + U[2] * U[2]);
}

// the terms of point n of element e
__device__ __forceinline__ void sph_terms(int N, int64_t stride, int64_t plane, const Ops<double>& ops,
                                          const double* __restrict__ q, const double* __restrict__ X,
                                          const double* __restrict__ invJ, double r_min, double r_max, int n_r,
                                          int n_t, int64_t e, int n, int& bin, double* val) {
  const int N3 = N * N * N;
  const int i = n % N, j = (n / N) % N, k = n / (N * N);
  double Q[9], x[3];
  for (int c = 0; c < 9; ++c) Q[c] = q[c * plane + e * stride + n];
  for (int c = 0; c < 3; ++c) x[c] = X[(e * 3 + c) * N3 + n];
  sph_point(Q, x, ops.w[i] * ops.w[j] * ops.w[k] / invJ[e * N3 + n], r_min, r_max, n_r, n_t, bin, val);
}

__global__ void __launch_bounds__(kSphThreads) sph_max_kernel(int N, int64_t stride, int64_t plane,
                                                              const Ops<double> ops, const double* __restrict__ q,
                                                              const double* __restrict__ X,
                                                              const double* __restrict__ invJ, double r_min,
                                                              double r_max, int n_r, int n_t,
                                                              unsigned long long* vmax) {
  __shared__ double red[kSphThreads / 32][kSphVals];
  const int64_t e = blockIdx.x;
  const int N3 = N * N * N;
  double m[kSphVals];
  for (int c = 0; c < kSphVals; ++c) m[c] = 0.0;
  for (int n = threadIdx.x; n < N3; n += kSphThreads) {
    int bin;
    double val[kSphVals];
    sph_terms(N, stride, plane, ops, q, X, invJ, r_min, r_max, n_r, n_t, e, n, bin, val);
    for (int c = 0; c < kSphVals; ++c) m[c] = isfinite(val[c]) ? fmax(m[c], fabs(val[c])) : INFINITY;
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int c = 0; c < kSphVals; ++c) {
    double v = m[c];
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) red[w][c] = v;
  }
  __syncthreads();
  if (threadIdx.x < kSphVals) {
    double v = 0.0;
    for (int k = 0; k < kSphThreads / 32; ++k) v = fmax(v, red[k][threadIdx.x]);
    atomicMax(vmax + threadIdx.x, (unsigned long long)__double_as_longlong(v));
  }
}

// s_c: the largest |term| of quantity c scaled by 2^s_c lies below 2^126 (0 when
// every term is zero or some term is not finite: the sum is then NaN)
__device__ __forceinline__ int sph_shift(unsigned long long bits) {
  const double m = __longlong_as_double((long long)bits);
  if (!(m > 0.0) || !isfinite(m)) return 0;
  int ex;
  frexp(m, &ex);  // m < 2^ex
  return 126 - ex;
}

// x = t 2^s (|x| < 2^126) as l[0] + l[1] 2^32 + l[2] 2^64 + l[3] 2^96, |l[k]| < 2^32:
// every step but the last rounding is exact (a power-of-two scaling, a truncation,
// the subtraction of x's own leading bits)
__device__ __forceinline__ void sph_limbs(double t, int s, long long* l) {
  double x = ldexp(t, s);
  const double w96 = 0x1p96, w64 = 0x1p64, w32 = 0x1p32;
  const double a = trunc(x * 0x1p-96);
  x -= a * w96;
  const double b = trunc(x * 0x1p-64);
  x -= b * w64;
  const double c = trunc(x * 0x1p-32);
  x -= c * w32;
  l[3] = (long long)a;
  l[2] = (long long)b;
  l[1] = (long long)c;
  l[0] = __double2ll_rn(x);
}

__global__ void __launch_bounds__(kSphThreads) spherical_kernel(int N, int64_t stride, int64_t plane,
                                                                const Ops<double> ops, const double* __restrict__ q,
                                                                const double* __restrict__ X,
                                                                const double* __restrict__ invJ, double r_min,
                                                                double r_max, int n_r, int n_t,
                                                                const unsigned long long* __restrict__ vmax,
                                                                unsigned long long* acc) {
  __shared__ unsigned long long win[kSphWindow * kSphVals * kSphLimbs];
  __shared__ int lo_hi[2];
  __shared__ int shift[kSphVals];
  const int64_t e = blockIdx.x;
  const int N3 = N * N * N;
  if (threadIdx.x == 0) {
    lo_hi[0] = INT_MAX;
    lo_hi[1] = -1;
  }
  if (threadIdx.x < kSphVals) shift[threadIdx.x] = sph_shift(vmax[threadIdx.x]);
  for (int i = threadIdx.x; i < kSphWindow * kSphVals * kSphLimbs; i += kSphThreads) win[i] = 0ull;
  __syncthreads();
  // pass 1: the range of bins this element touches
  for (int n = threadIdx.x; n < N3; n += kSphThreads) {
    int bin;
    double val[kSphVals];
    sph_terms(N, stride, plane, ops, q, X, invJ, r_min, r_max, n_r, n_t, e, n, bin, val);
    atomicMin(&lo_hi[0], bin);
    atomicMax(&lo_hi[1], bin);
  }
  __syncthreads();
  const int lo = lo_hi[0], span = lo_hi[1] - lo_hi[0] + 1;
  const bool local = span <= kSphWindow;
  // pass 2: limb sums (two's complement: an unsigned addition adds the signed limbs)
  for (int n = threadIdx.x; n < N3; n += kSphThreads) {
    int bin;
    double val[kSphVals];
    sph_terms(N, stride, plane, ops, q, X, invJ, r_min, r_max, n_r, n_t, e, n, bin, val);
    for (int c = 0; c < kSphVals; ++c) {
      if (!isfinite(val[c])) continue;  // the finish kernel writes NaN for this quantity
      long long l[kSphLimbs];
      sph_limbs(val[c], shift[c], l);
      unsigned long long* dst =
          local ? win + ((bin - lo) * kSphVals + c) * kSphLimbs : acc + ((int64_t)bin * kSphVals + c) * kSphLimbs;
      for (int k = 0; k < kSphLimbs; ++k)
        if (l[k] != 0) atomicAdd(dst + k, (unsigned long long)l[k]);
    }
  }
  __syncthreads();
  if (local)
    for (int t = threadIdx.x; t < span * kSphVals * kSphLimbs; t += kSphThreads)
      if (win[t] != 0ull) atomicAdd(acc + (int64_t)lo * kSphVals * kSphLimbs + t, win[t]);
}

__global__ void sph_finish_kernel(int64_t n_entries, const unsigned long long* __restrict__ vmax,
                                  const unsigned long long* __restrict__ acc, double* __restrict__ out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_entries) return;
  const int c = (int)(t % kSphVals);
  long long L[kSphLimbs];
  for (int k = 0; k < kSphLimbs; ++k) L[k] = (long long)acc[t * kSphLimbs + k];
  // carries: limbs 0..2 into [0, 2^32), the sign in limb 3
  for (int k = 0; k < kSphLimbs - 1; ++k) {
    const long long low = (long long)((unsigned long long)L[k] & 0xffffffffull);
    L[k + 1] += (L[k] - low) / 4294967296ll;
    L[k] = low;
  }
  const double r = ldexp((double)L[3], 96) + (ldexp((double)L[2], 64) + (ldexp((double)L[1], 32) + (double)L[0]));
  const double m = __longlong_as_double((long long)vmax[c]);
  out[t] = isfinite(m) ? ldexp(r, -sph_shift(vmax[c])) : __longlong_as_double(0x7ff8000000000000ll);
}

// ---------------------------------------------------------------------------
// Viscous record of the FP32-mixed background: the energy component of the
// background's viscous residual (its residual with viscous fluxes less the one
// without, both FP64), grad T0 and grad S0 at the solution points (values 9..11
// and 12..14 of the FP64 viscous record) and their face traces, in FP32.
// ---------------------------------------------------------------------------

__global__ void bg_visc_kernel(int N, int64_t n_e, int64_t stride, const double* __restrict__ R0,
                               const double* __restrict__ R0v, const double* __restrict__ grad,
                               const double* __restrict__ gtr, float* __restrict__ vrec, float* __restrict__ vtr) {
  const int N2 = N * N, N3 = N2 * N;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t plane = n_e * stride;
  if (t < n_e * N3) {
    const int64_t e = t / N3;
    const int n = (int)(t - e * N3);
    const int64_t g = e * stride + n;
    vrec[t] = (float)(R0v[4 * plane + g] - R0[4 * plane + g]);
    for (int k = 0; k < 6; ++k) vrec[(1 + k) * n_e * N3 + t] = (float)grad[(e * MV_REC + 9 + k) * N3 + n];
  }
  if (t < n_e * 6 * N2) {
    const int64_t ef = t / N2;
    const int pt = (int)(t - ef * N2);
    for (int k = 0; k < 6; ++k) vtr[(ef * 6 + k) * N2 + pt] = (float)gtr[(ef * MV_REC + 9 + k) * N2 + pt];
  }
}

cudaError_t launch_bg_visc(const sd_mesh* m, const double* R0, const double* R0v, const double* grad,
                           const double* gtr, float* vrec, float* vtr, cudaStream_t s) {
  const int64_t N2 = (int64_t)m->N * m->N, N3 = N2 * m->N;
  const int64_t tot = m->n_e * (N3 > 6 * N2 ? N3 : 6 * N2);
  if (tot == 0) return cudaSuccess;
  bg_visc_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(m->N, m->n_e, m->stride, R0, R0v, grad, gtr, vrec, vtr);
  return cudaGetLastError();
}

cudaError_t launch_spherical(const sd_mesh* m, const double* q, double r_min, double r_max, int n_r, int n_t,
                             double* out, cudaStream_t s) {
  const int64_t n_entries = (int64_t)n_r * n_t * kSphVals;
  const size_t acc_bytes = (size_t)n_entries * kSphLimbs * sizeof(unsigned long long);
  unsigned long long* scratch = nullptr;  // [8] maxima, then the limbs [n_r * n_t][8][4]
  cudaError_t err = cudaMallocAsync((void**)&scratch, acc_bytes + kSphVals * sizeof(unsigned long long), s);
  if (err != cudaSuccess) return err;
  unsigned long long* vmax = scratch;
  unsigned long long* acc = scratch + kSphVals;
  err = cudaMemsetAsync(scratch, 0, acc_bytes + kSphVals * sizeof(unsigned long long), s);
  const int64_t plane = m->n_e * m->stride;
  if (err == cudaSuccess && m->n_e > 0) {
    sph_max_kernel<<<(unsigned)m->n_e, kSphThreads, 0, s>>>(m->N, m->stride, plane, m->ops64, q, m->X64, m->invJ64,
                                                            r_min, r_max, n_r, n_t, vmax);
    err = cudaGetLastError();
    if (err == cudaSuccess) {
      spherical_kernel<<<(unsigned)m->n_e, kSphThreads, 0, s>>>(m->N, m->stride, plane, m->ops64, q, m->X64,
                                                                m->invJ64, r_min, r_max, n_r, n_t, vmax, acc);
      err = cudaGetLastError();
    }
  }
  if (err == cudaSuccess) {
    sph_finish_kernel<<<(unsigned)((n_entries + 255) / 256), 256, 0, s>>>(n_entries, vmax, acc, out);
    err = cudaGetLastError();
  }
  cudaError_t err2 = cudaFreeAsync(scratch, s);
  return err != cudaSuccess ? err : err2;
}

// ---------------------------------------------------------------------------
// FP32-mixed background: rho0 and p0 rounded to FP32 define the background Q0
// exactly; its FP64 residual R0 and its FP64 face jumps are stored in FP32.
// ---------------------------------------------------------------------------

__global__ void bg_prepare_kernel(int N, int64_t n_e, int64_t stride, double gamma, double inv_gm1,
                                  const double* __restrict__ qbg, double* q0, float* rec) {
  const int N3 = N * N * N;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_e * stride) return;
  const int64_t e = t / stride;
  const int n = (int)(t % stride);
  const int64_t plane = n_e * stride;
  double Q[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  if (n < N3) {
    const float r0 = (float)qbg[e * stride + n];
    const float p0 = (float)((gamma - 1.0) * qbg[4 * plane + e * stride + n]);
    rec[e * N3 + n] = r0;
    rec[n_e * N3 + e * N3 + n] = p0;
    Q[0] = (double)r0;
    Q[4] = (double)p0 * inv_gm1;  // the definition of E0 every mixed kernel uses
  }
  for (int v = 0; v < 9; ++v) q0[v * plane + e * stride + n] = Q[v];
}

__global__ void bg_finish_kernel(int N, int64_t n_e, int64_t stride, double gamma, const double* __restrict__ R0,
                                 const double* __restrict__ tr, const int* __restrict__ nbr,
                                 const int* __restrict__ meta, float* rec, float* jump) {
  const int N2 = N * N, N3 = N2 * N;
  const int64_t plane = n_e * stride;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n_e * N3) {
    const int64_t e = t / N3;
    const int n = (int)(t % N3);
    for (int c = 0; c < 3; ++c) rec[(2 + c) * n_e * N3 + t] = (float)R0[(1 + c) * plane + e * stride + n];
  }
  if (t < n_e * 6 * N2) {
    const int64_t e = t / (6 * N2);
    const int F = (int)((t / N2) % 6), pt = (int)(t % N2), a = pt % N, b = pt / N;
    const int nb = nbr[e * 6 + F], mt = meta[e * 6 + F];
    float jr = 0.0f, jp = 0.0f;
    if (nb >= 0) {
      const int code = meta_code(mt);
      const int u = (code & 4) ? b : a, w = (code & 4) ? a : b;
      const int a2 = (code & 2) ? N - 1 - u : u, b2 = (code & 1) ? N - 1 - w : w;
      const double* To = tr + (e * 6 + F) * 9 * N2 + pt;
      const double* Tn = tr + ((int64_t)nb * 6 + meta_nbF(mt)) * 9 * N2 + a2 + N * b2;
      jr = (float)(Tn[0] - To[0]);
      jp = (float)((gamma - 1.0) * (Tn[4 * N2] - To[4 * N2]));
    }
    jump[((e * 6 + F) * 2 + 0) * N2 + pt] = jr;
    jump[((e * 6 + F) * 2 + 1) * N2 + pt] = jp;
  }
}

cudaError_t launch_bg_prepare(const sd_mesh* m, double gamma, double inv_gm1, const double* q_bg, double* q0,
                              float* rec, cudaStream_t s) {
  const int64_t tot = m->n_e * m->stride;
  if (tot == 0) return cudaSuccess;
  bg_prepare_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(m->N, m->n_e, m->stride, gamma, inv_gm1, q_bg, q0,
                                                                  rec);
  return cudaGetLastError();
}

cudaError_t launch_bg_finish(const sd_mesh* m, double gamma, const double* R0, float* rec, float* jump,
                             const double* tr, cudaStream_t s) {
  const int64_t N2 = (int64_t)m->N * m->N;
  const int64_t tot = m->n_e * (6 * N2 > N2 * m->N ? 6 * N2 : N2 * m->N);
  if (tot == 0) return cudaSuccess;
  bg_finish_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(m->N, m->n_e, m->stride, gamma, R0, tr, m->nbr,
                                                                 m->meta, rec, jump);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Step control: dt = cfl * (smallest solution-point spacing) / lambda_max, the
// spacing being h_min times the first gap of the Chebyshev-Gauss points;
// c_h = lambda_max unless fixed.
// ---------------------------------------------------------------------------

// One block of LAM_SLOTS threads: lambda_max = largest of the partial maxima
// (compared as bit patterns, as the atomics wrote them), which are cleared for
// the next reduction; then dt and c_h.
// For the diffusive limit of the step: the smallest density over the solution
// points of the FP64 state q (atomicMin on the bits of a positive double into
// lo[0]; a NaN or a non-positive density, whose bits order above every positive
// double, is passed over: the state's lambda_max is NaN then and so is dt) and,
// when kappa_r varies, the largest gamma kappa_r(|x|) (atomicMax into hi[0]).
// No division per point: the step control forms 4/3 mu / rho_min once.
__global__ void visc_extrema_kernel(int N3, int64_t n_e, int64_t stride, const double* __restrict__ q,
                                    const double* __restrict__ X, double gamma, double kr0, double kr1, double kr2,
                                    unsigned long long* lo, unsigned long long* hi) {
  const bool kr_varies = kr1 != 0.0 || kr2 != 0.0;
  double rmin = INFINITY, kmax = 0.0;
  const int64_t n = n_e * N3;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = t / N3;
    const int k = (int)(t - e * N3);
    const double rho = q[e * stride + k];
    rmin = rho > 0.0 && rho < rmin ? rho : rmin;
    if (kr_varies) {
      const double* x = X + e * 3 * N3 + k;
      const double r = sqrt(x[0] * x[0] + x[N3] * x[N3] + x[2 * N3] * x[2 * N3]);
      const double g = gamma * (kr0 + kr1 * r + kr2 * r * r);
      kmax = g > kmax ? g : kmax;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double r2 = __shfl_xor_sync(0xffffffffu, rmin, o), k2 = __shfl_xor_sync(0xffffffffu, kmax, o);
    rmin = r2 < rmin ? r2 : rmin;
    kmax = k2 > kmax ? k2 : kmax;
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(lo, (unsigned long long)__double_as_longlong(rmin));
    if (kr_varies) atomicMax(hi, (unsigned long long)__double_as_longlong(kmax));
  }
}

cudaError_t launch_visc_numax(const sd_mesh* m, const sd_phys* ph, const double* q, cudaStream_t s) {
  unsigned long long* lo = reinterpret_cast<unsigned long long*>(m->dyn + 3);
  unsigned long long* hi = reinterpret_cast<unsigned long long*>(m->dyn + 4 + LAM_SLOTS);
  cudaError_t err = cudaMemsetAsync(lo, 0xff, sizeof(unsigned long long), s);  // above every positive double
  if (err == cudaSuccess) err = cudaMemsetAsync(hi, 0, sizeof(unsigned long long), s);
  if (err != cudaSuccess || m->n_e == 0) return err;
  const int N3 = m->N * m->N * m->N;
  const int64_t n = m->n_e * N3;
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 152 * 8);
  visc_extrema_kernel<<<(unsigned)blocks, 256, 0, s>>>(N3, m->n_e, m->stride, q, m->X64, ph->gamma, ph->kappa_r,
                                                       ph->kappa_r1, ph->kappa_r2, lo, hi);
  return cudaGetLastError();
}

// The step-control kernel.  visc_dx2 > 0: also dt <= visc_dx2 / nu_max, nu_max =
// max(mu43 / rho_min, nu_c, the largest gamma kappa_r(r)) from the extrema that
// visc_extrema_kernel left in dyn[3] and dyn[4 + LAM_SLOTS].
__global__ void __launch_bounds__(LAM_SLOTS) step_control_kernel(double* dyn, double cfl, double dx_min,
                                                                 double ch_fixed, double* dt_out, double* dyn_s,
                                                                 double dt_scale, double visc_dx2, double mu43,
                                                                 double nu_c) {
  __shared__ unsigned long long part[LAM_SLOTS / 32];
  unsigned long long* slots = reinterpret_cast<unsigned long long*>(dyn + 4);
  unsigned long long b = slots[threadIdx.x];
  slots[threadIdx.x] = 0ull;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long other = __shfl_xor_sync(0xffffffffu, b, o);
    b = other > b ? other : b;
  }
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = b;
  __syncthreads();
  if (threadIdx.x != 0) return;
  for (int w = 1; w < LAM_SLOTS / 32; ++w) b = part[w] > b ? part[w] : b;
  const double lam = __longlong_as_double((long long)b);
  double dt = cfl * dx_min / lam;
  if (visc_dx2 > 0.0) {
    double nu = mu43 / dyn[3];
    nu = nu_c > nu ? nu_c : nu;
    nu = dyn[4 + LAM_SLOTS] > nu ? dyn[4 + LAM_SLOTS] : nu;
    const double dtv = visc_dx2 / nu;
    dt = (dtv < dt || dtv != dtv) ? dtv : dt;
  }
  const double ch = ch_fixed > 0.0 ? ch_fixed : lam;
  dyn[0] = dt;
  dyn[1] = ch;
  dyn[2] = lam;
  if (dyn_s) {  // the pair the FP64 stages of the five-stage method read: (dt / r, c_h)
    dyn_s[0] = dt * dt_scale;
    dyn_s[1] = ch;
  }
  if (dt_out) {
    dt_out[0] = dt;
    dt_out[1] = ch;
  }
}

cudaError_t launch_step_control(const sd_mesh* m, double cfl, double c_h_fixed, double* dt_out, cudaStream_t s,
                                double* dyn_s, double dt_scale, const sd_phys* visc) {
  const double dx_min = m->h_min * (m->ops64.xs[1] - m->ops64.xs[0]);
  double visc_dx2 = 0.0, mu43 = 0.0, nu_c = 0.0;
  if (visc && visc->viscous && visc->visc_cfl > 0.0) {
    visc_dx2 = visc->visc_cfl * dx_min * dx_min;
    mu43 = 4.0 / 3.0 * visc->mu;
    const double kr_c = (visc->kappa_r1 != 0.0 || visc->kappa_r2 != 0.0) ? 0.0 : visc->gamma * visc->kappa_r;
    nu_c = visc->eta > visc->kappa ? visc->eta : visc->kappa;
    nu_c = kr_c > nu_c ? kr_c : nu_c;
  }
  step_control_kernel<<<1, LAM_SLOTS, 0, s>>>(m->dyn, cfl, dx_min, c_h_fixed, dt_out, dyn_s, dt_scale, visc_dx2,
                                              mu43, nu_c);
  return cudaGetLastError();
}

// out = a x + b y over n FP64 values (the five-stage method's W = a61 y2 + a62 y3)
__global__ void axpby_f64_kernel(double* out, double a, const double* __restrict__ x, double b,
                                 const double* __restrict__ y, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = a * x[i] + b * y[i];
}

cudaError_t launch_axpby_f64(double* out, double a, const double* x, double b, const double* y, int64_t n,
                             cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 152 * 16);
  axpby_f64_kernel<<<(unsigned)blocks, 256, 0, s>>>(out, a, x, b, y, n);
  return cudaGetLastError();
}

// out = q + W for an FP64 state q ([9][n_e stride]) and an FP32 register W ([9][n_e dstride]),
// the padding of q copied
__global__ void add_reg_f64_kernel(double* out, const double* __restrict__ q, const float* __restrict__ w,
                                   int64_t n_e, int N3, int64_t stride, int64_t dstride) {
  const int64_t per_v = n_e * stride, n = 9 * per_v;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = i / per_v, r = i - v * per_v, e = r / stride, k = r - e * stride;
    out[i] = k < N3 ? q[i] + (double)w[(v * n_e + e) * dstride + k] : q[i];
  }
}

cudaError_t launch_add_reg_f64(const sd_mesh* m, double* out, const double* q, const float* w, int64_t dstride,
                               cudaStream_t s) {
  const int64_t n = 9 * m->n_e * m->stride;
  if (n == 0) return cudaSuccess;
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 152 * 16);
  add_reg_f64_kernel<<<(unsigned)blocks, 256, 0, s>>>(out, q, w, m->n_e, m->N * m->N * m->N, m->stride, dstride);
  return cudaGetLastError();
}

}  // namespace sd
