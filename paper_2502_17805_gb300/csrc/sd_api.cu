// sd_api.cu -- host side of the C ABI declared in include/sdmhd.h.
//
// Mesh construction (face matching, orientation codes, boundary tagging,
// operator tables) runs on the host; everything per solution point or flux
// point runs in the CUDA kernels of this library.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <string>
#include <vector>

#include "sd_internal.h"

namespace {

thread_local std::string g_err;
thread_local std::string g_stale;  // a CUDA error left pending by an earlier, unrelated call

sd_status fail(sd_status st, const std::string& msg) {
  g_err = g_stale.empty() ? msg : msg + " (a CUDA error was already pending before this call: " + g_stale + ")";
  return st;
}

// Clear a pending error of this thread's CUDA runtime state, so that the error
// checks of this call see only this call's work; remember it for the message.
void take_stale() {
  const cudaError_t e = cudaGetLastError();
  g_stale = e == cudaSuccess ? std::string() : std::string(cudaGetErrorString(e));
}

sd_status cuda_fail(cudaError_t e, const char* what) {
  return fail(SD_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define SD_CUDA(call)                                          \
  do {                                                         \
    cudaError_t e_ = (call);                                   \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);        \
  } while (0)

struct DeviceGuard {
  int prev = -1;
  bool switched = false;
  explicit DeviceGuard(int dev) {
    take_stale();
    if (cudaGetDevice(&prev) != cudaSuccess) {
      prev = -1;
      cudaGetLastError();
      return;
    }
    if (prev != dev) {
      switched = cudaSetDevice(dev) == cudaSuccess;
      if (!switched) cudaGetLastError();
    }
  }
  ~DeviceGuard() {
    if (switched && cudaSetDevice(prev) != cudaSuccess) cudaGetLastError();
  }
};

// ---------------------------------------------------------------- 1D operators

// Legendre polynomial P_M and its derivative at x (Bonnet recurrence)
void legendre(int M, double x, double* P, double* dP) {
  double a = 1.0, b = x;
  if (M == 0) {
    *P = 1.0;
    *dP = 0.0;
    return;
  }
  for (int k = 2; k <= M; ++k) {
    const double c = ((2.0 * k - 1.0) * x * b - (k - 1.0) * a) / k;
    a = b;
    b = c;
  }
  *P = b;
  *dP = M * (a - x * b) / (1.0 - x * x);
}

// Gauss-Legendre nodes (ascending) and weights on [-1, 1] by Newton iteration
void gauss_legendre(int M, std::vector<double>& x, std::vector<double>& w) {
  x.assign(M, 0.0);
  w.assign(M, 0.0);
  for (int k = 0; k < M; ++k) {
    double t = -cos(M_PI * (k + 0.75) / (M + 0.5));
    for (int it = 0; it < 60; ++it) {
      double P, dP;
      legendre(M, t, &P, &dP);
      const double step = P / dP;
      t -= step;
      if (fabs(step) < 1e-16) break;
    }
    double P, dP;
    legendre(M, t, &P, &dP);
    x[k] = t;
    w[k] = 2.0 / ((1.0 - t * t) * dP * dP);
  }
  std::sort(x.begin(), x.end());
  for (int k = 0; k < M; ++k) {
    double P, dP;
    legendre(M, x[k], &P, &dP);
    w[k] = 2.0 / ((1.0 - x[k] * x[k]) * dP * dP);
  }
}

double lagr(const double* z, int n, int i, double t) {
  double v = 1.0;
  for (int s = 0; s < n; ++s)
    if (s != i) v *= (t - z[s]) / (z[i] - z[s]);
  return v;
}

double lagr_d(const double* z, int n, int i, double t) {
  double sum = 0.0;
  for (int m = 0; m < n; ++m) {
    if (m == i) continue;
    double pr = 1.0 / (z[i] - z[m]);
    for (int s = 0; s < n; ++s)
      if (s != i && s != m) pr *= (t - z[s]) / (z[i] - z[s]);
    sum += pr;
  }
  return sum;
}

// Solution points: Chebyshev-Gauss, X_s,n = (1 - cos((2n-1) pi / 2N)) / 2.
// Flux points: 0, the N-1 roots of P_{N-1} mapped to [0, 1], and 1 (N+1 points).
void build_ops(int N, sd::Ops<double>& o) {
  memset(&o, 0, sizeof(o));
  for (int n = 0; n < N; ++n) o.xs[n] = 0.5 * (1.0 - cos((2.0 * n + 1.0) * M_PI / (2.0 * N)));
  std::vector<double> r, wr;
  gauss_legendre(N - 1, r, wr);
  o.xf[0] = 0.0;
  for (int k = 0; k < N - 1; ++k) o.xf[k + 1] = 0.5 * (r[k] + 1.0);
  o.xf[N] = 1.0;
  for (int f = 0; f <= N; ++f)
    for (int i = 0; i < N; ++i) o.E[f * N + i] = lagr(o.xs, N, i, o.xf[f]);
  for (int i = 0; i < N; ++i)
    for (int f = 0; f <= N; ++f) o.D[i * (N + 1) + f] = lagr_d(o.xf, N + 1, f, o.xs[i]);
  // even-odd split: solution indices i <= N-1-i, flux indices f <= N-f
  for (int f = 0; 2 * f <= N; ++f)
    for (int i = 0; 2 * i <= N - 1; ++i) {
      const double a = o.E[f * N + i], b = o.E[f * N + N - 1 - i];
      o.Es[f * N + i] = (2 * i == N - 1) ? a : 0.5 * (a + b);
      o.Ed[f * N + i] = (2 * i == N - 1) ? 0.0 : 0.5 * (a - b);
    }
  for (int i = 0; 2 * i <= N - 1; ++i)
    for (int f = 0; 2 * f <= N; ++f) {
      const double a = o.D[i * (N + 1) + f], b = o.D[i * (N + 1) + N - f];
      o.Ds[i * (N + 1) + f] = (2 * f == N) ? a : 0.5 * (a + b);
      o.Dd[i * (N + 1) + f] = (2 * f == N) ? 0.0 : 0.5 * (a - b);
    }
  std::vector<double> g, gw;
  gauss_legendre(N + 3, g, gw);
  for (int i = 0; i < N; ++i) {
    double s = 0.0;
    for (int k = 0; k < N + 3; ++k) s += 0.5 * gw[k] * lagr(o.xs, N, i, 0.5 * (g[k] + 1.0));
    o.w[i] = s;
  }
}

void ops_to_f32(const sd::Ops<double>& a, sd::Ops<float>& b) {
  for (int i = 0; i < (sd::kMaxN + 1) * sd::kMaxN; ++i) {
    b.E[i] = (float)a.E[i];
    b.D[i] = (float)a.D[i];
    b.Es[i] = (float)a.Es[i];
    b.Ed[i] = (float)a.Ed[i];
    b.Ds[i] = (float)a.Ds[i];
    b.Dd[i] = (float)a.Dd[i];
  }
  for (int i = 0; i < sd::kMaxN; ++i) {
    b.w[i] = (float)a.w[i];
    b.xs[i] = (float)a.xs[i];
  }
  for (int i = 0; i <= sd::kMaxN; ++i) b.xf[i] = (float)a.xf[i];
}

void ops_to_pairs(int N, const sd::Ops<float>& a, sd::Ops2& b) {
  memset(&b, 0, sizeof(b));
  for (int i = 0; i < (sd::kMaxN + 1) * sd::kMaxN; ++i) {
    b.Es[i] = make_float2(a.Es[i], a.Es[i]);
    b.Ed[i] = make_float2(a.Ed[i], a.Ed[i]);
    b.Ds[i] = make_float2(a.Ds[i], a.Ds[i]);
    b.Dd[i] = make_float2(a.Dd[i], a.Dd[i]);
  }
  for (int i = 0; i < N; ++i) {
    b.E0[i] = make_float2(a.E[i], a.E[i]);
    b.EN[i] = make_float2(a.E[N * N + i], a.E[N * N + i]);
  }
}

// ---------------------------------------------------------------- mesh topology

// corner of face F at face-local corner (s, t); the face-local axes are the two
// remaining directions in increasing order
int face_corner(int F, int s, int t) {
  const int d = F >> 1, side = F & 1;
  int c[3];
  c[d] = side;
  c[d == 0 ? 1 : 0] = s;
  c[d == 2 ? 1 : 2] = t;
  return c[0] + 2 * c[1] + 4 * c[2];
}

// orientation code of the map (a, b) on face F1 of e1 -> (a', b') on face F2 of e2
int orientation(const int64_t* hex, int64_t e1, int F1, int64_t e2, int F2) {
  int s0 = -1, t0 = -1, s1 = -1, t1 = -1, s2 = -1, t2 = -1;
  const int64_t v00 = hex[8 * e1 + face_corner(F1, 0, 0)];
  const int64_t v10 = hex[8 * e1 + face_corner(F1, 1, 0)];
  const int64_t v01 = hex[8 * e1 + face_corner(F1, 0, 1)];
  for (int s = 0; s < 2; ++s)
    for (int t = 0; t < 2; ++t) {
      const int64_t v = hex[8 * e2 + face_corner(F2, s, t)];
      if (v == v00) { s0 = s; t0 = t; }
      if (v == v10) { s1 = s; t1 = t; }
      if (v == v01) { s2 = s; t2 = t; }
    }
  if (s0 < 0 || s1 < 0 || s2 < 0) return -1;
  // the second face must be reached consistently: the two probed axes must differ
  if ((s1 != s0) == (s2 != s0)) return -1;
  if (s1 != s0) {
    if (t1 != t0 || s2 != s0 || t2 == t0) return -1;
    return (0 << 2) | ((s0 == 1) << 1) | (t0 == 1);
  }
  if (t1 == t0 || s2 == s0 || t2 != t0) return -1;
  return (1 << 2) | ((s0 == 1) << 1) | (t0 == 1);
}

int64_t round_stride(int N) {
  const int64_t n3 = (int64_t)N * N * N;
  return (n3 + 1) / 2 * 2;  // 16-byte aligned element starts for FP64
}

template <typename T>
cudaError_t dalloc(T** p, size_t count, int64_t* bytes) {
  *bytes += (int64_t)(count * sizeof(T));
  return cudaMalloc((void**)p, count * sizeof(T) + 16);
}

void free_mesh(sd_mesh* m) {
  if (!m) return;
  for (cudaEvent_t ev : m->prof_ev) cudaEventDestroy(ev);
  void* ptrs[] = {m->own_faces, m->face_k, m->gface64, m->Sfam64, m->invJ64, m->X64, m->Sfam32, m->invJ32, m->X32,
                  m->nbr, m->meta,
                  m->tr64[0], m->tr64[1], m->tr32[0], m->tr32[1], m->dyn, m->diag_part, m->diag_out, m->divb,
                  m->err, m->grad, m->gtr, m->rvis64, m->grad32, m->mvf32, m->rvis32, m->dyn_s, m->work2, m->wreg32};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (m->host_diag) cudaFreeHost(m->host_diag);
  delete m;
}

sd_status check_state_ptr(const void* p, const char* name) {
  if (!p) return fail(SD_ERR_INVALID_ARGUMENT, std::string(name) + " is NULL");
  if (((uintptr_t)p & 15) != 0) return fail(SD_ERR_INVALID_ARGUMENT, std::string(name) + " is not 16-byte aligned");
  return SD_OK;
}

sd::StageParams base_params(const sd_mesh* m, const sd_phys* ph, int prec) {
  sd::StageParams P;
  memset(&P, 0, sizeof(P));
  P.n_e = m->n_e;
  P.stride = m->stride;
  P.plane = m->n_e * m->stride;
  P.gamma = ph->gamma;
  P.GM = ph->GM;
  P.omega = ph->omega;
  P.alpha = ph->glm_alpha;
  P.inv_gm1 = 1.0 / (ph->gamma - 1.0);
  P.c_h = ph->c_h;
  P.powell = ph->powell;
  P.gravity = ph->gravity;
  P.coriolis = ph->coriolis;
  for (int v = 0; v < 9; ++v) P.farfield[v] = ph->farfield[v];
  if (prec == SD_FP64) {
    P.Sfam = m->Sfam64;
    P.invJ = m->invJ64;
    P.X = m->X64;
  } else {
    P.Sfam = m->Sfam32;
    P.invJ = m->invJ32;
    P.X = m->X32;
  }
  P.nbr = m->nbr;
  P.meta = m->meta;
  P.err = m->err;
  P.wait_spins = m->wait_spins;
  P.n_own = m->n_own;
  P.own_faces = m->own_faces;
  P.face_k = m->face_k;
  P.gface = m->gface64;
  P.visc = ph->viscous ? 1 : 0;
  P.mu = ph->mu;
  P.eta = ph->eta;
  P.kappa = ph->kappa;
  P.kappa_r = ph->kappa_r;
  P.kappa_r1 = ph->kappa_r1;
  P.kappa_r2 = ph->kappa_r2;
  P.R_gas = ph->R_gas;
  P.visc_walls = ph->visc_walls ? 1 : 0;
  P.q_bottom = ph->q_bottom;
  P.T_top = ph->T_top;
  return P;
}


void* trace_buf(sd_mesh* m, int prec, int b) { return prec == SD_FP64 ? (void*)m->tr64[b] : (void*)m->tr32[b]; }

// Kernel timing: CUDA events on the launching stream around one launch.
enum { PROF_STAGE = 0, PROF_TRACE = 1, PROF_OTHER = 2 };
constexpr size_t kMaxProf = 65536;

struct ProfScope {
  sd_mesh* m;
  cudaStream_t s;
  bool on;
  ProfScope(const sd_mesh* mc, int cls, cudaStream_t st) : m(const_cast<sd_mesh*>(mc)), s(st), on(false) {
    if (!m->prof_on || m->prof_used >= kMaxProf) return;
    const size_t i = m->prof_used;
    while (m->prof_ev.size() < 2 * (i + 1)) {
      cudaEvent_t ev;
      if (cudaEventCreate(&ev) != cudaSuccess) return;
      m->prof_ev.push_back(ev);
    }
    if (m->prof_cls.size() < i + 1) m->prof_cls.resize(i + 1);
    m->prof_cls[i] = cls;
    on = cudaEventRecord(m->prof_ev[2 * i], s) == cudaSuccess;
  }
  ~ProfScope() {
    if (!on) return;
    if (cudaEventRecord(m->prof_ev[2 * m->prof_used + 1], s) == cudaSuccess) m->prof_used++;
  }
};

// Viscous FP32-mixed path: the perturbation gradients of the stage state that P
// describes (whose face traces are P.tr_in) and their face traces, then the
// viscous residual of that state (the background's included) into the mesh's
// buffers (allocated on first use); P then points the stage kernel at it.
cudaError_t prepare_viscous_mixed(sd_mesh* m, sd::StageParams& P, const sd_background* bg, cudaStream_t s) {
  const size_t N2 = (size_t)m->N * m->N, N3 = N2 * m->N, ne = (size_t)std::max<int64_t>(m->n_e, 1);
  cudaError_t err = cudaSuccess;
  struct Buf {
    float** p;
    size_t count;
  } bufs[3] = {{&m->grad32, ne * sd::MV_REC * N3}, {&m->mvf32, ne * 6 * 7 * N2}, {&m->rvis32, 7 * ne * N3}};
  for (const Buf& b : bufs)
    if (!*b.p) {
      err = cudaMalloc((void**)b.p, b.count * sizeof(float));
      if (err != cudaSuccess) return err;
      m->device_bytes += (int64_t)(b.count * sizeof(float));
    }
  if (!bg || !bg->vrec || !bg->vtr) return cudaErrorInvalidValue;
  // both kernels read the background's viscous record: the gradient kernel its face
  // traces (grad T0, grad S0 at this side's face points), the residual kernel all of it
  sd::StageParams Pg = P;
  Pg.bg_visc = bg->vrec;
  Pg.bg_vtr = bg->vtr;
  sd::StageParams Pv = Pg;
  Pg.mgrad_out = m->grad32;
  Pg.mvf_out = m->mvf32;
  Pv.mgrad = m->grad32;
  Pv.mvf_in = m->mvf32;
  Pv.rvis_out = m->rvis32;
  {
    ProfScope ps(m, PROF_OTHER, s);
    err = sd::launch_mixed_visc(m, Pg, Pv, s);
  }
  P.rvis = m->rvis32;
  return err;
}

// Viscous FP64 path: the BR1 gradient record of P.q_in (whose face traces are
// P.tr_in): its face traces and the interior viscous divergence into the mesh's
// buffers (allocated on first use), the record itself too when `record` (the
// background's viscous record); P then points the face-flux and element kernels at
// them.  The FP32-mixed path goes through prepare_viscous_mixed.  No-op without
// viscous fluxes.
cudaError_t prepare_viscous(sd_mesh* m, sd::StageParams& P, cudaStream_t s, int prec = SD_FP64,
                            const sd_background* bg = nullptr, bool record = false) {
  if (!P.visc) return cudaSuccess;
  if (prec == SD_FP32_MIXED) return prepare_viscous_mixed(m, P, bg, s);
  const size_t N2 = (size_t)m->N * m->N, N3 = N2 * m->N, ne = (size_t)std::max<int64_t>(m->n_e, 1);
  cudaError_t err = cudaSuccess;
  struct Buf {
    double** p;
    size_t count;
    bool want;
  } bufs[3] = {{&m->grad, ne * sd::MV_REC * N3, record},
               {&m->gtr, ne * 6 * sd::MV_REC * N2, true},
               {&m->rvis64, ne * 7 * N3, true}};
  for (const Buf& b : bufs)
    if (b.want && !*b.p) {
      err = cudaMalloc((void**)b.p, b.count * sizeof(double));
      if (err != cudaSuccess) return err;
      m->device_bytes += (int64_t)(b.count * sizeof(double));
    }
  sd::StageParams G = P;
  G.grad_out = record ? m->grad : nullptr;
  G.gtr_out = m->gtr;
  G.rvis64_out = m->rvis64;
  {
    ProfScope ps(m, PROF_OTHER, s);
    err = sd::launch_grad(m, G, s);
  }
  P.gtr_in = m->gtr;
  P.rvis64 = m->rvis64;
  return err;
}

sd_status check_common(const sd_mesh* m, const sd_phys* ph, int prec, const sd_background* bg) {
  if (!m) return fail(SD_ERR_INVALID_ARGUMENT, "mesh is NULL");
  if (!ph) return fail(SD_ERR_INVALID_ARGUMENT, "phys is NULL");
  if (prec != SD_FP64 && prec != SD_FP32_MIXED) return fail(SD_ERR_INVALID_ARGUMENT, "unknown precision");
  if (ph->rk_scheme != SD_RK_SSP33 && ph->rk_scheme != SD_RK_SSP53)
    return fail(SD_ERR_INVALID_ARGUMENT, "rk_scheme must be SD_RK_SSP33 or SD_RK_SSP53");
  if (!(ph->visc_cfl >= 0.0) || !isfinite(ph->visc_cfl))
    return fail(SD_ERR_INVALID_ARGUMENT, "visc_cfl must be finite and not negative");
  if (!(ph->gamma > 1.0)) return fail(SD_ERR_INVALID_ARGUMENT, "gamma must exceed 1");
  if (ph->viscous) {
    if (prec == SD_FP32_MIXED) {
      if (!bg || bg->visc_coef[7] != 1.0)
        return fail(SD_ERR_INVALID_ARGUMENT, "viscous fluxes on the FP32-mixed path need a background built with them");
      const double want[7] = {ph->mu, ph->eta, ph->kappa, ph->kappa_r, ph->kappa_r1, ph->kappa_r2, ph->R_gas};
      for (int i = 0; i < 7; ++i)
        if (bg->visc_coef[i] != want[i])
          return fail(SD_ERR_INVALID_ARGUMENT, "background was built with other viscous coefficients");
      if (ph->visc_walls)
        return fail(SD_ERR_UNSUPPORTED, "the wall conditions of the viscous path (visc_walls) run on SD_FP64 only");
      if (m->has_farfield)
        return fail(SD_ERR_UNSUPPORTED, "viscous fluxes on the FP32-mixed path take no far-field faces");
    }
    if (!(ph->mu >= 0.0) || !(ph->eta >= 0.0) || !(ph->kappa >= 0.0) || !(ph->kappa_r >= 0.0) ||
        !isfinite(ph->mu + ph->eta + ph->kappa + ph->kappa_r) || !isfinite(ph->kappa_r1) || !isfinite(ph->kappa_r2))
      return fail(SD_ERR_INVALID_ARGUMENT, "viscous coefficients must be finite and non-negative");
    if (!(ph->R_gas > 0.0) || !isfinite(ph->R_gas)) return fail(SD_ERR_INVALID_ARGUMENT, "R_gas must be positive");
    if (ph->visc_walls && (!(ph->T_top > 0.0) || !isfinite(ph->T_top) || !isfinite(ph->q_bottom)))
      return fail(SD_ERR_INVALID_ARGUMENT, "viscous walls need T_top > 0 and a finite q_bottom");
  }
  if (prec == SD_FP32_MIXED) {
    if (!bg) return fail(SD_ERR_INVALID_ARGUMENT, "the FP32-mixed path needs a background (sd_background_create)");
    if (bg->mesh != m) return fail(SD_ERR_INVALID_ARGUMENT, "background belongs to another mesh");
    if (bg->gamma != ph->gamma) return fail(SD_ERR_INVALID_ARGUMENT, "background was built with another gamma");
  }
  return SD_OK;
}

// polytrope pressure at radius r (Sec. Initial Conditions), for the dipole scaling
double polytrope_p(double r, double Nr, double rb, double rt, double rhob, double Rg, double g, double GM) {
  const double Cp = g * Rg / (g - 1.0);
  const double Tb = (GM / rb - GM / rt) / (Cp * (1.0 - exp(-(g - 1.0) * Nr)));
  const double zeta = 1.0 - (GM / rb - GM / r) / (Cp * Tb);
  return rhob * Rg * Tb * pow(zeta, g / (g - 1.0));
}

// Almost flux-balanced shell profile (Sec. Initial Conditions): S and rho on
// n + 1 uniform nodes over [r_b, r_t] with their derivatives, integrated by
// classical RK4 from the polytrope's bottom state.  P = (N_rho, r_b, r_t, rho_b,
// R, noise, dipole, L, kappa, kappa_r, kappa_r1, kappa_r2), the radiative
// diffusivity kappa_r(r) = kappa_r + kappa_r1 r + kappa_r2 r^2.
constexpr int kFluxNodes = 4096;

struct FluxProfile {
  int n = 0;
  double rb = 0.0, h = 1.0, Cp = 1.0, gamma = 1.0;
  std::vector<double> tab;  // [4][n + 1]: rho, S, drho/dr, dS/dr
};

FluxProfile flux_profile(const double* P, double gamma, double GM, int n) {
  const double Nr = P[0], rb = P[1], rt = P[2], rhob = P[3], Rg = P[4], L = P[7], kap = P[8];
  const double kr0 = P[9], kr1 = P[10], kr2 = P[11];
  FluxProfile F;
  F.n = n;
  F.rb = rb;
  F.h = (rt - rb) / n;
  F.gamma = gamma;
  F.Cp = gamma * Rg / (gamma - 1.0);
  const double Cp = F.Cp;
  const double Tb = (GM / rb - GM / rt) / (Cp * (1.0 - exp(-(gamma - 1.0) * Nr)));
  // polytrope rho_p, T_p and dT_p/dr at radius r
  auto poly = [&](double r, double& rp, double& Tp, double& dTp) {
    const double z = 1.0 - (GM / rb - GM / r) / (Cp * Tb);
    rp = rhob * pow(z, 1.0 / (gamma - 1.0));
    Tp = Tb * z;
    dTp = -GM / (Cp * r * r);
  };
  auto dS = [&](double r) {
    double rp, Tp, dTp;
    poly(r, rp, Tp, dTp);
    const double kapr = kr0 + kr1 * r + kr2 * r * r;
    return (L / (4.0 * M_PI * r * r) + kapr * rp * Cp * dTp) / (kap * rp * Tp);
  };
  auto drho = [&](double r, double rho, double S, double Sp) {
    return -(rho * Sp / Cp + GM / (r * r) / gamma * pow(rho, 2.0 - gamma) * exp(-gamma * S / Cp));
  };
  F.tab.assign(4 * (size_t)(n + 1), 0.0);
  double* T_rho = F.tab.data();
  double* T_S = T_rho + (n + 1);
  double* T_drho = T_S + (n + 1);
  double* T_dS = T_drho + (n + 1);
  const double pb = rhob * Rg * Tb;
  double rho = rhob, S = Cp * (log(pb) / gamma - log(rhob));
  const double h = F.h;
  for (int k = 0; k <= n; ++k) {
    const double r = rb + k * h;
    const double s1 = dS(r), q1 = drho(r, rho, S, s1);
    T_rho[k] = rho;
    T_S[k] = S;
    T_drho[k] = q1;
    T_dS[k] = s1;
    if (k == n) break;
    const double s2 = dS(r + 0.5 * h);
    const double q2 = drho(r + 0.5 * h, rho + 0.5 * h * q1, S + 0.5 * h * s1, s2);
    const double q3 = drho(r + 0.5 * h, rho + 0.5 * h * q2, S + 0.5 * h * s2, s2);
    const double s4 = dS(r + h);
    const double q4 = drho(r + h, rho + h * q3, S + h * s2, s4);
    rho += h * (q1 + 2.0 * q2 + 2.0 * q3 + q4) / 6.0;
    S += h * (s1 + 4.0 * s2 + s4) / 6.0;
  }
  return F;
}

// pressure of the profile at r (the device kernel interpolates the same way)
double flux_profile_p(const FluxProfile& F, double r) {
  double u = (r - F.rb) / F.h;
  int k = (int)floor(u);
  k = k < 0 ? 0 : (k >= F.n ? F.n - 1 : k);
  const double t = u - k, h = F.h;
  const double* T = F.tab.data();
  const int n1 = F.n + 1;
  const double a = (1 + 2 * t) * (1 - t) * (1 - t), b = t * (1 - t) * (1 - t), c = t * t * (3 - 2 * t),
               d = t * t * (t - 1);
  const double rho = a * T[k] + b * h * T[2 * n1 + k] + c * T[k + 1] + d * h * T[2 * n1 + k + 1];
  const double S = a * T[n1 + k] + b * h * T[3 * n1 + k] + c * T[n1 + k + 1] + d * h * T[3 * n1 + k + 1];
  return pow(rho * exp(S / F.Cp), F.gamma);
}

}  // namespace

namespace sd {
// message for sd_last_error() from entry points defined in other translation units
void set_last_error(const std::string& msg) { g_err = msg; }
}  // namespace sd

extern "C" {

const char* sd_last_error(void) { return g_err.c_str(); }

sd_status sd_mesh_create(const sd_mesh_desc* desc, void* stream, sd_mesh** out) {
  if (!out) return fail(SD_ERR_INVALID_ARGUMENT, "out is NULL");
  *out = nullptr;
  if (!desc) return fail(SD_ERR_INVALID_ARGUMENT, "desc is NULL");
  const int N = desc->order;
  if (N < 2 || N > sd::kMaxN) return fail(SD_ERR_UNSUPPORTED, "order N must be in [2, 8]");
  if (desc->n_elements < 0 || desc->n_vertices < 0) return fail(SD_ERR_INVALID_ARGUMENT, "negative size");
  if (desc->n_elements == 0) return fail(SD_ERR_INVALID_ARGUMENT, "a mesh needs at least one element");
  if (!desc->hex || !desc->vertices) return fail(SD_ERR_INVALID_ARGUMENT, "vertices or hex is NULL");
  if (desc->geom != 0 && desc->geom != 1) return fail(SD_ERR_INVALID_ARGUMENT, "geom must be 0 or 1");
  if (desc->n_elements > (int64_t)1 << 30) return fail(SD_ERR_INVALID_ARGUMENT, "too many elements");
  const int bcs[2] = {desc->bc_inner, desc->bc_outer};
  for (int b : bcs)
    if (b < SD_BC_PERIODIC || b > SD_BC_FARFIELD) return fail(SD_ERR_INVALID_ARGUMENT, "unknown boundary condition");
  const int64_t n_e = desc->n_elements, n_v = desc->n_vertices;
  const int64_t* hex = desc->hex;
  for (int64_t i = 0; i < 8 * n_e; ++i)
    if (hex[i] < 0 || hex[i] >= n_v) return fail(SD_ERR_INVALID_ARGUMENT, "vertex index out of range");
  double per[3] = {0.0, 0.0, 0.0};
  if (desc->periodic_lengths)
    for (int d = 0; d < 3; ++d) per[d] = desc->periodic_lengths[d] > 0.0 ? desc->periodic_lengths[d] : 0.0;

  // ---- corners, unwrapped across periodic directions relative to corner 0
  std::vector<double> corners((size_t)n_e * 24);
  for (int64_t e = 0; e < n_e; ++e) {
    const double* v0 = desc->vertices + 3 * hex[8 * e];
    for (int c = 0; c < 8; ++c) {
      const double* v = desc->vertices + 3 * hex[8 * e + c];
      for (int d = 0; d < 3; ++d) {
        double x = v[d];
        if (per[d] > 0.0) x += per[d] * std::nearbyint((v0[d] - v[d]) / per[d]);
        corners[e * 24 + 3 * c + d] = x;
      }
    }
    for (int c = 0; c < 8; ++c)
      for (int c2 = c + 1; c2 < 8; ++c2)
        if (hex[8 * e + c] == hex[8 * e + c2]) return fail(SD_ERR_MESH_TOPOLOGY, "element with repeated corners");
  }

  // ---- face matching: sort the 6 n_e faces by their sorted corner ids
  struct FaceKey {
    std::array<int64_t, 4> k;
    int64_t e;
    int F;
  };
  std::vector<FaceKey> faces((size_t)n_e * 6);
  for (int64_t e = 0; e < n_e; ++e)
    for (int F = 0; F < 6; ++F) {
      FaceKey& fk = faces[e * 6 + F];
      for (int s = 0; s < 2; ++s)
        for (int t = 0; t < 2; ++t) fk.k[2 * s + t] = hex[8 * e + face_corner(F, s, t)];
      std::sort(fk.k.begin(), fk.k.end());
      fk.e = e;
      fk.F = F;
    }
  std::sort(faces.begin(), faces.end(), [](const FaceKey& a, const FaceKey& b) {
    if (a.k != b.k) return a.k < b.k;
    if (a.e != b.e) return a.e < b.e;
    return a.F < b.F;
  });
  std::vector<int> nbr((size_t)n_e * 6, -1), meta((size_t)n_e * 6, 0);
  int64_t n_bf = 0, n_if = 0;
  bool has_ff = false;
  for (size_t i = 0; i < faces.size();) {
    size_t j = i + 1;
    while (j < faces.size() && faces[j].k == faces[i].k) ++j;
    if (j - i > 2) return fail(SD_ERR_MESH_TOPOLOGY, "a face is shared by more than two elements");
    if (j - i == 2) {
      const FaceKey& A = faces[i];
      const FaceKey& B = faces[i + 1];
      const int cab = orientation(hex, A.e, A.F, B.e, B.F), cba = orientation(hex, B.e, B.F, A.e, A.F);
      if (cab < 0 || cba < 0) return fail(SD_ERR_MESH_TOPOLOGY, "matched faces with inconsistent corners");
      nbr[A.e * 6 + A.F] = (int)B.e;
      nbr[B.e * 6 + B.F] = (int)A.e;
      meta[A.e * 6 + A.F] = B.F | (cab << 3) | (1 << 9);
      meta[B.e * 6 + B.F] = A.F | (cba << 3);
      ++n_if;
    } else {
      const FaceKey& A = faces[i];
      int bc = desc->bc_inner, outer = 0;
      if (desc->geom == 1) {
        double c[3] = {0, 0, 0};
        for (int s = 0; s < 2; ++s)
          for (int t = 0; t < 2; ++t) {
            const int cc = face_corner(A.F, s, t);
            for (int d = 0; d < 3; ++d) c[d] += 0.25 * corners[A.e * 24 + 3 * cc + d];
          }
        const double rc = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
        bc = rc < 0.5 * (desc->r_inner + desc->r_outer) ? desc->bc_inner : desc->bc_outer;
        outer = rc < 0.5 * (desc->r_inner + desc->r_outer) ? 0 : 1;
      }
      if (bc == SD_BC_PERIODIC) return fail(SD_ERR_MESH_TOPOLOGY, "unmatched face under a periodic boundary");
      if (bc == SD_BC_FARFIELD) has_ff = true;
      meta[A.e * 6 + A.F] = (bc << 6) | (outer << 10);
      ++n_bf;
    }
    i = j;
  }

  // ---- smallest edge chord
  static const int edges[12][2] = {{0, 1}, {2, 3}, {4, 5}, {6, 7}, {0, 2}, {1, 3},
                                   {4, 6}, {5, 7}, {0, 4}, {1, 5}, {2, 6}, {3, 7}};
  double hmin = INFINITY;
  for (int64_t e = 0; e < n_e; ++e)
    for (int k = 0; k < 12; ++k) {
      const double* a = &corners[e * 24 + 3 * edges[k][0]];
      const double* b = &corners[e * 24 + 3 * edges[k][1]];
      const double l = sqrt((a[0] - b[0]) * (a[0] - b[0]) + (a[1] - b[1]) * (a[1] - b[1]) + (a[2] - b[2]) * (a[2] - b[2]));
      hmin = std::min(hmin, l);
    }

  // ---- device objects
  take_stale();
  sd_mesh* m = new sd_mesh();
  if (cudaGetDevice(&m->device) != cudaSuccess) {
    delete m;
    return fail(SD_ERR_CUDA, "no CUDA device");
  }
  m->N = N;
  m->p = N / 2;
  m->n_e = n_e;
  m->stride = round_stride(N);
  m->n_bf = n_bf;
  m->n_if = n_if;
  m->h_min = hmin;
  m->geom = desc->geom;
  m->has_farfield = has_ff ? 1 : 0;
  m->wait_spins = sd::kWaitSpins;
  build_ops(N, m->ops64);
  ops_to_f32(m->ops64, m->ops32);
  ops_to_pairs(N, m->ops32, m->ops2);
  const int64_t N2 = (int64_t)N * N, N3 = N2 * N, NF = N + 1;
  const size_t ne = (size_t)std::max<int64_t>(n_e, 1);
  int64_t bytes = 0;
  // faces owned by an element (the first of a matched pair, or a boundary face): the FP64
  // face-flux kernel computes each of them once, for both sides
  std::vector<int> own_faces, face_k((size_t)n_e * 6, -1);
  for (int64_t e = 0; e < n_e; ++e)
    for (int F = 0; F < 6; ++F)
      if (nbr[e * 6 + F] < 0 || sd::meta_owner(meta[e * 6 + F])) {
        face_k[e * 6 + F] = (int)own_faces.size();
        own_faces.push_back((int)(e * 6 + F));
      }
  for (int64_t e = 0; e < n_e; ++e)
    for (int F = 0; F < 6; ++F)
      if (face_k[e * 6 + F] < 0) face_k[e * 6 + F] = face_k[(int64_t)nbr[e * 6 + F] * 6 + sd::meta_nbF(meta[e * 6 + F])];
  m->n_own = (int64_t)own_faces.size();
  cudaError_t err = cudaSuccess;
#define ALLOC(ptr, cnt)                                   \
  if (err == cudaSuccess) err = dalloc(&(ptr), (cnt), &bytes);
  ALLOC(m->own_faces, (size_t)m->n_own);
  ALLOC(m->face_k, ne * 6);
  ALLOC(m->gface64, (size_t)m->n_own * 10 * N2);
  ALLOC(m->Sfam64, ne * 9 * N2 * NF);
  ALLOC(m->invJ64, ne * N3);
  ALLOC(m->X64, ne * 3 * N3);
  ALLOC(m->Sfam32, ne * 9 * N2 * NF);
  ALLOC(m->invJ32, ne * N3);
  ALLOC(m->X32, ne * 3 * N3);
  ALLOC(m->nbr, ne * 6);
  ALLOC(m->meta, ne * 6);
  ALLOC(m->tr64[0], ne * 6 * 9 * N2);
  ALLOC(m->tr64[1], ne * 6 * 9 * N2);
  ALLOC(m->tr32[0], ne * 6 * 9 * N2);
  ALLOC(m->tr32[1], ne * 6 * 9 * N2);
  ALLOC(m->dyn, 5 + sd::LAM_SLOTS);  // dt, c_h, lambda, rho_min | lambda slots | gamma kappa_r max
  ALLOC(m->diag_part, ne * 12);
  ALLOC(m->diag_out, 12);
  ALLOC(m->divb, ne * N3);
  ALLOC(m->err, 4);
#undef ALLOC
  if (err == cudaSuccess) err = cudaMallocHost((void**)&m->host_diag, 12 * sizeof(double));
  m->device_bytes = bytes;
  if (err != cudaSuccess) {
    free_mesh(m);
    cudaGetLastError();
    return fail(err == cudaErrorMemoryAllocation ? SD_ERR_OUT_OF_MEMORY : SD_ERR_CUDA,
                std::string("allocation failed: ") + cudaGetErrorString(err));
  }
  cudaStream_t s = (cudaStream_t)stream;
  double* d_corners = nullptr;
  int* d_flag = nullptr;
  int h_flag = 0;
  auto cleanup = [&]() {
    if (d_corners) cudaFree(d_corners);
    if (d_flag) cudaFree(d_flag);
  };
  err = cudaMalloc((void**)&d_corners, ne * 24 * sizeof(double));
  if (err == cudaSuccess) err = cudaMalloc((void**)&d_flag, sizeof(int));
  if (err == cudaSuccess && n_e > 0)
    err = cudaMemcpyAsync(d_corners, corners.data(), n_e * 24 * sizeof(double), cudaMemcpyHostToDevice, s);
  if (err == cudaSuccess && n_e > 0)
    err = cudaMemcpyAsync(m->nbr, nbr.data(), n_e * 6 * sizeof(int), cudaMemcpyHostToDevice, s);
  if (err == cudaSuccess && n_e > 0)
    err = cudaMemcpyAsync(m->meta, meta.data(), n_e * 6 * sizeof(int), cudaMemcpyHostToDevice, s);
  if (err == cudaSuccess && n_e > 0)
    err = cudaMemcpyAsync(m->face_k, face_k.data(), n_e * 6 * sizeof(int), cudaMemcpyHostToDevice, s);
  if (err == cudaSuccess && m->n_own > 0)
    err = cudaMemcpyAsync(m->own_faces, own_faces.data(), m->n_own * sizeof(int), cudaMemcpyHostToDevice, s);
  if (err == cudaSuccess) err = cudaMemsetAsync(d_flag, 0, sizeof(int), s);
  if (err == cudaSuccess) err = cudaMemsetAsync(m->err, 0, sizeof(int), s);
  if (err == cudaSuccess) err = sd::launch_geometry(m, d_corners, d_flag, s);
  if (err == cudaSuccess) err = sd::launch_canonical_faces(m, s);
  if (err == cudaSuccess) err = cudaMemcpyAsync(&h_flag, d_flag, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  cleanup();
  if (err != cudaSuccess) {
    free_mesh(m);
    return cuda_fail(err, "mesh geometry");
  }
  if (h_flag) {
    free_mesh(m);
    return fail(SD_ERR_MESH_GEOMETRY, "non-positive Jacobian in the element map (left-handed or degenerate element)");
  }
  *out = m;
  return SD_OK;
}

sd_status sd_mesh_destroy(sd_mesh* m) {
  if (!m) return SD_OK;
  DeviceGuard g(m->device);
  free_mesh(m);
  return SD_OK;
}

sd_status sd_mesh_query(const sd_mesh* m, sd_mesh_info* out) {
  if (!m || !out) return fail(SD_ERR_INVALID_ARGUMENT, "null argument");
  out->order = m->N;
  out->p_map = m->p;
  out->n_elements = m->n_e;
  out->n_points = m->n_e * m->N * m->N * m->N;
  out->elem_stride = m->stride;
  out->state_bytes = 9 * m->n_e * m->stride * (int64_t)sizeof(double);
  out->n_boundary_faces = m->n_bf;
  out->n_interior_faces = m->n_if;
  out->h_min = m->h_min;
  out->device_bytes = m->device_bytes;
  // three FP32 trace buffers (the packed step's stage cycle) and 16 partial maxima of lambda
  out->trace_bytes = 3 * m->n_e * 6 * 9 * (int64_t)m->N * m->N * (int64_t)sizeof(float) + 16 * 8;
  return SD_OK;
}

sd_status sd_state_init(const sd_mesh* m, const sd_phys* ph, const sd_init* in, double* q, double* qbg, void* stream) {
  if (!m || !ph || !in) return fail(SD_ERR_INVALID_ARGUMENT, "null argument");
  sd_status st = check_state_ptr(q, "q");
  if (st != SD_OK) return st;
  if (qbg && (((uintptr_t)qbg & 15) != 0)) return fail(SD_ERR_INVALID_ARGUMENT, "q_background is not 16-byte aligned");
  if (in->kind < SD_INIT_UNIFORM || in->kind > SD_INIT_SHELL_FLUX_BALANCED)
    return fail(SD_ERR_INVALID_ARGUMENT, "unknown init kind");
  if (!(ph->gamma > 1.0)) return fail(SD_ERR_INVALID_ARGUMENT, "gamma must exceed 1");
  DeviceGuard g(m->device);
  double B0 = 0.0;
  const bool fluxbal = in->kind == SD_INIT_SHELL_FLUX_BALANCED;
  FluxProfile F;
  if (in->kind == SD_INIT_SHELL_POLYTROPE || fluxbal) {
    const double* P = in->params;
    const double Nr = P[0], rb = P[1], rt = P[2], rhob = P[3], Rg = P[4], ratio = P[6];
    if (!(rt > rb && rb > 0.0 && rhob > 0.0 && Rg > 0.0 && ph->GM > 0.0))
      return fail(SD_ERR_INVALID_ARGUMENT, "polytrope needs 0 < r_b < r_t, rho_b > 0, R_gas > 0, GM > 0");
    if (fluxbal) {
      if (!(P[8] > 0.0) || !(P[9] >= 0.0) || !isfinite(P[7]))
        return fail(SD_ERR_INVALID_ARGUMENT, "flux-balanced profile needs kappa > 0, kappa_r >= 0, finite L");
      F = flux_profile(P, ph->gamma, ph->GM, kFluxNodes);
      for (int k = 0; k <= F.n; ++k)  // rho and S at every node
        if (!(F.tab[k] > 0.0) || !isfinite(F.tab[k]) || !isfinite(F.tab[F.n + 1 + k]))
          return fail(SD_ERR_INVALID_ARGUMENT,
                      "the flux-balanced profile does not stay positive and finite with these parameters");
    }
    // magnetic energy of the unit dipole over the ideal shell: 8 pi (r_b^-3 - r_t^-3) / 3 (times 1/2 below);
    // internal energy: 4 pi / (gamma - 1) int p0 r^2 dr by 64-point Gauss-Legendre
    std::vector<double> x, w;
    gauss_legendre(64, x, w);
    double Ip = 0.0;
    for (int k = 0; k < 64; ++k) {
      const double r = 0.5 * (rb + rt) + 0.5 * (rt - rb) * x[k];
      const double p0 = fluxbal ? flux_profile_p(F, r) : polytrope_p(r, Nr, rb, rt, rhob, Rg, ph->gamma, ph->GM);
      Ip += 0.5 * (rt - rb) * w[k] * p0 * r * r;
    }
    Ip *= 4.0 * M_PI / (ph->gamma - 1.0);
    const double IB = 8.0 * M_PI * (1.0 / (rb * rb * rb) - 1.0 / (rt * rt * rt)) / 3.0;
    B0 = sqrt(2.0 * ratio * Ip / IB);
  }
  // the flux-balanced profile's table goes to the device for the duration of the kernel
  double* dtab = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  if (fluxbal) {
    const size_t bytes = F.tab.size() * sizeof(double);
    cudaError_t e1 = cudaMallocAsync((void**)&dtab, bytes, s);
    if (e1 == cudaSuccess) e1 = cudaMemcpyAsync(dtab, F.tab.data(), bytes, cudaMemcpyHostToDevice, s);
    if (e1 != cudaSuccess) return cuda_fail(e1, "flux-balanced profile table");
  }
  const sd::ProfileTable tab{dtab, F.n, F.rb, F.h, F.Cp};
  cudaError_t err = sd::launch_state_init(m, ph, in, B0, tab, q, qbg, s);
  if (dtab) cudaFreeAsync(dtab, s);
  if (err != cudaSuccess) return cuda_fail(err, "state init kernel");
  return SD_OK;
}

sd_status sd_background_create(const sd_mesh* m, const sd_phys* ph, const double* q_bg, void* stream,
                               sd_background** out) {
  if (!out) return fail(SD_ERR_INVALID_ARGUMENT, "out is NULL");
  *out = nullptr;
  sd_status st = check_common(m, ph, SD_FP64, nullptr);
  if (st != SD_OK) return st;
  st = check_state_ptr(q_bg, "q_background");
  if (st != SD_OK) return st;
  DeviceGuard g(m->device);
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t N2 = (int64_t)m->N * m->N, N3 = N2 * m->N;
  const size_t ne = (size_t)std::max<int64_t>(m->n_e, 1);
  sd_background* bg = new sd_background;
  bg->mesh = m;
  bg->gamma = ph->gamma;
  bg->rec = nullptr;
  bg->jump = nullptr;
  bg->dreg = nullptr;
  bg->qp = nullptr;
  bg->dstride = (N3 + 3) / 4 * 4;
  bg->device = m->device;
  bg->vrec = nullptr;
  bg->vtr = nullptr;
  for (int i = 0; i < 8; ++i) bg->visc_coef[i] = 0.0;
  const bool visc = ph->viscous != 0;
  if (visc && ph->visc_walls) {
    delete bg;
    return fail(SD_ERR_UNSUPPORTED, "the wall conditions of the viscous path (visc_walls) run on SD_FP64 only");
  }
  if (visc && m->has_farfield) {
    delete bg;
    return fail(SD_ERR_UNSUPPORTED, "viscous fluxes on the FP32-mixed path take no far-field faces");
  }
  double *q0 = nullptr, *R0 = nullptr, *R0v = nullptr;
  const size_t state = 9 * ne * m->stride;
  // stream-ordered allocations: building a background never waits for the device
  cudaError_t err = cudaMallocAsync((void**)&bg->rec, 5 * ne * N3 * sizeof(float), s);
  if (err == cudaSuccess) err = cudaMallocAsync((void**)&bg->jump, ne * 6 * 2 * N2 * sizeof(float), s);
  // D and q' of the mixed step: 18 planes of n_e * dstride floats
  if (err == cudaSuccess) err = cudaMallocAsync((void**)&bg->dreg, 18 * ne * bg->dstride * sizeof(float), s);
  if (err == cudaSuccess) bg->qp = bg->dreg + 9 * ne * bg->dstride;
  if (err == cudaSuccess) err = cudaMallocAsync((void**)&q0, state * sizeof(double), s);
  if (err == cudaSuccess) err = cudaMallocAsync((void**)&R0, state * sizeof(double), s);
  if (err == cudaSuccess) err = sd::launch_bg_prepare(m, ph->gamma, 1.0 / (ph->gamma - 1.0), q_bg, q0, bg->rec, s);
  sd_mesh* mm = const_cast<sd_mesh*>(m);
  if (err == cudaSuccess) {
    sd::StageParams P = base_params(m, ph, SD_FP64);
    P.q_in = q0;
    P.tr_out = mm->tr64[0];
    err = sd::launch_traces(m, SD_FP64, P, s);
    if (err == cudaSuccess) {
      // background residual: pressure-gradient flux with central face average, plus rho0 g.  A
      // far-field face takes the element's own background as its ghost: the mixed stages carry the
      // far field as the perturbation Q_ff - Q0 about that same background, so the two parts add
      // up to the full flux there.
      P.tr_out = nullptr;
      P.tr_in = mm->tr64[0];
      P.mode = sd::MODE_RESIDUAL;
      P.central = 1;
      P.ff_own = 1;
      P.c_h = 0.0;
      P.powell = 0;
      P.coriolis = 0;
      P.alpha = 0.0;
      P.out = R0;
      err = sd::launch_stage(m, SD_FP64, P, s);
    }
  }
  if (err == cudaSuccess && visc) {
    // the background's viscous residual (its residual with the viscous fluxes less the one above,
    // both FP64: only the heat flux of Q0 is left, in the energy component), grad T0 and grad S0
    err = cudaMallocAsync((void**)&bg->vrec, 7 * ne * N3 * sizeof(float), s);
    if (err == cudaSuccess) err = cudaMallocAsync((void**)&bg->vtr, ne * 6 * 6 * N2 * sizeof(float), s);
    if (err == cudaSuccess) err = cudaMallocAsync((void**)&R0v, state * sizeof(double), s);
    if (err == cudaSuccess) {
      sd::StageParams P = base_params(m, ph, SD_FP64);
      P.q_in = q0;
      P.tr_in = mm->tr64[0];
      P.mode = sd::MODE_RESIDUAL;
      P.central = 1;
      P.ff_own = 1;
      P.c_h = 0.0;
      P.powell = 0;
      P.coriolis = 0;
      P.alpha = 0.0;
      P.out = R0v;
      err = prepare_viscous(mm, P, s, SD_FP64, nullptr, true);  // FP64 BR1 record of Q0 into the mesh's buffers
      if (err == cudaSuccess) err = sd::launch_stage(m, SD_FP64, P, s);
      if (err == cudaSuccess) err = sd::launch_bg_visc(m, R0, R0v, mm->grad, mm->gtr, bg->vrec, bg->vtr, s);
    }
    const double coef[8] = {ph->mu, ph->eta, ph->kappa, ph->kappa_r, ph->kappa_r1, ph->kappa_r2, ph->R_gas, 1.0};
    for (int i = 0; i < 8; ++i) bg->visc_coef[i] = coef[i];
  }
  if (err == cudaSuccess) err = sd::launch_bg_finish(m, ph->gamma, R0, bg->rec, bg->jump, mm->tr64[0], s);
  mm->tr_tag[0] = mm->tr_tag[1] = nullptr;
  if (q0) cudaFreeAsync(q0, s);
  if (R0) cudaFreeAsync(R0, s);
  if (R0v) cudaFreeAsync(R0v, s);
  if (err != cudaSuccess) {
    if (bg->rec) cudaFreeAsync(bg->rec, s);
    if (bg->jump) cudaFreeAsync(bg->jump, s);
    if (bg->dreg) cudaFreeAsync(bg->dreg, s);
    if (bg->vrec) cudaFreeAsync(bg->vrec, s);
    if (bg->vtr) cudaFreeAsync(bg->vtr, s);
    delete bg;
    cudaGetLastError();
    return err == cudaErrorMemoryAllocation ? fail(SD_ERR_OUT_OF_MEMORY, "background allocation failed")
                                            : cuda_fail(err, "background preparation");
  }
  *out = bg;
  return SD_OK;
}

sd_status sd_background_destroy(sd_background* bg) {
  if (!bg) return SD_OK;
  DeviceGuard g(bg->device);
  // stream-ordered on the legacy default stream: after all work already issued
  // to it and to the blocking streams
  cudaFreeAsync(bg->rec, 0);
  cudaFreeAsync(bg->jump, 0);
  cudaFreeAsync(bg->dreg, 0);
  if (bg->vrec) cudaFreeAsync(bg->vrec, 0);
  if (bg->vtr) cudaFreeAsync(bg->vtr, 0);
  delete bg;
  return SD_OK;
}

sd_status sd_residual(const sd_mesh* m, const sd_phys* ph, sd_precision prec, const double* q, const sd_background* bg,
                      double* dqdt, void* stream) {
  sd_status st = check_common(m, ph, prec, bg);
  if (st != SD_OK) return st;
  if ((st = check_state_ptr(q, "q")) != SD_OK) return st;
  if ((st = check_state_ptr(dqdt, "dqdt")) != SD_OK) return st;
  if (q == dqdt) return fail(SD_ERR_INVALID_ARGUMENT, "dqdt must not alias q");
  DeviceGuard g(m->device);
  sd_mesh* mm = const_cast<sd_mesh*>(m);
  cudaStream_t s = (cudaStream_t)stream;
  sd::StageParams P = base_params(m, ph, prec);
  if (bg) {
    P.bg = bg->rec;
    P.bg_jump = bg->jump;
  }
  P.q_in = q;
  P.tr_out = trace_buf(mm, prec, 0);
  cudaError_t err;
  {
    ProfScope ps(m, PROF_TRACE, s);
    err = sd::launch_traces(m, prec, P, s);
  }
  if (err != cudaSuccess) return cuda_fail(err, "trace kernel");
  mm->tr_tag[0] = mm->tr_tag[1] = nullptr;
  P.tr_in = P.tr_out;
  P.tr_out = nullptr;
  P.mode = sd::MODE_RESIDUAL;
  P.out = dqdt;
  if ((err = prepare_viscous(mm, P, s, prec, bg)) != cudaSuccess) return cuda_fail(err, "gradient kernel");
  {
    ProfScope ps(m, PROF_STAGE, s);
    err = sd::launch_stage(m, prec, P, s);
  }
  if (err != cudaSuccess) return cuda_fail(err, "residual kernel");
  return SD_OK;
}

static sd_status rk_stage_impl(sd_mesh* m, const sd_phys* ph, int prec, int stage, double dt, const double* dyn,
                               const double* q_n, const double* q_in, double* q_out, const sd_background* bg,
                               bool want_traces, cudaStream_t s, int lsr_read = 0, int lsr_write = 0) {
  static const double A[3] = {0.0, 0.75, 1.0 / 3.0};
  static const double B[3] = {1.0, 0.25, 2.0 / 3.0};
  sd::StageParams P = base_params(m, ph, prec);
  if (bg) {
    P.bg = bg->rec;
    P.bg_jump = bg->jump;
  }
  // traces of q_in: reuse those written by the previous stage when it produced q_in
  int bin = -1;
  if (stage > 0)
    for (int b = 0; b < 2; ++b)
      if (m->tr_tag[b] == q_in && m->tr_prec[b] == prec) bin = b;
  if (bin < 0) {
    bin = 0;
    P.q_in = q_in;
    P.tr_out = trace_buf(m, prec, bin);
    cudaError_t err;
    {
      ProfScope ps(m, PROF_TRACE, s);
      err = sd::launch_traces(m, prec, P, s);
    }
    if (err != cudaSuccess) return cuda_fail(err, "trace kernel");
  }
  const int bout = 1 - bin;
  P.q_in = q_in;
  P.q_n = q_n;
  P.out = q_out;
  P.mode = sd::MODE_RK;
  P.rk_a = A[stage];
  P.rk_b = B[stage];
  P.dt = dt;
  P.dyn = dyn;
  P.tr_in = trace_buf(m, prec, bin);
  P.tr_out = want_traces ? trace_buf(m, prec, bout) : nullptr;
  if (bg && (lsr_read || lsr_write)) {
    P.dreg = bg->dreg;
    P.dstride = bg->dstride;
    P.lsr_read = lsr_read;
    P.lsr_write = lsr_write;
  }
  cudaError_t err = prepare_viscous(m, P, s, prec, bg);
  if (err != cudaSuccess) return cuda_fail(err, "gradient kernel");
  {
    ProfScope ps(m, PROF_STAGE, s);
    err = sd::launch_stage(m, prec, P, s);
  }
  if (err != cudaSuccess) return cuda_fail(err, "stage kernel");
  m->tr_tag[bin] = nullptr;
  m->tr_tag[bout] = want_traces ? q_out : nullptr;
  m->tr_prec[bout] = prec;
  return SD_OK;
}

sd_status sd_rk_stage(const sd_mesh* m, const sd_phys* ph, sd_precision prec, int32_t stage, double dt,
                      const double* q_n, const double* q_in, double* q_out, const sd_background* bg, void* stream) {
  sd_status st = check_common(m, ph, prec, bg);
  if (st != SD_OK) return st;
  if (stage < 0 || stage > 2) return fail(SD_ERR_INVALID_ARGUMENT, "stage must be 0, 1 or 2");
  if (ph->rk_scheme != SD_RK_SSP33)
    return fail(SD_ERR_UNSUPPORTED, "sd_rk_stage runs the stages of the three-stage method (rk_scheme SD_RK_SSP33)");
  if ((st = check_state_ptr(q_in, "q_in")) != SD_OK) return st;
  if ((st = check_state_ptr(q_out, "q_out")) != SD_OK) return st;
  if (stage > 0 && (st = check_state_ptr(q_n, "q_n")) != SD_OK) return st;
  if (!isfinite(dt)) return fail(SD_ERR_INVALID_ARGUMENT, "dt is not finite");
  DeviceGuard g(m->device);
  return rk_stage_impl(const_cast<sd_mesh*>(m), ph, prec, stage, dt, nullptr, stage > 0 ? q_n : q_in, q_in, q_out, bg,
                       stage < 2, (cudaStream_t)stream);
}

// The five-stage third-order SSP method (sd_phys.rk_scheme = SD_RK_SSP53; Sec. SD Method, last
// paragraph: SSPRK(5,3)): an optimal method of that class (SSP coefficient r), the member of least
// principal error of the family that attains r.  With c = 1/r and L the SD residual:
//   y2 = y1 + c dt L(y1),  y3 = y2 + c dt L(y2),  y4 = (1 - a43) y1 + a43 (y3 + c dt L(y3)),
//   y5 = (1 - a54) y1 + a54 (y4 + c dt L(y4)),  q^(n+1) = a61 y2 + a62 y3 + a65 (y5 + c dt L(y5)).
namespace ssp53 {
constexpr double r = 2.6506291914393882, a43 = 0.47329099097408517, a54 = 0.85150069298830050;
constexpr double a61 = 0.16614637524614647, a62 = 0.063691005655456475, a65 = 0.77016261909839706;
constexpr double c = 1.0 / r;
}  // namespace ssp53

// n_steps of the five-stage method, device-side step control as in advance_impl.
// FP64: y2 -> work, y3 -> work2, then work = a61 y2 + a62 y3 and y4, y5 in place in work2;
// every FP64 stage runs with dt / r (the step-control kernel's second pair), so each stage
// is q_out = a q_n + b (q_in + (dt/r) R) with the coefficients above.  FP32-mixed, increment
// form (D = y - q^n in FP32): stage 2 also leaves W = a61 D2 + a62 D3 in a second register,
// and the last stage adds its D + t to q^n + W (formed in work, FP64).
static sd_status advance53_impl(sd_mesh* mm, const sd_phys* ph, sd_precision prec, double cfl, int32_t n_steps,
                                double* q, double* work, const sd_background* bg, double* dt_out, cudaStream_t s) {
  using namespace ssp53;
  const bool mixed = prec == SD_FP32_MIXED;
  const size_t ne = (size_t)std::max<int64_t>(mm->n_e, 1);
  if (!mm->dyn_s) {
    SD_CUDA(cudaMalloc((void**)&mm->dyn_s, 2 * sizeof(double)));
    mm->device_bytes += 2 * sizeof(double);
  }
  if (!mixed && !mm->work2) {
    const size_t bytes = 9 * ne * (size_t)mm->stride * sizeof(double);
    SD_CUDA(cudaMalloc((void**)&mm->work2, bytes));
    mm->device_bytes += (int64_t)bytes;
  }
  if (mixed && !mm->wreg32) {
    const size_t bytes = 9 * ne * (size_t)bg->dstride * sizeof(float);
    SD_CUDA(cudaMalloc((void**)&mm->wreg32, bytes));
    mm->device_bytes += (int64_t)bytes;
  }
  auto stage_params = [&]() {
    sd::StageParams S = base_params(mm, ph, prec);
    if (bg) {
      S.bg = bg->rec;
      S.bg_jump = bg->jump;
    }
    S.mode = sd::MODE_RK;
    S.dyn = mixed ? mm->dyn : mm->dyn_s;
    if (mixed) {
      S.dreg = bg->dreg;
      S.dstride = bg->dstride;
      S.incr = 1;
      S.qp_in = bg->qp;
    }
    return S;
  };
  auto run = [&](sd::StageParams& S) -> cudaError_t {
    cudaError_t err = prepare_viscous(mm, S, s, prec, bg);
    if (err != cudaSuccess) return err;
    ProfScope ps(mm, PROF_STAGE, s);
    return sd::launch_stage(mm, prec, S, s);
  };
  int a = 0, b = 1;
  for (int32_t k = 0; k < n_steps; ++k) {
    const bool last = k == n_steps - 1;
    if (k == 0) {  // lambda_max of q fused with the traces of q (mixed: and q' of q)
      sd::StageParams P = base_params(mm, ph, prec);
      if (bg) {
        P.bg = bg->rec;
        P.bg_jump = bg->jump;
      }
      SD_CUDA(cudaMemsetAsync(mm->dyn + 4, 0, sd::LAM_SLOTS * sizeof(double), s));
      P.mode = sd::MODE_RESIDUAL;
      P.q_in = q;
      P.tr_out = trace_buf(mm, prec, a);
      P.lam_max = reinterpret_cast<unsigned long long*>(mm->dyn + 4);
      P.lam_nslot = sd::LAM_SLOTS;
      if (mixed) {
        P.qp_out = bg->qp;
        P.dstride = bg->dstride;
      }
      ProfScope ps(mm, PROF_TRACE, s);
      SD_CUDA(sd::launch_traces(mm, prec, P, s));
    }
    {
      ProfScope ps(mm, PROF_OTHER, s);
      if (ph->viscous && ph->visc_cfl > 0.0) SD_CUDA(sd::launch_visc_numax(mm, ph, q, s));
      SD_CUDA(sd::launch_step_control(mm, cfl, ph->c_h, dt_out ? dt_out + 2 * (int64_t)k : nullptr, s, mm->dyn_s, c, ph));
    }
    // stage 1: y2 = q + c dt L(q)
    sd::StageParams S = stage_params();
    S.q_in = S.q_n = q;
    S.out = work;
    S.rk_a = 0.0;
    S.rk_b = mixed ? c : 1.0;
    S.tr_in = trace_buf(mm, prec, a);
    S.tr_out = trace_buf(mm, prec, b);
    if (mixed) S.lsr_write = 1;
    SD_CUDA(run(S));
    // stage 2: y3 = y2 + c dt L(y2) (mixed: and W = a61 D2 + a62 D3)
    S = stage_params();
    S.q_in = mixed ? q : work;
    S.q_n = q;
    S.out = mixed ? work : mm->work2;
    S.rk_a = 0.0;
    S.rk_b = mixed ? c : 1.0;
    S.tr_in = trace_buf(mm, prec, b);
    S.tr_out = trace_buf(mm, prec, a);
    if (mixed) {
      S.lsr_read = 1;
      S.lsr_write = 2;
      S.wreg = mm->wreg32;
      S.w_old = (float)a61;
      S.w_new = (float)a62;
    }
    SD_CUDA(run(S));
    if (!mixed) {  // work = W = a61 y2 + a62 y3
      ProfScope ps(mm, PROF_OTHER, s);
      SD_CUDA(sd::launch_axpby_f64(work, a61, work, a62, mm->work2, 9 * mm->n_e * mm->stride, s));
    }
    // stages 3 and 4: y4 = (1 - a43) q + a43 (y3 + c dt L(y3)), y5 likewise with a54
    for (int st = 3; st <= 4; ++st) {
      const double al = st == 3 ? a43 : a54;
      S = stage_params();
      S.q_in = mixed ? q : mm->work2;
      S.q_n = q;
      S.out = mixed ? work : mm->work2;
      S.rk_a = 1.0 - al;
      S.rk_b = mixed ? al * c : al;
      S.tr_in = trace_buf(mm, prec, st == 3 ? a : b);
      S.tr_out = trace_buf(mm, prec, st == 3 ? b : a);
      if (mixed) {
        S.lsr_read = 1;
        S.lsr_write = 2;
      }
      SD_CUDA(run(S));
    }
    // stage 5: q = a61 y2 + a62 y3 + a65 (y5 + c dt L(y5)); with another step to come it
    // also writes the traces and lambda_max of the new q (mixed: and its q')
    if (mixed) {
      ProfScope ps(mm, PROF_OTHER, s);
      SD_CUDA(sd::launch_add_reg_f64(mm, work, q, mm->wreg32, bg->dstride, s));
    }
    S = stage_params();
    S.q_in = mixed ? work : mm->work2;
    S.q_n = mixed ? q : work;
    S.out = q;
    S.rk_a = mixed ? 1.0 - a65 : 1.0;
    S.rk_b = mixed ? a65 * c : a65;
    S.tr_in = trace_buf(mm, prec, a);
    S.tr_out = last ? nullptr : trace_buf(mm, prec, b);
    S.lam_max = last ? nullptr : reinterpret_cast<unsigned long long*>(mm->dyn + 4);
    S.lam_nslot = sd::LAM_SLOTS;
    if (mixed) {
      S.lsr_read = 1;
      S.lsr_write = 0;
      S.qp_out = last ? nullptr : bg->qp;
    }
    SD_CUDA(run(S));
    std::swap(a, b);
  }
  mm->tr_tag[0] = mm->tr_tag[1] = nullptr;
  return SD_OK;
}

// n_steps SSP-RK3 steps with device-side step control.  Trace buffer `a` holds
// the traces of q at the start of a step: from the trace pass (first step) or
// from the last stage of the previous step, which also leaves lambda_max of q in
// the partial maxima dyn[4 ...] (cleared by the step-control kernel that reads
// them).  Stages: q -> work (a -> b), work -> work (b -> a), work -> q (a -> b
// when another step follows); the buffers then swap roles.
static sd_status advance_impl(sd_mesh* mm, const sd_phys* ph, sd_precision prec, double cfl, int32_t n_steps,
                              double* q, double* work, const sd_background* bg, double* dt_out, cudaStream_t s) {
  if (ph->rk_scheme == SD_RK_SSP53) return advance53_impl(mm, ph, prec, cfl, n_steps, q, work, bg, dt_out, s);
  const bool mixed = prec == SD_FP32_MIXED;
  auto stage_params = [&]() {
    sd::StageParams S = base_params(mm, ph, prec);
    if (bg) {
      S.bg = bg->rec;
      S.bg_jump = bg->jump;
    }
    S.mode = sd::MODE_RK;
    S.dyn = mm->dyn;
    return S;
  };
  int a = 0, b = 1;
  for (int32_t k = 0; k < n_steps; ++k) {
    const bool last = k == n_steps - 1;
    if (k == 0) {  // lambda_max of q fused with the traces of q
      sd::StageParams P = stage_params();
      SD_CUDA(cudaMemsetAsync(mm->dyn + 4, 0, sd::LAM_SLOTS * sizeof(double), s));
      P.mode = sd::MODE_RESIDUAL;
      P.dyn = nullptr;
      P.q_in = q;
      P.tr_out = trace_buf(mm, prec, a);
      P.lam_max = reinterpret_cast<unsigned long long*>(mm->dyn + 4);
      P.lam_nslot = sd::LAM_SLOTS;
      if (mixed) {  // and q' of q for the increment-form stages
        P.qp_out = bg->qp;
        P.dstride = bg->dstride;
      }
      ProfScope ps(mm, PROF_TRACE, s);
      SD_CUDA(sd::launch_traces(mm, prec, P, s));
    }
    {
      ProfScope ps(mm, PROF_OTHER, s);
      if (ph->viscous && ph->visc_cfl > 0.0) SD_CUDA(sd::launch_visc_numax(mm, ph, q, s));
      SD_CUDA(sd::launch_step_control(mm, cfl, ph->c_h, dt_out ? dt_out + 2 * (int64_t)k : nullptr, s, nullptr, 1.0, ph));
    }
    // stage 0: work = q + dt R(q).  The mixed path runs the increment form: it keeps
    // no FP64 intermediate state, only D = q^(s) - q^n in FP32 (D = dt R(q) here),
    // and every stage reads q^n.
    sd::StageParams S = stage_params();
    S.q_in = S.q_n = q;
    S.out = work;
    S.rk_a = 0.0;
    S.rk_b = 1.0;
    S.tr_in = trace_buf(mm, prec, a);
    S.tr_out = trace_buf(mm, prec, b);
    if (mixed) {
      S.dreg = bg->dreg;
      S.dstride = bg->dstride;
      S.lsr_write = 1;
      S.incr = 1;
      S.qp_in = bg->qp;
    }
    SD_CUDA(prepare_viscous(mm, S, s, prec, bg));
    {
      ProfScope ps(mm, PROF_STAGE, s);
      SD_CUDA(sd::launch_stage(mm, prec, S, s));
    }
    // stage 1: work = 3/4 q + 1/4 (work + dt R(work)), in place (mixed: D advances)
    S.q_in = mixed ? q : work;
    S.out = work;
    S.q_n = q;
    S.rk_a = 0.75;
    S.rk_b = 0.25;
    S.tr_in = trace_buf(mm, prec, b);
    S.tr_out = trace_buf(mm, prec, a);
    if (mixed) {
      S.lsr_read = 1;
      S.lsr_write = 2;
    }
    SD_CUDA(prepare_viscous(mm, S, s, prec, bg));
    {
      ProfScope ps(mm, PROF_STAGE, s);
      SD_CUDA(sd::launch_stage(mm, prec, S, s));
    }
    // stage 2: q = 1/3 q + 2/3 (work + dt R(work)); with another step to come it
    // also writes the traces and lambda_max of the new q (mixed: q = q + D + t)
    S.q_in = mixed ? q : work;
    S.q_n = S.out = q;
    S.rk_a = 1.0 / 3.0;
    S.rk_b = 2.0 / 3.0;
    S.tr_in = trace_buf(mm, prec, a);
    S.tr_out = last ? nullptr : trace_buf(mm, prec, b);
    S.lam_max = last ? nullptr : reinterpret_cast<unsigned long long*>(mm->dyn + 4);
    S.lam_nslot = sd::LAM_SLOTS;
    if (mixed) {
      S.lsr_read = 1;
      S.lsr_write = 0;
      S.qp_out = last ? nullptr : bg->qp;  // q' of the new q, for the next step
    }
    SD_CUDA(prepare_viscous(mm, S, s, prec, bg));
    {
      ProfScope ps(mm, PROF_STAGE, s);
      SD_CUDA(sd::launch_stage(mm, prec, S, s));
    }
    std::swap(a, b);
  }
  mm->tr_tag[0] = mm->tr_tag[1] = nullptr;
  return SD_OK;
}

static sd_status check_step(const sd_mesh* m, const sd_phys* ph, sd_precision prec, double cfl, double* q,
                            double* work, const sd_background* bg) {
  sd_status st = check_common(m, ph, prec, bg);
  if (st != SD_OK) return st;
  if ((st = check_state_ptr(q, "q")) != SD_OK) return st;
  if ((st = check_state_ptr(work, "work")) != SD_OK) return st;
  if (q == work) return fail(SD_ERR_INVALID_ARGUMENT, "work must not alias q");
  if (!(cfl > 0.0)) return fail(SD_ERR_INVALID_ARGUMENT, "cfl must be positive");
  return SD_OK;
}

sd_status sd_step(const sd_mesh* m, const sd_phys* ph, sd_precision prec, double cfl, double* q, double* work,
                  const sd_background* bg, double* dt_out, void* stream) {
  sd_status st = check_step(m, ph, prec, cfl, q, work, bg);
  if (st != SD_OK) return st;
  DeviceGuard g(m->device);
  return advance_impl(const_cast<sd_mesh*>(m), ph, prec, cfl, 1, q, work, bg, dt_out, (cudaStream_t)stream);
}

sd_status sd_advance(const sd_mesh* m, const sd_phys* ph, sd_precision prec, double cfl, int32_t n_steps, double* q,
                     double* work, const sd_background* bg, double* dt_out, void* stream) {
  sd_status st = check_step(m, ph, prec, cfl, q, work, bg);
  if (st != SD_OK) return st;
  if (n_steps < 0) return fail(SD_ERR_INVALID_ARGUMENT, "n_steps must not be negative");
  DeviceGuard g(m->device);
  return advance_impl(const_cast<sd_mesh*>(m), ph, prec, cfl, n_steps, q, work, bg, dt_out, (cudaStream_t)stream);
}

sd_status sd_spherical_sums(const sd_mesh* m, const double* q, double r_min, double r_max, int32_t n_r,
                            int32_t n_theta, double* out, void* stream) {
  if (!m) return fail(SD_ERR_INVALID_ARGUMENT, "mesh is NULL");
  sd_status st = check_state_ptr(q, "q");
  if (st != SD_OK) return st;
  if (!out) return fail(SD_ERR_INVALID_ARGUMENT, "out is NULL");
  if (!(r_max > r_min) || !isfinite(r_min) || !isfinite(r_max))
    return fail(SD_ERR_INVALID_ARGUMENT, "need finite r_min < r_max");
  if (n_r < 1 || n_theta < 1 || (int64_t)n_r * n_theta > (1 << 24))
    return fail(SD_ERR_INVALID_ARGUMENT, "n_r and n_theta must be >= 1 with n_r * n_theta <= 2^24");
  if (m->n_e * (int64_t)m->N * m->N * m->N >= ((int64_t)1 << 31))
    return fail(SD_ERR_INVALID_ARGUMENT, "the spherical sums take meshes of fewer than 2^31 points");
  DeviceGuard g(m->device);
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t err;
  {
    ProfScope ps(m, PROF_OTHER, s);
    err = sd::launch_spherical(m, q, r_min, r_max, n_r, n_theta, out, s);
  }
  if (err == cudaErrorMemoryAllocation) return fail(SD_ERR_OUT_OF_MEMORY, "spherical sums: limb accumulators");
  if (err != cudaSuccess) return cuda_fail(err, "spherical sums kernel");
  return SD_OK;
}

sd_status sd_diagnostics(const sd_mesh* m, const sd_phys* ph, const double* q, sd_diag* out, void* stream) {
  sd_status st = check_common(m, ph, SD_FP64, nullptr);
  if (st != SD_OK) return st;
  if ((st = check_state_ptr(q, "q")) != SD_OK) return st;
  if (!out) return fail(SD_ERR_INVALID_ARGUMENT, "out is NULL");
  DeviceGuard g(m->device);
  sd_mesh* mm = const_cast<sd_mesh*>(m);
  cudaStream_t s = (cudaStream_t)stream;
  sd::StageParams P = base_params(m, ph, SD_FP64);
  P.q_in = q;
  P.tr_out = mm->tr64[0];
  {
    ProfScope ps(m, PROF_OTHER, s);
    SD_CUDA(sd::launch_traces(m, SD_FP64, P, s));
  }
  mm->tr_tag[0] = mm->tr_tag[1] = nullptr;
  P.tr_in = mm->tr64[0];
  P.tr_out = nullptr;
  P.mode = sd::MODE_DIVB;
  P.divb = mm->divb;
  {
    ProfScope ps(m, PROF_OTHER, s);
    SD_CUDA(sd::launch_stage(m, SD_FP64, P, s));
    SD_CUDA(sd::launch_diag(m, ph, q, s));
  }
  SD_CUDA(cudaMemcpyAsync(mm->host_diag, mm->diag_out, 10 * sizeof(double), cudaMemcpyDeviceToHost, s));
  SD_CUDA(cudaMemcpyAsync(mm->host_diag + 10, mm->err, sizeof(int), cudaMemcpyDeviceToHost, s));
  SD_CUDA(cudaStreamSynchronize(s));
  if (*reinterpret_cast<const int*>(mm->host_diag + 10) != 0) {
    // reported once: the word is cleared for the calls that follow
    SD_CUDA(cudaMemsetAsync(mm->err, 0, sizeof(int), s));
    SD_CUDA(cudaStreamSynchronize(s));
    return fail(SD_ERR_TIMEOUT, "a bounded device-side wait of a stage kernel ran out since the last sd_diagnostics call");
  }
  const double* h = mm->host_diag;
  const double vol = h[4];
  out->ke = h[0] / vol;
  out->eb = h[1] / vol;
  out->mass = h[2];
  out->energy = h[3];
  out->volume = vol;
  out->max_divb = h[5];
  out->lambda_max = h[6];
  out->min_rho = h[7];
  out->min_p = h[8];
  if (h[9] > 0.0 || h[5] != h[5] || h[6] != h[6])
    return fail(SD_ERR_NONPHYSICAL, "non-physical state: rho <= 0, p <= 0 or NaN at " +
                                        std::to_string((long long)h[9]) + " solution points");
  return SD_OK;
}

sd_status sd_memory_pool_keep(int64_t bytes) {
  int dev = -1;
  cudaError_t err = cudaGetDevice(&dev);
  cudaMemPool_t pool = nullptr;
  if (err == cudaSuccess) err = cudaDeviceGetDefaultMemPool(&pool, dev);
  uint64_t keep = bytes < 0 ? UINT64_MAX : (uint64_t)bytes;
  if (err == cudaSuccess) err = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  if (err != cudaSuccess) return cuda_fail(err, "memory pool release threshold");
  return SD_OK;
}

sd_status sd_mesh_set_wait_limit(sd_mesh* m, int32_t spins) {
  if (!m) return fail(SD_ERR_INVALID_ARGUMENT, "mesh is NULL");
  m->wait_spins = spins < 0 ? sd::kWaitSpins : spins;
  return SD_OK;
}

sd_status sd_profile_enable(sd_mesh* m, int32_t enable) {
  if (!m) return fail(SD_ERR_INVALID_ARGUMENT, "mesh is NULL");
  m->prof_on = enable ? 1 : 0;
  m->prof_used = 0;
  return SD_OK;
}

sd_status sd_profile_read(sd_mesh* m, sd_profile_stats* out) {
  if (!m || !out) return fail(SD_ERR_INVALID_ARGUMENT, "null argument");
  DeviceGuard g(m->device);
  memset(out, 0, sizeof(*out));
  for (size_t i = 0; i < m->prof_used; ++i) {
    SD_CUDA(cudaEventSynchronize(m->prof_ev[2 * i + 1]));
    float ms = 0.0f;
    SD_CUDA(cudaEventElapsedTime(&ms, m->prof_ev[2 * i], m->prof_ev[2 * i + 1]));
    if (m->prof_cls[i] == PROF_STAGE) {
      out->stage_launches++;
      out->stage_ms += ms;
    } else if (m->prof_cls[i] == PROF_TRACE) {
      out->trace_launches++;
      out->trace_ms += ms;
    } else {
      out->other_launches++;
      out->other_ms += ms;
    }
  }
  m->prof_used = 0;
  return SD_OK;
}

}  // extern "C"
