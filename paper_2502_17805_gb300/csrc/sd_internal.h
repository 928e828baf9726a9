// sd_internal.h -- structures shared by the host API and the CUDA kernels of the
// SD MHD+GLM library.  Not part of the public ABI (include/sdmhd.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/sdmhd.h"

namespace sd {

constexpr int kMaxN = 8;
// nodes per direction of the element map (degree floor(N/2) <= 4)
constexpr int kMaxGeoP1 = kMaxN / 2 + 1;
constexpr int kNV = 9;  // conserved variables

// 1D operators of one order N (Sec. SD Method): solution points xs, flux points
// xf, extrapolation E[f][i] = h_i(xf_f), derivative D[i][f] = l_f'(xs_i),
// quadrature weights w_i = int_0^1 h_i.  Passed to kernels by value.
template <typename R>
struct Ops {
  R E[(kMaxN + 1) * kMaxN];
  R D[kMaxN * (kMaxN + 1)];
  // Even-odd split of E and D.  Solution and flux points are symmetric about
  // 1/2, so E[N-f][N-1-i] = E[f][i] and D[N-1-i][f] = -D[i][N-f].  For f <= N/2,
  // i <= (N-1)/2: Es[f N + i] = (E[f][i] + E[f][N-1-i]) / 2, Ed = the half
  // difference (the middle solution point: Es = E, Ed = 0); Ds[i (N+1) + f] and
  // Dd alike over the flux-point pairs (f, N-f) (the middle flux point: Ds = D).
  R Es[(kMaxN + 1) * kMaxN];
  R Ed[(kMaxN + 1) * kMaxN];
  R Ds[kMaxN * (kMaxN + 1)];
  R Dd[kMaxN * (kMaxN + 1)];
  R w[kMaxN];
  R xs[kMaxN];
  R xf[kMaxN + 1];
};

// The FP32 line operators for Blackwell's paired FP32 arithmetic: every
// coefficient of the even-odd split of E and D (Ops::Es, Ed, Ds, Dd) and of the
// extrapolation to the two ends of a line (E[0][i], E[N][i]) held twice,
// {c, c}, so that one paired FMA applies it to two variables at once.
struct Ops2 {
  float2 Es[(kMaxN + 1) * kMaxN];
  float2 Ed[(kMaxN + 1) * kMaxN];
  float2 Ds[kMaxN * (kMaxN + 1)];
  float2 Dd[kMaxN * (kMaxN + 1)];
  float2 E0[kMaxN];
  float2 EN[kMaxN];
};

// Face metadata word: neighbour face (3 bits) | orientation code << 3 |
// boundary condition << 6 | owner << 9.  Orientation code: bit 2 swaps the
// two face-local indices, bits 1 and 0 flip the first and second.
__host__ __device__ inline int meta_nbF(int m) { return m & 7; }
__host__ __device__ inline int meta_code(int m) { return (m >> 3) & 7; }
__host__ __device__ inline int meta_bc(int m) { return (m >> 6) & 7; }
// boundary face on the outer sphere of a shell (bit 10)
__host__ __device__ inline int meta_outer(int m) { return (m >> 10) & 1; }
__host__ __device__ inline int meta_owner(int m) { return (m >> 9) & 1; }

// Offset, within one element's block of the FP32 metrics S^d (9 (N+1) N^2
// values), of component c of S^d at flux point f of line `line` of family d.
// The N^2 lines of one (d, f, c) are contiguous, so that the threads of a warp,
// which take consecutive lines of one flux point, read consecutive words.
__host__ __device__ constexpr inline int s32_index(int N, int d, int f, int c, int line) {
  return ((d * (N + 1) + f) * 3 + c) * N * N + line;
}

enum StageMode { MODE_RESIDUAL = 0, MODE_RK = 1, MODE_DIVB = 2 };

// Arguments of the fused element kernels.  Geometry pointers are float or
// double according to the precision policy of the kernel.
struct StageParams {
  int64_t n_e;
  int64_t stride;  // element stride of state arrays
  int64_t plane;   // n_e * stride
  const double* q_in;
  const double* q_n;
  double* out;     // dqdt (residual) or q_out (RK)
  int mode;
  int central;     // 1: face flux is the central average (no Rusanov dissipation)
  int ff_own;      // 1: a far-field face takes this side's own state as its ghost (the background pass)
  double rk_a, rk_b;
  double dt, c_h;
  const double* dyn;  // device (dt, c_h) or nullptr
  double gamma, GM, omega, alpha;
  double inv_gm1;  // 1/(gamma-1); the mixed background energy is E0 = p0 * inv_gm1
  int powell, gravity, coriolis, pad_;
  double farfield[9];
  const void* Sfam;   // FP64: [e][d][c][line][f]; FP32: [e][d][f][c][line] (s32_index)
  const void* invJ;   // [e][n]
  const void* X;      // [e][c][n]
  const int* nbr;     // [e][6] neighbour element or -1
  const int* meta;    // [e][6]
  const void* tr_in;  // [e][F][v][N^2] traces of q_in
  void* tr_out;       // traces of the output state (RK) or nullptr
  const float* bg;       // [5][n_e * N^3] rho0, p0, R0x, R0y, R0z (FP32 mixed)
  const float* bg_jump;  // [e][F][2][N^2] background jumps (rho0, p0), neighbour minus own
  double* divb;          // [n_e * N^3] (MODE_DIVB)
  unsigned long long* lam_max;  // partial maxima of lambda (bits of positive doubles), or nullptr
  int lam_nslot;                // number of partial maxima at lam_max (a power of two; 0 or 1: one)
  // low-storage form of the mixed RK stages (sd_step): D = q^(s) - q^n in FP32,
  // [9][n_e * dstride]; lsr_read: use D instead of q_n; lsr_write: 1 store D = t, 2 store D += t
  float* dreg;
  int64_t dstride;
  int lsr_read, lsr_write;
  // five-stage method, increment form: a stage that advances D in place (lsr_write 2)
  // also stores W = w_old D + w_new (D + t) here, [9][n_e * dstride] (nullptr: not)
  float* wreg;
  float w_old, w_new;
  // increment form (FP32-mixed sd_step): q_in is q^n in every stage and the stage's
  // state is q^n + D; stages with lsr_write only advance D, the last writes q^n + D + t
  int incr;
  // FP32 q' of q^n, [9][n_e * dstride], rounded from q^n as a load of it rounds
  // it: read by the increment-form stages (qp_in) in place of q^n; written by a
  // mixed trace pass and by an exact last stage (qp_out, for the new state)
  const float* qp_in;
  float* qp_out;
  // packed trace launch: this request's traces are already current, the CTA returns at once
  int skip;
  int* err;  // device error word (bounded waits that ran out)
  int wait_spins;  // polls of a bounded wait before it reports a time-out
  // FP64 face fluxes, computed once per face by its owner: the faces this mesh's
  // elements own (e * 6 + F, boundary faces included), the index k of the face of
  // (e, F) in that list (for either side), and the values [k][10][N^2]
  int64_t n_own;
  const int* own_faces;
  const int* face_k;
  void* gface;
  // viscous, resistive and thermal fluxes (FP64 policy): coefficients; the viscous kernel
  // writes the face traces [e][F][15][N^2] of the record (tau, J, grad T, grad S) to gtr_out,
  // the record at the solution points [e][15][N^3] to grad_out when set, and the interior
  // part of the viscous divergence [e][7][N^3] to rvis64_out; the face-flux kernel reads
  // gtr_in, the element kernel rvis64
  int visc, visc_walls;
  double mu, eta, kappa, kappa_r, R_gas;
  double kappa_r1, kappa_r2;  // kappa_r(r) = kappa_r + kappa_r1 r + kappa_r2 r^2
  double q_bottom, T_top;  // wall conditions of the viscous path (visc_walls)
  const double* gtr_in;
  double* grad_out;
  double* gtr_out;
  const double* rvis64;
  double* rvis64_out;
  // viscous fluxes on the FP32-mixed path: the perturbation gradient record [e][15][N^3], each
  // element's own F_vis . n at its face points along its outward unit normal [e][F][7][N^2]
  // (components rho U, E, B; mvf), the background's viscous record [7][n_e N^3] (its energy
  // residual, grad T0, grad S0) and its face traces [e][F][6][N^2], and the viscous residual of the
  // stage state [7][n_e N^3] (components rho U, E, B) that the mixed stage kernel adds
  const float* mgrad;
  const float* mvf_in;
  float* mgrad_out;
  float* mvf_out;
  const float* bg_visc;
  const float* bg_vtr;
  float* rvis_out;
  const float* rvis;
};

}  // namespace sd

struct sd_mesh {
  int device;
  int N, p;
  int64_t n_e;
  int64_t stride;
  int64_t n_bf, n_if;
  double h_min;
  int geom;
  // device geometry
  double* Sfam64;
  double* invJ64;
  double* X64;
  float* Sfam32;
  float* invJ32;
  float* X32;
  int* nbr;
  int* meta;
  // scratch: face traces (ping-pong), small device scalars
  double* tr64[2];
  float* tr32[2];
  const double* tr_tag[2];  // state whose traces buffer b holds (stage chaining)
  int tr_prec[2];
  double* dyn;              // [4 + LAM_SLOTS]: dt, c_h, lambda_max, spare, then the partial maxima of lambda
  double* diag_part;        // [n_e][12]
  double* diag_out;         // [12]
  double* divb;             // [n_e * N^3]
  double* host_diag;        // pinned [12]
  int* own_faces;           // [n_own] e * 6 + F of the faces the elements own (boundary faces included)
  int* face_k;              // [n_e][6] index in own_faces of the face of (e, F), either side
  int64_t n_own;
  double* gface64;          // [n_own][10][N^2] FP64 common face fluxes of the current stage
  int* err;                 // device error word of the stage kernels
  int wait_spins;           // polls of a stage kernel's bounded wait before a time-out (sd_mesh_set_wait_limit)
  double* grad;             // viscous FP64 path, allocated on first use: the record [e][15][N^3]
  double* gtr;              //   (the background only), its face traces [e][F][15][N^2]
  double* rvis64;           //   and the interior viscous divergence [e][7][N^3]
  float* grad32;            // viscous FP32-mixed path, allocated on first use: the gradient record,
  float* mvf32;             //   each side's F_vis . n at the faces
  float* rvis32;            //   and the viscous residual [7][n_e N^3]
  // five-stage time integrator (sd_phys.rk_scheme), allocated on first use: (dt/r, c_h)
  // for the FP64 stages, a second FP64 stage state, the FP32 register W of the mixed path
  double* dyn_s;
  double* work2;
  float* wreg32;
  int has_farfield;         // the mesh has far-field boundary faces
  int64_t device_bytes;
  sd::Ops<double> ops64;
  sd::Ops<float> ops32;
  sd::Ops2 ops2;
  // kernel timing: event pairs (start, stop) with a kernel class
  int prof_on;
  std::vector<cudaEvent_t> prof_ev;
  std::vector<int> prof_cls;
  size_t prof_used;
};

struct sd_background {
  const sd_mesh* mesh;
  float* rec;    // [5][n_e * N^3]
  float* jump;   // [n_e][6][2][N^2]
  float* dreg;   // [9][n_e * dstride]: FP32 difference register of the mixed sd_step
  float* qp;     // [9][n_e * dstride]: FP32 q' of q^n (same allocation as dreg)
  int64_t dstride;
  double gamma;
  int device;
  // built with viscous fluxes: the background's viscous energy residual, grad T0, grad S0
  // [7][n_e N^3] and the face traces of the gradients [e][F][6][N^2], with the coefficients used
  float* vrec;
  float* vtr;
  double visc_coef[8];  // mu, eta, kappa, kappa_r, kappa_r1, kappa_r2, R_gas, 1 when built with viscous fluxes
};

namespace sd {
// polls of a bounded mbarrier wait before it reports a time-out (about a millisecond)
constexpr int kWaitSpins = 1 << 16;
// partial maxima of lambda per mesh: the warps of a launch spread their atomics over these
constexpr int LAM_SLOTS = 256;
// gradients the viscous fluxes need: 8 primitive variables x 3 directions, index 3 c + j
constexpr int NGRAD = 24;
// Values per point of the viscous paths' gradient record: the viscous stress (6),
// the current (3), grad T and grad S (their perturbations on the FP32-mixed path).
constexpr int MV_REC = 15;
// kernels launched from the API (defined in the .cu files)
cudaError_t launch_stage(const sd_mesh* m, int prec, const StageParams& P, cudaStream_t s);
cudaError_t launch_traces(const sd_mesh* m, int prec, const StageParams& P, cudaStream_t s);
// longitude averages on the shell: volume sums per bin of radius x colatitude into out[n_r][n_t][8]
cudaError_t launch_spherical(const sd_mesh* m, const double* q, double r_min, double r_max, int n_r, int n_t,
                             double* out, cudaStream_t s);
// viscous FP64 path: the BR1 gradient record's face traces (and the record itself when
// P.grad_out is set) and the interior viscous divergence of P.q_in
cudaError_t launch_grad(const sd_mesh* m, const StageParams& P, cudaStream_t s);
// viscous FP32-mixed path: perturbation gradients (Pg), then the viscous residual (Pv)
cudaError_t launch_mixed_visc(const sd_mesh* m, const StageParams& Pg, const StageParams& Pv, cudaStream_t s);
// the background's viscous record from the FP64 residuals with and without viscous fluxes and the
// FP64 gradients of the background
cudaError_t launch_bg_visc(const sd_mesh* m, const double* R0, const double* R0v, const double* grad,
                           const double* gtr, float* vrec, float* vtr, cudaStream_t s);
cudaError_t launch_geometry(sd_mesh* m, const double* d_corners, int* d_flag, cudaStream_t s);
cudaError_t launch_canonical_faces(sd_mesh* m, cudaStream_t s);
// radial profile table of the flux-balanced initial state: [4][n + 1] = rho, S, drho/dr, dS/dr on
// uniform nodes r_b + k h (tab = nullptr for the other kinds)
struct ProfileTable {
  const double* tab;
  int n;
  double rb, h, Cp;
};
cudaError_t launch_state_init(const sd_mesh* m, const sd_phys* ph, const sd_init* in, double B0dip,
                              const ProfileTable& tab, double* q,
                              double* qbg, cudaStream_t s);
cudaError_t launch_diag(const sd_mesh* m, const sd_phys* ph, const double* q, cudaStream_t s);
cudaError_t launch_bg_prepare(const sd_mesh* m, double gamma, double inv_gm1, const double* q_bg, double* q0,
                              float* rec, cudaStream_t s);
cudaError_t launch_bg_finish(const sd_mesh* m, double gamma, const double* R0, float* rec, float* jump,
                             const double* tr, cudaStream_t s);
// visc with viscous != 0 and visc_cfl > 0: also dt <= visc_cfl dx_min^2 / nu_max, from the extrema
// launch_visc_numax left
cudaError_t launch_step_control(const sd_mesh* m, double cfl, double c_h_fixed, double* dt_out, cudaStream_t s,
                                double* dyn_s = nullptr, double dt_scale = 1.0, const sd_phys* visc = nullptr);
// the extrema the diffusive limit of the step needs (the smallest density over the solution points
// of the FP64 state q; the largest gamma kappa_r(r) when kappa_r varies), for the next step control
cudaError_t launch_visc_numax(const sd_mesh* m, const sd_phys* ph, const double* q, cudaStream_t s);
cudaError_t launch_axpby_f64(double* out, double a, const double* x, double b, const double* y, int64_t n,
                             cudaStream_t s);
cudaError_t launch_add_reg_f64(const sd_mesh* m, double* out, const double* q, const float* w, int64_t dstride,
                               cudaStream_t s);
}  // namespace sd
