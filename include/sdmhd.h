/*
 * sdmhd.h -- C ABI of the GB300 spectral-difference (SD) MHD+GLM library.
 *
 * The library computes, on one GPU, the SD residual and the explicit SSP
 * Runge-Kutta update of ideal compressible MHD with GLM divergence cleaning
 * on curved hexahedra (arXiv 2502.17805, "Fully Compressible
 * Magnetohydrodynamic Simulations of Solar Convection Zones with CHORUS++"):
 *
 *   dQ/dt + div F(Q) = M(Q)                     Eq. (1), Sec. MHD Governing Equations
 *   Q = (rho, rho U, E, B, psi)                 Eq. (2); E as Eq. (3)
 *   F = inviscid MHD + GLM flux                 Eq. (invF)
 *   M = gravity, Coriolis, Powell, -a psi       source vector M, same section
 *   cubed-sphere shell mesh                     Sec. Meshing
 *   transfinite map, |J|, contravariant flux    Sec. Spectral Difference Method
 *   Chebyshev-Gauss solution points, Legendre
 *   flux points, Lagrange extrapolation and
 *   derivative, BR1 average, Rusanov flux       Sec. Spectral Difference Method
 *   polytropic hydrostatic initial state        Sec. Initial Conditions
 *   wall boundary conditions                    Sec. Problem Formulation and Boundary Conditions
 *   KE and E_B volume averages                  Sec. Results
 *
 * Conventions (all calls)
 *   - State arrays are device pointers to FP64 data in the layout
 *       q[v * 9-plane][e * elem_stride + n],  n = i + N*(j + N*k),
 *     v in (rho, rho u, rho v, rho w, E, Bx, By, Bz, psi), i along xi;
 *     one plane holds n_elements * elem_stride values, elem_stride >= N^3 is
 *     rounded up so every element starts on a 16-byte boundary
 *     (see sd_mesh_query).  Q is the physical state (not |J|-weighted).
 *   - The caller owns every state buffer.  The library owns the mesh,
 *     geometry, background tables and its scratch buffers.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Work is
 *     stream-ordered and asynchronous, except where a call says it
 *     synchronises.
 *   - No call aborts, prints or exits.  Every failure returns a status and
 *     leaves a message for sd_last_error().  Device-side waits are bounded.
 *   - Functions are not thread-safe on one mesh object; distinct mesh objects
 *     may be used from distinct host threads.
 */
#ifndef SDMHD_H
#define SDMHD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SD_OK = 0,
  SD_ERR_INVALID_ARGUMENT = 1, /* null pointer, bad size, bad enum value, misaligned buffer */
  SD_ERR_UNSUPPORTED = 2,      /* order N outside [2, 8] */
  SD_ERR_MESH_TOPOLOGY = 3,    /* non-conforming mesh: a face shared by >2 elements, corners that do not match */
  SD_ERR_MESH_GEOMETRY = 4,    /* |J| <= 0 somewhere in an element */
  SD_ERR_OUT_OF_MEMORY = 5,    /* a device or host allocation failed */
  SD_ERR_CUDA = 6,             /* a CUDA runtime call or kernel launch failed */
  SD_ERR_NONPHYSICAL = 7,      /* rho <= 0, p <= 0 or NaN met by sd_diagnostics */
  SD_ERR_TIMEOUT = 8           /* a bounded device-side wait ran out */
} sd_status;

typedef enum { SD_FP64 = 0, SD_FP32_MIXED = 1 } sd_precision;

/* sd_phys.rk_scheme */
enum { SD_RK_SSP33 = 0, SD_RK_SSP53 = 1 };

/* Boundary conditions of unmatched faces (Sec. Problem Formulation and Boundary
 * Conditions).  Walls are impenetrable (U.n = 0); the inviscid ghost state
 * copies rho, p, psi and E, reflects U, and for the magnetic field either
 * reflects B (perfectly conducting, B_n -> -B_n) or reverses the tangential
 * field (perfectly radial, B_t -> -B_t).  FARFIELD uses sd_phys.farfield as
 * the ghost state (for tests).  PERIODIC is only valid for matched faces. */
typedef enum { SD_BC_PERIODIC = 0, SD_BC_WALL_CONDUCTING = 1, SD_BC_WALL_RADIAL = 2, SD_BC_FARFIELD = 3 } sd_bc;

/* Initial states (sd_init.kind) and their params[]:
 *  SD_INIT_UNIFORM         rho, u, v, w, p, Bx, By, Bz, psi
 *  SD_INIT_ALFVEN          rho, p, |B0|, amplitude, kx, ky, kz, t: circularly polarised
 *                          Alfven wave along k, B0 parallel to k, U = -dB/sqrt(rho)
 *  SD_INIT_SHELL_POLYTROPE N_rho, r_b, r_t, rho_b, R_gas, noise amplitude, dipole ratio:
 *                          polytrope of Sec. Initial Conditions (Eq. polytrop eqns, T_b), gamma and
 *                          GM from sd_phys; density noise at fixed pressure,
 *                          rho0 (1 - A xi sin(pi (r - r_b)/(r_t - r_b))), xi = SplitMix64 draw in
 *                          [-1, 1) keyed by (seed, e*N^3 + n); dipole B0 (3 (z.r)r - z)/r^3 scaled
 *                          so that its magnetic energy is `ratio` times the internal energy
 *  SD_INIT_DIVB_PULSE      rho, p, amplitude, cx, cy, cz, sigma: Bx Gaussian bump, U = 0
 *  SD_INIT_SHELL_FLUX_BALANCED  as SD_INIT_SHELL_POLYTROPE, then L, kappa, kappa_r, kappa_r1,
 *                          kappa_r2: the almost flux-balanced profile (Sec. Initial Conditions):
 *                          the entropy gradient dS/dr = (L / (4 pi r^2) + kappa_r(r) rho_p C_p
 *                          dT_p/dr) / (kappa rho_p T_p), kappa_r(r) = kappa_r + kappa_r1 r + kappa_r2 r^2,
 *                          of the polytrope rho_p, T_p, integrated from the polytrope's bottom
 *                          entropy, and the hydrostatic density drho/dr = -(rho S'/C_p +
 *                          (g/gamma) rho^(2-gamma) exp(-gamma S/C_p)) from rho_b (RK4 on 4,096
 *                          nodes, cubic Hermite interpolation); p = (rho exp(S/C_p))^gamma */
typedef enum {
  SD_INIT_UNIFORM = 0,
  SD_INIT_ALFVEN = 1,
  SD_INIT_SHELL_POLYTROPE = 2,
  SD_INIT_DIVB_PULSE = 3,
  SD_INIT_SHELL_FLUX_BALANCED = 4
} sd_init_kind;

typedef struct {
  int32_t order;              /* N: solution points per direction, 2..8 (Sec. SD Method) */
  int32_t geom;               /* 0: straight edges (trilinear); 1: spherical shell about the origin */
  int64_t n_vertices;
  const double* vertices;     /* host [n_vertices][3] */
  int64_t n_elements;
  const int64_t* hex;         /* host [n_elements][8]; corner (i,j,k) -> i + 2j + 4k, right-handed */
  const double* periodic_lengths; /* host [3] or NULL; entries > 0 make that direction periodic */
  double r_inner, r_outer;    /* shell radii (geom = 1): classify boundary faces as inner / outer */
  int32_t bc_inner, bc_outer; /* sd_bc of inner / outer boundary faces (geom 0: bc_inner for all) */
} sd_mesh_desc;

typedef struct {
  double gamma;     /* ratio of specific heats */
  double GM;        /* gravity g = -GM x / |x|^3 (source M) */
  double omega;     /* rotation rate about z (Coriolis -2 rho Omega x U) */
  double glm_alpha; /* damping a of the GLM source -a psi */
  double c_h;       /* GLM speed used in the flux and the Rusanov speed */
  int32_t powell;   /* 1: Powell terms -(div B)(B, U.B, U) in M */
  int32_t gravity;  /* 1: rho g and rho U.g in M */
  int32_t coriolis; /* 1: Coriolis force in M */
  /* Time integrator of sd_step and sd_advance: SD_RK_SSP33, the three-stage Shu-Osher SSP-RK3
   * (0, the default), or SD_RK_SSP53, the five-stage third-order SSP method the paper names
   * (Sec. SD Method, last paragraph: SSPRK(5,3)), with the coefficients of an optimal method of
   * that class derived in the oracle (SSP coefficient r = 2.6506..., so cfl up to r times the
   * three-stage method's for the same strong-stability bound).  sd_rk_stage and sd_step_packed
   * run the three-stage stages only and refuse SD_RK_SSP53. */
  int32_t rk_scheme;
  double farfield[9]; /* conserved ghost state of SD_BC_FARFIELD faces */
  /* Viscous, resistive and thermal fluxes F_vis (Sec. MHD Governing Equations; F = F_inv - F_vis),
   * with gradients of (U, T, S, B) by the BR1 scheme (Sec. SD Method), when viscous != 0 (both
   * precisions; SD_FP32_MIXED needs a background built with the same coefficients): mu dynamic
   * viscosity (lambda = -2/3 mu), eta magnetic diffusivity, kappa thermal diffusivity of the entropy
   * term (constants), kappa_r radiative diffusivity (with kappa_r1 and kappa_r2 below: kappa_r(r) =
   * kappa_r + kappa_r1 r + kappa_r2 r^2, r = |x| at the point of the heat flux; the caller keeps it
   * non-negative on the mesh), R_gas specific gas constant (T = p / (rho R_gas), C_p = gamma R_gas /
   * (gamma - 1)).  The time step of sd_step is the inviscid one unless visc_cfl (below) is set: the
   * caller then keeps cfl within the viscous limit (measured on the 41,472-element N = 6 shell,
   * N_rho = 3, with mu = 1e-4 and SSP-RK3: the stiff modes of the viscous stress reach NaN within 10
   * steps at cfl 0.2 and stay near the inviscid run's level at 0.01). */
  double mu, eta, kappa, kappa_r, R_gas;
  int32_t viscous;
  int32_t pad2_;
  /* Walls of the viscous path (Sec. Problem Formulation) when visc_walls != 0: stress-free and
   * impenetrable (only the normal viscous stress acts, on the face state whose normal velocity
   * vanishes), the heat flux q_bottom (per area, into the shell) through the inner sphere and the
   * temperature T_top held on the outer sphere (the common value of T in the BR1 gradients); a
   * perfectly conducting wall keeps only the normal part of the current in the resistive terms
   * (J = J_r r^), a radial-field wall holds B_theta = B_phi = 0 through its face state.  Otherwise a
   * wall passes its own F_vis.  visc_walls runs on SD_FP64 only. */
  double q_bottom, T_top;
  int32_t visc_walls;
  int32_t pad3_;
  double kappa_r1, kappa_r2; /* radius dependence of kappa_r (Sec. Benchmark Problem Definition) */
  /* Diffusive limit of the step (not in the paper; viscous != 0 only; 0 = off): sd_step and
   * sd_advance take dt = min(cfl dx_min / lambda_max, visc_cfl dx_min^2 / nu_max), nu_max the
   * largest diffusivity of the step's start state over the solution points,
   * max(4/3 mu / rho, eta, kappa, gamma kappa_r(r)), dx_min the smallest solution-point spacing.
   * One reduction over the state per step.  Measured with SSP-RK3 on the 41,472-element N = 6
   * shell (N_rho = 3, mu = eta = kappa = kappa_r = 1e-4): 0.0157 gives the step at which the stiff
   * modes of the viscous stress stay near the inviscid run's level over 200 steps; twice and four
   * times that let them grow.  SSPRK(5,3)'s stability interval on the negative real axis is 2.47
   * times SSP-RK3's. */
  double visc_cfl;
} sd_phys;

typedef struct {
  int32_t kind; /* sd_init_kind */
  int32_t pad_;
  double params[16];
  uint64_t seed;
} sd_init;

typedef struct {
  double ke;         /* (1/V) int 1/2 rho |U|^2 dV        (Sec. Results, KE) */
  double eb;         /* (1/V) int 1/2 |B|^2 dV            (Sec. Results, E_B) */
  double max_divb;   /* max over solution points of |div B| (discrete SD divergence, BR1 faces) */
  double mass;       /* int rho dV */
  double energy;     /* int E dV */
  double lambda_max; /* max over solution points of |U| + sqrt(gamma p / rho + |B|^2 / rho) */
  double min_rho, min_p;
  double volume;     /* int dV */
} sd_diag;

typedef struct {
  int32_t order;
  int32_t p_map;           /* degree of the polynomial geometry map, floor(N/2) */
  int64_t n_elements;
  int64_t n_points;        /* n_elements * N^3: the degrees of freedom per variable (Sec. Meshing) */
  int64_t elem_stride;     /* values between consecutive elements in one variable plane */
  int64_t state_bytes;     /* bytes of one state array: 9 * n_elements * elem_stride * 8 */
  int64_t n_boundary_faces;
  int64_t n_interior_faces;
  double h_min;            /* smallest element edge chord, for the time-step rule */
  int64_t device_bytes;    /* bytes the library holds on the device for this mesh */
  int64_t trace_bytes;     /* scratch one sd_step_req needs: three FP32 face-trace buffers and 128
                              bytes of lambda_max partial maxima */
} sd_mesh_info;

typedef struct {
  int64_t stage_launches; /* fused element kernels (residual / RK stages) */
  double stage_ms;        /* their summed device time */
  int64_t trace_launches; /* face-trace kernels (with lambda_max in sd_step) */
  double trace_ms;
  int64_t other_launches; /* step control, geometry-free helpers, diagnostics */
  double other_ms;
} sd_profile_stats;

typedef struct sd_mesh sd_mesh;
typedef struct sd_background sd_background;

/* Last error message of the calling host thread ("" when none). */
const char* sd_last_error(void);

/* Build a mesh on the current device: copies the host description, matches
 * faces (sorted corner ids; periodic directions unwrap corners by the period),
 * computes orientation codes, then runs the geometry kernel: the transfinite
 * map of each hexahedron (bilinear edge projectors minus twice the trilinear
 * corner projector, Sec. SD Method) sampled at Chebyshev-Lobatto nodes as a
 * degree-floor(N/2) polynomial map, its contravariant metrics S^d = |J| grad xi_d
 * at the flux points, |J| and x at the solution points.  Synchronises `stream`.
 * A mesh has at least one element (an empty description is
 * SD_ERR_INVALID_ARGUMENT).  Errors: SD_ERR_INVALID_ARGUMENT, SD_ERR_UNSUPPORTED,
 * SD_ERR_MESH_TOPOLOGY, SD_ERR_MESH_GEOMETRY, SD_ERR_OUT_OF_MEMORY, SD_ERR_CUDA.
 * *out is NULL on error. */
sd_status sd_mesh_create(const sd_mesh_desc* desc, void* stream, sd_mesh** out);
sd_status sd_mesh_destroy(sd_mesh* mesh);
sd_status sd_mesh_query(const sd_mesh* mesh, sd_mesh_info* out);

/* Write the initial state (Sec. Initial Conditions) at the solution points.
 * q: device state (layout above).  q_background: device state or NULL; for
 * SD_INIT_SHELL_POLYTROPE and SD_INIT_SHELL_FLUX_BALANCED it receives the
 * noise-free, field-free profile (rho0, 0, p0/(gamma-1), 0, 0), otherwise zeros.
 * Asynchronous. */
sd_status sd_state_init(const sd_mesh* mesh, const sd_phys* phys, const sd_init* init, double* q,
                        double* q_background, void* stream);

/* Prepare the FP32-mixed precision path around a hydrostatic background Q0
 * (device state, only rho and E are read; U = B = psi = 0 is assumed):
 * rounds rho0 and p0 to FP32, computes in FP64 the background residual R0
 * (pressure gradient with central face average, plus rho0 g; at a far-field
 * face the background is its own ghost, the far field entering the mixed
 * stages as a perturbation) and the FP64 jumps of the background across faces.  The handle also holds the FP32 scratch of
 * the mixed sd_step (the register D and the FP32 perturbation q' of the step's
 * starting state, 72 bytes per solution point), so one background serves one
 * sd_step / sd_advance / packed request at a time.  The handle stays valid
 * while the mesh lives.  Asynchronous: its device memory comes from the stream-ordered
 * allocator on `stream`, and the tables are complete once the work issued to
 * `stream` so far is (use the handle on `stream`, or after synchronising it).
 * q_background may be released once that work is complete.
 * With phys->viscous set the background also carries, for the viscous fluxes of
 * the mixed path, its own viscous residual (FP64, rounded to FP32: the heat flux
 * of Q0, in the energy component) and grad T0, grad S0 with their face traces
 * (28 more bytes per solution point); the mixed path then takes the viscous
 * fluxes of the perturbation in FP32 (gradients of (U, T', S', B)) for phys
 * with the same mu, eta, kappa, kappa_r(r) and R_gas.  Not taken with viscous
 * set: visc_walls != 0 or far-field faces (SD_ERR_UNSUPPORTED). */
sd_status sd_background_create(const sd_mesh* mesh, const sd_phys* phys, const double* q_background, void* stream,
                               sd_background** out);
/* Releases the background's device memory in stream order on the legacy default
 * stream (after all work issued so far to it and to blocking streams); work on
 * a non-blocking stream that uses the background must be complete first. */
sd_status sd_background_destroy(sd_background* bg);

/* dqdt = -div F / |J| + M at every solution point (Sec. SD Method: extrapolate to
 * the flux points, contravariant flux, Rusanov / BR1 common values at element
 * faces, derivative of the flux polynomials).  q and dqdt: device states.
 * SD_FP64: every step in FP64.  SD_FP32_MIXED: needs `bg`; the perturbation
 * about the background is carried through the SD operators in FP32 and added
 * to the FP64 background residual.  Asynchronous. */
sd_status sd_residual(const sd_mesh* mesh, const sd_phys* phys, sd_precision prec, const double* q,
                      const sd_background* bg, double* dqdt, void* stream);

/* One stage of the Shu-Osher SSP-RK3 scheme with the residual fused in:
 *   stage 0: q_out = q_in + dt R(q_in)                       (q_n ignored)
 *   stage 1: q_out = 3/4 q_n + 1/4 (q_in + dt R(q_in))
 *   stage 2: q_out = 1/3 q_n + 2/3 (q_in + dt R(q_in))
 * The RK combination is always FP64.  q_out may alias q_in or q_n.  Stage 0
 * recomputes the face traces of q_in; stages 1 and 2 reuse the traces the
 * previous stage wrote for its q_out when q_in is that buffer, so the
 * intermediate states must not be changed outside the library between the
 * stages of one step.  Asynchronous. */
sd_status sd_rk_stage(const sd_mesh* mesh, const sd_phys* phys, sd_precision prec, int32_t stage, double dt,
                      const double* q_n, const double* q_in, double* q_out, const sd_background* bg, void* stream);

/* One full SSP-RK3 step with device-side step control: lambda_max of q (max of
 * |U| + fast speed over the solution points), dt = cfl * dx_min / lambda_max with
 * dx_min = h_min (X_s,2 - X_s,1) the smallest solution-point spacing (with
 * the viscous terms and phys->visc_cfl > 0 at most visc_cfl dx_min^2 / nu_max),
 * c_h = lambda_max when phys->c_h <= 0 (else phys->c_h), then the three fused
 * stages.  q (in/out) and work: device states; dt_out: device double[2] or NULL,
 * receives (dt, c_h).  SD_FP32_MIXED keeps no FP64 intermediate state: the
 * lambda_max pass also stores q' = q^n - Q0 in FP32 in the background, every
 * stage reads q' and the background's FP32 register D = q^(s) - q^n, and only
 * the last stage reads and writes q (work is then not written).  No host
 * synchronisation.
 * With phys->rk_scheme = SD_RK_SSP53 the step is the five-stage SSPRK(5,3) (Sec. SD
 * Method) instead: SD_FP64 then also uses a second stage state, and SD_FP32_MIXED a
 * second FP32 register, both allocated by the mesh on first use, and work holds
 * q^n plus that register's combination of stages 2 and 3 for the last stage.
 * Asynchronous. */
sd_status sd_step(const sd_mesh* mesh, const sd_phys* phys, sd_precision prec, double cfl, double* q, double* work,
                  const sd_background* bg, double* dt_out, void* stream);

/* n_steps >= 0 consecutive sd_step calls in one call, with the same results bit
 * for bit.  The last stage of every step but the final one also returns the
 * face traces and lambda_max of the state it writes, which the next step uses in
 * place of its own trace pass (one read of the state per step fewer).  dt_out:
 * device double[2 * n_steps] or NULL, receives (dt, c_h) of each step in order.
 * Same arguments and errors as sd_step otherwise.  Asynchronous. */
sd_status sd_advance(const sd_mesh* mesh, const sd_phys* phys, sd_precision prec, double cfl, int32_t n_steps,
                     double* q, double* work, const sd_background* bg, double* dt_out, void* stream);

/* Longitude averages on a spherical shell (Sec. Results: differential rotation
 * <V_phi>, meridional circulation from <V_r> and <V_theta>, poloidal and
 * toroidal magnetic energy): the shell r in [r_min, r_max] about the origin is
 * divided into n_r bins of equal radial width and n_theta bins of equal
 * colatitude width over [0, pi]; every solution point adds its quadrature weight
 * w |J| times (1, V_r, V_theta, V_phi, (B_r^2 + B_theta^2)/2, B_phi^2/2, rho,
 * rho |U|^2/2) to the bin that holds it (points outside [r_min, r_max] go to the
 * nearest radial bin; on the rotation axis phi is taken as 0).  Dividing by the
 * first entry gives the bin means.  out: device double[n_r][n_theta][8],
 * overwritten.  Reproducible: each quantity is summed exactly in a 128-bit
 * fixed-point accumulator scaled to its largest |term| over the mesh (terms
 * resolved to 2^-126 of that term), then converted to double within about one
 * unit in the last place, so the result does not depend on the order of the
 * points or of the elements (bitwise).  A quantity with a non-finite term sums
 * to NaN.  Meshes of 2^31 points or more: SD_ERR_INVALID_ARGUMENT.  Scratch of
 * 256 bytes per bin is allocated on the stream for the call
 * (SD_ERR_OUT_OF_MEMORY when that fails).  The paper's B^2 / 8 pi is B^2 / 2 in
 * the library's units.  Asynchronous. */
sd_status sd_spherical_sums(const sd_mesh* mesh, const double* q, double r_min, double r_max, int32_t n_r,
                            int32_t n_theta, double* out, void* stream);

/* ---- Packed stepping of many independent solves (serving).
 * One request is one shell (or box) solve on its own mesh with its own physics,
 * background and states.  sd_step_packed advances every request by one
 * SSP-RK3 step of the FP32-mixed path (the same arithmetic as sd_step with
 * SD_FP32_MIXED): per order N present it launches one lambda_max/trace kernel,
 * one step-control kernel and three stage kernels over the elements of all
 * requests of that order, so small solves share launches and fill the GPU.
 * Each request's result does not depend on the others in the pack. */
typedef struct {
  const sd_mesh* mesh;
  sd_phys phys;             /* c_h <= 0: c_h = lambda_max of the request each step */
  const sd_background* bg;  /* required, and not shared with another request of the call */
  double* q;                /* device state, advanced in place */
  double* work;             /* device state used inside the step */
  void* traces;             /* device scratch of sd_mesh_info.trace_bytes bytes, 16-byte aligned */
  double* dyn;              /* device double[4]: receives (dt, c_h, lambda_max) of the step in [0..2] */
  double cfl;               /* dt = cfl * dx_min / lambda_max as in sd_step */
  int32_t flags;            /* SD_REQ_* bits below, 0 for a plain step */
  int32_t pad_;
} sd_step_req;

/* sd_step_req.flags.  SD_REQ_KEEP_TRACES: the last stage also leaves the face
 * traces and lambda_max of the new q (and its FP32 perturbation, in the
 * background) in `traces`, as sd_advance does between its steps.
 * SD_REQ_TRACES_READY: `traces` holds what the previous call of this request
 * left with SD_REQ_KEEP_TRACES, and q has not been changed since; the call then
 * skips the request's lambda_max/trace pass.  The results are the same bits
 * with or without the flags. */
enum { SD_REQ_KEEP_TRACES = 1, SD_REQ_TRACES_READY = 2 };

typedef struct sd_packer sd_packer;

/* A packer holds the device tables of up to max_requests requests per call. */
sd_status sd_packer_create(int32_t max_requests, sd_packer** out);
sd_status sd_packer_destroy(sd_packer* packer);
/* reqs: host array of n requests (n <= max_requests), all meshes on the current
 * device.  Asynchronous on `stream`; a second call may be issued before the
 * first finishes (the packer keeps its tables until the GPU has read them). */
sd_status sd_step_packed(sd_packer* packer, int32_t n, const sd_step_req* reqs, void* stream);

/* Global diagnostics of q in FP64 (Sec. Results: KE, E_B), with the discrete
 * div B of the residual (BR1 face average) for max|div B|.  Sums run in a fixed
 * order (deterministic).  Synchronises `stream`; returns SD_ERR_NONPHYSICAL
 * (with *out filled) when rho <= 0, p <= 0 or a NaN is found, and
 * SD_ERR_TIMEOUT (*out not filled) when a bounded device-side wait of a stage
 * kernel on this mesh ran out since the previous sd_diagnostics call. */
sd_status sd_diagnostics(const sd_mesh* mesh, const sd_phys* phys, const double* q, sd_diag* out, void* stream);

/* sd_residual_noalloc -- the FP64 residual of sd_residual (same result within
 * FP64 round-off; the same kernels run) without any memory allocation.  The
 * paper has no counterpart: this call exists for callers that cannot call
 * cudaMalloc when they need a residual, for example an application whose memory
 * pool already holds all the device memory it may use, or a latency-bound loop
 * that must not risk the device-wide synchronisation an allocation can cause.
 * Its scratch (the face traces of q and the common face fluxes) is a fixed
 * 8 MiB device array inside the library, held on every GPU that loads the
 * library until the process exits; meshes that need more ((n_elements * 54 +
 * n_owned_faces * 10) * N^2 * 8 bytes > 8 MiB, where every interior face counts
 * once and every boundary face once: about 25 KB per element of a closed mesh
 * at N = 6, i.e. about 330 elements) are rejected with SD_ERR_INVALID_ARGUMENT
 * and a message.  The first call on each device looks up the array's device address
 * with that device current; make that first call before any stream capture.
 * All calls share the one array, which keeps the last call's contents (every
 * entry a call reads is written earlier in the same call), so calls whose work
 * overlaps on the GPU (other streams, other threads) race.  q and dqdt: device
 * states; the mesh must belong to the current device.  Inviscid only: phys with
 * viscous set is rejected with SD_ERR_UNSUPPORTED (the viscous fluxes need
 * gradient buffers).  Asynchronous. */
sd_status sd_residual_noalloc(const sd_mesh* mesh, const sd_phys* phys, const double* q, double* dqdt, void* stream);

/* Stream-ordered memory for serving: sd_background_create takes its device
 * memory from the current device's default memory pool (cudaMallocAsync), which
 * by default returns freed memory to the system at every synchronisation, so a
 * service that creates and releases backgrounds continually pays for fresh
 * allocations.  This call keeps up to `bytes` of freed memory in that pool for
 * reuse (its release threshold; bytes < 0 keeps all of it).  The setting
 * belongs to the device's default pool and so applies to every user of that
 * pool in the process.  Errors: SD_ERR_CUDA. */
sd_status sd_memory_pool_keep(int64_t bytes);

/* Failure-detection test hook: the number of polls a stage kernel makes on
 * each of its bounded device-side waits (the shared-memory bulk copies of the
 * FP32-mixed stages) before it records a time-out.  spins < 0 restores the
 * default (65536 polls, about a millisecond).  A wait that runs out still lets
 * its copies land before the kernel goes on (a second bounded wait), so the
 * results stay valid; the time-out is recorded in the mesh's error word, which
 * the next sd_diagnostics call reports as SD_ERR_TIMEOUT and then clears.
 * With spins = 0 every wait of the next stage launches runs out at once. */
sd_status sd_mesh_set_wait_limit(sd_mesh* mesh, int32_t spins);

/* Kernel timing (tracing): with enable = 1 every kernel the library launches
 * for this mesh is bracketed by CUDA events on its launching stream; the
 * counters restart.  At most 65536 launches are recorded.  enable = 0 stops
 * recording. */
sd_status sd_profile_enable(sd_mesh* mesh, int32_t enable);
/* Waits for the recorded events, sums the device time per kernel class into
 * *out and clears the record. */
sd_status sd_profile_read(sd_mesh* mesh, sd_profile_stats* out);

#ifdef __cplusplus
}
#endif
#endif /* SDMHD_H */
