/*
 * sdref.h -- plain FP64 CPU oracle of the spectral-difference (SD) MHD+GLM
 * residual, SSP-RK3 stage, diagnostics and initial states.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this library: only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark use it.  It shares no code with the CUDA library.
 *
 * It follows the paper ("Fully Compressible MHD Simulations of Solar
 * Convection Zones with CHORUS++", arXiv 2502.17805):
 *   - conservative form and variables ........ Eq. (1)-(3) (divergence form, Q, E)
 *   - source vector M ......................... Sec. "MHD Governing Equations", M
 *   - inviscid MHD+GLM flux ................... Eq. (invF)
 *   - cubed-sphere mesh ....................... Sec. "Meshing"
 *   - transfinite map, Jacobian, transformed
 *     equations ............................... Sec. "Spectral Difference Method"
 *   - solution/flux points, Lagrange bases .... Sec. "Spectral Difference Method"
 *   - BR1 average, Rusanov common flux ........ Sec. "Spectral Difference Method"
 *   - polytropic initial state ................ Sec. "Initial Conditions", Eq. (polytrop eqns), T_b
 *   - impenetrable / conducting / radial walls  Sec. "Problem Formulation and Boundary Conditions"
 *   - KE and E_B volume averages .............. Sec. "Results"
 * Readings of passages the paper leaves open are listed at each function.
 *
 * State layout: q[v][e][n], v in (rho, rho u, rho v, rho w, E, Bx, By, Bz, psi),
 * n = i + N*(j + N*k) with i along xi.  Dense: element stride is N^3.
 * All pointers are host pointers.  Functions return 0 on success and a
 * nonzero code on failure, with a message in sdref_last_error().
 */
#ifndef SDREF_H
#define SDREF_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { SDREF_BC_PERIODIC = 0, SDREF_BC_WALL_CONDUCTING = 1, SDREF_BC_WALL_RADIAL = 2, SDREF_BC_FARFIELD = 3 };
enum { SDREF_INIT_UNIFORM = 0, SDREF_INIT_ALFVEN = 1, SDREF_INIT_SHELL_POLYTROPE = 2,
       SDREF_INIT_DIVB_PULSE = 3, SDREF_INIT_SINB = 4, SDREF_INIT_SHELL_FLUX_BALANCED = 5 };

typedef struct {
  double gamma, GM, omega, glm_alpha, c_h;
  int32_t powell, gravity, coriolis, pad_;
  double farfield[9]; /* conserved ghost state for SDREF_BC_FARFIELD faces */
  /* viscous, resistive and thermal fluxes F_vis (Sec. MHD Governing Equations), used when viscous != 0:
   * dynamic viscosity mu (lambda = -2/3 mu), magnetic diffusivity eta, thermal diffusivity kappa of the
   * entropy term, radiative diffusivity kappa_r, specific gas constant R_gas (T = p / (rho R_gas),
   * C_p = gamma R_gas / (gamma - 1)), all constant */
  double mu, eta, kappa, kappa_r, R_gas;
  int32_t viscous, pad2_;
  /* walls of the viscous path (Sec. Problem Formulation; readings W1, W2), when visc_walls != 0:
   * stress-free and impenetrable walls, the heat flux q_bottom (per area, into the shell) through the
   * inner sphere, the temperature T_top on the outer sphere; otherwise a wall takes its own F_vis */
  double q_bottom, T_top;
  int32_t visc_walls, pad3_;
  /* radius-dependent radiative diffusivity (reading V7): kappa_r(r) = kappa_r + kappa_r1 r + kappa_r2 r^2,
   * r = |x| at the point where the heat flux is evaluated */
  double kappa_r1, kappa_r2;
} sdref_phys;

typedef struct {
  double ke, eb, max_divb, mass, energy, lambda_max, min_rho, min_p, volume;
} sdref_diag;

typedef struct sdref_mesh sdref_mesh;

const char* sdref_last_error(void);

/* 1D operators of order N (2..8): solution points xs[N], flux points xf[N+1],
 * extrapolation E[(N+1)*N] (E[f*N+i] = h_i(xf[f])), derivative
 * D[N*(N+1)] (D[i*(N+1)+f] = l_f'(xs[i])), quadrature weights w[N] = int_0^1 h_i. */
int sdref_nodes(int N, double* xs, double* xf, double* E, double* D, double* w);

/* Mesh from corner geometry and hexahedral connectivity (corner (i,j,k) -> i+2j+4k).
 * periodic: NULL or [3] lengths (0 = not periodic).  geom: 0 straight edges,
 * 1 spherical shell about the origin (constant-radius edges are great-circle arcs). */
sdref_mesh* sdref_mesh_create(int N, int64_t n_v, const double* verts, int64_t n_e, const int64_t* hex,
                              const double* periodic, int geom, double r_in, double r_out,
                              int bc_in, int bc_out);
void sdref_mesh_destroy(sdref_mesh* m);
/* n_boundary_faces, n_interior_face_pairs, h_min */
int sdref_mesh_info(const sdref_mesh* m, int64_t* n_bfaces, int64_t* n_ifaces, double* h_min);
/* face table of element e: nb_e[6], nb_f[6], owner[6], code[6] (orientation code, see sdref.c) */
int sdref_mesh_faces(const sdref_mesh* m, int64_t e, int64_t* nb_e, int32_t* nb_f, int32_t* owner, int32_t* code);
/* geometry of element e: S[3][(N+1)*N*N][3] (family d, point f+(N+1)*(a+N*b)), J[N^3], X[N^3][3],
 * Xp[(p+1)^3][3] polynomial map nodes.  Any output may be NULL. */
int sdref_geometry(sdref_mesh* m, int64_t e, double* S, double* J, double* X, double* Xp);

/* Full residual dQ/dt (physical).  divb[n_e*N^3] and scale[9] (un-cancelled magnitude per variable)
 * may be NULL. */
int sdref_residual(sdref_mesh* m, const sdref_phys* ph, const double* q, double* dqdt, double* divb, double* scale);
/* Residual on a list of elements only; out[list][9][N^3]. */
/* gradients of the primitive variables (u, v, w, T, S, Bx, By, Bz) at the solution points with the
 * BR1 common solution at element faces: grad[e][3 c + j][N^3] = d w_c / d x_j (viscous fluxes) */
int sdref_gradients(sdref_mesh* m, const sdref_phys* ph, const double* q, double* grad);
/* volume sums over bins of radius x colatitude on the shell: out[n_r][n_theta][8] =
 * (volume, V_r, V_theta, V_phi, (B_r^2 + B_theta^2)/2, B_phi^2/2, rho, rho |U|^2/2), each times w |J| */
int sdref_spherical_averages(sdref_mesh* m, const double* q, int n_r, int n_theta, double* out);
/* almost flux-balanced profile (Sec. Initial Conditions) at radii r[n_r]: rho, p; P as for
 * SDREF_INIT_SHELL_FLUX_BALANCED (N_rho, r_b, r_t, rho_b, R, noise, dipole, L, kappa, kappa_r,
 * kappa_r1, kappa_r2): kappa_r(r) = kappa_r + kappa_r1 r + kappa_r2 r^2 */
int sdref_flux_balanced(const double* P, double gam, double GM, int n_nodes, int n_r, const double* r, double* rho,
                        double* p);
int sdref_residual_elements(sdref_mesh* m, const sdref_phys* ph, const double* q, int64_t n_list,
                            const int64_t* elems, double* out, double* scale);
/* One Shu-Osher SSP-RK3 stage: q_out = a_s q_n + b_s (q_in + dt R(q_in)). */
int sdref_rk_stage(sdref_mesh* m, const sdref_phys* ph, int stage, double dt, const double* q_n,
                   const double* q_in, double* q_out);
/* One step of the five-stage third-order SSP method (SSPRK(5,3), coefficients of reading R23):
 * q_out = q^(n+1) from q = q^n; q_out may not alias q. */
int sdref_rk53_step(sdref_mesh* m, const sdref_phys* ph, double dt, const double* q, double* q_out);
int sdref_diagnostics(sdref_mesh* m, const sdref_phys* ph, const double* q, sdref_diag* out);
/* Initial state at the solution points; q_background (NULL allowed) receives the noise-free,
 * field-free hydrostatic background for SHELL_POLYTROPE. */
int sdref_state_init(sdref_mesh* m, const sdref_phys* ph, int kind, const double* params, uint64_t seed,
                     double* q, double* q_background);
/* Polytrope profile (rho, p, T) at radius r: Eq. (polytrop eqns) with T_b. */
int sdref_polytrope(double r, double N_rho, double r_b, double r_t, double rho_b, double R_gas,
                    double gamma, double GM, double* rho, double* p, double* T);
/* Counter-based uniform draw in [-1,1): the (index+1)-th SplitMix64 output of seed. */
double sdref_uniform(uint64_t seed, uint64_t index);
uint64_t sdref_splitmix64(uint64_t seed, uint64_t index);
/* Physical flux in direction n (not normalised), fast speed and Rusanov flux (unit n). */
void sdref_flux(const double* q, const double* n, double gamma, double c_h, double* F);
double sdref_fast_speed(const double* q, const double* n_unit, double gamma);
void sdref_rusanov(const double* qL, const double* qR, const double* n_unit, double gamma, double c_h, double* F);
/* Threads the OpenMP loops over elements use (0 = library default). */
void sdref_set_threads(int n);
int sdref_get_threads(void);

#ifdef __cplusplus
}
#endif
#endif
