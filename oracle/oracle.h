/*
 * Plain FP64 CPU oracle for the nodal-DG large-eddy-simulation right-hand side
 * of Sridhar et al., "Large-eddy simulations with ClimateMachine" (GMD).
 *
 * TEST INFRASTRUCTURE ONLY.  This code is the correctness reference for the
 * CUDA path.  It shares no code, header, table or constant generator with the
 * product library; the product never links, loads or calls it.  Only the
 * tests, the smoke check and the benchmark's CPU-baseline leg use it.
 *
 * Everything here is written as plain loops in the order of the paper:
 *   Sec. 2   thermodynamics, equation of state, saturation adjustment
 *   Sec. 3.1 nodal DG on LGL hexahedra (Eqs. expansion .. matrixProblem),
 *            Rusanov flux (Eq. nonviscFlux), BR1 auxiliary gradient
 *   Sec. 3.2 low-storage Runge-Kutta (Carpenter & Kennedy 1994, 5 stages)
 *   Sec. 4   Smagorinsky-Lilly and Vreman closures with the Richardson correction
 *   App. A   wall boundary conditions, prescribed wall fluxes, Rayleigh sponge
 *   App. C   Favre (density-weighted) horizontal means
 * Readings where the paper is silent or garbled are stated at the point of
 * use.
 *
 * Compiled with -O2 -ffp-contract=off (IEEE round-to-nearest, no FMA).
 */
#ifndef CMLES_ORACLE_H
#define CMLES_ORACLE_H

#include <stdint.h>

#define ORC_MAXQ 9  /* N <= 8 */

/* Closure kinds. */
#define ORC_CLOSURE_NONE 0
#define ORC_CLOSURE_SL 1
#define ORC_CLOSURE_MLP 2
#define ORC_CLOSURE_VREMAN 3
#define ORC_FLUX_RUSANOV 0
#define ORC_FLUX_HLLC 1
#define ORC_FLUX_ROE 2

typedef struct {
  int N;                      /* polynomial order */
  int nex, ney, nez;          /* elements per direction */
  double x0, y0, z0;          /* domain origin */
  double Lx, Ly, Lz;          /* domain extents */
  int periodic_x, periodic_y, periodic_z;
  int warp;                   /* 1: terrain-following Gaussian ridge */
  double hill_h, hill_a, hill_xc;
} orc_mesh;

typedef struct {
  /* thermodynamic constants (Table t:constants) and the readings for g, p0, p_tr, T_tr */
  double g, p0, Rd, Rv, cvd, cvv, cvl, cvi, T0, Lv0, Lf0, ptr, Ttr;
  /* closure */
  int closure;                /* ORC_CLOSURE_* */
  double Cs, Prt;
  int richardson;
  int moist;                  /* 1: saturation adjustment, 0: q_l = 0 always */
  /* Rayleigh sponge (App. A.2) */
  double sponge_alpha, sponge_zs, sponge_gamma;
  double u_relax[3];
  double lateral_sponge_frac; /* >0: also damp within this fraction of Lx at both x ends */
  /* prescribed bottom-wall fluxes (App. A.1, BOMEX-style SHF/LHF) */
  int surface_flux;
  double shf, lhf;
  double Omega[3];            /* planetary rotation for the Coriolis term */
  int flux;                   /* ORC_FLUX_*: numerical flux of F1 on faces (Sec. 3.1) */
  /* bottom wall: wall-parallel momentum flux by the aerodynamic drag law
   * (Eq. drag_law) with this constant C_d; 0: free slip */
  double drag_cd;
  /* wall faces (bit f: 0 -x, 1 +x, 2 -y, 3 +y, 4 bottom, 5 top) where the
   * velocity ghost is no-slip, u+ = -u- (App. A.3, u_bc = 0), instead of the
   * reflection of the normal component */
  int noslip;
} orc_params;

typedef struct orc_solver orc_solver;

/* ---- LGL basis (Sec. 3.1) ---- */
void orc_lgl(int N, double *xi, double *w, double *D /* (N+1)^2, row-major D[i][j] = L_j'(xi_i) */);

/* ---- thermodynamics (Sec. 2) ---- */
double orc_pvsat(const orc_params *p, double T);
double orc_qsat(const orc_params *p, double T, double rho);
/* Saturation adjustment: given rho, q_t and specific internal energy I,
 * returns T and q_l; returns number of Newton iterations (0 when unsaturated),
 * or -1 when the iteration did not converge. */
int orc_saturation_adjustment(const orc_params *p, double rho, double qt, double I, double *T, double *ql);
/* Internal energy I(T, q_t, q_l) of Eq. total_internal_energy (q_i = 0). */
double orc_internal_energy(const orc_params *p, double T, double qt, double ql);

/* Pointwise diagnostic state of one node from its conserved variables. */
typedef struct {
  double rho, u[3], qt, etot, I, T, ql, qv, Rm, cvm, cpm, p, c, htot, theta, thetav;
  int newton;
} orc_thermo_state;
int orc_thermo(const orc_params *p, const double Y[6], double z, orc_thermo_state *s);

/* ---- fluxes ---- */
/* Normal inviscid flux n.F1(Y) (Eq. eom_compact, Sec. 2) given p_r at the node. */
void orc_flux1_normal(const orc_params *p, const double Y[6], double z, double pr, const double n[3], double out[6]);
/* Rusanov numerical flux n.F1* (Eq. nonviscFlux, standard 1/2 lambda reading). */
void orc_rusanov(const orc_params *p, const double Ym[6], const double Yp[6], double z, double pr,
                 const double n[3], double out[6]);

/* HLLC numerical flux n.F1* (Toro, Spruce & Speares 1994; named in Sec. 3.1),
 * Davis wave-speed estimates (reading). */
void orc_hllc(const orc_params *p, const double Ym[6], const double Yp[6], double z, double pr, const double n[3],
              double out[6]);

/* Roe numerical flux n.F1* (Roe 1981; named in Sec. 3.1): flux Jacobian at
 * Roe's averaged state with the frozen (q_l = 0) moist equation of state
 * (reading), no entropy fix. */
void orc_roe(const orc_params *p, const double Ym[6], const double Yp[6], double z, double pr, const double n[3],
             double out[6]);

/* ---- exponential filter (Eq. exponential_filter) ---- */
/* One-dimensional filter matrix F = V diag(exp(-alpha (k/N)^order)) V^-1,
 * V_ik = P_k(xi_i), row-major (N+1)^2. */
void orc_filter_matrix(int N, const double *xi, int order, double alpha, double *F);
/* Apply the filter in place to the variables of Q [E][6][Np] selected by
 * mask (bit v for variable v). */
void orc_filter(orc_solver *s, double *Q, int order, double alpha, int mask);

/* ---- closure (Sec. 4) ---- */
/* Smagorinsky-Lilly nu_t from the velocity gradient gu[i][j] = du_i/dx_j,
 * d(theta_v)/dz, theta_v and Delta (Eqs. smago, richardson). */
double orc_smagorinsky(const orc_params *p, const double gu[9], double dthvdz, double thv, double Delta);
/* Vreman nu_t (Eq. vreman-sgs) from the velocity gradient gu[i][j] = du_i/dx_j
 * and the directional lengths Dm[m] = L_m / N, times the same Richardson
 * factor as Smagorinsky-Lilly when p->richardson is set (reading: the
 * correction multiplies "the eddy viscosity" of either model). */
double orc_vreman(const orc_params *p, const double gu[9], double dthvdz, double thv, const double Dm[3]);

/* ---- solver ---- */
orc_solver *orc_create(const orc_mesh *m, const orc_params *p);
void orc_destroy(orc_solver *s);
int64_t orc_num_nodes(const orc_solver *s);
int orc_num_elements(const orc_solver *s);
/* Node coordinates, Jacobian and quadrature weight w_i*J_i, each [E][Np]. */
void orc_geometry(const orc_solver *s, double *x, double *y, double *z, double *J, double *wJ);
/* Reference state p_r, rho_r per node [E][Np] (hydrostatic; set by the caller). */
void orc_set_reference(orc_solver *s, const double *rho_r, const double *p_r);
/* MLP closure weights (FP64 copy of the network), used when closure == MLP. */
void orc_set_mlp(orc_solver *s, const double *W1, const double *b1, const double *W2, const double *b2,
                 const double *W3, const double *b3, const double *in_scale, const double *out_scale);

/* RHS of Eq. matrixProblem for state Q [E][6][Np]; RHS same layout.
 * form: 0 strong form (default), 1 weak form (integration by parts of the
 * volume flux term, Eq. weakDG2); both must agree under LGL collocation.
 * Returns number of nodes where saturation adjustment failed (0 normally). */
int orc_rhs(orc_solver *s, const double *Q, double *RHS, int form);
/* Intermediates of the last orc_rhs call: per node [E][k][Np] arrays.
 * G: (u,v,w,h_tot,q_t,theta_v) (6); gradG: [6][3]; nu_t (1); F2: [dir 3][5]
 * (rho d_qt, rho tau_i. + d_i rho u_. (3), energy); aux: (p - p_r, c, T, q_l). */
void orc_intermediates(const orc_solver *s, double *G, double *gradG, double *nut, double *F2, double *aux);

/* LSRK(5,4) of Carpenter & Kennedy (1994): advance Q in place by nsteps of dt. */
int orc_lsrk54(orc_solver *s, double *Q, int nsteps, double dt);
void orc_lsrk54_coefficients(double A[5], double B[5], double c[5]);
int orc_lsrk144(orc_solver *s, double *Q, int nsteps, double dt);
/* HEVI (Sec. 3.2): the vertical acoustic-gravity operator linearised about
 * the reference (hevi.c); flat meshes. */
void orc_set_reference_qt(orc_solver *s, const double *qt_r /* [E][Np] */);
void orc_vlin_reference(orc_solver *s, double *Qref);
void orc_vlin_apply(orc_solver *s, const double *Q, double *out);
void orc_lsrk144_coefficients(double A[14], double B[14], double c[14]);

/* Global budgets sum_e sum_i w_i J_i Q_v for all 6 variables; returns 1 if any
 * entry of Q is non-finite. */
int orc_budgets(const orc_solver *s, const double *Q, double out[6]);
/* Favre means per horizontal node level (box meshes): out[level][k] for
 * k = 0 rho-mean, 1 theta_bar, 2 q_t bar, 3 q_l bar, 4 u bar, 5 v bar, 6 w bar,
 * 7 w'w' variance, 8 w'theta' flux, 9 w'q_t' flux, 10 theta_l bar.
 * Number of levels = nez*(N+1). */
void orc_favre_profiles(const orc_solver *s, const double *Q, double *out);

/* ---- initial conditions (case set-up, inputs for tests) ---- */
/* Counter-based uniform [0,1): SplitMix64 (Steele, Lea & Flood 2014) output
 * number `counter` of the generator seeded with `seed`. */
double orc_uniform(uint64_t seed, uint64_t counter);
/* Case ids: 1 dry bubble, 2 moist layer, 3 hill flow, 5 throughput box,
 * 10 isentropic vortex (dry, g = 0), 11 density current.
 * `modes` is the random-phase velocity table for case 5: nmodes rows of
 * (kx, ky, kz, ax, ay, az, phase); may be NULL otherwise.  Writes Q [E][6][Np]
 * and the hydrostatic reference rho_r, p_r [E][Np]. */
typedef struct {
  int id;
  uint64_t seed;
  double theta0;              /* surface / background potential temperature */
  double dtheta, r0, xc, yc, zc;  /* bubble */
  double noise_theta, noise_qt, noise_zmax;
  double NBV;                 /* Brunt-Vaisala frequency for stratified cases */
  double u0[3];               /* uniform background velocity */
  double qt_sfc, qt_ml, z_ml, qt_top, dthdz_above;  /* moist layer */
  double vortex_beta, vortex_R, vortex_U, vortex_T, vortex_rho;  /* isentropic vortex */
  int moist;
  int nmodes;
  const double *modes;
  double qt_H;                /* scale height of q_t for the moist throughput box */
} orc_case;
void orc_init_case(orc_solver *s, const orc_case *c, double *Q, double *rho_r, double *p_r);
/* Exact isentropic-vortex state at time t (translating with vortex_U along x). */
void orc_vortex_exact(orc_solver *s, const orc_case *c, double t, double *Q);

/* ---- learned closure network, FP64 (gradient checks of the GPU kernels) ---- */
/* 13 -> 64 -> 64 -> 2, SiLU hidden activations, linear output.
 * W1 [64][13], W2 [64][64], W3 [2][64] row-major (out, in). */
void orc_mlp_forward(int n, const double *X /*[n][13]*/, const double *W1, const double *b1,
                     const double *W2, const double *b2, const double *W3, const double *b3,
                     double *Y /*[n][2]*/);
/* BF16 rounding (FP32 first, then round-to-nearest-even to 8 significand bits). */
double orc_bf16(double x);
/* The closure network with BF16 inputs and hidden activations (the learned
 * closure's definition); used by orc_rhs when closure == MLP. */
void orc_mlp_forward_bf16(int n, const double *X, const double *W1, const double *b1, const double *W2,
                          const double *b2, const double *W3, const double *b3, double *Y);
/* Mean-squared-error loss 1/(2n) sum |Y - T|^2 and its gradients. */
double orc_mlp_loss_grad(int n, const double *X, const double *T, const double *W1, const double *b1,
                         const double *W2, const double *b2, const double *W3, const double *b3,
                         double *gW1, double *gb1, double *gW2, double *gb2, double *gW3, double *gb3);
/* One Adam step (Kingma & Ba 2015) on a flat parameter vector. */
void orc_adam(int n, double *theta, const double *g, double *m, double *v, int t,
              double lr, double beta1, double beta2, double eps);

/* ---- learned-closure training samples (closure.c; the paper has no learned
 * closure: these follow the readings stated there) ---- */
/* u, v, w and theta_v of every node's thermodynamic state, prim[E][4][Np]. */
void orc_closure_primitives(const orc_solver *s, const double *Q, double *prim);
/* Top-hat filter of the primitive field onto the nodes of the mesh coarser by
 * `factor` (flat meshes): X[n][13] network inputs, T[n][2] least-squares
 * (nu*, kappa*), thv_bar[n] filtered theta_v (may be NULL).  Returns the
 * sample count, or -1 if the element counts are not multiples of factor. */
long long orc_closure_samples(const orc_solver *s, const double *prim, int factor, double *X, double *T,
                              double *thv_bar);

#endif
