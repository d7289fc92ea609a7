/*
 * cmles: C ABI of the B300 (sm_103a) nodal-DG large-eddy-simulation hot path
 * of Sridhar et al., "Large-eddy simulations with ClimateMachine" (GMD 2021/22).
 *
 * The library evaluates the right-hand side of Eq. eom_compact,
 *     dY/dt = -div(F1 + F2) + S(Y),   Y = [rho, rho u, rho v, rho w, rho e_tot, rho q_t],
 * in the semi-discrete nodal-DG form of Eq. matrixProblem on hexahedral
 * Legendre-Gauss-Lobatto elements of order N, and advances it with the
 * five-stage fourth-order low-storage Runge-Kutta scheme of Carpenter and
 * Kennedy (cited in Sec. 3.2).  Every step of that path runs in the library's
 * own CUDA kernels.
 *
 * Conventions for every entry point:
 *  - State arrays are FP64, element-major: Q[e][v][n], v in 0..5 as above,
 *    node n = i + (N+1) (j + (N+1) k) (i along x, j along y, k along z),
 *    element e = ex + nex (ey + ney ez).  E*6*(N+1)^3 doubles.
 *  - "_dev" pointers are CUDA device pointers owned by the caller and only
 *    borrowed for the duration of the call; "_host" pointers are host memory.
 *  - The handle owns its internal device buffers; it is not thread-safe.
 *  - Every call returns a cmles_status and never aborts.  On error,
 *    cmles_last_error_message(h) describes the failure.  Device-side errors
 *    (Newton non-convergence, non-finite values) are counted on the device and
 *    reported by cmles_diagnostics.
 *  - Work is enqueued on the handle's stream (cmles_set_stream; default the
 *    legacy default stream) and is asynchronous unless stated otherwise.
 */
#ifndef CMLES_H
#define CMLES_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cmles_t *cmles_handle;

typedef enum {
  CMLES_OK = 0,
  CMLES_ERR_ARG = 1,       /* invalid argument (null pointer, bad size, unsupported order) */
  CMLES_ERR_OOM = 2,       /* device allocation failed */
  CMLES_ERR_CUDA = 3,      /* a CUDA runtime call failed */
  CMLES_ERR_SATADJ = 4,    /* saturation adjustment did not converge at some node */
  CMLES_ERR_NONFINITE = 5, /* the state holds NaN or Inf */
  CMLES_ERR_MESH = 6,      /* inconsistent mesh description */
  CMLES_ERR_STATE = 7,     /* call out of order (e.g. no reference state yet) */
  CMLES_ERR_TIMEOUT = 8    /* a bounded device-side wait (tensor-core MMA completion) gave up;
                              the results of that launch are invalid, the context stays usable */
} cmles_status;

enum { CMLES_CLOSURE_NONE = 0, CMLES_CLOSURE_SL = 1, CMLES_CLOSURE_MLP = 2, CMLES_CLOSURE_VREMAN = 3 };
/* Numerical flux of F1 on element faces (Sec. 3.1): Rusanov (Eq. nonviscFlux,
 * lambda/2 reading), HLLC (Toro, Spruce & Speares 1994, Davis wave speeds) or
 * Roe (Roe 1981; Jacobian at Roe's averaged state with the frozen moist
 * equation of state, no entropy fix). */
enum { CMLES_FLUX_RUSANOV = 0, CMLES_FLUX_HLLC = 1, CMLES_FLUX_ROE = 2 };
/* Time integrators of cmles_step (Sec. 3.2): the 2N-storage fourth-order
 * explicit schemes with five stages (Carpenter & Kennedy 1994) or fourteen
 * stages and a larger stability region (Niegemann, Diehl & Busch 2012); or
 * HEVI, horizontally explicit and vertically implicit: the three-stage
 * second-order IMEX additive Runge-Kutta method ARK2 of Giraldo, Kelly &
 * Constantinescu (2013) with the vertical acoustic-gravity operator,
 * linearised about the hydrostatic reference and the rest state (linear
 * equation of state of dry air at rest, Rusanov flux at the reference sound
 * speed), implicit, and everything else explicit; each implicit stage is one
 * block-tridiagonal solve per vertical line of nodes (FP64; the stage
 * tendencies in the handle's precision).  HEVI requires a flat mesh and
 * walls at the bottom and top. */
enum { CMLES_LSRK54 = 0, CMLES_LSRK144 = 1, CMLES_ARK2_HEVI = 2 };

/* Arithmetic of the RHS kernels.
 *   CMLES_FP64       all FP64 ("plain" method).
 *   CMLES_FP32_ACC64 volume, face and gradient kernels in FP32 on a state
 *                    stored as FP32 deviations from the hydrostatic reference
 *                    (the reference subtraction done in FP64).  The state
 *                    itself is FP64: within a step the stage increments
 *                    B_s dQ_s are summed in FP32, and the last stage adds the
 *                    sum to the FP64 state and rewrites the FP32 shadow from
 *                    it, so at every step boundary the FP64 state is the
 *                    authority (get_state, diagnostics, checkpoints). */
enum { CMLES_FP64 = 0, CMLES_FP32_ACC64 = 1 };

/* Structured hexahedral mesh of nex x ney x nez elements (Sec. 3.1).  With
 * warp = 1, node heights follow z' = z + z_s(x)(1 - (z - z0)/Lz),
 * z_s(x) = hill_h exp(-((x - hill_xc)/hill_a)^2): elements stacked over the
 * terrain with linear damping to a flat top (Sec. 4.3). */
typedef struct {
  int N;                 /* polynomial order, 1..7 */
  int nex, ney, nez;
  double x0, y0, z0;
  double Lx, Ly, Lz;
  int periodic[3];       /* per direction; non-periodic ends are walls */
  int warp;
  double hill_h, hill_a, hill_xc;
} cmles_mesh;

/* Physical and numerical parameters.  cmles_default_params fills the
 * thermodynamic constants of Table t:constants (Sec. 2.5) and the readings
 * g = 9.81 m s^-2, p0 = 1e5 Pa, p_tr = 611.657 Pa, T_tr = 273.16 K. */
typedef struct {
  double g, p0, Rd, Rv, cvd, cvv, cvl, cvi, T0, Lv0, Lf0, ptr, Ttr;
  int closure;           /* CMLES_CLOSURE_*: Smagorinsky-Lilly (Sec. 4.1), Vreman (Sec. 4.2,
                            Delta_m = h_m / N; flat meshes only) or learned MLP; the
                            Richardson factor multiplies SL and Vreman alike */
  double Cs, Prt;        /* Smagorinsky coefficient, turbulent Prandtl number (1/3) */
  int richardson;        /* apply the Richardson correction f_b (Eq. richardson) */
  int moist;             /* saturation adjustment on (Sec. 2.7) */
  double sponge_alpha, sponge_zs, sponge_gamma; /* Rayleigh sponge (App. A.2) */
  double u_relax[3];
  double lateral_sponge_frac;                   /* also damp within this fraction of Lx at both x ends */
  int surface_flux;      /* bottom wall: prescribed SHF + LHF energy and LHF/L_v0 water flux (App. A.1) */
  double shf, lhf;       /* W m^-2 */
  double Omega[3];       /* rotation vector of the Coriolis term of Eq. momentum */
  int precision;         /* CMLES_FP64 or CMLES_FP32_ACC64 */
  double dt;             /* time step of cmles_step */
  int satadj_max_iter;   /* Newton iteration cap (default 20) */
  int flux;              /* CMLES_FLUX_* (default Rusanov) */
  /* Exponential modal filter (Eq. exponential_filter), applied to the state
   * after every step: mode k of the Legendre expansion along each direction
   * is scaled by exp(-filter_alpha (k/N)^filter_order).  filter_order 0
   * disables it (default); filter_alpha defaults to -ln(2^-52) = 36.04;
   * filter_vars is a bit mask over the six variables and may select only the
   * momentum components (bits 1-3, default all three), whose balanced
   * background is zero. */
  int filter_order;
  double filter_alpha;
  int filter_vars;
  int integrator;        /* CMLES_LSRK54 (default), CMLES_LSRK144 or CMLES_ARK2_HEVI */
  /* Bottom wall (App. A.1): the wall-parallel momentum flux of the
   * aerodynamic drag law (Eq. drag_law), n.(rho tau) = -rho C_d |u_p| u_p,
   * with this constant C_d, n the inward normal, rho the density at the wall
   * node and u_p the wall-parallel velocity at the node of the first
   * interior layer above it; the energy flux is unchanged.  0 (default):
   * free slip.  Negative or non-finite: CMLES_ERR_ARG. */
  double drag_cd;
  /* Wall faces with no-slip velocity (App. A.3): bit f for face f (0 -x,
   * 1 +x, 2 -y, 3 +y, 4 bottom, 5 top).  There the velocity ghost of the
   * face fluxes and of the gradient is u+ = -u- (u_bc = 0), elsewhere the
   * reflection u+ = u- - 2 (n.u-) n; scalars are copied either way and the
   * wall's diffusive fluxes stay those specified (zero, the surface fluxes,
   * the drag law).  Bits of periodic directions have no effect; bits above
   * 5: CMLES_ERR_ARG.  0 (default): free slip everywhere. */
  int noslip;
} cmles_params;

typedef struct {
  double budget[6];      /* domain integrals sum_e sum_n w_n J_n Q_v (FP64 reduction) */
  double time;           /* model time advanced by cmles_step */
  long long steps;       /* steps taken */
  int nonfinite;         /* 1 if the state holds a NaN or Inf */
  int satadj_failures;   /* Newton non-convergence count since the previous call */
  int tc_timeouts;       /* CTAs whose tensor-core completion wait gave up since the previous call */
  int cold_saturated;    /* kernel threads (each counted at most once per launch) whose saturation
                            adjustment left condensate below freezing (273.15 K) since the previous
                            call.  Information, not an error: all condensate is kept liquid (no ice
                            phase), and the status is not changed */
} cmles_diag;

/* Initial-state description for cmles_init_case (synthetic cases; inputs,
 * not part of the method).  id: 1 dry bubble, 2 moist layer, 3 hill flow
 * (warped meshes), 5 throughput box, 11 density current (theta_c/2 (1 +
 * cos(pi r)) with radii r0 in x and r0/2 in z).  modes: nmodes rows (kx, ky, kz, ax, ay, az, phase) of a
 * random-phase velocity field, host memory, may be NULL. */
typedef struct {
  int id;
  uint64_t seed;
  double theta0;
  double dtheta, r0, xc, yc, zc;
  double noise_theta, noise_qt, noise_zmax;
  double NBV;
  double u0[3];
  double qt_sfc, qt_ml, z_ml, qt_top, dthdz_above;
  int moist;
  int nmodes;
  const double *modes;
  double qt_H;
} cmles_case;

/* Apply the exponential filter of the handle's parameters once to the
 * current state (the same operation cmles_step applies after each step when
 * filter_order > 0); asynchronous on the handle's stream.  Errors:
 * CMLES_ERR_ARG when filter_order is 0. */
cmles_status cmles_filter(cmles_handle h);

/* Fill p with the defaults described above (SL closure, FP64, dry, no sponge). */
void cmles_default_params(cmles_params *p);

/* Build LGL nodes, weights and the differentiation matrix (Sec. 3.1,
 * Eqs. expansion, basisDerivatives), the element connectivity, metric terms
 * (Eq. mapping) and sponge tables, and allocate the device work buffers.
 * Errors: CMLES_ERR_ARG (null pointers, N outside the instantiated orders),
 * CMLES_ERR_MESH (non-positive sizes), CMLES_ERR_OOM. */
cmles_status cmles_create(const cmles_mesh *mesh, const cmles_params *params, cmles_handle *out);
cmles_status cmles_destroy(cmles_handle h);
/* Text of the last error on this handle (never NULL; "" when none). */
const char *cmles_last_error_message(cmles_handle h);
/* Stream (cudaStream_t passed as void*) on which all later work is enqueued. */
cmles_status cmles_set_stream(cmles_handle h, void *stream);

/* Hydrostatic reference state p_r, rho_r of Eq. momentum (and the total water
 * q_r of the same profile, used only as the FP32 storage offset).  Host
 * arrays of n values: one per node level (n = nez (N+1), level = ez (N+1) + k)
 * for flat meshes, one per node (n = E (N+1)^3) for warped meshes.
 * qt_r may be NULL (zero).  On the FP32 path with z periodic the reference
 * state must repeat across the wrap (bottom and top levels equal, including
 * rho e_r with its g z, so g = 0): otherwise CMLES_ERR_ARG. */
cmles_status cmles_set_reference(cmles_handle h, const double *rho_r_host, const double *p_r_host,
                                 const double *qt_r_host, size_t n);

/* Evaluate a synthetic initial state on the device and set the reference
 * state of that case (hydrostatic profiles of Eqs. pressureDistrib,
 * pressure_hs_brunt and density_hs_brunt, or RK4 integration for moist
 * profiles; seeded SplitMix64 noise).  Replaces cmles_set_reference. */
cmles_status cmles_init_case(cmles_handle h, const cmles_case *c);

/* Copy a state into / out of the handle (device buffers, layout above). */
cmles_status cmles_set_state(cmles_handle h, const double *Q_dev);
cmles_status cmles_get_state(cmles_handle h, double *Q_dev);
/* Same with host buffers; the copies run on the handle's stream and the call
 * returns after they complete (pinned host memory gives full PCIe speed). */
cmles_status cmles_set_state_host(cmles_handle h, const double *Q_host);
cmles_status cmles_get_state_host(cmles_handle h, double *Q_host);

/* Double-buffered upload of host states, so that a step can run while the
 * next state is copied.  cmles_stage_state_host starts an asynchronous copy
 * of Q_host (same layout; pinned memory for full speed, and it must stay
 * unchanged until the copy is committed) into the handle's staging buffer on
 * an internal copy stream, after the work already queued on the handle's
 * stream, and returns at once.  cmles_commit_staged_state makes the handle's
 * stream wait for that copy and takes the staged state as the handle's state,
 * as cmles_set_state would; the previous state buffer becomes the next
 * staging buffer.  The staging buffer (one state) is allocated at the first
 * call.  Errors: CMLES_ERR_ARG, CMLES_ERR_OOM, CMLES_ERR_CUDA; commit without
 * a staged copy gives CMLES_ERR_STATE. */
cmles_status cmles_stage_state_host(cmles_handle h, const double *Q_host);
cmles_status cmles_commit_staged_state(cmles_handle h);

/* Asynchronous download of the state, the counterpart of the staged upload.
 * cmles_fetch_state_host starts copying the handle's current state (after
 * the work already queued on the handle's stream) into Q_host (same layout;
 * pinned memory for full speed) on an internal copy stream, in 32 chunks,
 * and returns at once; cmles_wait_fetch blocks until the latest download
 * has completed (at once if there is none).  Q_host must not be read or
 * changed by the caller before cmles_wait_fetch returns.  A
 * cmles_stage_state_host of the same host buffer that follows uploads each
 * chunk as soon as it has arrived, so that the two directions of a host
 * round trip overlap on the bus; cmles_set_state_host and
 * cmles_get_state_host of that buffer wait for the whole download.  Calls
 * that change a state buffer (set_state, set_state_host, commit, init_case,
 * step, filter) are ordered after the download on the device, without
 * blocking the host.  Errors: CMLES_ERR_ARG, CMLES_ERR_CUDA. */
cmles_status cmles_fetch_state_host(cmles_handle h, double *Q_host);
cmles_status cmles_wait_fetch(cmles_handle h);

/* RHS of Eq. matrixProblem for the state Q (device, FP64) into RHS (device,
 * FP64, same layout), in the handle's precision.  The handle's own state is
 * left unchanged. */
cmles_status cmles_tendency(cmles_handle h, const double *Q_dev, double *RHS_dev);

/* Advance the handle's state by nsteps steps of params.dt of the chosen
 * integrator (params.integrator: LSRK(5,4), LSRK(14,4) or ARK2 HEVI).  Each
 * explicit stage is two kernels: the gradient/closure pass and the flux-divergence pass
 * with the fused stage update; with filter_order > 0 the exponential filter
 * follows every step.  Every step starts from the FP64 state alone (the first
 * stage has A = 0), so a state saved between calls resumes bit-identically.
 * Asynchronous. */
cmles_status cmles_step(cmles_handle h, int nsteps);

/* FP64 budgets, non-finite flag and Newton failures of the current state.
 * Synchronises the handle's stream.  Returns CMLES_ERR_NONFINITE or
 * CMLES_ERR_SATADJ when those occurred (out is filled in either case). */
cmles_status cmles_diagnostics(cmles_handle h, cmles_diag *out);

/* Favre (density-weighted) horizontal means of the current state per node
 * level (App. C), flat meshes only.  out_host receives nez (N+1) rows of 11
 * values: <rho>, theta, q_t, q_l, u, v, w, w'w', w'theta', w'q_t', theta_l.
 * Synchronises the stream. */
cmles_status cmles_profiles(cmles_handle h, double *out_host);

/* Kinetic-energy spectrum of the current state (the turbulence diagnostic of
 * Sec. 5.5, a Fourier transform of the velocity field), on a flat mesh
 * periodic in x and y; synchronises the stream.  Readings: velocity
 * u = (rho u)/rho at the nodes; resampled onto a uniform grid of N points per
 * element and direction at the cell centres xi_s = -1 + (2s+1)/N of each
 * element (M_x = nex N, M_y = ney N points per level, M_z = nez N levels)
 * with the element's Lagrange polynomial; per level the discrete Fourier
 * coefficients u^(p,q) = 1/(M_x M_y) sum_ij u_ij exp(-2 pi i (p i/M_x +
 * q j/M_y)); E_host[s] (s < nshell) = the level average of the sum of
 * (|u^|^2 + |v^|^2 + |w^|^2)/2 over the shell s = round(L sqrt((p/L_x)^2 +
 * (q/L_y)^2)), L = max(L_x, L_y); higher shells are dropped.  By Parseval the
 * sum over all shells is the grid mean of |u|^2/2.  FP64 throughout; the call
 * allocates its scratch (the grid and two transforms, 9 doubles per grid
 * point) on the handle's stream.  Errors: CMLES_ERR_ARG (nshell < 1, warped,
 * partitioned or not periodic in x and y), CMLES_ERR_CUDA. */
cmles_status cmles_spectrum(cmles_handle h, int nshell, double *E_host);

/* Learned SGS closure (not in the paper; an extension of Sec. 4):
 * a per-node network 13 -> 64 -> 64 -> 2 with SiLU hidden activations, BF16
 * weights and activations and FP32 accumulation on tensor cores, evaluated
 * inside the FP32 gradient pass when params.closure == CMLES_CLOSURE_MLP
 * (FP32_ACC64 precision only).  Inputs: the nine velocity gradients
 * du_i/dx_j (index 3i+j), the three theta_v gradients and Delta, each times
 * in_scale; outputs nu_t = out_scale[0] max(y0, 0), D_t = out_scale[1] max(y1, 0).
 * Parameter vector (FP32, 5201 values): W1[64][13], b1[64], W2[64][64],
 * b2[64], W3[2][64], b3[2], in_scale[13], out_scale[2] (weights out-major).
 * cmles_set_closure_weights takes it from host memory (n must be 5201),
 * cmles_set_closure_weights_device from device memory (e.g. after training). */
cmles_status cmles_set_closure_weights(cmles_handle h, const float *params_host, size_t n);
cmles_status cmles_set_closure_weights_device(cmles_handle h, const float *params_dev);

/* Training kernels of the closure network on device buffers (no handle):
 * cmles_mlp_forward: Y[n][2] = network(X[n][13]) on the tcgen05 tensor cores
 *   (BF16 operands, FP32 accumulation, biases folded into the contraction);
 *   synchronises the stream and returns CMLES_ERR_TIMEOUT if an MMA
 *   completion wait gave up; n = 0 returns CMLES_OK at once (the pointers
 *   may then be null).
 * cmles_mlp_loss_grad: loss = 1/(2n) sum |y - t|^2 over T[n][2] and its
 *   gradient with respect to the first 5186 parameters (W1 .. b3), written
 *   to grad_dev[5186] and loss_dev[1] (both overwritten); forward and
 *   backward products on the tcgen05 tensor cores; synchronises the stream
 *   and returns CMLES_ERR_TIMEOUT if an MMA completion wait gave up.
 * cmles_mlp_adam: one Adam step (Kingma & Ba 2015) of those 5186 parameters
 *   with moment buffers m_dev, v_dev (5186 each, zero at t = 1); t >= 1.
 * All run on `stream`; errors CMLES_ERR_ARG (null/size), CMLES_ERR_CUDA. */
cmles_status cmles_mlp_forward(const float *params_dev, const float *X_dev, float *Y_dev, long long n, void *stream);
cmles_status cmles_mlp_loss_grad(const float *params_dev, const float *X_dev, const float *T_dev, long long n,
                                 float *grad_dev, float *loss_dev, void *stream);
cmles_status cmles_mlp_adam(float *params_dev, const float *grad_dev, float *m_dev, float *v_dev, int t, float lr,
                            float beta1, float beta2, float eps, void *stream);

/* Training samples for the learned closure from the handle's current state
 * (a fine-resolution run; flat meshes).  The paper has no learned closure;
 * these targets extend its Sec. 4.  The fine field's velocity and theta_v
 * (FP64 thermodynamics of Sec. 2) are top-hat filtered, width one coarse node
 * spacing H / N, onto the nodes of the mesh coarser by `factor` in every
 * direction (element counts must be multiples of factor): each fine node (a
 * node on a shared face once per element) within H / (2N) of the coarse node
 * in every direction, the edge included, weighs its LGL quadrature weight;
 * periodic directions wrap, walls cut the box.  Per coarse node (coarse
 * element-major, node-minor): X_dev[13] = filtered du_i/dx_j (index 3i+j,
 * element-local derivatives), filtered d theta_v/dx_j (3), Delta_c =
 * (H_x H_y H_z)^(1/3) / N; T_dev[2] = least-squares eddy viscosity and
 * diffusivity max(0, -tau:S/(2 S:S)), max(0, -tau_th.g/|g|^2) from the
 * filtered subgrid stress tau_ij = <u_i u_j> - <u_i><u_j> and theta_v flux
 * tau_th,j = <u_j th> - <u_j><th>, S the symmetric part of the filtered
 * velocity gradient and g the filtered theta_v gradient (0 where S or g
 * vanishes); thv_dev (may be NULL) = filtered theta_v.  Device FP32 outputs;
 * the call allocates its FP64 scratch (4 values per fine node) on the
 * handle's stream.  *n_out receives the sample count; CMLES_ERR_ARG if
 * capacity is smaller or the mesh is warped. */
cmles_status cmles_closure_samples(cmles_handle h, int factor, float *X_dev, float *T_dev, float *thv_dev,
                                   long long capacity, long long *n_out);

/* Per-kernel timing: when enabled, every launch is bracketed by CUDA events
 * on the handle's stream; cmles_kernel_times returns, for the kernels
 * launched since the last reset, count[k] and total milliseconds[k] for
 * k = 0 gradient pass, 1 flux/update pass, 2 other kernels, and the total
 * number of kernel launches.  Synchronises the stream. */
cmles_status cmles_enable_timing(cmles_handle h, int enable);
cmles_status cmles_kernel_times(cmles_handle h, long long count[3], double ms[3], long long *launches);
/* Kernel launches issued by this handle since creation (always counted). */
long long cmles_launch_count(cmles_handle h);

/* The HEVI pieces of a handle created with CMLES_ARK2_HEVI (Sec. 3.2), on
 * device states in the layout of cmles_set_state:
 * cmles_hevi_operator: out = L (Q - Q_ref), the vertical linear operator
 *   (all six components; Q_ref = (rho_r, 0, 0, 0, rho e_r, 0) with
 *   rho e_r = rho_r (c_vm (T_r - T_0) + q_r I_v0 + g z), T_r = p_r/(rho_r R_m),
 *   the mixture constants at the reference total water q_r given to
 *   cmles_set_reference, 0 if none).
 * cmles_hevi_solve: Y = Q_ref + (I - dt gamma L)^-1 (B - Q_ref) with
 *   gamma = 1 - 1/sqrt 2 and the handle's dt; B and Y must differ.
 * Asynchronous; CMLES_ERR_STATE for another integrator or no reference. */
cmles_status cmles_hevi_operator(cmles_handle h, const double *Q_dev, double *out_dev);
cmles_status cmles_hevi_solve(cmles_handle h, const double *B_dev, double *Y_dev);

/* Test hook for the failure path of the bounded device-side waits (no GPU
 * fault involved), in the learned-closure gradient pass:
 *   mode 1: each CTA also waits, with a bound, on an mbarrier that nothing
 *           arrives on; the wait runs out, the CTA finishes its work
 *           (results intact), frees its Tensor Memory and is counted;
 *   mode 2: each CTA's first MMA completion wait gives up at once, while its
 *           MMA is still in flight (a test instance of the pass); the CTA
 *           issues no further MMA, reads no Tensor Memory (results invalid),
 *           and at its tear-down waits (bounded) for that MMA's completion
 *           before freeing the columns.  The test instance exists for the
 *           128-thread CTAs of N <= 4; above, mode 2 gives CMLES_ERR_ARG.
 * Either way the next cmles_diagnostics returns CMLES_ERR_TIMEOUT with
 * cmles_diag.tc_timeouts = the number of CTAs that gave up (each counted
 * once).  Mode 0 restores normal operation; other values give
 * CMLES_ERR_ARG. */
cmles_status cmles_test_stall_tc(cmles_handle h, int mode);

/* Allocation-free budgets.  The paper has no counterpart: this is a service
 * for callers that cannot call cudaMalloc, such as applications whose own
 * pool allocator owns all device memory, or time-stepping loops that cannot
 * accept the device-wide synchronisation cudaMalloc/cudaFree imply.  It
 * computes the same FP64 quadrature sums as cmles_diagnostics,
 * out_dev[v] = sum_e sum_n w_n J Q_v for v = 0..5 and out_dev[6] = number of
 * non-finite entries, for a caller-owned device state Q_dev (layout above) of
 * a flat mesh with constant element Jacobian `jacobian` (h_x h_y h_z / 8), on
 * `stream`.  No handle is needed and nothing is allocated: the block partial
 * sums live in a file-scope device array of 2 MiB that every GPU loading the
 * library keeps until exit.  Limits: 1 <= N <= 7 and at most 2,097,152
 * elements; larger sizes return CMLES_ERR_ARG without launching.  The first
 * call on each device looks up the array's device address (with that device
 * current) and should come before any stream capture; the address is cached
 * for the life of the loaded library, so after cudaDeviceReset the library
 * must be loaded again (a new process) before this call is used on that
 * device.  All calls share the
 * array, so calls that overlap on the GPU race: serialise them.  Errors:
 * CMLES_ERR_ARG (null pointers, sizes), CMLES_ERR_CUDA (lookup, or the launch
 * of one of its two kernels; an earlier non-sticky error of other code is
 * left for that code to read). */
cmles_status cmles_budgets_noalloc(const double *Q_dev, long long num_elements, int N, double jacobian,
                                   double *out_dev, void *stream);

/* ---- Domain decomposition (Sec. 3.1: the element loop split over
 * partitions that exchange the face data their neighbours need) ----
 *
 * A cmles_group is one mesh split into px x py pencils of whole element
 * columns (x and y; every partition keeps all nez layers), each partition a
 * set of device buffers of its own: its interior elements plus one ghost
 * element on each side in x and y.  Every explicit stage makes two halo
 * exchanges: before the gradient pass, the state and its four thermodynamic
 * fields at the face nodes of the partition's boundary elements; before the
 * flux pass, the five components of the diffusive flux F2 of the face's
 * direction.  An exchange packs each side's face nodes into a send buffer (a
 * kernel), copies it into the neighbouring partition's receive buffer and
 * unpacks it into that partition's ghost elements (a kernel).  All
 * partitions live on the calling thread's current GPU and the copies are
 * device-to-device on the group's stream: the single-GPU form of the
 * decomposition, in which a multi-GPU run would replace each copy with a
 * point-to-point send and receive.  Results are bit-identical to the whole
 * mesh's handle (every element runs the same kernels on the same values);
 * budgets are summed over partitions, so they agree to rounding.
 *
 * Scope: flat meshes, both precisions, every closure and numerical flux, the
 * explicit integrators (LSRK(5,4), LSRK(14,4)); no exponential filter, HEVI
 * or warped meshes (CMLES_ERR_ARG).  px <= nex and py <= ney; element columns
 * are split into nearly equal runs (the first nex mod px partitions in x get
 * one more), partition rank = ix + px iy.  State arrays passed to the group
 * calls use the whole mesh's layout of the conventions above. */
typedef struct cmles_group_t *cmles_group;
cmles_status cmles_group_create(const cmles_mesh *mesh, const cmles_params *params, int px, int py,
                                cmles_group *out);
cmles_status cmles_group_destroy(cmles_group g);
const char *cmles_group_last_error_message(cmles_group g);
/* The stream of every partition's work and of the exchanges' copies. */
cmles_status cmles_group_set_stream(cmles_group g, void *stream);
/* As cmles_set_reference and cmles_set_closure_weights, for every partition
 * (the reference is per node level, which the (x, y) split does not cut). */
cmles_status cmles_group_set_reference(cmles_group g, const double *rho_r_host, const double *p_r_host,
                                       const double *qt_r_host, size_t n);
cmles_status cmles_group_set_closure_weights(cmles_group g, const float *params_host, size_t n);
/* Scatter a whole-mesh device state into the partitions / gather it back. */
cmles_status cmles_group_set_state(cmles_group g, const double *Q_dev);
cmles_status cmles_group_get_state(cmles_group g, double *Q_dev);
/* As cmles_tendency and cmles_step, with the halo exchanges. */
cmles_status cmles_group_tendency(cmles_group g, const double *Q_dev, double *RHS_dev);
cmles_status cmles_group_step(cmles_group g, int nsteps);
/* As cmles_diagnostics: budgets and failure counts summed over the
 * partitions (the allreduce of a multi-GPU run).  Synchronises the stream. */
cmles_status cmles_group_diagnostics(cmles_group g, cmles_diag *out);
/* Bytes the halo exchanges of one stage move between partitions. */
long long cmles_group_halo_bytes(cmles_group g);
/* Host-only (no GPU needed): the halo plan of partition `rank` of a px x py
 * split of `mesh`, the one the group uses.  For each side s (0 -x, 1 +x,
 * 2 -y, 3 +y): neighbour[s] = the partition across that side (the partition
 * itself across a periodic boundary when it spans the mesh; -1 at a wall)
 * and count[s] face nodes.  send_index and recv_index (may be NULL; else
 * room for count[0] + .. + count[3] entries) receive, side after side, the
 * partition's storage node indices e Np + n (storage element e = (ex + 1) +
 * (nx + 2) ((ey + 1) + (ny + 2) ez) of the interior coordinates ex, ey, ez,
 * -1 and nx / ny being the ghosts; nx x ny interior columns): send = the face
 * nodes of its boundary elements on side s, in the order the neighbour across
 * s receives them into its side s ^ 1; recv = the ghost nodes on side s that
 * the neighbour's send on side s ^ 1 fills, entry for entry.  Order within a
 * side: element layer ez, then the element's index along the side, then the
 * face node t1 + (N+1) t2 (the two in-face indices in x, y, z order).
 * Errors: CMLES_ERR_ARG for a bad split, order or null counts. */
cmles_status cmles_halo_plan(const cmles_mesh *mesh, int px, int py, int rank, int neighbour[4], long long count[4],
                             long long *send_index, long long *recv_index);

/* Sizes of the handle's problem. */
long long cmles_num_elements(cmles_handle h);
long long cmles_num_nodes(cmles_handle h);
/* Device bytes held by the handle's buffers. */
long long cmles_device_bytes(cmles_handle h);

#ifdef __cplusplus
}
#endif
#endif
