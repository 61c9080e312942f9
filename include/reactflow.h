/*
 * reactflow.h -- C ABI of the B300 reacting-flow right-hand-side library.
 *
 * The library evaluates the explicit right-hand side of the multicomponent
 * reacting Navier-Stokes equations on a uniform Cartesian grid and advances it
 * with SSP-RK3 (paper: Methods, Governing equations; Methods, Numerical method).
 * Each RHS evaluation recovers primitives (temperature by a Newton solve on the
 * NASA polynomial fits), evaluates Wilke / mixture-averaged transport,
 * reversible Arrhenius chemistry and a Gaussian laser source, and adds the
 * divergence of WENO3-Z local-Lax-Friedrichs inviscid fluxes and second-order
 * central viscous, heat and species-diffusion fluxes.
 *
 * Conventions
 *  - Every entry point returns int: RF_OK (0) or a negative RF_E* code; no C++
 *    exception, trap or device assert crosses the ABI.  rf_last_error() gives a
 *    thread-local message for the last failing call on this thread.
 *  - Arrays marked "device" are CUDA device pointers owned by the caller (for
 *    example torch tensors); the library never frees them.  Arrays marked "host"
 *    are read during the call only.
 *  - Field layout: structure of arrays, variable-major, x fastest:
 *    a[v][k][j][i] at offset v*N + (k*ny + j)*nx + i, N = nx*ny*nz.
 *    Conserved variables U (nv = Ns + 4 fields, FP64):
 *    rho*Y_1 .. rho*Y_Ns [kg/m^3], rho*u, rho*v, rho*w [kg/m^2/s], E [J/m^3]
 *    (total energy including formation enthalpy).  T: one FP64 field [K].
 *  - Device work is enqueued on the caller's stream and is asynchronous.
 *    Run-time failures detected on the device (Newton non-convergence,
 *    non-finite values, temperature out of range, a bounded wait that ran out)
 *    are recorded in a per-context status word; rf_status() synchronises the
 *    stream, returns the matching RF_E* code and clears the word.
 *  - SI units throughout.
 */
#ifndef REACTFLOW_H
#define REACTFLOW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *rf_stream;       /* = cudaStream_t */

enum rf_code {
    RF_OK = 0,
    RF_EINVAL = -1,       /* bad argument: null pointer, size, unsupported species count ... */
    RF_ENEWTON = -2,      /* temperature Newton solve did not converge in some cell */
    RF_ENONFINITE = -3,   /* NaN or Inf met in the state or its derived quantities */
    RF_ERANGE = -4,       /* temperature or density outside the admissible range */
    RF_ECUDA = -5,        /* a CUDA runtime call failed (message names it) */
    RF_ETIMEOUT = -6,     /* a bounded device-side wait gave up */
    RF_ENOMEM = -7        /* device allocation failed */
};

enum rf_precision {
    RF_FP64 = 0,          /* every operation in FP64 */
    RF_MIXED = 1          /* FP32 bulk arithmetic; FP64 for the temperature Newton solve,
                             Gibbs-energy equilibrium constants and reverse rates, and
                             the conserved-variable stage accumulation (its exponentials
                             and ln T to 2e-13 / 5e-14, the time-step estimate's rate
                             derivatives as FP32 mantissas with integer exponents) */
};

enum rf_bc {
    RF_BC_PERIODIC = 0,
    RF_BC_EXTRAPOLATE = 1, /* zero-gradient ghost cells (copies of the edge cell) */
    RF_BC_NSCBC = 2        /* Navier-Stokes characteristic boundaries at both ends of the axis
                              (see rf_set_nscbc; the axis needs >= 3 cells).  Single-grid RHS
                              and RK steps in both precisions, with either scheme, on Cartesian
                              and RF_MAPPED grids (normal: the boundary cell's mean area vector
                              of the axis; the metric part of the normal term kept) and in
                              batched ensembles (the boundary kernels run per member after
                              the cell state); rejected by rf_rhs_noalloc and the adjoint
                              entry points */
};

enum rf_flags {           /* term switches for tests (0 = full method) and the scheme */
    RF_NO_INVISCID = 1,
    RF_NO_VISCOUS = 2,
    RF_NO_CHEMISTRY = 4,
    RF_NO_LASER = 8,
    RF_TENO6 = 16,        /* inviscid fluxes by TENO6 (Results, Solver; Methods, Numerical
                             method: the paper's sixth-order targeted ENO scheme, after Fu,
                             Hu and Adams 2016) instead of WENO3-Z: candidate stencils of
                             three and four cells inside a six-cell stencil (halo 3), kept
                             where their smoothness share chi_k >= 1e-7, LLF alpha over the
                             six cells.  Single-grid RHS and RK steps in both precisions;
                             rejected by rf_ensemble_create and the adjoint entry points */
    RF_MAPPED = 32,       /* curvilinear grid given by its node coordinates (rf_set_nodes; Methods,
                             Numerical method: the equations mapped onto a uniform computational
                             grid, U~ = U / J, F~ = (xi_x F + xi_y G + xi_z H) / J).  Face metrics
                             are the faces' area vectors (the six of a cell sum to zero, so a
                             uniform flow stays uniform), frozen over each face's stencil;
                             volumes, cell metrics and centres from the nodes.  dx, dy, dz of
                             the grid descriptor are then unused (they must still be > 0).
                             Single-grid RHS and RK steps in both precisions and with either
                             scheme (global-memory sweeps), NSCBC axes included; ensembles run
                             mapped members in the member loop (mode 0) only; rejected by
                             rf_rhs_noalloc and the adjoint entry points */
    RF_CHARWISE = 64,     /* characteristic-wise flux splitting (Methods, Numerical method: the
                             optional reconstruction of characteristic instead of conserved
                             variables) with the scheme RF_TENO6 selects: the split fluxes of
                             each face's stencil projected on the left eigenvectors of the
                             multicomponent Euler flux Jacobian at the face (arithmetic means of
                             the two adjacent cells' Y_s, u, dp/d(rho_s), gamma - 1 and H),
                             reconstructed field by field (WENO3-Z eps from the components a
                             field is made of) and projected back.  Cartesian grids; single-grid
                             RHS and RK steps in both precisions (global-memory sweeps);
                             rejected with RF_MAPPED or an NSCBC axis by rf_create_ctx, and by
                             rf_rhs_noalloc, rf_ensemble_create and the adjoint entry points */
    RF_FLAGS_ALL = 127
};

/* Mechanism description (host arrays, copied by rf_init_mechanism).
 * Paper: Methods, Governing equations (EOS, NASA fits, Wilke's rule,
 * mixture-averaged diffusion) and Methods, Combustion chemistry (finite-rate
 * Arrhenius reactions).  Ns in {1, 2, 4, 9}; Nr <= 32; every species uses the
 * same T_mid; at most 3 reactant and 3 product molecules per reaction.  At most
 * five mechanisms can be in use on a device at a time (each occupies a slot of
 * constant memory from its first context until rf_free_mechanism). */
typedef struct {
    int n_species;            /* Ns */
    int n_reactions;          /* Nr */
    const double *W;          /* [Ns] molar mass, kg/mol */
    const double *nasa_low;   /* [Ns][7] NASA-7 a1..a7 for T <  T_mid */
    const double *nasa_high;  /* [Ns][7] NASA-7 a1..a7 for T >= T_mid */
    const double *T_mid;      /* [Ns] K */
    const double *mu_ref;     /* [Ns] species viscosity at 300 K, Pa s */
    const double *mu_exp;     /* [Ns] exponent n_s of mu_s = mu_ref (T/300)^n_s */
    const double *D_ref;      /* [Ns][Ns] binary diffusivity at 300 K and 1 atm, m^2/s (symmetric) */
    const double *A;          /* [Nr] pre-exponential factor, (m^3/mol)^(order-1)/s */
    const double *b;          /* [Nr] temperature exponent */
    const double *Theta;      /* [Nr] activation temperature Ea/R, K */
    const int *nu_f;          /* [Nr][Ns] reactant stoichiometric coefficients */
    const int *nu_r;          /* [Nr][Ns] product stoichiometric coefficients */
    const int *reversible;    /* [Nr] 1 = reversible (k_r = k_f / K_c), 0 = irreversible */
    /* Pressure-dependent reactions (the paper's CH4/O2 mechanisms, Methods - Combustion
     * chemistry, contain them; CHEMKIN conventions).  rxn_type NULL: every reaction is
     * elementary (the other five arrays are then ignored).  At most 8 reactions of a
     * mechanism may be pressure dependent. */
    const int *rxn_type;      /* [Nr] 0 elementary; 1 third body: both directions times
                                 [M] = sum_s efficiency_s C_s; 2 Lindemann, 3 Troe fall-off:
                                 k = k_inf P_r / (1 + P_r) F, P_r = k_0 [M] / k_inf, with
                                 (A, b, Theta) the high-pressure k_inf */
    const double *efficiency; /* [Nr][Ns] third-body efficiencies (rows of type 1..3) */
    const double *A0;         /* [Nr] low-pressure k_0 = A0 T^b0 exp(-Theta0 / T), (m^3/mol)^order / s */
    const double *b0;         /* [Nr] */
    const double *Theta0;     /* [Nr] K */
    const double *troe;       /* [Nr][4] alpha, T***, T*, T** of the Troe broadening factor (type 3) */
} rf_mech_desc;

typedef struct {
    int nx, ny, nz;           /* cells per axis, each >= 1; nx <= 1024 */
    double dx, dy, dz;        /* spacing, m */
    int bc[3];                /* per axis x, y, z: rf_bc */
} rf_grid_desc;

/* Gaussian laser deposition (paper: Methods, Diffusion flame, Eq. laser-qs):
 * q_L = E / ((2 pi)^2 sigma_r^3 sigma_t) exp(-r^2 / 2 sigma_r^2) exp(-(t - t0)^2 / 2 sigma_t^2)
 * on 3-D grids; nz = 1 uses the paper's per-unit-depth 2-D form. */
typedef struct {
    double E, x0, y0, z0, sigma_r, t0, sigma_t;
} rf_laser;

/* Grid totals after one evaluation (see rf_diagnostics). */
typedef struct {
    double total[32];         /* sum over cells of each conserved variable times the cell volume */
    double heat_release;      /* sum over cells of HRR = -sum_s h_s omega_s times the cell volume, W */
    double max_T;             /* K */
    int nv;
} rf_diag;

typedef struct rf_mech rf_mech;
typedef struct rf_ctx rf_ctx;

/* Thread-local text of the last error on this thread ("" if none). */
const char *rf_last_error(void);

/* Copies the mechanism to the device.  *out owns device memory until
 * rf_free_mechanism.  Errors: RF_EINVAL (sizes, unsupported Ns, T_mid not
 * shared, more than 3 molecules on a side), RF_ECUDA / RF_ENOMEM. */
int rf_init_mechanism(const rf_mech_desc *d, rf_mech **out);
void rf_free_mechanism(rf_mech *m);

/* Creates a solver context for one grid: allocates its device workspace
 * (primitive/coefficient fields, RHS accumulator, two RK stage states,
 * reduction scalars, status word).  `m` must outlive the context. */
int rf_create_ctx(const rf_mech *m, const rf_grid_desc *g, int precision, uint32_t flags, rf_ctx **out);
void rf_free_ctx(rf_ctx *c);

/* Device bytes held by the context's workspace. */
size_t rf_ctx_workspace_bytes(const rf_ctx *c);

/* Conserved state from primitive fields.
 * prim (device, FP64, [5+Ns][N]): p [Pa], T [K], u, v, w [m/s], Y_1..Y_Ns.
 * U (device, FP64, [Ns+4][N]) and T (device, FP64, [N]) are written.
 * Paper: Methods, Governing equations (EOS p = rho R T sum Y_s / W_s). */
int rf_init_state(rf_ctx *c, const double *prim, double *U, double *T, rf_stream s);

/* dU/dt at time t (paper: Methods, Governing equations and Numerical method).
 * U (device, FP64, [Ns+4][N]) is read; T (device, [N]) carries the Newton
 * warm start in and the temperature of U out; laser may be NULL (no source);
 * dUdt (device, FP64, [Ns+4][N]) is written.  Asynchronous; check rf_status. */
int rf_rhs(rf_ctx *c, const double *U, double *T, double t, const rf_laser *laser, double *dUdt, rf_stream s);

/* One SSP-RK3 step (Shu-Osher form, stage times t, t+dt, t+dt/2; paper:
 * Methods, Numerical method).  U (device, [Ns+4][N]) is advanced in place;
 * T (device, [N]) holds the Newton warm start (on exit: the temperature of the
 * last stage's input); t_dev (device, 1 double) is advanced by dt;
 * dt_fixed > 0 uses that step, otherwise dt = min(CFL / max sum_d (|u_d|+c)/h_d,
 * 0.25 h_min^2 / max(nu, lambda/(rho cp), D_s), 0.2 / max |d omega_s/d rho_s|,
 * laser clamp); dt_dev (device, 1 double) receives the step used.
 * Asynchronous; check rf_status. */
int rf_rk_step(rf_ctx *c, double *U, double *T, double *t_dev, double dt_fixed, double cfl,
               const rf_laser *laser, double *dt_dev, rf_stream s);

/* rf_rk_step on host buffers: U_in (host, FP64, [Ns+4][N]) and T_in (host, [N]) are
 * copied to device buffers owned by the context (allocated on the first call,
 * N (Ns+5) doubles, counted by rf_ctx_workspace_bytes), the step runs there, and the
 * new state is copied to U_out (host, may equal U_in) and, if not NULL, the
 * temperature to T_out (host, may equal T_in).  The state is copied in by eight
 * chunks of cells on a copy stream of the context, and the first stage's
 * cell-state kernel of each chunk starts once that chunk has arrived, so that the
 * transfer overlaps computation; the temperature is copied out on the copy stream
 * as soon as the last stage's cell state has written it, during that stage's sweeps;
 * the state is copied out by eight chunks on a second copy stream once the last stage
 * is done, and s waits for them.  A following call's copy in of chunk q waits only for
 * this step's last stage and its copy out of chunk q, so the copies out of one step and
 * in of the next run in both directions at once (with pinned host memory; pageable
 * memory works but copies synchronously).  t_dev, dt_fixed, cfl, laser, dt_dev as rf_rk_step.
 * Asynchronous on s: the host buffers must stay valid, and U_out unread, until s
 * has completed.  Errors: RF_EINVAL, RF_ENOMEM, RF_ECUDA. */
int rf_rk_step_host(rf_ctx *c, const double *U_in, const double *T_in, double *U_out, double *T_out, double *t_dev,
                    double dt_fixed, double cfl, const rf_laser *laser, double *dt_dev, rf_stream s);

/* Tuning and test options of a context (host-side, take effect on the next call):
 *   "newton_maxit" Newton iteration cap (default 30; 0 forces RF_ENEWTON, for tests)
 *   "x_block"      threads per block of the FP64 x sweep (multiple of 32, <= 256; default 256)
 *   "walk_block"   threads per block of the FP64 y / z sweeps (multiple of 32, <= 128; default 128)
 *                  (the mixed-precision sweeps use fixed 128-thread tiles staged in shared memory)
 *   "walk_seg"     cells walked per thread in the y / z sweeps (default 16 in FP64, 32 in mixed precision)
 *   "profile"      1: record a CUDA event pair on the launching stream around every
 *                  kernel launch of this context (read with rf_profile_read); 0: off
 * Errors: RF_EINVAL for an unknown key or a value out of range. */
int rf_set_option(rf_ctx *c, const char *key, double value);

/* Node (cell corner) coordinates of an RF_MAPPED context: device array, FP64,
 * [3][nz+1][ny+1][nx+1] (x, y, z of node (i, j, k) at ((k (ny+1) + j)(nx+1) + i) within
 * each component; a two-dimensional grid, nz = 1, gives its two node planes, one
 * cell deep).  Cell (i, j, k) has the corners (i..i+1, j..j+1, k..k+1), ordered so
 * that the cell's volume is positive.  Computes the face area vectors, cell volumes,
 * metrics (inverse of the mean edge Jacobian) and centres into the context
 * (synchronous on s); the nodes are not kept.  Periodic axes connect cells by index;
 * each cell's faces take its own nodes, so a mapping that is not periodic stays
 * freestream-preserving, and one that is translation-periodic is also conservative.
 * Must be called before rf_rhs / rf_rk_step / rf_rk_step_host / rf_diagnostics.
 * Errors: RF_EINVAL (null argument, context without RF_MAPPED, a cell with a
 * non-positive volume or a left-handed metric), RF_ECUDA. */
int rf_set_nodes(rf_ctx *c, const double *nodes, rf_stream s);

/* One end of an NSCBC axis (paper: Application examples - the diffusion flame's left
 * and right boundaries and the combustor's injector inlet and nozzle outlet use the
 * Navier-Stokes characteristic boundary conditions for reacting flows, after Poinsot &
 * Lele 1992 and Okong'o & Bellan 2002).  Along the axis the sweeps use zero-gradient
 * ghost cells; in the first and last cell layer the inviscid normal term is replaced
 * by its characteristic form: wave amplitudes from one-sided second-order normal
 * derivatives of (rho, u_n, u_t1, u_t2, p, Y_s) with the frozen sound speed c, the
 * amplitudes of waves entering the domain replaced as below, and the conserved
 * rates formed with the multicomponent energy closure.  With ell = length,
 * M = |u_n| / c and F = max(1 - M^2, 0):
 *   outflow (target NULL): entering acoustic wave sigma c F (p - p_inf) / ell
 *     (partially non-reflecting; sigma = 0 is perfectly non-reflecting), entering
 *     entropy, shear and species waves 0;
 *   inflow (target given): the entering waves relax u_n, T, u_t and Y_s towards the
 *     target at rates eta_u c F / (2 ell), eta_T c / (gamma ell), eta_t c / ell and
 *     eta_Y c / ell.
 * Defaults at rf_create_ctx (both ends of every NSCBC axis): outflow, p_inf = 101325 Pa,
 * sigma = 0.25, every eta 1, length the domain length along the axis. */
typedef struct {
    double p_inf;             /* outflow: far-field pressure, Pa (> 0) */
    double sigma;             /* outflow: pressure relaxation coefficient (>= 0) */
    double eta_u, eta_T, eta_t, eta_Y;  /* inflow: relaxation coefficients (>= 0) */
    double length;            /* ell, m; <= 0: the number of cells along the axis times its spacing
                                 (on an RF_MAPPED grid: times V / |S| of the boundary cell, S its
                                 mean area vector of the axis) */
    const double *target;     /* NULL: outflow.  Inflow: device array, FP64, [4 + Ns][plane] holding
                                 (u, v, w, T, Y_1 .. Y_Ns) for each cell of the boundary plane;
                                 plane index = i_t1 + n_t1 i_t2 with t1 < t2 the two other axes
                                 (x axis: j + ny k; y axis: i + nx k; z axis: i + nx j).  Owned
                                 by the caller and read at every evaluation: it must stay valid
                                 (and may be changed between calls) while the side is set. */
} rf_nscbc;

/* Sets one end (side 0: low, the cells with index 0; side 1: high, index n - 1) of the
 * NSCBC axis `axis` (0 x, 1 y, 2 z) of context c; takes effect from the next call.
 * Errors: RF_EINVAL (null argument, axis or side out of range, the axis not NSCBC,
 * a non-finite or negative coefficient, an outflow side with p_inf <= 0). */
int rf_set_nscbc(rf_ctx *c, int axis, int side, const rf_nscbc *b);

/* Kernel classes of rf_profile_read: cell state, x sweep, y sweep, z sweep, other. */
enum { RF_PROF_CELL = 0, RF_PROF_SWEEP_X = 1, RF_PROF_SWEEP_Y = 2, RF_PROF_SWEEP_Z = 3, RF_PROF_OTHER = 4, RF_PROF_N = 5 };

/* Sums the recorded event intervals per kernel class since profiling was
 * enabled (or last read): ms[k] total milliseconds, launches[k] launch count,
 * for k < RF_PROF_N (nclass >= RF_PROF_N).  Waits for the recorded events;
 * clears the record.  Errors: RF_EINVAL, RF_ECUDA. */
int rf_profile_read(rf_ctx *c, double *ms, int *launches, int nclass);

/* Synchronises s, returns the device-side status of the context as an RF_E*
 * code (RF_OK if clean) and clears it.  *cell_out (may be NULL) receives a
 * flat cell index that raised the first recorded failure, or -1. */
int rf_status(rf_ctx *c, rf_stream s, long long *cell_out);

/* Totals of every conserved variable, total heat release rate and max T of the
 * state U (with T as Newton warm start).  Synchronous (result on the host). */
int rf_diagnostics(rf_ctx *c, const double *U, double *T, rf_diag *out, rf_stream s);

/* Discrete adjoint of the FP64 RHS (paper: the sensitivity question of
 * Application examples, Ignition of a diffusion flame / model combustor;
 * the method's RHS as in rf_rhs).  FP64 contexts only (RF_EINVAL otherwise).
 * Parameters p = (E, x0, y0, z0, sigma_r, ln A_0 .. ln A_{Nr-1}); grad_params
 * (device, 5 + Nr doubles) is accumulated into, as is lam_U (device, [Ns+4][N]).
 *
 * rf_adjoint_rhs: lam_U += (dR/dU)^T lam_dUdt + w_hrr dH/dU and grad_params +=
 * (dR/dp)^T lam_dUdt + w_hrr dH/dp, R = dU/dt of U at time t, H = sum over cells
 * of the heat-release rate -sum_s h_s omega_s times the cell volume.  lam_dUdt
 * (device, [Ns+4][N]) may be NULL (objective term only).  T (device) is the
 * Newton warm start in and the temperature of U out.  Non-smooth points take the
 * subgradient of the branch the forward evaluation took.  Asynchronous. */
int rf_adjoint_rhs(rf_ctx *c, const double *U, double *T, double t, const rf_laser *laser, const double *lam_dUdt,
                   double w_hrr, double *lam_U, double *grad_params, rf_stream s);

/* One SSP-RK3 step at fixed dt through rf_rhs evaluations and stage
 * combinations (the arithmetic rf_adjoint_rk_step differentiates): U and T are
 * advanced in place and, if J (host) is not NULL, *J += dt (H(U^n) + H(U^(1)) +
 * 4 H(U^(2))) / 6 (with J NULL no heat release is evaluated: a plain step of the
 * same arithmetic, as the checkpoint recomputation needs).  Synchronous. */
int rf_rk_step_objective(rf_ctx *c, double *U, double *T, double t, double dt, const rf_laser *laser, double *J,
                         rf_stream s);

/* Reverse of rf_rk_step_objective from U_n (device, not modified) and its
 * temperature T_n: lam (device, [Ns+4][N]) holds dJ/dU_{n+1} on entry and
 * dJ/dU_n on exit, with the step's objective term weighted by w_hrr;
 * grad_params accumulates.  Recomputes the stages internally.  Asynchronous. */
int rf_adjoint_rk_step(rf_ctx *c, const double *Un, const double *Tn, double t, double dt, const rf_laser *laser,
                       double w_hrr, double *lam, double *grad_params, rf_stream s);

/* rf_rk_step_objective that also keeps the step's stage inputs for the reverse pass,
 * so that the checkpointed gradient need not recompute them (two RHS evaluations
 * of each step it reverses).  stages (device, (2 (Ns+4) + 3) N doubles, caller-owned)
 * receives, in order: U^(1) and U^(2) ([Ns+4][N] each), the converged temperature of
 * U^n, that of U^(1), and the Newton warm start of U^(2) (the same as U^(1)'s) ([N]
 * each).  U, T, J as in rf_rk_step_objective (with J NULL the stages are those of the
 * plain step the checkpoint recomputation runs).  Errors: RF_EINVAL for a null
 * context, state or stages pointer or dt <= 0, and the conditions of
 * rf_rk_step_objective.  Synchronous. */
int rf_rk_step_stages(rf_ctx *c, double *U, double *T, double t, double dt, const rf_laser *laser, double *J,
                      double *stages, rf_stream s);

/* rf_adjoint_rk_step from the stage inputs rf_rk_step_stages kept for the step from
 * U_n (device, not modified) instead of recomputing them; same lam, grad_params and
 * w_hrr.  The temperatures in stages serve as Newton warm starts and are overwritten
 * (use each stages buffer once).  The result equals rf_adjoint_rk_step's to the order
 * of the FP64 atomic sums.  Errors: RF_EINVAL for a null pointer or dt <= 0, and the
 * conditions of rf_adjoint_rk_step.  Asynchronous. */
int rf_adjoint_rk_step_stored(rf_ctx *c, const double *Un, double *stages, double t, double dt, const rf_laser *laser,
                              double w_hrr, double *lam, double *grad_params, rf_stream s);

/* Batched ensembles (workload shape of the paper's ensemble studies, Results,
 * Ensemble simulation; Methods, Diffusion flame): members are contexts of one
 * mechanism and precision with their own grid sizes, states and lasers.
 * rf_ensemble_create records, for member i, its context, its state U[i], T[i]
 * (device) and laser lasers[i] (host, may be NULL for none) and t_dev[i] (device
 * array of n doubles holding each member's time); it builds the member tables
 * and the (member, tile) work lists of every phase.  The buffers must outlive
 * the ensemble.  Errors: RF_EINVAL (mixed mechanisms or precisions), RF_ENOMEM. */
typedef struct rf_ensemble rf_ensemble;
int rf_ensemble_create(rf_ctx *const *members, int n, double *const *U, double *const *T, const rf_laser *lasers,
                       double *t_dev, rf_ensemble **out);
void rf_ensemble_free(rf_ensemble *e);

/* Options: "walk_seg" (cells walked per thread in the y / z sweeps; rebuilds the
 * work lists), "barrier_spins" (polls, ~100 ns each, before a grid barrier of the
 * persistent kernel gives up; default 2e7) and "barrier_extra" (0 or 1: arrivals
 * a barrier waits for beyond the grid, so that a test can make a wait run out). */
int rf_ensemble_set_option(rf_ensemble *e, const char *key, double value);

/* Advances every member by nsteps SSP-RK3 steps (rules as rf_rk_step).
 * mode 0: per-member launch loop (each member's own rf_rk_step launches);
 * mode 1: one launch per phase over all members' work items;
 * mode 2: mode 1 captured once as a CUDA graph of one step, replayed;
 * mode 3: per RK stage, the cell state and the x sweep as launches over all members'
 *         work items, the y and z sweeps in one persistent cooperative launch (a grid
 *         barrier between them, bounded: a wait that runs out returns RF_ETIMEOUT),
 *         and (mixed precision) the stage update as a launch over the cells; one
 *         step is captured as a CUDA graph, as in mode 2, and replayed.
 * Modes 1-3 need every member with nx, ny, nz > 1 and Cartesian (an ensemble with
 * RF_MAPPED members runs mode 0).  A member whose state fails
 * (Newton, non-finite, range) is frozen at its last good step and the others
 * continue; member_status (host, n ints, may be NULL) receives each member's
 * RF_E* code.  Synchronous.  Returns RF_ETIMEOUT if a barrier gave up, a member's
 * code if member_status is NULL and a member failed, else RF_OK.  Each member's
 * results are bitwise those of running it alone. */
int rf_run_ensemble(rf_ensemble *e, int nsteps, int mode, double cfl, double dt_fixed, int32_t *member_status,
                    rf_stream s);

/* Picks the y / z walk segment length of a batched mode (1-3) by timing trial
 * steps of the ensemble itself for 8, 16 and 32 cells, then restores every
 * member's state and time; *seg_out (may be NULL) receives the choice.  The halo
 * is fixed at two cells by the WENO3-Z stencil and is not a tuning parameter. */
int rf_ensemble_autotune(rf_ensemble *e, int mode, double cfl, int *seg_out, rf_stream s);

/* Measures the FMA throughput of the current device (kind 0: FP64, 1: FP32)
 * with independent FMA chains on every SM; *tflops receives 2 x FMAs / s / 1e12.
 * Synchronous.  The FP64 figure is the ALU roofline of the cell-state kernel. */
int rf_probe_peak(int kind, double *tflops, rf_stream s);

/* Self-test of the FP64 elementary functions of the kernels (table-driven, after
 * Tang's methods): fn 0, the exponential pair of the Gibbs factors G_s =
 * exp(g_s/RT) RT/p_atm and 1/G_s (equilibrium constants, Methods, chemistry):
 * y[i] = exp(x[i]), y2[i] = exp(-x[i]) from one argument reduction; fn 1: y[i] =
 * ln x[i] for normal x > 0 (ln T of the rates and Gibbs energies); fn 2: y[i] =
 * exp(x[i]) (FP64 Arrhenius rates and transport powers).  Exponentials saturate at
 * 2^(+-1020) beyond |x| ~ 707.  And of the binary32 <-> binary64 conversions the
 * mixed-precision kernels build from integer operations: fn 3: y[i] = the
 * kernels' binary32 rounding of x[i], y2[i] = the hardware's (both widened
 * exactly to double); fn 4: the low 32 bits of each x[i] are a binary32 pattern
 * f, y[i] = the kernels' widening of f, y2[i] = the hardware's.  And of the
 * mixed path's FP64 functions, whose results feed FP32 quantities: fn 5: the
 * exponential pair y[i] = exp(x[i]), y2[i] = exp(-x[i]) to 2e-13 relative for
 * |x| <= 700; fn 6: y[i] = ln x[i] to 5e-14 absolute for normal x > 0 with a
 * binary exponent of magnitude at most 64.  x, y, y2 (fn 0, 3, 4, 5; may be NULL
 * otherwise): device arrays of n doubles (caller-owned).
 * Asynchronous on s; RF_EINVAL for an unknown fn, n < 0 or a missing array with
 * n > 0. */
int rf_probe_math(int fn, const double *x, double *y, double *y2, long long n, rf_stream s);

/* Allocation-free RHS (the paper has no counterpart: this is a service of the
 * library, not a step of the method).  Computes the same dU/dt as rf_rhs for a
 * mechanism and grid without a context, for callers that cannot allocate device
 * memory: a host framework whose caching allocator already holds the device's
 * memory budget (a library cudaMalloc would fail, or fragment and shrink that
 * budget behind the framework's back), and latency-critical loops, where
 * cudaMalloc and cudaFree may synchronise the device and stall work already
 * queued on other streams.  Its scratch (primitive and coefficient fields, RHS
 * accumulator, status words) lives in one static device array of 16 MiB that
 * every GPU loading the library holds until the process exits; grids needing
 * more (n (12 + 4 Ns) values of the bulk type, plus the FP32 state copy in
 * mixed precision and a 256-byte header; e.g. at most 43,000 cells for 9
 * species in FP64) are rejected with RF_EINVAL before any device work.  The
 * first call on a device looks the array's device address up
 * (cudaGetSymbolAddress) and the first call per precision and species count
 * sets kernel attributes (shared-memory limits); make those first calls before
 * any stream capture.
 * Calls share the array and its last contents (the status word is cleared at
 * each call); calls that overlap on the GPU race, so issue them on one stream.
 * Arguments as rf_rhs; m, g, precision and flags as rf_create_ctx.  The call
 * waits for its stream (it copies the status word to the host and synchronises
 * s) and returns the device status as an RF_E* code.  It calls no cudaMalloc,
 * cudaFree or other allocating routine. */
int rf_rhs_noalloc(const rf_mech *m, const rf_grid_desc *g, int precision, uint32_t flags, const double *U,
                   double *T, double t, const rf_laser *laser, double *dUdt, rf_stream s);

#ifdef __cplusplus
}
#endif
#endif /* REACTFLOW_H */
