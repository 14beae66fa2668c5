/*
 * petto.h -- C ABI of the GB300 PeTTO hot path (pseudo-transient topology optimisation).
 *
 * Method: PeTTO, arXiv 2509.06971.  The library advances, on one GPU, the loop of
 * Fig. 5: accelerated pseudo-transient (APT) and pseudo-transient (PT) sweeps of the
 * state equation (Sec. 2.2; Sec. 3.2 PT/APT systems), the compliance sensitivity
 * (Sec. 2.3), the design update with its volume terms (Sec. 2.3, Sec. 3.1) and an
 * explicit Cahn-Hilliard step (Sec. 2.4).
 *
 * Conventions shared by every call
 *   - Every call returns a petto_status and never throws or aborts.  On failure the
 *     context keeps a message, readable with petto_last_error().
 *   - Grids: nx, ny (, nz) cells of size h; nodes (i, j, k) with 0 <= i <= nx etc.
 *     Host/device arrays exchanged through this API use the natural layouts
 *       cell field  [P][cells]          cell (i,j,k)  -> i + nx*(j + ny*k)
 *       node field  [C][nodes]          node (i,j,k)  -> i + (nx+1)*((j) + (ny+1)*k)
 *     with C = nrhs * ncomp components (ncomp = dim for elasticity, 1 for heat),
 *     component c = r*ncomp + a for load case r and displacement component a.
 *     2D problems have k = 0 only.
 *   - dtype arguments take PETTO_F32 or PETTO_F64 (design fields also PETTO_BF16 and
 *     PETTO_F16).  on_device != 0 means the pointer is device memory of the context's
 *     GPU, read or written on the context's stream; otherwise it is host memory and the
 *     call returns after the copy has completed.
 *   - Host arrays passed to petto_create are copied; the caller keeps ownership.
 *   - A context owns all its device memory and is not thread-safe.
 */
#ifndef PETTO_H
#define PETTO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct petto_ctx petto_ctx;

typedef enum {
    PETTO_OK = 0,
    PETTO_EINVAL = 1,        /* invalid argument or inconsistent sizes */
    PETTO_ENOMEM = 2,        /* device or host allocation failed */
    PETTO_ECUDA = 3,         /* a CUDA runtime call failed (message has the CUDA error) */
    PETTO_ENOTCONV = 4,      /* solve hit max_sweeps before the tolerance; report valid */
    PETTO_EDIVERGED = 5,     /* solve diverged even after the PT fallback */
    PETTO_ETIMEOUT = 6,      /* a bounded device-side wait ran out */
    PETTO_EUNSUPPORTED = 7   /* combination not built (e.g. dtype for this call) */
} petto_status;

enum { PETTO_ELASTIC = 0, PETTO_THERMAL = 1 };
enum { PETTO_SIMP_MODIFIED = 0, PETTO_SIMP_PAPER = 1 };
enum { PETTO_F32 = 0, PETTO_F64 = 1, PETTO_BF16 = 2, PETTO_F16 = 3 };
enum { PETTO_VOL_PROJECTED = 0, PETTO_VOL_PENALTY = 1 };
enum { PETTO_SOLVE_PAPER = 0, PETTO_SOLVE_TOL = 1 };
enum { PETTO_SWEEP_APT = 0, PETTO_SWEEP_PT = 1 };

/* Regular grid of nx x ny (x nz) cells of size h (dim = 2 or 3). */
typedef struct {
    int dim;
    int64_t nx, ny, nz;
    double h;
} petto_grid;

/* Material interpolation (Sec. 3.1 overall conductivity; Sec. 3.2 overall modulus).
 *   interp PETTO_SIMP_MODIFIED (n_phases = 1): E = e_min + rho^penal (modulus[0] - e_min)
 *   interp PETTO_SIMP_PAPER    (n_phases = P): E = sum_i modulus[i] rho_i^penal
 * rho = clamp(phi, 0, 1).  nu is Poisson's ratio (2D elasticity is plane strain).
 * modulus is copied (n_phases doubles). */
typedef struct {
    int physics;            /* PETTO_ELASTIC or PETTO_THERMAL */
    int n_phases;
    const double *modulus;
    double e_min;
    double nu;
    double penal;
    int interp;
} petto_materials;

/* Nodal loads (external force; Sec. 3.2 momentum balance) and a uniform heat source
 * (Sec. 2.2; each cell gives body_source * h^d / 2^d to each of its corners).
 *   node  [n][3]  (i, j, k) of each entry (k = 0 in 2D)
 *   comp  [n]     displacement component a (0 for heat)
 *   value [n]     force
 *   rhs   [n]     load case r in [0, nrhs), or NULL for all entries in case 0
 * Entries at the same node and component add.  All arrays are copied. */
typedef struct {
    int64_t n;
    const int64_t *node;
    const int32_t *comp;
    const double *value;
    const int32_t *rhs;
    double body_source;
} petto_loads;

/* Dirichlet supports u_a = 0 (Sec. 3.1, 3.2 boundary conditions) as axis-aligned node
 * boxes: box [n_boxes][6] = lo_i, lo_j, lo_k, hi_i, hi_j, hi_k (inclusive), and
 * comp_mask [n_boxes] with bit a fixing component a.  At most 16 boxes. */
typedef struct {
    int n_boxes;
    const int64_t *box;
    const uint32_t *comp_mask;
} petto_bcs;

/* precision: PETTO_F32 or PETTO_F64 for the state fields and sweeps.
 * storage:   design-field storage (PETTO_F32, PETTO_F64, PETTO_BF16, PETTO_F16); the
 *            interpolation and all updates compute in the sweep precision.
 * nrhs:      load cases solved together (1..4), sharing one modulus field.
 * stream:    cudaStream_t for all work of this context (NULL = legacy default stream). */
typedef struct {
    int precision;
    int storage;
    int nrhs;
    void *stream;
} petto_options;

/* Solve control (Sec. 2.2 hybrid schedule).
 *   mode PETTO_SOLVE_PAPER: exactly n_apt APT sweeps then n_pt PT sweeps.
 *   mode PETTO_SOLVE_TOL:   APT sweeps until a check sweep's input residual satisfies
 *                            ||R|| <= tol ||F||, at most max_sweeps in total.
 * APT sweep:  w <- a_k w + b' R,  u <- u + w;   PT sweep:  u <- u + s1' R;
 * with b' = b, s1' = s1 (global step, the paper's form) or b' = b / diag(K),
 * s1' = s1 / diag(K) per DOF when local_dt != 0 (local pseudo-time steps).
 * momentum 0: a_k = a (the paper's fixed damping).  momentum 1 (adaptive restart, an
 * extension): a_k = min(a, (k-1)/(k+2)) with k the sweeps since the last restart; the sweeps
 * with (t mod check_every) % 4 == 3 test <R, w> of their input and, when negative, restart
 * the momentum at the next sweep (decided on the device).  momentum 2: PT sweeps throughout
 * (the plain first-order method, for comparison; not taken by batches).  Whole check intervals are
 * replayed as CUDA graphs (unless PETTO_NO_GRAPHS is set); a context created with the
 * legacy default stream runs on a blocking stream of its own.
 * refine 1 (FP32 contexts, tolerance mode, tol < 1e-3): an FP32 state cannot represent a
 * solution much below relative residual ~1e-4 for stiff problems, so the solve sweeps the
 * FP32 state to 1e-2, then continues the same iteration on u = u64 + d with u64 in FP64:
 * whenever the check residual has fallen 8x (or stalls for 20 checks) d is added to u64,
 * the FP64 defect F - K u64 becomes the right-hand side of the sweeps (FP32; for the two-row
 * 3D marching kernel FP16 scaled by a power of two, see petto_kernel_info) and d restarts
 * at zero, while w and the momentum schedule carry on.  The solve ends when the FP64
 * defect meets the tolerance.  With the environment variable PETTO_TRACE set, every check
 * residual is printed to stderr.
 * w is zero at the start of every solve.  Every check_every-th sweep is a check sweep
 * (the last sweep of a paper-mode solve is one too).  Divergence guard: a non-finite
 * check residual resets u and w to zero, a residual above 10x (fixed momentum) or 100x
 * (adaptive) the best seen resets w; either switches the rest of the solve to PT. */
typedef struct {
    int mode;
    int64_t n_apt, n_pt;
    double a, b, s1;
    double tol;
    int64_t max_sweeps;
    int check_every;
    int local_dt;
    int momentum;
    int refine;
} petto_solve_opts;

/* res_norm = ||R|| over free DOFs and all load cases at the last check sweep's input
 * state; rel_res = res_norm / f_norm; r_pde = ||R / h^d|| / (number of nodes), the
 * paper's residual norm (Sec. 3.1). */
typedef struct {
    int64_t sweeps, apt_sweeps, pt_sweeps;
    double res_norm, f_norm, rel_res, r_pde;
    int converged, fell_back_to_pt;
} petto_solve_report;

/* Design update and phase field (Sec. 2.3, 2.4, 3.1).
 *   g_i = alpha_h s_i / max_c |s_i| + kappa_1 (sum_j phi_j - 1)
 *   vol_mode PETTO_VOL_PROJECTED: phi_i <- clamp(phi_i - g_i - lambda_i, 0, 1) with
 *            lambda_i from n_bisect bisection halvings of [-2, 2] on mean phi_i = V_i
 *   vol_mode PETTO_VOL_PENALTY:   phi_i <- phi_i - g_i - kappa_v (mean phi_i - V_i)
 *   Cahn-Hilliard (ch_steps times): mu = w'(phi) - gamma_g L phi; phi <- phi + tau L mu
 *   with w = sin^2(pi phi)/64 and L the no-flux cell Laplacian in grid units. */
typedef struct {
    int vol_mode;
    double alpha_h, kappa_v, kappa_1, gamma_g, tau;
    int ch_steps;
    int n_bisect;
} petto_pf_opts;

/* metrics[0..7]: step, compliance, work F.u, rel_res, sweeps, seconds, mean phi_0, lambda_0 */
typedef void (*petto_step_cb)(const double *metrics, void *user);

/* Create a context: copies the problem, allocates device state, sets phi_i = vol_frac[i]
 * (vol_frac has n_phases entries, the targets V_i of Sec. 2.3 J_v), u = w = 0.
 * Errors: PETTO_EINVAL for bad sizes/options, PETTO_ENOMEM, PETTO_ECUDA. */
petto_status petto_create(const petto_grid *grid, const petto_materials *mat, const petto_loads *loads,
                          const petto_bcs *bcs, const double *vol_frac, const petto_options *opt,
                          petto_ctx **out);

/* Free every resource of the context (NULL is a no-op). */
void petto_destroy(petto_ctx *ctx);

/* Last error message of the context ("" if none); static text if ctx is NULL. */
const char *petto_last_error(const petto_ctx *ctx);

/* Name of a status code. */
const char *petto_status_string(petto_status s);

/* Design field phi [P][cells] in dtype; recomputes the modulus field (Sec. 3.2). */
petto_status petto_set_design(petto_ctx *ctx, const void *phi, int dtype, int on_device);
petto_status petto_get_design(petto_ctx *ctx, void *phi, int dtype, int on_device);

/* State u (and APT increment w = u^n - u^{n-1}) [C][nodes]; w may be NULL (set: zero;
 * get: not returned). */
petto_status petto_set_state(petto_ctx *ctx, const void *u, const void *w, int dtype, int on_device);
petto_status petto_get_state(petto_ctx *ctx, void *u, void *w, int dtype, int on_device);

/* Modulus / conductivity field E [cells] (Sec. 3.1, 3.2 interpolation) of the design. */
petto_status petto_get_modulus(petto_ctx *ctx, void *E, int dtype, int on_device);

/* Exactly n sweeps of one kind (PETTO_SWEEP_APT / PETTO_SWEEP_PT) with the given
 * constants, continuing from the current u and w (Sec. 2.2; Sec. 3.2 PT/APT systems).
 * res_norm2 (may be NULL) receives sum R^2 of the last sweep's input state. */
petto_status petto_sweep(petto_ctx *ctx, int kind, int64_t n, double a, double b, double s1, int local_dt,
                         double *res_norm2);

/* Exactly n sweeps like petto_sweep with a dense right-hand side r in place of the loads:
 * R = r - K u.  These are the correction sweeps of the FP64 iterative refinement that FP32
 * solves use (K d = r with r the FP64 defect F - K u64; the sweep itself is Sec. 3.2's
 * PT/APT system with r as the force).  r is FP64 in the natural layout [C][nodes] (host,
 * or device when on_device), copied at the call; the context turns it into what its sweep
 * kernel reads, exactly as refinement does: FP64 contexts read it as is, FP32 contexts as
 * FP32, and the two-row marching kernels as FP16 holding r 2^k with 2^k the power of two
 * that takes max |r| into [2^14, 2^15) (restored by 2^-k in the kernel).  u and w continue
 * from the current state.  res_norm2 as in petto_sweep.  PETTO_EINVAL for a bad kind, n < 0
 * or r = NULL. */
petto_status petto_sweep_rhs(petto_ctx *ctx, int kind, int64_t n, double a, double b, double s1, int local_dt,
                             const double *r, int on_device, double *res_norm2);

/* Attempts of each bounded wait of the TMA marching sweeps for their ring copies (default
 * and maximum 16384, each attempt suspending the thread for at most 100 us; tries < 0
 * restores the default).  When a sweep's wait runs out, its CTAs let the copies already in
 * flight land (always with the default bound), record the time-out and return, and the
 * next residual check of a solve returns PETTO_ETIMEOUT; the next petto_pt_solve starts
 * afresh.  With 0 every such wait runs out at once: the way to exercise that path (no
 * counterpart in the paper; failure handling of this implementation).  PETTO_EINVAL above
 * the default. */
petto_status petto_set_wait_limit(petto_ctx *ctx, int tries);

/* R = F - K u on free DOFs (0 on supports) for the current state; R [C][nodes] may be
 * NULL; res_norm2 (may be NULL) receives sum R^2. */
petto_status petto_residual(petto_ctx *ctx, double *res_norm2, void *R, int dtype, int on_device);

/* The FP64 defect of the iterative refinement (petto_solve_opts.refine) for a given FP64
 * state: R = F - K(E) u in FP64 arithmetic with the context's FP32 cell moduli, 0 on
 * supports (the Sec. 3.2 operator; Sec. 2.2 systems).  u [C][nodes] (C = ncomp x load cases,
 * host or device memory as on_device says) is read, not kept: the current state is left as
 * it was.  res_norm2 (may be NULL) receives sum R^2 over free DOFs, R [C][nodes] (may be
 * NULL) the field, in the same memory kind as u.  On a 3D elastic grid (or a slab of one:
 * its own planes) this is the FP64 z-marching defect kernel (the node gather with
 * PETTO_DEFECT=gather), elsewhere the FP64 node gather.  Synchronises.  PETTO_EUNSUPPORTED for FP64 contexts (their own
 * petto_residual is the FP64 residual), PETTO_EINVAL for a null context or state. */
petto_status petto_residual64(petto_ctx *ctx, const double *u, int on_device, double *res_norm2, double *R);

/* Hybrid APT/PT solve of K(E) u = F from the current u (Sec. 2.2). */
petto_status petto_pt_solve(petto_ctx *ctx, const petto_solve_opts *opts, petto_solve_report *rep);

/* Compliance C = sum_c E_c e_c (Sec. 2.3 J_h; Sec. 3.2 J_m) summed over load cases,
 * external work F.u, and the sensitivity dC/dphi [P][cells] = -(dE/dphi_i) e_c (the
 * total derivative at the current state, a hand-written adjoint of the self-adjoint
 * compliance).  Any output pointer may be NULL.  The sensitivity is also kept in the
 * context for petto_design_update. */
petto_status petto_sensitivity(petto_ctx *ctx, double *compliance, double *work, void *dcdphi, int dtype,
                               int on_device);

/* Design update from the kept sensitivity (Sec. 2.3 combined objective, Sec. 3.1
 * normalised step); lambda [P] (may be NULL) receives lambda_i (projected mode) or the
 * mean of phi_i before the step (penalty mode).  Refreshes the modulus field. */
petto_status petto_design_update(petto_ctx *ctx, const petto_pf_opts *opts, double *lambda);

/* Keep-out region of the design update (Sec. 3.4, the drone's void region): adds
 * alpha_b dJ_b/dphi_i with J_b = sum_i (mean over the region of phi_i - target_i)^2 to the
 * update's gradient on the region's cells; the per-cell gradient 2 (mean - target) / N_b
 * is folded into kappa_b (= 2 alpha_b / N_b, as kappa_v is for J_v).
 *   box     host [lo_i, lo_j, lo_k, hi_i, hi_j, hi_k]: inclusive cell ranges (lo_k = hi_k =
 *           0 in 2D), or NULL to remove the region
 *   target  host [n_phases] targets (e.g. 0 for a solid phase, 1 for an explicit void)
 *   kappa_b >= 0
 * Copied; applies to every later petto_design_update.  PETTO_EINVAL for an empty or
 * out-of-grid box. */
petto_status petto_set_keepout(petto_ctx *ctx, const int64_t *box, const double *target, double kappa_b);

/* ---------------------------------------------------------------- slabs
 * A single 3D grid decomposed along z into slabs, one context each (one GPU each, or several
 * on one GPU).  The caller creates each slab's context for the node planes it owns plus one
 * neighbour plane on each interior side (the ghost planes; cells likewise extended), with
 * its loads, supports and design restricted to that range, and declares the owned planes
 * with petto_set_owned_planes: sweeps, residuals and their sums then cover the owned
 * planes only, and the ghost planes keep what was copied into them.  Before each sweep the
 * caller copies each interface plane from its owner into the neighbour's ghost plane
 * (petto_get_plane / petto_set_plane, or a collective between ranks); the owned planes then
 * take the same values as in the same sweeps of the whole grid, bit for bit (a node's update
 * reads its 3 x 3 x 3 node neighbourhood and its 8 cells only, in the same order).  Residual
 * sums of the slabs add up to the whole grid's.  The node gather and the two-row marching
 * kernel take slabs: a slab context whose kernel is another marching variant switches to
 * the node gather, and petto_select_kernel offers it only those two (PETTO_EINVAL for the
 * others). */

/* Node planes zlo..zhi (local indices, inclusive) are the ones this context's sweeps write;
 * zlo = 0, zhi = nz cells (the last node plane) restores the whole grid.  z_global is the
 * whole grid's index of local plane 0: the marching kernel starts its z segments on the
 * whole grid's even planes, which makes the slab's arithmetic that of the whole grid bit for
 * bit.  PETTO_EINVAL for an empty or out-of-grid range or a negative z_global,
 * PETTO_EUNSUPPORTED in 2D.  Synchronises the stream. */
petto_status petto_set_owned_planes(petto_ctx *ctx, int64_t zlo, int64_t zhi, int64_t z_global);

/* Hooks of a decomposed state solve, supplied by the caller's transport (NCCL or gloo
 * between ranks, copies between contexts of one process).
 *   exchange   fills this slab's ghost planes with its neighbours' interface planes and
 *              sends its own (petto_get_plane / petto_set_plane on ctx); called before every
 *              sweep, by every slab in the same order
 *   allreduce  replaces values[0..n) by their sums over all slabs (allreduce_max: by
 *              their maxima)
 * Each returns PETTO_OK, or a status that ends the solve with that status. */
typedef petto_status (*petto_exchange_fn)(petto_ctx *ctx, void *user);
typedef petto_status (*petto_allreduce_fn)(double *values, int n, void *user);

/* The state solve of petto_pt_solve (Sec. 2.2 hybrid APT -> PT schedule, checks every
 * check_every sweeps, the divergence guard) on one slab of a z-decomposed grid: before every
 * sweep exchange(ctx, user); the check residual and ||F|| are the whole grid's (allreduce of
 * the slabs' sums), so every slab takes the same decisions.  Adaptive-restart momentum
 * (momentum 1) tests the whole grid's <R, w> (allreduce on every fourth sweep, which
 * synchronises the stream) and restarts every slab together; fixed momentum (0) and PT only
 * (2) need no such test.  The FP64 refinement of FP32 contexts (opts->refine, as in
 * petto_pt_solve) runs slab by slab: each slab keeps the FP64 state of its planes and its
 * ghost planes (one more exchange before the FP64 state takes u or d), the FP64 defect of
 * its own planes with the whole grid's norm (allreduce), and the FP16 right-hand side of
 * the two-row marching kernel scaled by the whole grid's max |r| (allreduce_max, which may
 * be NULL when no refinement runs): a slab computes what the whole grid computes on its
 * planes.  rep as in petto_pt_solve, with the whole grid's residuals.  Every slab calls it
 * with the same opts.  PETTO_EINVAL for a null hook (allreduce_max when a refinement would
 * run) or bad options; PETTO_ENOTCONV as petto_pt_solve. */
petto_status petto_slab_solve(petto_ctx *ctx, const petto_solve_opts *opts, petto_exchange_fn exchange,
                              petto_allreduce_fn allreduce, petto_allreduce_fn allreduce_max, void *user,
                              petto_solve_report *rep);

/* Copy node plane k (local index) of the current state, every component (load cases
 * included), out to / in from a dense [ndof components][ny+1][nx+1] array in the sweep
 * precision (dtype must equal it).  on_device = 1: the array is device memory and the copy
 * is ordered on the context's stream; 0: host memory, and the call returns when the copy
 * is done.  PETTO_EINVAL for a plane outside the grid or another dtype. */
petto_status petto_get_plane(petto_ctx *ctx, int64_t k, void *dst, int dtype, int on_device);
petto_status petto_set_plane(petto_ctx *ctx, int64_t k, const void *src, int dtype, int on_device);

/* Cell layers of a slab's design fields, for the decomposed design step.  A slab owns the
 * cell layers whose lower node plane it owns; it holds one more below (its lower ghost
 * layer, between its lower ghost plane and its first own plane) and keeps a copy of the
 * layer above its top layer (local index nz), which only the Cahn-Hilliard step reads.
 *   field PETTO_LAYER_PHI: phase `phase` of the design, in the context's storage type
 *   field PETTO_LAYER_MU:  the Cahn-Hilliard chemical potential, in the sweep precision
 * petto_layer_bytes: bytes of one layer (nx ny elements), 0 for a bad field or a 2D grid.
 * petto_get_layer / petto_set_layer copy layer k (0..nz-1 local, or nz: the copy of the
 * layer above) out to / in from dst / src; on_device as petto_get_plane.  PETTO_EINVAL for
 * a bad field, phase or layer, PETTO_EUNSUPPORTED in 2D. */
enum { PETTO_LAYER_PHI = 0, PETTO_LAYER_MU = 1 };
int64_t petto_layer_bytes(const petto_ctx *ctx, int field);
petto_status petto_get_layer(petto_ctx *ctx, int field, int phase, int64_t k, void *dst, int on_device);
petto_status petto_set_layer(petto_ctx *ctx, int field, int phase, int64_t k, const void *src, int on_device);

/* Hook of the decomposed design step: for every interface, copy the lower slab's top layer
 * (local nz - 1) of `field` (phase `phase` of phi, or mu) into the upper slab's layer 0 and
 * the upper slab's layer 1 into the lower slab's layer nz (petto_get_layer /
 * petto_set_layer); called by every slab in the same order.  PETTO_OK or a status that ends
 * the step with that status. */
typedef petto_status (*petto_layer_exchange_fn)(petto_ctx *ctx, int field, int phase, void *user);

/* One design loop (Fig. 5: state solve, sensitivity, update, Cahn-Hilliard, modulus) on one
 * slab of a z-decomposed grid, every slab calling it with the same options: the state solve
 * of petto_slab_solve; one more exchange; the sensitivity of every held cell (a ghost layer
 * gets its owner's bits), with C and F.u summed over the slab's own layers and planes and
 * max |s_i| taken over the whole grid (allreduce, allreduce_max); the update with the whole
 * grid's means (penalty) or the bisection's bracket moved on the host from the whole grid's
 * sums, one allreduce per halving (projected), so every slab takes the same multiplier and
 * a ghost layer keeps its owner's values; each Cahn-Hilliard half step preceded by
 * exchange_layer of the field it reads (phi before mu is formed, mu before phi moves) and
 * phi's layers exchanged at the end; the modulus refreshed.  allreduce_max replaces
 * values[0..n) by their maxima over the slabs.  metrics [8] (may be NULL) receives, as the
 * petto_optimize callback does: step, C, F.u, rel_res, sweeps, seconds, mean phi_0, and the
 * multiplier of phase 0 (projected) or mean phi_0 before the step (penalty) -- all of the
 * whole grid.  Every slab owns two node planes or more (then a slab's top layer has a layer
 * above it exactly when the slab has an upper neighbour; PETTO_EINVAL for a slab of one).
 * Elasticity with one load case, no keep-out term (PETTO_EUNSUPPORTED otherwise); the
 * solve refines FP32 states as petto_slab_solve does.  PETTO_EINVAL for a null hook or bad
 * options; PETTO_ENOTCONV when the solve missed its tolerance (the step is still taken). */
petto_status petto_slab_design_step(petto_ctx *ctx, const petto_solve_opts *so, const petto_pf_opts *po,
                                    petto_exchange_fn exchange, petto_layer_exchange_fn exchange_layer,
                                    petto_allreduce_fn allreduce, petto_allreduce_fn allreduce_max, void *user,
                                    double *metrics);

/* opts->ch_steps explicit Cahn-Hilliard steps (Sec. 2.4); refreshes the modulus field. */
petto_status petto_cahn_hilliard(petto_ctx *ctx, const petto_pf_opts *opts);

/* Design update then Cahn-Hilliard (the phi half of one PeTTO loop, Fig. 5);
 * vol_out [P] (may be NULL) receives mean phi_i afterwards. */
petto_status petto_phase_field_step(petto_ctx *ctx, const petto_pf_opts *opts, double *vol_out);

/* n_steps PeTTO loops (Fig. 5): solve, sensitivity, update, Cahn-Hilliard.  cb (may be
 * NULL) is called on the host after each loop with the metrics described above.
 * Returns PETTO_ENOTCONV if any solve missed its tolerance (the loop still runs).  With the
 * paper's fixed-count schedule (PETTO_SOLVE_PAPER, check_every 0) no host decision falls
 * inside a loop: once a loop has run on the context, each loop is one replay of a captured
 * CUDA graph of the same launches (the same results), read back only for cb. */
petto_status petto_optimize(petto_ctx *ctx, int n_steps, const petto_solve_opts *sopts,
                            const petto_pf_opts *popts, petto_step_cb cb, void *user);

/* Checkpoint of design, state and step counter to a file / back (same problem). */
petto_status petto_save(petto_ctx *ctx, const char *path);
petto_status petto_load(petto_ctx *ctx, const char *path);

/* Wait for all work of the context's stream. */
petto_status petto_synchronize(petto_ctx *ctx);

/* Number of kernel launches this context has issued (for launch accounting). */
int64_t petto_launch_count(const petto_ctx *ctx);

/* Sweep-kernel timing.  While enabled, every sweep launch (or every graph replay of a check
 * interval of sweeps) is bracketed by a pair of CUDA events on the context's stream;
 * petto_profile_read waits for them and returns the summed device time (ms), the number of
 * sweeps timed and how many of those read a dense right-hand side (refinement sweeps), then
 * resets the counters.  Disabled by default.  Any output pointer may be NULL. */
petto_status petto_profile(petto_ctx *ctx, int enable);
petto_status petto_profile_read(petto_ctx *ctx, double *sweep_ms, int64_t *sweeps, int64_t *rhs_sweeps);

/* Sweep-kernel autotuner: times every kernel variant and tile shape that applies to this
 * problem (for 3D elasticity in FP32: TMA-staged marching kernels with one or two owner
 * rows per thread, 32x16 tiles, the register-staged kernel, several z-segment lengths;
 * in 2D with one load case: four and two sweeps per launch ("tb2d/k4/..", timed per
 * sweep over whole launches) and the y-marching kernel with several rows per warp; always
 * the node-gather kernel's block shapes) for n APT sweeps each from the current state,
 * restores the state, and keeps the fastest.  report (may be NULL) receives a JSON object
 * of milliseconds per sweep for each candidate, keyed by the names petto_select_kernel
 * takes.  Uses temporary device memory.  The first solve of a 3D elastic FP32 context of
 * 2^17 nodes or more runs it (unless a kernel was selected) and remembers the choice per
 * grid shape for the process. */
petto_status petto_autotune(petto_ctx *ctx, int n, char *report, int report_len);

/* Selects the sweep kernel by the name the autotuner reports ("tma2/zs16", "march2d/ly8",
 * "gather/32x8", ...); a kernel name alone ("tma2", "march2d", "gather") selects its first
 * listed variant (the default parameters).  PETTO_EINVAL when no such kernel applies.
 * Every variant computes the same sweep; they differ in tiling and summation order. */
petto_status petto_select_kernel(petto_ctx *ctx, const char *name);

/* The sweep kernel in use, by the name petto_select_kernel takes ("custom" if none
 * matches), copied NUL-terminated into name (at most name_len bytes; may be NULL), and in
 * *rhs_bytes (may be NULL) the bytes per node and component of the dense right-hand side
 * that its refinement sweeps read: 2 for the two-row 3D marching kernel, which reads the
 * defect as FP16 scaled by a power of two, else the size of the sweep precision. */
petto_status petto_kernel_info(petto_ctx *ctx, char *name, int name_len, int *rhs_bytes);

/* ---------------------------------------------------------------- batches
 * Many independent 2D problems advanced together (the paper solves one design problem at a
 * time; batching changes how the work is scheduled on the GPU, not what each problem
 * computes).  One kernel launch per sweep covers every problem still iterating, each
 * chunk of check_every sweeps is replayed as one CUDA graph, and the check residuals of
 * all problems are read with one copy.  Each problem keeps the iteration of
 * petto_pt_solve: its own checks, momentum restarts, divergence guard, PT fallback and
 * FP32 iterative refinement, with the same kernel arithmetic and reduction order as the
 * 2D marching kernel, so it ends in the same state as when solved alone on that kernel. */
typedef struct petto_batch petto_batch;

/* Borrows n contexts (they must outlive the batch): 2D, one load case (nrhs 1), and a
 * common precision and physics, else PETTO_EUNSUPPORTED.  The batched sweep is the 2D
 * y-marching kernel: each context keeps its marching variant ("march2d/ly*", chosen by
 * petto_select_kernel or petto_autotune), and a context on another sweep kernel is
 * switched to the default "march2d" variant (a problem matches its solve alone bit for
 * bit when solved alone with the same variant).
 * During batch calls the contexts' work runs on the first context's stream (joined to the
 * others' streams with events).  *out is NULL on failure. */
petto_status petto_batch_create(int n, petto_ctx *const *ctxs, petto_batch **out);
void petto_batch_destroy(petto_batch *b);
const char *petto_batch_last_error(const petto_batch *b);
/* kernel launches issued by the batch and by its contexts */
int64_t petto_batch_launch_count(const petto_batch *b);

/* Solves every problem (Sec. 2.2 PT / APT relaxation).  opts [n]: mode, n_apt, n_pt,
 * max_sweeps, check_every (even, >= 2), local_dt, momentum and refine must agree across
 * problems (PETTO_EINVAL otherwise); a, b, s1 and tol are per problem.  reps [n] (may be
 * NULL) receive each problem's report.  Returns PETTO_ENOTCONV when a tolerance-mode
 * problem did not converge, PETTO_EDIVERGED when a residual stayed non-finite. */
petto_status petto_batch_pt_solve(petto_batch *b, const petto_solve_opts *opts, petto_solve_report *reps);

/* n_steps PeTTO loops (Fig. 5) on every problem: batched solve, then per problem the
 * sensitivity, the design update and the Cahn-Hilliard steps with popts[i].  metrics
 * (may be NULL) receives [n_steps][n][8] values laid out as for petto_step_cb (entry 6,
 * the mean phase, is NaN). */
petto_status petto_batch_optimize(petto_batch *b, int n_steps, const petto_solve_opts *sopts,
                                  const petto_pf_opts *popts, double *metrics);

/* Timing of the batched sweeps with CUDA events around each graph replay: enable, then
 * read (and reset) the accumulated milliseconds and batch sweeps. */
petto_status petto_batch_profile(petto_batch *b, int enable);
petto_status petto_batch_profile_read(petto_batch *b, double *sweep_ms, int64_t *sweeps);

/* Allocation-free residual norm.  The paper has no counterpart: this entry point exists
 * for callers that must not allocate GPU memory themselves -- code running under a memory
 * manager that owns every device byte (a framework's caching allocator, a fixed arena of
 * a long-running service) or a time-critical loop in which a cudaMalloc would stall the
 * device.  It needs no context: the caller passes every input and output, and the kernel
 * keeps the scratch of its reduction in one array compiled into this library (about
 * 128 KB, present on every GPU that loads the library until the process exits).
 *
 * Computes *norm2 = sum over free DOFs of (F - K(E) u)^2 for linear elasticity in FP32
 * (the operator of petto_residual, plane strain in 2D):
 *   grid   dim 2 or 3, nx, ny (, nz) cells of size h; at most 4 194 304 nodes
 *          ((nx+1)(ny+1)(nz+1)); larger grids return PETTO_EINVAL
 *   nu     Poisson's ratio
 *   u      device [dim][nodes] displacements, natural node order
 *   E      device [cells] moduli, natural cell order
 *   F      device [dim][nodes] nodal loads, or NULL for none
 *   fixed  device [dim][nodes] bytes, nonzero = supported DOF (excluded), or NULL
 *   norm2  host double receiving the result; the call returns after it is written
 *   stream cudaStream_t to run on (NULL = legacy default stream)
 * It calls no cudaMalloc, cudaFree or other allocating routine.  The first call on a
 * device looks up the device address of the scratch array (cudaGetSymbolAddress) and keeps
 * it for that device, so make that first call before any stream capture; the kept address
 * belongs to the device context of that call, so do not call again after a
 * cudaDeviceReset of the device.  Each call waits on its stream for its result before it
 * returns.  Every call clears the ticket counter of the reduction before launching.  All
 * calls share the one scratch array: calls that overlap on the GPU (different streams, or
 * different host threads on one device) race and must be serialised by the caller. */
petto_status petto_residual_norm_static(const petto_grid *grid, double nu, const float *u, const float *E,
                                        const float *F, const uint8_t *fixed, double *norm2, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* PETTO_H */
