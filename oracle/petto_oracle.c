/*
 * petto_oracle.c -- plain, slow, FP64 CPU oracle of the PeTTO hot path.
 *
 * TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark may load this code.  It is compiled twice: plainly (the oracle
 * the tests hold the GPU against) and with OpenMP (the all-core CPU baseline only).  The GPU product path never links it,
 * shares no source, header, table or helper with it, and does not fall back to it.
 *
 * What it computes (paper: "PeTTO", arXiv 2509.06971):
 *   - steady heat conduction  -div(kappa grad T) = f            (Sec. 2.2, Eq. Poisson)
 *   - linear elasticity  div(sigma) + f = 0, isotropic Lame law   (Sec. 3.2, momentum balance,
 *     stress definition, Lame parameters; plane strain in 2D)
 *   - first-order pseudo-transient (PT) sweeps                    (Sec. 2.2, discretised heat eq.;
 *                                                                   Sec. 3.2 PT system)
 *   - accelerated PT (damped wave) sweeps                         (Sec. 2.2 discretised damped wave
 *                                                                   eq.; Sec. 3.2 APT system)
 *   - hybrid APT -> PT schedule                                   (Sec. 2.2, last paragraph)
 *   - SIMP / multi-phase material interpolation                   (Sec. 3.1 overall conductivity,
 *                                                                   Sec. 3.2 overall Young's modulus)
 *   - compliance and its design sensitivity                       (Sec. 2.3 thermal compliance,
 *                                                                   Sec. 3.2 J_m)
 *   - volume / partition-of-unity terms and the design update     (Sec. 2.3 J_v, J_1, combined J;
 *                                                                   Sec. 3.1 normalised update)
 *   - explicit Cahn-Hilliard phase-field step                     (Sec. 2.4, CH model, w(phi))
 *
 * Discretisation (the paper says only "finite difference"; reading R1):
 *   nodes carry u (d components) or T; cells carry the design fields.  In every cell
 *   and at each of its 2^d corners the gradient is taken from the one-sided
 *   differences along the d cell edges that meet at that corner; the cell energy is
 *   the average over its corners of the continuum energy density times the cell
 *   volume h^d.  K u is the gradient of that discrete energy.  This file evaluates
 *   the definition literally: a loop over cells and corners that scatters forces.
 *
 * Layout (oracle only): node (i,j,k) -> n = i + (nx+1)*(j + (ny+1)*k), DOF = n*ncomp + a
 * (interleaved components); cell (i,j,k) -> c = i + nx*(j + ny*k); phase fields [P][cells].
 * 2D problems use nz = 0 (one node layer).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int dim;        /* 2 or 3 */
    int nx, ny, nz; /* cells per axis; nz is ignored when dim == 2 */
    double h;       /* cell size */
    int physics;    /* 0 = elasticity, 1 = heat conduction */
    double nu;      /* Poisson ratio (elasticity); 2D is plane strain */
} or_grid;

/* ------------------------------------------------------------------ sizes */

int or_ncomp(const or_grid *g) { return g->physics == 0 ? g->dim : 1; }

int64_t or_nnodes(const or_grid *g) {
    int64_t nzn = g->dim == 3 ? (int64_t)g->nz + 1 : 1;
    return (int64_t)(g->nx + 1) * (g->ny + 1) * nzn;
}

int64_t or_ncells(const or_grid *g) {
    int64_t nzc = g->dim == 3 ? (int64_t)g->nz : 1;
    return (int64_t)g->nx * g->ny * nzc;
}

int64_t or_ndof(const or_grid *g) { return or_nnodes(g) * or_ncomp(g); }

static int64_t node_id(const or_grid *g, int i, int j, int k) {
    return (int64_t)i + (int64_t)(g->nx + 1) * ((int64_t)j + (int64_t)(g->ny + 1) * k);
}

/* Unit-modulus Lame constants (Sec. 3.2, Lame parameters with E = 1). */
static void lame_unit(double nu, double *lam, double *mu) {
    *lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    *mu = 1.0 / (2.0 * (1.0 + nu));
}

/* -------------------------------------------------- the cell-corner operator
 *
 * cell_forces: given the nodal values of one cell (local node q = qx + 2*qy + 4*qz,
 * ncomp values each) and its modulus Ec, return the local nodal forces
 * f = dW_c/du_local, where
 *     W_c = sum_corners (h^d / 2^d) * 1/2 * eps_q : sigma_q        (elasticity)
 *     W_c = sum_corners (h^d / 2^d) * 1/2 * Ec |grad_q T|^2         (heat)
 * and, at corner q, d(.)/dx_b is the difference along the cell edge in direction b
 * that contains q.  Also returns the corner-summed unit-modulus energy density
 * e = sum_q (h^d/2^d) eps_q : C0 : eps_q  (= 2 W_c / Ec).
 */
static double cell_forces(const or_grid *g, double Ec, const double *ul, double *fl) {
    const int d = g->dim, nc = or_ncomp(g), nq = 1 << d;
    const double h = g->h, wq = pow(h, d) / (double)nq;
    double lam, mu;
    lame_unit(g->nu, &lam, &mu);
    double e_unit = 0.0;
    for (int r = 0; r < nq * nc; ++r) fl[r] = 0.0;
    for (int q = 0; q < nq; ++q) {
        /* G[a][b] = d u_a / d x_b at corner q */
        double G[3][3] = {{0}};
        int nb[3];
        double sg[3];
        for (int b = 0; b < d; ++b) {
            int qb = (q >> b) & 1;
            nb[b] = q ^ (1 << b);          /* the other end of the b-edge through q */
            sg[b] = qb == 0 ? 1.0 : -1.0;  /* orientation of that edge */
            for (int a = 0; a < nc; ++a)
                G[a][b] = sg[b] * (ul[nb[b] * nc + a] - ul[q * nc + a]) / h;
        }
        double S[3][3] = {{0}}; /* dW/dG per unit weight, scaled by Ec below */
        if (g->physics == 0) {
            double eps[3][3], tr = 0.0;
            for (int a = 0; a < d; ++a)
                for (int b = 0; b < d; ++b) eps[a][b] = 0.5 * (G[a][b] + G[b][a]);
            for (int a = 0; a < d; ++a) tr += eps[a][a];
            double en = 0.0;
            for (int a = 0; a < d; ++a)
                for (int b = 0; b < d; ++b) {
                    double sig = 2.0 * mu * eps[a][b] + (a == b ? lam * tr : 0.0);
                    S[a][b] = sig;
                    en += eps[a][b] * sig;
                }
            e_unit += wq * en;
        } else {
            double en = 0.0;
            for (int b = 0; b < d; ++b) {
                S[0][b] = G[0][b];
                en += G[0][b] * G[0][b];
            }
            e_unit += wq * en;
        }
        for (int a = 0; a < nc; ++a)
            for (int b = 0; b < d; ++b) {
                double t = Ec * wq * S[a][b] * sg[b] / h;
                fl[nb[b] * nc + a] += t;
                fl[q * nc + a] -= t;
            }
    }
    return e_unit;
}

static void cell_nodes(const or_grid *g, int64_t c, int64_t *nodes) {
    int i = (int)(c % g->nx);
    int64_t rest = c / g->nx;
    int j = (int)(rest % g->ny);
    int k = (int)(rest / g->ny);
    int nq = 1 << g->dim;
    for (int q = 0; q < nq; ++q)
        nodes[q] = node_id(g, i + (q & 1), j + ((q >> 1) & 1), g->dim == 3 ? k + ((q >> 2) & 1) : 0);
}

/* Forces of cells [c0, c1) scattered into Ku. */
static void scatter_cells(const or_grid *g, const double *E, const double *u, double *Ku, int64_t c0, int64_t c1) {
    const int nc = or_ncomp(g), nq = 1 << g->dim;
    double ul[24], fl[24];
    int64_t nodes[8];
    for (int64_t c = c0; c < c1; ++c) {
        cell_nodes(g, c, nodes);
        for (int q = 0; q < nq; ++q)
            for (int a = 0; a < nc; ++a) ul[q * nc + a] = u[nodes[q] * nc + a];
        cell_forces(g, E[c], ul, fl);
        for (int q = 0; q < nq; ++q)
            for (int a = 0; a < nc; ++a) Ku[nodes[q] * nc + a] += fl[q * nc + a];
    }
}

/* Ku = K(E) u by a cell loop that scatters element forces. */
void or_apply_K(const or_grid *g, const double *E, const double *u, double *Ku) {
    const int64_t ncell = or_ncells(g);
    memset(Ku, 0, sizeof(double) * (size_t)or_ndof(g));
#ifdef _OPENMP
    /* OpenMP build, used only to time the CPU baseline on all host cores: the cells of one
     * layer (a row in 2D, a z layer in 3D) touch two node layers, so layers of one parity
     * touch disjoint nodes and scatter in parallel, even layers first.  The sum at a node
     * then runs in another order than the serial loop's (the results agree to rounding). */
    const int nl = g->dim == 3 ? g->nz : g->ny;
    const int64_t per = ncell / nl;
    for (int par = 0; par < 2; ++par) {
#pragma omp parallel for schedule(static)
        for (int l = par; l < nl; l += 2) scatter_cells(g, E, u, Ku, (int64_t)l * per, (int64_t)(l + 1) * per);
    }
#else
    scatter_cells(g, E, u, Ku, 0, ncell);
#endif
}

/* Unit-modulus cell energies e_c = sum_q (h^d/2^d) eps_q:C0:eps_q, so that the
 * compliance is C = sum_c E_c e_c = u.K u (Sec. 2.3 thermal compliance; Sec. 3.2 J_m). */
void or_cell_energy(const or_grid *g, const double *u, double *e) {
    const int nc = or_ncomp(g), nq = 1 << g->dim;
    const int64_t ncell = or_ncells(g);
    double ul[24], fl[24];
    int64_t nodes[8];
    for (int64_t c = 0; c < ncell; ++c) {
        cell_nodes(g, c, nodes);
        for (int q = 0; q < nq; ++q)
            for (int a = 0; a < nc; ++a) ul[q * nc + a] = u[nodes[q] * nc + a];
        e[c] = cell_forces(g, 1.0, ul, fl);
    }
}

/* Explicit sparse assembly: COO triplets of K from the element matrices, one column
 * per local unit vector.  Returns the number of triplets written (ncells*(2^d nc)^2). */
int64_t or_assemble_K(const or_grid *g, const double *E, int64_t *rows, int64_t *cols, double *vals) {
    const int nc = or_ncomp(g), nq = 1 << g->dim, nl = nq * nc;
    const int64_t ncell = or_ncells(g);
    double ul[24], fl[24];
    int64_t nodes[8], t = 0;
    for (int64_t c = 0; c < ncell; ++c) {
        cell_nodes(g, c, nodes);
        for (int s = 0; s < nl; ++s) {
            for (int r = 0; r < nl; ++r) ul[r] = (r == s) ? 1.0 : 0.0;
            cell_forces(g, E[c], ul, fl);
            for (int r = 0; r < nl; ++r) {
                rows[t] = nodes[r / nc] * nc + (r % nc);
                cols[t] = nodes[s / nc] * nc + (s % nc);
                vals[t] = fl[r];
                ++t;
            }
        }
    }
    return t;
}

/* diag(K): per DOF, the sum over adjacent cells of the element-matrix diagonal entry,
 * each obtained by applying the cell operator to a local unit vector. */
void or_diag_K(const or_grid *g, const double *E, double *diag) {
    const int nc = or_ncomp(g), nq = 1 << g->dim, nl = nq * nc;
    const int64_t ncell = or_ncells(g);
    double ul[24], fl[24];
    int64_t nodes[8];
    memset(diag, 0, sizeof(double) * (size_t)or_ndof(g));
    for (int64_t c = 0; c < ncell; ++c) {
        cell_nodes(g, c, nodes);
        for (int s = 0; s < nl; ++s) {
            for (int r = 0; r < nl; ++r) ul[r] = (r == s) ? 1.0 : 0.0;
            cell_forces(g, E[c], ul, fl);
            diag[nodes[s / nc] * nc + (s % nc)] += fl[s];
        }
    }
}

/* Nodal load of a uniform source f: each cell gives f h^d / 2^d to each corner. */
void or_body_load(const or_grid *g, double f, double *F) {
    const int nq = 1 << g->dim;
    const int64_t ncell = or_ncells(g);
    int64_t nodes[8];
    double share = f * pow(g->h, g->dim) / (double)nq;
    for (int64_t c = 0; c < ncell; ++c) {
        cell_nodes(g, c, nodes);
        for (int q = 0; q < nq; ++q) F[nodes[q]] += share;
    }
}

/* ------------------------------------------------------- residual and sweeps */

/* R = F - K u on free DOFs, 0 on Dirichlet DOFs.  Returns sum R^2 over free DOFs. */
double or_residual(const or_grid *g, const double *E, const double *F, const uint8_t *fixed,
                   const double *u, double *R) {
    const int64_t nd = or_ndof(g);
    or_apply_K(g, E, u, R);
    double s = 0.0;
#ifdef _OPENMP
#pragma omp parallel for reduction(+ : s) schedule(static)
#endif
    for (int64_t r = 0; r < nd; ++r) {
        R[r] = fixed[r] ? 0.0 : F[r] - R[r];
        s += R[r] * R[r];
    }
    return s;
}

/* First-order PT (Sec. 2.2 discretised heat equation; Sec. 3.2 PT system), written in
 * grid units: u <- u + s1 R with s1 = dt1 / h^d.  With dinv != NULL the pseudo-time step
 * is local: u <- u + s1 dinv R, dinv = 1/diag(K) (local time stepping, an extension).
 * Returns sum R^2 of the input state. */
double or_pt_sweep(const or_grid *g, const double *E, const double *F, const uint8_t *fixed,
                   double s1, const double *dinv, double *u, double *Rwork) {
    const int64_t nd = or_ndof(g);
    double s = or_residual(g, E, F, fixed, u, Rwork);
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int64_t r = 0; r < nd; ++r)
        u[r] = fixed[r] ? 0.0 : u[r] + s1 * (dinv ? dinv[r] : 1.0) * Rwork[r];
    return s;
}

/* Accelerated PT (damped wave; Sec. 2.2 and Sec. 3.2 APT system) as a three-level
 * scheme: with w^n = u^n - u^{n-1},  w^{n+1} = a w^n + b R(u^n),  u^{n+1} = u^n + w^{n+1}.
 *   elastic (forward damping difference):  a = theta/(theta+dt2), b = dt2^2/((theta+dt2) h^d)
 *   thermal (backward damping difference): a = 1 - dt2/theta,      b = dt2^2/(theta h^d)
 * With dinv != NULL, b is replaced by b dinv (local time stepping, as for PT).
 * Returns sum R^2 of the input state; dot (may be NULL) receives sum R.w of the input
 * residual and the input increment. */
double or_apt_sweep(const or_grid *g, const double *E, const double *F, const uint8_t *fixed,
                    double a, double b, const double *dinv, double *u, double *w, double *Rwork, double *dot) {
    const int64_t nd = or_ndof(g);
    double s = or_residual(g, E, F, fixed, u, Rwork);
    if (dot) {
        double d = 0.0;
#ifdef _OPENMP
#pragma omp parallel for reduction(+ : d) schedule(static)
#endif
        for (int64_t r = 0; r < nd; ++r) d += Rwork[r] * w[r];
        *dot = d;
    }
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int64_t r = 0; r < nd; ++r) {
        if (fixed[r]) {
            w[r] = 0.0;
            u[r] = 0.0;
        } else {
            w[r] = a * w[r] + b * (dinv ? dinv[r] : 1.0) * Rwork[r];
            u[r] = u[r] + w[r];
        }
    }
    return s;
}

/* Hybrid schedule (Sec. 2.2 last paragraph; loops of Sec. 3): an APT block that starts
 * with w = 0, then a PT block.
 *   mode 0 ("paper"):     exactly n_apt APT sweeps, then n_pt PT sweeps.
 *   mode 1 ("tolerance"): APT sweeps until a check sweep sees ||R|| <= tol ||F||, at
 *                          most max_sweeps sweeps in total; n_pt is unused.
 * Every check_every-th sweep (counted from the start of the solve) is a check sweep: its
 * input residual is compared against the tolerance and the divergence guard.  The guard:
 * a non-finite residual resets u and w to 0; a residual above 10x the best seen resets
 * w to 0; either switches the rest of the solve to PT sweeps.
 * local_dt != 0 uses the local pseudo-time steps s1/diag(K), b/diag(K) throughout.
 * momentum 0 keeps the APT damping a fixed (the paper's form).  momentum 1 (adaptive
 * restart, an extension of the fixed damping): the APT sweep with index t (counted from 0
 * within the solve) uses a_t = min(a, (k-1)/(k+2)), k = t - t_restart (0 when k <= 0);
 * every sweep with (t mod check_every) % 4 == 3 (t % 4 == 3 when check_every = 0) computes
 * <R_t, w_t> of its input residual and increment
 * and, when that is negative (the last step went uphill in energy), sets t_restart = t + 1.
 * The guard factor is 10 for fixed and 100 for adaptive momentum.
 * rep: [0] sweeps, [1] APT sweeps, [2] PT sweeps, [3] last checked ||R||, [4] ||F||,
 *      [5] converged flag, [6] fell-back-to-PT flag.                              */
void or_solve(const or_grid *g, const double *E, const double *F, const uint8_t *fixed, int mode,
              int64_t n_apt, int64_t n_pt, double a, double b, double s1, double tol,
              int64_t max_sweeps, int check_every, int local_dt, int momentum, double *u, double *w, double *rep) {
    const int64_t nd = or_ndof(g);
    double *R = (double *)malloc(sizeof(double) * (size_t)nd);
    double *dinv = NULL;
    if (local_dt) {
        dinv = (double *)malloc(sizeof(double) * (size_t)nd);
        or_diag_K(g, E, dinv);
        for (int64_t r = 0; r < nd; ++r) dinv[r] = dinv[r] > 0.0 ? 1.0 / dinv[r] : 0.0;
    }
    double fn2 = 0.0;
    for (int64_t r = 0; r < nd; ++r)
        if (!fixed[r]) fn2 += F[r] * F[r];
    const double fnorm = sqrt(fn2);
    for (int64_t r = 0; r < nd; ++r) w[r] = 0.0;
    int64_t sweeps = 0, n_a = 0, n_p = 0;
    int use_pt = 0, fell = 0, conv = 0;
    double best = INFINITY, last = NAN;
    int64_t t_restart = 0;
    const double guard = momentum ? 100.0 : 10.0;
    const int64_t total = mode == 0 ? n_apt + n_pt : max_sweeps;
    while (sweeps < total) {
        int apt = !use_pt && (mode == 1 || sweeps < n_apt);
        double r2;
        if (apt) {
            double at = a, dot = 0.0;
            const int test = momentum && (((check_every > 0 ? sweeps % check_every : sweeps) % 4) == 3);
            if (momentum) {
                const int64_t k = sweeps - t_restart;
                const double sched = k <= 0 ? 0.0 : (double)(k - 1) / (double)(k + 2);
                at = sched < a ? sched : a;
            }
            r2 = or_apt_sweep(g, E, F, fixed, at, b, dinv, u, w, R, test ? &dot : NULL);
            if (test && dot < 0.0) t_restart = sweeps + 1;
        } else {
            r2 = or_pt_sweep(g, E, F, fixed, s1, dinv, u, R);
        }
        if (apt) ++n_a; else ++n_p;
        ++sweeps;
        if (check_every > 0 && sweeps % check_every == 0) {
            double rn = sqrt(r2);
            last = rn;
            if (!isfinite(rn)) {
                for (int64_t r = 0; r < nd; ++r) u[r] = w[r] = 0.0;
                use_pt = 1; fell = 1;
                continue;
            }
            if (rn > guard * best && !use_pt) {
                for (int64_t r = 0; r < nd; ++r) w[r] = 0.0;
                use_pt = 1; fell = 1;
            }
            if (rn < best) best = rn;
            if (mode == 1 && rn <= tol * fnorm) { conv = 1; break; }
        }
    }
    rep[0] = (double)sweeps; rep[1] = (double)n_a; rep[2] = (double)n_p;
    rep[3] = last; rep[4] = fnorm; rep[5] = conv; rep[6] = fell;
    free(R);
    free(dinv);
}

/* --------------------------------------------------------------- materials
 * interp 0 (modified SIMP, one phase):  E = Emin + rho^p (E0 - Emin)
 * interp 1 (paper, P phases):            E = sum_i E_i rho_i^p
 * with rho = clamp(phi, 0, 1) (Sec. 3.1 overall conductivity; Sec. 3.2 overall modulus). */
static double clamp01(double x) { return x < 0.0 ? 0.0 : (x > 1.0 ? 1.0 : x); }

void or_material(int64_t ncell, int P, const double *phi, const double *moduli, double e_min,
                 double p, int interp, double *E) {
    for (int64_t c = 0; c < ncell; ++c) {
        if (interp == 0) {
            double rho = clamp01(phi[c]);
            E[c] = e_min + pow(rho, p) * (moduli[0] - e_min);
        } else {
            double s = 0.0;
            for (int i = 0; i < P; ++i) s += moduli[i] * pow(clamp01(phi[(int64_t)i * ncell + c]), p);
            E[c] = s;
        }
    }
}

/* dE/dphi_i: the derivative of the interpolation, taken as 0 outside [0, 1] where the
 * clamp is flat, and as the interior one-sided value at phi in {0, 1}. */
static double dE_dphi(double phi, double Ei, double e_min, double p, int interp) {
    if (phi < 0.0 || phi > 1.0) return 0.0;
    double slope = interp == 0 ? (Ei - e_min) : Ei;
    return p * pow(phi, p - 1.0) * slope;
}

/* Sensitivity of the compliance (total derivative, reading R3):
 * s_{i,c} = dC/dphi_{i,c} = -(dE_c/dphi_{i,c}) e_c.  Returns C = sum_c E_c e_c. */
double or_sensitivity(int64_t ncell, int P, const double *phi, const double *moduli, double e_min,
                      double p, int interp, const double *E, const double *e, double *s) {
    double C = 0.0;
    for (int64_t c = 0; c < ncell; ++c) C += E[c] * e[c];
    for (int i = 0; i < P; ++i)
        for (int64_t c = 0; c < ncell; ++c) {
            int64_t ic = (int64_t)i * ncell + c;
            s[ic] = -dE_dphi(phi[ic], moduli[interp == 0 ? 0 : i], e_min, p, interp) * e[c];
        }
    return C;
}

/* ------------------------------------------------------------ design update
 * Normalised compliance step (Sec. 3.1): g_i = alpha_h s_i / max_c |s_i|, plus the
 * partition-of-unity gradient kappa_1 (sum_j phi_j - 1) (Sec. 2.3 J_1) when kappa_1 != 0.
 *   vol_mode 0 (projected): phi_i <- clamp(phi_i - g_i - lambda_i, 0, 1), lambda_i by
 *                            bisection on [-2, 2] so that mean phi_i = V_i (reading R8).
 *   vol_mode 1 (penalty):   phi_i <- phi_i - g_i - kappa_v (mean phi_i - V_i)  (Sec. 2.3 J_v;
 *                            reading R7: per-cell gradient of J_v is 2 (mean - V)/N, folded
 *                            into kappa_v by the caller).
 * lambda_out[i] receives lambda_i (projected) or mean phi_i before the step (penalty). */
/* The same update with the keep-out term of the drone problem (Sec. 3.4):
 * J_b = sum_i (mean over Omega_b of phi_i - Vb_i)^2 for the cells with keep[c] != 0
 * (reading R23: means over the region, as R7 reads J_v), whose per-cell gradient
 * 2 (mean_b phi_i - Vb_i) / N_b is folded into kappa_b by the caller and added to g_i on
 * the cells of Omega_b.  keep = NULL or kappa_b = 0 leaves the update unchanged. */
void or_update_b(int64_t ncell, int P, double *phi, const double *s, const double *V, int vol_mode,
                 double alpha_h, double kappa_v, double kappa_1, int n_bisect, const unsigned char *keep,
                 const double *Vb, double kappa_b, double *lambda_out) {
    double *d = (double *)malloc(sizeof(double) * (size_t)(ncell * P));
    double *smax = (double *)calloc((size_t)P, sizeof(double));
    double *mean = (double *)calloc((size_t)P, sizeof(double));
    double *mean_b = (double *)calloc((size_t)P, sizeof(double));
    int64_t nb = 0;
    if (keep)
        for (int64_t c = 0; c < ncell; ++c) nb += keep[c] != 0;
    for (int i = 0; i < P; ++i) {
        for (int64_t c = 0; c < ncell; ++c) {
            double a = fabs(s[(int64_t)i * ncell + c]);
            if (a > smax[i]) smax[i] = a;
            mean[i] += phi[(int64_t)i * ncell + c];
            if (keep && keep[c]) mean_b[i] += phi[(int64_t)i * ncell + c];
        }
        mean[i] /= (double)ncell;
        if (nb > 0) mean_b[i] /= (double)nb;
    }
    for (int64_t c = 0; c < ncell; ++c) {
        double tot = 0.0;
        for (int i = 0; i < P; ++i) tot += phi[(int64_t)i * ncell + c];
        for (int i = 0; i < P; ++i) {
            int64_t ic = (int64_t)i * ncell + c;
            double gi = smax[i] > 0.0 ? alpha_h * s[ic] / smax[i] : 0.0;
            gi += kappa_1 * (tot - 1.0);
            if (nb > 0 && keep[c]) gi += kappa_b * (mean_b[i] - Vb[i]);
            d[ic] = phi[ic] - gi;
        }
    }
    for (int i = 0; i < P; ++i) {
        double *di = d + (int64_t)i * ncell, *pi = phi + (int64_t)i * ncell;
        if (vol_mode == 0) {
            double lo = -2.0, hi = 2.0;
            for (int it = 0; it < n_bisect; ++it) {
                double mid = 0.5 * (lo + hi), m = 0.0;
                for (int64_t c = 0; c < ncell; ++c) m += clamp01(di[c] - mid);
                m /= (double)ncell;
                if (m > V[i]) lo = mid; else hi = mid;
            }
            double lam = 0.5 * (lo + hi);
            for (int64_t c = 0; c < ncell; ++c) pi[c] = clamp01(di[c] - lam);
            lambda_out[i] = lam;
        } else {
            for (int64_t c = 0; c < ncell; ++c) pi[c] = di[c] - kappa_v * (mean[i] - V[i]);
            lambda_out[i] = mean[i];
        }
    }
    free(d); free(smax); free(mean); free(mean_b);
}

void or_update(int64_t ncell, int P, double *phi, const double *s, const double *V, int vol_mode,
               double alpha_h, double kappa_v, double kappa_1, int n_bisect, double *lambda_out) {
    or_update_b(ncell, P, phi, s, V, vol_mode, alpha_h, kappa_v, kappa_1, n_bisect, NULL, NULL, 0.0, lambda_out);
}

/* ---------------------------------------------------------- Cahn-Hilliard
 * Double well w(phi) = sin^2(pi phi)/64 (Sec. 2.4); its derivative written out. */
double or_double_well(double phi) { double s = sin(M_PI * phi); return s * s / 64.0; }
double or_double_well_deriv(double phi) { return 2.0 * sin(M_PI * phi) * cos(M_PI * phi) * M_PI / 64.0; }

/* No-flux cell Laplacian in grid units: (L v)_c = sum over in-domain face neighbours
 * c' of (v_c' - v_c).  Missing neighbours carry no flux (Sec. 2.4 boundary conditions). */
void or_cell_laplacian(const or_grid *g, const double *v, double *Lv) {
    const int nx = g->nx, ny = g->ny, nz = g->dim == 3 ? g->nz : 1;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int64_t c = (int64_t)i + (int64_t)nx * ((int64_t)j + (int64_t)ny * k);
                double s = 0.0;
                if (i > 0) s += v[c - 1] - v[c];
                if (i < nx - 1) s += v[c + 1] - v[c];
                if (j > 0) s += v[c - nx] - v[c];
                if (j < ny - 1) s += v[c + nx] - v[c];
                if (g->dim == 3) {
                    if (k > 0) s += v[c - (int64_t)nx * ny] - v[c];
                    if (k < nz - 1) s += v[c + (int64_t)nx * ny] - v[c];
                }
                Lv[c] = s;
            }
}

/* One forward-Euler step of the (multi-)phase Cahn-Hilliard model (Sec. 2.4), per phase,
 * in grid units:  mu = w'(phi) - gamma_g L phi;  phi <- phi + tau L mu,
 * with tau = D dt3 / h^2 and gamma_g = gamma / h^2. */
void or_ch_step(const or_grid *g, int P, double gamma_g, double tau, double *phi) {
    const int64_t ncell = or_ncells(g);
    double *L = (double *)malloc(sizeof(double) * (size_t)ncell);
    double *mu = (double *)malloc(sizeof(double) * (size_t)ncell);
    for (int i = 0; i < P; ++i) {
        double *pi = phi + (int64_t)i * ncell;
        or_cell_laplacian(g, pi, L);
        for (int64_t c = 0; c < ncell; ++c) mu[c] = or_double_well_deriv(pi[c]) - gamma_g * L[c];
        or_cell_laplacian(g, mu, L);
        for (int64_t c = 0; c < ncell; ++c) pi[c] += tau * L[c];
    }
    free(L); free(mu);
}
