// sweep_ops.cuh -- the discrete operator and the per-DOF update shared by the sweep
// kernels (sweep.cu: node gather, 2D y-marching, batched 2D; sweep2d_tb.cu: 2D sweeps
// several per launch).  The operator is the corner-quadrature energy described at the top
// of sweep.cu (Sec. 3.2 stress law, Sec. 2.2 PT / APT updates); every kernel that calls
// these functions evaluates a node with the same arithmetic, so kernels that gather a
// node the same way give the same bits.
#pragma once

#include "petto_internal.cuh"

namespace petto {
namespace {
__device__ __forceinline__ unsigned fixed_mask(const BoxSet &bs, int i, int j, int k) {
    unsigned m = 0;
    for (int q = 0; q < bs.n; ++q) {
        const Box &b = bs.b[q];
        if (i >= b.lo[0] && i <= b.hi[0] && j >= b.lo[1] && j <= b.hi[1] && k >= b.lo[2] && k <= b.hi[2]) m |= b.mask;
    }
    return m;
}

// Sweep constants in the compute type: FP32 kernels use the host-converted FP32 copies.
template <typename T> struct KC {
    T ce_par, ce_perp, cf_lam, cf_mu, cdiag, ct, src, a, b, s1;
};
template <typename T> __device__ __forceinline__ KC<T> kconst(const SweepArgs &A);
template <> __device__ __forceinline__ KC<float> kconst<float>(const SweepArgs &A) {
    const OpConstF &f = A.kf;
    return {f.ce_par, f.ce_perp, f.cf_lam, f.cf_mu, f.cdiag, f.ct, f.src, f.a, f.b, f.s1};
}
template <> __device__ __forceinline__ KC<double> kconst<double>(const SweepArgs &A) {
    const OpConst &k = A.k;
    return {k.ce_par, k.ce_perp, k.cf_lam, k.cf_mu, k.cdiag, k.ct, k.src, A.a, A.b, A.s1};
}

template <typename T> __device__ __forceinline__ T load_val(const LoadEntry &e);
template <> __device__ __forceinline__ float load_val<float>(const LoadEntry &e) { return e.valf; }
template <> __device__ __forceinline__ double load_val<double>(const LoadEntry &e) { return e.vald; }

// ------------------------------------------------------------- 2D operator
// U[dy][dx][a] for offsets -1..1 around the node, Ec[cy][cx] for the 4 adjacent cells
// (cell (i-1+cx, j-1+cy)).
template <typename T>
__device__ __forceinline__ void ku_elastic_2d(const T (&U)[3][3][2], const T (&Ec)[2][2], const KC<T> &k,
                                              T (&Ku)[2]) {
    const T cpar = k.ce_par, cperp = k.ce_perp, cl = k.cf_lam, cm = k.cf_mu;
    Ku[0] = Ku[1] = T(0);
    // edges along x (b = 0) and y (b = 1)
    {
        const T Em = Ec[0][0] + Ec[1][0], Ep = Ec[0][1] + Ec[1][1];  // x-edges: cells left / right
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            const T c = a == 0 ? cpar : cperp;
            Ku[a] += c * (Em * (U[1][1][a] - U[1][0][a]) - Ep * (U[1][2][a] - U[1][1][a]));
        }
    }
    {
        const T Em = Ec[0][0] + Ec[0][1], Ep = Ec[1][0] + Ec[1][1];  // y-edges: cells below / above
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            const T c = a == 1 ? cpar : cperp;
            Ku[a] += c * (Em * (U[1][1][a] - U[0][1][a]) - Ep * (U[2][1][a] - U[1][1][a]));
        }
    }
    // the four cells as faces spanned by (x, y); the node is at local corner (al, be)
#pragma unroll
    for (int al = 0; al < 2; ++al)
#pragma unroll
        for (int be = 0; be < 2; ++be) {
            const T Et = Ec[1 - be][1 - al];
            // offsets of the face's corner (0,0) relative to the node
            const int x0 = 1 - al, y0 = 1 - be;  // index into U of local corner (0,0)
            T SA[2], SB[2];
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                SA[c] = (U[y0][x0 + 1][c] - U[y0][x0][c]) + (U[y0 + 1][x0 + 1][c] - U[y0 + 1][x0][c]);
                SB[c] = (U[y0 + 1][x0][c] - U[y0][x0][c]) + (U[y0 + 1][x0 + 1][c] - U[y0][x0 + 1][c]);
            }
            // a = x, b = y
            const T Ga = Et * (cl * SB[1] + cm * SA[1]);
            const T Gb = Et * (cm * SB[0] + cl * SA[0]);
            const T Ha = Et * (cl * SB[1] - cm * SA[1]);
            const T Hb = Et * (cm * SB[0] - cl * SA[0]);
            if (al == 1 && be == 1) { Ku[0] += Ga; Ku[1] += Gb; }
            if (al == 0 && be == 0) { Ku[0] -= Ga; Ku[1] -= Gb; }
            if (al == 1 && be == 0) { Ku[0] += Ha; Ku[1] += Hb; }
            if (al == 0 && be == 1) { Ku[0] -= Ha; Ku[1] -= Hb; }
        }
}

template <typename T>
__device__ __forceinline__ T ku_thermal_2d(const T (&U)[3][3], const T (&Ec)[2][2], const KC<T> &k) {
    const T ct = k.ct;
    const T Exm = Ec[0][0] + Ec[1][0], Exp = Ec[0][1] + Ec[1][1];
    const T Eym = Ec[0][0] + Ec[0][1], Eyp = Ec[1][0] + Ec[1][1];
    return ct * (Exm * (U[1][1] - U[1][0]) - Exp * (U[1][2] - U[1][1]) + Eym * (U[1][1] - U[0][1]) -
                 Eyp * (U[2][1] - U[1][1]));
}

// Products rounded on their own and fused multiply-adds written out (the compiler fuses
// nothing it is not told to), so that every kernel that evaluates an expression built from
// them gets the same bits whatever code surrounds it.
__device__ __forceinline__ float rn_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rn_mul(double a, double b) { return __dmul_rn(a, b); }
// a b + c rounded once, wherever it stands
__device__ __forceinline__ float rn_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double rn_fma(double a, double b, double c) { return __fma_rn(a, b, c); }

// The owner terms of the 2D y-marching form: at node (i, j), the x-edge to (i+1, j), the
// y-edge to (i, j+1) and the face of cell (i, j), from u at the four corners of that cell
// (u0 = u(i, j), un = u(i+1, j), u1 = u(i, j+1), un1 = u(i+1, j+1)) and the moduli of cells
// (i, j-1) (Eb), (i, j) (Ec) and (i-1, j) (El).  Their forces go to four nodes: own to (i, j),
// tx (x-message) to (i+1, j), cyn (carried up) to (i, j+1) and tg (diagonal) to (i+1, j+1);
// the node's K u is then own + tx(i-1, j) + cyn(i, j-1) + tg(i-1, j-1), summed in that order
// (m2_ku).  Every kernel of the marching form evaluates these expressions, so they agree
// bit for bit.
template <typename T, int PHYS>
__device__ __forceinline__ void m2_terms(const T *u0, const T *un, const T *u1, const T *un1, T Eb, T Ec, T El,
                                         const KC<T> &k, T *own, T *tx, T *cyn, T *tg) {
    const T Ex = Eb + Ec, Ey = El + Ec;
    if (PHYS == 0) {
        const T ax0 = un[0] - u0[0], ax1 = un[1] - u0[1];
        const T ay0 = u1[0] - u0[0], ay1 = u1[1] - u0[1];
        const T fx0 = rn_mul(rn_mul(k.ce_par, Ex), ax0), fx1 = rn_mul(rn_mul(k.ce_perp, Ex), ax1);
        const T fy0 = rn_mul(rn_mul(k.ce_perp, Ey), ay0), fy1 = rn_mul(rn_mul(k.ce_par, Ey), ay1);
        const T SA0 = ax0 + (un1[0] - u1[0]), SA1 = ax1 + (un1[1] - u1[1]);
        const T SB0 = ay0 + (un1[0] - un[0]), SB1 = ay1 + (un1[1] - un[1]);
        const T ma1 = rn_mul(k.cf_mu, SA1), la0 = rn_mul(k.cf_lam, SA0);
        const T G0 = rn_mul(Ec, rn_fma(k.cf_lam, SB1, ma1)), G1 = rn_mul(Ec, rn_fma(k.cf_mu, SB0, la0));
        const T H0 = rn_mul(Ec, rn_fma(k.cf_lam, SB1, -ma1)), H1 = rn_mul(Ec, rn_fma(k.cf_mu, SB0, -la0));
        own[0] = -fx0 - fy0 - G0;
        own[1] = -fx1 - fy1 - G1;
        tx[0] = fx0 + H0;
        tx[1] = fx1 + H1;
        tg[0] = G0;
        tg[1] = G1;
        cyn[0] = fy0 - H0;
        cyn[1] = fy1 - H1;
    } else {
        const T fx = rn_mul(rn_mul(k.ct, Ex), un[0] - u0[0]);
        const T fy = rn_mul(rn_mul(k.ct, Ey), u1[0] - u0[0]);
        own[0] = -fx - fy;
        tx[0] = fx;
        tg[0] = T(0);
        cyn[0] = fy;
    }
}
template <typename T>
__device__ __forceinline__ T m2_ku(T own, T mx, T cy, T gd) {
    return own + mx + cy + gd;
}
// diag(K) of node (i, j) from its four cells (i-1, j-1), (i, j-1), (i-1, j), (i, j)
template <typename T>
__device__ __forceinline__ T m2_diag(const KC<T> &k, T Elb, T Eb, T El, T Ec) {
    return k.cdiag * ((Elb + Eb) + (El + Ec));
}

// ------------------------------------------------------------- 3D operator
// U[dz][dy][dx][a], Ec[cz][cy][cx] (cell (i-1+cx, j-1+cy, k-1+cz)).
template <typename T>
__device__ __forceinline__ T Uat(const T (&U)[3][3][3][3], int ox, int oy, int oz, int c) {
    return U[oz + 1][oy + 1][ox + 1][c];
}

template <typename T>
__device__ __forceinline__ T Eat(const T (&Ec)[2][2][2], int cx, int cy, int cz) {
    return Ec[cz][cy][cx];
}

template <typename T>
__device__ __forceinline__ void ku_elastic_3d(const T (&U)[3][3][3][3], const T (&Ec)[2][2][2], const KC<T> &k,
                                              T (&Ku)[3]) {
    const T cpar = k.ce_par, cperp = k.ce_perp, cl = k.cf_lam, cm = k.cf_mu;
    Ku[0] = Ku[1] = Ku[2] = T(0);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        T Em = 0, Ep = 0;
#pragma unroll
        for (int p = 0; p < 2; ++p)
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                int c0[3], c1[3];
                // the two free cell indices run over the other axes
                const int o1 = (b + 1) % 3, o2 = (b + 2) % 3;
                c0[b] = 0; c0[o1] = p; c0[o2] = q;
                c1[b] = 1; c1[o1] = p; c1[o2] = q;
                Em += Eat(Ec, c0[0], c0[1], c0[2]);
                Ep += Eat(Ec, c1[0], c1[1], c1[2]);
            }
        int m[3] = {0, 0, 0}, pl[3] = {0, 0, 0};
        m[b] = -1;
        pl[b] = 1;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const T c = a == b ? cpar : cperp;
            const T u0 = Uat(U, 0, 0, 0, a);
            Ku[a] += c * (Em * (u0 - Uat(U, m[0], m[1], m[2], a)) - Ep * (Uat(U, pl[0], pl[1], pl[2], a) - u0));
        }
    }
    // faces spanned by (a, b) with a < b; c is the third axis
#pragma unroll
    for (int pa = 0; pa < 3; ++pa) {
        const int a = pa == 2 ? 1 : 0;
        const int b = pa == 0 ? 1 : 2;
        const int c = 3 - a - b;
#pragma unroll
        for (int al = 0; al < 2; ++al)
#pragma unroll
            for (int be = 0; be < 2; ++be) {
                T Et = 0;
#pragma unroll
                for (int cc = 0; cc < 2; ++cc) {
                    int ci[3];
                    ci[a] = 1 - al; ci[b] = 1 - be; ci[c] = cc;
                    Et += Eat(Ec, ci[0], ci[1], ci[2]);
                }
                T SA[2], SB[2];  // components (a, b) only
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int comp = q == 0 ? a : b;
                    T sa = 0, sb = 0;
#pragma unroll
                    for (int t = 0; t < 2; ++t) {
                        int s0[3] = {0, 0, 0}, s1[3] = {0, 0, 0};
                        // a-edge at local b-offset t: (-al, t-be) -> (1-al, t-be)
                        s0[a] = -al; s0[b] = t - be;
                        s1[a] = 1 - al; s1[b] = t - be;
                        sa += Uat(U, s1[0], s1[1], s1[2], comp) - Uat(U, s0[0], s0[1], s0[2], comp);
                        // b-edge at local a-offset t: (t-al, -be) -> (t-al, 1-be)
                        int r0[3] = {0, 0, 0}, r1[3] = {0, 0, 0};
                        r0[a] = t - al; r0[b] = -be;
                        r1[a] = t - al; r1[b] = 1 - be;
                        sb += Uat(U, r1[0], r1[1], r1[2], comp) - Uat(U, r0[0], r0[1], r0[2], comp);
                    }
                    SA[q] = sa;
                    SB[q] = sb;
                }
                const T Ga = Et * (cl * SB[1] + cm * SA[1]);
                const T Gb = Et * (cm * SB[0] + cl * SA[0]);
                const T Ha = Et * (cl * SB[1] - cm * SA[1]);
                const T Hb = Et * (cm * SB[0] - cl * SA[0]);
                if (al == 1 && be == 1) { Ku[a] += Ga; Ku[b] += Gb; }
                if (al == 0 && be == 0) { Ku[a] -= Ga; Ku[b] -= Gb; }
                if (al == 1 && be == 0) { Ku[a] += Ha; Ku[b] += Hb; }
                if (al == 0 && be == 1) { Ku[a] -= Ha; Ku[b] -= Hb; }
            }
    }
}

template <typename T>
__device__ __forceinline__ T ku_thermal_3d(const T (&U)[3][3][3], const T (&Ec)[2][2][2], const KC<T> &k) {
    const T ct = k.ct;
    T acc = 0;
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        T Em = 0, Ep = 0;
#pragma unroll
        for (int p = 0; p < 2; ++p)
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                int c0[3], c1[3];
                const int o1 = (b + 1) % 3, o2 = (b + 2) % 3;
                c0[b] = 0; c0[o1] = p; c0[o2] = q;
                c1[b] = 1; c1[o1] = p; c1[o2] = q;
                Em += Ec[c0[2]][c0[1]][c0[0]];
                Ep += Ec[c1[2]][c1[1]][c1[0]];
            }
        int m[3] = {0, 0, 0}, pl[3] = {0, 0, 0};
        m[b] = -1;
        pl[b] = 1;
        const T u0 = U[1][1][1];
        acc += Em * (u0 - U[m[2] + 1][m[1] + 1][m[0] + 1]) - Ep * (U[pl[2] + 1][pl[1] + 1][pl[0] + 1] - u0);
    }
    return ct * acc;
}

// ------------------------------------------------------------- update
// APT momentum of a sweep k sweeps after the last restart: fixed a, or the adaptive
// schedule min(a, (k-1)/(k+2)) (the same value in every thread of every block).
template <typename T> __device__ __forceinline__ T momentum_k(int adaptive, T a, long long k);
template <> __device__ __forceinline__ float momentum_k<float>(int adaptive, float a, long long k) {
    return adaptive ? fminf(a, apt_schedule_k(k)) : a;
}
template <> __device__ __forceinline__ double momentum_k<double>(int adaptive, double a, long long k) {
    if (!adaptive) return a;
    if (k <= 0) return 0.0;
    const double sched = (double)(k - 1) / (double)(k + 2);
    return sched < a ? sched : a;
}
template <typename T>
__device__ __forceinline__ T apt_momentum(const SweepArgs &A, const KC<T> &k) {
    return momentum_k<T>(A.adaptive, k.a,
                         A.adaptive ? sweep_index(A) - reinterpret_cast<const long long *>(A.ctrl)[CT_RESTART_AT] : 0);
}

// The per-DOF update of one sweep (APT, PT or residual only), with the block's sums of
// R^2 and R.w (restart test) accumulated in T.
template <typename T>
struct Upd {
    KC<T> k;
    T a_eff;
    int mode, local_dt, want_res, test_dot;
    const T *rhs;
    T res, dot;
    __device__ __forceinline__ void apply(int64_t idx_c, bool fixed, T Ku, T F, T diag, T *uo, const T *ui, T *w) {
        if (rhs) F = rhs[idx_c];
        T R = fixed ? T(0) : F - Ku;
        if (want_res) res += R * R;
        const T u = ui[idx_c];
        if (mode == 0) {
            const T step = local_dt ? k.b * fast_rcp(diag) : k.b;
            const T wi = w[idx_c];
            if (test_dot) dot += R * wi;
            const T wn = fixed ? T(0) : a_eff * wi + step * R;
            w[idx_c] = wn;
            uo[idx_c] = fixed ? T(0) : u + wn;
        } else if (mode == 1) {
            const T step = local_dt ? k.s1 * fast_rcp(diag) : k.s1;
            uo[idx_c] = fixed ? T(0) : u + step * R;
        } else {
            w[idx_c] = R;
        }
    }
    // the same update with u and w (APT) already in registers (the marching kernels: products
    // rounded on their own, so that every kernel of that form gets the same bits)
    __device__ __forceinline__ void apply_v(int64_t idx_c, bool fixed, T Ku, T F, T diag, T u, T wi, T *uo, T *w) {
        T R = fixed ? T(0) : F - Ku;
        if (want_res) res += R * R;
        if (mode == 0) {
            const T step = local_dt ? k.b * fast_rcp(diag) : k.b;
            if (test_dot) dot += R * wi;
            const T wn = fixed ? T(0) : rn_fma(a_eff, wi, rn_mul(step, R));
            w[idx_c] = wn;
            uo[idx_c] = fixed ? T(0) : u + wn;
        } else if (mode == 1) {
            const T step = local_dt ? k.s1 * fast_rcp(diag) : k.s1;
            uo[idx_c] = fixed ? T(0) : rn_fma(step, R, u);
        } else {
            w[idx_c] = R;
        }
    }
};
template <typename T>
__device__ __forceinline__ Upd<T> make_upd(const SweepArgs &A, const KC<T> &kc) {
    return Upd<T>{kc, apt_momentum<T>(A, kc), A.mode, A.local_dt, A.want_res, A.test_dot,
                  static_cast<const T *>(A.rhs), T(0), T(0)};
}

// Block totals of sum R^2 and sum R.w, then one deterministic grid reduction: partials
// of R^2 at [0, nb), of R.w at [nb, 2 nb); the last block writes *res2 and, on a test
// sweep, schedules a momentum restart at the next sweep when <R, w> < 0.
__device__ __forceinline__ void finish_sweep(const SweepArgs &A, double res, double dot, int64_t bid) {
    __shared__ double sh[32];
    if (!A.want_res && !A.test_dot) return;
    const unsigned nb = gridDim.x * gridDim.y * gridDim.z;
    const double r = A.want_res ? block_sum(res, sh) : 0.0;
    const double d = A.test_dot ? block_sum(dot, sh) : 0.0;
    if (block_tid() == 0) A.red.partials[(int64_t)nb + bid] = d;
    if (publish_partial(r, A.red, bid, nb)) {
        const double t = A.want_res ? sum_partials(A.red, 0, nb, sh) : 0.0;
        const double td = A.test_dot ? sum_partials(A.red, nb, nb, sh) : 0.0;
        if (block_tid() == 0) {
            if (A.want_res) *A.res2 = t;
            if (A.test_dot) {
                A.ctrl[CT_DOT] = td;
                if (td < 0.0) reinterpret_cast<long long *>(A.ctrl)[CT_RESTART_AT] = sweep_index(A) + 1;
            }
            *A.red.counter = 0u;
        }
    }
}

}  // namespace
}  // namespace petto
