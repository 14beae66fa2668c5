// sweep.cu -- fused PT / APT sweep kernels (Sec. 2.2; Sec. 3.2 PT and APT systems).
//
// The discrete operator.  The paper discretises the momentum balance and the heat
// equation by finite differences without fixing the stencil.  This library uses the
// corner-quadrature energy: in every cell, at each corner, the gradient is taken from
// the one-sided differences along the cell edges meeting there, and the cell energy is
// the corner average times h^d.  Expanding that energy gives two kinds of terms, which
// is the form the kernels evaluate:
//   * edge terms   W_e = h^(d-2)/2^d * Ebar_e * [(lam+2mu) A_par^2 + mu |A_perp|^2]
//                  with A = u(end) - u(start) along the grid edge e and Ebar_e the sum of
//                  the moduli of the 2^(d-1) cells around e;
//   * face terms   W_f = h^(d-2)/2^(d-2) * Etil_f * [lam Abar_a Bbar_b + mu Abar_b Bbar_a]
//                  for each face f spanned by axes (a, b), with Abar (Bbar) the mean of the
//                  difference vectors of its two a- (b-) edges and Etil_f the sum of the
//                  moduli of the cells sharing f (elasticity only; Sec. 3.2 stress law with
//                  the Lame parameters of Sec. 3.2, plane strain in 2D).
// Heat conduction keeps only the edge terms with the scalar temperature.  K u is the
// gradient of sum_e W_e + sum_f W_f.  The FP64 oracle evaluates the corner definition
// literally with a cell loop; the kernels here either gather, per node, the forces of its
// incident edges and faces (node-gather kernels), or evaluate each edge and face once at
// its owner node and pass the shares on (2D y-marching kernel below, 3D z-marching kernels
// in sweep3d_march.cu), so the two agree only if the expansion above is right.
//
// One sweep (APT):  R = F - K u (0 on supports);  w <- a w + b' R;  u' <- u + w
//          (PT):    u' <- u + s1' R
// with b' = b or b / diag(K) (local pseudo-time step), u read from one buffer and written
// to the other (ping-pong), w updated in place.  sum R^2 over free DOFs is accumulated in
// FP64 when requested (the residual norm of Sec. 3.1, for convergence checks).
#include <algorithm>
#include <cstdlib>
#include <cstring>

#include "petto_internal.cuh"
#include "sweep_ops.cuh"

namespace petto {

Layout make_layout(int dim, int nx, int ny, int nz) {
    Layout L{};
    L.dim = dim;
    L.nx = nx;
    L.ny = ny;
    L.nz = dim == 3 ? nz : 1;
    L.NX = nx + 1;
    L.NY = ny + 1;
    L.NZ = dim == 3 ? nz + 1 : 1;
    auto rup = [](int64_t v, int64_t m) { return (v + m - 1) / m * m; };
    L.SX = rup(L.NX + OX + 1, 32);
    L.SY = L.NY + 2;
    L.SZ = dim == 3 ? L.NZ + 2 : 1;
    L.CX = rup(nx + OX + 1, 32);
    L.CY = ny + 2;
    L.CZ = dim == 3 ? L.nz + 2 : 1;
    L.cstride = L.SX * L.SY * L.SZ;
    L.estride = L.CX * L.CY * L.CZ;
    return L;
}

namespace {

constexpr int GATHER3_ZS = 4;


// ------------------------------------------------------------- 2D gather kernel
// One node (i, j) of a 2D sweep: gathers the 3x3 neighbourhood and the 4 cell moduli,
// evaluates K u and hands each DOF to the update (multi-load-case 2D sweeps and the
// autotuner's alternative to the marching kernel below).
template <typename T, int PHYS, typename TE>
__device__ __forceinline__ void sweep2d_node(const Layout &L, const KC<T> &kc, const BoxSet &boxes, int nrhs,
                                             const T *__restrict__ ui, T *__restrict__ uo, T *__restrict__ w,
                                             const TE *__restrict__ E, const int *__restrict__ tile_ptr,
                                             const LoadEntry *__restrict__ loads, int tile, int i, int j,
                                             Upd<T> &up) {
    T Ec[2][2];
#pragma unroll
    for (int cy = 0; cy < 2; ++cy)
#pragma unroll
        for (int cx = 0; cx < 2; ++cx) Ec[cy][cx] = (T)__ldg(&E[L.cell(i - 1 + cx, j - 1 + cy, 0)]);
    const T S = Ec[0][0] + Ec[0][1] + Ec[1][0] + Ec[1][1];
    const T diag = kc.cdiag * S;
    const unsigned fm = fixed_mask(boxes, i, j, 0);
    const int64_t n0 = L.node(i, j, 0);
    const int l0 = tile_ptr[tile], l1 = tile_ptr[tile + 1];
    const int ncnt = ((i > 0) + (i < L.nx)) * ((j > 0) + (j < L.ny));
    for (int r = 0; r < nrhs; ++r) {
        if (PHYS == 0) {
            T U[3][3][2];
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                const T *uc = ui + (int64_t)(r * 2 + a) * L.cstride;
#pragma unroll
                for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                    for (int dx = 0; dx < 3; ++dx) U[dy][dx][a] = __ldg(&uc[n0 + (dy - 1) * L.SX + (dx - 1)]);
            }
            T Ku[2];
            ku_elastic_2d<T>(U, Ec, kc, Ku);
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                const int c = r * 2 + a;
                T F = 0;
                for (int l = l0; l < l1; ++l)
                    if (loads[l].node == n0 && loads[l].comp == c) F += load_val<T>(loads[l]);
                const int64_t idx = (int64_t)c * L.cstride + n0;
                up.apply(idx, (fm >> a) & 1u, Ku[a], F, diag, uo, ui, w);
            }
        } else {
            T U[3][3];
            const T *uc = ui + (int64_t)r * L.cstride;
#pragma unroll
            for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                for (int dx = 0; dx < 3; ++dx) U[dy][dx] = __ldg(&uc[n0 + (dy - 1) * L.SX + (dx - 1)]);
            const T Ku = ku_thermal_2d<T>(U, Ec, kc);
            T F = kc.src * (T)ncnt;
            for (int l = l0; l < l1; ++l)
                if (loads[l].node == n0 && loads[l].comp == r) F += load_val<T>(loads[l]);
            const int64_t idx = (int64_t)r * L.cstride + n0;
            up.apply(idx, fm & 1u, Ku, F, diag, uo, ui, w);
        }
    }
}

template <typename T, int PHYS, typename TE = T>
__global__ void __launch_bounds__(256) sweep2d_gather(const SweepArgs A) {
    const Layout &L = A.L;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const KC<T> kc = kconst<T>(A);
    Upd<T> up = make_upd<T>(A, kc);
    if (i < L.NX && j < L.NY)
        sweep2d_node<T, PHYS, TE>(L, kc, A.boxes, A.nrhs, static_cast<const T *>(A.u_in), static_cast<T *>(A.u_out),
                                  static_cast<T *>(A.w), static_cast<const TE *>(A.E), A.tile_ptr, A.loads,
                                  blockIdx.x + gridDim.x * blockIdx.y, i, j, up);
    finish_sweep(A, (double)up.res, (double)up.dot, blockIdx.x + (int64_t)gridDim.x * blockIdx.y);
}

// ------------------------------------------------------------- 2D y-marching kernel
// Each warp owns 32 node columns (the lane's column i = 30 * bx - 1 + lane) and marches up
// ly rows.  At row j a lane evaluates once the terms whose lower-left corner is its node:
// the x-edge to (i+1, j), the y-edge to (i, j+1) and the face of cell (i, j), and
// distributes their forces: -fx - fy - G to itself, fx + H to (i+1, j) (shuffled up one
// lane), fy - H to (i, j+1) (kept in registers for the next row) and G to (i+1, j+1)
// (shuffled, then kept).  Neighbour values of column i+1 and cell column i-1 come by warp
// shuffles, the next rows by loads issued one row ahead; no shared memory, no barriers.
// Lanes 1..30 produce output (lanes 0 and 31 are the halo), and each warp starts one row
// early to receive the messages from below.
template <typename T, typename TE>
struct M2View {
    Layout L;
    KC<T> kc;
    const BoxSet *boxes;
    const T *ui;
    T *uo;
    T *w;
    const TE *E;
    const T *rhs;
    const int *tile_ptr;
    const LoadEntry *loads;
    int gx, ly;
};

template <typename T, int PHYS, typename TE, int LY>
__device__ __forceinline__ void march2d_tile(const M2View<T, TE> &V, int tile, Upd<T> &up) {
    constexpr int C = PHYS == 0 ? 2 : 1;
    constexpr unsigned FULL = 0xffffffffu;
    const Layout &L = V.L;
    const KC<T> &k = V.kc;
    const int lane = threadIdx.x;
    const int bxi = tile % V.gx, byi = tile / V.gx;
    const int i = bxi * 30 - 1 + lane;
    const int y0 = (byi * M2W + (int)threadIdx.y) * LY;
    if (y0 >= L.NY) return;  // warp-uniform
    const int yend = min(y0 + LY, L.NY);
    const bool ucol = i >= -1 && i <= L.NX;      // node column inside the zero ring
    const bool ecol = i >= -1 && i <= L.nx;      // cell column inside the zero ring
    const bool out = lane >= 1 && lane <= 30 && i < L.NX;
    const int l0 = V.tile_ptr[tile], l1 = V.tile_ptr[tile + 1];
    // 32-bit offsets (a 2D field has fewer than 2^31 elements per component pair; checked
    // when the kernel is selected)
    const int cs = (int)L.cstride, SX = (int)L.SX, CXp = (int)L.CX;
    const int ncol = i + OX, ecolo = i + OX;
    // supports whose x-range holds this column; their y-ranges are tested per row
    unsigned bbits = 0;
    for (int q = 0; q < V.boxes->n; ++q)
        if (i >= V.boxes->b[q].lo[0] && i <= V.boxes->b[q].hi[0]) bbits |= 1u << q;
    auto ld_u = [&](int j, T (&v)[C]) {
        const bool ok = ucol && j >= -1 && j <= L.NY;
        const int n = ok ? (j + 1) * SX + ncol : 0;
#pragma unroll
        for (int c = 0; c < C; ++c) v[c] = ok ? __ldg(&V.ui[c * cs + n]) : T(0);
    };
    auto ld_e = [&](int j) -> T {
        const bool ok = ecol && j >= -1 && j <= L.ny;
        return ok ? (T)__ldg(&V.E[(j + 1) * CXp + ecolo]) : T(0);
    };
    T u0[C], u1[C], u2[C], un[C], un1[C], wv[C], fv[C], wv2[C], fv2[C];
    ld_u(y0 - 1, u0);
    ld_u(y0, u1);
    ld_u(y0 + 1, u2);
    T Eb = ld_e(y0 - 2), Ec = ld_e(y0 - 1), E2 = ld_e(y0);
#pragma unroll
    for (int c = 0; c < C; ++c) {
        un[c] = __shfl_down_sync(FULL, u0[c], 1);
        wv[c] = fv[c] = wv2[c] = fv2[c] = T(0);
    }
    T Elb = __shfl_up_sync(FULL, Eb, 1);
    // w and the dense right-hand side of output row j, two rows ahead of their use
    auto ld_wf = [&](int j, T (&wd)[C], T (&fd)[C]) {
        if (!out || j >= yend) return;
        const int n = (j + 1) * SX + ncol;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            if (up.mode == 0) wd[c] = V.w[c * cs + n];
            if (V.rhs) fd[c] = V.rhs[c * cs + n];
        }
    };
    ld_wf(y0, wv, fv);
    ld_wf(y0 + 1, wv2, fv2);
    T cy[C], gd[C];
#pragma unroll
    for (int c = 0; c < C; ++c) cy[c] = gd[c] = T(0);
    // rows are a compile-time count: the loop unrolls fully and the row rotation below
    // becomes register renaming, so loads stay in flight until their first real use
#pragma unroll
    for (int r = 0; r <= LY; ++r) {
        const int j = y0 - 1 + r;
        if (j >= yend) break;  // warp-uniform
        const T El = __shfl_up_sync(FULL, Ec, 1);
#pragma unroll
        for (int c = 0; c < C; ++c) un1[c] = __shfl_down_sync(FULL, u1[c], 1);
        T own[C], mx[C], gn[C], cyn[C], tx[C], tg[C];
        m2_terms<T, PHYS>(u0, un, u1, un1, Eb, Ec, El, k, own, tx, cyn, tg);
#pragma unroll
        for (int c = 0; c < C; ++c) {
            mx[c] = __shfl_up_sync(FULL, tx[c], 1);
            gn[c] = PHYS == 0 ? __shfl_up_sync(FULL, tg[c], 1) : T(0);
        }
        if (j >= y0 && out) {
            const int n = (j + 1) * SX + ncol;
            unsigned fm = 0;
            for (unsigned bb = bbits; bb; bb &= bb - 1) {
                const Box &bx = V.boxes->b[__ffs(bb) - 1];
                if (j >= bx.lo[1] && j <= bx.hi[1]) fm |= bx.mask;
            }
            const T diag = m2_diag(k, Elb, Eb, El, Ec);
            T F[C];
#pragma unroll
            for (int c = 0; c < C; ++c) F[c] = fv[c];
            if (!V.rhs) {
                if (PHYS == 1) F[0] = k.src * (T)(((i > 0) + (i < L.nx)) * ((j > 0) + (j < L.ny)));
                const int64_t nl = L.node(i, j, 0);
                for (int l = l0; l < l1; ++l) {
                    const LoadEntry &le = V.loads[l];
                    if (le.node == nl) {
#pragma unroll
                        for (int c = 0; c < C; ++c)
                            if (le.comp == c) F[c] += load_val<T>(le);
                    }
                }
            }
#pragma unroll
            for (int c = 0; c < C; ++c)
                up.apply_v(c * cs + n, (fm >> c) & 1u, m2_ku(own[c], mx[c], cy[c], gd[c]), F[c], diag, u0[c], wv[c],
                           V.uo, V.w);
        }
#pragma unroll
        for (int c = 0; c < C; ++c) {
            cy[c] = cyn[c];
            gd[c] = gn[c];
            u0[c] = u1[c];
            u1[c] = u2[c];
            un[c] = un1[c];
        }
        Eb = Ec;
        Ec = E2;
        Elb = El;
        if (j + 3 <= L.NY) ld_u(j + 3, u2);
        E2 = ld_e(j + 2);
        if (j >= y0) {
#pragma unroll
            for (int c = 0; c < C; ++c) {
                wv[c] = wv2[c];
                fv[c] = fv2[c];
            }
            ld_wf(j + 2, wv2, fv2);
        }
    }
}

// rows per warp: the variants compiled (a tiling's ly is one of these)
template <typename T, int PHYS, typename TE>
__device__ __forceinline__ void march2d_tile_ly(const M2View<T, TE> &V, int tile, Upd<T> &up) {
    switch (V.ly) {
        case 4: march2d_tile<T, PHYS, TE, 4>(V, tile, up); break;
        case 16: march2d_tile<T, PHYS, TE, 16>(V, tile, up); break;
        default: march2d_tile<T, PHYS, TE, 8>(V, tile, up); break;
    }
}

template <typename T, int PHYS, typename TE = T>
__global__ void __launch_bounds__(32 * M2W) sweep2d_march(const __grid_constant__ SweepArgs A) {
    const int tile = blockIdx.x + gridDim.x * blockIdx.y;
    const KC<T> kc = kconst<T>(A);
    Upd<T> up = make_upd<T>(A, kc);
    const M2View<T, TE> V{A.L, kc, &A.boxes, static_cast<const T *>(A.u_in), static_cast<T *>(A.u_out),
                          static_cast<T *>(A.w), static_cast<const TE *>(A.E), static_cast<const T *>(A.rhs),
                          A.tile_ptr, A.loads, (int)gridDim.x, A.zseg};
    march2d_tile_ly<T, PHYS, TE>(V, tile, up);
    finish_sweep(A, (double)up.res, (double)up.dot, tile);
}

// ------------------------------------------------------------- batched 2D kernel
// One launch sweeps every active problem of a batch.  Block b takes tile tiles[b] (its
// problem and the tile's index inside that problem's own 32 x 8 tiling), so each problem
// sees exactly the blocks, the arithmetic and the reduction order of its own
// single-problem sweep; the deterministic reduction runs per problem (its own partials,
// ticket counter, residual slot and restart word).
template <typename T> __device__ __forceinline__ KC<T> kconst_inst(const BatchInst &I);
template <> __device__ __forceinline__ KC<float> kconst_inst<float>(const BatchInst &I) {
    const OpConstF &f = I.kf;
    return {f.ce_par, f.ce_perp, f.cf_lam, f.cf_mu, f.cdiag, f.ct, f.src, f.a, f.b, f.s1};
}
template <> __device__ __forceinline__ KC<double> kconst_inst<double>(const BatchInst &I) {
    const OpConst &k = I.k;
    return {k.ce_par, k.ce_perp, k.cf_lam, k.cf_mu, k.cdiag, k.ct, k.src, I.a, I.b, I.s1};
}

template <typename T, int PHYS>
__device__ __forceinline__ void sweep2d_batch_tile(const BatchLaunch &P, int t, long long sidx, double *sh) {
    const BatchTile bt = P.tiles[t];
    const BatchInst &I = P.inst[bt.inst];
    const int nb = I.gx * I.gy;
    const int mode = sidx < I.apt_until ? 0 : 1;
    const KC<T> kc = kconst_inst<T>(I);
    const long long since = P.adaptive ? sidx - reinterpret_cast<const long long *>(I.ctrl)[CT_RESTART_AT] : 0;
    const int test_dot = mode == 0 && P.adaptive ? P.test_dot : 0;
    Upd<T> up{kc, momentum_k<T>(P.adaptive, kc.a, since), mode, P.local_dt, P.want_res, test_dot,
              static_cast<const T *>(I.rhs), T(0), T(0)};
    const M2View<T, T> V{I.L, kc, &I.boxes, static_cast<const T *>(I.u[P.cur]), static_cast<T *>(I.u[1 - P.cur]),
                         static_cast<T *>(I.w), static_cast<const T *>(I.E), static_cast<const T *>(I.rhs),
                         I.tile_ptr, I.loads, I.gx, I.ly};
    march2d_tile_ly<T, PHYS, T>(V, bt.tile, up);
    // per-problem deterministic reduction, as finish_sweep does for a whole grid
    if (!P.want_res && !test_dot) return;
    const double r = P.want_res ? block_sum((double)up.res, sh) : 0.0;
    const double d = test_dot ? block_sum((double)up.dot, sh) : 0.0;
    if (block_tid() == 0) I.red.partials[(int64_t)nb + bt.tile] = d;
    if (publish_partial(r, I.red, bt.tile, nb)) {
        const double tot = P.want_res ? sum_partials(I.red, 0, nb, sh) : 0.0;
        const double td = test_dot ? sum_partials(I.red, nb, nb, sh) : 0.0;
        if (block_tid() == 0) {
            if (P.want_res) *I.res2 = tot;
            if (test_dot) {
                I.ctrl[CT_DOT] = td;
                if (td < 0.0) reinterpret_cast<long long *>(I.ctrl)[CT_RESTART_AT] = sidx + 1;
            }
            *I.red.counter = 0u;
        }
    }
}

// One block per active tile (the grid is the active tile count, set by the host whenever
// problems finish), so finished problems cost nothing and every block's latency overlaps
// with the other blocks resident on the SM.
template <typename T, int PHYS>
__global__ void __launch_bounds__(32 * M2W, sizeof(T) == 4 ? 6 : 2) sweep2d_batch(const BatchLaunch P) {
    __shared__ double sh[32];
    sweep2d_batch_tile<T, PHYS>(P, blockIdx.x, *P.base + P.sweep_idx, sh);
}

// ------------------------------------------------------------- 3D gather kernel
template <typename T, int PHYS, typename TE = T>
__global__ void __launch_bounds__(128) sweep3d_gather(const SweepArgs A) {
    const Layout &L = A.L;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int kb = A.zb + blockIdx.z * GATHER3_ZS;
    const T *__restrict__ ui = static_cast<const T *>(A.u_in);
    T *__restrict__ uo = static_cast<T *>(A.u_out);
    T *__restrict__ w = static_cast<T *>(A.w);
    const TE *__restrict__ E = static_cast<const TE *>(A.E);
    const KC<T> kc = kconst<T>(A);
    Upd<T> up = make_upd<T>(A, kc);
    const int tile = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    const int l0 = A.tile_ptr[tile], l1 = A.tile_ptr[tile + 1];
    if (i < L.NX && j < L.NY) {
        const int ke = min(kb + GATHER3_ZS, A.zhi + 1);
        for (int k = max(kb, A.zlo); k < ke; ++k) {
            T Ec[2][2][2];
#pragma unroll
            for (int cz = 0; cz < 2; ++cz)
#pragma unroll
                for (int cy = 0; cy < 2; ++cy)
#pragma unroll
                    for (int cx = 0; cx < 2; ++cx) Ec[cz][cy][cx] = (T)__ldg(&E[L.cell(i - 1 + cx, j - 1 + cy, k - 1 + cz)]);
            T S = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) S += Ec[q >> 2][(q >> 1) & 1][q & 1];
            const T diag = kc.cdiag * S;
            const unsigned fm = fixed_mask(A.boxes, i, j, k);
            const int64_t n0 = L.node(i, j, k);
            const int ncnt = ((i > 0) + (i < L.nx)) * ((j > 0) + (j < L.ny)) * ((k > 0) + (k < L.nz));
            for (int r = 0; r < A.nrhs; ++r) {
                if (PHYS == 0) {
                    T U[3][3][3][3];
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        const T *uc = ui + (int64_t)(r * 3 + a) * L.cstride;
#pragma unroll
                        for (int dz = 0; dz < 3; ++dz)
#pragma unroll
                            for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                                for (int dx = 0; dx < 3; ++dx)
                                    U[dz][dy][dx][a] = __ldg(&uc[n0 + (dz - 1) * L.SX * L.SY + (dy - 1) * L.SX + (dx - 1)]);
                    }
                    T Ku[3];
                    ku_elastic_3d<T>(U, Ec, kc, Ku);
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        const int c = r * 3 + a;
                        T F = 0;
                        for (int l = l0; l < l1; ++l)
                            if (A.loads[l].node == n0 && A.loads[l].comp == c) F += load_val<T>(A.loads[l]);
                        up.apply((int64_t)c * L.cstride + n0, (fm >> a) & 1u, Ku[a], F, diag, uo, ui, w);
                    }
                } else {
                    T U[3][3][3];
                    const T *uc = ui + (int64_t)r * L.cstride;
#pragma unroll
                    for (int dz = 0; dz < 3; ++dz)
#pragma unroll
                        for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                            for (int dx = 0; dx < 3; ++dx)
                                U[dz][dy][dx] = __ldg(&uc[n0 + (dz - 1) * L.SX * L.SY + (dy - 1) * L.SX + (dx - 1)]);
                    const T Ku = ku_thermal_3d<T>(U, Ec, kc);
                    T F = kc.src * (T)ncnt;
                    for (int l = l0; l < l1; ++l)
                        if (A.loads[l].node == n0 && A.loads[l].comp == r) F += load_val<T>(A.loads[l]);
                    up.apply((int64_t)r * L.cstride + n0, fm & 1u, Ku, F, diag, uo, ui, w);
                }
            }
        }
    }
    finish_sweep(A, (double)up.res, (double)up.dot, tile);
}

}  // namespace

Tiling gather_tiling(const Layout &L) {
    Tiling t{};
    if (L.dim == 2) {
        t.bx = 32; t.by = 8; t.zs = 1; t.kind = 0;
    } else {
        t.bx = 32; t.by = 4; t.zs = GATHER3_ZS; t.kind = 0;
    }
    t.ox = t.bx;
    t.oy = t.by;
    t.gx = (L.NX + t.ox - 1) / t.ox;
    t.gy = (L.NY + t.oy - 1) / t.oy;
    t.gz = (L.NZ + t.zs - 1) / t.zs;
    return t;
}

Tiling march2d_tiling(const Layout &L, int ly) {
    Tiling t{};
    t.kind = 5;
    t.bx = 32;
    t.by = M2W;
    t.zs = 1;
    t.ox = 30;
    t.gx = (L.NX + t.ox - 1) / t.ox;
    // 4 rows per warp unless asked otherwise: the shortest segments (each warp recomputes one
    // row below its own) measured fastest from 512^2 to 2048 x 1024 nodes, single problems
    // and batches alike -- the kernel is bound by the latency of a warp's row chain
    if (ly <= 0) ly = 4;
    ly = ly >= 16 ? 16 : (ly >= 8 ? 8 : 4);  // the compiled variants
    t.ly = ly;
    t.oy = M2W * ly;
    t.gy = (L.NY + t.oy - 1) / t.oy;
    t.gz = 1;
    return t;
}

Tiling choose_tiling(const Layout &L, int physics, int precision, int nrhs) {
    // 2D, one load case: four sweeps per launch on a shared-memory copy of each tile
    // (sweep2d_tb.cu); PETTO_SWEEP2D=march selects the y-marching kernel (from about
    // 500 x 400 nodes, 32-bit offsets required; the node gather below that), =gather the gather
    const char *env2 = std::getenv("PETTO_SWEEP2D");
    if (L.dim == 2 && nrhs == 1 && !(env2 && (std::strcmp(env2, "march") == 0 || std::strcmp(env2, "gather") == 0)))
        return tb2d_tiling(L, physics, precision, 4);
    if (L.dim == 2 && nrhs == 1 && !(env2 && std::strcmp(env2, "gather") == 0) && (int64_t)L.NX * L.NY >= 200000 &&
        2 * L.cstride < (int64_t(1) << 31) && L.estride < (int64_t(1) << 31))
        return march2d_tiling(L);
    if (L.dim == 3 && physics == 0 && precision == 0) {
        // z-marching kernel: TMA-staged with two owner rows per thread, lean per-plane path,
        // by default; PETTO_MARCH=tma2 selects the two-row kernel it was derived from,
        // tma8 / tma16 one row per thread (32x8 / 32x16 tiles), v1 the register-staged kernel
        Tiling t{};
        const char *env = std::getenv("PETTO_MARCH");
        // the TMA kernel addresses a node column with 32-bit offsets
        if ((env && std::strcmp(env, "v1") == 0 && nrhs == 1) || 3 * nrhs * L.cstride >= (int64_t(1) << 31)) {
            if (nrhs != 1) return gather_tiling(L);
            march3d_tiling(L, t);
        }
        else if (env && std::strcmp(env, "tma8") == 0) march3d_tma_tiling(L, 8, t);
        else if (env && std::strcmp(env, "tma16") == 0) march3d_tma_tiling(L, 16, t);
        else if (env && std::strcmp(env, "tma2") == 0) march3d_tma2_tiling(L, t);
        else march3d_tma3_tiling(L, t);
        return t;
    }
    return gather_tiling(L);
}

// FP64 residual R = F - K(E) u of an FP64 state with the FP32 modulus field (mode 2):
// the defect of the iterative refinement around FP32 sweeps.
cudaError_t launch_residual64(const SweepArgs &a0, const Tiling &t, cudaStream_t s) {
    if (t.kind == 8) return launch_defect3d(a0, t, s);
    SweepArgs a = a0;
    a.zb = t.zn ? t.zb : 0;
    dim3 block(t.bx, t.by, 1), grid(t.gx, t.gy, t.gz);
    if (a.L.dim == 2) {
        if (a.physics == 0) sweep2d_gather<double, 0, float><<<grid, block, 0, s>>>(a);
        else sweep2d_gather<double, 1, float><<<grid, block, 0, s>>>(a);
    } else {
        if (a.physics == 0) sweep3d_gather<double, 0, float><<<grid, block, 0, s>>>(a);
        else sweep3d_gather<double, 1, float><<<grid, block, 0, s>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_sweep(const SweepArgs &a0, const Tiling &t, int precision, cudaStream_t s, const TmaMaps *maps) {
    SweepArgs a = a0;
    a.zseg = t.zs;
    a.zb = t.zn ? t.zb : 0;
    if (t.kind == 1) return launch_march3d(a, t, s);
    if (t.kind == 2 || t.kind == 3) {
        if (!maps || !maps->valid) return cudaErrorInvalidValue;
        return launch_march3d_tma(a, t, *maps, s);
    }
    if (t.kind == 4) {
        if (!maps || !maps->valid) return cudaErrorInvalidValue;
        return launch_march3d_tma2(a, t, *maps, s);
    }
    if (t.kind == 6) {
        if (!maps || !maps->valid) return cudaErrorInvalidValue;
        return launch_march3d_tma3(a, t, *maps, s);
    }
    if (t.kind == 7) return launch_sweep2d_tb(a, t, precision, s);
    if (t.kind == 5) {
        a.zseg = t.ly;
        dim3 block(32, M2W, 1), grid(t.gx, t.gy, 1);
        if (precision == 0) {
            if (a.physics == 0) sweep2d_march<float, 0><<<grid, block, 0, s>>>(a);
            else sweep2d_march<float, 1><<<grid, block, 0, s>>>(a);
        } else {
            if (a.physics == 0) sweep2d_march<double, 0><<<grid, block, 0, s>>>(a);
            else sweep2d_march<double, 1><<<grid, block, 0, s>>>(a);
        }
        return cudaGetLastError();
    }
    dim3 block(t.bx, t.by, 1), grid(t.gx, t.gy, t.gz);
    if (a.L.dim == 2) {
        if (precision == 0) {
            if (a.physics == 0) sweep2d_gather<float, 0><<<grid, block, 0, s>>>(a);
            else sweep2d_gather<float, 1><<<grid, block, 0, s>>>(a);
        } else {
            if (a.physics == 0) sweep2d_gather<double, 0><<<grid, block, 0, s>>>(a);
            else sweep2d_gather<double, 1><<<grid, block, 0, s>>>(a);
        }
    } else {
        if (precision == 0) {
            if (a.physics == 0) sweep3d_gather<float, 0><<<grid, block, 0, s>>>(a);
            else sweep3d_gather<float, 1><<<grid, block, 0, s>>>(a);
        } else {
            if (a.physics == 0) sweep3d_gather<double, 0><<<grid, block, 0, s>>>(a);
            else sweep3d_gather<double, 1><<<grid, block, 0, s>>>(a);
        }
    }
    return cudaGetLastError();
}

template <typename T, int PHYS>
static cudaError_t launch_batch_kernel(const BatchLaunch &p, int ntiles, cudaStream_t s) {
    sweep2d_batch<T, PHYS><<<ntiles, dim3(32, M2W, 1), 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_sweep2d_batch(const BatchLaunch &p, int ntiles, int precision, cudaStream_t s) {
    if (ntiles <= 0) return cudaSuccess;
    if (precision == 0) return p.physics == 0 ? launch_batch_kernel<float, 0>(p, ntiles, s)
                                              : launch_batch_kernel<float, 1>(p, ntiles, s);
    return p.physics == 0 ? launch_batch_kernel<double, 0>(p, ntiles, s) : launch_batch_kernel<double, 1>(p, ntiles, s);
}

}  // namespace petto

// ============================================================================
// Allocation-free residual norm (petto_residual_norm_static in include/petto.h).
//
// A variant of the residual mode of the gather kernel above for callers that cannot
// allocate device memory: inputs in the natural layouts, bounds handled per neighbour
// instead of by the zero ring, and the scratch of the deterministic grid reduction (one
// partial per block, the result, the ticket counter) in one file-scope device array of
// fixed size instead of context-owned memory.
// ============================================================================
#include <mutex>

#include "../../include/petto.h"

namespace petto {
namespace {

constexpr int NA_BLOCK = 256;                    // threads (nodes) per block
constexpr int NA_MAX_BLOCKS = 16384;             // at most 16384 * 256 = 4 194 304 nodes
constexpr int NA_RESULT = NA_MAX_BLOCKS;         // slot of the total
constexpr int NA_TICKET = NA_MAX_BLOCKS + 1;     // slot whose low word is the ticket counter
constexpr int NA_WORDS = NA_MAX_BLOCKS + 8;      // 131 136 bytes in all

// Shared by every call of the entry point on a device, kept between calls.
static __device__ __align__(256) double g_na_scratch[NA_WORDS];

template <int DIM>
__global__ void __launch_bounds__(NA_BLOCK) residual_norm_natural(int nx, int ny, int nz, KC<float> kf,
                                                                   const float *__restrict__ u,
                                                                   const float *__restrict__ E,
                                                                   const float *__restrict__ F,
                                                                   const unsigned char *__restrict__ fixed,
                                                                   double *scratch) {
    __shared__ double sh[32];
    const int NX = nx + 1, NY = ny + 1, NZ = DIM == 3 ? nz + 1 : 1;
    const int64_t nn = (int64_t)NX * NY * NZ;
    const int64_t n = (int64_t)blockIdx.x * NA_BLOCK + threadIdx.x;
    double acc = 0.0;
    if (n < nn) {
        const int i = (int)(n % NX);
        const int64_t r = n / NX;
        const int j = (int)(r % NY), kk = (int)(r / NY);
        auto uat = [&](int a, int di, int dj, int dk) -> float {
            const int ii = i + di, jj = j + dj, k2 = kk + dk;
            if (ii < 0 || ii >= NX || jj < 0 || jj >= NY || k2 < 0 || k2 >= NZ) return 0.f;
            return __ldg(&u[(int64_t)a * nn + ii + (int64_t)NX * (jj + (int64_t)NY * k2)]);
        };
        auto eat = [&](int ci, int cj, int ck) -> float {
            if (ci < 0 || ci >= nx || cj < 0 || cj >= ny || (DIM == 3 && (ck < 0 || ck >= nz))) return 0.f;
            return __ldg(&E[ci + (int64_t)nx * (cj + (int64_t)ny * (DIM == 3 ? ck : 0))]);
        };
        float Ku[3] = {0.f, 0.f, 0.f};
        if (DIM == 2) {
            float U[3][3][2], Ec[2][2];
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                    for (int dx = 0; dx < 3; ++dx) U[dy][dx][a] = uat(a, dx - 1, dy - 1, 0);
#pragma unroll
            for (int cy = 0; cy < 2; ++cy)
#pragma unroll
                for (int cx = 0; cx < 2; ++cx) Ec[cy][cx] = eat(i - 1 + cx, j - 1 + cy, 0);
            float K2[2];
            ku_elastic_2d<float>(U, Ec, kf, K2);
            Ku[0] = K2[0];
            Ku[1] = K2[1];
        } else {
            float U[3][3][3][3], Ec[2][2][2];
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int dz = 0; dz < 3; ++dz)
#pragma unroll
                    for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                        for (int dx = 0; dx < 3; ++dx) U[dz][dy][dx][a] = uat(a, dx - 1, dy - 1, dz - 1);
#pragma unroll
            for (int cz = 0; cz < 2; ++cz)
#pragma unroll
                for (int cy = 0; cy < 2; ++cy)
#pragma unroll
                    for (int cx = 0; cx < 2; ++cx) Ec[cz][cy][cx] = eat(i - 1 + cx, j - 1 + cy, kk - 1 + cz);
            ku_elastic_3d<float>(U, Ec, kf, Ku);
        }
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            const int64_t idx = (int64_t)a * nn + n;
            if (fixed && fixed[idx]) continue;
            const float R = (F ? F[idx] : 0.f) - Ku[a];
            acc += (double)R * (double)R;
        }
    }
    // deterministic reduction through the static scratch: partials in block order
    const double b = block_sum(acc, sh);
    __shared__ bool last;
    if (threadIdx.x == 0) {
        scratch[blockIdx.x] = b;
        __threadfence();
        last = atomicAdd(reinterpret_cast<unsigned *>(&scratch[NA_TICKET]), 1u) == gridDim.x - 1u;
    }
    __syncthreads();
    if (last) {
        __threadfence();
        const volatile double *p = scratch;
        double s = 0.0;
        for (int q = threadIdx.x; q < (int)gridDim.x; q += NA_BLOCK) s += p[q];
        const double t = block_sum(s, sh);
        if (threadIdx.x == 0) {
            scratch[NA_RESULT] = t;
            *reinterpret_cast<unsigned *>(&scratch[NA_TICKET]) = 0u;
        }
    }
}

// Device address of g_na_scratch, looked up once per device (host code may not use the
// symbol itself as a device address).
std::mutex g_na_mutex;
double *g_na_ptr[64] = {nullptr};

}  // namespace
}  // namespace petto

extern "C" petto_status petto_residual_norm_static(const petto_grid *grid, double nu, const float *u,
                                                   const float *E, const float *F, const uint8_t *fixed,
                                                   double *norm2, void *stream) {
    using namespace petto;
    if (!grid || !u || !E || !norm2) return PETTO_EINVAL;
    if (grid->dim != 2 && grid->dim != 3) return PETTO_EINVAL;
    if (grid->nx < 1 || grid->ny < 1 || (grid->dim == 3 && grid->nz < 1) || !(grid->h > 0)) return PETTO_EINVAL;
    if (!(nu > -1.0 && nu < 0.5)) return PETTO_EINVAL;
    const int64_t NX = grid->nx + 1, NY = grid->ny + 1, NZ = grid->dim == 3 ? grid->nz + 1 : 1;
    if (NX > (1 << 24) || NY > (1 << 24) || NZ > (1 << 24)) return PETTO_EINVAL;
    const int64_t nn = NX * NY * NZ;
    const int64_t blocks = (nn + NA_BLOCK - 1) / NA_BLOCK;
    if (blocks > NA_MAX_BLOCKS) return PETTO_EINVAL;  // more than 4 194 304 nodes
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return PETTO_ECUDA;
    double *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_na_mutex);
        if (!g_na_ptr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_na_scratch) != cudaSuccess || !p) return PETTO_ECUDA;
            g_na_ptr[dev] = static_cast<double *>(p);
        }
        scratch = g_na_ptr[dev];
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the ticket counter must start at zero (an interrupted earlier call could have left it)
    if (cudaMemsetAsync(scratch + NA_TICKET, 0, sizeof(double), s) != cudaSuccess) return PETTO_ECUDA;
    const int d = grid->dim;
    const double hs = std::pow(grid->h, d - 2), nq = (double)(1 << d);
    const double lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu)), mu = 1.0 / (2.0 * (1.0 + nu));
    KC<float> k{};
    k.ce_par = (float)(2.0 / nq * hs * (lam + 2.0 * mu));
    k.ce_perp = (float)(2.0 / nq * hs * mu);
    k.cf_lam = (float)(hs * lam / nq);
    k.cf_mu = (float)(hs * mu / nq);
    if (d == 2)
        residual_norm_natural<2><<<(unsigned)blocks, NA_BLOCK, 0, s>>>((int)grid->nx, (int)grid->ny, 0, k, u, E, F,
                                                                       fixed, scratch);
    else
        residual_norm_natural<3><<<(unsigned)blocks, NA_BLOCK, 0, s>>>((int)grid->nx, (int)grid->ny, (int)grid->nz, k,
                                                                       u, E, F, fixed, scratch);
    if (cudaGetLastError() != cudaSuccess) return PETTO_ECUDA;
    if (cudaMemcpyAsync(norm2, scratch + NA_RESULT, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return PETTO_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return PETTO_ECUDA;
    return PETTO_OK;
}
