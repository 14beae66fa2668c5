// sweep2d_tb.cu -- 2D sweeps, several per launch (temporal blocking of the PT / APT sweeps
// of Sec. 2.2 and the Sec. 3.2 systems).
//
// A block owns an output tile of ox x oy nodes.  It stages in shared memory the region of
// (ox + 2K) x (oy + 2K) nodes around the tile -- u, w, the right-hand side F and the support
// mask of each node, and the moduli of the region's cells -- and runs K sweeps on that copy:
// sweep s updates the region shrunk by s nodes on every side, the nodes whose 3 x 3
// neighbourhood sweep s - 1 has updated.  After the K-th sweep it writes the output tile
// back.  Halo nodes are updated redundantly, by every block that stages them, with the same
// arithmetic as in the block that owns them, so every node ends with the value K single
// sweeps give.  A node is evaluated as the y-marching kernel evaluates it (m2_terms: each
// edge and face term once, at its owner node, its shares passed by warp shuffles along x and
// in registers along y; m2_ku, m2_diag, Upd::apply_v; loads added in list order after the
// source term), so the two agree bit for bit.  One read of the grid (from L2 or HBM) and one
// launch then serve K sweeps.
//
// The u field ping-pongs between two global buffers as with single sweeps.  w is updated in
// place within a launch, in shared memory, but a launch of K > 1 sweeps reads the w of its
// halo nodes, which neighbouring blocks own and rewrite: it writes w to a second buffer
// (SweepArgs::w_out).  The sums of R^2 (residual checks) and <R, w> (the restart test of
// the adaptive momentum) are taken on the launch's last sweep, over the output tile; the
// host groups a solve's sweeps so that every check and test sweep ends a launch, so the
// momentum restart, decided on the device after that sweep, applies from the next launch.
#include <algorithm>
#include <cmath>

#include "petto_internal.cuh"
#include "sweep_ops.cuh"

namespace petto {
namespace {

// Asynchronous copy of one element from global to shared memory; the element is zero when
// !valid (source size 0: nothing is read, and src only has to be a valid address).
template <typename T>
__device__ __forceinline__ void cp_async_zfill(T *dst, const T *src, bool valid) {
    static_assert(sizeof(T) == 4 || sizeof(T) == 8, "4- or 8-byte elements");
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    if (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 4 : 0) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 8 : 0) : "memory");
}

// MODE: 0 APT, 1 PT, 2 residual only; LOCAL: local pseudo-time steps (both compile-time, so
// the per-node update carries no branches on them)
template <typename T, int PHYS, int MODE, int LOCAL>
__global__ void __launch_bounds__(TB_THREADS, 2) sweep2d_tb(const __grid_constant__ SweepArgs A, int ox, int oy, int halo) {
    constexpr int C = PHYS == 0 ? 2 : 1;
    extern __shared__ __align__(16) unsigned char tb_raw[];
    const Layout &L = A.L;
    // the region is the output tile and a halo of the tiling's sweeps per launch; a launch of
    // K sweeps (fewer at the end of a run) starts d = halo - K nodes further in
    const int K = A.tb_k, d = halo - K;
    const int RX = ox + 2 * halo, RY = oy + 2 * halo, RN = RX * RY;
    T *su0 = reinterpret_cast<T *>(tb_raw);  // [C][RN], the state before odd sweeps
    T *su1 = su0 + C * RN;                   // [C][RN], the state before even sweeps
    T *sw = su1 + C * RN;                    // [C][RN] w (APT), or R (residual mode)
    T *sf = sw + C * RN;                     // [C][RN] F
    T *se = sf + C * RN;                     // [RY][RX] moduli of the cells whose lower-left node is
                                             // the region node of the same index
    unsigned char *sm = reinterpret_cast<unsigned char *>(se + RN);  // [RN] support mask
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + 32 * ty;
    const int x0 = (int)blockIdx.x * ox - halo, y0 = (int)blockIdx.y * oy - halo;  // grid node of region node (0, 0)
    const KC<T> kc = kconst<T>(A);
    const T *__restrict__ ui = static_cast<const T *>(A.u_in);
    const T *__restrict__ wi = static_cast<const T *>(A.w);
    const T *__restrict__ rhs = static_cast<const T *>(A.rhs);
    const T *__restrict__ E = static_cast<const T *>(A.E);
    const int64_t cs = L.cstride;

    // ---- stage the region with asynchronous copies (cp.async, zero-filled where the source
    // is outside the grid or not needed), so that every load of the block is in flight at once
    for (int ly = ty; ly < RY; ly += 8) {
        const int j = y0 + ly;
        for (int lx = tx; lx < RX; lx += 32) {
            const int i = x0 + lx;
            const int n = ly * RX + lx;
            const bool in = i >= 0 && i < L.NX && j >= 0 && j < L.NY;
            // w is read only where the first sweep updates (the region's border is never
            // updated, and a one-sweep launch reads no node its neighbours write)
            const bool upd = in && lx >= d + 1 && lx < RX - d - 1 && ly >= d + 1 && ly < RY - d - 1;
            const int64_t g = in ? L.node(i, j, 0) : 0;
#pragma unroll
            for (int c = 0; c < C; ++c) {
                cp_async_zfill(&su0[c * RN + n], ui + c * cs + g, in);  // outside the grid: 0
                if (!in) su1[c * RN + n] = T(0);
                cp_async_zfill(&sw[c * RN + n], wi + c * cs + g, upd && MODE == 0);
                if (rhs) cp_async_zfill(&sf[c * RN + n], rhs + c * cs + g, in);
                else sf[c * RN + n] = (PHYS == 1 && in) ? kc.src * (T)(((i > 0) + (i < L.nx)) * ((j > 0) + (j < L.ny)))
                                                        : T(0);
            }
            // a node outside the grid is staged as held in every component: its update writes
            // the zeros it already has, with no branch in the sweep loop
            sm[n] = in ? (unsigned char)fixed_mask(A.boxes, i, j, 0) : (unsigned char)((1u << C) - 1u);
        }
    }
    // cells (outside the grid: modulus 0, as in the zero ring of the global layout)
    for (int cy = ty; cy < RY; cy += 8) {
        const int cj = y0 + cy;
        for (int cx = tx; cx < RX; cx += 32) {
            const int ci = x0 + cx;
            const bool in = ci >= 0 && ci < L.nx && cj >= 0 && cj < L.ny;
            cp_async_zfill(&se[cy * RX + cx], E + (in ? L.cell(ci, cj, 0) : 0), in);
        }
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncthreads();
    // point loads of the region's nodes, from the load lists of the 3 x 3 tiles around this
    // one (the halo is narrower than a tile): one thread per list, so a node's loads are
    // added in list order after the source term, as in the single-sweep kernels
    if (!rhs && tid < 9) {
        const int bx = (int)blockIdx.x + tid % 3 - 1, by = (int)blockIdx.y + tid / 3 - 1;
        if (bx >= 0 && bx < (int)gridDim.x && by >= 0 && by < (int)gridDim.y) {
            const int t = bx + (int)gridDim.x * by;
            for (int l = A.tile_ptr[t]; l < A.tile_ptr[t + 1]; ++l) {
                const LoadEntry le = A.loads[l];
                const int lx = (int)(le.node % L.SX) - OX - x0, ly = (int)(le.node / L.SX) - 1 - y0;
                if (lx >= 0 && lx < RX && ly >= 0 && ly < RY && le.comp < C)
                    sf[le.comp * RN + ly * RX + lx] += load_val<T>(le);
            }
        }
    }
    __syncthreads();

    // ---- K sweeps on the staged copy, in the y-marching form of the single-sweep kernel
    // (m2_terms): the block's 8 warps are nsx column strips x (8 / nsx) row segments.  A warp's
    // lanes hold 32 consecutive region columns, lanes 1..30 its outputs (lane 0 and 31 only
    // pass messages), and it marches its segment's rows from the row below the first, which
    // only produces the messages that row receives.
    constexpr unsigned FULL = 0xffffffffu;
    const int nsx = (RX - 2) / 30, nsy = 8 / nsx;
    const int lane = tx, strip = ty % nsx, segm = ty / nsx;
    const int lx = 30 * strip + lane;  // this lane's region column
    const long long last = sweep_index(A);  // index of this launch's last sweep
    const long long rst = A.adaptive ? reinterpret_cast<const long long *>(A.ctrl)[CT_RESTART_AT] : 0;
    Upd<T> up{kc, T(0), MODE, LOCAL, 0, 0, nullptr, T(0), T(0)};
    for (int s = 1; s <= K; ++s) {
        const T *rd = (s & 1) ? su0 : su1;
        T *wr = (s & 1) ? su1 : su0;
        up.a_eff = momentum_k<T>(A.adaptive, kc.a, A.adaptive ? last - (K - s) - rst : 0);
        // the sums are taken over the output tile on the last sweep only
        const bool sums = s == K && (A.want_res || A.test_dot);
        up.want_res = up.test_dot = 0;
        const int e = s + d;  // sweep s updates the region shrunk by e nodes on every side
        const int sl = (RY - 2 * e + nsy - 1) / nsy;
        const int ys = e + segm * sl, ye = min(ys + sl, RY - e);
        const bool xin = lane >= 1 && lane <= 30 && lx >= e && lx < RX - e;
        if (ys < ye) {  // warp-uniform
            int j = ys - 1;
            T u0[C], u1[C], un[C], un1[C], cy[C], gd[C];
#pragma unroll
            for (int c = 0; c < C; ++c) {
                u0[c] = rd[c * RN + j * RX + lx];
                u1[c] = rd[c * RN + (j + 1) * RX + lx];
                un[c] = __shfl_down_sync(FULL, u0[c], 1);
                cy[c] = gd[c] = T(0);
            }
            T Eb = j >= 1 ? se[(j - 1) * RX + lx] : T(0), Ec = se[j * RX + lx], Elb = T(0);
            for (; j < ye; ++j) {
                const T El = __shfl_up_sync(FULL, Ec, 1);
#pragma unroll
                for (int c = 0; c < C; ++c) un1[c] = __shfl_down_sync(FULL, u1[c], 1);
                T own[C], tx_[C], cyn[C], tg[C], mx[C], gn[C];
                m2_terms<T, PHYS>(u0, un, u1, un1, Eb, Ec, El, kc, own, tx_, cyn, tg);
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    mx[c] = __shfl_up_sync(FULL, tx_[c], 1);
                    gn[c] = PHYS == 0 ? __shfl_up_sync(FULL, tg[c], 1) : T(0);
                }
                if (j >= ys && xin) {
                    const int n = j * RX + lx;
                    const unsigned m = sm[n];
                    if (sums) {
                        const bool own_node = j >= halo && j < halo + oy && lx >= halo && lx < halo + ox;
                        up.want_res = own_node && A.want_res;
                        up.test_dot = own_node && MODE == 0 && A.test_dot;
                    }
                    const T diag = m2_diag(kc, Elb, Eb, El, Ec);
#pragma unroll
                    for (int c = 0; c < C; ++c)
                        up.apply_v(c * RN + n, (m >> c) & 1u, m2_ku(own[c], mx[c], cy[c], gd[c]), sf[c * RN + n], diag,
                                   u0[c], sw[c * RN + n], wr, sw);
                }
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    cy[c] = cyn[c];
                    gd[c] = gn[c];
                    u0[c] = u1[c];
                    un[c] = un1[c];
                }
                Eb = Ec;
                Elb = El;
                if (j + 1 < ye) {
#pragma unroll
                    for (int c = 0; c < C; ++c) u1[c] = rd[c * RN + (j + 2) * RX + lx];
                    Ec = se[(j + 1) * RX + lx];
                }
            }
        }
        __syncthreads();
    }

    // ---- write the output tile back
    const T *fin = (K & 1) ? su1 : su0;
    T *uo = static_cast<T *>(A.u_out);
    T *wo = static_cast<T *>(A.w_out);
    for (int ly = halo + ty; ly < halo + oy; ly += 8) {
        const int j = y0 + ly;
        if (j >= L.NY) break;
        for (int lx = halo + tx; lx < halo + ox; lx += 32) {
            const int i = x0 + lx;
            if (i >= L.NX) break;
            const int n = ly * RX + lx;
            const int64_t g = L.node(i, j, 0);
#pragma unroll
            for (int c = 0; c < C; ++c) {
                if (MODE != 2) uo[c * cs + g] = fin[c * RN + n];
                if (MODE != 1) wo[c * cs + g] = sw[c * RN + n];
            }
        }
    }
    finish_sweep(A, (double)up.res, (double)up.dot, blockIdx.x + (int64_t)gridDim.x * blockIdx.y);
}

}  // namespace

template <typename T, int PHYS, int MODE>
cudaError_t tb2d_set_smem2(int mx) {
    cudaError_t e = cudaFuncSetAttribute(sweep2d_tb<T, PHYS, MODE, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(sweep2d_tb<T, PHYS, MODE, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    return e;
}
template <typename T>
cudaError_t tb2d_set_smem(int mx) {
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = tb2d_set_smem2<T, 0, 0>(mx);
    if (e == cudaSuccess) e = tb2d_set_smem2<T, 0, 1>(mx);
    if (e == cudaSuccess) e = tb2d_set_smem2<T, 0, 2>(mx);
    if (e == cudaSuccess) e = tb2d_set_smem2<T, 1, 0>(mx);
    if (e == cudaSuccess) e = tb2d_set_smem2<T, 1, 1>(mx);
    if (e == cudaSuccess) e = tb2d_set_smem2<T, 1, 2>(mx);
    return e;
}

cudaError_t tb2d_prepare() {
    static unsigned long long prepared = 0;  // one bit per device
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev >= 64 || ((prepared >> dev) & 1ull)) return e;
    int mx = 0;
    e = cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    mx -= 1024;  // the reduction scratch of finish_sweep is static shared memory
    if (e == cudaSuccess) e = tb2d_set_smem<float>(mx);
    if (e == cudaSuccess) e = tb2d_set_smem<double>(mx);
    if (e == cudaSuccess) prepared |= 1ull << dev;
    return e;
}

size_t tb2d_smem(int rx, int ry, int ncomp, int precision) {
    const size_t ts = precision == 0 ? sizeof(float) : sizeof(double);
    return (size_t)(4 * ncomp + 1) * rx * ry * ts + (size_t)rx * ry;
}

// The regions the kernel takes: rx = 30 nsx + 2 columns for nsx = 1, 2, 4 or 8 column
// strips of warps (the other 8 / nsx warps split the rows), any ry.
bool tb2d_region_ok(int rx, int ry, int k) {
    const int nsx = (rx - 2) / 30;
    return rx == 30 * nsx + 2 && (nsx == 1 || nsx == 2 || nsx == 4 || nsx == 8) && rx - 2 * k >= 4 &&
           ry - 2 * k >= 4;
}

// Cost model of a region shape: the busiest SM's tiles x the warp row steps of one tile over
// K sweeps (each warp marches its share of the rows plus one row below it), plus the
// staging, with a penalty for one block per SM (its barriers leave the SM idle while the
// slowest warp finishes a sweep).
Tiling tb2d_tiling(const Layout &L, int physics, int precision, int k, int rx, int ry) {
    Tiling t{};
    t.kind = 7;
    t.bx = 32;
    t.by = 8;
    t.zs = 1;
    t.gz = 1;
    k = k >= 4 ? 4 : (k >= 2 ? 2 : 1);
    t.ly = k;
    const int C = physics == 0 ? 2 : 1;
    if (!tb2d_region_ok(rx, ry, k)) {
        int dev = 0, sms = 152, opt = 232448, per_sm = 233472;
        if (cudaGetDevice(&dev) == cudaSuccess) {
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            cudaDeviceGetAttribute(&opt, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
            cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        }
        double best = INFINITY;
        rx = ry = 0;
        for (int nsx : {1, 2, 4, 8})
            for (int ryc = 8; ryc <= 256; ryc += 4) {
                const int rxc = 30 * nsx + 2, nsy = 8 / nsx;
                if (!tb2d_region_ok(rxc, ryc, k)) continue;
                const size_t smem = tb2d_smem(rxc, ryc, C, precision) + 1024;
                if (smem > (size_t)opt) continue;
                const int blocks_sm = std::min<int>(8, (int)((size_t)per_sm / (smem + 1024)));
                if (blocks_sm < 1) continue;
                const int ox = rxc - 2 * k, oy = ryc - 2 * k;
                const int64_t tiles = (int64_t)((L.NX + ox - 1) / ox) * ((L.NY + oy - 1) / oy);
                double work = 0.25 * rxc * ryc / 32.0;  // staging, in warp row steps
                for (int s = 1; s <= k; ++s) work += 8.0 * ((ryc - 2 * s + nsy - 1) / nsy + 1);
                const double busiest = std::ceil((double)tiles / sms);
                const double cost = busiest * work / (blocks_sm >= 2 ? 1.0 : 0.8);
                if (cost < best * 0.999) {
                    best = cost;
                    rx = rxc;
                    ry = ryc;
                }
            }
        if (rx == 0) {  // nothing fits (a very small device): the smallest region
            rx = 32;
            ry = 2 * k + 4;
        }
    }
    t.ox = rx - 2 * k;
    t.oy = ry - 2 * k;
    t.gx = (L.NX + t.ox - 1) / t.ox;
    t.gy = (L.NY + t.oy - 1) / t.oy;
    return t;
}

template <typename T, int PHYS, int MODE>
void tb2d_launch3(const SweepArgs &a, const Tiling &t, dim3 grid, dim3 block, size_t smem, cudaStream_t s) {
    if (a.local_dt) sweep2d_tb<T, PHYS, MODE, 1><<<grid, block, smem, s>>>(a, t.ox, t.oy, t.ly);
    else sweep2d_tb<T, PHYS, MODE, 0><<<grid, block, smem, s>>>(a, t.ox, t.oy, t.ly);
}
template <typename T, int PHYS>
void tb2d_launch2(const SweepArgs &a, const Tiling &t, dim3 grid, dim3 block, size_t smem, cudaStream_t s) {
    if (a.mode == 0) tb2d_launch3<T, PHYS, 0>(a, t, grid, block, smem, s);
    else if (a.mode == 1) tb2d_launch3<T, PHYS, 1>(a, t, grid, block, smem, s);
    else tb2d_launch3<T, PHYS, 2>(a, t, grid, block, smem, s);
}
template <typename T>
void tb2d_launch(const SweepArgs &a, const Tiling &t, dim3 grid, dim3 block, size_t smem, cudaStream_t s) {
    if (a.physics == 0) tb2d_launch2<T, 0>(a, t, grid, block, smem, s);
    else tb2d_launch2<T, 1>(a, t, grid, block, smem, s);
}

cudaError_t launch_sweep2d_tb(const SweepArgs &a0, const Tiling &t, int precision, cudaStream_t s) {
    SweepArgs a = a0;
    if (!a.w_out) a.w_out = a.w;
    a.tb_k = std::max(1, std::min(a.tb_k, t.ly));  // a launch runs at most the tiling's halo of sweeps
    cudaError_t e = tb2d_prepare();
    if (e != cudaSuccess) return e;
    const int C = a.physics == 0 ? 2 : 1;
    const size_t smem = tb2d_smem(t.ox + 2 * t.ly, t.oy + 2 * t.ly, C, precision);
    const dim3 grid(t.gx, t.gy, 1), block(32, 8, 1);
    if (precision == 0) tb2d_launch<float>(a, t, grid, block, smem, s);
    else tb2d_launch<double>(a, t, grid, block, smem, s);
    return cudaGetLastError();
}

}  // namespace petto
