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
// sweeps give: a node is evaluated as the node-gather kernel evaluates it (ku_elastic_2d /
// ku_thermal_2d, Upd::apply, loads added in list order), so the two agree bit for bit.
// One read of the grid (from L2 or HBM) and one launch then serve K sweeps.
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

constexpr unsigned char TB_OUTSIDE = 0x80;  // mask bit of a staged node outside the grid

template <typename T, int PHYS>
__global__ void __launch_bounds__(TB_THREADS, 2) sweep2d_tb(const __grid_constant__ SweepArgs A, int ox, int oy) {
    constexpr int C = PHYS == 0 ? 2 : 1;
    extern __shared__ __align__(16) unsigned char tb_raw[];
    const Layout &L = A.L;
    const int K = A.tb_k;
    const int RX = ox + 2 * K, RY = oy + 2 * K, RN = RX * RY, EX = RX - 1;
    T *su0 = reinterpret_cast<T *>(tb_raw);  // [C][RN], the state before odd sweeps
    T *su1 = su0 + C * RN;                   // [C][RN], the state before even sweeps
    T *sw = su1 + C * RN;                    // [C][RN] w (APT), or R (residual mode)
    T *sf = sw + C * RN;                     // [C][RN] F
    T *se = sf + C * RN;                     // [RY - 1][RX - 1] cell moduli
    unsigned char *sm = reinterpret_cast<unsigned char *>(se + (RY - 1) * EX);  // [RN] support mask
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + 32 * ty;
    const int x0 = (int)blockIdx.x * ox - K, y0 = (int)blockIdx.y * oy - K;  // grid node of region node (0, 0)
    const KC<T> kc = kconst<T>(A);
    const T *__restrict__ ui = static_cast<const T *>(A.u_in);
    const T *__restrict__ wi = static_cast<const T *>(A.w);
    const T *__restrict__ rhs = static_cast<const T *>(A.rhs);
    const T *__restrict__ E = static_cast<const T *>(A.E);
    const int64_t cs = L.cstride;

    // ---- stage the region: nodes (outside the grid: 0 in both state copies, never updated)
    for (int ly = ty; ly < RY; ly += 8) {
        const int j = y0 + ly;
        for (int lx = tx; lx < RX; lx += 32) {
            const int i = x0 + lx;
            const int n = ly * RX + lx;
            const bool in = i >= 0 && i < L.NX && j >= 0 && j < L.NY;
            // w is read only where the first sweep updates (the region's border is never
            // updated, and a one-sweep launch reads no node its neighbours write)
            const bool upd = in && lx >= 1 && lx < RX - 1 && ly >= 1 && ly < RY - 1;
            const int64_t g = in ? L.node(i, j, 0) : 0;
#pragma unroll
            for (int c = 0; c < C; ++c) {
                su0[c * RN + n] = in ? ui[c * cs + g] : T(0);
                if (!in) su1[c * RN + n] = T(0);
                sw[c * RN + n] = (upd && A.mode == 0) ? wi[c * cs + g] : T(0);
                T f = T(0);
                if (rhs) f = in ? rhs[c * cs + g] : T(0);
                else if (PHYS == 1 && in) f = kc.src * (T)(((i > 0) + (i < L.nx)) * ((j > 0) + (j < L.ny)));
                sf[c * RN + n] = f;
            }
            sm[n] = in ? (unsigned char)fixed_mask(A.boxes, i, j, 0) : TB_OUTSIDE;
        }
    }
    // cells (outside the grid: modulus 0, as in the zero ring of the global layout)
    for (int cy = ty; cy < RY - 1; cy += 8) {
        const int cj = y0 + cy;
        for (int cx = tx; cx < EX; cx += 32) {
            const int ci = x0 + cx;
            const bool in = ci >= 0 && ci < L.nx && cj >= 0 && cj < L.ny;
            se[cy * EX + cx] = in ? E[L.cell(ci, cj, 0)] : T(0);
        }
    }
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

    // ---- K sweeps on the staged copy
    const long long last = sweep_index(A);  // index of this launch's last sweep
    const long long rst = A.adaptive ? reinterpret_cast<const long long *>(A.ctrl)[CT_RESTART_AT] : 0;
    Upd<T> up{kc, T(0), A.mode, A.local_dt, 0, 0, nullptr, T(0), T(0)};
    for (int s = 1; s <= K; ++s) {
        const T *rd = (s & 1) ? su0 : su1;
        T *wr = (s & 1) ? su1 : su0;
        up.a_eff = momentum_k<T>(A.adaptive, kc.a, A.adaptive ? last - (K - s) - rst : 0);
        const bool final_sweep = s == K;
        for (int ly = s + ty; ly < RY - s; ly += 8) {
            const bool own_row = final_sweep && ly >= K && ly < K + oy;
            for (int lx = s + tx; lx < RX - s; lx += 32) {
                const int n = ly * RX + lx;
                const unsigned m = sm[n];
                if (m & TB_OUTSIDE) continue;
                const bool own = own_row && lx >= K && lx < K + ox;
                up.want_res = own && A.want_res;
                up.test_dot = own && A.test_dot;
                T Ec[2][2];
                Ec[0][0] = se[(ly - 1) * EX + lx - 1];
                Ec[0][1] = se[(ly - 1) * EX + lx];
                Ec[1][0] = se[ly * EX + lx - 1];
                Ec[1][1] = se[ly * EX + lx];
                const T S = Ec[0][0] + Ec[0][1] + Ec[1][0] + Ec[1][1];
                const T diag = kc.cdiag * S;
                if (PHYS == 0) {
                    T U[3][3][2];
#pragma unroll
                    for (int a = 0; a < 2; ++a)
#pragma unroll
                        for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                            for (int dx = 0; dx < 3; ++dx) U[dy][dx][a] = rd[a * RN + n + (dy - 1) * RX + (dx - 1)];
                    T Ku[2];
                    ku_elastic_2d<T>(U, Ec, kc, Ku);
#pragma unroll
                    for (int a = 0; a < 2; ++a) up.apply(a * RN + n, (m >> a) & 1u, Ku[a], sf[a * RN + n], diag, wr, rd, sw);
                } else {
                    T U[3][3];
#pragma unroll
                    for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                        for (int dx = 0; dx < 3; ++dx) U[dy][dx] = rd[n + (dy - 1) * RX + (dx - 1)];
                    const T Ku = ku_thermal_2d<T>(U, Ec, kc);
                    up.apply(n, m & 1u, Ku, sf[n], diag, wr, rd, sw);
                }
            }
        }
        __syncthreads();
    }

    // ---- write the output tile back
    const T *fin = (K & 1) ? su1 : su0;
    T *uo = static_cast<T *>(A.u_out);
    T *wo = static_cast<T *>(A.w_out);
    for (int ly = K + ty; ly < K + oy; ly += 8) {
        const int j = y0 + ly;
        if (j >= L.NY) break;
        for (int lx = K + tx; lx < K + ox; lx += 32) {
            const int i = x0 + lx;
            if (i >= L.NX) break;
            const int n = ly * RX + lx;
            const int64_t g = L.node(i, j, 0);
#pragma unroll
            for (int c = 0; c < C; ++c) {
                if (A.mode != 2) uo[c * cs + g] = fin[c * RN + n];
                if (A.mode != 1) wo[c * cs + g] = sw[c * RN + n];
            }
        }
    }
    finish_sweep(A, (double)up.res, (double)up.dot, blockIdx.x + (int64_t)gridDim.x * blockIdx.y);
}

}  // namespace

cudaError_t tb2d_prepare() {
    static unsigned long long prepared = 0;  // one bit per device
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev >= 64 || ((prepared >> dev) & 1ull)) return e;
    int mx = 0;
    e = cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    mx -= 1024;  // the reduction scratch of finish_sweep is static shared memory
    if (e == cudaSuccess) e = cudaFuncSetAttribute(sweep2d_tb<float, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(sweep2d_tb<float, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(sweep2d_tb<double, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(sweep2d_tb<double, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (e == cudaSuccess) prepared |= 1ull << dev;
    return e;
}

size_t tb2d_smem(int rx, int ry, int ncomp, int precision) {
    const size_t ts = precision == 0 ? sizeof(float) : sizeof(double);
    return ((size_t)4 * ncomp * rx * ry + (size_t)(rx - 1) * (ry - 1)) * ts + (size_t)rx * ry;
}

// Cost model of a region shape: the busiest SM's tiles x the node updates of one tile over
// K sweeps (rows split over 8 warps and 32-lane column groups, as the loops run), plus half
// a node update per staged node, with a penalty for one block per SM (its barriers leave the
// SM idle while the slowest warp finishes a sweep).
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
    if (rx <= 0 || ry <= 0) {
        int dev = 0, sms = 152, opt = 232448, per_sm = 233472;
        if (cudaGetDevice(&dev) == cudaSuccess) {
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            cudaDeviceGetAttribute(&opt, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
            cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        }
        double best = INFINITY;
        for (int rxc : {32, 48, 64, 80, 96, 128, 160, 192})
            for (int ryc : {12, 16, 20, 24, 32, 40, 48, 56, 64, 80, 96, 128}) {
                const int ox = rxc - 2 * k, oy = ryc - 2 * k;
                if (ox < 8 || oy < 4) continue;
                const size_t smem = tb2d_smem(rxc, ryc, C, precision) + 1024;
                if (smem > (size_t)opt) continue;
                const int blocks_sm = std::min<int>(8, (int)((size_t)per_sm / (smem + 1024)));
                if (blocks_sm < 1) continue;
                const int64_t tiles = (int64_t)((L.NX + ox - 1) / ox) * ((L.NY + oy - 1) / oy);
                double work = 0.5 * rxc * ryc;
                for (int s = 1; s <= k; ++s)
                    work += (double)((rxc - 2 * s + 31) / 32 * 32) * ((ryc - 2 * s + 7) / 8 * 8);
                const double busiest = std::ceil((double)tiles / sms);
                const double cost = busiest * work / (blocks_sm >= 2 ? 1.0 : 0.8);
                if (cost < best * 0.999) {
                    best = cost;
                    rx = rxc;
                    ry = ryc;
                }
            }
        if (rx <= 0) {  // nothing fits (a very small device): the smallest region
            rx = 32;
            ry = 12;
        }
    }
    t.ox = rx - 2 * k;
    t.oy = ry - 2 * k;
    t.gx = (L.NX + t.ox - 1) / t.ox;
    t.gy = (L.NY + t.oy - 1) / t.oy;
    return t;
}

cudaError_t launch_sweep2d_tb(const SweepArgs &a0, const Tiling &t, int precision, cudaStream_t s) {
    SweepArgs a = a0;
    if (!a.w_out) a.w_out = a.w;
    a.tb_k = std::max(1, std::min(a.tb_k, t.ly));  // a launch runs at most the tiling's halo of sweeps
    cudaError_t e = tb2d_prepare();
    if (e != cudaSuccess) return e;
    const int C = a.physics == 0 ? 2 : 1;
    const size_t smem = tb2d_smem(t.ox + 2 * a.tb_k, t.oy + 2 * a.tb_k, C, precision);
    const dim3 grid(t.gx, t.gy, 1), block(32, 8, 1);
    if (precision == 0) {
        if (a.physics == 0) sweep2d_tb<float, 0><<<grid, block, smem, s>>>(a, t.ox, t.oy);
        else sweep2d_tb<float, 1><<<grid, block, smem, s>>>(a, t.ox, t.oy);
    } else {
        if (a.physics == 0) sweep2d_tb<double, 0><<<grid, block, smem, s>>>(a, t.ox, t.oy);
        else sweep2d_tb<double, 1><<<grid, block, smem, s>>>(a, t.ox, t.oy);
    }
    return cudaGetLastError();
}

}  // namespace petto
