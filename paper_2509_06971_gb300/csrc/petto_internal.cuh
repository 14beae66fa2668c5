// petto_internal.cuh -- device layout, kernel parameter blocks and launchers of libpetto.
//
// Device layout (GB300 HBM).  Every node field is stored per component (structure of
// arrays) with a one-node ring of zeros around the grid, so that the stencil kernels
// read neighbours without bounds tests; rows are padded to a multiple of 32 elements
// (128 B in FP32) and node i = 0 sits at element offset OX = 4 of its row (16-byte
// aligned).  Cell fields used by the sweeps (the modulus E) carry the same zero ring,
// so missing cells outside the domain contribute nothing.  Design fields phi, the
// sensitivity and the update scratch use the compact natural layout [P][cells].
#pragma once

#include <cstdint>
#include <cuda.h>  // CUtensorMap (type only; maps are encoded through the runtime's driver entry point)
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace petto {

constexpr int OX = 4;          // element offset of node/cell i = 0 within a padded row
constexpr int MAX_BOXES = 16;  // Dirichlet boxes per problem
constexpr int MAX_RHS = 4;     // load cases solved together
constexpr int MAX_PHASES = 8;  // design phases

struct Layout {
    int dim;
    int nx, ny, nz;        // cells (nz = 1 in 2D)
    int NX, NY, NZ;        // nodes (NZ = 1 in 2D)
    int64_t SX, SY, SZ;    // padded node pitches (elements); SZ = 1 plane in 2D
    int64_t CX, CY, CZ;    // padded cell pitches
    int64_t cstride;       // elements per node component (SX * SY * SZ)
    int64_t estride;       // elements of the padded cell field (CX * CY * CZ)

    __host__ __device__ __forceinline__ int64_t node(int i, int j, int k) const {
        return ((int64_t)(k + (dim == 3 ? 1 : 0)) * SY + (j + 1)) * SX + (i + OX);
    }
    __host__ __device__ __forceinline__ int64_t cell(int i, int j, int k) const {
        return ((int64_t)(k + (dim == 3 ? 1 : 0)) * CY + (j + 1)) * CX + (i + OX);
    }
    __host__ __device__ __forceinline__ int64_t ncells() const { return (int64_t)nx * ny * nz; }
    __host__ __device__ __forceinline__ int64_t nnodes() const { return (int64_t)NX * NY * NZ; }
};

Layout make_layout(int dim, int nx, int ny, int nz);

struct Box {
    int lo[3], hi[3];
    unsigned mask;
};

struct BoxSet {
    int n;
    Box b[MAX_BOXES];
};

// Sparse nodal load, stored in the padded node index space and grouped per sweep tile.
struct LoadEntry {
    int64_t node;   // padded node index
    int comp;       // component c = r * ncomp + a
    float valf;
    double vald;
};

// Scratch of the deterministic grid reductions (see publish_partial below).
struct RedBuf {
    double *partials;
    unsigned *counter;
};

// Constants of the discrete operator (unit modulus, scaled by h^(d-2)); see sweep.cu.
struct OpConst {
    double ce_par, ce_perp;   // edge force: (2/2^d) h^(d-2) (lam+2mu), (2/2^d) h^(d-2) mu
    double cf_lam, cf_mu;     // face corner force: h^(d-2)/2^d * lam, * mu
    double cdiag;             // diag(K) = cdiag * (sum of adjacent cell moduli)
    double ct;                // thermal edge conductance factor (2/2^d) h^(d-2)
    double src;               // nodal body source per adjacent cell: f h^d / 2^d
};

// Device-side solve control words (doubles in the ctrl array).
constexpr int CT_RESTART_AT = 0;  // sweep index (int64 bits) at which the APT momentum last restarted
constexpr int CT_DOT = 1;         // last tested <R, w> (for inspection)
constexpr int CT_ERR = 2;         // nonzero after a bounded device-side wait ran out
constexpr int CT_BASE = 3;        // (int64) index of the first sweep of a graph-replayed chunk
constexpr int CT_RMAX = 4;        // max |r| of the refinement defect (scaling of its FP16 copy)
constexpr int CT_RSCALE = 5;      // 2^-k: the FP16 right-hand side holds r 2^k
constexpr int CT_N = 8;
constexpr int WAIT_TRIES = 1 << 14;  // default attempts of a bounded ring wait (about 1.6 s at most)

// FP32 copies of the constants, converted once on the host (a double-to-float conversion
// in a kernel runs on the narrow FP64 pipe of GB300).
struct OpConstF {
    float ce_par, ce_perp, cf_lam, cf_mu, cdiag, ct, src;
    float a, b, s1;
};

struct SweepArgs {
    Layout L;
    OpConstF kf;
    int physics;              // 0 elastic, 1 thermal
    int ncomp, nrhs;
    int mode;                 // 0 APT, 1 PT, 2 residual only (writes R to w_or_r)
    int local_dt;
    int want_res;
    int adaptive;             // APT momentum a_k = min(a, (k-1)/(k+2)), k sweeps since the last restart
    int test_dot;             // this sweep tests <R, w_in> < 0 and schedules a restart
    long long sweep_idx;      // index of this sweep within the solve (offset within the chunk when
                              // base_from_ctrl: the chunk's first index is read from the device)
    int base_from_ctrl;
    int zseg;                 // output planes per z segment of the marching kernels
    int rhs_index;            // marching kernels: load case of this launch (one launch per case)
    int zlo, zhi;             // 3D: node planes written by the sweep (a slab of a decomposed grid;
                              // the planes outside hold a neighbour's copied values)
    int zb;                   // 3D: first plane of the first z tile / marching segment (<= zlo)
    double *ctrl;             // solve control words (CT_*)
    const void *rhs;          // dense right-hand side [C][cstride] replacing the loads, or null
    int rhs_half;             // rhs is FP16 holding r 2^k, 2^-k in ctrl[CT_RSCALE] (two-row marching kernel)
    double a, b, s1;
    OpConst k;
    BoxSet boxes;
    const void *u_in;
    void *u_out;
    void *w;                  // APT increment (in place) or R output (mode 2)
    const void *E;
    const int *tile_ptr;      // per-tile CSR of loads
    const LoadEntry *loads;
    double *res2;             // receives sum R^2 (if want_res)
    RedBuf red;
    int wait_tries = WAIT_TRIES;  // TMA marching kernels: attempts of each bounded ring wait
    // 2D sweeps several per launch (sweep2d_tb, kind 7): this launch runs tb_k sweeps, the
    // last of them with index sweep_idx (the R^2 and <R, w> sums are taken on that one); w
    // is read from w and written to w_out, a second buffer when tb_k > 1 (a block reads the
    // old w of the halo nodes it shares with its neighbours)
    int tb_k = 1;
    void *w_out = nullptr;
};

// ---------------------------------------------------------------- batches
// One problem of a batch of 2D problems that advance together, one launch per sweep
// (sweep2d_batch).  Device-resident; the host rewrites it between sweep chunks.
struct BatchInst {
    Layout L;
    OpConstF kf;            // FP32 constants, with this problem's a, b, s1
    OpConst k;              // FP64 constants
    double a, b, s1;
    BoxSet boxes;
    void *u[2];             // state ping-pong buffers
    void *w;                // APT increment
    const void *E;          // cell moduli
    const void *rhs;        // dense right-hand side (refinement correction) or null
    const int *tile_ptr;    // per-tile CSR of loads for the marching tiling
    const LoadEntry *loads;
    RedBuf red;             // this problem's partial sums and ticket counter
    double *res2;           // receives sum R^2 on check sweeps
    double *ctrl;           // CT_RESTART_AT, CT_DOT of this problem
    int gx, gy;             // tiles of this problem (2D marching tiling: 30 x M2W*ly nodes)
    int ly;                 // output rows per warp
    long long apt_until;    // APT while the sweep index is below this, PT from there on
};

struct BatchTile {
    int inst;               // problem
    int tile;               // tile index inside the problem's own tiling (x fastest)
};

struct BatchLaunch {
    const BatchInst *inst;
    const BatchTile *tiles;       // active problems' tiles first; one block per active tile
    const long long *base;        // device word: index of the first sweep of the chunk
    long long sweep_idx;          // this sweep's offset in the chunk
    int cur;                      // u[cur] is read, u[1 - cur] written
    int physics, nrhs, local_dt, want_res, test_dot, adaptive;
};

// ntiles: the active tiles (the leading entries of p.tiles)
cudaError_t launch_sweep2d_batch(const BatchLaunch &p, int ntiles, int precision, cudaStream_t s);

// ---------------------------------------------------------------- reductions

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_max(float v) {
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ double warp_max(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Block-wide sum of one double per thread; result valid in thread 0.  Needs a
// 32-double shared scratch.  All threads of the block must call it.
__device__ __forceinline__ double block_sum(double v, double *sh) {
    const int lane = threadIdx.x & 31;
    const int wid = (threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z)) >> 5;
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nw = (blockDim.x * blockDim.y * blockDim.z + 31) >> 5;
    (void)lane;
    v = warp_sum(v);
    __syncthreads();
    if ((tid & 31) == 0) sh[wid] = v;
    __syncthreads();
    double r = 0.0;
    if (tid < 32) {
        r = tid < nw ? sh[tid] : 0.0;
        r = warp_sum(r);
    }
    return r;
}

// Deterministic grid reduction: every block publishes its partial at partials[idx];
// the last block to arrive (atomic ticket) sums the partials in index order, so the
// result does not depend on block scheduling.  The ticket counter is reset by that last
// block, so kernels on one stream can reuse the same buffer one after another.
__device__ __forceinline__ int block_tid() { return threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z); }
__device__ __forceinline__ int block_nthreads() { return blockDim.x * blockDim.y * blockDim.z; }

// v: the block's total, valid in thread 0.  Returns true in every thread of the last block.
__device__ __forceinline__ bool publish_partial(double v, const RedBuf &rb, int64_t idx, unsigned total) {
    __shared__ bool last;
    if (block_tid() == 0) {
        rb.partials[idx] = v;
        __threadfence();
        last = (atomicAdd(rb.counter, 1u) == total - 1u);
    }
    __syncthreads();
    return last;
}

// Called by all threads of the last block: ordered sum of partials[off, off + n).
__device__ __forceinline__ double sum_partials(const RedBuf &rb, int64_t off, int64_t n, double *sh) {
    __threadfence();
    const volatile double *p = rb.partials;
    double acc = 0.0;
    for (int64_t i = block_tid(); i < n; i += block_nthreads()) acc += p[off + i];
    return block_sum(acc, sh);
}

// Momentum of the adaptive-restart schedule for this sweep: (k-1)/(k+2), k sweeps since the
// last restart (0 for k <= 0).  Integer arithmetic until one FP32 division.
__device__ __forceinline__ long long sweep_index(const SweepArgs &A) {
    return A.base_from_ctrl ? reinterpret_cast<const long long *>(A.ctrl)[CT_BASE] + A.sweep_idx : A.sweep_idx;
}

__device__ __forceinline__ float apt_schedule_k(long long k) {
    if (k <= 0) return 0.f;
    const int ki = k < (1 << 30) ? (int)k : (1 << 30);
    return __fdividef((float)(ki - 1), (float)(ki + 2));
}
__device__ __forceinline__ float apt_schedule(const SweepArgs &A) {
    return apt_schedule_k(sweep_index(A) - reinterpret_cast<const long long *>(A.ctrl)[CT_RESTART_AT]);
}

// Approximate reciprocal (MUFU, ~1 ulp): the local pseudo-time step only scales the update.
__device__ __forceinline__ float fast_rcp(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double fast_rcp(double x) { return 1.0 / x; }

// atomic max for non-negative floating values through their ordered bit patterns
__device__ __forceinline__ void atomic_max_nonneg(double *addr, double v) {
    atomicMax(reinterpret_cast<unsigned long long *>(addr), (unsigned long long)__double_as_longlong(v));
}

// ---------------------------------------------------------------- storage types

template <typename S> struct Store;
template <> struct Store<float> {
    __device__ __forceinline__ static float ld(const float *p, int64_t i) { return p[i]; }
    __device__ __forceinline__ static void st(float *p, int64_t i, float v) { p[i] = v; }
};
template <> struct Store<double> {
    __device__ __forceinline__ static double ld(const double *p, int64_t i) { return p[i]; }
    __device__ __forceinline__ static void st(double *p, int64_t i, double v) { p[i] = v; }
};
template <> struct Store<__nv_bfloat16> {
    __device__ __forceinline__ static float ld(const __nv_bfloat16 *p, int64_t i) { return __bfloat162float(p[i]); }
    __device__ __forceinline__ static void st(__nv_bfloat16 *p, int64_t i, float v) { p[i] = __float2bfloat16_rn(v); }
};
template <> struct Store<__half> {
    __device__ __forceinline__ static float ld(const __half *p, int64_t i) { return __half2float(p[i]); }
    __device__ __forceinline__ static void st(__half *p, int64_t i, float v) { p[i] = __float2half_rn(v); }
};

// ---------------------------------------------------------------- launchers

// Sweep tiling used by the load lists: returns the tile id of a node for the kernel
// that will run (all sweep kernels of one context share one tiling).
struct Tiling {
    int bx, by;        // threads per block in x, y (nodes per tile in x, y)
    int zs;            // nodes per tile in z (3D), 1 in 2D
    int gx, gy, gz;    // tiles per axis
    int ox, oy;        // output nodes per tile in x, y (== bx, by for gather kernels)
    int kind;          // 0 gather, 1 3D z-marching (register-staged), 2/3 3D TMA one row per
                       // thread (32x8 / 32x16), 4 3D TMA two rows per thread, 5 2D y-marching,
                       // 6 3D TMA two rows per thread, lean per-plane path, 7 2D sweeps several per
                       // launch on a shared-memory copy of the tile and its halo, 8 3D FP64 defect
                       // (z-marching, residual only)
    int ly;            // kind 5: output rows per warp (a block's warps take consecutive segments);
                       // kind 7: sweeps per launch (1, 2 or 4)
    int zlo, zn;       // 3D: output node planes [zlo, zlo + zn) (zn = 0: all planes, zlo = 0)
    int zb;            // first plane of the first z tile / segment (<= zlo)
    int order;         // 0: tiles numbered x fastest; 1: z fastest (tile column by column)
    // tile of node (i, j, k), or -1 for a node outside the output planes
    __host__ int tile_of(int i, int j, int k) const {
        if (zn && (k < zlo || k >= zlo + zn)) return -1;
        if (order) return ((i / ox) + gx * (j / oy)) * gz + (k - zb) / zs;
        return (i / ox) + gx * ((j / oy) + gy * ((k - zb) / zs));
    }
    int ntiles() const { return gx * gy * gz; }
};

// The z-marching kernel serves 3D elasticity in FP32 with one load case; every other
// combination uses the node-gather kernels.
Tiling choose_tiling(const Layout &L, int physics, int precision, int nrhs);
Tiling gather_tiling(const Layout &L);
// 2D y-marching tiling: blocks of 32 x M2W threads, 30 output columns per warp and ly rows
// per warp (ly = 0: chosen from the grid size)
Tiling march2d_tiling(const Layout &L, int ly = 0);
constexpr int M2W = 4;  // warps per block of the 2D marching kernel
// FP64 residual R = F - K(E) u of an FP64 state (the defect of the refinement), with the
// node-gather kernels or, on a whole 3D elastic grid, the FP64 z-marching kernel (kind 8)
cudaError_t launch_residual64(const SweepArgs &a, const Tiling &t, cudaStream_t s);
void defect3d_tiling(const Layout &L, Tiling &t);
cudaError_t launch_defect3d(const SweepArgs &a, const Tiling &t, cudaStream_t s);
// z segment length of a marching tiling: fewest (waves of `resident` blocks) x (planes per
// block, with the one-plane halo) over `columns` tile columns
int choose_zseg(int NZ, int columns, int resident);
void march3d_tiling(const Layout &L, Tiling &t);
cudaError_t launch_march3d(const SweepArgs &a, const Tiling &t, cudaStream_t s);

// Tensor maps of the TMA-staged marching kernel: u (4D: x, y, z, component) for each of the
// two ping-pong buffers, and the modulus (3D).
struct TmaMaps {
    bool valid = false;
    CUtensorMap u[2];
    CUtensorMap w;
    CUtensorMap e;
    const void *ubuf[2] = {nullptr, nullptr};
    // FP16 refinement right-hand side of the two-row kernel (made when refinement starts)
    bool rvalid = false;
    CUtensorMap r;
    const void *rbuf = nullptr;
};
bool make_tma_rhs_map(const Layout &L, int ncomp, const void *rhs16, TmaMaps &m);
void march3d_tma_tiling(const Layout &L, int ty, Tiling &t);
void march3d_tma2_tiling(const Layout &L, Tiling &t);
cudaError_t march3d_prepare();
cudaError_t launch_march3d_tma2(const SweepArgs &a, const Tiling &t, const TmaMaps &m, cudaStream_t s);
cudaError_t launch_march3d_tma(const SweepArgs &a, const Tiling &t, const TmaMaps &m, cudaStream_t s);
void march3d_tma3_tiling(const Layout &L, Tiling &t);
cudaError_t launch_march3d_tma3(const SweepArgs &a, const Tiling &t, const TmaMaps &m, cudaStream_t s);
// the two-row marching kernels (kinds 4 and 6): one tiling, one set of tensor maps, FP16
// refinement right-hand side, slabs of a decomposed grid
inline bool two_row_kind(int kind) { return kind == 4 || kind == 6; }

// 2D sweeps several per launch (kind 7).  A block stages the region of (ox + 2 ly) x
// (oy + 2 ly) nodes around its ox x oy output tile; rx, ry give that region for ly sweeps.
constexpr int TB_THREADS = 256;  // 32 x 8
size_t tb2d_smem(int rx, int ry, int ncomp, int precision);
cudaError_t tb2d_prepare();  // shared-memory opt-in of the kernels on the current device (host, once)
// the regions the kernel takes: rx = 30 nsx + 2 (nsx = 1, 2, 4, 8 warp column strips), an
// output tile of at least 4 x 4
bool tb2d_region_ok(int rx, int ry, int k);
// the region (rx, ry) for k sweeps per launch with the lowest modelled cost (rx = ry = 0
// picks it), or the given one; ox = rx - 2k, oy = ry - 2k
Tiling tb2d_tiling(const Layout &L, int physics, int precision, int k, int rx = 0, int ry = 0);
cudaError_t launch_sweep2d_tb(const SweepArgs &a, const Tiling &t, int precision, cudaStream_t s);
bool make_tma_maps(const Layout &L, int ty, int ncomp, void *u0, void *u1, void *w, const void *E, TmaMaps &m);

cudaError_t launch_sweep(const SweepArgs &a, const Tiling &t, int precision, cudaStream_t s,
                         const TmaMaps *maps = nullptr);

struct DesignArgs {
    Layout L;
    int P, interp, storage, precision;
    double penal, e_min;
    double moduli[MAX_PHASES];
};

cudaError_t launch_material(const DesignArgs &d, const void *phi, void *E, cudaStream_t s);

struct SensArgs {
    Layout L;
    int physics, ncomp, nrhs;
    OpConst k;
    double lam, mu;      // unit Lame constants (elastic)
    double h;
    int zc0 = 0, zc1 = 1 << 30;  // cell layers whose energy enters the compliance (a slab's own)
};

// scal layout (device doubles): [0] sum R^2, [1] compliance, [2] work, [8..8+P) max|s_i|,
// [16..16+P) lo_i, [24..24+P) hi_i, [32..32+P) sums, [40..40+P) mean_i, [48..48+P) lambda_i,
// [56..56+P) mean of phi_i over the keep-out region
constexpr int SC_RES = 0, SC_C = 1, SC_W = 2, SC_SMAX = 8, SC_LO = 16, SC_HI = 24, SC_SUM = 32,
              SC_MEAN = 40, SC_LAM = 48, SC_BMEAN = 56, SC_N = 64;

cudaError_t launch_sensitivity(const SensArgs &sa, const DesignArgs &d, const void *u, const void *E,
                               const void *phi, void *s, double *scal, RedBuf rb, cudaStream_t st);

cudaError_t launch_work(const Layout &L, int ncomp, int nrhs, int precision, const LoadEntry *loads, int n_loads,
                        const void *u, double body_src, double *scal, RedBuf rb, cudaStream_t st);

// partial-sum capacity (doubles) a problem of this size needs
int64_t reduction_capacity(const Layout &L, int ntiles, int P);

struct UpdateArgs {
    int64_t ncell;
    int P, vol_mode, n_bisect, precision, storage;
    double alpha_h, kappa_v, kappa_1;
    double V[MAX_PHASES];
    // keep-out region (Sec. 3.4 J_b): cells lo..hi (inclusive) of an nx x ny (x nz) grid
    int keep;                 // 0: no keep-out term
    int nx, ny;
    int klo[3], khi[3];
    double kappa_b;
    double Vb[MAX_PHASES];
    // a slab of a decomposed grid (ext = 1): the bisection sums its own cell layers zc0 .. zc1 - 1
    // (layer cells each) into scal[SC_SUM + p] and the host moves the bracket
    int ext = 0;
    int zc0 = 0, zc1 = 0;
    int64_t layer = 0;
};

cudaError_t launch_update(const UpdateArgs &ua, void *phi, const void *s, void *dscratch, double *scal,
                          RedBuf rb, cudaStream_t st, int64_t *launches);

// One half of a Cahn-Hilliard step for phase p (half 0: mu, 1: phi), with the cell layers above
// the top layer taken from phi_hi ([P][layer]) / mu_hi ([layer]) when given (a slab's neighbour)
cudaError_t launch_ch_half(const Layout &L, int p, int half, int storage, int precision, double gamma_g, double tau,
                           void *phi, void *mu_scratch, const void *phi_hi, const void *mu_hi, cudaStream_t st);
// scal[slot + p] = sum of phase p over cell layers zc0 .. zc1 - 1
cudaError_t launch_layer_sums(const Layout &L, int P, int storage, const void *phi, int zc0, int zc1, double *scal,
                              int slot, RedBuf rb, cudaStream_t st);
// the bisection's sums at the bracket midpoint (ua.ext), and the clamp at lambda = its final midpoint
cudaError_t launch_bisect_sums(const UpdateArgs &ua, const void *dscratch, double *scal, RedBuf rb, cudaStream_t st);
cudaError_t launch_update_apply(const UpdateArgs &ua, void *phi, const void *dscratch, double *scal, cudaStream_t st);
cudaError_t launch_ch(const Layout &L, int P, int storage, int precision, double gamma_g, double tau,
                      void *phi, void *mu_scratch, cudaStream_t st, int64_t *launches);

cudaError_t launch_mean(const Layout &L, int P, int storage, const void *phi, double *scal, RedBuf rb,
                        cudaStream_t st);

}  // namespace petto
