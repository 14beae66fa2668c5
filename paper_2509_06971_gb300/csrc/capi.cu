// capi.cu -- the C ABI of libpetto (declared in include/petto.h): context, buffers,
// problem descriptors, and the host-side control of the PeTTO loop (Fig. 5 of the paper):
// hybrid APT/PT solve with convergence checks every k sweeps (Sec. 2.2), sensitivity
// (Sec. 2.3), design update and Cahn-Hilliard step (Sec. 2.3, 2.4).
#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/petto.h"
#include "petto_internal.cuh"

using namespace petto;

// 3D grids from this many nodes get their sweep kernel picked by the autotuner on the first
// solve (the tuning then costs well under one solve; below it the default choice stands).
// On small or thin grids the one-row TMA kernel can beat the two-row one (the paper's
// 256 x 17 x 85 multi-material grid: 17.6 against 23.8 us per sweep), since it has more
// blocks to spread over the SMs.
constexpr int64_t AUTOTUNE_MIN_NODES = 1 << 17;

struct petto_ctx {
    // problem
    int dim = 2, physics = 0, ncomp = 2, nrhs = 1, P = 1, interp = 0, precision = 0, storage = 0;
    int nx = 0, ny = 0, nz = 1;
    double h = 1.0, nu = 0.3, e_min = 1e-9, penal = 3.0, body_source = 0.0;
    std::vector<double> moduli, vol;
    cudaStream_t stream = nullptr;
    Layout L{};
    Tiling tiling{};   // tiling of the sweep kernel
    Tiling gtiling{};  // tiling of the node-gather kernels (FP64 defect of the refinement)
    TmaMaps tma{};     // tensor maps of the TMA-staged marching kernel
    OpConst k{};
    BoxSet boxes{};
    double lam0 = 0.0, mu0 = 0.0;
    double f_norm = 0.0;
    // keep-out region of the design update (Sec. 3.4 J_b)
    int keep = 0;
    int klo[3] = {0, 0, 0}, khi[3] = {0, 0, 0};
    double kappa_b = 0.0;
    double Vb[MAX_PHASES] = {0};
    // device buffers
    void *u[2] = {nullptr, nullptr};
    void *w = nullptr, *E = nullptr, *phi = nullptr, *s = nullptr, *dscr = nullptr, *mu = nullptr;
    void *rbuf = nullptr, *stage = nullptr;
    void *w_alt = nullptr;  // second w buffer of the 2D sweeps several per launch (kind 7)
    // a slab's copies of the cell layer above its top layer (the neighbour's first own layer):
    // phi ([P][nx ny], storage type) and mu ([nx ny]), for the Cahn-Hilliard step
    void *phi_hi = nullptr, *mu_hi = nullptr;
    size_t stage_bytes = 0;
    double *scal = nullptr;
    unsigned *counter = nullptr;
    double *partials = nullptr;
    int *tile_ptr = nullptr, *gtile_ptr = nullptr;
    LoadEntry *loads = nullptr, *gloads = nullptr;
    int n_loads = 0;
    int ntiles_alloc = 0;
    int64_t partial_cap = 0;
    std::vector<std::pair<std::pair<int64_t, int>, double>> load_list;  // merged (node, component) -> value
    double *ctrl = nullptr;
    void *u64 = nullptr, *r64 = nullptr, *rhs32 = nullptr;
    bool rhs_half = false;  // rhs32 holds the scaled FP16 copy (two-row marching kernel)
    int own_lo = 0, own_n = 0;  // 3D slab of a decomposed grid: node planes the sweeps write
                                // (own_n = 0: every plane)
    int64_t own_z0 = 0;         // plane of the whole grid that local plane 0 is
    int cur = 0;
    int64_t launches = 0;
    int64_t step = 0;
    bool have_sens = false;
    bool profiling = false;
    bool owns_stream = false;
    bool use_graphs = true;  // replay sweep chunks between checks as CUDA graphs
    struct GraphEntry {
        int apt, local_dt, adaptive, cur, ce, res_last;
        const void *rhs;
        double a, b, s1;
        cudaGraphExec_t exec;
        const void *w;     // the w buffer current when the chunk starts
        int flips, swaps;  // ping-pong flips of u and swaps of w over the chunk (its launches)
        int launches;      // kernel launches of the chunk
    };
    std::vector<GraphEntry> graphs;
    // whole design loops of the paper's fixed-count schedule, one graph per starting buffer
    // state (u's ping-pong parity, the current w buffer)
    struct StepGraph {
        int cur;
        const void *w;
        petto_solve_opts so;
        petto_pf_opts po;
        cudaGraphExec_t exec;
        int flips, swaps;
        int64_t launches;
        int profiled;                      // event records around the sweeps (kernel timing)
        cudaGraph_t graph;                 // kept for its event-record nodes
        cudaGraphNode_t ev_node[2];
    };
    std::vector<StepGraph> step_graphs;
    bool trace = false;  // PETTO_TRACE set: print every check residual to stderr
    int wait_tries = WAIT_TRIES;  // attempts of each bounded ring wait of the TMA sweeps
    bool tune_pending = false;    // the first solve picks the sweep kernel by timing (large 3D grids)
    long long slab_restart_at = 0;  // petto_slab_solve: the last restart of the whole grid's momentum
    std::vector<cudaEvent_t> ev_free;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pending;
    std::vector<int> ev_count;  // sweeps covered by each pending event pair
    double prof_ms = 0.0;
    int64_t prof_sweeps = 0, prof_rhs_sweeps = 0;
    std::vector<int> ev_rhs;  // 1 where the timed sweeps read a dense right-hand side
    std::string err;

    size_t tsize() const { return precision == 0 ? 4 : 8; }
    size_t ssize() const { return storage == 0 ? 4 : (storage == 1 ? 8 : 2); }
    int ndofc() const { return nrhs * ncomp; }
    size_t node_bytes() const { return (size_t)ndofc() * L.cstride * tsize(); }
    RedBuf red() const { return RedBuf{partials, counter}; }
};

// The 2D marching kernel: one load case, 32-bit element offsets within a field.
static bool march2d_ok(const petto_ctx *ctx) {
    return ctx->L.dim == 2 && ctx->nrhs == 1 && (int64_t)ctx->ncomp * ctx->L.cstride < (int64_t(1) << 31) &&
           ctx->L.estride < (int64_t(1) << 31);
}

static void clear_graphs(petto_ctx *ctx) {
    for (auto &g : ctx->graphs) cudaGraphExecDestroy(g.exec);
    ctx->graphs.clear();
    for (auto &g : ctx->step_graphs) {
        cudaGraphExecDestroy(g.exec);
        if (g.graph) cudaGraphDestroy(g.graph);
    }
    ctx->step_graphs.clear();
}

namespace {

petto_status fail(petto_ctx *c, petto_status st, const std::string &msg) {
    if (c) c->err = msg;
    return st;
}

#define CK(call)                                                                                       \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess)                                                                         \
            return fail(ctx, PETTO_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));        \
    } while (0)

// ---------------------------------------------------------------- layout packing kernels

template <typename A, typename B> __device__ __forceinline__ B cvt(A v) { return (B)v; }

// natural [C][nodes] <-> padded [C][cstride]
template <typename Src, typename Dst>
__global__ void pack_nodes(Layout L, int C, const Src *__restrict__ src, Dst *__restrict__ dst, int to_padded) {
    const int64_t nn = L.nnodes();
    const int64_t tot = nn * C;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(t / nn);
        const int64_t n = t % nn;
        const int i = (int)(n % L.NX);
        const int64_t r = n / L.NX;
        const int j = (int)(r % L.NY), k = (int)(r / L.NY);
        const int64_t p = (int64_t)c * L.cstride + L.node(i, j, k);
        if (to_padded) dst[p] = (Dst)src[t];
        else dst[t] = (Dst)src[p];
    }
}

// padded cell field -> natural [cells]
template <typename Src, typename Dst>
__global__ void unpack_cells(Layout L, const Src *__restrict__ src, Dst *__restrict__ dst) {
    const int64_t nc = L.ncells();
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc; c += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(c % L.nx);
        const int64_t r = c / L.nx;
        const int j = (int)(r % L.ny), k = (int)(r / L.ny);
        dst[c] = (Dst)src[L.cell(i, j, k)];
    }
}

template <typename Src, typename Dst> __device__ __forceinline__ Dst conv(Src v) { return (Dst)v; }
template <> __device__ __forceinline__ __nv_bfloat16 conv<float, __nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 conv<double, __nv_bfloat16>(double v) { return __double2bfloat16(v); }
template <> __device__ __forceinline__ __half conv<float, __half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __half conv<double, __half>(double v) { return __double2half(v); }
template <> __device__ __forceinline__ float conv<__nv_bfloat16, float>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <> __device__ __forceinline__ double conv<__nv_bfloat16, double>(__nv_bfloat16 v) { return (double)__bfloat162float(v); }
template <> __device__ __forceinline__ float conv<__half, float>(__half v) { return __half2float(v); }
template <> __device__ __forceinline__ double conv<__half, double>(__half v) { return (double)__half2float(v); }
template <> __device__ __forceinline__ __nv_bfloat16 conv<__nv_bfloat16, __nv_bfloat16>(__nv_bfloat16 v) { return v; }
template <> __device__ __forceinline__ __half conv<__half, __half>(__half v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 conv<__half, __nv_bfloat16>(__half v) { return __float2bfloat16_rn(__half2float(v)); }
template <> __device__ __forceinline__ __half conv<__nv_bfloat16, __half>(__nv_bfloat16 v) { return __float2half_rn(__bfloat162float(v)); }

template <typename Src, typename Dst>
__global__ void convert_flat(int64_t n, const Src *__restrict__ src, Dst *__restrict__ dst) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        dst[t] = conv<Src, Dst>(src[t]);
}

__global__ void fill_phase(int64_t nc, int P, const double *__restrict__ vals, int storage, void *phi) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nc * P; t += (int64_t)gridDim.x * blockDim.x) {
        const double v = vals[t / nc];
        if (storage == 0) static_cast<float *>(phi)[t] = (float)v;
        else if (storage == 1) static_cast<double *>(phi)[t] = v;
        else if (storage == 2) static_cast<__nv_bfloat16 *>(phi)[t] = __double2bfloat16(v);
        else static_cast<__half *>(phi)[t] = __double2half(v);
    }
}

int grid_of(int64_t n) {
    int64_t g = (n + 255) / 256;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 8));
}

template <typename F>
cudaError_t dispatch_dtype(int dtype, F &&f) {
    switch (dtype) {
        case PETTO_F32: return f(float{});
        case PETTO_F64: return f(double{});
        case PETTO_BF16: return f(__nv_bfloat16{});
        case PETTO_F16: return f(__half{});
        default: return cudaErrorInvalidValue;
    }
}

size_t dtype_size(int dtype) { return dtype == PETTO_F64 ? 8 : (dtype == PETTO_F32 ? 4 : 2); }

petto_status ensure_stage(petto_ctx *ctx, size_t bytes) {
    if (ctx->stage_bytes >= bytes) return PETTO_OK;
    if (ctx->stage) cudaFree(ctx->stage);
    ctx->stage = nullptr;
    ctx->stage_bytes = 0;
    CK(cudaMalloc(&ctx->stage, bytes));
    ctx->stage_bytes = bytes;
    return PETTO_OK;
}

DesignArgs design_args(const petto_ctx *ctx) {
    DesignArgs d{};
    d.L = ctx->L;
    d.P = ctx->P;
    d.interp = ctx->interp;
    d.storage = ctx->storage;
    d.precision = ctx->precision;
    d.penal = ctx->penal;
    d.e_min = ctx->e_min;
    for (int p = 0; p < (int)ctx->moduli.size() && p < MAX_PHASES; ++p) d.moduli[p] = ctx->moduli[p];
    return d;
}

petto_status refresh_material(petto_ctx *ctx) {
    DesignArgs d = design_args(ctx);
    CK(launch_material(d, ctx->phi, ctx->E, ctx->stream));
    ctx->launches++;
    return PETTO_OK;
}

// --- node field transfer (natural layout, dtype) to/from a padded device buffer
petto_status node_in(petto_ctx *ctx, const void *src, int dtype, int on_device, void *dst_padded) {
    const int C = ctx->ndofc();
    const int64_t n = (int64_t)C * ctx->L.nnodes();
    const void *dsrc = src;
    if (dtype != PETTO_F32 && dtype != PETTO_F64) return fail(ctx, PETTO_EUNSUPPORTED, "node fields are f32/f64");
    if (!on_device) {
        petto_status st = ensure_stage(ctx, n * dtype_size(dtype));
        if (st != PETTO_OK) return st;
        CK(cudaMemcpyAsync(ctx->stage, src, n * dtype_size(dtype), cudaMemcpyHostToDevice, ctx->stream));
        dsrc = ctx->stage;
    }
    const Layout L = ctx->L;
    cudaStream_t s = ctx->stream;
    const int prec = ctx->precision;
    CK(dispatch_dtype(dtype, [&](auto sv) -> cudaError_t {
        using S = decltype(sv);
        if (prec == 0) pack_nodes<S, float><<<grid_of(n), 256, 0, s>>>(L, C, (const S *)dsrc, (float *)dst_padded, 1);
        else pack_nodes<S, double><<<grid_of(n), 256, 0, s>>>(L, C, (const S *)dsrc, (double *)dst_padded, 1);
        return cudaGetLastError();
    }));
    ctx->launches++;
    if (!on_device) CK(cudaStreamSynchronize(ctx->stream));
    return PETTO_OK;
}

petto_status node_out(petto_ctx *ctx, const void *src_padded, void *dst, int dtype, int on_device) {
    const int C = ctx->ndofc();
    const int64_t n = (int64_t)C * ctx->L.nnodes();
    if (dtype != PETTO_F32 && dtype != PETTO_F64) return fail(ctx, PETTO_EUNSUPPORTED, "node fields are f32/f64");
    void *ddst = dst;
    if (!on_device) {
        petto_status st = ensure_stage(ctx, n * dtype_size(dtype));
        if (st != PETTO_OK) return st;
        ddst = ctx->stage;
    }
    const Layout L = ctx->L;
    cudaStream_t s = ctx->stream;
    const int prec = ctx->precision;
    CK(dispatch_dtype(dtype, [&](auto dv) -> cudaError_t {
        using D = decltype(dv);
        if (prec == 0) pack_nodes<float, D><<<grid_of(n), 256, 0, s>>>(L, C, (const float *)src_padded, (D *)ddst, 0);
        else pack_nodes<double, D><<<grid_of(n), 256, 0, s>>>(L, C, (const double *)src_padded, (D *)ddst, 0);
        return cudaGetLastError();
    }));
    ctx->launches++;
    if (!on_device) {
        CK(cudaMemcpyAsync(dst, ctx->stage, n * dtype_size(dtype), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    return PETTO_OK;
}

// flat cell-field transfer with dtype conversion (design phi, sensitivity)
petto_status flat_in(petto_ctx *ctx, const void *src, int dtype, int on_device, void *dst, int dst_dtype, int64_t n) {
    const void *dsrc = src;
    if (!on_device) {
        petto_status st = ensure_stage(ctx, n * dtype_size(dtype));
        if (st != PETTO_OK) return st;
        CK(cudaMemcpyAsync(ctx->stage, src, n * dtype_size(dtype), cudaMemcpyHostToDevice, ctx->stream));
        dsrc = ctx->stage;
    }
    cudaStream_t s = ctx->stream;
    CK(dispatch_dtype(dtype, [&](auto sv) -> cudaError_t {
        using S = decltype(sv);
        return dispatch_dtype(dst_dtype, [&](auto dv) -> cudaError_t {
            using D = decltype(dv);
            convert_flat<S, D><<<grid_of(n), 256, 0, s>>>(n, (const S *)dsrc, (D *)dst);
            return cudaGetLastError();
        });
    }));
    ctx->launches++;
    if (!on_device) CK(cudaStreamSynchronize(ctx->stream));
    return PETTO_OK;
}

petto_status flat_out(petto_ctx *ctx, const void *src, int src_dtype, void *dst, int dtype, int on_device, int64_t n) {
    void *ddst = dst;
    if (!on_device) {
        petto_status st = ensure_stage(ctx, n * dtype_size(dtype));
        if (st != PETTO_OK) return st;
        ddst = ctx->stage;
    }
    cudaStream_t s = ctx->stream;
    CK(dispatch_dtype(src_dtype, [&](auto sv) -> cudaError_t {
        using S = decltype(sv);
        return dispatch_dtype(dtype, [&](auto dv) -> cudaError_t {
            using D = decltype(dv);
            convert_flat<S, D><<<grid_of(n), 256, 0, s>>>(n, (const S *)src, (D *)ddst);
            return cudaGetLastError();
        });
    }));
    ctx->launches++;
    if (!on_device) {
        CK(cudaMemcpyAsync(dst, ctx->stage, n * dtype_size(dtype), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    return PETTO_OK;
}

SweepArgs base_sweep_args(petto_ctx *ctx) {
    SweepArgs a{};
    a.L = ctx->L;
    a.physics = ctx->physics;
    a.ncomp = ctx->ncomp;
    a.nrhs = ctx->nrhs;
    a.k = ctx->k;
    a.boxes = ctx->boxes;
    a.E = ctx->E;
    a.tile_ptr = ctx->tile_ptr;
    a.loads = ctx->loads;
    a.res2 = ctx->scal + SC_RES;
    a.red = ctx->red();
    a.ctrl = ctx->ctrl;
    a.rhs = nullptr;
    a.zlo = ctx->own_n ? ctx->own_lo : 0;
    a.zhi = ctx->own_n ? ctx->own_lo + ctx->own_n - 1 : ctx->L.NZ - 1;
    a.wait_tries = ctx->wait_tries;
    const OpConst &k = ctx->k;
    a.kf = OpConstF{(float)k.ce_par, (float)k.ce_perp, (float)k.cf_lam, (float)k.cf_mu, (float)k.cdiag, (float)k.ct,
                    (float)k.src, 0.f, 0.f, 0.f};
    return a;
}

// Per-sweep controls beyond the constants: adaptive momentum, its restart test, the
// index of the sweep within the solve, and an optional dense right-hand side.
struct SweepCtl {
    int adaptive = 0;
    int test_dot = 0;
    long long idx = 0;
    int base_from_ctrl = 0;
    const void *rhs = nullptr;
};

// Sweeps of one kind (0 APT, 1 PT) from u[cur] into u[1-cur] in one launch, flipping cur:
// one sweep, or (the 2D kernel that runs several per launch, kind 7) nsw sweeps with indices
// sc.idx .. sc.idx + nsw - 1, the last of them the one that sums R^2 / tests <R, w> (the
// caller ends its groups on those sweeps); APT sweeps then write w to the second buffer
// and the two swap (PT sweeps leave w alone).
petto_status one_sweep(petto_ctx *ctx, int kind, double a, double b, double s1, int local_dt, bool want_res,
                       const SweepCtl &sc = SweepCtl(), int nsw = 1) {
    if (nsw > 1 && (ctx->tiling.kind != 7 || nsw > ctx->tiling.ly || !ctx->w_alt))
        return fail(ctx, PETTO_EINVAL, "several sweeps per launch need the 2D kernel that runs them");
    SweepArgs A = base_sweep_args(ctx);
    A.mode = kind;
    A.local_dt = local_dt;
    A.want_res = want_res ? 1 : 0;
    A.adaptive = sc.adaptive;
    A.test_dot = kind == 0 && sc.adaptive ? sc.test_dot : 0;
    A.sweep_idx = sc.idx + nsw - 1;
    A.base_from_ctrl = sc.base_from_ctrl;
    A.rhs = sc.rhs;
    A.rhs_half = sc.rhs && sc.rhs == ctx->rhs32 && ctx->rhs_half;
    A.a = a;
    A.b = b;
    A.s1 = s1;
    A.kf.a = (float)a;
    A.kf.b = (float)b;
    A.kf.s1 = (float)s1;
    A.u_in = ctx->u[ctx->cur];
    A.u_out = ctx->u[1 - ctx->cur];
    A.w = ctx->w;
    A.tb_k = nsw;
    const bool w_swap = nsw > 1 && kind == 0;  // PT sweeps neither read nor write w
    A.w_out = w_swap ? ctx->w_alt : ctx->w;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (ctx->profiling && !sc.base_from_ctrl) {
        for (cudaEvent_t *e : {&e0, &e1}) {
            if (!ctx->ev_free.empty()) {
                *e = ctx->ev_free.back();
                ctx->ev_free.pop_back();
            } else {
                CK(cudaEventCreate(e));
            }
        }
        CK(cudaEventRecord(e0, ctx->stream));
    }
    CK(launch_sweep(A, ctx->tiling, ctx->precision, ctx->stream, &ctx->tma));
    if (ctx->profiling && !sc.base_from_ctrl) {
        CK(cudaEventRecord(e1, ctx->stream));
        ctx->ev_pending.emplace_back(e0, e1);
        ctx->ev_count.push_back(nsw);
        ctx->ev_rhs.push_back(sc.rhs != nullptr);
    }
    ctx->launches++;
    ctx->cur ^= 1;
    if (w_swap) std::swap(ctx->w, ctx->w_alt);
    return PETTO_OK;
}

// Sweeps per launch for the group starting at sweep j of a run of n (indices counted from
// the run's start, which sits on a multiple of 4): the kernel's count, halved until the
// group starts on a multiple of its size and fits the run.  Groups of 1, 2 or 4 aligned so
// end every test sweep (j mod 4 = 3) and the run's last sweep.
int sweep_group(const petto_ctx *ctx, int64_t j, int64_t n) {
    int g = ctx->tiling.kind == 7 && ctx->w_alt ? ctx->tiling.ly : 1;
    while (g > 1 && (j % g != 0 || j + g > n)) g >>= 1;
    return g;
}

petto_status read_scal(petto_ctx *ctx, double *host) {
    double ctrl[CT_N];
    CK(cudaMemcpyAsync(host, ctx->scal, sizeof(double) * SC_N, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(ctrl, ctx->ctrl, sizeof(double) * CT_N, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (ctrl[CT_ERR] != 0.0) return fail(ctx, PETTO_ETIMEOUT, "a bounded device-side wait ran out in a sweep");
    return PETTO_OK;
}


void build_opconst(petto_ctx *ctx) {
    const int d = ctx->dim;
    const double hs = std::pow(ctx->h, d - 2);
    const double nq = (double)(1 << d);
    const double lam = ctx->nu / ((1.0 + ctx->nu) * (1.0 - 2.0 * ctx->nu));
    const double mu = 1.0 / (2.0 * (1.0 + ctx->nu));
    ctx->lam0 = lam;
    ctx->mu0 = mu;
    OpConst &k = ctx->k;
    k.ce_par = 2.0 / nq * hs * (lam + 2.0 * mu);
    k.ce_perp = 2.0 / nq * hs * mu;
    k.cf_lam = hs * lam / nq;
    k.cf_mu = hs * mu / nq;
    k.ct = 2.0 / nq * hs;
    k.cdiag = ctx->physics == 0 ? 2.0 / nq * hs * (lam + (d + 1) * mu) : 2.0 / nq * hs * d;
    k.src = ctx->body_source * std::pow(ctx->h, d) / nq;
}

petto_status drain_profile(petto_ctx *ctx) {
    for (size_t q = 0; q < ctx->ev_pending.size(); ++q) {
        auto &pr = ctx->ev_pending[q];
        CK(cudaEventSynchronize(pr.second));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, pr.first, pr.second));
        ctx->prof_ms += ms;
        const int cnt = q < ctx->ev_count.size() ? ctx->ev_count[q] : 1;
        ctx->prof_sweeps += cnt;
        if (q < ctx->ev_rhs.size() && ctx->ev_rhs[q]) ctx->prof_rhs_sweeps += cnt;
        ctx->ev_free.push_back(pr.first);
        ctx->ev_free.push_back(pr.second);
    }
    ctx->ev_pending.clear();
    ctx->ev_count.clear();
    ctx->ev_rhs.clear();
    return PETTO_OK;
}


// Switch the sweep kernel's tiling: rebuild the per-tile load table (and the tensor maps of
// the TMA-staged kernels), growing the tile and partial-sum buffers when needed.
// A tiling restricted to the context's output planes (a slab of a decomposed grid): z tiles
// (gather) or z segments (marching) start at the slab's first plane.
// Tiling of the FP64 defect of the refinement: the FP64 z-marching kernel on 3D elastic
// grids and their slabs, the node gather otherwise (2D, heat; PETTO_DEFECT=gather forces it)
Tiling defect_tiling(const petto_ctx *ctx) {
    const char *env = std::getenv("PETTO_DEFECT");
    if (ctx->dim == 3 && ctx->physics == 0 && !(env && std::strcmp(env, "gather") == 0)) {
        Tiling t{};
        defect3d_tiling(ctx->L, t);
        return t;
    }
    return gather_tiling(ctx->L);
}

Tiling own_planes(const petto_ctx *ctx, Tiling t) {
    if (!ctx->own_n) return t;
    t.zlo = ctx->own_lo;
    t.zn = ctx->own_n;
    t.zb = t.zlo;
    if (two_row_kind(t.kind)) {
        // marching segments start on even planes of the whole grid, as the whole grid's do
        // (its segment length is even), so every plane is computed as it is there
        if ((t.zlo + ctx->own_z0) & 1) t.zb = std::max(t.zlo - 1, 0);
        const int span = t.zlo + t.zn - t.zb;
        t.zs = std::min(t.zs, span);
        if (t.zs < span && (t.zs & 1)) ++t.zs;
        t.gz = (span + t.zs - 1) / t.zs;
    } else {
        t.gz = (t.zn + t.zs - 1) / t.zs;
    }
    return t;
}

petto_status set_tiling(petto_ctx *ctx, const Tiling &t0) {
    if (ctx->own_n && t0.kind != 0 && !two_row_kind(t0.kind))
        return fail(ctx, PETTO_EUNSUPPORTED, "a slab context sweeps with the node-gather or two-row marching kernel");
    const Tiling t = own_planes(ctx, t0);
    const int NX = ctx->L.NX, NY = ctx->L.NY;
    const int nt = t.ntiles();
    std::vector<int> tptr(nt + 1, 0);
    std::vector<std::pair<int, LoadEntry>> tmp;
    for (auto &kv : ctx->load_list) {
        const int64_t n = kv.first.first;
        const int i = (int)(n % NX), j = (int)((n / NX) % NY), k = (int)(n / ((int64_t)NX * NY));
        LoadEntry le{};
        le.node = ctx->L.node(i, j, k);
        le.comp = kv.first.second;
        le.vald = kv.second;
        le.valf = (float)kv.second;
        const int tl = t.tile_of(i, j, k);
        if (tl >= 0) tmp.emplace_back(tl, le);  // loads on planes outside a slab belong to a neighbour
    }
    std::stable_sort(tmp.begin(), tmp.end(), [](const auto &x, const auto &y) { return x.first < y.first; });
    std::vector<LoadEntry> ent;
    for (auto &pr : tmp) {
        tptr[pr.first + 1]++;
        ent.push_back(pr.second);
    }
    for (int q = 0; q < nt; ++q) tptr[q + 1] += tptr[q];
    CK(cudaStreamSynchronize(ctx->stream));
    clear_graphs(ctx);
    if (nt > ctx->ntiles_alloc) {
        CK(cudaFree(ctx->tile_ptr));
        ctx->tile_ptr = nullptr;
        CK(cudaMalloc(&ctx->tile_ptr, sizeof(int) * (nt + 1)));
        ctx->ntiles_alloc = nt;
    }
    const int64_t cap = reduction_capacity(ctx->L, std::max(nt, ctx->gtiling.ntiles()), ctx->P);
    if (cap > ctx->partial_cap) {
        CK(cudaFree(ctx->partials));
        ctx->partials = nullptr;
        CK(cudaMalloc(&ctx->partials, sizeof(double) * cap));
        ctx->partial_cap = cap;
    }
    if (t.kind == 7) {
        CK(tb2d_prepare());
        if (!ctx->w_alt) {
            CK(cudaMalloc(&ctx->w_alt, ctx->node_bytes()));
            CK(cudaMemset(ctx->w_alt, 0, ctx->node_bytes()));
        }
    }
    CK(cudaMemcpy(ctx->tile_ptr, tptr.data(), sizeof(int) * (nt + 1), cudaMemcpyHostToDevice));
    if (!ent.empty()) CK(cudaMemcpy(ctx->loads, ent.data(), sizeof(LoadEntry) * ent.size(), cudaMemcpyHostToDevice));
    if ((t.kind >= 2 && t.kind <= 4) || t.kind == 6) {
        const int ty = t.kind == 2 ? 8 : 16;
        if (!make_tma_maps(ctx->L, ty, ctx->ndofc(), ctx->u[0], ctx->u[1], ctx->w, ctx->E, ctx->tma))
            return fail(ctx, PETTO_ECUDA, "tensor map creation failed");
    }
    ctx->tiling = t;
    return PETTO_OK;
}
}  // namespace

// ==================================================================== C ABI

extern "C" {

const char *petto_status_string(petto_status s) {
    switch (s) {
        case PETTO_OK: return "PETTO_OK";
        case PETTO_EINVAL: return "PETTO_EINVAL";
        case PETTO_ENOMEM: return "PETTO_ENOMEM";
        case PETTO_ECUDA: return "PETTO_ECUDA";
        case PETTO_ENOTCONV: return "PETTO_ENOTCONV";
        case PETTO_EDIVERGED: return "PETTO_EDIVERGED";
        case PETTO_ETIMEOUT: return "PETTO_ETIMEOUT";
        case PETTO_EUNSUPPORTED: return "PETTO_EUNSUPPORTED";
    }
    return "PETTO_UNKNOWN";
}

const char *petto_last_error(const petto_ctx *ctx) {
    if (!ctx) return "no context";
    return ctx->err.c_str();
}

int64_t petto_launch_count(const petto_ctx *ctx) { return ctx ? ctx->launches : 0; }

petto_status petto_profile(petto_ctx *ctx, int enable) {
    if (!ctx) return PETTO_EINVAL;
    petto_status st = drain_profile(ctx);
    if (st != PETTO_OK) return st;
    ctx->profiling = enable != 0;
    return PETTO_OK;
}

petto_status petto_profile_read(petto_ctx *ctx, double *sweep_ms, int64_t *sweeps, int64_t *rhs_sweeps) {
    if (!ctx) return PETTO_EINVAL;
    petto_status st = drain_profile(ctx);
    if (st != PETTO_OK) return st;
    if (sweep_ms) *sweep_ms = ctx->prof_ms;
    if (sweeps) *sweeps = ctx->prof_sweeps;
    if (rhs_sweeps) *rhs_sweeps = ctx->prof_rhs_sweeps;
    ctx->prof_ms = 0.0;
    ctx->prof_sweeps = 0;
    ctx->prof_rhs_sweeps = 0;
    return PETTO_OK;
}

void petto_destroy(petto_ctx *ctx) {
    if (!ctx) return;
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    for (auto &pr : ctx->ev_pending) {
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
    }
    for (auto e : ctx->ev_free) cudaEventDestroy(e);
    clear_graphs(ctx);
    void *bufs[] = {ctx->u[0], ctx->u[1], ctx->w, ctx->w_alt, ctx->E, ctx->phi, ctx->s, ctx->dscr, ctx->mu, ctx->rbuf,
                    ctx->stage, ctx->scal, ctx->counter, ctx->tile_ptr, ctx->loads, ctx->partials,
                    ctx->gtile_ptr, ctx->gloads, ctx->ctrl, ctx->u64, ctx->r64, ctx->rhs32, ctx->phi_hi, ctx->mu_hi};
    for (void *b : bufs)
        if (b) cudaFree(b);
    if (ctx->owns_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

petto_status petto_create(const petto_grid *grid, const petto_materials *mat, const petto_loads *loads,
                          const petto_bcs *bcs, const double *vol_frac, const petto_options *opt, petto_ctx **out) {
    if (!out) return PETTO_EINVAL;
    *out = nullptr;
    if (!grid || !mat || !vol_frac || !opt) return PETTO_EINVAL;
    if (grid->dim != 2 && grid->dim != 3) return PETTO_EINVAL;
    if (grid->nx < 1 || grid->ny < 1 || (grid->dim == 3 && grid->nz < 1)) return PETTO_EINVAL;
    if (grid->nx > (1 << 24) || grid->ny > (1 << 24) || grid->nz > (1 << 24) || !(grid->h > 0)) return PETTO_EINVAL;
    if (opt->precision != PETTO_F32 && opt->precision != PETTO_F64) return PETTO_EINVAL;
    if (opt->storage < PETTO_F32 || opt->storage > PETTO_F16) return PETTO_EINVAL;
    if (opt->nrhs < 1 || opt->nrhs > MAX_RHS) return PETTO_EINVAL;
    if (mat->physics != PETTO_ELASTIC && mat->physics != PETTO_THERMAL) return PETTO_EINVAL;
    if (mat->n_phases < 1 || mat->n_phases > MAX_PHASES || !mat->modulus) return PETTO_EINVAL;
    if (mat->interp == PETTO_SIMP_MODIFIED && mat->n_phases != 1) return PETTO_EINVAL;
    if (mat->physics == PETTO_ELASTIC && !(mat->nu > -1.0 && mat->nu < 0.5)) return PETTO_EINVAL;

    petto_ctx *ctx = new (std::nothrow) petto_ctx();
    if (!ctx) return PETTO_ENOMEM;
    ctx->dim = grid->dim;
    ctx->nx = (int)grid->nx;
    ctx->ny = (int)grid->ny;
    ctx->nz = grid->dim == 3 ? (int)grid->nz : 1;
    ctx->h = grid->h;
    ctx->physics = mat->physics;
    ctx->ncomp = mat->physics == PETTO_ELASTIC ? grid->dim : 1;
    ctx->nrhs = opt->nrhs;
    ctx->P = mat->n_phases;
    ctx->interp = mat->interp;
    ctx->nu = mat->nu;
    ctx->e_min = mat->e_min;
    ctx->penal = mat->penal;
    ctx->precision = opt->precision;
    ctx->storage = opt->storage;
    ctx->stream = (cudaStream_t)opt->stream;
    if (!ctx->stream) {
        // the legacy default stream cannot be captured: use a blocking stream of our own, which
        // still orders with work on the legacy default stream
        if (cudaStreamCreate(&ctx->stream) != cudaSuccess) {
            delete ctx;
            return PETTO_ECUDA;
        }
        ctx->owns_stream = true;
    }
    ctx->use_graphs = std::getenv("PETTO_NO_GRAPHS") == nullptr;
    ctx->moduli.assign(mat->modulus, mat->modulus + mat->n_phases);
    ctx->vol.assign(vol_frac, vol_frac + mat->n_phases);
    ctx->body_source = loads ? loads->body_source : 0.0;
    if (ctx->body_source != 0.0 && ctx->physics != PETTO_THERMAL) {
        delete ctx;
        return PETTO_EINVAL;
    }
    ctx->trace = std::getenv("PETTO_TRACE") != nullptr;
    ctx->L = make_layout(ctx->dim, ctx->nx, ctx->ny, ctx->nz);
    ctx->tiling = choose_tiling(ctx->L, ctx->physics, ctx->precision, ctx->nrhs);
    // large 3D elastic FP32 grids: the first solve times the applicable sweep kernels and
    // keeps the fastest (once per grid shape in the process), unless a kernel is chosen first
    ctx->tune_pending = ctx->dim == 3 && ctx->physics == 0 && ctx->precision == PETTO_F32 &&
                        ctx->L.nnodes() >= AUTOTUNE_MIN_NODES && !std::getenv("PETTO_MARCH");
    build_opconst(ctx);

    // supports
    if (bcs && bcs->n_boxes > 0) {
        if (bcs->n_boxes > MAX_BOXES || !bcs->box || !bcs->comp_mask) {
            petto_destroy(ctx);
            return PETTO_EINVAL;
        }
        ctx->boxes.n = bcs->n_boxes;
        for (int q = 0; q < bcs->n_boxes; ++q) {
            for (int a = 0; a < 3; ++a) {
                ctx->boxes.b[q].lo[a] = (int)bcs->box[6 * q + a];
                ctx->boxes.b[q].hi[a] = (int)bcs->box[6 * q + 3 + a];
            }
            ctx->boxes.b[q].mask = bcs->comp_mask[q];
        }
    }
    auto is_fixed = [&](int i, int j, int k, int a) {
        for (int q = 0; q < ctx->boxes.n; ++q) {
            const Box &b = ctx->boxes.b[q];
            if (i >= b.lo[0] && i <= b.hi[0] && j >= b.lo[1] && j <= b.hi[1] && k >= b.lo[2] && k <= b.hi[2] &&
                ((b.mask >> a) & 1u))
                return true;
        }
        return false;
    };

    // nodal loads: merge duplicates (node, component) and keep them sorted by the tile of
    // each sweep kernel that looks them up
    std::map<std::pair<int64_t, int>, double> merged;  // (natural node, component) -> value
    const int NX = ctx->L.NX, NY = ctx->L.NY, NZ = ctx->L.NZ;
    if (loads && loads->n > 0) {
        if (!loads->node || !loads->comp || !loads->value) {
            petto_destroy(ctx);
            return PETTO_EINVAL;
        }
        for (int64_t e = 0; e < loads->n; ++e) {
            const int i = (int)loads->node[3 * e], j = (int)loads->node[3 * e + 1];
            const int k = ctx->dim == 3 ? (int)loads->node[3 * e + 2] : 0;
            const int a = loads->comp[e];
            const int r = loads->rhs ? loads->rhs[e] : 0;
            if (i < 0 || i >= NX || j < 0 || j >= NY || k < 0 || k >= NZ || a < 0 || a >= ctx->ncomp || r < 0 ||
                r >= ctx->nrhs) {
                ctx->err = "load entry out of range";
                petto_destroy(ctx);
                return PETTO_EINVAL;
            }
            const int64_t n = (int64_t)i + (int64_t)NX * ((int64_t)j + (int64_t)NY * k);
            merged[std::make_pair(n, r * ctx->ncomp + a)] += loads->value[e];
        }
    }
    ctx->gtiling = defect_tiling(ctx);
    ctx->load_list.assign(merged.begin(), merged.end());
    auto table = [&](const Tiling &t, std::vector<int> &tptr, std::vector<LoadEntry> &ent) {
        const int nt = t.ntiles();
        tptr.assign(nt + 1, 0);
        std::vector<std::pair<int, LoadEntry>> tmp;
        for (auto &kv : merged) {
            const int64_t n = kv.first.first;
            const int i = (int)(n % NX), j = (int)((n / NX) % NY), k = (int)(n / ((int64_t)NX * NY));
            LoadEntry le{};
            le.node = ctx->L.node(i, j, k);
            le.comp = kv.first.second;
            le.vald = kv.second;
            le.valf = (float)kv.second;
            tmp.emplace_back(t.tile_of(i, j, k), le);
        }
        std::stable_sort(tmp.begin(), tmp.end(), [](const auto &x, const auto &y) { return x.first < y.first; });
        ent.clear();
        for (auto &pr : tmp) {
            tptr[pr.first + 1]++;
            ent.push_back(pr.second);
        }
        for (int q = 0; q < nt; ++q) tptr[q + 1] += tptr[q];
    };
    std::vector<int> tptr, gptr;
    std::vector<LoadEntry> tent, gent;
    table(ctx->tiling, tptr, tent);
    table(ctx->gtiling, gptr, gent);
    // the defect's load table also serves the node-gather tiling a slab switches to
    const int ntiles = ctx->tiling.ntiles(),
              gntiles = std::max(ctx->gtiling.ntiles(), gather_tiling(ctx->L).ntiles());
    ctx->n_loads = (int)tent.size();
    // ||F|| over free DOFs (point loads plus the body source)
    double f2 = 0.0;
    for (auto &kv : merged) {
        const int64_t n = kv.first.first;
        const int i = (int)(n % NX), j = (int)((n / NX) % NY), k = (int)(n / ((int64_t)NX * NY));
        const int a = kv.first.second % ctx->ncomp;
        if (is_fixed(i, j, k, a)) continue;
        double F = kv.second;
        if (ctx->body_source != 0.0) {
            const int cnt = ((i > 0) + (i < ctx->nx)) * ((j > 0) + (j < ctx->ny)) *
                            (ctx->dim == 3 ? ((k > 0) + (k < ctx->nz)) : 1);
            F += ctx->k.src * cnt;
        }
        f2 += F * F;
    }
    if (ctx->body_source != 0.0) {
        for (int r = 0; r < ctx->nrhs; ++r)
            for (int k = 0; k < NZ; ++k)
                for (int j = 0; j < NY; ++j)
                    for (int i = 0; i < NX; ++i) {
                        const int64_t n = (int64_t)i + (int64_t)NX * (j + (int64_t)NY * k);
                        if (merged.count(std::make_pair(n, r)) || is_fixed(i, j, k, 0)) continue;
                        const int cnt = ((i > 0) + (i < ctx->nx)) * ((j > 0) + (j < ctx->ny)) *
                                        (ctx->dim == 3 ? ((k > 0) + (k < ctx->nz)) : 1);
                        const double F = ctx->k.src * cnt;
                        f2 += F * F;
                    }
    }
    ctx->f_norm = std::sqrt(f2);

    // device buffers
    const size_t nb = ctx->node_bytes();
    const size_t eb = ctx->L.estride * ctx->tsize();
    const int64_t nc = ctx->L.ncells();
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void **p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(p, std::max<size_t>(bytes, 16));
    };
    alloc(&ctx->u[0], nb);
    alloc(&ctx->u[1], nb);
    alloc(&ctx->w, nb);
    if (ctx->tiling.kind == 7) alloc(&ctx->w_alt, nb);  // 2D sweeps several per launch
    alloc(&ctx->E, eb);
    alloc(&ctx->phi, (size_t)ctx->P * nc * ctx->ssize());
    alloc(&ctx->s, (size_t)ctx->P * nc * ctx->tsize());
    alloc(&ctx->dscr, (size_t)ctx->P * nc * ctx->tsize());
    alloc(&ctx->mu, (size_t)nc * ctx->tsize());
    alloc((void **)&ctx->scal, sizeof(double) * SC_N);
    alloc((void **)&ctx->counter, sizeof(unsigned) * 4);
    ctx->partial_cap = reduction_capacity(ctx->L, std::max(ntiles, gntiles), ctx->P);
    alloc((void **)&ctx->partials, sizeof(double) * ctx->partial_cap);
    ctx->ntiles_alloc = ntiles;
    alloc((void **)&ctx->tile_ptr, sizeof(int) * (ntiles + 1));
    alloc((void **)&ctx->loads, sizeof(LoadEntry) * std::max(1, ctx->n_loads));
    alloc((void **)&ctx->gtile_ptr, sizeof(int) * (gntiles + 1));
    alloc((void **)&ctx->gloads, sizeof(LoadEntry) * std::max(1, ctx->n_loads));
    alloc((void **)&ctx->ctrl, sizeof(double) * CT_N);
    if (e != cudaSuccess) {
        petto_status st = e == cudaErrorMemoryAllocation ? PETTO_ENOMEM : PETTO_ECUDA;
        cudaGetLastError();
        petto_destroy(ctx);
        return st;
    }
    cudaStream_t s = ctx->stream;
    e = cudaMemsetAsync(ctx->u[0], 0, nb, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->u[1], 0, nb, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->w, 0, nb, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->E, 0, eb, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->scal, 0, sizeof(double) * SC_N, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->counter, 0, sizeof(unsigned) * 4, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ctx->tile_ptr, tptr.data(), sizeof(int) * (ntiles + 1), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ctx->gtile_ptr, gptr.data(), sizeof(int) * gptr.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && ctx->n_loads > 0)
        e = cudaMemcpyAsync(ctx->loads, tent.data(), sizeof(LoadEntry) * ctx->n_loads, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && ctx->n_loads > 0)
        e = cudaMemcpyAsync(ctx->gloads, gent.data(), sizeof(LoadEntry) * ctx->n_loads, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->ctrl, 0, sizeof(double) * CT_N, s);
    if (e == cudaSuccess && ctx->w_alt) e = cudaMemsetAsync(ctx->w_alt, 0, nb, s);
    if (e == cudaSuccess && ctx->tiling.kind == 7) e = tb2d_prepare();
    // phi = V
    double *dvol = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&dvol, sizeof(double) * ctx->P);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dvol, ctx->vol.data(), sizeof(double) * ctx->P, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        fill_phase<<<grid_of(nc * ctx->P), 256, 0, s>>>(nc, ctx->P, dvol, ctx->storage, ctx->phi);
        e = cudaGetLastError();
        ctx->launches++;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (dvol) cudaFree(dvol);
    if (e != cudaSuccess) {
        petto_destroy(ctx);
        return PETTO_ECUDA;
    }
    if (ctx->dim == 3 && ctx->physics == 0 && ctx->precision == PETTO_F32 && march3d_prepare() != cudaSuccess) {
        ctx->err = "cannot configure the marching kernels";
        petto_destroy(ctx);
        return PETTO_ECUDA;
    }
    if (ctx->tiling.kind == 2 || ctx->tiling.kind == 3 || two_row_kind(ctx->tiling.kind)) {
        const int ty = ctx->tiling.kind == 2 ? 8 : 16;
        if (!make_tma_maps(ctx->L, ty, ctx->ndofc(), ctx->u[0], ctx->u[1], ctx->w, ctx->E, ctx->tma)) {
            if (ctx->tiling.kind == 2) {
                march3d_tiling(ctx->L, ctx->tiling);  // same tile shape, register-staged kernel
            } else {
                ctx->err = "tensor map creation failed";
                petto_destroy(ctx);
                return PETTO_ECUDA;
            }
        }
    }
    petto_status st = refresh_material(ctx);
    if (st != PETTO_OK) {
        petto_destroy(ctx);
        return st;
    }
    *out = ctx;
    return PETTO_OK;
}

petto_status petto_synchronize(petto_ctx *ctx) {
    if (!ctx) return PETTO_EINVAL;
    CK(cudaStreamSynchronize(ctx->stream));
    return PETTO_OK;
}

petto_status petto_set_design(petto_ctx *ctx, const void *phi, int dtype, int on_device) {
    if (!ctx || !phi) return fail(ctx, PETTO_EINVAL, "null argument");
    const int64_t n = (int64_t)ctx->P * ctx->L.ncells();
    petto_status st = flat_in(ctx, phi, dtype, on_device, ctx->phi, ctx->storage, n);
    if (st != PETTO_OK) return st;
    ctx->have_sens = false;
    return refresh_material(ctx);
}

petto_status petto_get_design(petto_ctx *ctx, void *phi, int dtype, int on_device) {
    if (!ctx || !phi) return fail(ctx, PETTO_EINVAL, "null argument");
    return flat_out(ctx, ctx->phi, ctx->storage, phi, dtype, on_device, (int64_t)ctx->P * ctx->L.ncells());
}

petto_status petto_set_state(petto_ctx *ctx, const void *u, const void *w, int dtype, int on_device) {
    if (!ctx || !u) return fail(ctx, PETTO_EINVAL, "null argument");
    petto_status st = node_in(ctx, u, dtype, on_device, ctx->u[ctx->cur]);
    if (st != PETTO_OK) return st;
    if (w) return node_in(ctx, w, dtype, on_device, ctx->w);
    CK(cudaMemsetAsync(ctx->w, 0, ctx->node_bytes(), ctx->stream));
    if (!on_device) CK(cudaStreamSynchronize(ctx->stream));
    return PETTO_OK;
}

petto_status petto_get_state(petto_ctx *ctx, void *u, void *w, int dtype, int on_device) {
    if (!ctx || !u) return fail(ctx, PETTO_EINVAL, "null argument");
    petto_status st = node_out(ctx, ctx->u[ctx->cur], u, dtype, on_device);
    if (st != PETTO_OK || !w) return st;
    return node_out(ctx, ctx->w, w, dtype, on_device);
}

petto_status petto_get_modulus(petto_ctx *ctx, void *E, int dtype, int on_device) {
    if (!ctx || !E) return fail(ctx, PETTO_EINVAL, "null argument");
    if (dtype != PETTO_F32 && dtype != PETTO_F64) return fail(ctx, PETTO_EUNSUPPORTED, "modulus is f32/f64");
    const int64_t nc = ctx->L.ncells();
    void *ddst = E;
    if (!on_device) {
        petto_status st = ensure_stage(ctx, nc * dtype_size(dtype));
        if (st != PETTO_OK) return st;
        ddst = ctx->stage;
    }
    const Layout L = ctx->L;
    cudaStream_t s = ctx->stream;
    if (ctx->precision == 0) {
        if (dtype == PETTO_F32) unpack_cells<float, float><<<grid_of(nc), 256, 0, s>>>(L, (const float *)ctx->E, (float *)ddst);
        else unpack_cells<float, double><<<grid_of(nc), 256, 0, s>>>(L, (const float *)ctx->E, (double *)ddst);
    } else {
        if (dtype == PETTO_F32) unpack_cells<double, float><<<grid_of(nc), 256, 0, s>>>(L, (const double *)ctx->E, (float *)ddst);
        else unpack_cells<double, double><<<grid_of(nc), 256, 0, s>>>(L, (const double *)ctx->E, (double *)ddst);
    }
    CK(cudaGetLastError());
    ctx->launches++;
    if (!on_device) {
        CK(cudaMemcpyAsync(E, ctx->stage, nc * dtype_size(dtype), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    return PETTO_OK;
}

petto_status petto_sweep(petto_ctx *ctx, int kind, int64_t n, double a, double b, double s1, int local_dt,
                         double *res_norm2) {
    if (!ctx || n < 0 || (kind != PETTO_SWEEP_APT && kind != PETTO_SWEEP_PT))
        return fail(ctx, PETTO_EINVAL, "bad sweep arguments");
    for (int64_t t = 0; t < n;) {
        const int g = sweep_group(ctx, t, n);
        SweepCtl sc;
        sc.idx = t;
        petto_status st = one_sweep(ctx, kind, a, b, s1, local_dt, res_norm2 && t + g == n, sc, g);
        if (st != PETTO_OK) return st;
        t += g;
    }
    if (res_norm2) {
        if (n == 0) {
            *res_norm2 = 0.0;
            return PETTO_OK;
        }
        CK(cudaMemcpyAsync(res_norm2, ctx->scal + SC_RES, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    return PETTO_OK;
}

petto_status petto_residual(petto_ctx *ctx, double *res_norm2, void *R, int dtype, int on_device) {
    if (!ctx) return PETTO_EINVAL;
    if (!ctx->rbuf) CK(cudaMalloc(&ctx->rbuf, ctx->node_bytes()));
    CK(cudaMemsetAsync(ctx->rbuf, 0, ctx->node_bytes(), ctx->stream));
    SweepArgs A = base_sweep_args(ctx);
    A.mode = 2;
    A.want_res = 1;
    A.u_in = ctx->u[ctx->cur];
    A.u_out = nullptr;
    A.w = ctx->rbuf;
    CK(launch_sweep(A, ctx->tiling, ctx->precision, ctx->stream, &ctx->tma));
    ctx->launches++;
    if (res_norm2) {
        CK(cudaMemcpyAsync(res_norm2, ctx->scal + SC_RES, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    if (R) return node_out(ctx, ctx->rbuf, R, dtype, on_device);
    return PETTO_OK;
}

}  // extern "C"

// set one device control word (stream-ordered, no host staging)
__global__ void set_ctrl_kernel(double *ctrl, int slot, long long v) { reinterpret_cast<long long *>(ctrl)[slot] = v; }

namespace {

// flat conversions / updates over whole padded node fields
__global__ void f32_to_f64(int64_t n, const float *__restrict__ a, double *__restrict__ b) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        b[t] = (double)a[t];
}
__global__ void f64_to_f32(int64_t n, const double *__restrict__ a, float *__restrict__ b) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        b[t] = (float)a[t];
}
// max |a| into *m (which starts at 0): the bit patterns of non-negative doubles order as integers
__global__ void abs_max_f64(int64_t n, const double *__restrict__ a, double *m) {
    double v = 0.0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        v = fmax(v, fabs(a[t]));
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0 && v > 0.0)
        atomicMax(reinterpret_cast<unsigned long long *>(m), (unsigned long long)__double_as_longlong(v));
}
// b = FP16(a 2^k) with 2^k the power of two taking max |a| = m into [2^14, 2^15) (all
// entries stay below the FP16 maximum); 2^-k, the factor that restores a, goes to *inv
__global__ void f64_to_f16_scaled(int64_t n, const double *__restrict__ a, const double *m, double *inv,
                                  __half *__restrict__ b) {
    int e = 0;
    frexp(*m, &e);  // m < 2^e
    const int k = 15 - e;
    if (blockIdx.x == 0 && threadIdx.x == 0) *inv = ldexp(1.0, -k);
    const double sc = ldexp(1.0, k);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        b[t] = __float2half_rn((float)(a[t] * sc));
}
__global__ void add_f32_to_f64(int64_t n, const float *__restrict__ d, double *__restrict__ u) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        u[t] += (double)d[t];
}

struct SolveState {
    int64_t sweeps = 0, na = 0, np = 0, total = 0;
    bool use_pt = false, fell = false;
    double best = INFINITY, last = NAN;
    int since_improve = 0;
    double improve_ref = INFINITY;
};

petto_status set_ctrl(petto_ctx *ctx, int slot, long long v) {
    set_ctrl_kernel<<<1, 1, 0, ctx->stream>>>(ctx->ctrl, slot, v);
    CK(cudaGetLastError());
    ctx->launches++;
    return PETTO_OK;
}

// One chunk of ce sweeps (the last a check sweep) as a CUDA graph: captured once per set of
// sweep constants and starting buffer, replayed with the chunk's first sweep index read
// from the device control words.
petto_status graph_chunk(petto_ctx *ctx, const petto_solve_opts *o, bool apt, int ce, long long base,
                         const void *rhs, bool *done, bool res_last = true) {
    *done = false;
    const int adaptive = o->momentum == 1 ? 1 : 0;
    petto_ctx::GraphEntry *ge = nullptr;
    for (auto &g : ctx->graphs)
        if (g.apt == apt && g.local_dt == o->local_dt && g.adaptive == adaptive && g.cur == ctx->cur && g.ce == ce &&
            g.res_last == (res_last ? 1 : 0) && g.rhs == rhs && g.a == o->a && g.b == o->b && g.s1 == o->s1 &&
            g.w == ctx->w)
            ge = &g;
    if (!ge) {
        if (ctx->graphs.size() >= 8) clear_graphs(ctx);
        cudaGraph_t graph = nullptr;
        CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
        const int cur0 = ctx->cur;
        void *const w0 = ctx->w;
        const int64_t l0 = ctx->launches;
        petto_status st = PETTO_OK;
        int flips = 0, swaps = 0;
        for (int j = 0; j < ce && st == PETTO_OK;) {
            const int g = sweep_group(ctx, j, ce);
            SweepCtl sc;
            sc.adaptive = adaptive;
            sc.test_dot = ((j + g - 1) % 4) == 3;
            sc.idx = j;
            sc.base_from_ctrl = 1;
            sc.rhs = rhs;
            st = one_sweep(ctx, apt ? 0 : 1, o->a, o->b, o->s1, o->local_dt, res_last && j + g == ce, sc, g);
            ++flips;
            if (g > 1 && apt) ++swaps;
            j += g;
        }
        cudaError_t ec = cudaStreamEndCapture(ctx->stream, &graph);
        ctx->cur = cur0;
        if (ctx->w != w0) std::swap(ctx->w, ctx->w_alt);
        ctx->launches = l0;
        if (st != PETTO_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        CK(ec);
        cudaGraphExec_t exec = nullptr;
        cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        CK(ei);
        petto_ctx::GraphEntry g{apt ? 1 : 0, o->local_dt, adaptive, ctx->cur, ce, res_last ? 1 : 0, rhs, o->a, o->b,
                                o->s1, exec, w0, flips, swaps, flips};
        ctx->graphs.push_back(g);
        ge = &ctx->graphs.back();
    }
    set_ctrl_kernel<<<1, 1, 0, ctx->stream>>>(ctx->ctrl, CT_BASE, base);
    CK(cudaGetLastError());
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (ctx->profiling) {
        for (cudaEvent_t *e : {&e0, &e1}) {
            if (!ctx->ev_free.empty()) {
                *e = ctx->ev_free.back();
                ctx->ev_free.pop_back();
            } else {
                CK(cudaEventCreate(e));
            }
        }
        CK(cudaEventRecord(e0, ctx->stream));
    }
    CK(cudaGraphLaunch(ge->exec, ctx->stream));
    if (ctx->profiling) {
        CK(cudaEventRecord(e1, ctx->stream));
        ctx->ev_pending.emplace_back(e0, e1);
        ctx->ev_count.push_back(ce);
        ctx->ev_rhs.push_back(rhs != nullptr);
    }
    ctx->launches += ge->launches + 1;
    // the buffer roles after the chunk's launches
    if (ge->flips & 1) ctx->cur ^= 1;
    if (ge->swaps & 1) std::swap(ctx->w, ctx->w_alt);
    *done = true;
    return PETTO_OK;
}

// One check residual rn applied to the phase state: the divergence guard (a non-finite
// residual zeroes u and w and falls back to PT; one above guard x the best so far zeroes w
// and falls back to PT), the stop test and the stall test.  *ended is set when the phase
// ends; *reached when rn <= stop_abs.  check = false (the budget's last, unchecked sweep)
// ends the phase.
petto_status apply_check(petto_ctx *ctx, const petto_solve_opts *o, SolveState &S, double rn, bool check,
                         double stop_abs, int stall_checks, bool *ended, int *reached) {
    const double guard = o->momentum == 1 ? 100.0 : 10.0;
    *ended = false;
    if (!check) {
        *ended = true;
        return PETTO_OK;
    }
    if (!std::isfinite(rn)) {
        CK(cudaMemsetAsync(ctx->u[ctx->cur], 0, ctx->node_bytes(), ctx->stream));
        CK(cudaMemsetAsync(ctx->w, 0, ctx->node_bytes(), ctx->stream));
        S.use_pt = true;
        S.fell = true;
        return PETTO_OK;
    }
    if (rn > guard * S.best && !S.use_pt) {
        CK(cudaMemsetAsync(ctx->w, 0, ctx->node_bytes(), ctx->stream));
        S.use_pt = true;
        S.fell = true;
    }
    if (rn < S.best) S.best = rn;
    if (rn <= stop_abs) {
        *reached = 1;
        *ended = true;
        return PETTO_OK;
    }
    if (rn < 0.9 * S.improve_ref) {
        S.improve_ref = rn;
        S.since_improve = 0;
    } else if (stall_checks > 0 && ++S.since_improve >= stall_checks) {
        *ended = true;
    }
    return PETTO_OK;
}

// ---- iterative refinement around FP32 sweeps (steps shared by the single and batched solves)
// FP32 sweeps on the state itself run down to REFINE_FROM x ||F|| (well above the FP32 floor
// of these problems, 3.5e-5 .. 9.5e-4) or until the check residual stalls; the refinement,
// whose sweeps also read a dense right-hand side, takes over from there.  (Measured on the
// 3D cantilever: switching at 3e-2 or 1e-2 takes the same sweeps; at 2e-3 the plain sweeps
// slow down near the floor and a design step takes 30 % more sweeps.)
constexpr double REFINE_FROM = 1e-2;
constexpr int REFINE_STALL = 20;

// the FP64 state, defect and right-hand side buffers of the refinement
petto_status refine_alloc(petto_ctx *ctx) {
    const size_t nb64 = (size_t)ctx->ndofc() * ctx->L.cstride * sizeof(double);
    if (!ctx->u64) {
        CK(cudaMalloc(&ctx->u64, nb64));
        // the node-gather defect reads the padding around the grid: zero, as in every state
        CK(cudaMemsetAsync(ctx->u64, 0, nb64, ctx->stream));
    }
    if (!ctx->r64) {
        CK(cudaMalloc(&ctx->r64, nb64));
        // the defect kernel writes grid nodes only: the padding stays zero (it enters max |r|)
        CK(cudaMemsetAsync(ctx->r64, 0, nb64, ctx->stream));
    }
    if (!ctx->rhs32) CK(cudaMalloc(&ctx->rhs32, ctx->node_bytes()));
    return PETTO_OK;
}

// u64 <- u (FP32 state), allocating the FP64 state, defect and right-hand side buffer
petto_status refine_begin(petto_ctx *ctx) {
    const int64_t nel = (int64_t)ctx->ndofc() * ctx->L.cstride;
    petto_status st = refine_alloc(ctx);
    if (st != PETTO_OK) return st;
    f32_to_f64<<<grid_of(nel), 256, 0, ctx->stream>>>(nel, (const float *)ctx->u[ctx->cur], (double *)ctx->u64);
    CK(cudaGetLastError());
    ctx->launches++;
    return PETTO_OK;
}

// FP64 defect r64 = F - K u64 and its norm (synchronises)
petto_status refine_defect(petto_ctx *ctx, double *norm) {
    SweepArgs R = base_sweep_args(ctx);
    R.mode = 2;
    R.want_res = 1;
    R.u_in = ctx->u64;
    R.w = ctx->r64;
    R.tile_ptr = ctx->gtile_ptr;
    R.loads = ctx->gloads;
    CK(launch_residual64(R, ctx->gtiling, ctx->stream));
    ctx->launches++;
    double scal[SC_N];
    petto_status st = read_scal(ctx, scal);
    if (st != PETTO_OK) return st;
    *norm = std::sqrt(scal[SC_RES]);
    return PETTO_OK;
}

// the defect becomes the right-hand side of the correction sweeps, which restart from d = 0.
// The two-row 3D marching kernel reads it as FP16 scaled by a power of two (one TMA box per
// stage, 6 bytes a node instead of 12); FP16 keeps 11 bits, so the correction solved to the
// FP32 floor (about 1e-4 of its right-hand side) loses nothing the next defect does not see.
// r64 -> the right-hand side the sweep kernel reads (FP16 scaled or FP32, in rhs32)
petto_status refine_rhs(petto_ctx *ctx) {
    const int64_t nel = (int64_t)ctx->ndofc() * ctx->L.cstride;
    ctx->rhs_half = two_row_kind(ctx->tiling.kind);
    if (ctx->rhs_half) {
        CK(cudaMemsetAsync(ctx->ctrl + CT_RMAX, 0, sizeof(double), ctx->stream));
        abs_max_f64<<<grid_of(nel), 256, 0, ctx->stream>>>(nel, (const double *)ctx->r64, ctx->ctrl + CT_RMAX);
        f64_to_f16_scaled<<<grid_of(nel), 256, 0, ctx->stream>>>(nel, (const double *)ctx->r64, ctx->ctrl + CT_RMAX,
                                                                  ctx->ctrl + CT_RSCALE, (__half *)ctx->rhs32);
        ctx->launches += 2;
        if (!ctx->tma.rvalid || ctx->tma.rbuf != ctx->rhs32) {
            if (!make_tma_rhs_map(ctx->L, ctx->ndofc(), ctx->rhs32, ctx->tma))
                return fail(ctx, PETTO_ECUDA, "tensor map creation failed");
            clear_graphs(ctx);
        }
    } else {
        f64_to_f32<<<grid_of(nel), 256, 0, ctx->stream>>>(nel, (const double *)ctx->r64, (float *)ctx->rhs32);
    }
    CK(cudaGetLastError());
    ctx->launches++;
    return PETTO_OK;
}

petto_status refine_correction(petto_ctx *ctx) {
    petto_status st = refine_rhs(ctx);
    if (st != PETTO_OK) return st;
    CK(cudaMemsetAsync(ctx->u[ctx->cur], 0, ctx->node_bytes(), ctx->stream));
    return PETTO_OK;
}

// u64 += d
petto_status refine_absorb(petto_ctx *ctx) {
    const int64_t nel = (int64_t)ctx->ndofc() * ctx->L.cstride;
    add_f32_to_f64<<<grid_of(nel), 256, 0, ctx->stream>>>(nel, (const float *)ctx->u[ctx->cur], (double *)ctx->u64);
    CK(cudaGetLastError());
    ctx->launches++;
    return PETTO_OK;
}

// u <- u64 rounded to FP32, w <- 0
petto_status refine_finish(petto_ctx *ctx) {
    const int64_t nel = (int64_t)ctx->ndofc() * ctx->L.cstride;
    f64_to_f32<<<grid_of(nel), 256, 0, ctx->stream>>>(nel, (const double *)ctx->u64, (float *)ctx->u[ctx->cur]);
    CK(cudaGetLastError());
    CK(cudaMemsetAsync(ctx->w, 0, ctx->node_bytes(), ctx->stream));
    ctx->launches++;
    return PETTO_OK;
}

// Sweep until a check sweep's residual is <= stop_abs, the budget ends, or (stall_checks > 0)
// the residual has not fallen 10% over stall_checks checks.  Returns 1 when stop_abs was
// reached, 0 otherwise.  Applies the divergence guard.
petto_status sweep_phase(petto_ctx *ctx, const petto_solve_opts *o, SolveState &S, double stop_abs, int64_t n_apt,
                         int stall_checks, const void *rhs, int *reached) {
    *reached = 0;
    const int ce = o->check_every;
    double scal[SC_N];
    while (S.sweeps < S.total) {
        const bool apt = !S.use_pt && (o->mode == PETTO_SOLVE_TOL || S.sweeps < n_apt);
        // a whole check interval of one sweep kind: replay it as a graph
        const bool same_kind = o->mode == PETTO_SOLVE_TOL || S.use_pt || S.sweeps + ce <= n_apt || S.sweeps >= n_apt;
        if (ctx->use_graphs && ctx->stream && ce >= 4 && ce % 2 == 0 && S.sweeps % ce == 0 &&
            S.sweeps + ce <= S.total && same_kind) {
            bool done = false;
            petto_status st = graph_chunk(ctx, o, apt, ce, S.sweeps, rhs, &done);
            if (st != PETTO_OK) return st;
            if (done) {
                if (apt) S.na += ce; else S.np += ce;
                S.sweeps += ce;
                goto checked;
            }
        }
        if (ctx->use_graphs && ctx->stream && ce == 0 && S.sweeps % 4 == 0) {
            // no checks (the paper's fixed counts): replay runs of up to 64 sweeps of one kind,
            // keeping the budget's last sweep (which reports the residual) for the loop below
            int64_t len = S.total - S.sweeps - 1;
            if (o->mode == PETTO_SOLVE_PAPER && !S.use_pt && S.sweeps < n_apt) len = std::min(len, n_apt - S.sweeps);
            len = std::min<int64_t>(len, 64) & ~int64_t(3);
            if (len >= 4) {
                bool done = false;
                petto_status st = graph_chunk(ctx, o, apt, (int)len, S.sweeps, rhs, &done, false);
                if (st != PETTO_OK) return st;
                if (done) {
                    if (apt) S.na += len; else S.np += len;
                    S.sweeps += len;
                    continue;
                }
            }
        }
        {
            const bool check = ce > 0 && (S.sweeps + 1) % ce == 0;
            const bool final_report = (S.sweeps + 1 == S.total);
            SweepCtl sc;
            sc.adaptive = o->momentum == 1 ? 1 : 0;
            sc.test_dot = ((ce > 0 ? S.sweeps % ce : S.sweeps) % 4) == 3;
            sc.idx = S.sweeps;
            sc.rhs = rhs;
            petto_status st = one_sweep(ctx, apt ? 0 : 1, o->a, o->b, o->s1, o->local_dt, check || final_report, sc);
            if (st != PETTO_OK) return st;
            if (apt) ++S.na; else ++S.np;
            ++S.sweeps;
            if (!(check || final_report)) continue;
        }
    checked:
        const bool check = ce > 0 && S.sweeps % ce == 0;
        petto_status st = read_scal(ctx, scal);
        if (st != PETTO_OK) return st;
        const double rn = std::sqrt(scal[SC_RES]);
        S.last = rn;
        if (ctx->trace) {
            double ctrl[CT_N];
            cudaMemcpy(ctrl, ctx->ctrl, sizeof(ctrl), cudaMemcpyDeviceToHost);
            long long ra = 0;
            std::memcpy(&ra, &ctrl[CT_RESTART_AT], sizeof(ra));
            std::fprintf(stderr, "petto: sweep %lld res %.6e rel %.3e restart@%lld%s\n", (long long)S.sweeps, rn,
                         ctx->f_norm > 0 ? rn / ctx->f_norm : 0.0, ra,
                         rhs ? " (correction)" : "");
        }
        bool ended = false;
        st = apply_check(ctx, o, S, rn, check, stop_abs, stall_checks, &ended, reached);
        if (st != PETTO_OK) return st;
        if (ended) break;
    }
    return PETTO_OK;
}

// The first solve of a large 3D grid times the applicable sweep kernels (petto_autotune) and
// keeps the fastest; the choice is remembered per grid shape for the rest of the process.
std::mutex g_tune_mutex;
std::map<std::string, std::string> g_tuned;

petto_status tune_first_solve(petto_ctx *ctx) {
    if (!ctx->tune_pending) return PETTO_OK;
    ctx->tune_pending = false;
    const std::string key = std::to_string(ctx->dim) + ":" + std::to_string(ctx->nx) + "x" + std::to_string(ctx->ny) +
                            "x" + std::to_string(ctx->nz) + ":r" + std::to_string(ctx->nrhs) + ":p" +
                            std::to_string(ctx->physics) + std::to_string(ctx->precision);
    std::string name;
    {
        std::lock_guard<std::mutex> lk(g_tune_mutex);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) name = it->second;
    }
    if (!name.empty()) return petto_select_kernel(ctx, name.c_str());
    petto_status st = petto_autotune(ctx, 10, nullptr, 0);
    if (st != PETTO_OK) return st;
    char nm[64];
    st = petto_kernel_info(ctx, nm, sizeof nm, nullptr);
    if (st != PETTO_OK) return st;
    std::lock_guard<std::mutex> lk(g_tune_mutex);
    g_tuned[key] = nm;
    return PETTO_OK;
}

}  // namespace

extern "C" {

petto_status petto_residual64(petto_ctx *ctx, const double *u, int on_device, double *res_norm2, double *R) {
    if (!ctx || !u) return fail(ctx, PETTO_EINVAL, "null argument");
    if (ctx->precision != PETTO_F32) return fail(ctx, PETTO_EUNSUPPORTED, "the FP64 defect belongs to FP32 contexts");
    petto_status st = refine_alloc(ctx);
    if (st != PETTO_OK) return st;
    const int C = ctx->ndofc();
    const int64_t nn = (int64_t)C * ctx->L.nnodes();
    const double *src = u;
    if (!on_device) {
        st = ensure_stage(ctx, nn * sizeof(double));
        if (st != PETTO_OK) return st;
        CK(cudaMemcpyAsync(ctx->stage, u, nn * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
        src = static_cast<const double *>(ctx->stage);
    }
    pack_nodes<double, double><<<grid_of(nn), 256, 0, ctx->stream>>>(ctx->L, C, src, (double *)ctx->u64, 1);
    CK(cudaGetLastError());
    ctx->launches++;
    double norm = 0.0;
    st = refine_defect(ctx, &norm);
    if (st != PETTO_OK) return st;
    if (res_norm2) *res_norm2 = norm * norm;
    if (!R) return PETTO_OK;
    double *dst = R;
    if (!on_device) {
        st = ensure_stage(ctx, nn * sizeof(double));
        if (st != PETTO_OK) return st;
        dst = static_cast<double *>(ctx->stage);
    }
    pack_nodes<double, double><<<grid_of(nn), 256, 0, ctx->stream>>>(ctx->L, C, (const double *)ctx->r64, dst, 0);
    CK(cudaGetLastError());
    ctx->launches++;
    if (!on_device) CK(cudaMemcpyAsync(R, ctx->stage, nn * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return PETTO_OK;
}

petto_status petto_pt_solve(petto_ctx *ctx, const petto_solve_opts *o, petto_solve_report *rep) {
    if (!ctx || !o) return fail(ctx, PETTO_EINVAL, "null argument");
    if (o->mode != PETTO_SOLVE_PAPER && o->mode != PETTO_SOLVE_TOL) return fail(ctx, PETTO_EINVAL, "bad mode");
    if (o->n_apt < 0 || o->n_pt < 0 || o->max_sweeps < 0 || o->check_every < 0)
        return fail(ctx, PETTO_EINVAL, "negative count");
    if (o->momentum < 0 || o->momentum > 2) return fail(ctx, PETTO_EINVAL, "momentum is 0, 1 or 2");
    CK(cudaMemsetAsync(ctx->w, 0, ctx->node_bytes(), ctx->stream));
    petto_status st = tune_first_solve(ctx);
    if (st == PETTO_OK) st = set_ctrl(ctx, CT_RESTART_AT, 0);
    if (st == PETTO_OK) st = set_ctrl(ctx, CT_ERR, 0);  // a new solve: no wait has run out yet
    if (st != PETTO_OK) return st;
    SolveState S;
    S.use_pt = o->momentum == 2;  // the plain first-order method throughout
    S.total = o->mode == PETTO_SOLVE_PAPER ? o->n_apt + o->n_pt : o->max_sweeps;
    const double fn = ctx->f_norm;
    const bool refine = o->mode == PETTO_SOLVE_TOL && o->refine && ctx->precision == PETTO_F32 && o->tol < 1e-3;
    bool conv = false;
    int reached = 0;
    double true_res = NAN;
    if (!refine) {
        const double stop = o->mode == PETTO_SOLVE_TOL ? o->tol * fn : -1.0;
        st = sweep_phase(ctx, o, S, stop, o->n_apt, 0, nullptr, &reached);
        if (st != PETTO_OK) return st;
        conv = reached != 0;
    } else {
        // FP32 sweeps on the state itself down to REFINE_FROM, then the same iteration
        // continued on u = u64 + d: u64 (FP64) absorbs d whenever the check residual has fallen 8x, the
        // FP64 defect F - K u64 becomes the right-hand side of the sweeps, d restarts
        // from zero and the increment w and the momentum schedule carry on unchanged (the
        // APT recursion is the same in the shifted variable).
        st = sweep_phase(ctx, o, S, REFINE_FROM * fn, 0, REFINE_STALL, nullptr, &reached);
        if (st != PETTO_OK) return st;
        st = refine_begin(ctx);
        if (st != PETTO_OK) return st;
        while (true) {
            st = refine_defect(ctx, &true_res);
            if (st != PETTO_OK) return st;
            if (ctx->trace)
                std::fprintf(stderr, "petto: FP64 defect %.6e rel %.3e after %lld sweeps\n", true_res,
                             fn > 0 ? true_res / fn : 0.0, (long long)S.sweeps);
            if (true_res <= o->tol * fn) {
                conv = true;
                break;
            }
            if (S.sweeps >= S.total || !std::isfinite(true_res)) break;
            st = refine_correction(ctx);
            if (st != PETTO_OK) return st;
            S.improve_ref = INFINITY;
            S.since_improve = 0;
            const double stop = std::max(true_res / 8.0, 0.5 * o->tol * fn);
            st = sweep_phase(ctx, o, S, stop, 0, 20, ctx->rhs32, &reached);
            if (st != PETTO_OK) return st;
            st = refine_absorb(ctx);
            if (st != PETTO_OK) return st;
        }
        st = refine_finish(ctx);
        if (st != PETTO_OK) return st;
        S.last = true_res;
    }
    if (rep) {
        rep->sweeps = S.sweeps;
        rep->apt_sweeps = S.na;
        rep->pt_sweeps = S.np;
        rep->res_norm = S.last;
        rep->f_norm = fn;
        rep->rel_res = fn > 0 ? S.last / fn : NAN;
        rep->r_pde = S.last / std::pow(ctx->h, ctx->dim) / (double)ctx->L.nnodes();
        rep->converged = conv ? 1 : 0;
        rep->fell_back_to_pt = S.fell ? 1 : 0;
    }
    if (!std::isfinite(S.last)) return fail(ctx, PETTO_EDIVERGED, "residual not finite after PT fallback");
    if (o->mode == PETTO_SOLVE_TOL && !conv) return PETTO_ENOTCONV;
    return PETTO_OK;
}

int64_t petto_layer_bytes(const petto_ctx *ctx, int field) {
    if (!ctx || ctx->dim != 3 || (field != PETTO_LAYER_PHI && field != PETTO_LAYER_MU)) return 0;
    return (int64_t)ctx->L.nx * ctx->L.ny * (field == PETTO_LAYER_PHI ? ctx->ssize() : ctx->tsize());
}

}  // extern "C"

namespace {

// the address of cell layer k of a field (k = nz: the copy of the layer above the grid)
petto_status layer_ptr(petto_ctx *ctx, int field, int phase, int64_t k, char **out) {
    if (ctx->dim != 3) return fail(ctx, PETTO_EUNSUPPORTED, "cell layers are z layers of a 3D grid");
    if (field != PETTO_LAYER_PHI && field != PETTO_LAYER_MU) return fail(ctx, PETTO_EINVAL, "field is phi or mu");
    if (field == PETTO_LAYER_PHI && (phase < 0 || phase >= ctx->P)) return fail(ctx, PETTO_EINVAL, "no such phase");
    if (k < 0 || k > ctx->L.nz) return fail(ctx, PETTO_EINVAL, "cell layer outside the grid");
    const int64_t pl = (int64_t)ctx->L.nx * ctx->L.ny, nc = ctx->L.ncells();
    const size_t es = field == PETTO_LAYER_PHI ? ctx->ssize() : ctx->tsize();
    if (k == ctx->L.nz) {
        void *&hi = field == PETTO_LAYER_PHI ? ctx->phi_hi : ctx->mu_hi;
        if (!hi) {
            const size_t bytes = (size_t)(field == PETTO_LAYER_PHI ? ctx->P : 1) * pl * es;
            CK(cudaMalloc(&hi, bytes));
            CK(cudaMemsetAsync(hi, 0, bytes, ctx->stream));
        }
        *out = static_cast<char *>(hi) + (field == PETTO_LAYER_PHI ? (int64_t)phase * pl * es : 0);
        return PETTO_OK;
    }
    char *base = static_cast<char *>(field == PETTO_LAYER_PHI ? ctx->phi : ctx->mu);
    *out = base + ((field == PETTO_LAYER_PHI ? (int64_t)phase * nc : 0) + k * pl) * (int64_t)es;
    return PETTO_OK;
}

petto_status copy_layer(petto_ctx *ctx, int field, int phase, int64_t k, void *dst, const void *src, int on_device) {
    if (!ctx || (!dst && !src)) return fail(ctx, PETTO_EINVAL, "null argument");
    char *lp = nullptr;
    petto_status st = layer_ptr(ctx, field, phase, k, &lp);
    if (st != PETTO_OK) return st;
    const size_t bytes = (size_t)petto_layer_bytes(ctx, field);
    if (dst) CK(cudaMemcpyAsync(dst, lp, bytes, cudaMemcpyDefault, ctx->stream));
    else CK(cudaMemcpyAsync(lp, src, bytes, cudaMemcpyDefault, ctx->stream));
    if (!on_device) CK(cudaStreamSynchronize(ctx->stream));  // host memory is the caller's again on return
    return PETTO_OK;
}

}  // namespace

extern "C" {

}  // extern "C"

namespace {

struct SlabHooks {
    petto_exchange_fn exchange;
    petto_allreduce_fn allreduce, allreduce_max;
    void *user;
};

// The sweeps of one phase of a slab's solve, as sweep_phase runs them on a whole grid: an
// exchange of the ghost planes before every sweep, the whole grid's <R, w> deciding each
// restart test and the whole grid's residual each check.
petto_status slab_phase(petto_ctx *ctx, const petto_solve_opts *o, SolveState &S, double stop_abs, int64_t n_apt,
                        int stall_checks, const void *rhs, const SlabHooks &H, int *reached) {
    *reached = 0;
    const int ce = o->check_every;
    while (S.sweeps < S.total) {
        const bool apt = !S.use_pt && (o->mode == PETTO_SOLVE_TOL || S.sweeps < n_apt);
        petto_status st = H.exchange(ctx, H.user);
        if (st != PETTO_OK) return st;
        const bool check = ce > 0 && (S.sweeps + 1) % ce == 0;
        const bool final_report = S.sweeps + 1 == S.total;
        SweepCtl sc;
        sc.adaptive = o->momentum == 1 ? 1 : 0;
        // the restart test of the adaptive momentum, on the whole grid's <R, w>
        sc.test_dot = apt && sc.adaptive && ((ce > 0 ? S.sweeps % ce : S.sweeps) % 4) == 3;
        sc.idx = S.sweeps;
        sc.rhs = rhs;
        st = one_sweep(ctx, apt ? 0 : 1, o->a, o->b, o->s1, o->local_dt, check || final_report, sc);
        if (st != PETTO_OK) return st;
        if (apt) ++S.na; else ++S.np;
        ++S.sweeps;
        if (sc.test_dot) {
            // the kernel decided on this slab's own sum; the decision is the whole grid's
            double ctrl[CT_N];
            CK(cudaMemcpyAsync(ctrl, ctx->ctrl, sizeof(ctrl), cudaMemcpyDeviceToHost, ctx->stream));
            CK(cudaStreamSynchronize(ctx->stream));
            double dot = ctrl[CT_DOT];
            st = H.allreduce(&dot, 1, H.user);
            if (st != PETTO_OK) return st;
            long long at = 0;
            std::memcpy(&at, &ctrl[CT_RESTART_AT], sizeof(at));
            if (dot < 0.0) at = S.sweeps;
            else if (at == S.sweeps) {
                // this slab's own sum was negative but the grid's is not: undo its restart
                at = ctx->slab_restart_at;
            }
            ctx->slab_restart_at = at;
            st = set_ctrl(ctx, CT_RESTART_AT, at);
            if (st != PETTO_OK) return st;
        }
        if (!(check || final_report)) continue;
        double scal[SC_N];
        st = read_scal(ctx, scal);
        if (st != PETTO_OK) return st;
        double r2 = scal[SC_RES];
        st = H.allreduce(&r2, 1, H.user);
        if (st != PETTO_OK) return st;
        const double rn = std::sqrt(r2);
        S.last = rn;
        if (ctx->trace)
            std::fprintf(stderr, "petto: slab %d sweep %lld res %.6e%s\n", ctx->own_lo, (long long)S.sweeps, rn,
                         rhs ? " (correction)" : "");
        bool ended = false;
        st = apply_check(ctx, o, S, rn, check, stop_abs, stall_checks, &ended, reached);
        if (st != PETTO_OK) return st;
        if (ended) break;
    }
    return PETTO_OK;
}

// The FP64 defect of a slab's own planes and the whole grid's norm of it (the ghost planes
// of u64 hold the neighbours' values)
petto_status slab_defect(petto_ctx *ctx, const SlabHooks &H, double *norm) {
    double local = 0.0;
    petto_status st = refine_defect(ctx, &local);
    if (st != PETTO_OK) return st;
    double r2 = local * local;
    st = H.allreduce(&r2, 1, H.user);
    if (st != PETTO_OK) return st;
    *norm = std::sqrt(r2);
    return PETTO_OK;
}

// The defect as the correction sweeps' right-hand side, d <- 0.  The FP16 form takes its
// power-of-two scale from the whole grid's max |r| (the ghost planes of r64 stay zero), so
// every slab rounds as the whole grid does.
petto_status slab_correction(petto_ctx *ctx, const SlabHooks &H) {
    const int64_t nel = (int64_t)ctx->ndofc() * ctx->L.cstride;
    ctx->rhs_half = two_row_kind(ctx->tiling.kind);
    if (ctx->rhs_half) {
        CK(cudaMemsetAsync(ctx->ctrl + CT_RMAX, 0, sizeof(double), ctx->stream));
        abs_max_f64<<<grid_of(nel), 256, 0, ctx->stream>>>(nel, (const double *)ctx->r64, ctx->ctrl + CT_RMAX);
        CK(cudaGetLastError());
        double m = 0.0;
        CK(cudaMemcpyAsync(&m, ctx->ctrl + CT_RMAX, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        petto_status st = H.allreduce_max(&m, 1, H.user);
        if (st != PETTO_OK) return st;
        CK(cudaMemcpyAsync(ctx->ctrl + CT_RMAX, &m, sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
        f64_to_f16_scaled<<<grid_of(nel), 256, 0, ctx->stream>>>(nel, (const double *)ctx->r64, ctx->ctrl + CT_RMAX,
                                                                  ctx->ctrl + CT_RSCALE, (__half *)ctx->rhs32);
        CK(cudaGetLastError());
        // the copy above reads m from this frame: done before it returns
        CK(cudaStreamSynchronize(ctx->stream));
        ctx->launches += 2;
        if (!ctx->tma.rvalid || ctx->tma.rbuf != ctx->rhs32) {
            if (!make_tma_rhs_map(ctx->L, ctx->ndofc(), ctx->rhs32, ctx->tma))
                return fail(ctx, PETTO_ECUDA, "tensor map creation failed");
            clear_graphs(ctx);
        }
    } else {
        f64_to_f32<<<grid_of(nel), 256, 0, ctx->stream>>>(nel, (const double *)ctx->r64, (float *)ctx->rhs32);
        CK(cudaGetLastError());
        ctx->launches++;
    }
    CK(cudaMemsetAsync(ctx->u[ctx->cur], 0, ctx->node_bytes(), ctx->stream));
    return PETTO_OK;
}

}  // namespace

extern "C" {

petto_status petto_slab_solve(petto_ctx *ctx, const petto_solve_opts *o, petto_exchange_fn exchange,
                              petto_allreduce_fn allreduce, petto_allreduce_fn allreduce_max, void *user,
                              petto_solve_report *rep) {
    if (!ctx || !o || !exchange || !allreduce) return fail(ctx, PETTO_EINVAL, "null argument");
    if (o->mode != PETTO_SOLVE_PAPER && o->mode != PETTO_SOLVE_TOL) return fail(ctx, PETTO_EINVAL, "bad mode");
    if (o->n_apt < 0 || o->n_pt < 0 || o->max_sweeps < 0 || o->check_every < 0)
        return fail(ctx, PETTO_EINVAL, "negative count");
    if (o->momentum < 0 || o->momentum > 2) return fail(ctx, PETTO_EINVAL, "momentum is 0, 1 or 2");
    const bool refine = o->mode == PETTO_SOLVE_TOL && o->refine && ctx->precision == PETTO_F32 && o->tol < 1e-3;
    if (refine && !allreduce_max) return fail(ctx, PETTO_EINVAL, "the refinement of a slab solve needs allreduce_max");
    const SlabHooks H{exchange, allreduce, allreduce_max, user};
    petto_status st = tune_first_solve(ctx);
    // ||F|| of the whole grid: each slab holds the loads of its own planes
    double fn2 = ctx->f_norm * ctx->f_norm;
    if (st == PETTO_OK) st = allreduce(&fn2, 1, user);
    if (st != PETTO_OK) return st;
    const double fn = std::sqrt(fn2);
    CK(cudaMemsetAsync(ctx->w, 0, ctx->node_bytes(), ctx->stream));
    st = set_ctrl(ctx, CT_RESTART_AT, 0);
    if (st == PETTO_OK) st = set_ctrl(ctx, CT_ERR, 0);
    if (st != PETTO_OK) return st;
    ctx->slab_restart_at = 0;
    SolveState S;
    S.use_pt = o->momentum == 2;
    S.total = o->mode == PETTO_SOLVE_PAPER ? o->n_apt + o->n_pt : o->max_sweeps;
    int reached = 0;
    bool conv = false;
    if (!refine) {
        const double stop = o->mode == PETTO_SOLVE_TOL ? o->tol * fn : -1.0;
        st = slab_phase(ctx, o, S, stop, o->n_apt, 0, nullptr, H, &reached);
        if (st != PETTO_OK) return st;
        conv = reached != 0;
    } else {
        // the refinement of petto_pt_solve, slab by slab: FP32 sweeps of the state down to
        // REFINE_FROM, then rounds of (FP64 defect, correction sweeps of d, u64 += d).  Before
        // u64 takes u or d, one more exchange brings their ghost planes up to date, so a
        // slab's u64 holds its neighbours' values on its ghost planes throughout.
        st = slab_phase(ctx, o, S, REFINE_FROM * fn, 0, REFINE_STALL, nullptr, H, &reached);
        if (st == PETTO_OK) st = exchange(ctx, user);
        if (st == PETTO_OK) st = refine_begin(ctx);
        if (st != PETTO_OK) return st;
        double true_res = NAN;
        while (true) {
            st = slab_defect(ctx, H, &true_res);
            if (st != PETTO_OK) return st;
            if (ctx->trace)
                std::fprintf(stderr, "petto: slab %d FP64 defect %.6e after %lld sweeps\n", ctx->own_lo, true_res,
                             (long long)S.sweeps);
            if (true_res <= o->tol * fn) {
                conv = true;
                break;
            }
            if (S.sweeps >= S.total || !std::isfinite(true_res)) break;
            st = slab_correction(ctx, H);
            if (st != PETTO_OK) return st;
            S.improve_ref = INFINITY;
            S.since_improve = 0;
            const double stop = std::max(true_res / 8.0, 0.5 * o->tol * fn);
            st = slab_phase(ctx, o, S, stop, 0, 20, ctx->rhs32, H, &reached);
            if (st == PETTO_OK) st = exchange(ctx, user);
            if (st == PETTO_OK) st = refine_absorb(ctx);
            if (st != PETTO_OK) return st;
        }
        st = refine_finish(ctx);
        if (st != PETTO_OK) return st;
        S.last = true_res;
    }
    if (rep) {
        rep->sweeps = S.sweeps;
        rep->apt_sweeps = S.na;
        rep->pt_sweeps = S.np;
        rep->res_norm = S.last;
        rep->f_norm = fn;
        rep->rel_res = fn > 0 ? S.last / fn : NAN;
        rep->r_pde = NAN;
        rep->converged = conv ? 1 : 0;
        rep->fell_back_to_pt = S.fell ? 1 : 0;
    }
    if (!std::isfinite(S.last) && S.sweeps > 0) return fail(ctx, PETTO_EDIVERGED, "residual not finite after PT fallback");
    if (o->mode == PETTO_SOLVE_TOL && !conv) return PETTO_ENOTCONV;
    return PETTO_OK;
}

petto_status petto_slab_design_step(petto_ctx *ctx, const petto_solve_opts *so, const petto_pf_opts *po,
                                    petto_exchange_fn exchange, petto_layer_exchange_fn exchange_layer,
                                    petto_allreduce_fn allreduce, petto_allreduce_fn allreduce_max, void *user,
                                    double *metrics) {
    if (!ctx || !so || !po || !exchange || !exchange_layer || !allreduce || !allreduce_max)
        return fail(ctx, PETTO_EINVAL, "null argument");
    if (ctx->dim != 3) return fail(ctx, PETTO_EUNSUPPORTED, "slabs are z ranges of a 3D grid");
    if (ctx->physics != PETTO_ELASTIC || ctx->keep || ctx->nrhs != 1)
        return fail(ctx, PETTO_EUNSUPPORTED, "the slab design step covers one-load-case elasticity without keep-out");
    if (po->vol_mode != PETTO_VOL_PROJECTED && po->vol_mode != PETTO_VOL_PENALTY)
        return fail(ctx, PETTO_EINVAL, "bad vol_mode");
    if (po->n_bisect < 0 || po->n_bisect > 200 || po->ch_steps < 0) return fail(ctx, PETTO_EINVAL, "bad counts");
    if (ctx->own_n == 1) return fail(ctx, PETTO_EINVAL, "a slab of the design step owns two node planes or more");
    const auto t0 = std::chrono::steady_clock::now();
    const int P = ctx->P;
    const Layout &L = ctx->L;
    const int64_t pl = (int64_t)L.nx * L.ny;
    // the cell layers this slab counts: those whose lower node plane it owns
    const int zc0 = ctx->own_n ? ctx->own_lo : 0;
    const int zc1 = ctx->own_n ? std::min(ctx->own_lo + ctx->own_n, L.nz) : L.nz;
    double ncount = (double)pl * (zc1 - zc0);
    petto_status st = allreduce(&ncount, 1, user);
    if (st != PETTO_OK) return st;
    // 1. the state solve, then the ghost planes brought up to date for the sensitivity
    petto_solve_report rep{};
    st = petto_slab_solve(ctx, so, exchange, allreduce, allreduce_max, user, &rep);
    const bool notconv = st == PETTO_ENOTCONV;
    if (st != PETTO_OK && !notconv) return st;
    st = exchange(ctx, user);
    if (st != PETTO_OK) return st;
    // 2. sensitivity of every held cell (a ghost layer gets its owner's bits); C and F.u over
    //    this slab's own layers and planes, max |s_i| over the whole grid
    CK(cudaMemsetAsync(ctx->scal + SC_SMAX, 0, sizeof(double) * MAX_PHASES, ctx->stream));
    SensArgs sa{};
    sa.L = L;
    sa.physics = ctx->physics;
    sa.ncomp = ctx->ncomp;
    sa.nrhs = ctx->nrhs;
    sa.k = ctx->k;
    sa.lam = ctx->lam0;
    sa.mu = ctx->mu0;
    sa.h = ctx->h;
    sa.zc0 = zc0;
    sa.zc1 = zc1;
    DesignArgs d = design_args(ctx);
    CK(launch_sensitivity(sa, d, ctx->u[ctx->cur], ctx->E, ctx->phi, ctx->s, ctx->scal, ctx->red(), ctx->stream));
    CK(launch_work(L, ctx->ncomp, ctx->nrhs, ctx->precision, ctx->loads, ctx->n_loads, ctx->u[ctx->cur], 0.0,
                   ctx->scal, ctx->red(), ctx->stream));
    ctx->launches += 2;
    double sc[SC_N];
    st = read_scal(ctx, sc);
    if (st != PETTO_OK) return st;
    double cw[2] = {sc[SC_C], sc[SC_W]};
    double smax[MAX_PHASES];
    for (int q = 0; q < P; ++q) smax[q] = sc[SC_SMAX + q];
    st = allreduce(cw, 2, user);
    if (st == PETTO_OK) st = allreduce_max(smax, P, user);
    if (st != PETTO_OK) return st;
    CK(cudaMemcpyAsync(ctx->scal + SC_SMAX, smax, sizeof(double) * P, cudaMemcpyHostToDevice, ctx->stream));
    // 3. the design update on every held cell, with the whole grid's sums: the means (penalty)
    //    and the bisection's bracket (projected) move on the host
    auto grid_means = [&](double *mean) -> petto_status {
        CK(launch_layer_sums(L, P, ctx->storage, ctx->phi, zc0, zc1, ctx->scal, SC_SUM, ctx->red(), ctx->stream));
        ctx->launches++;
        double s2[SC_N];
        petto_status e = read_scal(ctx, s2);
        if (e != PETTO_OK) return e;
        for (int q = 0; q < P; ++q) mean[q] = s2[SC_SUM + q];
        e = allreduce(mean, P, user);
        if (e != PETTO_OK) return e;
        for (int q = 0; q < P; ++q) mean[q] /= ncount;
        return PETTO_OK;
    };
    UpdateArgs ua{};
    ua.ncell = L.ncells();
    ua.P = P;
    ua.vol_mode = po->vol_mode;
    ua.n_bisect = po->n_bisect;
    ua.precision = ctx->precision;
    ua.storage = ctx->storage;
    ua.alpha_h = po->alpha_h;
    ua.kappa_v = po->kappa_v;
    ua.kappa_1 = po->kappa_1;
    for (int q = 0; q < P; ++q) ua.V[q] = ctx->vol[q];
    ua.nx = L.nx;
    ua.ny = L.ny;
    ua.ext = 1;
    ua.zc0 = zc0;
    ua.zc1 = zc1;
    ua.layer = pl;
    double mean[MAX_PHASES] = {0}, lam[MAX_PHASES] = {0};
    if (po->vol_mode == PETTO_VOL_PENALTY) {
        st = grid_means(mean);
        if (st != PETTO_OK) return st;
        CK(cudaMemcpyAsync(ctx->scal + SC_MEAN, mean, sizeof(double) * P, cudaMemcpyHostToDevice, ctx->stream));
        for (int q = 0; q < P; ++q) lam[q] = mean[q];
    }
    CK(launch_update(ua, ctx->phi, ctx->s, ctx->dscr, ctx->scal, ctx->red(), ctx->stream, &ctx->launches));
    if (po->vol_mode == PETTO_VOL_PROJECTED) {
        double br[2 * MAX_PHASES];  // [lo_0 .. lo_P-1 | hi_0 .. hi_P-1] as in scal
        for (int q = 0; q < P; ++q) {
            br[q] = -2.0;
            br[MAX_PHASES + q] = 2.0;
        }
        for (int it = 0; it <= po->n_bisect; ++it) {
            CK(cudaMemcpyAsync(ctx->scal + SC_LO, br, sizeof(double) * P, cudaMemcpyHostToDevice, ctx->stream));
            CK(cudaMemcpyAsync(ctx->scal + SC_HI, br + MAX_PHASES, sizeof(double) * P, cudaMemcpyHostToDevice,
                               ctx->stream));
            if (it == po->n_bisect) break;  // the final bracket is on the device
            CK(launch_bisect_sums(ua, ctx->dscr, ctx->scal, ctx->red(), ctx->stream));
            ctx->launches++;
            double s2[SC_N], sums[MAX_PHASES];
            st = read_scal(ctx, s2);
            if (st != PETTO_OK) return st;
            for (int q = 0; q < P; ++q) sums[q] = s2[SC_SUM + q];
            st = allreduce(sums, P, user);
            if (st != PETTO_OK) return st;
            for (int q = 0; q < P; ++q) {
                const double m = sums[q] / ncount, md = 0.5 * (br[q] + br[MAX_PHASES + q]);
                if (m > ua.V[q]) br[q] = md;
                else br[MAX_PHASES + q] = md;
            }
        }
        CK(launch_update_apply(ua, ctx->phi, ctx->dscr, ctx->scal, ctx->stream));
        ctx->launches++;
        for (int q = 0; q < P; ++q) lam[q] = 0.5 * (br[q] + br[MAX_PHASES + q]);
    }
    ctx->have_sens = false;
    // 4. Cahn-Hilliard: phi's layers next to each interface are exchanged before mu is formed,
    //    mu's before phi moves, and phi's again at the end (the ghost layer and the copy of the
    //    layer above then hold their owners' values)
    for (int t = 0; t < po->ch_steps; ++t)
        for (int q = 0; q < P; ++q) {
            char *dummy = nullptr;
            st = layer_ptr(ctx, PETTO_LAYER_PHI, q, L.nz, &dummy);  // makes the copies of the layer above
            if (st == PETTO_OK) st = layer_ptr(ctx, PETTO_LAYER_MU, 0, L.nz, &dummy);
            if (st == PETTO_OK) st = exchange_layer(ctx, PETTO_LAYER_PHI, q, user);
            if (st != PETTO_OK) return st;
            const void *phh = ctx->own_n && ctx->own_lo + ctx->own_n < L.NZ ? ctx->phi_hi : nullptr;
            const void *muh = ctx->own_n && ctx->own_lo + ctx->own_n < L.NZ ? ctx->mu_hi : nullptr;
            CK(launch_ch_half(L, q, 0, ctx->storage, ctx->precision, po->gamma_g, po->tau, ctx->phi, ctx->mu, phh, muh,
                              ctx->stream));
            st = exchange_layer(ctx, PETTO_LAYER_MU, q, user);
            if (st != PETTO_OK) return st;
            CK(launch_ch_half(L, q, 1, ctx->storage, ctx->precision, po->gamma_g, po->tau, ctx->phi, ctx->mu, phh, muh,
                              ctx->stream));
            ctx->launches += 2;
        }
    if (po->ch_steps > 0)
        for (int q = 0; q < P; ++q) {
            st = exchange_layer(ctx, PETTO_LAYER_PHI, q, user);
            if (st != PETTO_OK) return st;
        }
    st = refresh_material(ctx);
    if (st != PETTO_OK) return st;
    ctx->step++;
    if (metrics) {
        double vol[MAX_PHASES];
        st = grid_means(vol);
        if (st != PETTO_OK) return st;
        const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        const double m[8] = {(double)ctx->step, cw[0], cw[1], rep.rel_res, (double)rep.sweeps, secs, vol[0], lam[0]};
        std::memcpy(metrics, m, sizeof(m));
    }
    return notconv ? PETTO_ENOTCONV : PETTO_OK;
}

petto_status petto_set_wait_limit(petto_ctx *ctx, int tries) {
    if (!ctx || tries > WAIT_TRIES) return fail(ctx, PETTO_EINVAL, "wait limit above the default");
    ctx->wait_tries = tries < 0 ? WAIT_TRIES : tries;
    clear_graphs(ctx);  // captured sweeps carry the limit in their arguments
    return PETTO_OK;
}

petto_status petto_sweep_rhs(petto_ctx *ctx, int kind, int64_t n, double a, double b, double s1, int local_dt,
                             const double *r, int on_device, double *res_norm2) {
    if (!ctx || n < 0 || !r || (kind != PETTO_SWEEP_APT && kind != PETTO_SWEEP_PT))
        return fail(ctx, PETTO_EINVAL, "bad sweep arguments");
    petto_status st = refine_alloc(ctx);
    if (st != PETTO_OK) return st;
    const int C = ctx->ndofc();
    const int64_t nn = (int64_t)C * ctx->L.nnodes();
    const double *src = r;
    if (!on_device) {
        st = ensure_stage(ctx, nn * sizeof(double));
        if (st != PETTO_OK) return st;
        CK(cudaMemcpyAsync(ctx->stage, r, nn * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
        src = static_cast<const double *>(ctx->stage);
    }
    pack_nodes<double, double><<<grid_of(nn), 256, 0, ctx->stream>>>(ctx->L, C, src, (double *)ctx->r64, 1);
    CK(cudaGetLastError());
    ctx->launches++;
    const void *rhs = ctx->r64;
    if (ctx->precision == PETTO_F32) {
        st = refine_rhs(ctx);
        if (st != PETTO_OK) return st;
        rhs = ctx->rhs32;
    }
    SweepCtl sc;
    sc.rhs = rhs;
    for (int64_t t = 0; t < n;) {
        const int g = sweep_group(ctx, t, n);
        sc.idx = t;
        st = one_sweep(ctx, kind, a, b, s1, local_dt, res_norm2 && t + g == n, sc, g);
        if (st != PETTO_OK) return st;
        t += g;
    }
    if (res_norm2) {
        if (n == 0) {
            *res_norm2 = 0.0;
            return PETTO_OK;
        }
        CK(cudaMemcpyAsync(res_norm2, ctx->scal + SC_RES, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    } else if (!on_device) {
        CK(cudaStreamSynchronize(ctx->stream));
    }
    return PETTO_OK;
}

petto_status petto_sensitivity(petto_ctx *ctx, double *compliance, double *work, void *dcdphi, int dtype,
                               int on_device) {
    if (!ctx) return PETTO_EINVAL;
    CK(cudaMemsetAsync(ctx->scal + SC_SMAX, 0, sizeof(double) * MAX_PHASES, ctx->stream));
    SensArgs sa{};
    sa.L = ctx->L;
    sa.physics = ctx->physics;
    sa.ncomp = ctx->ncomp;
    sa.nrhs = ctx->nrhs;
    sa.k = ctx->k;
    sa.lam = ctx->lam0;
    sa.mu = ctx->mu0;
    sa.h = ctx->h;
    DesignArgs d = design_args(ctx);
    CK(launch_sensitivity(sa, d, ctx->u[ctx->cur], ctx->E, ctx->phi, ctx->s, ctx->scal, ctx->red(), ctx->stream));
    ctx->launches++;
    CK(launch_work(ctx->L, ctx->ncomp, ctx->nrhs, ctx->precision, ctx->loads, ctx->n_loads, ctx->u[ctx->cur],
                   ctx->k.src, ctx->scal, ctx->red(), ctx->stream));
    ctx->launches++;
    ctx->have_sens = true;
    if (compliance || work) {
        double sc[SC_N];
        petto_status st = read_scal(ctx, sc);
        if (st != PETTO_OK) return st;
        if (compliance) *compliance = sc[SC_C];
        if (work) *work = sc[SC_W];
    }
    if (dcdphi)
        return flat_out(ctx, ctx->s, ctx->precision == 0 ? PETTO_F32 : PETTO_F64, dcdphi, dtype, on_device,
                        (int64_t)ctx->P * ctx->L.ncells());
    return PETTO_OK;
}

petto_status petto_design_update(petto_ctx *ctx, const petto_pf_opts *o, double *lambda) {
    if (!ctx || !o) return fail(ctx, PETTO_EINVAL, "null argument");
    if (!ctx->have_sens) return fail(ctx, PETTO_EINVAL, "petto_design_update needs petto_sensitivity first");
    if (o->vol_mode != PETTO_VOL_PROJECTED && o->vol_mode != PETTO_VOL_PENALTY)
        return fail(ctx, PETTO_EINVAL, "bad vol_mode");
    if (o->n_bisect < 0 || o->n_bisect > 200) return fail(ctx, PETTO_EINVAL, "n_bisect out of range");
    UpdateArgs ua{};
    ua.ncell = ctx->L.ncells();
    ua.P = ctx->P;
    ua.vol_mode = o->vol_mode;
    ua.n_bisect = o->n_bisect;
    ua.precision = ctx->precision;
    ua.storage = ctx->storage;
    ua.alpha_h = o->alpha_h;
    ua.kappa_v = o->kappa_v;
    ua.kappa_1 = o->kappa_1;
    for (int p = 0; p < ctx->P; ++p) ua.V[p] = ctx->vol[p];
    ua.keep = ctx->keep;
    ua.nx = ctx->L.nx;
    ua.ny = ctx->L.ny;
    for (int a = 0; a < 3; ++a) {
        ua.klo[a] = ctx->klo[a];
        ua.khi[a] = ctx->khi[a];
    }
    ua.kappa_b = ctx->kappa_b;
    for (int p = 0; p < ctx->P; ++p) ua.Vb[p] = ctx->Vb[p];
    if (o->vol_mode == PETTO_VOL_PENALTY) {
        CK(launch_mean(ctx->L, ctx->P, ctx->storage, ctx->phi, ctx->scal, ctx->red(), ctx->stream));
        ctx->launches++;
    }
    CK(launch_update(ua, ctx->phi, ctx->s, ctx->dscr, ctx->scal, ctx->red(), ctx->stream, &ctx->launches));
    ctx->have_sens = false;
    petto_status st = refresh_material(ctx);
    if (st != PETTO_OK) return st;
    if (lambda) {
        double sc[SC_N];
        st = read_scal(ctx, sc);
        if (st != PETTO_OK) return st;
        for (int p = 0; p < ctx->P; ++p) lambda[p] = o->vol_mode == PETTO_VOL_PROJECTED ? sc[SC_LAM + p] : sc[SC_MEAN + p];
    }
    return PETTO_OK;
}

petto_status petto_set_keepout(petto_ctx *ctx, const int64_t *box, const double *target, double kappa_b) {
    if (!ctx) return PETTO_EINVAL;
    CK(cudaStreamSynchronize(ctx->stream));
    clear_graphs(ctx);  // captured design loops carry the update's keep-out term
    if (!box) {
        ctx->keep = 0;
        return PETTO_OK;
    }
    if (!target) return fail(ctx, PETTO_EINVAL, "keep-out targets missing");
    const int64_t n[3] = {ctx->L.nx, ctx->L.ny, ctx->dim == 3 ? ctx->L.nz : 1};
    for (int a = 0; a < 3; ++a)
        if (box[a] < 0 || box[3 + a] >= n[a] || box[a] > box[3 + a])
            return fail(ctx, PETTO_EINVAL, "keep-out box outside the grid or empty");
    if (!(kappa_b >= 0.0)) return fail(ctx, PETTO_EINVAL, "kappa_b must be >= 0");
    for (int a = 0; a < 3; ++a) {
        ctx->klo[a] = (int)box[a];
        ctx->khi[a] = (int)box[3 + a];
    }
    for (int p = 0; p < ctx->P; ++p) ctx->Vb[p] = target[p];
    ctx->kappa_b = kappa_b;
    ctx->keep = 1;
    return PETTO_OK;
}

petto_status petto_set_owned_planes(petto_ctx *ctx, int64_t zlo, int64_t zhi, int64_t z_global) {
    if (ctx) ctx->tune_pending = false;  // a slab keeps the kernel its decomposition chose
    if (!ctx) return PETTO_EINVAL;
    if (ctx->dim != 3) return fail(ctx, PETTO_EUNSUPPORTED, "slabs are z ranges of a 3D grid");
    const int NZ = ctx->L.NZ;
    if (zlo < 0 || zhi >= NZ || zlo > zhi) return fail(ctx, PETTO_EINVAL, "owned planes outside the grid or empty");
    if (z_global < 0) return fail(ctx, PETTO_EINVAL, "negative global plane offset");
    ctx->own_z0 = z_global;
    const bool whole = zlo == 0 && zhi == NZ - 1;
    Tiling t = ctx->tiling;
    if (!whole && t.kind != 0 && !two_row_kind(t.kind)) {
        // another marching variant is selected: a slab sweeps with the node gather instead
        t = gather_tiling(ctx->L);
    }
    t.zlo = 0;
    t.zn = 0;
    ctx->own_lo = whole ? 0 : (int)zlo;
    ctx->own_n = whole ? 0 : (int)(zhi - zlo + 1);
    // the tiling of the FP64 defect (the node gather on a slab), restricted the same way
    const Tiling g = own_planes(ctx, defect_tiling(ctx));
    const int NX = ctx->L.NX, NY = ctx->L.NY, gnt = g.ntiles();
    std::vector<int> gptr(gnt + 1, 0);
    std::vector<std::pair<int, LoadEntry>> tmp;
    for (auto &kv : ctx->load_list) {
        const int64_t n = kv.first.first;
        const int i = (int)(n % NX), j = (int)((n / NX) % NY), k = (int)(n / ((int64_t)NX * NY));
        LoadEntry le{};
        le.node = ctx->L.node(i, j, k);
        le.comp = kv.first.second;
        le.vald = kv.second;
        le.valf = (float)kv.second;
        const int tl = g.tile_of(i, j, k);
        if (tl >= 0) tmp.emplace_back(tl, le);
    }
    std::stable_sort(tmp.begin(), tmp.end(), [](const auto &x, const auto &y) { return x.first < y.first; });
    std::vector<LoadEntry> gent;
    for (auto &pr : tmp) {
        gptr[pr.first + 1]++;
        gent.push_back(pr.second);
    }
    for (int q = 0; q < gnt; ++q) gptr[q + 1] += gptr[q];
    CK(cudaStreamSynchronize(ctx->stream));
    // fewer (or as many) tiles than the whole-grid table allocated at creation
    CK(cudaMemcpy(ctx->gtile_ptr, gptr.data(), sizeof(int) * (gnt + 1), cudaMemcpyHostToDevice));
    if (!gent.empty())
        CK(cudaMemcpy(ctx->gloads, gent.data(), sizeof(LoadEntry) * gent.size(), cudaMemcpyHostToDevice));
    ctx->gtiling = g;
    return set_tiling(ctx, t);
}

namespace {
// one node plane k of the current state, every component, as [C][NY][NX] at dst/src
petto_status copy_plane(petto_ctx *ctx, int64_t k, void *dst, const void *src, int dtype, int on_device) {
    if (!ctx || (!dst && !src)) return fail(ctx, PETTO_EINVAL, "null argument");
    if (k < 0 || k >= ctx->L.NZ) return fail(ctx, PETTO_EINVAL, "plane outside the grid");
    if (dtype != ctx->precision) return fail(ctx, PETTO_EINVAL, "planes are copied in the sweep precision");
    const Layout &L = ctx->L;
    const size_t T = ctx->tsize();
    char *u = static_cast<char *>(ctx->u[ctx->cur]);
    const size_t plane = (size_t)L.NX * L.NY * T;
    for (int c = 0; c < ctx->ndofc(); ++c) {
        char *field = u + ((int64_t)c * L.cstride + L.node(0, 0, (int)k)) * T;
        if (dst)
            CK(cudaMemcpy2DAsync(static_cast<char *>(dst) + c * plane, L.NX * T, field, L.SX * T, L.NX * T, L.NY,
                                 cudaMemcpyDefault, ctx->stream));
        else
            CK(cudaMemcpy2DAsync(field, L.SX * T, static_cast<const char *>(src) + c * plane, L.NX * T, L.NX * T,
                                 L.NY, cudaMemcpyDefault, ctx->stream));
    }
    if (!on_device) CK(cudaStreamSynchronize(ctx->stream));  // host memory is the caller's again on return
    return PETTO_OK;
}
}  // namespace

petto_status petto_get_plane(petto_ctx *ctx, int64_t k, void *dst, int dtype, int on_device) {
    return copy_plane(ctx, k, dst, nullptr, dtype, on_device);
}

petto_status petto_set_plane(petto_ctx *ctx, int64_t k, const void *src, int dtype, int on_device) {
    return copy_plane(ctx, k, nullptr, src, dtype, on_device);
}

petto_status petto_get_layer(petto_ctx *ctx, int field, int phase, int64_t k, void *dst, int on_device) {
    return copy_layer(ctx, field, phase, k, dst, nullptr, on_device);
}

petto_status petto_set_layer(petto_ctx *ctx, int field, int phase, int64_t k, const void *src, int on_device) {
    return copy_layer(ctx, field, phase, k, nullptr, src, on_device);
}

petto_status petto_cahn_hilliard(petto_ctx *ctx, const petto_pf_opts *o) {
    if (!ctx || !o) return fail(ctx, PETTO_EINVAL, "null argument");
    if (o->ch_steps < 0) return fail(ctx, PETTO_EINVAL, "negative ch_steps");
    for (int t = 0; t < o->ch_steps; ++t)
        CK(launch_ch(ctx->L, ctx->P, ctx->storage, ctx->precision, o->gamma_g, o->tau, ctx->phi, ctx->mu, ctx->stream,
                     &ctx->launches));
    return refresh_material(ctx);
}

petto_status petto_phase_field_step(petto_ctx *ctx, const petto_pf_opts *o, double *vol_out) {
    petto_status st = petto_design_update(ctx, o, nullptr);
    if (st != PETTO_OK) return st;
    st = petto_cahn_hilliard(ctx, o);
    if (st != PETTO_OK) return st;
    if (vol_out) {
        CK(launch_mean(ctx->L, ctx->P, ctx->storage, ctx->phi, ctx->scal, ctx->red(), ctx->stream));
        ctx->launches++;
        double sc[SC_N];
        st = read_scal(ctx, sc);
        if (st != PETTO_OK) return st;
        for (int p = 0; p < ctx->P; ++p) vol_out[p] = sc[SC_MEAN + p];
    }
    return PETTO_OK;
}

}  // extern "C"

namespace {

// A design loop of the paper's fixed-count schedule (Fig. 5 with n_apt APT and n_pt PT
// sweeps, no checks) takes no host decision between its launches: the solve's sweeps, the
// sensitivity, the update (its bisection runs on the device), Cahn-Hilliard, the modulus and
// the volume means.  After a first loop on the ordinary path (which also runs the
// autotuner), petto_optimize captures one loop as a CUDA graph and replays it, one host read
// of the scalars per loop.  The graph holds the same launches in the same order, so the
// loops give the same bits.
bool step_graph_ok(const petto_ctx *ctx, const petto_solve_opts *so) {
    return so->mode == PETTO_SOLVE_PAPER && so->check_every == 0 && ctx->use_graphs && ctx->stream &&
           !ctx->trace && !ctx->tune_pending && so->n_apt >= 0 && so->n_pt >= 0 && so->n_apt + so->n_pt > 0;
}

bool same_opts(const petto_solve_opts &a, const petto_solve_opts &b) { return std::memcmp(&a, &b, sizeof a) == 0; }
bool same_opts(const petto_pf_opts &a, const petto_pf_opts &b) { return std::memcmp(&a, &b, sizeof a) == 0; }

// the launches of one loop, on the context's stream (captured by the caller)
petto_status step_launches(petto_ctx *ctx, const petto_solve_opts *so, const petto_pf_opts *po, int *flips,
                           int *swaps, cudaEvent_t ev0, cudaEvent_t ev1) {
    *flips = *swaps = 0;
    CK(cudaMemsetAsync(ctx->w, 0, ctx->node_bytes(), ctx->stream));
    petto_status st = set_ctrl(ctx, CT_RESTART_AT, 0);
    if (st == PETTO_OK) st = set_ctrl(ctx, CT_ERR, 0);
    if (st == PETTO_OK && ev0) CK(cudaEventRecordWithFlags(ev0, ctx->stream, cudaEventRecordExternal));
    const int64_t n_apt = so->momentum == 2 ? 0 : so->n_apt;
    const int64_t total = so->n_apt + so->n_pt;
    for (int64_t t = 0; t < total && st == PETTO_OK;) {
        const bool apt = t < n_apt;
        const int g = apt ? sweep_group(ctx, t, n_apt) : sweep_group(ctx, t - n_apt, total - n_apt);
        SweepCtl sc;
        sc.adaptive = so->momentum == 1 ? 1 : 0;
        sc.test_dot = apt && sc.adaptive && ((t + g - 1) % 4) == 3;
        sc.idx = t;
        st = one_sweep(ctx, apt ? 0 : 1, so->a, so->b, so->s1, so->local_dt, t + g == total, sc, g);
        ++*flips;
        if (g > 1 && apt) ++*swaps;
        t += g;
    }
    if (st == PETTO_OK && ev1) CK(cudaEventRecordWithFlags(ev1, ctx->stream, cudaEventRecordExternal));
    if (st == PETTO_OK) st = petto_sensitivity(ctx, nullptr, nullptr, nullptr, PETTO_F64, 0);
    if (st == PETTO_OK) st = petto_design_update(ctx, po, nullptr);
    if (st == PETTO_OK && po->vol_mode == PETTO_VOL_PENALTY)  // keep the pre-step means (the penalty's lambda)
        CK(cudaMemcpyAsync(ctx->scal + SC_SUM, ctx->scal + SC_MEAN, sizeof(double) * ctx->P, cudaMemcpyDeviceToDevice,
                           ctx->stream));
    if (st == PETTO_OK) st = petto_cahn_hilliard(ctx, po);
    if (st == PETTO_OK) {
        CK(launch_mean(ctx->L, ctx->P, ctx->storage, ctx->phi, ctx->scal, ctx->red(), ctx->stream));
        ctx->launches++;
    }
    return st;
}

petto_status take_event(petto_ctx *ctx, cudaEvent_t *e) {
    if (!ctx->ev_free.empty()) {
        *e = ctx->ev_free.back();
        ctx->ev_free.pop_back();
        return PETTO_OK;
    }
    CK(cudaEventCreate(e));
    return PETTO_OK;
}

petto_status step_graph(petto_ctx *ctx, const petto_solve_opts *so, const petto_pf_opts *po) {
    const int prof = ctx->profiling ? 1 : 0;
    petto_ctx::StepGraph *ge = nullptr;
    for (auto &g : ctx->step_graphs)
        if (g.cur == ctx->cur && g.w == ctx->w && g.profiled == prof && same_opts(g.so, *so) && same_opts(g.po, *po))
            ge = &g;
    if (!ge) {
        if (ctx->step_graphs.size() >= 4) clear_graphs(ctx);
        const int cur0 = ctx->cur;
        void *const w0 = ctx->w;
        const int64_t l0 = ctx->launches;
        // the sweeps are timed as a whole (event records in the graph, given fresh events at
        // every replay), not launch by launch
        cudaEvent_t mark[2] = {nullptr, nullptr};
        if (prof)
            for (cudaEvent_t &e : mark) {
                petto_status se = take_event(ctx, &e);
                if (se != PETTO_OK) return se;
            }
        cudaGraph_t graph = nullptr;
        CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
        int flips = 0, swaps = 0;
        ctx->profiling = false;
        petto_status st = step_launches(ctx, so, po, &flips, &swaps, mark[0], mark[1]);
        ctx->profiling = prof != 0;
        cudaError_t ec = cudaStreamEndCapture(ctx->stream, &graph);
        const int64_t nl = ctx->launches - l0;
        ctx->cur = cur0;
        if (ctx->w != w0) std::swap(ctx->w, ctx->w_alt);
        ctx->launches = l0;
        for (cudaEvent_t e : mark)
            if (e) ctx->ev_free.push_back(e);
        if (st != PETTO_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        CK(ec);
        petto_ctx::StepGraph sg{cur0, w0, *so, *po, nullptr, flips, swaps, nl, prof, graph, {nullptr, nullptr}};
        if (prof) {
            size_t nn = 0;
            CK(cudaGraphGetNodes(graph, nullptr, &nn));
            std::vector<cudaGraphNode_t> nodes(nn);
            CK(cudaGraphGetNodes(graph, nodes.data(), &nn));
            for (cudaGraphNode_t nd : nodes) {
                cudaGraphNodeType ty;
                CK(cudaGraphNodeGetType(nd, &ty));
                if (ty != cudaGraphNodeTypeEventRecord) continue;
                cudaEvent_t e = nullptr;
                CK(cudaGraphEventRecordNodeGetEvent(nd, &e));
                if (e == mark[0]) sg.ev_node[0] = nd;
                if (e == mark[1]) sg.ev_node[1] = nd;
            }
            if (!sg.ev_node[0] || !sg.ev_node[1]) {
                cudaGraphDestroy(graph);
                return fail(ctx, PETTO_ECUDA, "event records missing from the captured loop");
            }
        }
        cudaError_t ei = cudaGraphInstantiate(&sg.exec, graph, 0);
        if (ei != cudaSuccess) {
            cudaGraphDestroy(graph);
            CK(ei);
        }
        if (!prof) {
            cudaGraphDestroy(graph);
            sg.graph = nullptr;
        }
        ctx->step_graphs.push_back(sg);
        ge = &ctx->step_graphs.back();
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (prof) {
        petto_status se = take_event(ctx, &e0);
        if (se == PETTO_OK) se = take_event(ctx, &e1);
        if (se != PETTO_OK) return se;
        CK(cudaGraphExecEventRecordNodeSetEvent(ge->exec, ge->ev_node[0], e0));
        CK(cudaGraphExecEventRecordNodeSetEvent(ge->exec, ge->ev_node[1], e1));
    }
    CK(cudaGraphLaunch(ge->exec, ctx->stream));
    if (prof) {
        ctx->ev_pending.emplace_back(e0, e1);
        ctx->ev_count.push_back((int)(so->n_apt + so->n_pt));
        ctx->ev_rhs.push_back(0);
    }
    ctx->launches += ge->launches;
    if (ge->flips & 1) ctx->cur ^= 1;
    if (ge->swaps & 1) std::swap(ctx->w, ctx->w_alt);
    ctx->have_sens = false;
    return PETTO_OK;
}

}  // namespace

extern "C" {

petto_status petto_optimize(petto_ctx *ctx, int n_steps, const petto_solve_opts *so, const petto_pf_opts *po,
                            petto_step_cb cb, void *user) {
    if (!ctx || !so || !po || n_steps < 0) return fail(ctx, PETTO_EINVAL, "bad arguments");
    bool notconv = false;
    for (int t = 0; t < n_steps; ++t) {
        const auto t0 = std::chrono::steady_clock::now();
        // (a first loop on this context, here or in an earlier call, ran the ordinary path)
        if ((t > 0 || ctx->step > 0) && step_graph_ok(ctx, so)) {
            // the paper's fixed-count loop: the whole loop is one graph replay
            petto_status st = step_graph(ctx, so, po);
            if (st != PETTO_OK) return st;
            ctx->step++;
            if (cb) {
                double sc[SC_N];
                st = read_scal(ctx, sc);
                if (st != PETTO_OK) return st;
                const double lam0 = po->vol_mode == PETTO_VOL_PROJECTED ? sc[SC_LAM] : sc[SC_SUM];
                const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
                const double fn = ctx->f_norm;
                const double m[8] = {(double)ctx->step, sc[SC_C], sc[SC_W], fn > 0 ? std::sqrt(sc[SC_RES]) / fn : NAN,
                                     (double)(so->n_apt + so->n_pt), secs, sc[SC_MEAN], lam0};
                cb(m, user);
            }
            continue;
        }
        petto_solve_report rep{};
        petto_status st = petto_pt_solve(ctx, so, &rep);
        if (st == PETTO_ENOTCONV) notconv = true;
        else if (st != PETTO_OK) return st;
        // the design half without host round trips; one read of the scalars at the end
        st = petto_sensitivity(ctx, nullptr, nullptr, nullptr, PETTO_F64, 0);
        if (st != PETTO_OK) return st;
        st = petto_design_update(ctx, po, nullptr);
        if (st != PETTO_OK) return st;
        if (po->vol_mode == PETTO_VOL_PENALTY)  // keep the pre-step means (the penalty's lambda)
            CK(cudaMemcpyAsync(ctx->scal + SC_SUM, ctx->scal + SC_MEAN, sizeof(double) * ctx->P,
                               cudaMemcpyDeviceToDevice, ctx->stream));
        st = petto_cahn_hilliard(ctx, po);
        if (st != PETTO_OK) return st;
        ctx->step++;
        if (cb) {
            CK(launch_mean(ctx->L, ctx->P, ctx->storage, ctx->phi, ctx->scal, ctx->red(), ctx->stream));
            ctx->launches++;
            double sc[SC_N];
            st = read_scal(ctx, sc);
            if (st != PETTO_OK) return st;
            const double lam0 = po->vol_mode == PETTO_VOL_PROJECTED ? sc[SC_LAM] : sc[SC_SUM];
            const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            const double m[8] = {(double)ctx->step, sc[SC_C], sc[SC_W], rep.rel_res, (double)rep.sweeps, secs,
                                 sc[SC_MEAN], lam0};
            cb(m, user);
        }
    }
    if (!cb && n_steps > 0 && ctx->step > 1 && step_graph_ok(ctx, so)) {
        // the replayed loops read nothing back: surface a run-out ring wait here
        double sc[SC_N];
        petto_status st = read_scal(ctx, sc);
        if (st != PETTO_OK) return st;
    }
    return notconv ? PETTO_ENOTCONV : PETTO_OK;
}

}  // extern "C"

// ============================================================================ batches
// A batch advances many independent 2D problems together: one launch of sweep2d_batch per
// sweep covers the tiles of every problem still iterating, each chunk of check_every
// sweeps is one CUDA graph, and all residual checks of a chunk are read with one copy.
// Per problem, the iteration, its checks, restarts, PT fallback and FP32 refinement are
// those of petto_pt_solve (the same helpers and the same kernel arithmetic), so a problem
// solved in a batch ends in the same state as when solved alone.
struct petto_batch {
    std::vector<petto_ctx *> ctx;   // borrowed
    cudaStream_t stream = nullptr;  // the first context's stream
    int precision = 0, physics = 0;
    std::vector<BatchInst> inst;    // host mirror of the device table
    BatchInst *d_inst = nullptr;
    std::vector<BatchTile> tiles;   // active problems' tiles first
    BatchTile *d_tiles = nullptr;
    int ntiles = 0;                 // all tiles
    int nact = 0;                   // tiles of the active problems (the launch grid)
    long long *d_base = nullptr;    // device word: first sweep index of the chunk
    double *d_res = nullptr;        // sum R^2 of each problem's last check sweep
    std::vector<int> active;
    int cur = 0;
    int64_t launches = 0;
    struct Graph {
        int len, cur, adaptive, local_dt;
        int nact;  // grid the graph's launches currently have
        cudaGraphExec_t exec;
    };
    std::vector<Graph> graphs;
    cudaEvent_t ev = nullptr;
    bool profiling = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pending;
    std::vector<int> ev_count;
    std::vector<cudaEvent_t> ev_free;
    double prof_ms = 0.0;
    int64_t prof_sweeps = 0;
    std::string err;
};

namespace {

petto_status bfail(petto_batch *b, petto_status st, const std::string &msg) {
    if (b) b->err = msg;
    return st;
}

#define BCK(call)                                                                                      \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess)                                                                         \
            return bfail(b, PETTO_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));         \
    } while (0)

__global__ void set_word_kernel(long long *w, long long v) { *w = v; }

// problems' contexts run on the batch stream for the duration of a batch call
struct StreamJoin {
    petto_batch *b;
    std::vector<cudaStream_t> saved;
    explicit StreamJoin(petto_batch *bb) : b(bb) {
        for (petto_ctx *c : b->ctx) {
            saved.push_back(c->stream);
            if (c->stream != b->stream) {
                cudaEventRecord(b->ev, c->stream);
                cudaStreamWaitEvent(b->stream, b->ev, 0);
                c->stream = b->stream;
            }
        }
    }
    ~StreamJoin() {
        for (size_t i = 0; i < b->ctx.size(); ++i) {
            petto_ctx *c = b->ctx[i];
            if (saved[i] != b->stream) {
                c->stream = saved[i];
                cudaEventRecord(b->ev, b->stream);
                cudaStreamWaitEvent(saved[i], b->ev, 0);
            }
        }
    }
};

// re-read each problem's buffers and tiling from its context (a context may have been
// re-tiled or used alone since the last batch call) and bring every state to u[cur]
petto_status batch_refresh(petto_batch *b) {
    int ntiles = 0;
    for (size_t i = 0; i < b->ctx.size(); ++i) {
        petto_ctx *ctx = b->ctx[i];
        if (!march2d_ok(ctx)) return bfail(b, PETTO_EUNSUPPORTED, "a problem is too large for the batched sweep");
        if (ctx->tiling.kind != 5) {
            petto_status st = set_tiling(ctx, march2d_tiling(ctx->L));
            if (st != PETTO_OK) return bfail(b, st, ctx->err);
        }
        const Tiling &g = ctx->tiling;
        ntiles += g.gx * g.gy;
        if (ctx->cur != b->cur) {
            BCK(cudaMemcpyAsync(ctx->u[b->cur], ctx->u[ctx->cur], ctx->node_bytes(), cudaMemcpyDeviceToDevice,
                                b->stream));
            ctx->cur = b->cur;
        }
        BatchInst &I = b->inst[i];
        I.L = ctx->L;
        I.kf = base_sweep_args(ctx).kf;
        I.k = ctx->k;
        I.boxes = ctx->boxes;
        I.u[0] = ctx->u[0];
        I.u[1] = ctx->u[1];
        I.w = ctx->w;
        I.E = ctx->E;
        I.rhs = nullptr;
        I.tile_ptr = ctx->tile_ptr;
        I.loads = ctx->loads;
        I.red = ctx->red();
        I.ctrl = ctx->ctrl;
        I.gx = g.gx;
        I.gy = g.gy;
        I.ly = g.ly;
        I.res2 = b->d_res + i;
    }
    if (ntiles > b->ntiles) {
        BCK(cudaStreamSynchronize(b->stream));
        // the captured chunk graphs hold the old tile list's address
        for (auto &g : b->graphs) cudaGraphExecDestroy(g.exec);
        b->graphs.clear();
        if (b->d_tiles) BCK(cudaFree(b->d_tiles));
        b->d_tiles = nullptr;
        BCK(cudaMalloc(&b->d_tiles, sizeof(BatchTile) * ntiles));
    }
    b->ntiles = ntiles;
    return PETTO_OK;
}

// rebuild the tile list (active problems first) and upload it with the problem table
petto_status batch_upload(petto_batch *b) {
    b->tiles.clear();
    for (int pass = 0; pass < 2; ++pass)
        for (size_t i = 0; i < b->inst.size(); ++i) {
            if ((b->active[i] != 0) != (pass == 0)) continue;
            const int nt = b->inst[i].gx * b->inst[i].gy;
            for (int t = 0; t < nt; ++t) b->tiles.push_back(BatchTile{(int)i, t});
        }
    b->nact = 0;
    for (size_t i = 0; i < b->inst.size(); ++i)
        if (b->active[i]) b->nact += b->inst[i].gx * b->inst[i].gy;
    BCK(cudaMemcpyAsync(b->d_tiles, b->tiles.data(), sizeof(BatchTile) * b->tiles.size(), cudaMemcpyHostToDevice,
                        b->stream));
    BCK(cudaMemcpyAsync(b->d_inst, b->inst.data(), sizeof(BatchInst) * b->inst.size(), cudaMemcpyHostToDevice,
                        b->stream));
    // the host copies above are pageable: make sure they were taken before the mirrors change
    BCK(cudaStreamSynchronize(b->stream));
    return PETTO_OK;
}

BatchLaunch batch_launch(petto_batch *b, const petto_solve_opts *o, long long j, int len) {
    BatchLaunch p{};
    p.inst = b->d_inst;
    p.tiles = b->d_tiles;
    p.base = b->d_base;
    p.sweep_idx = j;
    p.cur = (b->cur + (int)j) & 1;
    p.physics = b->physics;
    p.nrhs = 1;
    p.local_dt = o->local_dt;
    p.want_res = j == len - 1;
    p.test_dot = (j % 4) == 3;
    p.adaptive = o->momentum ? 1 : 0;
    return p;
}

// capture len batched sweeps from u[cur] over the active tiles
petto_status batch_capture(petto_batch *b, const petto_solve_opts *o, int len, cudaGraph_t *graph) {
    *graph = nullptr;
    BCK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t el = cudaSuccess;
    for (int j = 0; j < len && el == cudaSuccess; ++j)
        el = launch_sweep2d_batch(batch_launch(b, o, j, len), b->nact, b->precision, b->stream);
    cudaError_t ec = cudaStreamEndCapture(b->stream, graph);
    if (el != cudaSuccess || ec != cudaSuccess) {
        if (*graph) cudaGraphDestroy(*graph);
        *graph = nullptr;
        BCK(el != cudaSuccess ? el : ec);
    }
    return PETTO_OK;
}

// len sweeps of every active problem from u[cur]: one graph per (len, cur, momentum, step)
// kind, its launch grids updated in place when the set of active problems changes
petto_status batch_chunk(petto_batch *b, const petto_solve_opts *o, long long base, int len) {
    set_word_kernel<<<1, 1, 0, b->stream>>>(b->d_base, base);
    BCK(cudaGetLastError());
    const int adaptive = o->momentum ? 1 : 0;
    petto_batch::Graph *ge = nullptr;
    for (auto &g : b->graphs)
        if (g.len == len && g.cur == b->cur && g.adaptive == adaptive && g.local_dt == o->local_dt) ge = &g;
    if (!ge || ge->nact != b->nact) {
        cudaGraph_t graph = nullptr;
        petto_status st = batch_capture(b, o, len, &graph);
        if (st != PETTO_OK) return st;
        bool updated = false;
        if (ge) {
            cudaGraphExecUpdateResultInfo info{};
            updated = cudaGraphExecUpdate(ge->exec, graph, &info) == cudaSuccess;
            if (!updated) {
                cudaGetLastError();
                cudaGraphExecDestroy(ge->exec);
                ge->exec = nullptr;
            }
        }
        if (!updated) {
            cudaGraphExec_t exec = nullptr;
            cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
            if (ei != cudaSuccess) {
                cudaGraphDestroy(graph);
                BCK(ei);
            }
            if (ge) ge->exec = exec;
            else {
                b->graphs.push_back(petto_batch::Graph{len, b->cur, adaptive, o->local_dt, b->nact, exec});
                ge = &b->graphs.back();
            }
        }
        ge->nact = b->nact;
        cudaGraphDestroy(graph);
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (b->profiling) {
        for (cudaEvent_t *e : {&e0, &e1}) {
            if (!b->ev_free.empty()) {
                *e = b->ev_free.back();
                b->ev_free.pop_back();
            } else {
                BCK(cudaEventCreate(e));
            }
        }
        BCK(cudaEventRecord(e0, b->stream));
    }
    BCK(cudaGraphLaunch(ge->exec, b->stream));
    if (b->profiling) {
        BCK(cudaEventRecord(e1, b->stream));
        b->ev_pending.emplace_back(e0, e1);
        b->ev_count.push_back(len);
    }
    b->launches += len + 1;
    if (len & 1) {
        // an odd chunk moves the active problems' state to the other buffer: move the
        // finished ones' along so that every problem's state is in u[cur]
        for (size_t i = 0; i < b->ctx.size(); ++i)
            if (!b->active[i]) {
                petto_ctx *c = b->ctx[i];
                BCK(cudaMemcpyAsync(c->u[1 - b->cur], c->u[b->cur], c->node_bytes(), cudaMemcpyDeviceToDevice,
                                    b->stream));
            }
        b->cur ^= 1;
    }
    for (petto_ctx *c : b->ctx) c->cur = b->cur;
    return PETTO_OK;
}

// per-problem solve state of a batched solve
struct BatchSolve {
    SolveState S;
    int phase = 0;          // 0 sweeps on the state, 1 refinement correction, 2 done
    double stop = 0.0;      // this phase's residual target
    int stall = 0;
    double true_res = NAN;
    bool conv = false;
};

}  // namespace

extern "C" {

petto_status petto_batch_create(int n, petto_ctx *const *ctxs, petto_batch **out) {
    if (!out || n <= 0 || !ctxs) return PETTO_EINVAL;
    *out = nullptr;
    for (int i = 0; i < n; ++i)
        if (!ctxs[i]) return PETTO_EINVAL;
    const petto_ctx *c0 = ctxs[0];
    for (int i = 0; i < n; ++i) {
        const petto_ctx *c = ctxs[i];
        if (c->dim != 2 || c->nrhs != 1 || c->precision != c0->precision || c->physics != c0->physics)
            return PETTO_EUNSUPPORTED;
    }
    petto_batch *b = new petto_batch();
    b->ctx.assign(ctxs, ctxs + n);
    b->stream = c0->stream;
    b->precision = c0->precision;
    b->physics = c0->physics;
    b->active.assign(n, 0);
    auto cleanup = [&](petto_status st, const char *msg) {
        petto_batch_destroy(b);
        (void)msg;
        return st;
    };
    if (cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming) != cudaSuccess) return cleanup(PETTO_ECUDA, "event");
    b->inst.assign(n, BatchInst{});
    if (cudaMalloc(&b->d_inst, sizeof(BatchInst) * n) != cudaSuccess ||
        cudaMalloc(&b->d_base, sizeof(long long)) != cudaSuccess ||
        cudaMalloc(&b->d_res, sizeof(double) * n) != cudaSuccess)
        return cleanup(PETTO_ENOMEM, "device memory");
    if (batch_refresh(b) != PETTO_OK) return cleanup(PETTO_ECUDA, "tiling");
    *out = b;
    return PETTO_OK;
}

void petto_batch_destroy(petto_batch *b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (auto &g : b->graphs) cudaGraphExecDestroy(g.exec);
    for (auto &pr : b->ev_pending) {
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
    }
    for (auto e : b->ev_free) cudaEventDestroy(e);
    if (b->ev) cudaEventDestroy(b->ev);
    void *bufs[] = {b->d_inst, b->d_tiles, b->d_base, b->d_res};
    for (void *p : bufs)
        if (p) cudaFree(p);
    delete b;
}

const char *petto_batch_last_error(const petto_batch *b) { return b ? b->err.c_str() : "null batch"; }

int64_t petto_batch_launch_count(const petto_batch *b) {
    if (!b) return 0;
    int64_t n = b->launches;
    for (const petto_ctx *c : b->ctx) n += c->launches;
    return n;
}

petto_status petto_batch_profile(petto_batch *b, int enable) {
    if (!b) return PETTO_EINVAL;
    b->profiling = enable != 0;
    return PETTO_OK;
}

petto_status petto_batch_profile_read(petto_batch *b, double *sweep_ms, int64_t *sweeps) {
    if (!b) return PETTO_EINVAL;
    for (size_t q = 0; q < b->ev_pending.size(); ++q) {
        auto &pr = b->ev_pending[q];
        BCK(cudaEventSynchronize(pr.second));
        float ms = 0.f;
        BCK(cudaEventElapsedTime(&ms, pr.first, pr.second));
        b->prof_ms += ms;
        b->prof_sweeps += b->ev_count[q];
        b->ev_free.push_back(pr.first);
        b->ev_free.push_back(pr.second);
    }
    b->ev_pending.clear();
    b->ev_count.clear();
    if (sweep_ms) *sweep_ms = b->prof_ms;
    if (sweeps) *sweeps = b->prof_sweeps;
    b->prof_ms = 0.0;
    b->prof_sweeps = 0;
    return PETTO_OK;
}

petto_status petto_batch_pt_solve(petto_batch *b, const petto_solve_opts *opts, petto_solve_report *reps) {
    if (!b || !opts) return bfail(b, PETTO_EINVAL, "null argument");
    const int n = (int)b->ctx.size();
    const petto_solve_opts &o0 = opts[0];
    for (int i = 0; i < n; ++i) {
        const petto_solve_opts &o = opts[i];
        if (o.mode != o0.mode || o.n_apt != o0.n_apt || o.n_pt != o0.n_pt || o.max_sweeps != o0.max_sweeps ||
            o.check_every != o0.check_every || o.local_dt != o0.local_dt || o.momentum != o0.momentum ||
            o.refine != o0.refine)
            return bfail(b, PETTO_EINVAL, "batched problems share mode, counts, check interval, step kind, momentum "
                                          "and refinement; only a, b, s1 and tol may differ");
    }
    if (o0.mode != PETTO_SOLVE_PAPER && o0.mode != PETTO_SOLVE_TOL) return bfail(b, PETTO_EINVAL, "bad mode");
    if (o0.n_apt < 0 || o0.n_pt < 0 || o0.max_sweeps < 0) return bfail(b, PETTO_EINVAL, "negative count");
    if (o0.check_every < 2 || o0.check_every % 2) return bfail(b, PETTO_EINVAL, "check_every must be even and >= 2");
    if (o0.momentum < 0 || o0.momentum > 1) return bfail(b, PETTO_EINVAL, "batches take momentum 0 or 1");
    StreamJoin join(b);
    petto_status st = batch_refresh(b);
    if (st != PETTO_OK) return st;
    const int64_t total = o0.mode == PETTO_SOLVE_PAPER ? o0.n_apt + o0.n_pt : o0.max_sweeps;
    const bool refine = o0.mode == PETTO_SOLVE_TOL && o0.refine && b->precision == PETTO_F32;
    std::vector<BatchSolve> BS(n);
    for (int i = 0; i < n; ++i) {
        petto_ctx *ctx = b->ctx[i];
        const petto_solve_opts &o = opts[i];
        ctx->cur = b->cur;
        BCK(cudaMemsetAsync(ctx->w, 0, ctx->node_bytes(), b->stream));
        st = set_ctrl(ctx, CT_RESTART_AT, 0);
        if (st != PETTO_OK) return bfail(b, st, ctx->err);
        BatchSolve &q = BS[i];
        q.S.total = total;
        const bool ref_i = refine && o.tol < 1e-3;
        q.stop = ref_i ? REFINE_FROM * ctx->f_norm : (o.mode == PETTO_SOLVE_TOL ? o.tol * ctx->f_norm : -1.0);
        q.stall = ref_i ? REFINE_STALL : 0;
        BatchInst &I = b->inst[i];
        I.kf.a = (float)o.a;
        I.kf.b = (float)o.b;
        I.kf.s1 = (float)o.s1;
        I.a = o.a;
        I.b = o.b;
        I.s1 = o.s1;
        I.rhs = nullptr;
        I.apt_until = o.mode == PETTO_SOLVE_TOL ? LLONG_MAX : o.n_apt;
        b->active[i] = total > 0 ? 1 : 0;
        if (!b->active[i]) q.phase = 2;
    }
    st = batch_upload(b);
    if (st != PETTO_OK) return st;
    const int ce = o0.check_every;
    int64_t sweeps = 0;
    std::vector<double> res(n);
    auto refine_of = [&](int i) { return refine && opts[i].tol < 1e-3; };
    while (sweeps < total) {
        bool any = false;
        for (int i = 0; i < n; ++i) any = any || b->active[i];
        if (!any) break;
        const int len = (int)std::min<int64_t>(ce, total - sweeps);
        st = batch_chunk(b, &o0, sweeps, len);
        if (st != PETTO_OK) return st;
        BCK(cudaMemcpyAsync(res.data(), b->d_res, sizeof(double) * n, cudaMemcpyDeviceToHost, b->stream));
        BCK(cudaStreamSynchronize(b->stream));
        const int64_t s0 = sweeps;
        sweeps += len;
        const bool check = sweeps % ce == 0;
        bool changed = false;
        for (int i = 0; i < n; ++i) {
            if (!b->active[i]) continue;
            petto_ctx *ctx = b->ctx[i];
            const petto_solve_opts &o = opts[i];
            BatchSolve &q = BS[i];
            BatchInst &I = b->inst[i];
            // sweeps of each kind in this chunk
            const int64_t na = std::max<int64_t>(0, std::min<int64_t>(sweeps, I.apt_until) - s0);
            q.S.na += na;
            q.S.np += len - na;
            q.S.sweeps = sweeps;
            const double rn = std::sqrt(res[i]);
            q.S.last = rn;
            bool ended = false;
            int reached = 0;
            const bool was_pt = q.S.use_pt;
            st = apply_check(ctx, &o, q.S, rn, check, q.stop, q.stall, &ended, &reached);
            if (st != PETTO_OK) return bfail(b, st, ctx->err);
            if (q.S.use_pt && !was_pt) {
                I.apt_until = 0;
                changed = true;
            }
            if (!ended && sweeps < total) continue;
            // the phase has ended
            if (!refine_of(i)) {
                q.conv = o.mode == PETTO_SOLVE_TOL && reached != 0;
                q.phase = 2;
            } else {
                st = q.phase == 0 ? refine_begin(ctx) : refine_absorb(ctx);
                if (st != PETTO_OK) return bfail(b, st, ctx->err);
                st = refine_defect(ctx, &q.true_res);
                if (st != PETTO_OK) return bfail(b, st, ctx->err);
                const double fn = ctx->f_norm;
                if (q.true_res <= o.tol * fn || sweeps >= total || !std::isfinite(q.true_res)) {
                    q.conv = q.true_res <= o.tol * fn;
                    st = refine_finish(ctx);
                    if (st != PETTO_OK) return bfail(b, st, ctx->err);
                    q.S.last = q.true_res;
                    q.phase = 2;
                } else {
                    st = refine_correction(ctx);
                    if (st != PETTO_OK) return bfail(b, st, ctx->err);
                    q.S.improve_ref = INFINITY;
                    q.S.since_improve = 0;
                    q.stop = std::max(q.true_res / 8.0, 0.5 * o.tol * fn);
                    q.stall = 20;
                    q.phase = 1;
                    I.rhs = ctx->rhs32;
                }
            }
            if (q.phase == 2) {
                b->active[i] = 0;
                I.rhs = nullptr;
            }
            changed = true;
        }
        if (changed) {
            st = batch_upload(b);
            if (st != PETTO_OK) return st;
        }
    }
    // problems still active when the budget ran out between checks (cannot happen with an
    // even check interval dividing the budget, kept for safety)
    for (int i = 0; i < n; ++i)
        if (b->active[i]) {
            b->active[i] = 0;
            BS[i].phase = 2;
        }
    bool all_conv = true, bad = false;
    for (int i = 0; i < n; ++i) {
        petto_ctx *ctx = b->ctx[i];
        BatchSolve &q = BS[i];
        const double fn = ctx->f_norm;
        if (reps) {
            petto_solve_report &r = reps[i];
            r.sweeps = q.S.sweeps;
            r.apt_sweeps = q.S.na;
            r.pt_sweeps = q.S.np;
            r.res_norm = q.S.last;
            r.f_norm = fn;
            r.rel_res = fn > 0 ? q.S.last / fn : NAN;
            r.r_pde = q.S.last / std::pow(ctx->h, ctx->dim) / (double)ctx->L.nnodes();
            r.converged = q.conv ? 1 : 0;
            r.fell_back_to_pt = q.S.fell ? 1 : 0;
        }
        if (!std::isfinite(q.S.last)) bad = true;
        if (o0.mode == PETTO_SOLVE_TOL && !q.conv) all_conv = false;
    }
    if (bad) return bfail(b, PETTO_EDIVERGED, "a residual was not finite after PT fallback");
    if (!all_conv) return PETTO_ENOTCONV;
    return PETTO_OK;
}

petto_status petto_batch_optimize(petto_batch *b, int n_steps, const petto_solve_opts *sopts,
                                  const petto_pf_opts *popts, double *metrics) {
    if (!b || !sopts || !popts || n_steps < 0) return bfail(b, PETTO_EINVAL, "bad arguments");
    const int n = (int)b->ctx.size();
    bool notconv = false;
    std::vector<petto_solve_report> reps(n);
    for (int t = 0; t < n_steps; ++t) {
        const auto t0 = std::chrono::steady_clock::now();
        petto_status st = petto_batch_pt_solve(b, sopts, reps.data());
        if (st == PETTO_ENOTCONV) notconv = true;
        else if (st != PETTO_OK) return st;
        StreamJoin join(b);
        for (int i = 0; i < n; ++i) {
            petto_ctx *ctx = b->ctx[i];
            double C = 0, W = 0, lam[MAX_PHASES] = {0};
            st = petto_sensitivity(ctx, &C, &W, nullptr, PETTO_F64, 0);
            if (st == PETTO_OK) st = petto_design_update(ctx, &popts[i], lam);
            if (st == PETTO_OK) st = petto_cahn_hilliard(ctx, &popts[i]);
            if (st != PETTO_OK) return bfail(b, st, ctx->err);
            ctx->step++;
            if (metrics) {
                double *m = metrics + ((int64_t)t * n + i) * 8;
                m[0] = (double)ctx->step;
                m[1] = C;
                m[2] = W;
                m[3] = reps[i].rel_res;
                m[4] = (double)reps[i].sweeps;
                m[5] = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
                m[6] = NAN;
                m[7] = lam[0];
            }
        }
    }
    return notconv ? PETTO_ENOTCONV : PETTO_OK;
}

// checkpoint: magic, sizes, step, then phi (storage dtype), u, w (precision, natural layout)
petto_status petto_save(petto_ctx *ctx, const char *path) {
    if (!ctx || !path) return fail(ctx, PETTO_EINVAL, "null argument");
    const int64_t nc = (int64_t)ctx->P * ctx->L.ncells();
    const int64_t nn = (int64_t)ctx->ndofc() * ctx->L.nnodes();
    const int pdt = ctx->precision == 0 ? PETTO_F32 : PETTO_F64;
    std::vector<char> phi(nc * ctx->ssize()), u(nn * ctx->tsize()), w(nn * ctx->tsize());
    petto_status st = flat_out(ctx, ctx->phi, ctx->storage, phi.data(), ctx->storage, 0, nc);
    if (st == PETTO_OK) st = node_out(ctx, ctx->u[ctx->cur], u.data(), pdt, 0);
    if (st == PETTO_OK) st = node_out(ctx, ctx->w, w.data(), pdt, 0);
    if (st != PETTO_OK) return st;
    FILE *f = std::fopen(path, "wb");
    if (!f) return fail(ctx, PETTO_EINVAL, std::string("cannot open ") + path);
    const int64_t hdr[10] = {0x6f74746570LL, 1, ctx->dim, ctx->nx, ctx->ny, ctx->nz, ctx->P, ctx->ndofc(),
                             ctx->precision * 16 + ctx->storage, ctx->step};
    bool ok = std::fwrite(hdr, sizeof(hdr), 1, f) == 1 && std::fwrite(phi.data(), 1, phi.size(), f) == phi.size() &&
              std::fwrite(u.data(), 1, u.size(), f) == u.size() && std::fwrite(w.data(), 1, w.size(), f) == w.size();
    ok = (std::fclose(f) == 0) && ok;
    return ok ? PETTO_OK : fail(ctx, PETTO_EINVAL, "write failed");
}

petto_status petto_load(petto_ctx *ctx, const char *path) {
    if (!ctx || !path) return fail(ctx, PETTO_EINVAL, "null argument");
    FILE *f = std::fopen(path, "rb");
    if (!f) return fail(ctx, PETTO_EINVAL, std::string("cannot open ") + path);
    int64_t hdr[10];
    const int64_t nc = (int64_t)ctx->P * ctx->L.ncells();
    const int64_t nn = (int64_t)ctx->ndofc() * ctx->L.nnodes();
    bool ok = std::fread(hdr, sizeof(hdr), 1, f) == 1 && hdr[0] == 0x6f74746570LL && hdr[1] == 1 &&
              hdr[2] == ctx->dim && hdr[3] == ctx->nx && hdr[4] == ctx->ny && hdr[5] == ctx->nz && hdr[6] == ctx->P &&
              hdr[7] == ctx->ndofc() && hdr[8] == ctx->precision * 16 + ctx->storage;
    std::vector<char> phi(nc * ctx->ssize()), u(nn * ctx->tsize()), w(nn * ctx->tsize());
    ok = ok && std::fread(phi.data(), 1, phi.size(), f) == phi.size() && std::fread(u.data(), 1, u.size(), f) == u.size() &&
         std::fread(w.data(), 1, w.size(), f) == w.size();
    std::fclose(f);
    if (!ok) return fail(ctx, PETTO_EINVAL, "checkpoint does not match this problem");
    const int pdt = ctx->precision == 0 ? PETTO_F32 : PETTO_F64;
    petto_status st = flat_in(ctx, phi.data(), ctx->storage, 0, ctx->phi, ctx->storage, nc);
    if (st == PETTO_OK) st = node_in(ctx, u.data(), pdt, 0, ctx->u[ctx->cur]);
    if (st == PETTO_OK) st = node_in(ctx, w.data(), pdt, 0, ctx->w);
    if (st != PETTO_OK) return st;
    ctx->step = hdr[9];
    ctx->have_sens = false;
    return refresh_material(ctx);
}

}  // extern "C"

namespace {

// The sweep-kernel variants that apply to a problem, by name: the 3D marching kernels
// (TMA two-row, TMA one-row 32x8 / 32x16, register-staged) x z-segment lengths, the 2D
// kernel running several sweeps per launch x sweeps per launch (region in nodes), the 2D
// y-marching kernel x rows per warp, and the node-gather kernel x block shapes.
std::vector<std::pair<std::string, Tiling>> kernel_candidates_all(const petto_ctx *ctx);

// the candidates a context can take: a slab of a decomposed grid only the node gather and
// the two-row marching kernel (both write a range of planes), restricted to that range
std::vector<std::pair<std::string, Tiling>> kernel_candidates(const petto_ctx *ctx) {
    std::vector<std::pair<std::string, Tiling>> all = kernel_candidates_all(ctx), cand;
    for (auto &c : all)
        if (!ctx->own_n || c.second.kind == 0 || two_row_kind(c.second.kind)) cand.push_back(c);
    return cand;
}

std::vector<std::pair<std::string, Tiling>> kernel_candidates_all(const petto_ctx *ctx) {
    std::vector<std::pair<std::string, Tiling>> cand;
    const Layout &L = ctx->L;
    if (L.dim == 3 && ctx->physics == 0 && ctx->precision == PETTO_F32) {
        Tiling t{};
        const bool tma_ok = 3 * (int64_t)ctx->nrhs * L.cstride < (int64_t(1) << 31);
        if (tma_ok) {
            for (int zs : {0, 8, 16, 32}) {
                march3d_tma2_tiling(L, t);
                if (zs) {
                    t.zs = std::min(zs, L.NZ);
                    t.gz = (L.NZ + t.zs - 1) / t.zs;
                }
                cand.emplace_back("tma2/zs" + std::to_string(t.zs), t);
                march3d_tma_tiling(L, 8, t);
                if (zs) {
                    t.zs = std::min(zs, L.NZ);
                    t.gz = (L.NZ + t.zs - 1) / t.zs;
                }
                cand.emplace_back("tma8/zs" + std::to_string(t.zs), t);
            }
            march3d_tma_tiling(L, 16, t);
            cand.emplace_back("tma16/zs" + std::to_string(t.zs), t);
            for (int zs : {0, 8, 16, 24}) {
                march3d_tma3_tiling(L, t);
                if (zs && zs != t.zs) {
                    if (zs >= L.NZ) continue;
                    t.zs = zs;
                    t.gz = (L.NZ + t.zs - 1) / t.zs;
                } else if (zs) {
                    continue;  // the default length already listed
                }
                cand.emplace_back("tma3/zs" + std::to_string(t.zs), t);
            }
        }
        if (ctx->nrhs == 1) {
            march3d_tiling(L, t);
            cand.emplace_back("v1/zs" + std::to_string(t.zs), t);
        }
        // and the node gather below (slower here, but it takes slabs of any kind)
    }
    if (L.dim == 2 && ctx->nrhs == 1)
        for (int k : {4, 2}) {
            const Tiling t = tb2d_tiling(L, ctx->physics, ctx->precision, k);
            cand.emplace_back("tb2d/k" + std::to_string(k) + "/" + std::to_string(t.ox + 2 * k) + "x" +
                                  std::to_string(t.oy + 2 * k),
                              t);
        }
    if (march2d_ok(ctx))
        for (int ly : {4, 8, 16}) {
            const Tiling t = march2d_tiling(L, ly);
            cand.emplace_back("march2d/ly" + std::to_string(t.ly), t);
        }
    for (auto bxby : {std::make_pair(32, 8), std::make_pair(64, 4), std::make_pair(128, 2), std::make_pair(16, 16),
                      std::make_pair(32, 4)}) {
        Tiling t = gather_tiling(L);
        if (L.dim == 3 && bxby.first * bxby.second > 128) continue;
        t.bx = t.ox = bxby.first;
        t.by = t.oy = bxby.second;
        t.gx = (L.NX + t.ox - 1) / t.ox;
        t.gy = (L.NY + t.oy - 1) / t.oy;
        t.gz = (L.NZ + t.zs - 1) / t.zs;
        cand.emplace_back("gather/" + std::to_string(t.bx) + "x" + std::to_string(t.by), t);
    }
    return cand;
}

}  // namespace

extern "C" {

petto_status petto_select_kernel(petto_ctx *ctx, const char *name) {
    if (!ctx || !name) return fail(ctx, PETTO_EINVAL, "null argument");
    ctx->tune_pending = false;
    const std::string want(name);
    // "tb2d/k<K>/<rx>x<ry>": the 2D kernel of K sweeps per launch on a region of rx x ry
    // nodes (rx = 32, 62, 122 or 242; output tile rx - 2K by ry - 2K, at least 4 x 4; shared
    // memory within the limit)
    int k = 0, rx = 0, ry = 0;
    if (ctx->L.dim == 2 && ctx->nrhs == 1 && std::sscanf(name, "tb2d/k%d/%dx%d", &k, &rx, &ry) == 3) {
        if ((k != 1 && k != 2 && k != 4) || !tb2d_region_ok(rx, ry, k))
            return fail(ctx, PETTO_EINVAL,
                        "tb2d: K is 1, 2 or 4, rx is 32, 62, 122 or 242 and the output tile at least 4 x 4");
        int dev = 0, opt = 0;
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&opt, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        if (tb2d_smem(rx, ry, ctx->ncomp, ctx->precision) + 1024 > (size_t)opt)
            return fail(ctx, PETTO_EINVAL, "tb2d: the region does not fit in shared memory");
        return set_tiling(ctx, tb2d_tiling(ctx->L, ctx->physics, ctx->precision, k, rx, ry));
    }
    for (auto &c : kernel_candidates(ctx)) {
        // "march2d" or "tma2" alone: the first (default-parameter) entry of that kernel
        if (c.first == want || c.first.compare(0, want.size() + 1, want + "/") == 0) return set_tiling(ctx, c.second);
    }
    return fail(ctx, PETTO_EINVAL, "no sweep kernel named " + want + " applies to this problem");
}

petto_status petto_kernel_info(petto_ctx *ctx, char *name, int name_len, int *rhs_bytes) {
    if (!ctx) return fail(ctx, PETTO_EINVAL, "null context");
    const Tiling &t = ctx->tiling;
    std::string nm = "custom";
    if (t.kind == 7)
        nm = "tb2d/k" + std::to_string(t.ly) + "/" + std::to_string(t.ox + 2 * t.ly) + "x" +
             std::to_string(t.oy + 2 * t.ly);
    else for (auto &c : kernel_candidates(ctx)) {
        const Tiling q = own_planes(ctx, c.second);
        if (q.kind == t.kind && q.bx == t.bx && q.by == t.by && q.zs == t.zs && q.ox == t.ox && q.oy == t.oy &&
            ((q.kind != 5 && q.kind != 7) || q.ly == t.ly)) {
            nm = c.first;
            break;
        }
    }
    if (name && name_len > 0) {
        std::strncpy(name, nm.c_str(), name_len - 1);
        name[name_len - 1] = 0;
    }
    // refinement sweeps of the two-row 3D marching kernel read an FP16 right-hand side
    if (rhs_bytes) *rhs_bytes = two_row_kind(t.kind) ? 2 : (ctx->precision == PETTO_F32 ? 4 : 8);
    return PETTO_OK;
}

// Time each sweep-kernel variant that applies to this problem for n sweeps from the
// current state (restored afterwards) and keep the fastest.
petto_status petto_autotune(petto_ctx *ctx, int n, char *report, int report_len) {
    if (!ctx || n < 1) return fail(ctx, PETTO_EINVAL, "bad arguments");
    ctx->tune_pending = false;
    const std::vector<std::pair<std::string, Tiling>> cand = kernel_candidates(ctx);
    // keep the state: u (current) and w
    void *su = nullptr, *sw = nullptr;
    CK(cudaMalloc(&su, ctx->node_bytes()));
    CK(cudaMalloc(&sw, ctx->node_bytes()));
    CK(cudaMemcpyAsync(su, ctx->u[ctx->cur], ctx->node_bytes(), cudaMemcpyDeviceToDevice, ctx->stream));
    CK(cudaMemcpyAsync(sw, ctx->w, ctx->node_bytes(), cudaMemcpyDeviceToDevice, ctx->stream));
    const int cur0 = ctx->cur;
    const bool prof0 = ctx->profiling;
    std::string rep = "{";
    double best = INFINITY;
    Tiling best_t = ctx->tiling;
    petto_status st = PETTO_OK;
    for (auto &c : cand) {
        st = set_tiling(ctx, c.second);
        if (st != PETTO_OK) break;
        st = petto_profile(ctx, 1);
        if (st != PETTO_OK) break;
        double ms = 0;
        int64_t cnt = 0;
        // launches of as many sweeps as the kernel runs per launch: two to warm up, then n sweeps
        const int g = sweep_group(ctx, 0, 4);
        for (int64_t t = 0; t < n + 2 * g && st == PETTO_OK; t += g) {
            if (t == 2 * g) st = petto_profile_read(ctx, &ms, &cnt, nullptr);
            if (st == PETTO_OK) st = one_sweep(ctx, 0, 0.99, 0.5, 0.5, 1, false, SweepCtl(), g);
        }
        if (st == PETTO_OK) st = petto_profile_read(ctx, &ms, &cnt, nullptr);
        if (st != PETTO_OK) break;
        const double per = ms / std::max<int64_t>(cnt, 1);
        rep += (rep.size() > 1 ? ", \"" : "\"") + c.first + "\": " + std::to_string(per);
        if (per < best) {
            best = per;
            best_t = c.second;
        }
        ctx->cur = cur0;
        CK(cudaMemcpyAsync(ctx->u[ctx->cur], su, ctx->node_bytes(), cudaMemcpyDeviceToDevice, ctx->stream));
        CK(cudaMemcpyAsync(ctx->w, sw, ctx->node_bytes(), cudaMemcpyDeviceToDevice, ctx->stream));
    }
    petto_profile(ctx, prof0 ? 1 : 0);
    if (st == PETTO_OK) st = set_tiling(ctx, best_t);
    cudaStreamSynchronize(ctx->stream);
    cudaFree(su);
    cudaFree(sw);
    rep += "}";
    if (report && report_len > 0) {
        std::strncpy(report, rep.c_str(), (size_t)report_len - 1);
        report[report_len - 1] = 0;
    }
    return st;
}

}  // extern "C"
