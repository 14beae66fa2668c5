// design.cu -- material interpolation, compliance sensitivity, design update with its
// volume multiplier, and the explicit Cahn-Hilliard step (PeTTO, arXiv 2509.06971).
//
//   material      E_c = e_min + rho^p (E0 - e_min)      (one phase, modified SIMP) or
//                 E_c = sum_i E_i rho_i^p               (P phases; Sec. 3.1 overall
//                 conductivity, Sec. 3.2 overall Young's modulus), rho = clamp(phi, 0, 1)
//   sensitivity   s_{i,c} = dC/dphi_{i,c} = -(dE_c/dphi_{i,c}) e_c, the total derivative
//                 of the self-adjoint compliance (Sec. 2.3 J_h, Sec. 3.2 J_m), with the
//                 unit-modulus cell energy e_c evaluated from the edge/face expansion of
//                 the corner-quadrature energy (see sweep.cu)
//   update        g_i = alpha_h s_i / max|s_i| + kappa_1 (sum_j phi_j - 1)  (Sec. 2.3, 3.1);
//                 projected: phi_i <- clamp(phi_i - g_i - lambda_i, 0, 1), lambda_i by
//                 bisection on [-2, 2] with FP64 sums, all on the device (no host sync);
//                 penalty:   phi_i <- phi_i - g_i - kappa_v (mean phi_i - V_i)
//   Cahn-Hilliard mu = w'(phi) - gamma_g L phi,  phi <- phi + tau L mu,  w = sin^2(pi phi)/64,
//                 L the no-flux cell Laplacian (Sec. 2.4; forward Euler in pseudo-time)
#include <algorithm>

#include "petto_internal.cuh"

namespace petto {
namespace {

__device__ __forceinline__ void cell_ijk(const Layout &L, int64_t c, int &i, int &j, int &k) {
    i = (int)(c % L.nx);
    const int64_t r = c / L.nx;
    j = (int)(r % L.ny);
    k = (int)(r / L.ny);
}

template <typename T> __device__ __forceinline__ T clamp01(T x) { return x < T(0) ? T(0) : (x > T(1) ? T(1) : x); }

template <typename T>
__device__ __forceinline__ T interp_E(const DesignArgs &d, const T (&rho)[MAX_PHASES]) {
    if (d.interp == 0) return (T)d.e_min + pow(rho[0], (T)d.penal) * ((T)d.moduli[0] - (T)d.e_min);
    T s = 0;
#pragma unroll
    for (int p = 0; p < MAX_PHASES; ++p) {
        if (p >= d.P) break;
        s += (T)d.moduli[p] * pow(rho[p], (T)d.penal);
    }
    return s;
}

// derivative of the interpolation; 0 where the clamp is flat (phi outside [0, 1])
template <typename T>
__device__ __forceinline__ T interp_dE(const DesignArgs &d, int p, T phi) {
    if (phi < T(0) || phi > T(1)) return T(0);
    const T slope = d.interp == 0 ? (T)d.moduli[0] - (T)d.e_min : (T)d.moduli[p];
    return (T)d.penal * pow(phi, (T)d.penal - T(1)) * slope;
}

template <typename T, typename S>
__global__ void material_kernel(const DesignArgs d, const S *__restrict__ phi, T *__restrict__ E) {
    const int64_t nc = d.L.ncells();
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc; c += (int64_t)gridDim.x * blockDim.x) {
        T rho[MAX_PHASES];
#pragma unroll
        for (int p = 0; p < MAX_PHASES; ++p)
            rho[p] = p < d.P ? clamp01<T>((T)Store<S>::ld(phi, (int64_t)p * nc + c)) : T(0);
        int i, j, k;
        cell_ijk(d.L, c, i, j, k);
        E[d.L.cell(i, j, k)] = interp_E<T>(d, rho);
    }
}

// unit-modulus cell energy e_c (twice the corner-quadrature strain energy per unit E);
// DIM and PHYS are compile-time so the corner table ul stays in registers
template <typename T, int DIM, int PHYS>
__device__ __forceinline__ T cell_energy(T lam, T mu, T hs, const T (&ul)[8][3]) {
    constexpr int nq = 1 << DIM;
    T edge = 0, face = 0;
    if (PHYS == 1) {
#pragma unroll
        for (int b = 0; b < DIM; ++b)
#pragma unroll
            for (int q = 0; q < nq; ++q)
                if (!((q >> b) & 1)) {
                    const T t = ul[q | (1 << b)][0] - ul[q][0];
                    edge += t * t;
                }
        return T(2) * hs * edge / (T)nq;
    }
#pragma unroll
    for (int b = 0; b < DIM; ++b)
#pragma unroll
        for (int q = 0; q < nq; ++q)
            if (!((q >> b) & 1)) {
#pragma unroll
                for (int a = 0; a < DIM; ++a) {
                    const T t = ul[q | (1 << b)][a] - ul[q][a];
                    edge += (a == b ? lam + T(2) * mu : mu) * t * t;
                }
            }
    // faces spanned by (a, b); in 3D two of each (third-axis bit t = 0, 1)
#pragma unroll
    for (int a = 0; a < DIM; ++a)
#pragma unroll
        for (int b = a + 1; b < DIM; ++b) {
            const int c = 3 - a - b;
            constexpr int nt = DIM == 3 ? 2 : 1;
#pragma unroll
            for (int t = 0; t < nt; ++t) {
                T Aa = 0, Ab = 0, Ba = 0, Bb = 0;  // sums of the two a-edges / b-edges
#pragma unroll
                for (int q = 0; q < nq; ++q) {
                    if (DIM == 3 && (((q >> c) & 1) != t)) continue;
                    if (!((q >> a) & 1)) {
                        Aa += ul[q | (1 << a)][a] - ul[q][a];
                        Ab += ul[q | (1 << a)][b] - ul[q][b];
                    }
                    if (!((q >> b) & 1)) {
                        Ba += ul[q | (1 << b)][a] - ul[q][a];
                        Bb += ul[q | (1 << b)][b] - ul[q][b];
                    }
                }
                // means are sums / 2
                face += lam * (Aa * Bb) * T(0.25) + mu * (Ab * Ba) * T(0.25);
            }
        }
    // e = 2 h^(d-2) [ edge / 2^d + face / 2^(d-2) ]
    return T(2) * hs * (edge / (T)nq + face * T(4) / (T)nq);
}

// Grid-stride over cells: s_{p,c} = -(dE/dphi_p) e_c and C = sum_c E_c e_c.  Per-thread
// sums and maxima stay in T; one FP64 block sum per thread at the end (deterministic order).
template <typename T, typename S, int DIM, int PHYS>
__global__ void __launch_bounds__(256) sensitivity_kernel(const SensArgs sa, const DesignArgs d,
                                                          const T *__restrict__ u, const T *__restrict__ E,
                                                          const S *__restrict__ phi, T *__restrict__ s,
                                                          double *scal, const RedBuf rb) {
    __shared__ double sh[32];
    const Layout &L = sa.L;
    constexpr int ncomp = PHYS == 1 ? 1 : DIM;
    const int64_t nc = L.ncells();
    const T lam = (T)sa.lam, mu = (T)sa.mu, hs = (T)(DIM == 3 ? sa.h : 1.0);
    T comp = 0;
    T smax[MAX_PHASES];
#pragma unroll
    for (int p = 0; p < MAX_PHASES; ++p) smax[p] = 0;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc; c += (int64_t)gridDim.x * blockDim.x) {
        int i, j, k;
        cell_ijk(L, c, i, j, k);
        const int64_t n0 = L.node(i, j, DIM == 3 ? k : 0);
        T e = 0;
        for (int r = 0; r < sa.nrhs; ++r) {
            T ul[8][3];
            const T *ur = u + (int64_t)r * ncomp * L.cstride + n0;
#pragma unroll
            for (int q = 0; q < (1 << DIM); ++q) {
                const int64_t o = (q & 1) + ((q >> 1) & 1) * L.SX + (DIM == 3 ? ((q >> 2) & 1) * L.SX * L.SY : 0);
#pragma unroll
                for (int a = 0; a < ncomp; ++a) ul[q][a] = ur[(int64_t)a * L.cstride + o];
            }
            e += cell_energy<T, DIM, PHYS>(lam, mu, hs, ul);
        }
        const T Ec = E[L.cell(i, j, k)];
        if (k >= sa.zc0 && k < sa.zc1) comp += Ec * e;  // a slab counts its own cell layers
#pragma unroll
        for (int p = 0; p < MAX_PHASES; ++p) {
            if (p >= d.P) break;
            const T ph = (T)Store<S>::ld(phi, (int64_t)p * nc + c);
            const T sv = -interp_dE<T>(d, p, ph) * e;
            s[(int64_t)p * nc + c] = sv;
            smax[p] = fmax(smax[p], sv < T(0) ? -sv : sv);
        }
    }
#pragma unroll
    for (int p = 0; p < MAX_PHASES; ++p) {
        if (p >= d.P) break;
        const T m = warp_max(smax[p]);
        if ((threadIdx.x & 31) == 0 && m > T(0)) atomic_max_nonneg(&scal[SC_SMAX + p], (double)m);
    }
    const double tot = block_sum((double)comp, sh);
    if (publish_partial(tot, rb, blockIdx.x, gridDim.x)) {
        const double t = sum_partials(rb, 0, gridDim.x, sh);
        if (threadIdx.x == 0) {
            scal[SC_C] = t;
            *rb.counter = 0u;
        }
    }
}

template <typename T>
__global__ void work_kernel(const Layout L, int ncomp, int nrhs, const LoadEntry *__restrict__ loads, int n_loads,
                            const T *__restrict__ u, double src, double *scal, const RedBuf rb) {
    __shared__ double sh[32];
    double acc = 0.0;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t l = tid; l < n_loads; l += stride) acc += loads[l].vald * (double)u[(int64_t)loads[l].comp * L.cstride + loads[l].node];
    if (src != 0.0) {
        const int64_t nn = L.nnodes();
        for (int64_t n = tid; n < nn; n += stride) {
            const int i = (int)(n % L.NX);
            const int64_t r = n / L.NX;
            const int j = (int)(r % L.NY), k = (int)(r / L.NY);
            const int cnt = ((i > 0) + (i < L.nx)) * ((j > 0) + (j < L.ny)) * (L.dim == 3 ? ((k > 0) + (k < L.nz)) : 1);
            for (int rr = 0; rr < nrhs; ++rr) acc += src * cnt * (double)u[(int64_t)(rr * ncomp) * L.cstride + L.node(i, j, k)];
        }
    }
    const double t = block_sum(acc, sh);
    if (publish_partial(t, rb, blockIdx.x, gridDim.x)) {
        const double tt = sum_partials(rb, 0, gridDim.x, sh);
        if (threadIdx.x == 0) {
            scal[SC_W] = tt;
            *rb.counter = 0u;
        }
    }
}

// -------------------------------------------------------------- design update

template <typename T, typename S>
__global__ void upd_prepare(const UpdateArgs ua, S *__restrict__ phi, const T *__restrict__ s, T *__restrict__ dbuf,
                            const double *__restrict__ scal) {
    const int64_t nc = ua.ncell;
    // per-phase factors hoisted out of the cell loop (phase loops unrolled: registers, not stack)
    T scale[MAX_PHASES], shift[MAX_PHASES];
#pragma unroll
    for (int p = 0; p < MAX_PHASES; ++p) {
        scale[p] = 0;
        shift[p] = 0;
        if (p < ua.P) {
            const double smax = scal[SC_SMAX + p];
            scale[p] = smax > 0.0 ? (T)(ua.alpha_h / smax) : T(0);
            shift[p] = (T)(ua.kappa_v * (scal[SC_MEAN + p] - ua.V[p]));
        }
    }
    const T k1 = (T)ua.kappa_1;
    // keep-out term (Sec. 3.4 J_b): kappa_b (mean over the region of phi_i - Vb_i) on its cells
    T kb[MAX_PHASES];
#pragma unroll
    for (int p = 0; p < MAX_PHASES; ++p)
        kb[p] = ua.keep && p < ua.P ? (T)(ua.kappa_b * (scal[SC_BMEAN + p] - ua.Vb[p])) : T(0);
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc; c += (int64_t)gridDim.x * blockDim.x) {
        bool inb = false;
        if (ua.keep) {
            const int i = (int)(c % ua.nx);
            const int64_t r = c / ua.nx;
            const int j = (int)(r % ua.ny), k = (int)(r / ua.ny);
            inb = i >= ua.klo[0] && i <= ua.khi[0] && j >= ua.klo[1] && j <= ua.khi[1] && k >= ua.klo[2] &&
                  k <= ua.khi[2];
        }
        T tot = 0;
        T ph[MAX_PHASES];
#pragma unroll
        for (int p = 0; p < MAX_PHASES; ++p) {
            ph[p] = 0;
            if (p < ua.P) {
                ph[p] = (T)Store<S>::ld(phi, (int64_t)p * nc + c);
                tot += ph[p];
            }
        }
#pragma unroll
        for (int p = 0; p < MAX_PHASES; ++p) {
            if (p >= ua.P) break;
            T g = scale[p] * s[(int64_t)p * nc + c] + k1 * (tot - T(1));
            if (inb) g += kb[p];
            const T dv = ph[p] - g;
            if (ua.vol_mode == 0) dbuf[(int64_t)p * nc + c] = dv;
            else Store<S>::st(phi, (int64_t)p * nc + c, dv - shift[p]);
        }
    }
}

__global__ void bis_init(int P, double *scal) {
    const int p = threadIdx.x;
    if (p < P) {
        scal[SC_LO + p] = -2.0;
        scal[SC_HI + p] = 2.0;
    }
}

// One bisection halving for every phase: grid (blocks, P).  Each block publishes its
// partial sum of clamp(d - mid, 0, 1); the last block sums each phase's partials in block
// order and moves that phase's bracket.
template <typename T>
__global__ void __launch_bounds__(256) bis_step(const UpdateArgs ua, const T *__restrict__ dbuf, double *scal,
                                                const RedBuf rb) {
    __shared__ double sh[32];
    const int p = blockIdx.y;
    const int64_t nc = ua.ncell;
    // element arithmetic in T (FP32 for the FP32 path: the FP64 pipe is narrow), FP64 block sums
    const T mid = (T)(0.5 * (scal[SC_LO + p] + scal[SC_HI + p]));
    T acc = 0;
    // ext: a slab of a decomposed grid sums its own cell layers only and leaves the
    // bracket to the host, which adds the slabs' sums
    const int64_t c0 = ua.ext ? (int64_t)ua.zc0 * ua.layer : 0, c1 = ua.ext ? (int64_t)ua.zc1 * ua.layer : nc;
    for (int64_t c = c0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < c1; c += (int64_t)gridDim.x * blockDim.x)
        acc += clamp01<T>(dbuf[(int64_t)p * nc + c] - mid);
    const double t = block_sum((double)acc, sh);
    if (publish_partial(t, rb, (int64_t)p * gridDim.x + blockIdx.x, gridDim.x * gridDim.y)) {
#pragma unroll
        for (int q = 0; q < MAX_PHASES; ++q) {
            if (q >= ua.P) break;
            const double sq = sum_partials(rb, (int64_t)q * gridDim.x, gridDim.x, sh);
            if (ua.ext) {
                if (threadIdx.x == 0) scal[SC_SUM + q] = sq;
                continue;
            }
            const double m = sq / (double)nc;
            if (threadIdx.x == 0) {
                volatile double *vs = scal;
                const double md = 0.5 * (vs[SC_LO + q] + vs[SC_HI + q]);
                if (m > ua.V[q]) vs[SC_LO + q] = md;
                else vs[SC_HI + q] = md;
            }
        }
        if (threadIdx.x == 0) *rb.counter = 0u;
    }
}

template <typename T, typename S>
__global__ void upd_apply(const UpdateArgs ua, S *__restrict__ phi, const T *__restrict__ dbuf, double *scal) {
    const int p = blockIdx.y;
    const int64_t nc = ua.ncell;
    const double lam = 0.5 * (scal[SC_LO + p] + scal[SC_HI + p]);
    if (blockIdx.x == 0 && threadIdx.x == 0) scal[SC_LAM + p] = lam;
    const T lamT = (T)lam;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc; c += (int64_t)gridDim.x * blockDim.x)
        Store<S>::st(phi, (int64_t)p * nc + c, clamp01<T>(dbuf[(int64_t)p * nc + c] - lamT));
}

// -------------------------------------------------------------- Cahn-Hilliard

// hi: the cell layer above the grid's top layer (a slab's neighbour), or null for the no-flux
// boundary there
template <typename T, typename S>
__device__ __forceinline__ T lap_at(const Layout &L, const S *v, int64_t c, int i, int j, int k, const S *hi) {
    const T x = (T)Store<S>::ld(v, c);
    T s = 0;
    if (i > 0) s += (T)Store<S>::ld(v, c - 1) - x;
    if (i < L.nx - 1) s += (T)Store<S>::ld(v, c + 1) - x;
    if (j > 0) s += (T)Store<S>::ld(v, c - L.nx) - x;
    if (j < L.ny - 1) s += (T)Store<S>::ld(v, c + L.nx) - x;
    if (L.dim == 3) {
        const int64_t pl = (int64_t)L.nx * L.ny;
        if (k > 0) s += (T)Store<S>::ld(v, c - pl) - x;
        if (k < L.nz - 1) s += (T)Store<S>::ld(v, c + pl) - x;
        else if (hi) s += (T)Store<S>::ld(hi, c - (int64_t)k * pl) - x;
    }
    return s;
}

__device__ __forceinline__ float dwell(float x) { return sinpif(2.0f * x) * (float)(3.14159265358979323846 / 64.0); }
__device__ __forceinline__ double dwell(double x) { return sinpi(2.0 * x) * (3.14159265358979323846 / 64.0); }

template <typename T, typename S>
__global__ void ch_mu(const Layout L, const S *__restrict__ phi, T *__restrict__ mu, double gamma_g,
                      const S *__restrict__ phi_hi) {
    const int64_t nc = L.ncells();
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc; c += (int64_t)gridDim.x * blockDim.x) {
        int i, j, k;
        cell_ijk(L, c, i, j, k);
        const T ph = (T)Store<S>::ld(phi, c);
        mu[c] = dwell(ph) - (T)gamma_g * lap_at<T, S>(L, phi, c, i, j, k, phi_hi);
    }
}

template <typename T, typename S>
__global__ void ch_phi(const Layout L, S *__restrict__ phi, const T *__restrict__ mu, double tau,
                       const T *__restrict__ mu_hi) {
    const int64_t nc = L.ncells();
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc; c += (int64_t)gridDim.x * blockDim.x) {
        int i, j, k;
        cell_ijk(L, c, i, j, k);
        const T nv = (T)Store<S>::ld(phi, c) + (T)tau * lap_at<T, T>(L, mu, c, i, j, k, mu_hi);
        Store<S>::st(phi, c, nv);
    }
}

// scal[slot + p] = (sum of phase p over cells c0 .. c1 - 1) / div, in FP64 with the
// deterministic reduction
template <typename S>
__global__ void mean_kernel(int64_t nc, int P, const S *__restrict__ phi, double *scal, const RedBuf rb, int64_t c0,
                            int64_t c1, double div, int slot) {
    __shared__ double sh[32];
    const int p = blockIdx.y;
    double acc = 0.0;
    for (int64_t c = c0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < c1; c += (int64_t)gridDim.x * blockDim.x)
        acc += (double)Store<S>::ld(phi, (int64_t)p * nc + c);
    const double t = block_sum(acc, sh);
    if (publish_partial(t, rb, (int64_t)p * gridDim.x + blockIdx.x, gridDim.x * gridDim.y)) {
        for (int q = 0; q < P; ++q) {
            const double m = sum_partials(rb, (int64_t)q * gridDim.x, gridDim.x, sh);
            if (threadIdx.x == 0) scal[slot + q] = m / div;
        }
        if (threadIdx.x == 0) *rb.counter = 0u;
    }
}

// mean of each phase over the keep-out cells, in FP64 with the deterministic reduction
template <typename S>
__global__ void box_mean_kernel(const UpdateArgs ua, const S *__restrict__ phi, double *scal, const RedBuf rb) {
    __shared__ double sh[32];
    const int p = blockIdx.y;
    const int bx = ua.khi[0] - ua.klo[0] + 1, by = ua.khi[1] - ua.klo[1] + 1, bz = ua.khi[2] - ua.klo[2] + 1;
    const int64_t nb = (int64_t)bx * by * bz;
    double acc = 0.0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nb; t += (int64_t)gridDim.x * blockDim.x) {
        const int i = ua.klo[0] + (int)(t % bx);
        const int64_t r = t / bx;
        const int j = ua.klo[1] + (int)(r % by), k = ua.klo[2] + (int)(r / by);
        const int64_t c = (int64_t)i + (int64_t)ua.nx * ((int64_t)j + (int64_t)ua.ny * k);
        acc += (double)Store<S>::ld(phi, (int64_t)p * ua.ncell + c);
    }
    const double tot = block_sum(acc, sh);
    if (publish_partial(tot, rb, (int64_t)p * gridDim.x + blockIdx.x, gridDim.x * gridDim.y)) {
#pragma unroll
        for (int q = 0; q < MAX_PHASES; ++q) {
            if (q >= ua.P) break;
            const double m = sum_partials(rb, (int64_t)q * gridDim.x, gridDim.x, sh);
            if (threadIdx.x == 0) scal[SC_BMEAN + q] = m / (double)nb;
        }
        if (threadIdx.x == 0) *rb.counter = 0u;
    }
}

int grid_for(int64_t n, int block, int cap = 152 * 16) {
    int64_t g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

}  // namespace

// ---------------------------------------------------------------- dispatch helpers

#define PETTO_DISPATCH_STORAGE(storage, SVAR, ...)                      \
    switch (storage) {                                                  \
        case 0: { using SVAR = float; __VA_ARGS__; } break;             \
        case 1: { using SVAR = double; __VA_ARGS__; } break;            \
        case 2: { using SVAR = __nv_bfloat16; __VA_ARGS__; } break;     \
        case 3: { using SVAR = __half; __VA_ARGS__; } break;            \
        default: return cudaErrorInvalidValue;                          \
    }

#define PETTO_DISPATCH_PREC(prec, TVAR, ...)                            \
    if ((prec) == 0) { using TVAR = float; __VA_ARGS__; }               \
    else { using TVAR = double; __VA_ARGS__; }

cudaError_t launch_material(const DesignArgs &d, const void *phi, void *E, cudaStream_t s) {
    const int g = grid_for(d.L.ncells(), 256);
    PETTO_DISPATCH_PREC(d.precision, T,
        PETTO_DISPATCH_STORAGE(d.storage, S,
            material_kernel<T, S><<<g, 256, 0, s>>>(d, static_cast<const S *>(phi), static_cast<T *>(E))))
    return cudaGetLastError();
}

int64_t reduction_capacity(const Layout &L, int ntiles, int P) {
    int64_t c = ntiles;
    c = std::max<int64_t>(c, (L.ncells() + 255) / 256);
    c = std::max<int64_t>(c, (int64_t)152 * 4 * P);
    c = std::max<int64_t>(c, (int64_t)152 * 16);
    return 2 * c + 64;
}

cudaError_t launch_sensitivity(const SensArgs &sa, const DesignArgs &d, const void *u, const void *E,
                               const void *phi, void *sbuf, double *scal, RedBuf rb, cudaStream_t st) {
    const int64_t nc = sa.L.ncells();
    const int g = grid_for(nc, 256, 152 * 8);
#define PETTO_SENS(DIM, PHYS)                                                                                       \
    PETTO_DISPATCH_PREC(d.precision, T,                                                                             \
        PETTO_DISPATCH_STORAGE(d.storage, S,                                                                        \
            sensitivity_kernel<T, S, DIM, PHYS><<<g, 256, 0, st>>>(sa, d, static_cast<const T *>(u),                \
                                                                  static_cast<const T *>(E),                        \
                                                                  static_cast<const S *>(phi),                      \
                                                                  static_cast<T *>(sbuf), scal, rb)))
    if (sa.L.dim == 3) {
        if (sa.physics == 1) PETTO_SENS(3, 1) else PETTO_SENS(3, 0)
    } else {
        if (sa.physics == 1) PETTO_SENS(2, 1) else PETTO_SENS(2, 0)
    }
#undef PETTO_SENS
    return cudaGetLastError();
}

cudaError_t launch_work(const Layout &L, int ncomp, int nrhs, int precision, const LoadEntry *loads, int n_loads,
                        const void *u, double body_src, double *scal, RedBuf rb, cudaStream_t st) {
    const int g = body_src != 0.0 ? grid_for(L.nnodes(), 256) : 1;
    PETTO_DISPATCH_PREC(precision, T,
        work_kernel<T><<<g, 256, 0, st>>>(L, ncomp, nrhs, loads, n_loads, static_cast<const T *>(u), body_src, scal, rb))
    return cudaGetLastError();
}

// The phase sums take eight cells per thread before the block sum: on small grids fewer
// blocks publish partials (a 65 K-cell grid of six phases: 192 blocks instead of 1 536).
cudaError_t launch_mean(const Layout &L, int P, int storage, const void *phi, double *scal, RedBuf rb,
                        cudaStream_t st) {
    const int64_t nc = L.ncells();
    dim3 grid(grid_for(nc, 256 * 8, 152 * 4), P);
    PETTO_DISPATCH_STORAGE(storage, S,
        mean_kernel<S><<<grid, 256, 0, st>>>(nc, P, static_cast<const S *>(phi), scal, rb, 0, nc, (double)nc,
                                             SC_MEAN))
    return cudaGetLastError();
}

cudaError_t launch_layer_sums(const Layout &L, int P, int storage, const void *phi, int zc0, int zc1, double *scal,
                              int slot, RedBuf rb, cudaStream_t st) {
    const int64_t nc = L.ncells(), pl = (int64_t)L.nx * L.ny;
    dim3 grid(grid_for(nc, 256 * 8, 152 * 4), P);
    PETTO_DISPATCH_STORAGE(storage, S,
        mean_kernel<S><<<grid, 256, 0, st>>>(nc, P, static_cast<const S *>(phi), scal, rb, (int64_t)zc0 * pl,
                                             (int64_t)zc1 * pl, 1.0, slot))
    return cudaGetLastError();
}

cudaError_t launch_bisect_sums(const UpdateArgs &ua, const void *dscratch, double *scal, RedBuf rb, cudaStream_t st) {
    dim3 grid(grid_for(ua.ncell, 256, 152 * 4), ua.P);
    PETTO_DISPATCH_PREC(ua.precision, T, bis_step<T><<<grid, 256, 0, st>>>(ua, static_cast<const T *>(dscratch), scal, rb))
    return cudaGetLastError();
}

cudaError_t launch_update_apply(const UpdateArgs &ua, void *phi, const void *dscratch, double *scal, cudaStream_t st) {
    dim3 grid2(grid_for(ua.ncell, 256), ua.P);
    PETTO_DISPATCH_PREC(ua.precision, T,
        PETTO_DISPATCH_STORAGE(ua.storage, S,
            upd_apply<T, S><<<grid2, 256, 0, st>>>(ua, static_cast<S *>(phi), static_cast<const T *>(dscratch), scal)))
    return cudaGetLastError();
}

cudaError_t launch_update(const UpdateArgs &ua, void *phi, const void *s, void *dscratch, double *scal,
                          RedBuf rb, cudaStream_t st, int64_t *launches) {
    const int g = grid_for(ua.ncell, 256);
    if (ua.keep) {
        const int64_t nb = (int64_t)(ua.khi[0] - ua.klo[0] + 1) * (ua.khi[1] - ua.klo[1] + 1) *
                           (ua.khi[2] - ua.klo[2] + 1);
        dim3 gb(grid_for(nb, 256, 152 * 4), ua.P);
        PETTO_DISPATCH_STORAGE(ua.storage, S,
            box_mean_kernel<S><<<gb, 256, 0, st>>>(ua, static_cast<const S *>(phi), scal, rb))
        *launches += 1;
    }
    PETTO_DISPATCH_PREC(ua.precision, T,
        PETTO_DISPATCH_STORAGE(ua.storage, S,
            upd_prepare<T, S><<<g, 256, 0, st>>>(ua, static_cast<S *>(phi), static_cast<const T *>(s),
                                                 static_cast<T *>(dscratch), scal)))
    *launches += 1;
    if (ua.vol_mode != 0 || ua.ext) return cudaGetLastError();  // ext: the host runs the bisection
    bis_init<<<1, 32, 0, st>>>(ua.P, scal);
    *launches += 1;
    dim3 grid(grid_for(ua.ncell, 256, 152 * 4), ua.P);
    for (int it = 0; it < ua.n_bisect; ++it) {
        PETTO_DISPATCH_PREC(ua.precision, T,
            bis_step<T><<<grid, 256, 0, st>>>(ua, static_cast<const T *>(dscratch), scal, rb))
        *launches += 1;
    }
    dim3 grid2(g, ua.P);
    PETTO_DISPATCH_PREC(ua.precision, T,
        PETTO_DISPATCH_STORAGE(ua.storage, S,
            upd_apply<T, S><<<grid2, 256, 0, st>>>(ua, static_cast<S *>(phi), static_cast<const T *>(dscratch), scal)))
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_ch(const Layout &L, int P, int storage, int precision, double gamma_g, double tau, void *phi,
                      void *mu_scratch, cudaStream_t st, int64_t *launches) {
    const int64_t nc = L.ncells();
    const int g = grid_for(nc, 256);
    for (int p = 0; p < P; ++p) {
        PETTO_DISPATCH_PREC(precision, T,
            PETTO_DISPATCH_STORAGE(storage, S,
                S *ph = static_cast<S *>(phi) + (int64_t)p * nc;
                ch_mu<T, S><<<g, 256, 0, st>>>(L, ph, static_cast<T *>(mu_scratch), gamma_g, nullptr);
                ch_phi<T, S><<<g, 256, 0, st>>>(L, ph, static_cast<const T *>(mu_scratch), tau, nullptr)))
        *launches += 2;
    }
    return cudaGetLastError();
}

cudaError_t launch_ch_half(const Layout &L, int p, int half, int storage, int precision, double gamma_g, double tau,
                           void *phi, void *mu_scratch, const void *phi_hi, const void *mu_hi, cudaStream_t st) {
    const int64_t nc = L.ncells(), pl = (int64_t)L.nx * L.ny;
    const int g = grid_for(nc, 256);
    PETTO_DISPATCH_PREC(precision, T,
        PETTO_DISPATCH_STORAGE(storage, S,
            S *ph = static_cast<S *>(phi) + (int64_t)p * nc;
            const S *phh = phi_hi ? static_cast<const S *>(phi_hi) + (int64_t)p * pl : nullptr;
            if (half == 0) ch_mu<T, S><<<g, 256, 0, st>>>(L, ph, static_cast<T *>(mu_scratch), gamma_g, phh);
            else ch_phi<T, S><<<g, 256, 0, st>>>(L, ph, static_cast<const T *>(mu_scratch), tau,
                                                  static_cast<const T *>(mu_hi))))
    return cudaGetLastError();
}

}  // namespace petto
