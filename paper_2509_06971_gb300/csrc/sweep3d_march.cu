// sweep3d_march.cu -- z-marching fused APT/PT sweep for 3D elasticity in FP32, the hot
// kernel of the 3D workloads (Sec. 3.3 of the paper solves the 3D cantilever with this
// iteration; Sec. 3.2 gives the PT/APT systems).
//
// Same operator as sweep.cu (edge terms + face terms of the corner-quadrature energy),
// organised so that every edge and every face is evaluated once:
//   * a thread block owns a tile of TX x TY node columns and marches them in z over a
//     segment of ZS node planes;
//   * the thread of node n owns the three edges n->n+x, n->n+y, n->n+z and the three faces
//     with lower corner n.  It computes their forces once and sends the shares of other
//     nodes as three combined messages: to n+x (via shared memory), to n+y (shared memory),
//     to n+z (itself, next plane) and one diagonal share to n+x+y;
//   * the tile overlaps its neighbours by one owner column/row on the low side, so every
//     output node receives all of its messages inside the block (31 x (TY-1) outputs);
//   * u planes and modulus layers pass through a two-plane shared-memory ring; the global
//     loads of plane z+2 are issued into registers while plane z is computed.
// Per output node and sweep the kernel reads u, w and E once from HBM and writes u', w'
// once (52 B in FP32, the algorithmic minimum); halo re-reads hit L2.
#include "petto_internal.cuh"

namespace petto {
namespace {

constexpr int MX = 32;           // threads (owner columns) per tile row
constexpr int MTY = 8;           // owner rows per tile
constexpr int MZS = 16;          // output planes per z segment
constexpr int MWX = MX + 1;      // tile width in nodes / cells
constexpr int MWY = MTY + 1;     // tile height
constexpr int MNT = MX * MTY;    // threads per block
constexpr int MENT = MWX * MWY;  // tile entries per plane

struct Staged {
    float u[2][3];
    float e[2];
    bool v[2];
};

__device__ __forceinline__ void stage_plane(const Layout &L, const float *__restrict__ u, const float *__restrict__ E,
                                            int x0, int y0, int p, int tid, Staged &s) {
    // u plane p (nodes x0-1 .. x0+31, y0-1 .. y0+TY-1) and E layer p-1 (cells x0-2.., y0-2..)
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int e = tid + r * MNT;
        s.v[r] = e < MENT;
        const int ex = e % MWX, ey = e / MWX;
        const int x = x0 - 1 + ex, y = y0 - 1 + ey;
        const bool okn = s.v[r] && x <= L.NX && y <= L.NY && p >= 0 && p < L.NZ;
        const int64_t n = L.node(min(x, L.NX), min(y, L.NY), p);
#pragma unroll
        for (int c = 0; c < 3; ++c) s.u[r][c] = okn ? __ldg(&u[(int64_t)c * L.cstride + n]) : 0.f;
        const int cx = x - 1, cy = y - 1, l = p - 1;
        const bool oke = s.v[r] && cx >= -1 && cx <= L.nx && cy >= -1 && cy <= L.ny && l >= 0 && l < L.nz;
        s.e[r] = oke ? __ldg(&E[L.cell(max(cx, -1), max(cy, -1), max(l, 0))]) : 0.f;
    }
}

__global__ void __launch_bounds__(MNT, 3) sweep3d_march_f32(const SweepArgs A) {
    __shared__ float su[2][3][MWY][MWX];
    __shared__ float se[2][MWY][MWX];
    __shared__ float4 ma[2][MTY][MX];
    __shared__ float4 mb[2][MTY][MX];
    __shared__ double shred[32];

    const Layout &L = A.L;
    const float *__restrict__ ui = static_cast<const float *>(A.u_in);
    float *__restrict__ uo = static_cast<float *>(A.u_out);
    float *__restrict__ w = static_cast<float *>(A.w);
    const float *__restrict__ E = static_cast<const float *>(A.E);

    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * MX + tx;
    const int x0 = blockIdx.x * (MX - 1), y0 = blockIdx.y * (MTY - 1), z0 = blockIdx.z * MZS;
    const int X = x0 - 1 + tx, Y = y0 - 1 + ty;
    const bool outxy = tx >= 1 && ty >= 1 && X < L.NX && Y < L.NY;
    const int zend = min(z0 + MZS, L.NZ);

    const float cpar = (float)A.k.ce_par, cperp = (float)A.k.ce_perp;
    const float cl = (float)A.k.cf_lam, cm = (float)A.k.cf_mu, cdg = (float)A.k.cdiag;
    float fa = (float)A.a;
    const float fb = (float)A.b, fs1 = (float)A.s1;
    if (A.adaptive) {
        const long long k = A.sweep_idx - (long long)A.ctrl[CT_RESTART_AT];
        const float sched = k <= 0 ? 0.f : (float)(k - 1) / (float)(k + 2);
        fa = fminf(fa, sched);
    }
    const float *__restrict__ rhs = static_cast<const float *>(A.rhs);

    // supports: boxes that contain this (X, Y) column
    unsigned boxbits = 0;
    for (int q = 0; q < A.boxes.n; ++q) {
        const Box &b = A.boxes.b[q];
        if (X >= b.lo[0] && X <= b.hi[0] && Y >= b.lo[1] && Y <= b.hi[1]) boxbits |= 1u << q;
    }
    const int tile = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    const int l0 = A.tile_ptr[tile], l1 = A.tile_ptr[tile + 1];

    // prologue: planes z0-1 (into the ring) and z0 (staged in registers)
    Staged st;
    stage_plane(L, ui, E, x0, y0, z0 - 1, tid, st);
#pragma unroll
    for (int r = 0; r < 2; ++r)
        if (st.v[r]) {
            const int e = tid + r * MNT, ex = e % MWX, ey = e / MWX;
#pragma unroll
            for (int c = 0; c < 3; ++c) su[(z0 - 1) & 1][c][ey][ex] = st.u[r][c];
            se[(z0 - 1) & 1][ey][ex] = st.e[r];
        }
    stage_plane(L, ui, E, x0, y0, z0, tid, st);
    __syncthreads();

    float U0[4][3], E0[4];
    {
        const int s = (z0 - 1) & 1;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            U0[0][c] = su[s][c][ty][tx];
            U0[1][c] = su[s][c][ty][tx + 1];
            U0[2][c] = su[s][c][ty + 1][tx];
            U0[3][c] = su[s][c][ty + 1][tx + 1];
        }
        // E layer z0-2: the ring holds layer p-1 for plane p, i.e. layer z0-2 here
        E0[0] = se[s][ty + 1][tx + 1];  // c(n)
        E0[1] = se[s][ty + 1][tx];      // c(n-x)
        E0[2] = se[s][ty][tx + 1];      // c(n-y)
        E0[3] = se[s][ty][tx];          // c(n-x-y)
    }
    float Szp[3] = {0.f, 0.f, 0.f}, Gxzp[2] = {0.f, 0.f}, Gyzp[2] = {0.f, 0.f};
    float res = 0.f, dot = 0.f;

    for (int zp = z0 - 1; zp < zend; ++zp) {
        // ring slot of plane zp+1 (and E layer zp): write the staged data, then stage zp+2
        const int s1 = (zp + 1) & 1;
#pragma unroll
        for (int r = 0; r < 2; ++r)
            if (st.v[r]) {
                const int e = tid + r * MNT, ex = e % MWX, ey = e / MWX;
#pragma unroll
                for (int c = 0; c < 3; ++c) su[s1][c][ey][ex] = st.u[r][c];
                se[s1][ey][ex] = st.e[r];
            }
        // own w (for the update of plane zp) -- loaded before the barrier to hide latency
        float wv[3] = {0.f, 0.f, 0.f};
        const bool outp = outxy && zp >= z0;
        const int64_t nidx = outp ? L.node(X, Y, zp) : 0;
        if (outp && A.mode == 0) {
#pragma unroll
            for (int c = 0; c < 3; ++c) wv[c] = w[(int64_t)c * L.cstride + nidx];
        }
        float uown[3] = {0.f, 0.f, 0.f};
        if (zp + 2 <= zend) stage_plane(L, ui, E, x0, y0, zp + 2, tid, st);
        __syncthreads();

        float U1[3][3], E1[4];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            U1[0][c] = su[s1][c][ty][tx];
            U1[1][c] = su[s1][c][ty][tx + 1];
            U1[2][c] = su[s1][c][ty + 1][tx];
        }
        E1[0] = se[s1][ty + 1][tx + 1];
        E1[1] = se[s1][ty + 1][tx];
        E1[2] = se[s1][ty][tx + 1];
        E1[3] = se[s1][ty][tx];
#pragma unroll
        for (int c = 0; c < 3; ++c) uown[c] = U0[0][c];

        // ---- owned edges
        const float Ex = E1[0] + E1[2] + E0[0] + E0[2];   // x-edge: cells (X, Y-1..Y, zp-1..zp)
        const float Ey = E1[0] + E1[1] + E0[0] + E0[1];   // y-edge: cells (X-1..X, Y, zp-1..zp)
        const float Ez = E1[0] + E1[1] + E1[2] + E1[3];   // z-edge: cells (X-1..X, Y-1..Y, zp)
        float ax[3], ay[3], az[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            ax[c] = U0[1][c] - U0[0][c];
            ay[c] = U0[2][c] - U0[0][c];
            az[c] = U1[0][c] - U0[0][c];
        }
        const float exp_ = Ex * cpar, exq = Ex * cperp, eyp = Ey * cpar, eyq = Ey * cperp, ezp = Ez * cpar,
                    ezq = Ez * cperp;
        const float Fx[3] = {exp_ * ax[0], exq * ax[1], exq * ax[2]};
        const float Fy[3] = {eyq * ay[0], eyp * ay[1], eyq * ay[2]};
        const float Fz[3] = {ezq * az[0], ezq * az[1], ezp * az[2]};

        // ---- owned faces: G (to the far corner) and H (to the a-neighbour corner)
        // xy face (a = x, b = y) at plane zp: cells (X, Y, zp-1..zp)
        float Gxy[2], Hxy[2];
        {
            const float Et = E1[0] + E0[0];
            const float SAx = ax[0] + (U0[3][0] - U0[2][0]), SAy = ax[1] + (U0[3][1] - U0[2][1]);
            const float SBx = ay[0] + (U0[3][0] - U0[1][0]), SBy = ay[1] + (U0[3][1] - U0[1][1]);
            const float el = Et * cl, em = Et * cm;
            const float p = em * SAy, q = el * SAx;
            Gxy[0] = fmaf(el, SBy, p);
            Hxy[0] = fmaf(el, SBy, -p);
            Gxy[1] = fmaf(em, SBx, q);
            Hxy[1] = fmaf(em, SBx, -q);
        }
        // xz face (a = x, b = z) in the plane y = Y: cells (X, Y-1..Y, zp)
        float Gxz[2], Hxz[2];  // components (x, z)
        {
            const float Et = E1[0] + E1[2];
            const float SAx = ax[0] + (U1[1][0] - U1[0][0]), SAz = ax[2] + (U1[1][2] - U1[0][2]);
            const float SBx = az[0] + (U1[1][0] - U0[1][0]), SBz = az[2] + (U1[1][2] - U0[1][2]);
            const float el = Et * cl, em = Et * cm;
            const float p = em * SAz, q = el * SAx;
            Gxz[0] = fmaf(el, SBz, p);
            Hxz[0] = fmaf(el, SBz, -p);
            Gxz[1] = fmaf(em, SBx, q);
            Hxz[1] = fmaf(em, SBx, -q);
        }
        // yz face (a = y, b = z) in the plane x = X: cells (X-1..X, Y, zp)
        float Gyz[2], Hyz[2];  // components (y, z)
        {
            const float Et = E1[0] + E1[1];
            const float SAy = ay[1] + (U1[2][1] - U1[0][1]), SAz = ay[2] + (U1[2][2] - U1[0][2]);
            const float SBy = az[1] + (U1[2][1] - U0[2][1]), SBz = az[2] + (U1[2][2] - U0[2][2]);
            const float el = Et * cl, em = Et * cm;
            const float p = em * SAz, q = el * SAy;
            Gyz[0] = fmaf(el, SBz, p);
            Hyz[0] = fmaf(el, SBz, -p);
            Gyz[1] = fmaf(em, SBy, q);
            Hyz[1] = fmaf(em, SBy, -q);
        }

        // ---- messages
        const float Mx0 = Fx[0] + Hxy[0] + Hxz[0] + Gxzp[0];
        const float Mx1 = Fx[1] + Hxy[1];
        const float Mx2 = Fx[2] + Hxz[1] + Gxzp[1];
        const float My0 = Fy[0] - Hxy[0];
        const float My1 = Fy[1] - Hxy[1] + Hyz[0] + Gyzp[0];
        const float My2 = Fy[2] + Hyz[1] + Gyzp[1];
        const int sm = zp & 1;
        ma[sm][ty][tx] = make_float4(Mx0, Mx1, Mx2, Gxy[0]);
        mb[sm][ty][tx] = make_float4(My0, My1, My2, Gxy[1]);
        const float own0 = -(Fx[0] + Fy[0] + Fz[0]) - Gxy[0] - Gxz[0];
        const float own1 = -(Fx[1] + Fy[1] + Fz[1]) - Gxy[1] - Gyz[0];
        const float own2 = -(Fx[2] + Fy[2] + Fz[2]) - Gxz[1] - Gyz[1];
        const float Sz0 = Fz[0] - Hxz[0];
        const float Sz1 = Fz[1] - Hyz[0];
        const float Sz2 = Fz[2] - Hxz[1] - Hyz[1];
        __syncthreads();

        if (outp) {
            const float4 rx = ma[sm][ty][tx - 1];
            const float4 ry = mb[sm][ty - 1][tx];
            const float gxy0 = ma[sm][ty - 1][tx - 1].w;
            const float gxy1 = mb[sm][ty - 1][tx - 1].w;
            const float Ku[3] = {own0 + rx.x + ry.x + Szp[0] + gxy0, own1 + rx.y + ry.y + Szp[1] + gxy1,
                                 own2 + rx.z + ry.z + Szp[2]};
            unsigned fm = 0;
            for (int q = 0; q < A.boxes.n; ++q)
                if (((boxbits >> q) & 1u) && zp >= A.boxes.b[q].lo[2] && zp <= A.boxes.b[q].hi[2]) fm |= A.boxes.b[q].mask;
            float F[3] = {0.f, 0.f, 0.f};
            if (rhs) {
#pragma unroll
                for (int c = 0; c < 3; ++c) F[c] = rhs[(int64_t)c * L.cstride + nidx];
            } else {
                for (int l = l0; l < l1; ++l) {
                    const LoadEntry &le = A.loads[l];
                    if (le.node == nidx) F[le.comp] += le.valf;
                }
            }
            const float S8 = E0[0] + E0[1] + E0[2] + E0[3] + E1[0] + E1[1] + E1[2] + E1[3];
            const float dinv = A.local_dt ? 1.f / (cdg * S8) : 1.f;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const bool fixed = (fm >> c) & 1u;
                const float R = fixed ? 0.f : F[c] - Ku[c];
                res = fmaf(R, R, res);
                const int64_t idx = (int64_t)c * L.cstride + nidx;
                if (A.mode == 0) {
                    dot = fmaf(R, wv[c], dot);
                    const float wn = fixed ? 0.f : fmaf(fa, wv[c], fb * dinv * R);
                    w[idx] = wn;
                    uo[idx] = fixed ? 0.f : uown[c] + wn;
                } else if (A.mode == 1) {
                    uo[idx] = fixed ? 0.f : fmaf(fs1 * dinv, R, uown[c]);
                } else {
                    w[idx] = R;
                }
            }
        }
        // carry to the next plane
        Szp[0] = Sz0; Szp[1] = Sz1; Szp[2] = Sz2;
        Gxzp[0] = Gxz[0]; Gxzp[1] = Gxz[1];
        Gyzp[0] = Gyz[0]; Gyzp[1] = Gyz[1];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            U0[0][c] = U1[0][c];
            U0[1][c] = U1[1][c];
            U0[2][c] = U1[2][c];
            U0[3][c] = su[s1][c][ty + 1][tx + 1];
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) E0[q] = E1[q];
    }

    if (A.want_res || A.test_dot) {
        const unsigned nb = gridDim.x * gridDim.y * gridDim.z;
        const double r = A.want_res ? block_sum((double)res, shred) : 0.0;
        const double d = A.test_dot ? block_sum((double)dot, shred) : 0.0;
        if (tid == 0) A.red.partials[(int64_t)nb + tile] = d;
        if (publish_partial(r, A.red, tile, nb)) {
            const double t = A.want_res ? sum_partials(A.red, 0, nb, shred) : 0.0;
            const double td = A.test_dot ? sum_partials(A.red, nb, nb, shred) : 0.0;
            if (tid == 0) {
                if (A.want_res) *A.res2 = t;
                if (A.test_dot) {
                    A.ctrl[CT_DOT] = td;
                    if (td < 0.0) A.ctrl[CT_RESTART_AT] = (double)(A.sweep_idx + 1);
                }
                *A.red.counter = 0u;
            }
        }
    }
}

}  // namespace

void march3d_tiling(const Layout &L, Tiling &t) {
    t.bx = MX;
    t.by = MTY;
    t.zs = MZS;
    t.ox = MX - 1;
    t.oy = MTY - 1;
    t.kind = 1;
    t.gx = (L.NX + t.ox - 1) / t.ox;
    t.gy = (L.NY + t.oy - 1) / t.oy;
    t.gz = (L.NZ + t.zs - 1) / t.zs;
}

cudaError_t launch_march3d(const SweepArgs &a, const Tiling &t, cudaStream_t s) {
    dim3 block(MX, MTY, 1), grid(t.gx, t.gy, t.gz);
    sweep3d_march_f32<<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace petto

// ============================================================================
// TMA-staged variant.  Same owner/message scheme as above; the u planes and modulus
// layers arrive through cp.async.bulk.tensor into a 4-slot shared-memory ring, three
// planes ahead, each slot guarded by an mbarrier (one elected thread issues the copies and
// the expected byte count).  Tensor boxes start at a 16-byte aligned x (the tile origin
// rounded down) and the block reads them at a fixed column offset.  One block barrier per
// plane: the ring slot about to be refilled was last read before the previous barrier.
// Every mbarrier wait is bounded; on time-out the block records an error in the control
// words, drains its copies in flight (bounded) and leaves without writing.
// ============================================================================
namespace petto {
namespace {

constexpr int TBW = 40;        // box width (floats): covers the 33 tile columns at any offset 0..3
constexpr int TNS = 4;         // ring slots
constexpr int TD = 3;          // planes in flight ahead of the consumer
constexpr int TWAIT = 1 << 22; // try_wait attempts before a wait is declared timed out

template <int TY> struct TmaGeom {
    static constexpr int NT = 32 * TY, WY = TY + 1;
    static constexpr int UBYTES = 3 * WY * TBW * 4, EBYTES = WY * TBW * 4;
    static constexpr int USLOT = (UBYTES + 127) / 128 * 128, ESLOT = (EBYTES + 127) / 128 * 128;
    static constexpr int MSG = 2 * 2 * NT * 16;
    static constexpr int SMEM = TNS * (USLOT + ESLOT) + MSG + TNS * 8 + 128;  // + alignment slack
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (int it = 0; it < TWAIT; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
        : "memory");
}

template <int TY>
__global__ void __launch_bounds__(32 * TY, 24 / TY) sweep3d_march_tma(const __grid_constant__ SweepArgs A,
                                                             const __grid_constant__ CUtensorMap tmu,
                                                             const __grid_constant__ CUtensorMap tme) {
    using G = TmaGeom<TY>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // TMA destinations at 128-byte aligned shared addresses
    unsigned char *smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    float *su = reinterpret_cast<float *>(smem);                                  // TNS u slots
    float *se = reinterpret_cast<float *>(smem + TNS * G::USLOT);                 // TNS E slots
    float4 *msg = reinterpret_cast<float4 *>(smem + TNS * (G::USLOT + G::ESLOT)); // [2][2][NT]
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + TNS * (G::USLOT + G::ESLOT) + G::MSG);
    __shared__ double shred[32];

    const Layout &L = A.L;
    float *__restrict__ uo = static_cast<float *>(A.u_out);
    float *__restrict__ w = static_cast<float *>(A.w);
    const float *__restrict__ rhs = static_cast<const float *>(A.rhs);

    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
    const int x0 = blockIdx.x * 31, y0 = blockIdx.y * (TY - 1), z0 = blockIdx.z * MZS;
    const int X = x0 - 1 + tx, Y = y0 - 1 + ty;
    const bool outxy = tx >= 1 && ty >= 1 && X < L.NX && Y < L.NY;
    const int zend = min(z0 + MZS, L.NZ);
    const int xs = (x0 - 1 + OX) & ~3, xoff = (x0 - 1 + OX) - xs;    // u box origin / column offset
    const int xse = (x0 - 2 + OX) & ~3, xoffe = (x0 - 2 + OX) - xse; // E box origin / column offset

    const float cpar = (float)A.k.ce_par, cperp = (float)A.k.ce_perp;
    const float cl = (float)A.k.cf_lam, cm = (float)A.k.cf_mu, cdg = (float)A.k.cdiag;
    float fa = (float)A.a;
    const float fb = (float)A.b, fs1 = (float)A.s1;
    if (A.adaptive) {
        const long long k = A.sweep_idx - (long long)A.ctrl[CT_RESTART_AT];
        const float sched = k <= 0 ? 0.f : (float)(k - 1) / (float)(k + 2);
        fa = fminf(fa, sched);
    }
    unsigned boxbits = 0;
    for (int q = 0; q < A.boxes.n; ++q) {
        const Box &b = A.boxes.b[q];
        if (X >= b.lo[0] && X <= b.hi[0] && Y >= b.lo[1] && Y <= b.hi[1]) boxbits |= 1u << q;
    }
    const int tile = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    const int l0 = A.tile_ptr[tile], l1 = A.tile_ptr[tile + 1];
    const int64_t plane = L.SX * L.SY, cs = L.cstride;
    const int64_t nbase = outxy ? L.node(X, Y, 0) : 0;

    // stage r (relative to plane z0-1) holds u plane z0-1+r and E layer z0-2+r
    auto issue = [&](int r) {
        const int p = z0 - 1 + r;
        const int slot = r % TNS;
        const uint32_t bar = smem_u32(&bars[slot]);
        mbar_expect_tx(bar, (unsigned)(G::UBYTES + G::EBYTES));
        tma_load_4d(smem_u32(su + slot * (G::USLOT / 4)), &tmu, xs, y0, p + 1, 0, bar);
        tma_load_3d(smem_u32(se + slot * (G::ESLOT / 4)), &tme, xse, y0 - 1, p, bar);
    };
    const int nstage = zend - (z0 - 1) + 1;  // stages z0-1 .. zend
    if (tid == 0) {
        for (int s = 0; s < TNS; ++s) mbar_init(smem_u32(&bars[s]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0)
        for (int r = 0; r <= TD && r < nstage; ++r) issue(r);
    int issued = min(TD + 1, nstage);

    bool bad = !mbar_wait(smem_u32(&bars[0]), 0);
    float U0[4][3], E0[4];
    {
        const float *u0 = su;
        const float *e0 = se;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float *r0 = u0 + (c * G::WY + ty) * TBW + xoff + tx;
            U0[0][c] = r0[0];
            U0[1][c] = r0[1];
            U0[2][c] = r0[TBW];
            U0[3][c] = r0[TBW + 1];
        }
        const float *q0 = e0 + ty * TBW + xoffe + tx;
        E0[0] = q0[TBW + 1];
        E0[1] = q0[TBW];
        E0[2] = q0[1];
        E0[3] = q0[0];
    }
    bad = __syncthreads_or(bad);
    float Szp[3] = {0.f, 0.f, 0.f}, Gxzp[2] = {0.f, 0.f}, Gyzp[2] = {0.f, 0.f};
    float res = 0.f, dot = 0.f;

    for (int zp = z0 - 1; zp < zend && !bad; ++zp) {
        const int r1 = zp + 1 - (z0 - 1);  // stage read in this iteration
        if (tid == 0 && issued < nstage && issued <= r1 + TD - 1 + 1) {
            issue(issued);
        }
        issued = min(issued + 1, nstage);
        const int slot = r1 % TNS;
        const bool outp = outxy && zp >= z0;
        const int64_t nidx = nbase + (int64_t)zp * plane;
        float wv[3] = {0.f, 0.f, 0.f};
        if (outp && A.mode == 0) {
#pragma unroll
            for (int c = 0; c < 3; ++c) wv[c] = w[c * cs + nidx];
        }
        if (!mbar_wait(smem_u32(&bars[slot]), (r1 / TNS) & 1)) bad = true;
        float U1[4][3], E1[4];
        {
            const float *u1 = su + slot * (G::USLOT / 4);
            const float *e1 = se + slot * (G::ESLOT / 4);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float *r0 = u1 + (c * G::WY + ty) * TBW + xoff + tx;
                U1[0][c] = r0[0];
                U1[1][c] = r0[1];
                U1[2][c] = r0[TBW];
                U1[3][c] = r0[TBW + 1];
            }
            const float *q0 = e1 + ty * TBW + xoffe + tx;
            E1[0] = q0[TBW + 1];
            E1[1] = q0[TBW];
            E1[2] = q0[1];
            E1[3] = q0[0];
        }
        const float Ex = E1[0] + E1[2] + E0[0] + E0[2];
        const float Ey = E1[0] + E1[1] + E0[0] + E0[1];
        const float Ez = E1[0] + E1[1] + E1[2] + E1[3];
        float ax[3], ay[3], az[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            ax[c] = U0[1][c] - U0[0][c];
            ay[c] = U0[2][c] - U0[0][c];
            az[c] = U1[0][c] - U0[0][c];
        }
        const float exp_ = Ex * cpar, exq = Ex * cperp, eyp = Ey * cpar, eyq = Ey * cperp, ezp = Ez * cpar,
                    ezq = Ez * cperp;
        const float Fx[3] = {exp_ * ax[0], exq * ax[1], exq * ax[2]};
        const float Fy[3] = {eyq * ay[0], eyp * ay[1], eyq * ay[2]};
        const float Fz[3] = {ezq * az[0], ezq * az[1], ezp * az[2]};
        float Gxy[2], Hxy[2], Gxz[2], Hxz[2], Gyz[2], Hyz[2];
        {
            const float Et = E1[0] + E0[0];
            const float SAx = ax[0] + (U0[3][0] - U0[2][0]), SAy = ax[1] + (U0[3][1] - U0[2][1]);
            const float SBx = ay[0] + (U0[3][0] - U0[1][0]), SBy = ay[1] + (U0[3][1] - U0[1][1]);
            const float el = Et * cl, em = Et * cm, p = em * SAy, q = el * SAx;
            Gxy[0] = fmaf(el, SBy, p);
            Hxy[0] = fmaf(el, SBy, -p);
            Gxy[1] = fmaf(em, SBx, q);
            Hxy[1] = fmaf(em, SBx, -q);
        }
        {
            const float Et = E1[0] + E1[2];
            const float SAx = ax[0] + (U1[1][0] - U1[0][0]), SAz = ax[2] + (U1[1][2] - U1[0][2]);
            const float SBx = az[0] + (U1[1][0] - U0[1][0]), SBz = az[2] + (U1[1][2] - U0[1][2]);
            const float el = Et * cl, em = Et * cm, p = em * SAz, q = el * SAx;
            Gxz[0] = fmaf(el, SBz, p);
            Hxz[0] = fmaf(el, SBz, -p);
            Gxz[1] = fmaf(em, SBx, q);
            Hxz[1] = fmaf(em, SBx, -q);
        }
        {
            const float Et = E1[0] + E1[1];
            const float SAy = ay[1] + (U1[2][1] - U1[0][1]), SAz = ay[2] + (U1[2][2] - U1[0][2]);
            const float SBy = az[1] + (U1[2][1] - U0[2][1]), SBz = az[2] + (U1[2][2] - U0[2][2]);
            const float el = Et * cl, em = Et * cm, p = em * SAz, q = el * SAy;
            Gyz[0] = fmaf(el, SBz, p);
            Hyz[0] = fmaf(el, SBz, -p);
            Gyz[1] = fmaf(em, SBy, q);
            Hyz[1] = fmaf(em, SBy, -q);
        }
        const int sm = zp & 1;
        float4 *ma = msg + (sm * 2 + 0) * G::NT;
        float4 *mb = msg + (sm * 2 + 1) * G::NT;
        ma[tid] = make_float4(Fx[0] + Hxy[0] + Hxz[0] + Gxzp[0], Fx[1] + Hxy[1], Fx[2] + Hxz[1] + Gxzp[1], Gxy[0]);
        mb[tid] = make_float4(Fy[0] - Hxy[0], Fy[1] - Hxy[1] + Hyz[0] + Gyzp[0], Fy[2] + Hyz[1] + Gyzp[1], Gxy[1]);
        const float own0 = -(Fx[0] + Fy[0] + Fz[0]) - Gxy[0] - Gxz[0];
        const float own1 = -(Fx[1] + Fy[1] + Fz[1]) - Gxy[1] - Gyz[0];
        const float own2 = -(Fx[2] + Fy[2] + Fz[2]) - Gxz[1] - Gyz[1];
        const float Sz0 = Fz[0] - Hxz[0], Sz1 = Fz[1] - Hyz[0], Sz2 = Fz[2] - Hxz[1] - Hyz[1];
        if (__syncthreads_or(bad)) {
            bad = true;
            break;
        }
        if (outp) {
            const float4 rx = ma[tid - 1];
            const float4 ry = mb[tid - 32];
            const float gxy0 = ma[tid - 33].w, gxy1 = mb[tid - 33].w;
            const float Ku[3] = {own0 + rx.x + ry.x + Szp[0] + gxy0, own1 + rx.y + ry.y + Szp[1] + gxy1,
                                 own2 + rx.z + ry.z + Szp[2]};
            unsigned fm = 0;
            if (boxbits)
                for (int q = 0; q < A.boxes.n; ++q)
                    if (((boxbits >> q) & 1u) && zp >= A.boxes.b[q].lo[2] && zp <= A.boxes.b[q].hi[2])
                        fm |= A.boxes.b[q].mask;
            float F[3] = {0.f, 0.f, 0.f};
            if (rhs) {
#pragma unroll
                for (int c = 0; c < 3; ++c) F[c] = rhs[c * cs + nidx];
            } else {
                for (int l = l0; l < l1; ++l) {
                    const LoadEntry &le = A.loads[l];
                    if (le.node == nidx) F[le.comp] += le.valf;
                }
            }
            float dinv = 1.f;
            if (A.local_dt) {
                const float S8 = E0[0] + E0[1] + E0[2] + E0[3] + E1[0] + E1[1] + E1[2] + E1[3];
                dinv = __frcp_rn(cdg * S8);
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const bool fixed = (fm >> c) & 1u;
                const float R = fixed ? 0.f : F[c] - Ku[c];
                res = fmaf(R, R, res);
                const int64_t idx = c * cs + nidx;
                if (A.mode == 0) {
                    dot = fmaf(R, wv[c], dot);
                    const float wn = fixed ? 0.f : fmaf(fa, wv[c], fb * dinv * R);
                    w[idx] = wn;
                    uo[idx] = fixed ? 0.f : U0[0][c] + wn;
                } else if (A.mode == 1) {
                    uo[idx] = fixed ? 0.f : fmaf(fs1 * dinv, R, U0[0][c]);
                } else {
                    w[idx] = R;
                }
            }
        }
        Szp[0] = Sz0; Szp[1] = Sz1; Szp[2] = Sz2;
        Gxzp[0] = Gxz[0]; Gxzp[1] = Gxz[1];
        Gyzp[0] = Gyz[0]; Gyzp[1] = Gyz[1];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            U0[0][c] = U1[0][c];
            U0[1][c] = U1[1][c];
            U0[2][c] = U1[2][c];
            U0[3][c] = U1[3][c];
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) E0[q] = E1[q];
    }

    if (bad) {
        // record the time-out, let the copies already issued land (bounded), leave
        if (tid == 0) {
            A.ctrl[CT_ERR] = 1.0;
            for (int r = 0; r < issued; ++r) mbar_wait(smem_u32(&bars[r % TNS]), (r / TNS) & 1);
        }
        __syncthreads();
        return;
    }
    if (A.want_res || A.test_dot) {
        const unsigned nb = gridDim.x * gridDim.y * gridDim.z;
        const double r = A.want_res ? block_sum((double)res, shred) : 0.0;
        const double d = A.test_dot ? block_sum((double)dot, shred) : 0.0;
        if (tid == 0) A.red.partials[(int64_t)nb + tile] = d;
        if (publish_partial(r, A.red, tile, nb)) {
            const double t = A.want_res ? sum_partials(A.red, 0, nb, shred) : 0.0;
            const double td = A.test_dot ? sum_partials(A.red, nb, nb, shred) : 0.0;
            if (tid == 0) {
                if (A.want_res) *A.res2 = t;
                if (A.test_dot) {
                    A.ctrl[CT_DOT] = td;
                    if (td < 0.0) A.ctrl[CT_RESTART_AT] = (double)(A.sweep_idx + 1);
                }
                *A.red.counter = 0u;
            }
        }
    }
}

}  // namespace

void march3d_tma_tiling(const Layout &L, int ty, Tiling &t) {
    t.bx = 32;
    t.by = ty;
    t.zs = MZS;
    t.ox = 31;
    t.oy = ty - 1;
    t.kind = ty == 16 ? 3 : 2;
    t.gx = (L.NX + t.ox - 1) / t.ox;
    t.gy = (L.NY + t.oy - 1) / t.oy;
    t.gz = (L.NZ + t.zs - 1) / t.zs;
}

cudaError_t launch_march3d_tma(const SweepArgs &a, const Tiling &t, const TmaMaps &m, cudaStream_t s) {
    const CUtensorMap *mu = a.u_in == m.ubuf[0] ? &m.u[0] : (a.u_in == m.ubuf[1] ? &m.u[1] : nullptr);
    if (!mu) return cudaErrorInvalidValue;
    dim3 grid(t.gx, t.gy, t.gz);
    if (t.kind == 3) {
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(sweep3d_march_tma<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, TmaGeom<16>::SMEM);
            attr = true;
        }
        sweep3d_march_tma<16><<<grid, dim3(32, 16), TmaGeom<16>::SMEM, s>>>(a, *mu, m.e);
    } else {
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(sweep3d_march_tma<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, TmaGeom<8>::SMEM);
            attr = true;
        }
        sweep3d_march_tma<8><<<grid, dim3(32, 8), TmaGeom<8>::SMEM, s>>>(a, *mu, m.e);
    }
    return cudaGetLastError();
}

}  // namespace petto

// ---------------------------------------------------------------- tensor maps (host)
#include <cudaTypedefs.h>

namespace petto {

bool make_tma_maps(const Layout &L, int ty, void *u0, void *u1, const void *E, TmaMaps &m) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return false;
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    m.valid = false;
    const cuuint64_t udim[4] = {(cuuint64_t)L.SX, (cuuint64_t)L.SY, (cuuint64_t)L.SZ, 3};
    const cuuint64_t ustr[3] = {(cuuint64_t)L.SX * 4, (cuuint64_t)(L.SX * L.SY) * 4, (cuuint64_t)L.cstride * 4};
    const cuuint32_t ubox[4] = {TBW, (cuuint32_t)(ty + 1), 1, 3};
    const cuuint32_t one4[4] = {1, 1, 1, 1};
    void *ub[2] = {u0, u1};
    for (int q = 0; q < 2; ++q) {
        if (encode(&m.u[q], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, ub[q], udim, ustr, ubox, one4,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
        m.ubuf[q] = ub[q];
    }
    const cuuint64_t edim[3] = {(cuuint64_t)L.CX, (cuuint64_t)L.CY, (cuuint64_t)L.CZ};
    const cuuint64_t estr[2] = {(cuuint64_t)L.CX * 4, (cuuint64_t)(L.CX * L.CY) * 4};
    const cuuint32_t ebox[3] = {TBW, (cuuint32_t)(ty + 1), 1};
    if (encode(&m.e, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void *>(E), edim, estr, ebox, one4,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    m.valid = true;
    return true;
}

}  // namespace petto
