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
