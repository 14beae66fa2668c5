// FP64 defect of the iterative refinement on 3D elasticity: R = F - K(E) u for the FP64
// state u and the FP32 cell moduli E (the Sec. 3.2 corner-quadrature operator; the
// refinement around the FP32 sweeps of Sec. 2.2, one defect per refinement round).
//
// GB300's FP64 pipe issues about two operations per clock per SM -- a sixty-fourth of its
// FP32 rate -- so this kernel is bound by FP64 arithmetic, not bytes: what counts is the
// number of FP64 operations per node.  The node-gather form recomputes the terms of every
// edge and face at each of their nodes (about 420 operations a node); this kernel uses the
// owner-message form of the FP32 marching sweeps instead, where every edge and face term is
// computed once, by the node that owns it, and handed to the other nodes it touches:
//
//   * a block of 32 x 8 threads owns a tile of 31 x 7 node columns (lane 0 and thread row 0
//     are the halo that only sends messages) and marches a z segment of it, plane by plane,
//     one plane below the segment first (it only produces the z messages);
//   * node planes of u (FP64) and layers of E (FP32, converted once when staged) go through
//     a two-slot shared-memory ring, the next plane's loads in flight during the current
//     plane's arithmetic;
//   * x and y messages (with the xy-face corner term) go through shared memory, z messages
//     stay in registers from one plane to the next;
//   * the moduli sums of the edges and faces reuse each other and the previous plane's
//     (seven additions a node instead of twelve).
//
// One launch per load case.  On a slab of a z-decomposed grid the segments start at the
// slab's first plane (its ghost plane below is the first segment's warm-up plane) and only
// the slab's own planes are written; a node's arithmetic does not depend on where the
// segments start, so a slab's defect equals the whole grid's bit for bit.
#include "petto_internal.cuh"

namespace petto {
namespace {

constexpr int DX = 32;            // threads (owner columns) per tile row
constexpr int DTY = 8;            // owner rows per tile
constexpr int DWX = DX + 1;       // staged plane width (nodes) / layer width (cells)
constexpr int DWY = DTY + 1;      // staged plane height
constexpr int DNT = DX * DTY;     // threads per block
constexpr int DENT = DWX * DWY;   // staged entries per plane
constexpr int DST = (DENT + DNT - 1) / DNT;  // staged entries per thread

struct DStaged {
    double u[DST][3];
    double e[DST];
};

// u plane p (nodes x0-1 .. x0+31, y0-1 .. y0+7) and E layer p-1 (cells x0-2 .., y0-2 ..) into
// registers; zero outside the grid
__device__ __forceinline__ void d_stage(const Layout &L, const double *__restrict__ u, const float *__restrict__ E,
                                        int x0, int y0, int p, int tid, DStaged &s) {
#pragma unroll
    for (int r = 0; r < DST; ++r) {
        const int e = tid + r * DNT;
        const int ex = e % DWX, ey = e / DWX;
        const int x = x0 - 1 + ex, y = y0 - 1 + ey;
        const bool okn = e < DENT && x >= 0 && x < L.NX && y >= 0 && y < L.NY && p >= 0 && p < L.NZ;
        const int64_t n = okn ? L.node(x, y, p) : 0;
#pragma unroll
        for (int c = 0; c < 3; ++c) s.u[r][c] = okn ? __ldg(&u[(int64_t)c * L.cstride + n]) : 0.0;
        const int cx = x - 1, cy = y - 1, l = p - 1;
        const bool oke = e < DENT && cx >= 0 && cx < L.nx && cy >= 0 && cy < L.ny && l >= 0 && l < L.nz;
        s.e[r] = oke ? (double)__ldg(&E[L.cell(cx, cy, l)]) : 0.0;
    }
}

__global__ void __launch_bounds__(DNT, 2) defect3d_march(const SweepArgs A) {
    __shared__ double su[2][3][DWY][DWX];
    __shared__ double se[2][DWY][DWX];
    __shared__ double mx[4][DTY][DX];  // x message (3 components) and Gxy.x
    __shared__ double my[4][DTY][DX];  // y message (3 components) and Gxy.y
    __shared__ double shred[32];

    const Layout &L = A.L;
    const double *__restrict__ ui = static_cast<const double *>(A.u_in) + (int64_t)3 * A.rhs_index * L.cstride;
    double *__restrict__ ro = static_cast<double *>(A.w) + (int64_t)3 * A.rhs_index * L.cstride;
    const float *__restrict__ E = static_cast<const float *>(A.E);

    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * DX + tx;
    const int x0 = blockIdx.x * (DX - 1), y0 = blockIdx.y * (DTY - 1), z0 = A.zb + blockIdx.z * A.zseg;
    const int X = x0 - 1 + tx, Y = y0 - 1 + ty;
    const bool outxy = tx >= 1 && ty >= 1 && X < L.NX && Y < L.NY;
    const int zend = min(z0 + A.zseg, A.zhi + 1);
    const int zo = max(z0, A.zlo);  // first plane written
    const double cpar = A.k.ce_par, cperp = A.k.ce_perp, cl = A.k.cf_lam, cm = A.k.cf_mu;

    unsigned boxbits = 0;  // support boxes containing this (X, Y) column
    for (int q = 0; q < A.boxes.n; ++q) {
        const Box &b = A.boxes.b[q];
        if (X >= b.lo[0] && X <= b.hi[0] && Y >= b.lo[1] && Y <= b.hi[1]) boxbits |= 1u << q;
    }
    const int tile = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    const int l0 = A.tile_ptr[tile], l1 = A.tile_ptr[tile + 1];
    const int c0 = 3 * A.rhs_index;

    // prologue: plane z0-1 into ring slot (z0-1)&1, plane z0 staged in registers
    DStaged st;
    d_stage(L, ui, E, x0, y0, z0 - 1, tid, st);
#pragma unroll
    for (int r = 0; r < DST; ++r) {
        const int e = tid + r * DNT;
        if (e < DENT) {
            const int ex = e % DWX, ey = e / DWX;
#pragma unroll
            for (int c = 0; c < 3; ++c) su[(z0 + 1) & 1][c][ey][ex] = st.u[r][c];
            se[(z0 + 1) & 1][ey][ex] = st.e[r];
        }
    }
    d_stage(L, ui, E, x0, y0, z0, tid, st);
    __syncthreads();

    // plane zp (lo) values of this thread: u at (X, Y), (X+1, Y), (X, Y+1), (X+1, Y+1) and the
    // moduli sums of the xz and yz faces of the previous layer
    double U0[4][3], E0c;
    double pxz, pyz;
    {
        const int s = (z0 + 1) & 1;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            U0[0][c] = su[s][c][ty][tx];
            U0[1][c] = su[s][c][ty][tx + 1];
            U0[2][c] = su[s][c][ty + 1][tx];
            U0[3][c] = su[s][c][ty + 1][tx + 1];
        }
        // layer z0-2 (cells of plane z0-1's ring entry)
        E0c = se[s][ty + 1][tx + 1];
        pxz = E0c + se[s][ty][tx + 1];
        pyz = E0c + se[s][ty + 1][tx];
    }
    double Szp[3] = {0.0, 0.0, 0.0}, Gxzp[2] = {0.0, 0.0}, Gyzp[2] = {0.0, 0.0};
    double res = 0.0;

    for (int zp = z0 - 1; zp < zend; ++zp) {
        // ring slot of plane zp+1 (and E layer zp): write the staged data, then stage zp+2
        const int s1 = (zp + 1) & 1;
#pragma unroll
        for (int r = 0; r < DST; ++r) {
            const int e = tid + r * DNT;
            if (e < DENT) {
                const int ex = e % DWX, ey = e / DWX;
#pragma unroll
                for (int c = 0; c < 3; ++c) su[s1][c][ey][ex] = st.u[r][c];
                se[s1][ey][ex] = st.e[r];
            }
        }
        if (zp + 2 <= zend) d_stage(L, ui, E, x0, y0, zp + 2, tid, st);
        __syncthreads();

        double U1[3][3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            U1[0][c] = su[s1][c][ty][tx];
            U1[1][c] = su[s1][c][ty][tx + 1];
            U1[2][c] = su[s1][c][ty + 1][tx];
        }
        // layer zp: cells (X, Y), (X-1, Y), (X, Y-1), (X-1, Y-1)
        const double E1c = se[s1][ty + 1][tx + 1], E1x = se[s1][ty + 1][tx], E1y = se[s1][ty][tx + 1],
                     E1xy = se[s1][ty][tx];

        // ---- moduli sums: faces first, the edges from them and the previous layer's
        const double Exz = E1c + E1y;            // xz face: cells (X, Y-1..Y, zp)
        const double Eyz = E1c + E1x;            // yz face: cells (X-1..X, Y, zp)
        const double Exy = E1c + E0c;            // xy face: cells (X, Y, zp-1..zp)
        const double Ex = Exz + pxz;             // x edge: cells (X, Y-1..Y, zp-1..zp)
        const double Ey = Eyz + pyz;             // y edge: cells (X-1..X, Y, zp-1..zp)
        const double Ez = Eyz + (E1y + E1xy);    // z edge: cells (X-1..X, Y-1..Y, zp)

        // ---- owned edges
        double ax[3], ay[3], az[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            ax[c] = U0[1][c] - U0[0][c];
            ay[c] = U0[2][c] - U0[0][c];
            az[c] = U1[0][c] - U0[0][c];
        }
        const double exp_ = Ex * cpar, exq = Ex * cperp, eyp = Ey * cpar, eyq = Ey * cperp, ezp = Ez * cpar,
                     ezq = Ez * cperp;
        const double Fx[3] = {exp_ * ax[0], exq * ax[1], exq * ax[2]};
        const double Fy[3] = {eyq * ay[0], eyp * ay[1], eyq * ay[2]};
        const double Fz[3] = {ezq * az[0], ezq * az[1], ezp * az[2]};

        // ---- owned faces: G (to the far corner) and H (to the a-neighbour corner)
        double Gxy[2], Hxy[2];  // xy face at plane zp, components (x, y)
        {
            const double SAx = ax[0] + (U0[3][0] - U0[2][0]), SAy = ax[1] + (U0[3][1] - U0[2][1]);
            const double SBx = ay[0] + (U0[3][0] - U0[1][0]), SBy = ay[1] + (U0[3][1] - U0[1][1]);
            const double el = Exy * cl, em = Exy * cm;
            const double p = em * SAy, q = el * SAx;
            Gxy[0] = fma(el, SBy, p);
            Hxy[0] = fma(el, SBy, -p);
            Gxy[1] = fma(em, SBx, q);
            Hxy[1] = fma(em, SBx, -q);
        }
        double Gxz[2], Hxz[2];  // xz face in the plane y = Y, components (x, z)
        {
            const double SAx = ax[0] + (U1[1][0] - U1[0][0]), SAz = ax[2] + (U1[1][2] - U1[0][2]);
            const double SBx = az[0] + (U1[1][0] - U0[1][0]), SBz = az[2] + (U1[1][2] - U0[1][2]);
            const double el = Exz * cl, em = Exz * cm;
            const double p = em * SAz, q = el * SAx;
            Gxz[0] = fma(el, SBz, p);
            Hxz[0] = fma(el, SBz, -p);
            Gxz[1] = fma(em, SBx, q);
            Hxz[1] = fma(em, SBx, -q);
        }
        double Gyz[2], Hyz[2];  // yz face in the plane x = X, components (y, z)
        {
            const double SAy = ay[1] + (U1[2][1] - U1[0][1]), SAz = ay[2] + (U1[2][2] - U1[0][2]);
            const double SBy = az[1] + (U1[2][1] - U0[2][1]), SBz = az[2] + (U1[2][2] - U0[2][2]);
            const double el = Eyz * cl, em = Eyz * cm;
            const double p = em * SAz, q = el * SAy;
            Gyz[0] = fma(el, SBz, p);
            Hyz[0] = fma(el, SBz, -p);
            Gyz[1] = fma(em, SBy, q);
            Hyz[1] = fma(em, SBy, -q);
        }

        // ---- messages to (X+1, Y) and (X, Y+1); the xy-face G goes to (X+1, Y+1)
        mx[0][ty][tx] = Fx[0] + Hxy[0] + Hxz[0] + Gxzp[0];
        mx[1][ty][tx] = Fx[1] + Hxy[1];
        mx[2][ty][tx] = Fx[2] + Hxz[1] + Gxzp[1];
        mx[3][ty][tx] = Gxy[0];
        my[0][ty][tx] = Fy[0] - Hxy[0];
        my[1][ty][tx] = Fy[1] - Hxy[1] + Hyz[0] + Gyzp[0];
        my[2][ty][tx] = Fy[2] + Hyz[1] + Gyzp[1];
        my[3][ty][tx] = Gxy[1];
        __syncthreads();

        if (outxy && zp >= zo) {
            const double Ku0 = -(Fx[0] + Fy[0] + Fz[0]) - Gxy[0] - Gxz[0] + mx[0][ty][tx - 1] + my[0][ty - 1][tx] +
                               Szp[0] + mx[3][ty - 1][tx - 1];
            const double Ku1 = -(Fx[1] + Fy[1] + Fz[1]) - Gxy[1] - Gyz[0] + mx[1][ty][tx - 1] + my[1][ty - 1][tx] +
                               Szp[1] + my[3][ty - 1][tx - 1];
            const double Ku2 =
                -(Fx[2] + Fy[2] + Fz[2]) - Gxz[1] - Gyz[1] + mx[2][ty][tx - 1] + my[2][ty - 1][tx] + Szp[2];
            const int64_t nidx = L.node(X, Y, zp);
            unsigned fm = 0;
            for (int q = 0; q < A.boxes.n; ++q)
                if (((boxbits >> q) & 1u) && zp >= A.boxes.b[q].lo[2] && zp <= A.boxes.b[q].hi[2])
                    fm |= A.boxes.b[q].mask;
            double F0 = 0.0, F1 = 0.0, F2 = 0.0;
            for (int l = l0; l < l1; ++l) {
                const LoadEntry &le = A.loads[l];
                if (le.node != nidx) continue;
                const int cc = le.comp - c0;
                if (cc == 0) F0 += le.vald;
                else if (cc == 1) F1 += le.vald;
                else if (cc == 2) F2 += le.vald;
            }
            const double F[3] = {F0, F1, F2}, Ku[3] = {Ku0, Ku1, Ku2};
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const double R = ((fm >> c) & 1u) ? 0.0 : F[c] - Ku[c];
                res = fma(R, R, res);
                ro[(int64_t)c * L.cstride + nidx] = R;
            }
        }
        // ---- carry to the next plane: z messages, the face sums of layer zp, plane zp+1
        Szp[0] = Fz[0] - Hxz[0];
        Szp[1] = Fz[1] - Hyz[0];
        Szp[2] = Fz[2] - Hxz[1] - Hyz[1];
        Gxzp[0] = Gxz[0];
        Gxzp[1] = Gxz[1];
        Gyzp[0] = Gyz[0];
        Gyzp[1] = Gyz[1];
        pxz = Exz;
        pyz = Eyz;
        E0c = E1c;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            U0[0][c] = U1[0][c];
            U0[1][c] = U1[1][c];
            U0[2][c] = U1[2][c];
            U0[3][c] = su[s1][c][ty + 1][tx + 1];
        }
    }

    if (A.want_res) {
        const unsigned nb = gridDim.x * gridDim.y * gridDim.z;
        const double r = block_sum(res, shred);
        if (publish_partial(r, A.red, tile, nb)) {
            const double t = sum_partials(A.red, 0, nb, shred);
            if (tid == 0) {
                // one launch per load case: the sums accumulate in launch order
                *A.res2 = A.rhs_index == 0 ? t : *A.res2 + t;
                *A.red.counter = 0u;
            }
        }
    }
}

}  // namespace

void defect3d_tiling(const Layout &L, Tiling &t) {
    t.order = 0;
    t.bx = DX;
    t.by = DTY;
    t.ox = DX - 1;
    t.oy = DTY - 1;
    t.kind = 8;
    t.gx = (L.NX + t.ox - 1) / t.ox;
    t.gy = (L.NY + t.oy - 1) / t.oy;
    // FP64-bound: blocks sharing an SM share its FP64 pipe, so the cost of a segmentation is
    // the busiest SM's planes -- waves of one block per SM
    t.zs = choose_zseg(L.NZ, t.gx * t.gy, 152);
    t.gz = (L.NZ + t.zs - 1) / t.zs;
}

cudaError_t launch_defect3d(const SweepArgs &a0, const Tiling &t, cudaStream_t s) {
    const dim3 grid(t.gx, t.gy, t.gz), block(DX, DTY, 1);
    for (int r = 0; r < a0.nrhs; ++r) {
        SweepArgs a = a0;
        a.zseg = t.zs;
        a.zb = t.zn ? t.zb : 0;
        a.rhs_index = r;
        defect3d_march<<<grid, block, 0, s>>>(a);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace petto
