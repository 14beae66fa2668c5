"""Seeded synthetic workloads: grids, supports, loads, materials and initial designs.

This module holds problem *inputs* only -- no stencil, interpolation, update or any
other arithmetic of the method -- so that the GPU path and the FP64 oracle can be fed
identical instances without sharing code.  It imports nothing but numpy.

The paper (PeTTO, arXiv 2509.06971) uses no datasets: every workload is a parametric
box domain with supports and loads (Sec. 3.1 heat sink, Sec. 3.2 MBB beam, Sec. 3.3
cantilever, Sec. 3.4 drone).  The instances below restate those shapes on unit-size
cells; numbers that the paper does not fix are chosen here and documented.

Index conventions: a node is (i, j, k) with 0 <= i <= nx, 0 <= j <= ny, 0 <= k <= nz;
a Dirichlet box is ((lo_i, lo_j, lo_k), (hi_i, hi_j, hi_k), mask) with inclusive node
ranges and bit a of ``mask`` fixing component a; a load is ((i, j, k), comp, value) with
value the external nodal force (downward = negative y in 2D, negative z in 3D).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

ELASTIC, THERMAL = 0, 1
SIMP_MODIFIED, SIMP_PAPER = 0, 1
PROJECTED, PENALTY = 0, 1


@dataclass
class ProblemSpec:
    name: str
    dim: int
    nx: int
    ny: int
    nz: int = 0
    h: float = 1.0
    physics: int = ELASTIC
    nu: float = 0.3
    # materials (Sec. 3.1 / 3.2 interpolation); for SIMP_MODIFIED moduli = [E0]
    moduli: list = field(default_factory=lambda: [1.0])
    e_min: float = 1e-9
    penal: float = 3.0
    interp: int = SIMP_MODIFIED
    vol_frac: list = field(default_factory=lambda: [0.5])
    loads: list = field(default_factory=list)          # [((i,j,k), comp, value)]
    body_source: float = 0.0
    boxes: list = field(default_factory=list)          # [((lo),(hi),mask)]
    phi0: np.ndarray | None = None                     # [P, cells], cell (i,j,k) -> i + nx(j + ny k)
    # state solver parameters in grid units (Sec. 2.2; Sec. 3.2 PT/APT systems)
    apt_a: float = 0.99
    apt_b: float = 0.25
    pt_s1: float = 0.25
    tol: float = 1e-6
    check_every: int = 50
    max_sweeps: int = 200000
    local_dt: bool = True      # local pseudo-time steps b/diag(K), s1/diag(K) (an extension)
    momentum: int = 1          # 0: fixed APT damping a; 1: adaptive-restart momentum (an extension)
    solve_mode: int = 1        # 1: to tolerance; 0: the paper's fixed n_apt APT then n_pt PT sweeps
    n_apt: int = 0
    n_pt: int = 0
    # design update and phase field (Sec. 2.3, 2.4; Sec. 3.1 weights)
    vol_mode: int = PROJECTED
    alpha_h: float = 0.1
    kappa_v: float = 0.0
    kappa_1: float = 0.0
    gamma_g: float = 0.0
    tau: float = 0.0
    n_bisect: int = 60
    # keep-out region of the update (Sec. 3.4 J_b): ((lo_i, lo_j, lo_k), (hi_i, hi_j, hi_k))
    # inclusive cell ranges, per-phase targets and kappa_b = 2 alpha_b / N_b
    keepout: tuple | None = None
    keepout_target: list = field(default_factory=list)
    kappa_b: float = 0.0
    design_steps: int = 1
    precision: str = "f32"
    storage: str = "f32"

    @property
    def n_phases(self) -> int:
        return 1 if self.interp == SIMP_MODIFIED else len(self.moduli)

    @property
    def ncomp(self) -> int:
        return self.dim if self.physics == ELASTIC else 1

    @property
    def ncells(self) -> int:
        return self.nx * self.ny * (self.nz if self.dim == 3 else 1)

    @property
    def nnodes(self) -> int:
        return (self.nx + 1) * (self.ny + 1) * ((self.nz + 1) if self.dim == 3 else 1)

    def with_(self, **kw) -> "ProblemSpec":
        return replace(self, **kw)


# --------------------------------------------------------------- parameter maps

def apt_params(h_p: float, elastic: bool = True, theta: float = 1.0, dim: int = 2):
    """Paper constants in grid units (reading R5).  The paper's APT step is
    dt2 = h_p/2 and theta = 1 with h_p its own cell size (Sec. 3.1, Sec. 3.2); its PT step
    is dt1 = h_p^2/(2d) (Sec. 3.1: dx^2/4 in 2D; Sec. 3.3: dx^2/6 in 3D).  On a grid of
    unit cells the same iteration has
        elastic form: a = theta/(theta + dt2),  b = dt2^2/((theta + dt2) h_p^2)  (= a/4)
        thermal form: a = 1 - dt2/theta,       b = dt2^2/(theta h_p^2)           (= 1/4)
        PT:           s1 = 1/(2d)."""
    dt2 = h_p / 2.0
    if elastic:
        a = theta / (theta + dt2)
        b = (dt2 * dt2 / (theta + dt2)) / (h_p * h_p)
    else:
        a = 1.0 - dt2 / theta
        b = (dt2 * dt2 / theta) / (h_p * h_p)
    return a, b, 1.0 / (2 * dim)


def local_step_params(n_max: int, c_a: float = 0.15):
    """Defaults for local (Jacobi-scaled) pseudo-time steps: returns (a, b, s1) with
    momentum a = 1 - c_a / n_max (the slowest mode of an elliptic operator on n_max cells
    scales as n_max^-2, so the best damping rate scales as 1/n_max), APT step b = 0.9 and PT
    step s1 = 0.75.  The scaled operator diag(K)^-1 K has its largest eigenvalue near 2 for
    uniform moduli and up to about 2.4 for moduli varying cell by cell over nine decades, so
    PT stays inside s1 lam_max < 2 and APT inside b lam_max < 2 (1 + a) once a >= 1/4."""
    return 1.0 - c_a / float(n_max), 0.9, 0.75


def ch_params(h_p: float, dim: int, dt3_factor: float = 500.0, gamma: float = 3e-5, safety: float = 0.9):
    """Cahn-Hilliard constants in grid units (Sec. 3.1: dt3 = 500 dx^4, gamma = 3e-5; D = 1,
    reading R10): tau = dt3/h_p^2, gamma_g = gamma/h_p^2, with tau capped at ``safety`` times
    the explicit stability bound tau (w''_max lam_L + gamma_g lam_L^2) <= 2, lam_L = 4d,
    w''_max = 2 pi^2 / 64 for w = sin^2(pi phi)/64."""
    tau = dt3_factor * h_p ** 2
    gamma_g = gamma / h_p ** 2
    lam_l = 4.0 * dim
    wpp = 2.0 * math.pi ** 2 / 64.0
    bound = 2.0 / (wpp * lam_l + gamma_g * lam_l ** 2)
    return min(tau, safety * bound), gamma_g


# --------------------------------------------------------------- builders

def _uniform_phi(ncells: int, fracs) -> np.ndarray:
    return np.stack([np.full(ncells, float(v)) for v in fracs])


def mbb_halfbeam(nx: int = 60, ny: int = 20, seed: int = 1, precision: str = "f64") -> ProblemSpec:
    """2D MBB half-beam (symmetry edge at x = 0): u_x = 0 on the left edge, u_y = 0 at the
    bottom-right node, unit downward load at the top-left node; E0 = 1, Emin = 1e-9,
    nu = 0.3, p = 3, V = 0.5, initial density 0.5 + U[-0.01, 0.01] (PCG64 ``seed``)."""
    rng = np.random.default_rng(seed)
    phi0 = 0.5 + rng.uniform(-0.01, 0.01, size=(1, nx * ny))
    h_p = 1.0 / ny
    a, b, s1 = local_step_params(nx)
    tau, gg = ch_params(h_p, 2)
    return ProblemSpec(
        name=f"mbb_halfbeam_{nx}x{ny}", dim=2, nx=nx, ny=ny, vol_frac=[0.5],
        boxes=[((0, 0, 0), (0, ny, 0), 0b01), ((nx, 0, 0), (nx, 0, 0), 0b10)],
        loads=[((0, ny, 0), 1, -1.0)], phi0=phi0,
        apt_a=a, apt_b=b, pt_s1=s1, tol=1e-8, tau=tau, gamma_g=gg, design_steps=50,
        precision=precision, storage=precision)


def cantilever2d(nx: int = 1024, ny: int = 512, vol: float = 0.4, load_cells: int = 8,
                 precision: str = "f32") -> ProblemSpec:
    """2D cantilever: clamped left edge; unit downward traction over the ``load_cells``
    mid-height cell edges of the right edge, each edge's share split equally between its
    two end nodes (reading R16)."""
    assert ny % 2 == 0 and load_cells % 2 == 0 and load_cells <= ny
    j0 = ny // 2 - load_cells // 2
    per_edge = 1.0 / load_cells
    loads = {}
    for e in range(load_cells):
        for jj in (j0 + e, j0 + e + 1):
            loads[jj] = loads.get(jj, 0.0) + 0.5 * per_edge
    h_p = 1.0 / ny
    a, b, s1 = local_step_params(nx)
    tau, gg = ch_params(h_p, 2)
    return ProblemSpec(
        name=f"cantilever2d_{nx}x{ny}", dim=2, nx=nx, ny=ny, vol_frac=[vol],
        boxes=[((0, 0, 0), (0, ny, 0), 0b11)],
        loads=[((nx, jj, 0), 1, -v) for jj, v in sorted(loads.items())],
        phi0=_uniform_phi(nx * ny, [vol]),
        apt_a=a, apt_b=b, pt_s1=s1, tol=1e-6, tau=tau, gamma_g=gg, design_steps=200,
        precision=precision, storage=precision)


def heat2d(n: int = 1024, vol: float = 0.4, precision: str = "f32") -> ProblemSpec:
    """2D heat sink: k0 = 1, kmin = 1e-3, p = 3, uniform source 0.01 (Sec. 3.1), T = 0 on
    the nodes of the left edge with 0.45 <= j/n <= 0.55 (reading R16)."""
    j_lo = math.ceil(0.45 * n - 1e-9)
    j_hi = math.floor(0.55 * n + 1e-9)
    h_p = 1.0 / n
    a, b, s1 = local_step_params(n)
    tau, gg = ch_params(h_p, 2)
    return ProblemSpec(
        name=f"heat2d_{n}x{n}", dim=2, nx=n, ny=n, physics=THERMAL, moduli=[1.0], e_min=1e-3,
        vol_frac=[vol], boxes=[((0, j_lo, 0), (0, j_hi, 0), 0b1)], body_source=0.01,
        phi0=_uniform_phi(n * n, [vol]),
        apt_a=a, apt_b=b, pt_s1=s1, tol=1e-6, tau=tau, gamma_g=gg, design_steps=200,
        precision=precision, storage=precision)


def _line_load_3d(nx: int, ny: int, js=None):
    """Unit downward (-z) line load along the bottom edge (k = 0) of the x = nx face;
    equal share per edge segment, end nodes half weight (reading R16)."""
    loads = []
    for j in range(ny + 1):
        w = 1.0 / ny * (0.5 if j in (0, ny) else 1.0)
        loads.append(((nx, j, 0), 2, -w))
    return loads


def cantilever3d(nx: int = 256, ny: int = 128, nz: int = 128, vol: float = 0.12,
                 precision: str = "f32") -> ProblemSpec:
    """3D cantilever: clamped x = 0 face, unit downward line load along the bottom edge of
    the x = L face, E0 = 1, Emin = 1e-9, nu = 0.3, p = 3."""
    h_p = 2.0 / nx
    a, b, s1 = local_step_params(nx)
    tau, gg = ch_params(h_p, 3)
    return ProblemSpec(
        name=f"cantilever3d_{nx}x{ny}x{nz}", dim=3, nx=nx, ny=ny, nz=nz, vol_frac=[vol],
        boxes=[((0, 0, 0), (0, ny, nz), 0b111)], loads=_line_load_3d(nx, ny),
        phi0=_uniform_phi(nx * ny * nz, [vol]),
        apt_a=a, apt_b=b, pt_s1=s1, tol=1e-6, tau=tau, gamma_g=gg, design_steps=50,
        precision=precision, storage=precision)


def mbb_multimat2d(nx: int = 512, ny: int = 128, precision: str = "f32") -> ProblemSpec:
    """The paper's own multi-material MBB loop (Sec. 3.2): a 4 x 1 domain (nx = 4 ny cells),
    both bottom corners on rollers (u_y = 0), a unit downward load at the top-centre node,
    five materials E = [1.0, 0.775, 0.55, 0.325, 0.1] with V = 0.08 each plus an explicit
    void phase (E = 1e-6, V = 0.6), E = sum_i E_i phi_i^3, every phase starting at 0.5.
    Each loop: 20 APT then 20 PT sweeps with the paper's global steps (dt2 = dx/2,
    theta = 1, dt1 = dx^2/4; no local steps, fixed damping), the penalty update with
    alpha_h = 0.1, alpha_v = 1e4, alpha_1 = 1e3 (reading R7: kappa = 2 alpha / N_cells), and
    one Cahn-Hilliard step with dt3 = 500 dx^4, gamma = 3e-5.  The paper's grid is written
    "513 x 128"; 512 x 128 cells give its 4 : 1 aspect ratio at dx = 1/128."""
    h_p = 1.0 / ny
    a, b, s1 = apt_params(h_p, elastic=True, dim=2)
    tau, gg = ch_params(h_p, 2)
    moduli = [1e-6, 1.0, 0.775, 0.55, 0.325, 0.1]
    fr = [0.6, 0.08, 0.08, 0.08, 0.08, 0.08]
    n = nx * ny
    return ProblemSpec(
        name=f"mbb_multimat2d_{nx}x{ny}", dim=2, nx=nx, ny=ny, moduli=moduli, e_min=0.0, interp=SIMP_PAPER,
        vol_frac=fr, boxes=[((0, 0, 0), (0, 0, 0), 0b10), ((nx, 0, 0), (nx, 0, 0), 0b10)],
        loads=[((nx // 2, ny, 0), 1, -1.0)], phi0=np.full((len(fr), n), 0.5),
        apt_a=a, apt_b=b, pt_s1=s1, local_dt=False, momentum=0, solve_mode=0, n_apt=20, n_pt=20,
        check_every=0, vol_mode=PENALTY, alpha_h=0.1, kappa_v=2.0 * 1e4 / n, kappa_1=2.0 * 1e3 / n,
        tau=tau, gamma_g=gg, design_steps=200, precision=precision, storage=precision)


def heat2d_paper(n: int = 512, precision: str = "f32") -> ProblemSpec:
    """The paper's heat-conduction loop (Sec. 3.1): n x n cells, T = 0 on the top and left
    sides, no flux elsewhere, uniform source f = 0.01, one conductor (kappa = 1) with an
    explicit void phase (kappa = 1e-6), solid fraction 0.3, kappa = sum_i kappa_i phi_i^3,
    both phases starting at 1.0.  Each loop: 500 APT then 500 PT sweeps with the paper's
    global steps (thermal form, dt2 = dx/2, theta = 1, dt1 = dx^2/4), the penalty update with
    alpha_h = 0.1, alpha_v = 1e5, alpha_1 = 1e4 (reading R7), one Cahn-Hilliard step with
    dt3 = 500 dx^4.  Grid units with dx = 1/n (reading R12: the printed L = 4 is garbled)."""
    h_p = 1.0 / n
    a, b, s1 = apt_params(h_p, elastic=False, dim=2)
    tau, gg = ch_params(h_p, 2)
    fr = [0.7, 0.3]
    nc = n * n
    return ProblemSpec(
        name=f"heat2d_paper_{n}", dim=2, nx=n, ny=n, physics=THERMAL, moduli=[1e-6, 1.0], e_min=0.0,
        interp=SIMP_PAPER, vol_frac=fr, body_source=0.01,
        boxes=[((0, 0, 0), (0, n, 0), 1), ((0, n, 0), (n, n, 0), 1)], phi0=np.full((2, nc), 1.0),
        apt_a=a, apt_b=b, pt_s1=s1, local_dt=False, momentum=0, solve_mode=0, n_apt=500, n_pt=500,
        check_every=0, vol_mode=PENALTY, alpha_h=0.1, kappa_v=2.0 * 1e5 / nc, kappa_1=2.0 * 1e4 / nc,
        tau=tau, gamma_g=gg, design_steps=5000, precision=precision, storage=precision)


def multimat3d_paper(nx: int = 256, ny: int = 17, nz: int = 85, precision: str = "f32") -> ProblemSpec:
    """The paper's 3D multi-material cantilever loop (Sec. 3.3): 256 x 17 x 85 cells of size
    1/128 (2 x 2/15 x 2/3), the x = L face fixed, a unit force in +z spread along the
    horizontal centre line of the x = 0 face (nodes (0, j, nz/2), end nodes half weight;
    reading R24), three materials E = 1.0, 0.6, 0.2 with V = 0.1 each plus a void phase
    (E = 1e-6, V = 0.7).  Each loop: 100 APT then 100 PT sweeps with the paper's global
    steps (dt2 = dx/2, dt1 = dx^2/6), the penalty update with the MBB weights
    (alpha_v = 1e4, alpha_1 = 1e3), one Cahn-Hilliard step (dt3 = 500 dx^4)."""
    h_p = 1.0 / 128.0
    a, b, s1 = apt_params(h_p, elastic=True, dim=3)
    tau, gg = ch_params(h_p, 3)
    fr = [0.7, 0.1, 0.1, 0.1]
    n = nx * ny * nz
    kz = nz // 2
    w = [0.5 if j in (0, ny) else 1.0 for j in range(ny + 1)]
    tot = sum(w)
    return ProblemSpec(
        name=f"multimat3d_paper_{nx}x{ny}x{nz}", dim=3, nx=nx, ny=ny, nz=nz, moduli=[1e-6, 1.0, 0.6, 0.2],
        e_min=0.0, interp=SIMP_PAPER, vol_frac=fr, boxes=[((nx, 0, 0), (nx, ny, nz), 0b111)],
        loads=[((0, j, kz), 2, w[j] / tot) for j in range(ny + 1)], phi0=_uniform_phi(n, fr),
        apt_a=a, apt_b=b, pt_s1=s1, local_dt=False, momentum=0, solve_mode=0, n_apt=100, n_pt=100,
        check_every=0, vol_mode=PENALTY, alpha_h=0.1, kappa_v=2.0 * 1e4 / n, kappa_1=2.0 * 1e3 / n,
        tau=tau, gamma_g=gg, design_steps=4000, precision=precision, storage=precision)


def drone3d(nx: int = 128, ny: int = 64, nz: int = 128, vol: float = 0.12, precision: str = "f32") -> ProblemSpec:
    """The drone skeleton (Sec. 3.4): a 1.0 x 0.5 x 1.0 box (y vertical) on nx x ny x nz
    cells, rollers (u_y = 0) at the four top corners, a unit downward point load at the
    centre of the bottom face, one solid (E = 1) with an explicit void phase (E = 1e-6),
    solid fraction ``vol``.  A keep-out region must stay void: J_b with targets 1 (void) and
    0 (solid); the region is proposed here (the paper's figure is missing): the central
    quarter in x and z, the middle half in y.  Each loop: 50 APT then 50 PT sweeps with the
    paper's global steps, the penalty update with the MBB weights (alpha_v = 1e4,
    alpha_1 = 1e3) and alpha_b = alpha_v (reading R23), one Cahn-Hilliard step."""
    h_p = 1.0 / nx
    a, b, s1 = apt_params(h_p, elastic=True, dim=3)
    tau, gg = ch_params(h_p, 3)
    n = nx * ny * nz
    fr = [1.0 - vol, vol]
    lo = (3 * nx // 8, ny // 4, 3 * nz // 8)
    hi = (5 * nx // 8 - 1, 3 * ny // 4 - 1, 5 * nz // 8 - 1)
    nb = (hi[0] - lo[0] + 1) * (hi[1] - lo[1] + 1) * (hi[2] - lo[2] + 1)
    corners = [(0, ny, 0), (nx, ny, 0), (0, ny, nz), (nx, ny, nz)]
    return ProblemSpec(
        name=f"drone3d_{nx}x{ny}x{nz}", dim=3, nx=nx, ny=ny, nz=nz, moduli=[1e-6, 1.0], e_min=0.0,
        interp=SIMP_PAPER, vol_frac=fr, boxes=[(c, c, 0b010) for c in corners],
        loads=[((nx // 2, 0, nz // 2), 1, -1.0)], phi0=_uniform_phi(n, fr),
        apt_a=a, apt_b=b, pt_s1=s1, local_dt=False, momentum=0, solve_mode=0, n_apt=50, n_pt=50,
        check_every=0, vol_mode=PENALTY, alpha_h=0.1, kappa_v=2.0 * 1e4 / n, kappa_1=2.0 * 1e3 / n,
        keepout=(lo, hi), keepout_target=[1.0, 0.0], kappa_b=2.0 * 1e4 / nb,
        tau=tau, gamma_g=gg, design_steps=40000, precision=precision, storage=precision)


def multimat3d(nx: int = 384, ny: int = 192, nz: int = 192, storage: str = "bf16") -> ProblemSpec:
    """3D multi-material cantilever: phases (void, E = 1, E = 0.5) with volume fractions
    (0.8, 0.1, 0.1), paper interpolation E = sum_i E_i rho_i^p with the void modulus 1e-9
    (Sec. 3.3 uses three solids plus a soft void phase); BCs and load as the cantilever."""
    base = cantilever3d(nx, ny, nz)
    fr = [0.8, 0.1, 0.1]
    return base.with_(name=f"multimat3d_{nx}x{ny}x{nz}_{storage}", moduli=[1e-9, 1.0, 0.5],
                      interp=SIMP_PAPER, vol_frac=fr, phi0=_uniform_phi(nx * ny * nz, fr),
                      kappa_1=0.0, storage=storage)


def batch2d(n_instances: int = 48, seed: int = 5, lo: int = 128, hi_factor: float = 8.0) -> list:
    """Batched 2D instances: n_x = 128 * 8^U rounded to a multiple of 8 (so 128..1024),
    n_y = n_x / 2; cantilever or MBB half-beam by a fair coin; V ~ U[0.3, 0.5]; the load
    node drawn uniformly along the loaded edge (PCG64 ``seed``)."""
    rng = np.random.default_rng(seed)
    out = []
    for t in range(n_instances):
        nx = int(round(lo * hi_factor ** rng.uniform()) / 8.0) * 8
        nx = max(lo, min(int(lo * hi_factor), nx))
        ny = nx // 2
        vol = float(rng.uniform(0.3, 0.5))
        cant = bool(rng.integers(0, 2))
        j = int(rng.integers(0, ny + 1))
        h_p = 1.0 / ny
        a, b, s1 = local_step_params(nx)
        tau, gg = ch_params(h_p, 2)
        if cant:
            boxes = [((0, 0, 0), (0, ny, 0), 0b11)]
            loads = [((nx, j, 0), 1, -1.0)]
        else:
            boxes = [((0, 0, 0), (0, ny, 0), 0b01), ((nx, 0, 0), (nx, 0, 0), 0b10)]
            loads = [((0, max(j, ny // 2), 0), 1, -1.0)]
        out.append(ProblemSpec(
            name=f"batch{t}_{'cant' if cant else 'mbb'}_{nx}x{ny}", dim=2, nx=nx, ny=ny, vol_frac=[vol],
            boxes=boxes, loads=loads, phi0=_uniform_phi(nx * ny, [vol]),
            apt_a=a, apt_b=b, pt_s1=s1, tol=1e-6, tau=tau, gamma_g=gg))
    return out


def multirhs3d(nx: int = 192, ny: int = 96, nz: int = 96, n_rhs: int = 4, seed: int = 5):
    """3D cantilever with ``n_rhs`` unit downward point-load cases at seeded nodes on the
    bottom edge of the x = L face.  Returns (spec without loads, list of load lists)."""
    rng = np.random.default_rng(seed)
    base = cantilever3d(nx, ny, nz)
    js = rng.integers(0, ny + 1, size=n_rhs)
    cases = [[((nx, int(j), 0), 2, -1.0)] for j in js]
    return base.with_(name=f"multirhs3d_{nx}x{ny}x{nz}_r{n_rhs}", loads=cases[0]), cases


def random_design(spec: ProblemSpec, seed: int, lo: float = 0.05, hi: float = 0.95) -> np.ndarray:
    """A seeded non-uniform design field [P, cells] in [lo, hi] for operator tests."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=(spec.n_phases, spec.ncells))


def random_state(spec: ProblemSpec, seed: int, scale: float = 1.0) -> np.ndarray:
    """A seeded nodal field [ncomp, nodes] (node (i,j,k) -> i + (nx+1)(j + (ny+1)k))."""
    rng = np.random.default_rng(seed)
    return scale * rng.standard_normal(size=(spec.ncomp, spec.nnodes))


CONFIGS = {
    "mbb60x20_f64": lambda: mbb_halfbeam(),
    "cantilever2d_1024x512": lambda: cantilever2d(),
    "heat2d_1024": lambda: heat2d(),
    "cantilever3d_256x128x128": lambda: cantilever3d(),
    "multimat3d_384x192x192_bf16": lambda: multimat3d(storage="bf16"),
    "multimat3d_384x192x192_f16": lambda: multimat3d(storage="f16"),
}
