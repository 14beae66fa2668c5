"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed-form
solutions, convergence order, a direct sparse solve, energy identities, symmetry,
finite differences, exact piecewise-linear roots, and the paper's own discrete
equations (PeTTO, arXiv 2509.06971: Sec. 2.2 PT/APT, Sec. 2.3 J_v/J_1, Sec. 2.4 CH,
Sec. 3.2 stress law / PT / APT systems).  A plausible slip in the oracle (a dropped
term, a wrong sign, a transposed index) fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2509_06971_gb300 import workloads as W
from tests._util import node_coords, oracle_materials, oracle_problem

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _lame(nu):
    return nu / ((1 + nu) * (1 - 2 * nu)), 1 / (2 * (1 + nu))


# ----------------------------------------------------------------- operator

@pytest.mark.parametrize("dim,shape,phys,nullity", [
    (2, (5, 4, 0), O.ELASTIC, 3), (3, (3, 3, 2), O.ELASTIC, 6),
    (2, (5, 4, 0), O.THERMAL, 1), (3, (3, 3, 2), O.THERMAL, 1)])
def test_only_rigid_modes(dim, shape, phys, nullity):
    """K(E) with no supports has exactly the rigid-body null space: no hourglass modes."""
    p = O.OracleProblem(dim, *shape, physics=phys)
    E = np.random.default_rng(3).uniform(0.1, 1.0, p.ncells)
    K = p.assemble_K(E).toarray()
    assert np.abs(K - K.T).max() < 1e-14
    ev = np.linalg.eigvalsh(K)
    assert int(np.sum(np.abs(ev) < 1e-10 * ev[-1])) == nullity
    assert ev.min() > -1e-12


def test_apply_matches_assembly_and_diag():
    p = O.OracleProblem(3, 4, 3, 2)
    rng = np.random.default_rng(0)
    E = rng.uniform(0.1, 1, p.ncells)
    u = rng.standard_normal(p.ndof)
    K = p.assemble_K(E)
    assert np.allclose(K @ u, p.apply_K(E, u), rtol=0, atol=1e-12)
    assert np.allclose(K.diagonal(), p.diag_K(E), rtol=1e-14)


@pytest.mark.parametrize("dim", [2, 3])
def test_uniaxial_bar_closed_form(dim):
    """Bar on symmetry rollers pulled by a uniform traction t on x = L: the discrete
    solution is the continuum one (plane strain in 2D, Sec. 3.2 stress law):
    2D: u_x = t(1-nu^2)x/E, u_y = -t nu (1+nu) y/E;  3D: u_x = tx/E, u_y,z = -nu t y,z/E."""
    nx, ny, nz = (8, 5, 0) if dim == 2 else (5, 3, 4)
    Em, t, nu = 2.5, 0.7, 0.3
    h = 0.5
    boxes = [((0, 0, 0), (0, ny, nz), 0b001), ((0, 0, 0), (nx, 0, nz), 0b010)]
    if dim == 3:
        boxes.append(((0, 0, 0), (nx, ny, 0), 0b100))
    # traction t on the x = L face, each boundary cell face's force t h^(d-1) split equally
    loads = {}
    faces = [(j, k) for j in range(ny) for k in range(nz if dim == 3 else 1)]
    for (j, k) in faces:
        corners = [(j + dj, k + dk) for dj in (0, 1) for dk in ((0, 1) if dim == 3 else (0,))]
        for c in corners:
            loads[c] = loads.get(c, 0.0) + t * h ** (dim - 1) / len(corners)
    p = O.OracleProblem(dim, nx, ny, nz, h=h, nu=nu, boxes=boxes,
                        loads=[((nx, j, k), 0, v) for (j, k), v in loads.items()])
    E = np.full(p.ncells, Em)
    u = p.direct_solve(E, p.load_vector(), p.fixed_mask()).reshape(-1, dim)
    X = node_coords(p)
    if dim == 2:
        exact = np.stack([t * (1 - nu ** 2) * X[:, 0] / Em, -t * nu * (1 + nu) * X[:, 1] / Em], 1)
    else:
        exact = np.stack([t * X[:, 0] / Em, -nu * t * X[:, 1] / Em, -nu * t * X[:, 2] / Em], 1)
    assert np.abs(u - exact).max() <= 1e-12 * np.abs(exact).max()
    # golden fixture: the closed form at the far corner node
    g = json.load(open(os.path.join(GOLDEN, "uniaxial_bar.json")))[f"{dim}d"]
    far = p.node_id(nx, ny, nz if dim == 3 else 0)
    assert np.allclose(u[far], g["far_corner_u"], rtol=1e-12, atol=0)


def test_thermal_quadratic_exact():
    """T = 0 on x = 0, insulated elsewhere, uniform kappa and source f: the nodal values
    equal T = f x (2L - x) / (2 kappa) exactly (Sec. 2.2 Poisson equation)."""
    nx, ny, f, kap, h = 10, 4, 0.01, 2.0, 0.25
    p = O.OracleProblem(2, nx, ny, physics=O.THERMAL, body_source=f, h=h,
                        boxes=[((0, 0, 0), (0, ny, 0), 1)])
    T = p.direct_solve(np.full(p.ncells, kap), p.load_vector(), p.fixed_mask())
    x = node_coords(p)[:, 0]
    L = nx * h
    exact = f * x * (2 * L - x) / (2 * kap)
    assert np.abs(T - exact).max() <= 1e-12 * exact.max()


def _mms_error(dim, n):
    sp = pytest.importorskip("sympy")
    x, y, z = sp.symbols("x y z")
    X = [x, y, z][:dim]
    lam, mu = _lame(0.3)
    if dim == 2:
        U = [sp.sin(sp.pi * x) * sp.sin(sp.pi * y), sp.sin(2 * sp.pi * x) * sp.sin(sp.pi * y) / 2]
        Ef = 1 + sp.sin(sp.pi * x) * sp.cos(sp.pi * y / 2) / 2 + x * y
    else:
        U = [sp.sin(sp.pi * x) * sp.sin(sp.pi * y) * sp.sin(sp.pi * z),
             sp.sin(2 * sp.pi * x) * sp.sin(sp.pi * y) * sp.sin(sp.pi * z) / 2,
             sp.sin(sp.pi * x) * sp.sin(2 * sp.pi * y) * sp.sin(sp.pi * z) / 3]
        Ef = 1 + sp.sin(sp.pi * x) * sp.cos(sp.pi * y / 2) / 2 + x * y * z
    eps = [[(sp.diff(U[a], X[b]) + sp.diff(U[b], X[a])) / 2 for b in range(dim)] for a in range(dim)]
    tr = sum(eps[a][a] for a in range(dim))
    sig = [[Ef * (lam * tr * int(a == b) + 2 * mu * eps[a][b]) for b in range(dim)] for a in range(dim)]
    f = [-sum(sp.diff(sig[a][b], X[b]) for b in range(dim)) for a in range(dim)]
    fl = [sp.lambdify(X, fa, "numpy") for fa in f]
    ul = [sp.lambdify(X, ua, "numpy") for ua in U]
    El = sp.lambdify(X, Ef, "numpy")
    h = 1.0 / n
    p = O.OracleProblem(dim, n, n, n if dim == 3 else 0, h=h)
    N = node_coords(p)
    nzc = n if dim == 3 else 1
    kc, jc, ic = np.meshgrid(np.arange(nzc), np.arange(n), np.arange(n), indexing="ij")
    C = (np.stack([ic.reshape(-1), jc.reshape(-1), kc.reshape(-1)], 1) + 0.5) * h
    E = El(*[C[:, i] for i in range(dim)]) * np.ones(len(C))
    F = np.stack([fl[a](*[N[:, i] for i in range(dim)]) * np.ones(len(N)) for a in range(dim)], 1).reshape(-1) * h ** dim
    us = np.stack([ul[a](*[N[:, i] for i in range(dim)]) * np.ones(len(N)) for a in range(dim)], 1).reshape(-1)
    bd = np.any((N[:, :dim] < 1e-12) | (N[:, :dim] > 1 - 1e-12), axis=1)
    fixed = np.repeat(bd, dim).astype(np.uint8)
    F[fixed == 1] = 0
    return np.abs(p.direct_solve(E, F, fixed) - us).max()


@pytest.mark.parametrize("dim,ns", [(2, [8, 16, 32]), (3, [4, 8, 16])])
def test_manufactured_solution_second_order(dim, ns):
    """Smooth u* and smooth E(x) with the body force of the continuum operator (Sec. 3.2
    momentum balance and stress law): the nodal error falls at order >= 1.9."""
    errs = [_mms_error(dim, n) for n in ns]
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert min(orders) >= 1.9, (errs, orders)


def test_mirror_symmetry_full_mbb():
    """Full-span MBB with a centre load and rollers at both bottom corners (Sec. 3.2 setup):
    u_x is odd and u_y even about the centre line, and the sensitivity is mirrored."""
    nx, ny = 16, 6
    p = O.OracleProblem(2, nx, ny, boxes=[((0, 0, 0), (0, 0, 0), 0b11), ((nx, 0, 0), (nx, 0, 0), 0b10)],
                        loads=[((nx // 2, ny, 0), 1, -1.0)])
    # pin u_x at the left support only; a mirror-symmetric problem needs symmetric supports,
    # so use the symmetric pair (u_y on both) plus u_x on the centre-bottom node instead.
    p = O.OracleProblem(2, nx, ny, boxes=[((0, 0, 0), (0, 0, 0), 0b10), ((nx, 0, 0), (nx, 0, 0), 0b10),
                                          ((nx // 2, 0, 0), (nx // 2, 0, 0), 0b01)],
                        loads=[((nx // 2, ny, 0), 1, -1.0)])
    rng = np.random.default_rng(7)
    half = rng.uniform(0.2, 1.0, (ny, nx // 2))
    Ecell = np.concatenate([half, half[:, ::-1]], axis=1).reshape(-1)
    u = p.direct_solve(Ecell, p.load_vector(), p.fixed_mask()).reshape(ny + 1, nx + 1, 2)
    assert np.abs(u[:, :, 0] + u[:, ::-1, 0]).max() < 1e-12 * np.abs(u).max()
    assert np.abs(u[:, :, 1] - u[:, ::-1, 1]).max() < 1e-12 * np.abs(u).max()
    e = p.cell_energy(u.reshape(-1)).reshape(ny, nx)
    assert np.abs(e - e[:, ::-1]).max() < 1e-12 * e.max()


# ------------------------------------------------------------ solvers

def _small_cantilever(dim):
    spec = W.cantilever2d(12, 6, load_cells=2) if dim == 2 else W.cantilever3d(6, 4, 4)
    p = oracle_problem(spec)
    E = np.random.default_rng(11).uniform(0.2, 1.0, p.ncells)
    return p, E


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("kind", ["apt_global", "apt_local", "apt_adaptive", "pt_local"])
def test_iterations_converge_to_direct_solve(dim, kind):
    """PT and APT fixed points are K u = F: the converged field equals a sparse direct
    solve of the assembled K within 1e-8 relative."""
    p, E = _small_cantilever(dim)
    F, fixed = p.load_vector(), p.fixed_mask()
    ud = p.direct_solve(E, F, fixed)
    u = np.zeros(p.ndof)
    if kind == "apt_global":
        rep = p.solve(E, F, fixed, u, mode=1, a=0.97, b=0.2, tol=1e-12, max_sweeps=400000, check_every=10)
    elif kind == "apt_local":
        rep = p.solve(E, F, fixed, u, mode=1, a=0.97, b=1.0, tol=1e-12, max_sweeps=400000, check_every=10,
                      local_dt=True)
    elif kind == "apt_adaptive":
        rep = p.solve(E, F, fixed, u, mode=1, a=1.0, b=0.9, tol=1e-12, max_sweeps=400000, check_every=10,
                      local_dt=True, momentum=1)
    else:
        rep = p.solve(E, F, fixed, u, mode=0, n_apt=0, n_pt=400000, s1=0.75, check_every=0, local_dt=True)
    assert rep["fell_back_to_pt"] is False
    assert np.abs(u - ud).max() <= 1e-8 * np.abs(ud).max()


def test_energy_equals_external_work():
    """Compliance sum_c E_c e_c (Sec. 3.2 J_m) equals F.u at the solution of K u = F."""
    for dim in (2, 3):
        p, E = _small_cantilever(dim)
        F = p.load_vector()
        u = p.direct_solve(E, F, p.fixed_mask())
        C = float(np.dot(E, p.cell_energy(u)))
        assert abs(C - F @ u) <= 1e-10 * abs(C)


def test_sweeps_satisfy_paper_discrete_equations():
    """Three consecutive oracle states satisfy the paper's discrete PT / APT equations:
    elastic APT  theta (u+ - 2u + u-)/dt^2 + (u+ - u)/dt = R(u)/h^d   (Sec. 3.2 APT system)
    thermal APT  theta (T+ - 2T + T-)/dt^2 + (T - T-)/dt = R(T)/h^d   (Sec. 2.2 damped wave)
    PT           (u+ - u)/dt1 = R(u)/h^d                             (Sec. 2.2, Sec. 3.2 PT)."""
    theta, h = 1.3, 0.5
    dt2 = 0.37
    for phys in (O.ELASTIC, O.THERMAL):
        p = O.OracleProblem(2, 5, 4, h=h, physics=phys, boxes=[((0, 0, 0), (0, 4, 0), 0b11)],
                            loads=[((5, 2, 0), phys == O.ELASTIC and 1 or 0, -1.0)])
        E = np.random.default_rng(2).uniform(0.3, 1, p.ncells)
        F, fixed = p.load_vector(), p.fixed_mask()
        if phys == O.ELASTIC:
            a, b = theta / (theta + dt2), dt2 ** 2 / ((theta + dt2) * h ** 2)
        else:
            a, b = 1 - dt2 / theta, dt2 ** 2 / (theta * h ** 2)
        rng = np.random.default_rng(4)
        u_prev = rng.standard_normal(p.ndof) * (1 - fixed)
        u = u_prev + 0.1 * rng.standard_normal(p.ndof) * (1 - fixed)
        w = u - u_prev
        R, _ = p.residual(E, F, fixed, u)
        u_new, w_new = u.copy(), w.copy()
        p.apt_sweep(E, F, fixed, a, b, u_new, w_new)
        if phys == O.ELASTIC:
            lhs = theta * (u_new - 2 * u + u_prev) / dt2 ** 2 + (u_new - u) / dt2
        else:
            lhs = theta * (u_new - 2 * u + u_prev) / dt2 ** 2 + (u - u_prev) / dt2
        free = fixed == 0
        assert np.abs(lhs[free] - R[free] / h ** 2).max() <= 1e-11 * np.abs(R).max()
        dt1 = h * h / 4
        u_pt = u.copy()
        p.pt_sweep(E, F, fixed, dt1 / h ** 2, u_pt)
        assert np.abs((u_pt - u)[free] / dt1 - R[free] / h ** 2).max() <= 1e-11 * np.abs(R).max()


def test_grid_unit_parameters_reproduce_paper_units():
    """The grid-unit constants of the workloads (a, b, s1) give the same iteration as the
    paper's constants written in its own units (theta = 1, dt2 = dx/2, dt1 = dx^2/4,
    Sec. 3.1/3.2; golden fixture of the paper's constants)."""
    g = json.load(open(os.path.join(GOLDEN, "paper_constants.json")))
    h_p = 1.0 / 128
    p_phys = O.OracleProblem(2, 6, 4, h=h_p, boxes=[((0, 0, 0), (0, 4, 0), 0b11)], loads=[((6, 2, 0), 1, -1.0)])
    p_grid = O.OracleProblem(2, 6, 4, h=1.0, boxes=p_phys.boxes, loads=p_phys.loads)
    E = np.random.default_rng(5).uniform(0.3, 1, p_phys.ncells)
    F, fixed = p_phys.load_vector(), p_phys.fixed_mask()
    theta = g["mbb"]["theta"]
    dt2 = g["mbb"]["dt2_over_dx"] * h_p
    a_p, b_p = theta / (theta + dt2), dt2 ** 2 / ((theta + dt2) * h_p ** 2)
    a_g, b_g, s1_g = W.apt_params(h_p, elastic=True, dim=2)
    u1, w1 = np.zeros(p_phys.ndof), np.zeros(p_phys.ndof)
    u2, w2 = u1.copy(), w1.copy()
    for _ in range(7):
        p_phys.apt_sweep(E, F, fixed, a_p, b_p, u1, w1)
        p_grid.apt_sweep(E, F, fixed, a_g, b_g, u2, w2)
    assert np.allclose(u1, u2, rtol=1e-13, atol=1e-15)
    dt1 = g["mbb"]["dt1_over_dx2"] * h_p ** 2
    assert abs(s1_g - dt1 / h_p ** 2) < 1e-15
    # 3D: dt1 = dx^2/6 (Sec. 3.3)
    assert abs(W.apt_params(h_p, dim=3)[2] - g["cantilever3d"]["dt1_over_dx2"]) < 1e-15


# ------------------------------------------------------ design sensitivities

@pytest.mark.parametrize("case", ["simp2d", "simp3d", "paper3phase2d", "thermal2d"])
def test_sensitivity_central_differences(case):
    """dC/dphi from the oracle's adjoint formula equals central finite differences of the
    compliance C(phi) = F.u(phi) (each C from a direct solve), delta = 1e-4, on seeded cells."""
    if case == "simp2d":
        spec = W.mbb_halfbeam(10, 5)
    elif case == "simp3d":
        spec = W.cantilever3d(6, 3, 3)
    elif case == "paper3phase2d":
        spec = W.cantilever2d(10, 4, load_cells=2).with_(moduli=[0.05, 1.0, 0.5], interp=W.SIMP_PAPER,
                                                          vol_frac=[0.6, 0.2, 0.2])
    else:
        spec = W.heat2d(8).with_(boxes=[((0, 3, 0), (0, 5, 0), 1)])
    p, mat = oracle_problem(spec), oracle_materials(spec)
    F, fixed = p.load_vector(), p.fixed_mask()
    phi = W.random_design(spec, seed=9, lo=0.1, hi=0.9)

    def comp(ph):
        u = p.direct_solve(mat.modulus(ph), F, fixed)
        return float(F @ u), u

    C0, u0 = comp(phi)
    E = mat.modulus(phi)
    s, C = mat.sensitivity(phi, E, p.cell_energy(u0))
    assert abs(C - C0) <= 1e-9 * abs(C0)
    rng = np.random.default_rng(32)
    delta = 1e-4
    for _ in range(8):
        i = int(rng.integers(0, spec.n_phases))
        c = int(rng.integers(0, spec.ncells))
        pp, pm = phi.copy(), phi.copy()
        pp[i, c] += delta
        pm[i, c] -= delta
        fd = (comp(pp)[0] - comp(pm)[0]) / (2 * delta)
        assert abs(fd - s[i, c]) <= 1e-5 * abs(s[i, c]) + 1e-12 * abs(C0), (i, c, fd, s[i, c])


def test_material_interpolation_end_points():
    """Modified SIMP: E(0) = Emin, E(1) = E0; paper form: E = sum_i E_i phi_i^p (Sec. 3.2)."""
    m = O.OracleMaterials([2.0], 1e-9, 3.0, O.SIMP_MODIFIED)
    E = m.modulus(np.array([[0.0, 1.0, 0.5, -0.2, 1.3]]))
    assert np.allclose(E, [1e-9, 2.0, 1e-9 + 0.125 * (2.0 - 1e-9), 1e-9, 2.0], rtol=1e-15)
    mp = O.OracleMaterials([1e-6, 1.0, 0.5], 0.0, 3.0, O.SIMP_PAPER)
    phi = np.array([[0.2], [0.5], [0.3]])
    assert abs(mp.modulus(phi)[0] - (1e-6 * 0.008 + 0.125 + 0.5 * 0.027)) < 1e-15


# ------------------------------------------------------------ design update

def _exact_lambda(d, V):
    """Root of mean(clamp(d - lam, 0, 1)) = V by sorting the breakpoints (brute force)."""
    bps = np.unique(np.concatenate([d, d - 1.0]))
    f = lambda lam: np.clip(d - lam, 0, 1).mean() - V
    vals = np.array([f(b) for b in bps])
    k = np.flatnonzero((vals[:-1] >= 0) & (vals[1:] <= 0))[0]
    l0, l1, f0, f1 = bps[k], bps[k + 1], vals[k], vals[k + 1]
    return l0 if f0 == f1 else l0 + (l1 - l0) * f0 / (f0 - f1)


def test_projected_update_holds_volume():
    rng = np.random.default_rng(1)
    ncell = 500
    phi = rng.uniform(0, 1, (1, ncell))
    s = -rng.uniform(0, 3, (1, ncell))
    d = phi[0] - 0.1 * s[0] / np.abs(s).max()
    lam = O.update(phi, s, [0.37], alpha_h=0.1)
    assert abs(phi.mean() - 0.37) < 1e-13
    assert abs(lam[0] - _exact_lambda(d, 0.37)) < 1e-12
    assert phi.min() >= 0 and phi.max() <= 1


def test_penalty_update_is_gradient_of_volume_terms():
    """Penalty mode with alpha_h = 0 steps along -grad(alpha_v J_v + alpha_1 J_1) with
    J_v = sum_i (mean phi_i - V_i)^2, J_1 = mean_c (sum_i phi_i - 1)^2 (Sec. 2.3; reading R7:
    integrals over a unit-measure domain), checked by central differences."""
    rng = np.random.default_rng(2)
    P, N = 3, 40
    phi = rng.uniform(0, 1, (P, N))
    V = np.array([0.2, 0.3, 0.5])
    av, a1 = 0.7, 0.3

    def J(ph):
        return av * np.sum((ph.mean(axis=1) - V) ** 2) + a1 * np.mean((ph.sum(axis=0) - 1) ** 2)

    new = phi.copy()
    O.update(new, np.zeros((P, N)), V, vol_mode=O.PENALTY, alpha_h=0.0, kappa_v=2 * av / N, kappa_1=2 * a1 / N)
    step = phi - new
    for (i, c) in [(0, 3), (1, 17), (2, 39)]:
        e = np.zeros_like(phi)
        e[i, c] = 1e-6
        fd = (J(phi + e) - J(phi - e)) / 2e-6
        assert abs(step[i, c] - fd) < 1e-9


def test_keepout_term_is_gradient_of_void_region_constraint():
    """The keep-out term (Sec. 3.4): penalty mode with alpha_h = 0 steps along
    -grad(alpha_v J_v + alpha_1 J_1 + alpha_b J_b) with J_b = sum_i (mean over the region
    of phi_i - Vb_i)^2 (reading R23), checked by central differences inside and outside
    the region; in projected mode the term moves the region's density toward Vb."""
    rng = np.random.default_rng(4)
    P, N = 2, 48
    phi = rng.uniform(0, 1, (P, N))
    V = np.array([0.3, 0.7])
    Vb = np.array([0.0, 1.0])
    keep = np.zeros(N, bool)
    keep[10:22] = True
    av, a1, ab = 0.7, 0.3, 1.9
    nb = keep.sum()

    def J(ph):
        return (av * np.sum((ph.mean(axis=1) - V) ** 2) + a1 * np.mean((ph.sum(axis=0) - 1) ** 2)
                + ab * np.sum((ph[:, keep].mean(axis=1) - Vb) ** 2))

    new = phi.copy()
    O.update(new, np.zeros((P, N)), V, vol_mode=O.PENALTY, alpha_h=0.0, kappa_v=2 * av / N, kappa_1=2 * a1 / N,
             keepout=keep, Vb=Vb, kappa_b=2 * ab / nb)
    step = phi - new
    for (i, c) in [(0, 3), (1, 12), (0, 21), (1, 40)]:
        e = np.zeros_like(phi)
        e[i, c] = 1e-6
        fd = (J(phi + e) - J(phi - e)) / 2e-6
        assert abs(step[i, c] - fd) < 1e-9
    # projected mode: with a strong keep-out weight the region empties of phase 0
    ph = np.full((1, N), 0.5)
    O.update(ph, np.zeros((1, N)), [0.5], vol_mode=O.PROJECTED, alpha_h=0.0, keepout=keep, Vb=[0.0], kappa_b=2.0)
    assert ph[0, keep].max() < ph[0, ~keep].min()
    assert abs(ph.mean() - 0.5) < 1e-12


# ------------------------------------------------------------ phase field

def test_double_well():
    """w(phi) = sin^2(pi phi)/64 (Sec. 2.4): minima at 0 and 1, w' vanishes at 0, 1/2, 1,
    and the oracle's w' is the derivative of w."""
    for x in (0.0, 0.5, 1.0):
        assert abs(O.double_well_deriv(x)) < 1e-16
    assert O.double_well(0.0) == 0.0 and abs(O.double_well(1.0)) < 1e-32
    assert abs(O.double_well(0.5) - 1 / 64) < 1e-18
    for x in np.linspace(-0.3, 1.3, 17):
        fd = (O.double_well(x + 1e-6) - O.double_well(x - 1e-6)) / 2e-6
        assert abs(fd - O.double_well_deriv(x)) < 1e-10


def test_cell_laplacian_no_flux():
    """L is symmetric, sums to zero (no flux through the boundary), kills constants, and on
    a linear profile is zero inside and one-sided at the ends."""
    p = O.OracleProblem(3, 5, 4, 3)
    rng = np.random.default_rng(0)
    u, v = rng.standard_normal(p.ncells), rng.standard_normal(p.ncells)
    assert abs(u @ p.cell_laplacian(v) - v @ p.cell_laplacian(u)) < 1e-12
    assert abs(p.cell_laplacian(v).sum()) < 1e-12
    assert np.abs(p.cell_laplacian(np.ones(p.ncells))).max() == 0
    x = np.tile(np.arange(5.0), 4 * 3)
    Lx = p.cell_laplacian(x).reshape(3, 4, 5)
    assert np.abs(Lx[:, :, 1:4]).max() < 1e-14
    assert np.allclose(Lx[:, :, 0], 1.0) and np.allclose(Lx[:, :, 4], -1.0)


def test_cahn_hilliard_conserves_mass_and_separates():
    """The explicit CH step conserves sum phi exactly (no-flux BCs, Sec. 2.4) and drives a
    perturbed mixture toward the wells 0 and 1 (phase separation)."""
    spec = W.mbb_halfbeam(24, 12)
    p = oracle_problem(spec)
    rng = np.random.default_rng(3)
    phi = (0.5 + 0.05 * rng.standard_normal((1, p.ncells)))
    m0 = phi.sum()
    spread0 = np.abs(phi - 0.5).mean()
    for _ in range(400):
        p.ch_step(phi, spec.gamma_g, spec.tau)
    assert abs(phi.sum() - m0) < 1e-10
    assert np.abs(phi - 0.5).mean() > 4 * spread0


def test_design_loop_compliance_decreases():
    """Three PeTTO loops (Fig. 5) on a small MBB: volume held, compliance falls."""
    spec = W.mbb_halfbeam(12, 4)
    p, mat = oracle_problem(spec), oracle_materials(spec)
    F, fixed = p.load_vector(), p.fixed_mask()
    phi, u = spec.phi0.copy(), np.zeros(p.ndof)
    Cs = []
    for _ in range(4):
        m = O.design_step(p, mat, phi, u, F, fixed, spec.vol_frac,
                          dict(mode=1, a=1.0, b=0.9, s1=0.75, tol=1e-10, max_sweeps=200000, check_every=10,
                               local_dt=True, momentum=1),
                          dict(alpha_h=0.1, gamma_g=spec.gamma_g, tau=spec.tau))
        Cs.append(m["compliance"])
        assert abs(m["work"] - m["compliance"]) < 1e-8 * m["compliance"]
    assert Cs[-1] < Cs[0]


def _neumann_mode(shape, ks):
    """Eigenvector of the no-flux cell Laplacian (Sec. 2.4 boundary conditions): the tensor
    product of cos(pi k (i + 1/2) / n) over the axes, with eigenvalue
    -sum_a (2 - 2 cos(pi k_a / n_a))."""
    v = np.ones(1)
    lam = 0.0
    for n, k in zip(shape, ks):
        c = np.cos(math.pi * k * (np.arange(n) + 0.5) / n)
        v = np.multiply.outer(c, v)          # slowest axis outermost: [k][j][i]
        lam += 2.0 - 2.0 * math.cos(math.pi * k / n)
    return v.reshape(-1), lam


@pytest.mark.parametrize("dim,shape,modes", [
    (2, (24, 16), [(1, 0), (3, 2), (7, 5), (0, 15)]),
    (3, (10, 8, 6), [(1, 0, 0), (2, 3, 1), (5, 4, 3), (9, 7, 5)])])
def test_cahn_hilliard_linear_growth_factor(dim, shape, modes):
    """One explicit CH step (Sec. 2.4: mu = w'(phi) - gamma_g L phi, phi <- phi + tau L mu)
    on phi = 1/2 + eps v_k, v_k an eigenvector of the no-flux Laplacian (L v_k = -lam_k v_k),
    multiplies eps by exactly g_k = 1 - tau lam_k (w''(1/2) + gamma_g lam_k) up to O(eps^2)
    relative, with w''(1/2) = -2 pi^2 / 64 for the paper's double well sin^2(pi phi)/64.
    A wrong factor on gamma_g or tau, a sign slip in mu, or a mobility applied to the wrong
    term changes g_k for some of these modes by far more than the tolerance."""
    h_p = 1.0 / shape[1]
    tau, gg = W.ch_params(h_p, dim)
    p = O.OracleProblem(dim, *shape) if dim == 3 else O.OracleProblem(dim, shape[0], shape[1])
    wpp = -2.0 * math.pi ** 2 / 64.0
    eps = 1e-5
    for ks in modes:
        v, lam = _neumann_mode(shape, ks)
        assert np.allclose(p.cell_laplacian(v), -lam * v, atol=1e-12)
        phi = (0.5 + eps * v)[None, :].copy()
        p.ch_step(phi, gg, tau)
        g = 1.0 - tau * lam * (wpp + gg * lam)
        m = np.abs(v) > 0.05
        ratio = (phi[0, m] - 0.5) / (eps * v[m])
        assert np.abs(ratio - g).max() < 1e-8 * max(1.0, abs(g)), (ks, g, ratio.min(), ratio.max())


def test_ch_params_follow_the_paper_constants():
    """The grid-unit Cahn-Hilliard constants restate the paper's (Sec. 3.1: dt3 = 500 dx^4,
    gamma = 3e-5, D = 1): tau = D dt3 / h_p^2 = 500 h_p^2, gamma_g = gamma / h_p^2, unless tau
    exceeds 0.9 x the explicit bound tau (w''_max lam_L + gamma_g lam_L^2) <= 2 (reading R10),
    lam_L = 4 d the largest eigenvalue of the no-flux Laplacian's bound, w''_max = 2 pi^2/64."""
    with open(os.path.join(GOLDEN, "paper_constants.json")) as f:
        pc = json.load(f)["heat2d"]
    dt3, gamma = pc["dt3_over_dx4"], pc["gamma"]
    wpp_max = max(abs(O.double_well_deriv(x + 1e-6) - O.double_well_deriv(x - 1e-6)) / 2e-6
                  for x in np.linspace(0, 1, 201))
    assert abs(wpp_max - 2 * math.pi ** 2 / 64) < 1e-6
    for dim in (2, 3):
        for n in (8, 20, 64, 128, 512, 1024):
            h_p = 1.0 / n
            tau, gg = W.ch_params(h_p, dim)
            assert gg == pytest.approx(gamma / h_p ** 2, rel=1e-15)
            lam_l = 4.0 * dim
            bound = 2.0 / (wpp_max * lam_l + gg * lam_l ** 2)
            paper_tau = dt3 * h_p ** 4 / h_p ** 2
            if paper_tau <= 0.9 * bound * (1 - 1e-9):
                assert tau == pytest.approx(paper_tau, rel=1e-15)
            else:
                assert tau == pytest.approx(0.9 * bound, rel=1e-6)
            # the explicit step is stable on the Laplacian's actual largest eigenvalue
            assert tau * (wpp_max * lam_l + gg * lam_l ** 2) <= 1.8 + 1e-9
    # the product tau gamma_g of the paper's constants is scale free (Sec. 3.1: 0.015)
    tau, gg = W.ch_params(1.0 / 512, 2)
    assert tau * gg == pytest.approx(dt3 * gamma, rel=1e-12)


@pytest.mark.parametrize("dim,shape", [(2, (12, 6, 0)), (3, (6, 4, 3))])
def test_local_step_params_are_inside_the_stability_bound(dim, shape):
    """Local pseudo-time steps (reading R19) scale the step by 1/diag(K).  PT,
    u <- u + s1 D^-1 R, is stable when s1 lam_max(D^-1 K) < 2; APT with momentum a when
    b lam_max < 2 (1 + a).  With uniform moduli lam_max is near 2 (so b = 0.9 is stable even
    at a = 0); for moduli drawn log-uniform in [1e-9, 1] cell by cell it reaches 2.2 (2D) and
    2.4 (3D), still inside the PT bound for s1 = 0.75 and inside the APT bound from a = 1/4,
    the adaptive schedule's momentum on the second sweep after a restart."""
    a, b, s1 = W.local_step_params(64)
    assert (b, s1) == (0.9, 0.75) and 0.0 < a < 1.0
    p = O.OracleProblem(dim, *shape)

    def lam_max(E):
        K = p.assemble_K(E).toarray()
        d = np.diag(K)
        lam = np.linalg.eigvals(K / d[:, None]).real.max()
        assert lam <= (np.abs(K).sum(axis=1) / d).max() + 1e-9   # Gershgorin
        return lam

    lam = lam_max(np.ones(p.ncells))
    assert 2.0 <= lam < 2.1 and b * lam < 2.0
    rng = np.random.default_rng(11)
    for trial in range(3):
        lam = lam_max(10.0 ** rng.uniform(-9, 0, p.ncells))
        assert s1 * lam < 2.0 and b * lam < 2.0 * (1.0 + 0.25), lam


def _guard_setup():
    spec = W.mbb_halfbeam(12, 6)
    p, mat = oracle_problem(spec), oracle_materials(spec)
    return p, mat.modulus(spec.phi0), p.load_vector(), p.fixed_mask()


@pytest.mark.parametrize("momentum,a,b,factor", [(0, 1.3, 0.25, 10.0), (1, 1.0, 25.0, 100.0)])
def test_solve_guard_switches_to_pt_above_the_guard_factor(momentum, a, b, factor):
    """Divergence guard of the tolerance-mode solve: the first check whose residual exceeds
    factor x the best earlier check (10 with fixed damping, 100 with adaptive-restart
    momentum) zeroes w and switches to PT for the rest of the solve; u carries on from the
    state it reached.  Established from fresh solves cut at successive checks (each reports
    its last checked residual), then continued against plain PT sweeps."""
    p, E, F, fixed = _guard_setup()
    ce = 5
    kw = dict(mode=1, a=a, b=b, s1=0.25, tol=1e-30, check_every=ce, local_dt=False, momentum=momentum)
    res, fell, states = [], [], []
    for m in range(1, 13):
        u = np.zeros(p.ndof)
        rep = p.solve(E, F, fixed, u, max_sweeps=m * ce, **kw)
        res.append(rep["res_norm"])
        fell.append(rep["fell_back_to_pt"])
        states.append(u)
        if rep["fell_back_to_pt"]:
            break
    assert fell[-1], "the over-relaxed iteration must trip the guard"
    ms = len(res)
    for m in range(1, ms - 1):
        assert res[m] <= factor * min(res[:m])
    assert res[ms - 1] > factor * min(res[:ms - 1])
    q = 7
    u = np.zeros(p.ndof)
    rep = p.solve(E, F, fixed, u, max_sweeps=ms * ce + q, **kw)
    assert rep["fell_back_to_pt"] and rep["apt_sweeps"] == ms * ce and rep["pt_sweeps"] == q
    ref = states[-1].copy()
    for _ in range(q):
        p.pt_sweep(E, F, fixed, 0.25, ref)
    assert np.array_equal(u, ref)


@pytest.mark.parametrize("momentum", [0, 1])
def test_solve_guard_resets_a_non_finite_state(momentum):
    """A non-finite check residual zeroes u and w and switches to PT: from a state holding a
    NaN, the solve ends exactly where PT sweeps from zero end."""
    p, E, F, fixed = _guard_setup()
    ce, q = 4, 9
    u = np.zeros(p.ndof)
    u[np.flatnonzero(fixed == 0)[5]] = np.nan
    rep = p.solve(E, F, fixed, u, mode=1, a=0.9, b=0.25, s1=0.25, tol=1e-30, max_sweeps=ce + q, check_every=ce,
                  local_dt=False, momentum=momentum)
    assert rep["fell_back_to_pt"] and rep["apt_sweeps"] == ce and rep["pt_sweeps"] == q
    ref = np.zeros(p.ndof)
    for _ in range(q):
        p.pt_sweep(E, F, fixed, 0.25, ref)
    assert np.all(np.isfinite(u)) and np.array_equal(u, ref)


def test_openmp_build_agrees_with_the_oracle():
    """The OpenMP build (all-core CPU baseline only) runs the same sweeps as the oracle; its
    scatter sums each node's cell forces in another order, so the states agree to rounding."""
    if not O.openmp_available():
        pytest.skip("no OpenMP in the host compiler")
    for spec in (W.cantilever3d(18, 9, 7), W.mbb_halfbeam(30, 9)):
        out = []
        for omp in (False, True):
            op = O.OracleProblem(spec.dim, spec.nx, spec.ny, spec.nz, h=spec.h, physics=spec.physics, nu=spec.nu,
                                 loads=spec.loads, boxes=spec.boxes, openmp=omp)
            E = oracle_materials(spec).modulus(W.random_design(spec, seed=7))
            u = np.zeros(op.ndof)
            op.solve(E, op.load_vector(), op.fixed_mask(), u, mode=0, n_apt=25, n_pt=5, a=0.9, b=0.25, s1=0.25,
                     check_every=0)
            out.append((u, op.residual(E, op.load_vector(), op.fixed_mask(), u)[1]))
        assert np.abs(out[0][0] - out[1][0]).max() <= 1e-12 * np.abs(out[0][0]).max()
        assert abs(out[0][1] - out[1][1]) <= 1e-12 * out[0][1]
