"""2D sweeps several per launch (temporal blocking, kernel sweep2d_tb): K sweeps (Sec. 2.2
PT / APT updates of the Sec. 3.2 systems) run by each block on a shared-memory copy of its
tile and a K-node halo, against single sweeps and the oracle.

* FP64: K sweeps in one launch give, bit for bit, the field of K launches of the
  y-marching kernel (the same per-node arithmetic); ragged grids of many tiles, point loads
  and supports on tile edges and in halos, elastic (cantilever, MBB) and thermal, APT with
  global and local steps and PT, K = 2 and 4.  Also within 1e-12 of the oracle's K sweeps.
* FP32: within 1e-5 rel-L2 per field of the oracle's K sweeps, on the shapes the kernel
  picks by itself and on small tiles.
* A launch count that is not a multiple of K (grouped 4 + 2 + 1) and a dense right-hand
  side (refinement correction) follow the same rule.
* Solves: the adaptive-restart APT solve on this kernel takes the y-marching solve's
  decisions in FP64 (the same sweep count, the same field); the FP32 refined solve and a
  design loop land on the oracle's direct solve / FP64 loop.
* Degenerate grids (one cell, one cell row or column, grids narrower than a tile) follow the
  FP64 rule with the kernel's own region and with regions far larger than the grid.
"""
import numpy as np
import pytest

from paper_2509_06971_gb300 import workloads as W
from tests._util import nodes_to_oracle, oracle_materials, oracle_problem, oracle_to_nodes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2509_06971_gb300 import problem as PR
    return PR


def rel_l2(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def relmax(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def specs():
    c = W.cantilever2d(70, 46, load_cells=6)
    return {
        # loads on the top edge and inside the grid (halos of neighbouring tiles)
        "cantilever": c.with_(loads=c.loads + [((13, 46, 0), 0, 0.3), ((24, 8, 0), 1, -0.2), ((25, 9, 0), 0, 0.4)]),
        "mbb": W.mbb_halfbeam(67, 21),
        "heat": W.heat2d(66).with_(boxes=[((0, 29, 0), (0, 37, 0), 1), ((66, 0, 0), (66, 3, 0), 1)],
                                   loads=[((23, 17, 0), 0, 0.5)]),
    }


def _prob(P, spec, kernel, seed=1, precision="f64"):
    spec = spec.with_(precision=precision, storage=precision)
    prob = P.Problem(spec)
    if kernel:
        prob.select_kernel(kernel)
    phi = W.random_design(spec, seed=seed, lo=0.05, hi=0.95)
    prob.set_design(phi)
    return spec, prob, phi


def _state(spec, dt=np.float64):
    return W.random_state(spec, seed=2).astype(dt), W.random_state(spec, seed=3, scale=0.1).astype(dt)


def _run(P, spec, kernel, kind, n, consts, local, precision="f64"):
    spec, prob, phi = _prob(P, spec, kernel, precision=precision)
    dt = np.float64 if precision == "f64" else np.float32
    u0, w0 = _state(spec, dt)
    prob.set_state(u0, w0)
    a, b, s1 = consts
    r2 = prob.sweep(kind, n, a, b, s1, local)
    u, w = prob.get_state(with_w=True, dtype=dt)
    name = prob.kernel_info()[0]
    prob.close()
    return u, w, r2, name, phi


CONSTS = {"apt": (0, (0.93, 0.21, 0.0), False), "apt_local": (0, (0.93, 0.9, 0.0), True),
          "pt": (1, (0.0, 0.0, 0.17), False), "pt_local": (1, (0.0, 0.0, 0.7), True)}


@pytest.mark.parametrize("name", list(specs()))
@pytest.mark.parametrize("kind", list(CONSTS))
@pytest.mark.parametrize("kernel,n", [("tb2d/k4/32x16", 4), ("tb2d/k2/62x12", 2), ("tb2d/k4/62x20", 7),
                                      ("tb2d/k4/122x14", 4)])
def test_sweeps_per_launch_equal_single_sweeps_fp64(P, name, kind, kernel, n):
    spec = specs()[name]
    sk, consts, local = CONSTS[kind]
    ut, wt, r2t, kname, phi = _run(P, spec, kernel, sk, n, consts, local)
    assert kname == kernel
    ug, wg, r2g, gname, _ = _run(P, spec, "march2d", sk, n, consts, local)
    assert gname.startswith("march2d/")
    assert np.array_equal(ut, ug), relmax(ut, ug)
    assert np.array_equal(wt, wg), relmax(wt, wg)  # PT sweeps leave w as it was
    if sk == 1:
        assert np.array_equal(wt, _state(spec)[1])
    assert abs(r2t - r2g) <= 1e-13 * r2g  # the sum over the last sweep, in another order
    # and the oracle's n sweeps
    op, om = oracle_problem(spec), oracle_materials(spec)
    E, F, fixed = om.modulus(phi), op.load_vector(), op.fixed_mask()
    u0, w0 = _state(spec)
    uo, wo = nodes_to_oracle(u0), nodes_to_oracle(w0)
    a, b, s1 = consts
    for _ in range(n):
        r2o = op.apt_sweep(E, F, fixed, a, b, uo, wo, local_dt=local) if sk == 0 else \
            op.pt_sweep(E, F, fixed, s1, uo, local_dt=local)
    assert relmax(ut, oracle_to_nodes(uo, spec.ncomp)) < 1e-12
    assert abs(r2t - r2o) < 1e-11 * r2o


@pytest.mark.parametrize("name", ["cantilever", "heat"])
@pytest.mark.parametrize("kernel", [None, "tb2d/k4/32x16"])
def test_sweeps_per_launch_fp32_against_oracle(P, name, kernel):
    spec = specs()[name]
    n = 8
    ut, wt, r2t, kname, phi = _run(P, spec, kernel, 0, n, (0.93, 0.9, 0.0), True, precision="f32")
    assert kname.startswith("tb2d/k4/")  # the default 2D kernel
    op, om = oracle_problem(spec), oracle_materials(spec)
    E = om.modulus(np.asarray(phi, np.float32).astype(np.float64))
    F, fixed = op.load_vector(), op.fixed_mask()
    u0, w0 = _state(spec, np.float32)
    uo, wo = nodes_to_oracle(u0.astype(np.float64)), nodes_to_oracle(w0.astype(np.float64))
    for _ in range(n):
        r2o = op.apt_sweep(E, F, fixed, 0.93, 0.9, uo, wo, local_dt=True)
    un, wn = oracle_to_nodes(uo, spec.ncomp), oracle_to_nodes(wo, spec.ncomp)
    for c in range(spec.ncomp):
        assert rel_l2(ut[c], un[c]) < 1e-5, c
        assert rel_l2(wt[c], wn[c]) < 1e-5, c
    assert abs(r2t - r2o) < 1e-5 * r2o


def test_dense_right_hand_side_fp64(P):
    """The correction sweeps of the refinement read a dense right-hand side instead of the
    loads: 4 in one launch equal 4 y-marching sweeps."""
    spec = specs()["cantilever"]
    r = W.random_state(spec, seed=9, scale=1e-3)
    out = {}
    for kernel in ("tb2d/k4/32x16", "march2d"):
        spec64, prob, _ = _prob(P, spec, kernel)
        u0, w0 = _state(spec64)
        prob.set_state(u0, w0)
        r2 = prob.sweep_rhs(0, 4, r, 0.9, 0.8, 0.0, True)
        out[kernel] = prob.get_state(with_w=True) + (r2,)
        prob.close()
    a, b = out["tb2d/k4/32x16"], out["march2d"]
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert abs(a[2] - b[2]) <= 1e-13 * b[2]


@pytest.mark.parametrize("name", ["cantilever", "heat"])
def test_adaptive_solve_takes_the_marching_solves_decisions_fp64(P, name):
    spec = specs()[name]
    res = {}
    for kernel in ("tb2d/k4/62x24", "march2d"):
        spec64, prob, phi = _prob(P, spec, kernel, seed=4)
        rep = prob.solve(mode=1, tol=1e-10, momentum=1, local_dt=True, check_every=20, max_sweeps=400000)
        res[kernel] = (rep, prob.get_state())
        prob.close()
    (rt, ut), (rg, ug) = res["tb2d/k4/62x24"], res["march2d"]
    assert rt["converged"] and rg["converged"]
    assert rt["sweeps"] == rg["sweeps"], (rt, rg)
    assert np.array_equal(ut, ug), relmax(ut, ug)
    # and the solution is the oracle's
    op, om = oracle_problem(spec), oracle_materials(spec)
    F = op.load_vector()
    ud = op.direct_solve(om.modulus(phi), F, op.fixed_mask())
    assert relmax(ut, oracle_to_nodes(ud, spec.ncomp)) < 1e-8


@pytest.mark.parametrize("name", ["cantilever", "heat"])
def test_fp32_refined_solve_matches_direct_solve(P, name):
    """FP32 sweeps four per launch with the FP64 refinement (dense FP32 right-hand sides)
    to 1e-6: the compliance of the oracle's direct solve (elasticity and heat)."""
    spec = (W.cantilever2d(128, 64) if name == "cantilever" else W.heat2d(96)).with_(precision="f32",
                                                                                    storage="f32")
    prob = P.Problem(spec)
    assert prob.kernel_info()[0].startswith("tb2d/k4/")
    phi = W.random_design(spec, seed=7, lo=0.2, hi=0.9)
    prob.set_design(phi)
    rep = prob.solve(tol=1e-6)
    assert rep["converged"] and rep["rel_res"] <= 1e-6
    Cg, _, _ = prob.sensitivity(want_field=False)
    prob.close()
    op, om = oracle_problem(spec), oracle_materials(spec)
    F = op.load_vector()
    Co = float(F @ op.direct_solve(om.modulus(np.asarray(phi, np.float32).astype(np.float64)), F, op.fixed_mask()))
    assert abs(Cg - Co) < 1e-4 * abs(Co)


def test_bad_regions_are_rejected(P):
    from paper_2509_06971_gb300 import capi as C
    spec, prob, _ = _prob(P, specs()["cantilever"], None, precision="f32")
    for name in ("tb2d/k3/32x16", "tb2d/k4/10x16", "tb2d/k4/40x16", "tb2d/k4/32x11", "tb2d/k4/242x256"):
        with pytest.raises(C.PettoError) as e:
            prob.select_kernel(name)
        assert e.value.status == C.PETTO_EINVAL, name
    prob.select_kernel("tb2d/k2/62x24")
    assert prob.kernel_info() == ("tb2d/k2/62x24", 4)
    prob.close()


@pytest.mark.parametrize("shape", [(1, 1), (2, 1), (1, 5), (33, 1), (3, 200), (200, 3), (61, 47)])
@pytest.mark.parametrize("kernel", [None, "tb2d/k4/122x14", "tb2d/k2/32x16"])
def test_degenerate_grids_fp64(P, shape, kernel):
    """Grids of one cell, one cell row or column, and grids narrower than a tile (so one
    block's halo reaches past every edge): 9 sweeps (launches of 4 + 4 + 1, or 2 + ... + 1)
    equal 9 y-marching sweeps bit for bit and the oracle's 9 sweeps."""
    nx, ny = shape
    spec = W.ProblemSpec(name="thin", dim=2, nx=nx, ny=ny, nz=0, precision="f64", storage="f64",
                         boxes=[((0, 0, 0), (0, ny, 0), 3)], loads=[((nx, ny, 0), 1, -1.0)], vol_frac=[0.5])
    n, consts, local = 9, (0.93, 0.9, 0.0), True
    ut, wt, r2t, kname, phi = _run(P, spec, kernel, 0, n, consts, local)
    assert kname.startswith("tb2d/") and (kernel is None or kname == kernel)
    ug, wg, r2g, gname, _ = _run(P, spec, "march2d", 0, n, consts, local)
    assert np.array_equal(ut, ug), relmax(ut, ug)
    assert np.array_equal(wt, wg), relmax(wt, wg)
    assert abs(r2t - r2g) <= 1e-13 * r2g
    op, om = oracle_problem(spec), oracle_materials(spec)
    E, F, fixed = om.modulus(phi), op.load_vector(), op.fixed_mask()
    u0, w0 = _state(spec)
    uo, wo = nodes_to_oracle(u0), nodes_to_oracle(w0)
    for _ in range(n):
        op.apt_sweep(E, F, fixed, *consts[:2], uo, wo, local_dt=local)
    assert relmax(ut, oracle_to_nodes(uo, 2)) < 1e-12
