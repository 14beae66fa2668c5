"""Slab decomposition on one GPU: several slab contexts of one grid, planes exchanged device
to device before every sweep, against the same sweeps of the whole grid.  A node's update
reads only its 3 x 3 x 3 neighbourhood and its 8 cells, in the same order in both, so the
owned planes must match bit for bit (node-gather and two-row marching kernels, FP64 and
FP32); the FP64 decomposed solve is also held against the oracle's direct solve.  The FP64
refinement of FP32 solves, decomposed, gives the whole grid's refined solve bit for bit,
alone and inside the decomposed design loop."""
import numpy as np
import pytest

from paper_2509_06971_gb300 import slab as S
from paper_2509_06971_gb300 import workloads as W
from tests._util import oracle_materials, oracle_problem, nodes_to_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2509_06971_gb300 import problem as PR
    return PR


def _spec(nx=70, ny=40, nz=37, precision="f64"):
    """Several x/y tiles and z segments with ragged tails; loads on and next to slab
    interfaces; supports crossing them."""
    base = W.cantilever3d(nx, ny, nz)
    loads = base.loads + [((31, 7, 12), 0, 0.7), ((30, 6, 13), 1, -0.4), ((62, 14, 25), 2, 0.25),
                          ((5, 39, 19), 2, 1.0), ((nx, ny, nz), 1, 0.3)]
    boxes = base.boxes + [((nx, 0, 10), (nx, ny, 30), 0b010), ((10, 21, 0), (40, 22, 5), 0b101)]
    spec = base.with_(loads=loads, boxes=boxes, precision=precision, storage=precision)
    return spec.with_(phi0=W.random_design(spec, seed=31))


def _whole(P, spec, kernel, u0, w0, sweeps):
    p = P.Problem(spec)
    if kernel:
        p.select_kernel(kernel)
    p.set_state(u0, w0)
    r2 = [p.sweep(kind, n, a, b, s1, True) for kind, n, a, b, s1 in sweeps]
    u, w = p.get_state(with_w=True, dtype=p.np_dtype)
    p.close()
    return u, w, r2


SWEEPS = [(0, 3, 0.9, 0.8, 0.0), (1, 2, 0.0, 0.0, 0.15), (0, 2, 0.95, 0.7, 0.0)]


def _same(a, b, spec):
    """Bit-for-bit equality; on failure, report the size of the gap and the planes it is on."""
    if np.array_equal(a, b):
        return
    d = np.abs(np.asarray(a, np.float64) - b).reshape(a.shape[0], spec.nz + 1, spec.ny + 1, spec.nx + 1)
    planes = np.nonzero(d.max(axis=(0, 2, 3)))[0].tolist()
    pytest.fail(f"max |diff| {d.max():.3e} (rel {d.max() / np.abs(b).max():.3e}) on planes {planes}")


@pytest.mark.parametrize("precision,kernel", [("f64", None), ("f32", "tma3"), ("f32", "tma2"),
                                              ("f32", "gather/32x4")])
@pytest.mark.parametrize("n_slabs", [2, 3])
def test_slabs_equal_whole_grid_sweeps(P, precision, kernel, n_slabs):
    spec = _spec(precision=precision)
    dt = np.float64 if precision == "f64" else np.float32
    u0 = W.random_state(spec, seed=32).astype(dt)
    w0 = W.random_state(spec, seed=33, scale=0.1).astype(dt)
    uw, ww, r2w = _whole(P, spec, kernel, u0, w0, SWEEPS)
    with S.SlabGrid(spec, n_slabs, kernel=kernel) as g:
        if kernel:
            name = g.probs[0].kernel_info()[0]
            assert name.startswith(kernel.split("/")[0])
        g.set_state(u0, w0)
        r2s = [g.sweep(kind, n, a, b, s1, True) for kind, n, a, b, s1 in SWEEPS]
        us, ws = g.get_state(with_w=True, dtype=dt)
    _same(us, uw, spec)
    _same(ws, ww, spec)  # w of the last APT block
    tol = 1e-12 if precision == "f64" else 1e-5  # sums over slabs in another order
    for a, b in zip(r2s, r2w):
        assert abs(a - b) <= tol * b


def test_slab_solve_matches_direct_solve_fp64(P):
    """A fixed-momentum APT solve over three slabs, exchange before every sweep, to
    ||R|| <= 1e-9 ||F||: compliance within 1e-7 of the oracle's direct solve."""
    base = W.cantilever3d(24, 12, 14, precision="f64")
    spec = base.with_(loads=base.loads + [((12, 6, 5), 0, 0.5), ((20, 3, 9), 1, -0.3)],
                      phi0=W.random_design(base, seed=36, lo=0.3, hi=0.95))
    with S.SlabGrid(spec, 3) as g:
        rep = g.solve(tol=1e-9, check_every=50, max_sweeps=20000)  # about 6 600 sweeps
        u = g.get_state()
    assert rep["converged"], rep
    op, om = oracle_problem(spec), oracle_materials(spec)
    F = op.load_vector()
    ud = op.direct_solve(om.modulus(spec.phi0), F, op.fixed_mask())
    Cs, Cd = float(F @ nodes_to_oracle(u)), float(F @ ud)
    assert abs(Cs - Cd) <= 1e-7 * abs(Cd)


@pytest.mark.parametrize("kernel", ["tma3", "tma2"])
def test_slab_multi_rhs_two_row_equals_whole(P, kernel):
    spec, cases = W.multirhs3d(40, 18, 20, n_rhs=2, seed=5)
    spec = spec.with_(precision="f32", storage="f32", phi0=W.random_design(spec, seed=34))
    rng = np.random.default_rng(35)
    u0 = rng.standard_normal((6, spec.nnodes)).astype(np.float32)
    p = P.Problem(spec, nrhs=2, load_cases=cases)
    p.select_kernel(kernel)
    p.set_state(u0)
    p.sweep(0, 4, 0.9, 0.8, 0.0, True)
    uw = p.get_state(dtype=np.float32)
    p.close()
    with S.SlabGrid(spec, 2, kernel=kernel, nrhs=2, load_cases=cases) as g:
        g.set_state(u0)
        g.sweep(0, 4, 0.9, 0.8, 0.0, True)
        us = g.get_state(dtype=np.float32)
    _same(us, uw, spec)


def test_slab_argument_checks(P):
    from paper_2509_06971_gb300 import capi as C
    p2 = P.Problem(W.mbb_halfbeam(24, 8))
    with pytest.raises(C.PettoError) as e:
        p2.set_owned_planes(0, 0)
    assert e.value.status == C.PETTO_EUNSUPPORTED
    p2.close()
    p3 = P.Problem(W.cantilever3d(24, 12, 12).with_(precision="f32", storage="f32"))
    for lo, hi in ((-1, 3), (4, 3), (0, 13)):
        with pytest.raises(C.PettoError) as e:
            p3.set_owned_planes(lo, hi)
        assert e.value.status == C.PETTO_EINVAL
    p3.set_owned_planes(1, 11)
    with pytest.raises(C.PettoError) as e:
        p3.select_kernel("tma8")  # one-row marching kernels write whole columns
    assert e.value.status == C.PETTO_EINVAL
    p3.select_kernel("gather")
    assert p3.kernel_info()[0].startswith("gather/")
    with pytest.raises(C.PettoError) as e:
        p3.get_plane(13)
    assert e.value.status == C.PETTO_EINVAL
    with pytest.raises(ValueError):
        p3.get_plane(0, out=np.empty(p3.plane_shape(), np.float64))  # not the sweep precision
    # the whole range restores a whole-grid context; planes round-trip through the host
    p3.set_owned_planes(0, 12)
    pl = np.arange(np.prod(p3.plane_shape()), dtype=np.float32).reshape(p3.plane_shape())
    p3.set_plane(5, pl)
    assert np.array_equal(p3.get_plane(5), pl)
    u = p3.get_state(dtype=np.float32).reshape(3, 13, 13, 25)
    assert np.array_equal(u[:, 5], pl) and not u[:, 4].any()
    p3.close()


@pytest.mark.parametrize("precision,kernel,n_slabs", [("f64", None, 2), ("f64", None, 3), ("f32", "tma3", 3)])
def test_library_slab_solve_with_adaptive_momentum_equals_whole_grid(P, precision, kernel, n_slabs):
    """petto_slab_solve (the solve loop in the library, with the driver's exchange and
    all-reduce hooks) with the adaptive-restart momentum: its restart tests and checks use
    the whole grid's <R, w> and ||R|| (sums over the slabs), so it takes the whole grid's
    solve's decisions: the same sweep counts and the same field (sums in another order can
    only move a decision that sits on a tie)."""
    spec = _spec(precision=precision)
    tol = 1e-9 if precision == "f64" else 1e-3
    kw = dict(tol=tol, check_every=20, max_sweeps=60000)
    p = P.Problem(spec)
    if kernel:
        p.select_kernel(kernel)
    rep_w = p.solve(mode=1, momentum=1, refine=False, local_dt=True, **kw)
    uw = p.get_state(dtype=p.np_dtype)
    p.close()
    with S.SlabGrid(spec, n_slabs, kernel=kernel) as g:
        rep_s = g.solve(momentum=1, local_dt=True, **kw)
        us = g.get_state(dtype=uw.dtype)
    assert rep_w["converged"] and rep_s["converged"], (rep_w, rep_s)
    assert rep_s["sweeps"] == rep_w["sweeps"]
    _same(us, uw, spec)


def _design_spec(precision, vol_mode):
    base = W.cantilever3d(24, 12, 14).with_(precision=precision, storage=precision)
    spec = base.with_(loads=base.loads + [((12, 6, 5), 0, 0.5), ((20, 3, 9), 1, -0.3)],
                      phi0=W.random_design(base, seed=37, lo=0.2, hi=0.6))
    # the penalty form with a volume term, so that the step reads the whole grid's means
    return spec.with_(vol_mode=vol_mode, kappa_v=0.5 if vol_mode == 1 else spec.kappa_v)


@pytest.mark.parametrize("precision,kernel,n_slabs,vol_mode", [("f64", None, 2, 0), ("f64", None, 3, 0),
                                                               ("f64", None, 3, 1), ("f32", "tma3", 2, 0)])
def test_slab_design_steps_equal_whole_grid(P, precision, kernel, n_slabs, vol_mode):
    """petto_slab_design_step on every slab (Fig. 5 loop: solve, sensitivity, update,
    Cahn-Hilliard, modulus; plane and cell-layer exchanges, sums and maxima over the slabs)
    against petto_optimize on the whole grid, two loops from the same design: the same sweep
    counts, and compliance, multiplier, volume and design equal up to the order of the sums
    (the bisection and the means add the slabs' partial sums; FP64 1e-11, FP32 1e-5)."""
    spec = _design_spec(precision, vol_mode)
    tol = 1e-9 if precision == "f64" else 1e-3
    solve_kw = dict(tol=tol, check_every=20, max_sweeps=60000, momentum=1, local_dt=True, refine=False)
    p = P.Problem(spec)
    if kernel:
        p.select_kernel(kernel)
    hist, _ = p.optimize(2, solve_kw=solve_kw)
    phi_w = p.get_design()
    p.close()
    with S.SlabGrid(spec, n_slabs, kernel=kernel) as g:
        rows = [g.design_step(solve_kw=solve_kw) for _ in range(2)]
        phi_s = g.get_design()
    rtol = 1e-11 if precision == "f64" else 1e-5
    for a, b in zip(rows, hist):
        assert a["sweeps"] == b["sweeps"], (a, b)
        for key in ("compliance", "work", "mean_phi0", "lambda0"):
            assert abs(a[key] - b[key]) <= rtol * max(abs(b[key]), 1e-3), (key, a[key], b[key])
    assert np.abs(phi_s - phi_w).max() <= rtol * 10


def test_slab_design_step_oracle_loops_fp64(P):
    """Two decomposed design loops against the oracle's two loops (Sec. 3.3 update and
    Cahn-Hilliard step), FP64, three slabs: compliance within 1e-7, design within 1e-6."""
    from oracle import oracle as O
    spec = _design_spec("f64", 0)
    with S.SlabGrid(spec, 3) as g:
        rows = [g.design_step(solve_kw=dict(tol=1e-10, check_every=20, max_sweeps=100000, momentum=1,
                                            local_dt=True)) for _ in range(2)]
        phi_s = g.get_design()
    op, om = oracle_problem(spec), oracle_materials(spec)
    F, fixed = op.load_vector(), op.fixed_mask()
    phi, u = spec.phi0.copy(), np.zeros(op.ndof)
    for t in range(2):
        m = O.design_step(op, om, phi, u, F, fixed, spec.vol_frac,
                          dict(mode=1, a=1.0, b=spec.apt_b, s1=spec.pt_s1, tol=1e-10, max_sweeps=400000,
                               check_every=20, local_dt=True, momentum=1),
                          dict(alpha_h=spec.alpha_h, gamma_g=spec.gamma_g, tau=spec.tau, vol_mode=spec.vol_mode,
                               kappa_v=spec.kappa_v, kappa_1=spec.kappa_1, n_bisect=spec.n_bisect))
        assert abs(rows[t]["compliance"] - m["compliance"]) <= 1e-7 * m["compliance"]
    assert np.abs(phi_s - phi).max() <= 1e-6


def test_slab_design_step_checks(P):
    from paper_2509_06971_gb300 import capi as C
    spec = _design_spec("f64", 0)
    with S.SlabGrid(W.cantilever3d(8, 4, 2).with_(precision="f64", storage="f64"), 2) as g2:
        with pytest.raises(ValueError):
            g2.design_step()  # the upper slab would own one node plane and no cell layer
    with S.SlabGrid(spec, 2) as g:
        p = g.probs[1]
        nb = p.layer_bytes(C.PETTO_LAYER_PHI)
        assert nb == spec.nx * spec.ny * 8 and p.layer_bytes(C.PETTO_LAYER_MU) == nb
        buf = np.zeros(nb, np.uint8)
        for field, phase, k in ((2, 0, 0), (0, 1, 0), (0, 0, -1), (0, 0, p.spec.nz + 1)):
            with pytest.raises(C.PettoError) as e:
                p.get_layer(field, phase, k, buf)
            assert e.value.status == C.PETTO_EINVAL
        phi = p.get_design()
        p.get_layer(C.PETTO_LAYER_PHI, 0, 3, buf)
        assert np.array_equal(buf.view(np.float64), phi[0].reshape(p.spec.nz, -1)[3])


@pytest.mark.parametrize("kernel,n_slabs", [("tma3", 2), ("tma3", 3), ("gather/32x4", 2)])
def test_slab_refined_fp32_solve_equals_whole_grid(P, kernel, n_slabs):
    """The FP64 refinement of an FP32 solve, decomposed: each slab's FP64 state with its
    ghost planes, the defect of its own planes (the FP64 marching defect, whose per-node
    arithmetic does not depend on where its z segments start), the whole grid's defect norm
    and the whole grid's scale of the FP16 right-hand side (allreduce_max).  To 1e-6: the
    whole grid's refined solve's sweep count, residual and field bit for bit."""
    spec = _spec(precision="f32")
    kw = dict(tol=1e-6, check_every=20, max_sweeps=100000, momentum=1, local_dt=True)
    p = P.Problem(spec)
    p.select_kernel(kernel)
    rep_w = p.solve(mode=1, refine=True, **kw)
    uw = p.get_state(dtype=np.float32)
    p.close()
    with S.SlabGrid(spec, n_slabs, kernel=kernel) as g:
        rep_s = g.solve(refine=True, **kw)
        us = g.get_state(dtype=np.float32)
    assert rep_w["converged"] and rep_s["converged"], (rep_w, rep_s)
    assert rep_w["rel_res"] <= 1e-6
    assert rep_s["sweeps"] == rep_w["sweeps"], (rep_s, rep_w)
    assert abs(rep_s["rel_res"] - rep_w["rel_res"]) <= 1e-9 * rep_w["rel_res"]  # sums in another order
    _same(us, uw, spec)


def test_slab_refined_fp32_solve_matches_direct_solve(P):
    """An FP32 solve over three slabs (two-row marching kernel) refined to ||R|| <= 1e-6 ||F||:
    the compliance of the oracle's direct solve (FP64 moduli of the FP32 design) to 1e-5."""
    base = W.cantilever3d(24, 12, 14)
    spec = base.with_(loads=base.loads + [((12, 6, 5), 0, 0.5), ((20, 3, 9), 1, -0.3)],
                      phi0=W.random_design(base, seed=36, lo=0.3, hi=0.95))
    with S.SlabGrid(spec, 3, kernel="tma3") as g:
        rep = g.solve(tol=1e-6, check_every=20, max_sweeps=100000, momentum=1, local_dt=True)
        u = g.get_state(dtype=np.float64)
    assert rep["converged"] and rep["rel_res"] <= 1e-6, rep
    op, om = oracle_problem(spec), oracle_materials(spec)
    F = op.load_vector()
    ud = op.direct_solve(om.modulus(np.asarray(spec.phi0, np.float32).astype(np.float64)), F, op.fixed_mask())
    Cs, Cd = float(F @ nodes_to_oracle(u)), float(F @ ud)
    assert abs(Cs - Cd) <= 1e-5 * abs(Cd), (Cs, Cd)


def test_slab_refined_design_steps_equal_whole_grid(P):
    """Two decomposed design loops with FP32 state solves refined to 1e-6 (the benchmark's
    solve) against petto_optimize on the whole grid: the same sweep counts, the step's
    metrics and the design equal up to the order of the sums."""
    spec = _design_spec("f32", 0)
    solve_kw = dict(tol=1e-6, check_every=20, max_sweeps=100000, momentum=1, local_dt=True)
    p = P.Problem(spec)
    p.select_kernel("tma3")
    hist, _ = p.optimize(2, solve_kw=solve_kw)
    phi_w = p.get_design()
    p.close()
    with S.SlabGrid(spec, 2, kernel="tma3") as g:
        rows = [g.design_step(solve_kw=solve_kw) for _ in range(2)]
        phi_s = g.get_design()
    for a, b in zip(rows, hist):
        assert a["sweeps"] == b["sweeps"], (a, b)
        assert a["rel_res"] <= 1e-6 and b["rel_res"] <= 1e-6
        for key in ("compliance", "work", "mean_phi0", "lambda0"):
            assert abs(a[key] - b[key]) <= 1e-5 * max(abs(b[key]), 1e-3), (key, a[key], b[key])
    assert np.abs(phi_s - phi_w).max() <= 1e-4


def test_slab_refinement_needs_the_max_hook(P):
    """A one-slab decomposition of the whole grid (no-op exchange, identity all-reduces) is
    petto_pt_solve: the refined FP32 solve takes its decisions and gives its field; without
    allreduce_max the refinement is refused."""
    from paper_2509_06971_gb300 import capi as C
    spec = _spec(precision="f32")
    kw = dict(tol=1e-6, check_every=20, max_sweeps=100000, momentum=1, local_dt=True)
    p = P.Problem(spec)
    p.select_kernel("tma3")
    with pytest.raises(C.PettoError) as e:
        p.slab_solve(lambda: None, lambda v: v, mode=1, **kw)
    assert e.value.status == C.PETTO_EINVAL
    p.set_state(np.zeros((3, spec.nnodes), np.float32))
    rep_s = p.slab_solve(lambda: None, lambda v: v, allreduce_max=lambda v: v, mode=1, **kw)
    us = p.get_state(dtype=np.float32)
    p.set_state(np.zeros((3, spec.nnodes), np.float32))
    rep_w = p.solve(mode=1, **kw)
    uw = p.get_state(dtype=np.float32)
    p.close()
    assert rep_s["converged"] and rep_s["sweeps"] == rep_w["sweeps"]
    _same(us, uw, spec)
