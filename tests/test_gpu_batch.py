"""Batched 2D problems (petto_batch_*): one launch per sweep over every problem.

Each problem of a batch runs the iteration of the single-problem solve with the same
kernel arithmetic, tiles and reduction order as the 2D marching sweep, so its state,
sweep counts and residuals must equal (bit for bit) those of the same problem solved
alone on that kernel; against the default (node-gather) single-problem kernel they agree
to FP32 rounding.  The FP64 batch is also held against the oracle, which shares nothing
with either GPU path.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2509_06971_gb300 import workloads as W
from tests._util import oracle_materials, oracle_problem, oracle_to_nodes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2509_06971_gb300 import problem as PR
    return PR


def small_batch(n=5, seed=5, precision="f32"):
    """Instances of the batch recipe at reduced sizes (32x16 .. 128x64 cells)."""
    return [s.with_(precision=precision, storage=precision) for s in W.batch2d(n, seed=seed, lo=32, hi_factor=4.0)]


def relmax(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _alone(P, specs, seeds, kernel="march2d", **kw):
    out = []
    for spec, sd in zip(specs, seeds):
        p = P.Problem(spec)
        if kernel:
            p.select_kernel(kernel)  # the batched sweep's kernel
        p.set_design(W.random_design(spec, seed=sd))
        rep = p.solve(**kw)
        out.append((rep, p.get_state(dtype=p.np_dtype)))
        p.close()
    return out


def _batched(P, specs, seeds, **kw):
    probs = []
    for spec, sd in zip(specs, seeds):
        p = P.Problem(spec)
        p.set_design(W.random_design(spec, seed=sd))
        probs.append(p)
    b = P.Batch(probs)
    reps = b.solve(**kw)
    states = [p.get_state(dtype=p.np_dtype) for p in probs]
    launches = b.launches
    b.close()
    for p in probs:
        p.close()
    return reps, states, launches


def _same(alone, batched):
    reps, states, _ = batched
    for (ra, ua), rb, ub in zip(alone, reps, states):
        for key in ("sweeps", "apt_sweeps", "pt_sweeps", "converged", "fell_back_to_pt"):
            assert ra[key] == rb[key], (key, ra, rb)
        assert ra["res_norm"] == rb["res_norm"] or (np.isnan(ra["res_norm"]) and np.isnan(rb["res_norm"]))
        assert np.array_equal(ua, ub)


def test_batch_fp32_refined_equals_alone(P):
    """Tolerance mode with FP32 sweeps, adaptive momentum and FP64 refinement: problems of
    different sizes converge at different checks and leave the batch one by one."""
    specs = small_batch(5)
    seeds = list(range(30, 35))
    kw = dict(tol=1e-6, check_every=20, max_sweeps=40000)
    alone = _alone(P, specs, seeds, **kw)
    assert all(r["converged"] for r, _ in alone)
    assert len({r["sweeps"] for r, _ in alone}) > 1  # the problems finish at different sweeps
    batched = _batched(P, specs, seeds, **kw)
    _same(alone, batched)


def test_batch_fp64_equals_alone_and_oracle(P):
    """FP64 tolerance mode: equal to the single-problem path, and the converged fields
    equal the oracle's direct solve to 1e-8 relative."""
    specs = small_batch(3, seed=7, precision="f64")
    seeds = [40, 41, 42]
    kw = dict(tol=1e-11, check_every=20, max_sweeps=200000)
    alone = _alone(P, specs, seeds, **kw)
    batched = _batched(P, specs, seeds, **kw)
    _same(alone, batched)
    for spec, sd, ub in zip(specs, seeds, batched[1]):
        op, om = oracle_problem(spec), oracle_materials(spec)
        phi = W.random_design(spec, seed=sd)
        ud = op.direct_solve(om.modulus(phi), op.load_vector(), op.fixed_mask())
        assert relmax(ub, oracle_to_nodes(ud, 2)) < 1e-8


def test_batch_paper_schedule_equals_alone_and_oracle(P):
    """Paper schedule with the APT/PT switch inside a check interval (n_apt = 30, checks
    every 20): each problem switches at its own sweep 30 inside the batched chunk."""
    specs = small_batch(3, seed=9, precision="f64")
    seeds = [50, 51, 52]
    kw = dict(mode=0, n_apt=30, n_pt=10, momentum=0, a=0.95, check_every=20)
    alone = _alone(P, specs, seeds, **kw)
    batched = _batched(P, specs, seeds, **kw)
    _same(alone, batched)
    for (spec, sd), ub, rb in zip(zip(specs, seeds), batched[1], batched[0]):
        assert rb["apt_sweeps"] == 30 and rb["pt_sweeps"] == 10
        op, om = oracle_problem(spec), oracle_materials(spec)
        u = np.zeros(op.ndof)
        op.solve(om.modulus(W.random_design(spec, seed=sd)), op.load_vector(), op.fixed_mask(), u, mode=0,
                 n_apt=30, n_pt=10, a=0.95, b=spec.apt_b, s1=spec.pt_s1, check_every=20, local_dt=True)
        assert relmax(ub, oracle_to_nodes(u, 2)) < 1e-12


def test_batch_divergence_guard_equals_alone(P):
    """An over-relaxed fixed momentum trips the guard; the problem falls back to PT inside
    the batch exactly as it does alone."""
    specs = small_batch(3, seed=11)
    seeds = [60, 61, 62]
    kw = dict(tol=1e-5, momentum=0, a=1.3, b=0.9, check_every=10, max_sweeps=4000, refine=False)
    alone = _alone(P, specs, seeds, **kw)
    assert any(r["fell_back_to_pt"] for r, _ in alone)
    batched = _batched(P, specs, seeds, **kw)
    _same(alone, batched)


def test_batch_thermal_equals_alone(P):
    base = [W.heat2d(n) for n in (40, 64, 24)]
    specs = [s.with_(precision="f32", storage="f32",
                     boxes=[((0, s.ny // 2 - 3, 0), (0, s.ny // 2 + 3, 0), 1)]) for s in base]
    seeds = [70, 71, 72]
    kw = dict(tol=1e-6, check_every=20, max_sweeps=40000)
    alone = _alone(P, specs, seeds, **kw)
    batched = _batched(P, specs, seeds, **kw)
    _same(alone, batched)


def test_batch_optimize_equals_alone(P):
    """Two design loops: the batched solve plus per-problem design steps leave the same
    designs and compliances as petto_optimize on each problem alone."""
    specs = small_batch(3, seed=13)
    kw = dict(tol=1e-6, check_every=20, max_sweeps=40000)
    hist_alone, phis = [], []
    for spec in specs:
        p = P.Problem(spec)
        p.select_kernel("march2d")
        h, _ = p.optimize(2, solve_kw=kw)
        hist_alone.append(h)
        phis.append(p.get_design())
        p.close()
    probs = [P.Problem(spec) for spec in specs]
    b = P.Batch(probs)
    m, _ = b.optimize(2, solve_kw=kw)
    for i, p in enumerate(probs):
        assert np.array_equal(p.get_design(), phis[i])
        for t in range(2):
            assert m[t, i, 1] == hist_alone[i][t]["compliance"]
            assert m[t, i, 4] == hist_alone[i][t]["sweeps"]
    b.close()
    for p in probs:
        p.close()


def test_batch_rejects_mixed_problems(P):
    from paper_2509_06971_gb300 import capi as C
    a = P.Problem(W.mbb_halfbeam(24, 8).with_(precision="f32", storage="f32"))
    b64 = P.Problem(W.mbb_halfbeam(24, 8))
    c3 = P.Problem(W.cantilever3d(8, 4, 4))
    for other in (b64, c3):
        with pytest.raises(C.PettoError) as e:
            P.Batch([a, other])
        assert e.value.status == C.PETTO_EUNSUPPORTED
    bt = P.Batch([a])
    with pytest.raises(C.PettoError) as e:
        bt.solve(check_every=7)
    assert e.value.status == C.PETTO_EINVAL
    bt.close()
    for p in (a, b64, c3):
        p.close()


def test_batch_state_reused_after_alone_sweeps(P):
    """A problem swept alone an odd number of times (state in the other ping-pong buffer)
    is picked up correctly by the next batched solve."""
    specs = small_batch(2, seed=15)
    kw = dict(tol=1e-6, check_every=20, max_sweeps=40000)
    ref = []
    for spec in specs:
        p = P.Problem(spec)
        p.select_kernel("march2d")
        p.sweep(0, 3, 0.9, 0.9, 0.75, True)
        ref.append((p.solve(**kw), p.get_state(dtype=np.float32)))
        p.close()
    probs = [P.Problem(spec) for spec in specs]
    for p in probs:
        p.select_kernel("march2d")
        p.sweep(0, 3, 0.9, 0.9, 0.75, True)
    b = P.Batch(probs)
    reps = b.solve(**kw)
    for (ra, ua), rb, p in zip(ref, reps, probs):
        assert ra["sweeps"] == rb["sweeps"]
        assert np.array_equal(ua, p.get_state(dtype=np.float32))
    b.close()
    for p in probs:
        p.close()


def test_batch_matches_default_single_path_within_fp32(P):
    """Against problems solved alone on the default 2D kernel (four sweeps per launch,
    node-gather arithmetic): the same iteration in another summation order, so FP32 results
    agree to rounding: converged fields to the solve tolerance and compliance to 1e-4."""
    specs = small_batch(4, seed=17)
    seeds = [80, 81, 82, 83]
    kw = dict(tol=1e-6, check_every=20, max_sweeps=40000)
    alone = _alone(P, specs, seeds, kernel=None, **kw)
    reps, states, _ = _batched(P, specs, seeds, **kw)
    for (ra, ua), rb, ub, spec, sd in zip(alone, reps, states, specs, seeds):
        assert ra["converged"] and rb["converged"]
        op, om = oracle_problem(spec), oracle_materials(spec)
        E = om.modulus(np.asarray(W.random_design(spec, seed=sd), np.float32).astype(np.float64))
        F = op.load_vector()
        ca = float(F @ np.ascontiguousarray(np.asarray(ua, np.float64).T.reshape(-1)))
        cb = float(F @ np.ascontiguousarray(np.asarray(ub, np.float64).T.reshape(-1)))
        assert abs(ca - cb) / abs(ca) < 1e-4
        assert relmax(ub, ua) < 1e-3


def test_select_kernel_names(P):
    from paper_2509_06971_gb300 import capi as C
    p = P.Problem(small_batch(1)[0])
    for name in ("march2d", "march2d/ly8", "gather", "gather/32x4"):
        p.select_kernel(name)
    with pytest.raises(C.PettoError) as e:
        p.select_kernel("tma2")  # a 3D kernel
    assert e.value.status == C.PETTO_EINVAL
    p.close()
