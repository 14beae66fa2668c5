"""The benchmark's workload at full size -- the 3D cantilever 256 x 128 x 128 in FP32, on the
sweep kernel and launch configuration that bench.py times -- against the oracle; and the
2D cantilever 1024 x 512 and heat 1024 x 1024 grids on their default kernel (four sweeps
per launch on shared-memory copies of the tiles).

* APT and PT sweeps from a seeded random state and design (one each in 3D, one launch of
  four each in 2D), field by field against the oracle's sweeps.  Global pseudo-time steps: the oracle's local-step form recomputes
  diag(K) on every call, about a minute per sweep at this size; the local-step path is held
  element by element on the smaller grids of test_gpu_parity.py.
* The refined solve of the first design iteration (local steps, adaptive momentum, FP64
  refinement with FP16 right-hand sides), by what holds at any size: the oracle's energy
  of the returned state equals its work F . u (the state solves K u = F), and the GPU's
  compliance and sensitivity field equal the oracle's for that state.
"""
import numpy as np
import pytest

from paper_2509_06971_gb300 import workloads as W
from tests._util import nodes_to_oracle, oracle_materials, oracle_problem, oracle_to_nodes

pytestmark = pytest.mark.gpu

SIZE = (256, 128, 128)
# the other full-size workloads: the 2D cantilever and heat grids
FULL_2D = {"cantilever2d_1024x512": lambda: W.cantilever2d(1024, 512), "heat2d_1024x1024": lambda: W.heat2d(1024)}


@pytest.fixture(scope="module")
def P():
    from paper_2509_06971_gb300 import problem as PR
    return PR


def rel_l2(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _spec(name):
    return W.cantilever3d(*SIZE) if name == "cantilever3d" else FULL_2D[name]()


@pytest.mark.parametrize("name,kernel", [("cantilever3d", "tma3/"), ("cantilever2d_1024x512", "tb2d/k4/"),
                                         ("heat2d_1024x1024", "tb2d/k4/")])
def test_fullsize_sweeps_match_oracle(P, name, kernel):
    spec = _spec(name)
    phi = W.random_design(spec, seed=41)
    u0 = W.random_state(spec, seed=42).astype(np.float32)
    w0 = W.random_state(spec, seed=43, scale=0.1).astype(np.float32)
    a, b, s1 = 0.95, 0.05, 0.1
    prob = P.Problem(spec)
    assert prob.kernel_info()[0].startswith(kernel)  # the kernel the benchmark times
    prob.set_design(phi)
    prob.set_state(u0, w0)
    n = 4 if kernel.startswith("tb2d") else 1  # the 2D kernel runs four sweeps per launch
    r2a = prob.sweep(0, n, a, b, 0.0, False)
    r2p = prob.sweep(1, n, 0.0, 0.0, s1, False)
    ug, wg = prob.get_state(with_w=True)
    prob.close()

    op, om = oracle_problem(spec), oracle_materials(spec)
    E = om.modulus(np.asarray(phi, np.float32).astype(np.float64))
    F, fixed = op.load_vector(), op.fixed_mask()
    uo, wo = nodes_to_oracle(u0.astype(np.float64)), nodes_to_oracle(w0.astype(np.float64))
    for _ in range(n):
        r2a_o = op.apt_sweep(E, F, fixed, a, b, uo, wo)
    for _ in range(n):
        r2p_o = op.pt_sweep(E, F, fixed, s1, uo)
    un, wn = oracle_to_nodes(uo, spec.ncomp), oracle_to_nodes(wo, spec.ncomp)
    for c in range(spec.ncomp):
        assert rel_l2(ug[c], un[c]) < 1e-5
        assert rel_l2(wg[c], wn[c]) < 1e-5
    assert abs(r2a - r2a_o) < 1e-5 * r2a_o
    assert abs(r2p - r2p_o) < 1e-5 * r2p_o


def test_fullsize_refined_solve(P):
    spec = W.cantilever3d(*SIZE)
    prob = P.Problem(spec)
    rep = prob.solve(tol=1e-6)
    assert rep["converged"] and rep["rel_res"] <= 1e-6
    Cg, Wg, sg = prob.sensitivity()
    u = prob.get_state()
    prob.close()

    op, om = oracle_problem(spec), oracle_materials(spec)
    phi = np.asarray(spec.phi0, np.float32).astype(np.float64)
    uo = nodes_to_oracle(u)
    so, Co = om.sensitivity(phi, om.modulus(phi), op.cell_energy(uo))
    Wo = float(op.load_vector() @ uo)
    # energy equals work: the state solves K u = F.  C - W = -u . R, bounded by
    # ||u|| ||R|| <= ||u|| ||F|| 1e-6, about 1e-4 C on this grid (||u|| spans 12.8 M DOFs,
    # F one loaded edge); an unconverged or wrong state misses by far more
    assert abs(Co - Wo) < 1e-3 * Co
    assert abs(Cg - Co) < 1e-5 * Co    # the GPU's compliance of its own state
    assert abs(Wg - Wo) < 1e-5 * Co
    assert rel_l2(sg, so) < 1e-5


MULTIMAT = (384, 192, 192)


def test_fullsize_multimat_bf16_modulus_and_sweep(P):
    """The multi-material workload at full size (384 x 192 x 192, void + two solids, design
    stored in BF16, arithmetic in FP32): the modulus equals the oracle's interpolation of
    the stored design, and one APT sweep on that modulus matches the oracle's sweep."""
    spec = W.multimat3d(*MULTIMAT, storage="bf16")
    prob = P.Problem(spec)
    prob.set_design(W.random_design(spec, seed=45, lo=0.05, hi=0.9))
    phi_st = prob.get_design()  # the stored design, rounded to BF16
    Eg = prob.get_modulus()
    om = oracle_materials(spec)
    Eo = om.modulus(phi_st)
    assert np.abs(Eg - Eo).max() <= 1e-6 * np.abs(Eo).max()
    u0 = W.random_state(spec, seed=46).astype(np.float32)
    prob.set_state(u0)
    a, b = 0.95, 0.05
    r2 = prob.sweep(0, 1, a, b, 0.0, False)
    ug, wg = prob.get_state(with_w=True)
    prob.close()

    op = oracle_problem(spec)
    F, fixed = op.load_vector(), op.fixed_mask()
    uo = nodes_to_oracle(u0.astype(np.float64))
    wo = np.zeros_like(uo)
    r2o = op.apt_sweep(Eg, F, fixed, a, b, uo, wo)  # on the GPU's modulus, so both sweep the same E
    un, wn = oracle_to_nodes(uo, 3), oracle_to_nodes(wo, 3)
    for c in range(3):
        assert rel_l2(ug[c], un[c]) < 1e-5
        assert rel_l2(wg[c], wn[c]) < 1e-5
    assert abs(r2 - r2o) < 1e-5 * r2o


MULTIRHS = (192, 96, 96)


def test_fullsize_multi_rhs_sweep(P):
    """Four load cases at full size (192 x 96 x 96, one marching launch per case sharing the
    step constants): one APT sweep of every case matches the oracle's sweep of that case."""
    spec, cases = W.multirhs3d(*MULTIRHS, n_rhs=4)
    phi = W.random_design(spec, seed=47)
    u0 = np.concatenate([W.random_state(spec, seed=48 + r) for r in range(4)]).astype(np.float32)
    prob = P.Problem(spec, nrhs=4, load_cases=cases)
    assert prob.kernel_info()[0].startswith("tma3/")
    prob.set_design(phi)
    prob.set_state(u0)
    a, b = 0.95, 0.05
    r2 = prob.sweep(0, 1, a, b, 0.0, False)
    ug, wg = prob.get_state(with_w=True)
    prob.close()

    om = oracle_materials(spec)
    E = om.modulus(np.asarray(phi, np.float32).astype(np.float64))
    r2o = 0.0
    for r, case in enumerate(cases):
        op = oracle_problem(spec, loads=case)
        uo = nodes_to_oracle(u0[3 * r:3 * r + 3].astype(np.float64))
        wo = np.zeros_like(uo)
        r2o += op.apt_sweep(E, op.load_vector(), op.fixed_mask(), a, b, uo, wo)
        un, wn = oracle_to_nodes(uo, 3), oracle_to_nodes(wo, 3)
        for c in range(3):
            assert rel_l2(ug[3 * r + c], un[c]) < 1e-5
            assert rel_l2(wg[3 * r + c], wn[c]) < 1e-5
    assert abs(r2 - r2o) < 1e-5 * r2o


N_BATCH = 48


def test_fullsize_batch_paper_schedule(P):
    """The 48-problem batch at full size (128 x 64 .. 1024 x 512 cells, one launch per sweep
    over every problem): two APT and two PT sweeps of the paper's schedule (global steps,
    fixed damping); the smallest and the largest problem match the oracle's sweeps."""
    specs = W.batch2d(N_BATCH)
    probs = [P.Problem(s) for s in specs]
    b = P.Batch(probs)
    kw = dict(mode=0, n_apt=2, n_pt=2, a=0.9, b=0.05, s1=0.1, local_dt=False, momentum=0, check_every=2)
    reps = b.solve(**kw)
    sizes = [s.ncells for s in specs]
    picks = sorted({int(np.argmin(sizes)), int(np.argmax(sizes))})
    states = {i: probs[i].get_state() for i in picks}
    b.close()
    for p in probs:
        p.close()
    for i in picks:
        spec = specs[i]
        assert reps[i]["apt_sweeps"] == 2 and reps[i]["pt_sweeps"] == 2
        op, om = oracle_problem(spec), oracle_materials(spec)
        u = np.zeros(op.ndof)
        op.solve(om.modulus(np.asarray(spec.phi0, np.float32).astype(np.float64)), op.load_vector(), op.fixed_mask(),
                 u, mode=0, n_apt=2, n_pt=2, a=0.9, b=0.05, s1=0.1, check_every=2, local_dt=False)
        un = oracle_to_nodes(u, spec.ncomp)
        for c in range(spec.ncomp):
            assert rel_l2(states[i][c], un[c]) < 1e-5


PAPER_LOOPS = {
    "heat2d_paper_512": lambda: W.heat2d_paper(512),
    "mbb_multimat2d_512x128": lambda: W.mbb_multimat2d(512, 128),
    "multimat3d_paper_256x17x85": lambda: W.multimat3d_paper(256, 17, 85),
    "drone3d_128x64x128": lambda: W.drone3d(128, 64, 128),
}


@pytest.mark.parametrize("name", list(PAPER_LOOPS))
def test_fullsize_paper_loop_sweeps(P, name):
    """The paper's own loops at their full sizes (its grids, materials, global steps and
    fixed damping): the solve's first three APT and two PT sweeps from the initial design
    match the oracle's."""
    spec = PAPER_LOOPS[name]()
    prob = P.Problem(spec)
    rep = prob.solve(mode=0, n_apt=3, n_pt=2, check_every=0)
    assert rep["apt_sweeps"] == 3 and rep["pt_sweeps"] == 2
    ug = prob.get_state()
    prob.close()
    op, om = oracle_problem(spec), oracle_materials(spec)
    u = np.zeros(op.ndof)
    op.solve(om.modulus(np.asarray(spec.phi0, np.float32).astype(np.float64)), op.load_vector(), op.fixed_mask(), u,
             mode=0, n_apt=3, n_pt=2, a=spec.apt_a, b=spec.apt_b, s1=spec.pt_s1, check_every=0,
             local_dt=spec.local_dt, momentum=0)
    un = oracle_to_nodes(u, spec.ncomp)
    for c in range(spec.ncomp):
        assert rel_l2(ug[c], un[c]) < 1e-5
