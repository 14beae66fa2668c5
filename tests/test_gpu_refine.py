"""The refinement sweep and the adjoint on the 3D cantilever, against the oracle.

* The correction sweep of the FP64 refinement (the variant that does nearly all of the
  benchmark's sweeps: local pseudo-time steps, momentum, and a dense right-hand side that
  the two-row marching kernel reads as FP16 holding r 2^k) is held field by field against
  the oracle's APT sweep (Sec. 3.2 APT system) with F = that FP16 right-hand side restored
  to r: FP16(r 2^k) 2^-k, the power of two 2^k taking max |r| into [2^14, 2^15).  On a ragged
  70 x 40 x 37 grid (several tiles and z segments, supports and loads on tile edges) and on
  the benchmark's full 256 x 128 x 128 grid.
* The hand-written adjoint dC/dphi (Sec. 2.3; reading R3, the total derivative) of the 3D
  cantilever in FP64, on a 32 x 16 x 16 copy: against central finite differences (step
  1e-4) of the GPU compliance on 32 cells drawn by PCG64 seed 3, and against the oracle's
  gradient at the oracle's direct solution.
* The FP64 defect F - K(E) u of the refinement (the z-marching FP64 kernel and the node
  gather) against the oracle's FP64 residual, node by node to 1e-12 of max |R|, on ragged,
  tiny and full-size grids and with several load cases.
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


def fp16_scaled(r):
    """The right-hand side the two-row kernel reads, restored to r's scale: FP16 of r 2^k
    (rounded through FP32, as the conversion kernel does) times 2^-k."""
    m = np.abs(r).max()
    _, e = np.frexp(m)          # m < 2^e
    k = 15 - int(e)
    h = (r * 2.0 ** k).astype(np.float32).astype(np.float16)
    return h.astype(np.float64) * 2.0 ** -k


def _ragged():
    nx, ny, nz = 70, 40, 37
    base = W.cantilever3d(nx, ny, nz)
    loads = base.loads + [((31, 7, 16), 0, 0.7), ((62, 14, 32), 2, 0.25)]
    boxes = base.boxes + [((nx, 0, nz), (nx, ny, nz), 0b010), ((10, 21, 0), (40, 22, 5), 0b101)]
    return base.with_(loads=loads, boxes=boxes)


@pytest.mark.parametrize("name", ["ragged70x40x37", "cantilever3d_256x128x128"])
def test_refinement_sweep_matches_oracle(P, name):
    spec = _ragged() if name.startswith("ragged") else W.cantilever3d(256, 128, 128)
    phi = W.random_design(spec, seed=51)
    d0 = W.random_state(spec, seed=52, scale=1e-3).astype(np.float32)
    w0 = W.random_state(spec, seed=53, scale=1e-4).astype(np.float32)
    r = W.random_state(spec, seed=54, scale=1e-3)
    a, b, s1 = 0.93, 0.9, 0.75
    prob = P.Problem(spec)
    assert prob.kernel_info()[0].startswith("tma3/")  # the benchmark's sweep kernel
    prob.set_design(phi)
    prob.set_state(d0, w0)
    r2a = prob.sweep_rhs(0, 1, r, a, b, 0.0, True)
    ua, wa = prob.get_state(with_w=True)
    if name.startswith("ragged"):
        r2p = prob.sweep_rhs(1, 1, r, 0.0, 0.0, s1, True)
        up = prob.get_state()
    prob.close()

    op, om = oracle_problem(spec), oracle_materials(spec)
    E = om.modulus(np.asarray(phi, np.float32).astype(np.float64))
    fixed = op.fixed_mask()
    F = nodes_to_oracle(fp16_scaled(r))
    dinv = op.inverse_diag(E)
    uo, wo = nodes_to_oracle(d0.astype(np.float64)), nodes_to_oracle(w0.astype(np.float64))
    r2a_o = op.apt_sweep(E, F, fixed, a, b, uo, wo, local_dt=True, dinv=dinv)
    un, wn = oracle_to_nodes(uo, 3), oracle_to_nodes(wo, 3)
    for c in range(3):
        assert rel_l2(ua[c], un[c]) < 1e-5, c
        assert rel_l2(wa[c], wn[c]) < 1e-5, c
    assert abs(r2a - r2a_o) < 1e-5 * r2a_o
    if name.startswith("ragged"):
        r2p_o = op.pt_sweep(E, F, fixed, s1, uo, local_dt=True, dinv=dinv)
        un = oracle_to_nodes(uo, 3)
        for c in range(3):
            assert rel_l2(up[c], un[c]) < 1e-5, c
        assert abs(r2p - r2p_o) < 1e-5 * r2p_o


def test_adjoint_3d_cantilever_matches_finite_differences_and_oracle(P):
    torch = pytest.importorskip("torch")
    from paper_2509_06971_gb300.problem import PettoCompliance
    spec = W.cantilever3d(32, 16, 16).with_(precision="f64", storage="f64")
    prob = P.Problem(spec)
    phi0 = W.random_design(spec, seed=31, lo=0.2, hi=0.8)
    phi = torch.tensor(phi0, dtype=torch.float64, device="cuda", requires_grad=True)
    kw = dict(tol=1e-12, max_sweeps=2000000, check_every=20)
    Cv = PettoCompliance.apply(phi, prob, **kw)
    Cv.backward()
    g = phi.grad.detach().cpu().numpy()
    # each compliance is exact to |F . (u - u*)| = |u* . R| <= ||u|| ||R||, ||R|| <= tol ||F||:
    # the difference quotient carries at most 2 ||u|| tol ||F|| / (2 h) beside its O(h^2) term
    solve_err = np.linalg.norm(prob.get_state()) * kw["tol"] * np.linalg.norm(oracle_problem(spec).load_vector())
    cells = np.random.default_rng(3).choice(spec.ncells, size=32, replace=False)
    h = 1e-4
    for c in cells:
        d = torch.zeros_like(phi)
        d[0, c] = h
        cp = PettoCompliance.apply((phi + d).detach(), prob, **kw).item()
        cm = PettoCompliance.apply((phi - d).detach(), prob, **kw).item()
        fd = (cp - cm) / (2 * h)
        assert abs(fd - g[0, c]) < 1e-5 * abs(g[0, c]) + solve_err / h, (c, fd, g[0, c])
    prob.close()
    # the oracle's gradient at its own direct solution of the same design
    op, om = oracle_problem(spec), oracle_materials(spec)
    E = om.modulus(phi0)
    u = op.direct_solve(E, op.load_vector(), op.fixed_mask())
    s, Co = om.sensitivity(phi0, E, op.cell_energy(u))
    assert abs(Cv.item() - Co) < 1e-9 * Co
    assert np.abs(g - s).max() < 1e-7 * np.abs(s).max()


def _dyadic_design(spec, seed):
    """A seeded design of densities in {0, 1/4, 1/2, 3/4, 1}: rho^3 and the SIMP modulus
    rounded to FP32 are then the same whether computed in FP32 or in FP64 and rounded, so
    the oracle's FP64 moduli rounded to FP32 are the context's FP32 moduli exactly."""
    return np.round(np.asarray(W.random_design(spec, seed=seed), np.float64) * 4.0) / 4.0


def _defect_oracle(spec, phi, u, loads=None):
    """The oracle's FP64 residual F - K(E) u with its moduli rounded to FP32 (the defect
    runs with the FP32 moduli of an FP32 context)."""
    op, om = oracle_problem(spec, loads=loads), oracle_materials(spec)
    E = om.modulus(phi).astype(np.float32).astype(np.float64)
    R, r2 = op.residual(E, op.load_vector(), op.fixed_mask(), nodes_to_oracle(u))
    return oracle_to_nodes(R, spec.ncomp), r2


@pytest.mark.parametrize("name", ["ragged70x40x37", "tiny3x2x1", "cantilever3d_256x128x128"])
def test_fp64_defect_matches_oracle(P, name, monkeypatch):
    """The FP64 defect of the refinement, R = F - K(E) u in FP64 with the FP32 moduli (the
    z-marching defect kernel), field by field against the oracle's FP64 residual at the same
    state, and against the node-gather defect kernel: on a ragged grid of several tiles and z
    segments with supports ending inside segments and loads on tile edges, on a grid smaller
    than one tile, and on the benchmark's full grid."""
    if name.startswith("ragged"):
        spec = _ragged()
    elif name.startswith("tiny"):
        spec = W.cantilever3d(3, 2, 1)
    else:
        spec = W.cantilever3d(256, 128, 128)
    phi = _dyadic_design(spec, 61)
    u = W.random_state(spec, seed=62, scale=1e-2)
    out = {}
    for kernel in ("march", "gather"):
        if kernel == "gather":
            monkeypatch.setenv("PETTO_DEFECT", "gather")
        prob = P.Problem(spec)
        prob.set_design(phi)
        out[kernel] = prob.residual64(u)
        prob.close()
    monkeypatch.delenv("PETTO_DEFECT", raising=False)
    Ro, r2o = _defect_oracle(spec, phi, u)
    scale = np.abs(Ro).max()
    for kernel, (r2, R) in out.items():
        assert np.abs(R - Ro).max() <= 1e-12 * scale, (kernel, np.abs(R - Ro).max() / scale)
        assert abs(r2 - r2o) <= 1e-12 * r2o, kernel
    # supports hold R = 0 exactly
    fixed = oracle_to_nodes(oracle_problem(spec).fixed_mask().astype(np.float64), 3) != 0
    assert np.all(out["march"][1][fixed] == 0.0)


def test_fp64_defect_of_several_load_cases(P):
    """One defect launch per load case, the sums accumulated across them."""
    spec, cases = W.multirhs3d(40, 20, 20, n_rhs=3, seed=4)
    prob = P.Problem(spec, nrhs=3, load_cases=cases)
    phi = _dyadic_design(spec, 63)
    prob.set_design(phi)
    u = np.random.default_rng(64).standard_normal((9, spec.nnodes)) * 1e-2
    r2, R = prob.residual64(u)
    prob.close()
    r2o = 0.0
    for r, case in enumerate(cases):
        Ro, r2c = _defect_oracle(spec, phi, u[3 * r:3 * r + 3], loads=case)
        assert np.abs(R[3 * r:3 * r + 3] - Ro).max() <= 1e-12 * np.abs(Ro).max(), r
        r2o += r2c
    assert abs(r2 - r2o) <= 1e-12 * r2o


def test_fp64_defect_rejects_fp64_contexts(P):
    from paper_2509_06971_gb300 import capi as C
    spec = W.cantilever3d(8, 4, 4).with_(precision="f64", storage="f64")
    prob = P.Problem(spec)
    with pytest.raises(C.PettoError) as e:
        prob.residual64(np.zeros((3, spec.nnodes)))
    assert e.value.status == C.PETTO_EUNSUPPORTED
    prob.close()
