"""Host-side checks that need no GPU: the C ABI library builds, loads and exports every
function include/petto.h declares; argument validation fails cleanly; workload inputs
have the structure the paper's examples give them."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2509_06971_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "petto.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"typedef[^;]*;", "", src)  # function-pointer types of the hooks are not functions
    return sorted(set(re.findall(r"\b(petto_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_function():
    from paper_2509_06971_gb300 import capi
    lib = capi.load()
    declared = header_functions()
    assert len(declared) >= 20
    missing = [f for f in declared if not hasattr(lib, f)]
    assert not missing, missing
    assert sorted(capi.EXPORTED) == declared


def test_status_strings():
    from paper_2509_06971_gb300 import capi
    assert capi.status_string(capi.PETTO_ENOTCONV) == "PETTO_ENOTCONV"
    assert capi.load().petto_last_error(None) == b"no context"


def _create(grid, mat=None, opt=None):
    from paper_2509_06971_gb300 import capi as C
    lib = C.load()
    mod = (ctypes.c_double * 1)(1.0)
    mat = mat or C.petto_materials(C.PETTO_ELASTIC, 1, mod, 1e-9, 0.3, 3.0, C.PETTO_SIMP_MODIFIED)
    opt = opt or C.petto_options(C.PETTO_F32, C.PETTO_F32, 1, None)
    vol = (ctypes.c_double * 1)(0.5)
    ctx = ctypes.c_void_p()
    st = lib.petto_create(ctypes.byref(grid), ctypes.byref(mat), None, None, vol, ctypes.byref(opt),
                          ctypes.byref(ctx))
    if ctx:
        lib.petto_destroy(ctx)
    return st


def test_create_rejects_bad_arguments_before_touching_the_gpu():
    from paper_2509_06971_gb300 import capi as C
    assert _create(C.petto_grid(4, 8, 8, 0, 1.0)) == C.PETTO_EINVAL           # dim
    assert _create(C.petto_grid(2, 0, 8, 0, 1.0)) == C.PETTO_EINVAL           # empty grid
    assert _create(C.petto_grid(2, 8, 8, 0, 0.0)) == C.PETTO_EINVAL           # h
    assert _create(C.petto_grid(2, 8, 8, 0, 1.0),
                   opt=C.petto_options(C.PETTO_F32, C.PETTO_F32, 9, None)) == C.PETTO_EINVAL  # nrhs
    mod = (ctypes.c_double * 1)(1.0)
    bad_nu = C.petto_materials(C.PETTO_ELASTIC, 1, mod, 1e-9, 0.5, 3.0, C.PETTO_SIMP_MODIFIED)
    assert _create(C.petto_grid(2, 8, 8, 0, 1.0), mat=bad_nu) == C.PETTO_EINVAL
    lib = C.load()
    assert lib.petto_sweep(None, 0, 1, 0.9, 1.0, 0.5, 0, None) == C.PETTO_EINVAL
    assert lib.petto_pt_solve(None, None, None) == C.PETTO_EINVAL
    assert lib.petto_residual64(None, None, 0, None, None) == C.PETTO_EINVAL
    assert lib.petto_slab_solve(None, None, C.petto_exchange_fn(), C.petto_allreduce_fn(), C.petto_allreduce_fn(),
                                None, None) == C.PETTO_EINVAL


def test_create_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2509_06971_gb300 import capi as C
    st = _create(C.petto_grid(2, 8, 8, 0, 1.0))
    assert st in (C.PETTO_ECUDA, C.PETTO_ENOMEM)


def test_problem_layer_fails_loudly_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2509_06971_gb300 import capi as C, problem
    with pytest.raises(C.PettoError):
        problem.Problem(W.mbb_halfbeam(8, 4))


# ------------------------------------------------------------ workload inputs

def test_cantilever2d_traction_split():
    spec = W.cantilever2d(64, 32, load_cells=8)
    vals = {node[1]: v for node, comp, v in spec.loads}
    assert abs(sum(vals.values()) + 1.0) < 1e-15
    assert sorted(vals) == list(range(12, 21))
    assert abs(vals[12] + 1 / 16) < 1e-15 and abs(vals[16] + 1 / 8) < 1e-15
    assert all(node[0] == 64 and comp == 1 for node, comp, v in spec.loads)


def test_heat2d_dirichlet_nodes():
    spec = W.heat2d(1024)
    (lo, hi, mask), = spec.boxes
    assert (lo[1], hi[1]) == (461, 563) and hi[1] - lo[1] + 1 == 103 and lo[0] == hi[0] == 0


def test_line_load_3d():
    spec = W.cantilever3d(16, 8, 8)
    tot = sum(v for _, c, v in spec.loads)
    assert abs(tot + 1.0) < 1e-15 and len(spec.loads) == 9
    assert all(node[0] == 16 and node[2] == 0 and c == 2 for node, c, _ in spec.loads)


def test_batch_instances_are_seeded_and_in_range():
    a, b = W.batch2d(48, seed=5), W.batch2d(48, seed=5)
    assert [s.name for s in a] == [s.name for s in b]
    assert all(128 <= s.nx <= 1024 and s.nx % 8 == 0 and s.ny == s.nx // 2 for s in a)
    assert all(0.3 <= s.vol_frac[0] <= 0.5 for s in a)
    kinds = {s.name.split("_")[1] for s in a}
    assert kinds == {"cant", "mbb"}


def test_mbb_initial_design_noise():
    s = W.mbb_halfbeam()
    assert s.phi0.shape == (1, 1200)
    assert np.all(np.abs(s.phi0 - 0.5) <= 0.01) and s.phi0.std() > 0.004
    assert np.array_equal(s.phi0, W.mbb_halfbeam().phi0)


def test_ch_parameters_within_stability_bound():
    import math
    for h_p, dim in [(1 / 20, 2), (1 / 512, 2), (1 / 128, 3), (1 / 1024, 2)]:
        tau, gg = W.ch_params(h_p, dim)
        lam = 4 * dim
        assert tau * (2 * math.pi ** 2 / 64 * lam + gg * lam ** 2) <= 2.0
        assert abs(gg * h_p ** 2 - 3e-5) < 1e-18
