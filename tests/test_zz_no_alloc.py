"""The allocation-free residual norm (petto_residual_norm_static), for callers that may
not allocate GPU memory: it must give the same sum R^2 as the context-based
petto_residual on the same state, call after call (its reduction scratch is a fixed array
shared by every call).  Collected last on purpose."""
import ctypes

import numpy as np
import pytest

from paper_2509_06971_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _dense_inputs(spec):
    """Dense nodal loads and support flags [dim][nodes] from the workload description."""
    nx1, ny1 = spec.nx + 1, spec.ny + 1
    nz1 = spec.nz + 1 if spec.dim == 3 else 1
    F = np.zeros((spec.dim, nz1, ny1, nx1), np.float32)
    for node, comp, val in spec.loads:
        i, j, k = (list(node) + [0, 0])[:3]
        F[comp, k, j, i] += val
    fixed = np.zeros((spec.dim, nz1, ny1, nx1), np.uint8)
    for lo, hi, mask in spec.boxes:
        for a in range(spec.dim):
            if (mask >> a) & 1:
                fixed[a, lo[2]:hi[2] + 1, lo[1]:hi[1] + 1, lo[0]:hi[0] + 1] = 1
    return F.reshape(spec.dim, -1), fixed.reshape(spec.dim, -1)


CASES = {
    "2d": (W.cantilever2d(90, 40, load_cells=6), True, True),
    "3d": (W.cantilever3d(40, 18, 13), True, True),
    "3d_h0.5": (W.cantilever3d(40, 18, 13).with_(h=0.5), True, True),   # h^(d-2) scaling
    "3d_no_loads": (W.cantilever3d(24, 10, 9), False, True),            # F = NULL
    "3d_no_supports": (W.cantilever3d(24, 10, 9), True, False),         # fixed = NULL
    # exactly the limit of 4 194 304 nodes
    "2d_at_limit": (W.mbb_halfbeam(2047, 2047), True, True),
}


@pytest.mark.parametrize("name", list(CASES))
def test_static_residual_norm_matches_context_residual(name):
    torch = pytest.importorskip("torch")
    from paper_2509_06971_gb300 import capi as C, problem
    lib = C.load()
    spec, with_f, with_fixed = CASES[name]
    spec = spec.with_(precision="f32", storage="f32")
    # the context residual of the same problem: no loads / no supports where those are left out
    spec = spec.with_(loads=spec.loads if with_f else [], boxes=spec.boxes if with_fixed else [])
    prob = problem.Problem(spec)
    phi = W.random_design(spec, seed=31)
    prob.set_design(phi)
    grid = C.petto_grid(spec.dim, spec.nx, spec.ny, spec.nz if spec.dim == 3 else 0, spec.h)
    E = torch.tensor(prob.get_modulus(np.float32), device="cuda")
    Fh, fixh = _dense_inputs(spec)
    F = torch.tensor(Fh, device="cuda")
    fixed = torch.tensor(fixh, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):  # two calls in a row share the static scratch
        u = W.random_state(spec, seed=40 + call).astype(np.float32)
        prob.set_state(u)
        ref, _ = prob.residual(with_field=False)
        ud = torch.tensor(u, device="cuda")
        out = ctypes.c_double(-1.0)
        st = lib.petto_residual_norm_static(ctypes.byref(grid), spec.nu, ctypes.c_void_p(ud.data_ptr()),
                                            ctypes.c_void_p(E.data_ptr()),
                                            ctypes.c_void_p(F.data_ptr()) if with_f else None,
                                            ctypes.c_void_p(fixed.data_ptr()) if with_fixed else None,
                                            ctypes.byref(out), ctypes.c_void_p(stream))
        assert st == C.PETTO_OK
        assert abs(out.value - ref) <= 1e-5 * ref, (call, out.value, ref)
    prob.close()


def test_static_residual_norm_rejects_grids_above_the_limit():
    """One node more than the 4 194 304 the static scratch covers: PETTO_EINVAL, checked
    before any launch (the small buffers passed are never read)."""
    torch = pytest.importorskip("torch")
    from paper_2509_06971_gb300 import capi as C
    lib = C.load()
    buf = torch.zeros(16, device="cuda")
    out = ctypes.c_double(0.0)
    for grid in (C.petto_grid(2, 4, 838860, 0, 1.0),      # 5 x 838 861 = 4 194 305 nodes
                 C.petto_grid(3, 200, 200, 200, 1.0)):
        assert lib.petto_residual_norm_static(ctypes.byref(grid), 0.3, ctypes.c_void_p(buf.data_ptr()),
                                              ctypes.c_void_p(buf.data_ptr()), None, None, ctypes.byref(out),
                                              None) == C.PETTO_EINVAL
