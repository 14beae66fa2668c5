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


@pytest.mark.parametrize("spec", [W.cantilever2d(90, 40, load_cells=6), W.cantilever3d(40, 18, 13)],
                         ids=["2d", "3d"])
def test_static_residual_norm_matches_context_residual(spec):
    torch = pytest.importorskip("torch")
    from paper_2509_06971_gb300 import capi as C, problem
    lib = C.load()
    spec = spec.with_(precision="f32", storage="f32")
    prob = problem.Problem(spec)
    phi = W.random_design(spec, seed=31)
    prob.set_design(phi)
    grid = C.petto_grid(spec.dim, spec.nx, spec.ny, spec.nz if spec.dim == 3 else 0, spec.h)
    E = torch.tensor(prob.get_modulus(np.float32), device="cuda")
    Fh, fixh = _dense_inputs(spec)
    F = torch.tensor(Fh, device="cuda")
    fixed = torch.tensor(fixh, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        u = W.random_state(spec, seed=40 + call).astype(np.float32)
        prob.set_state(u)
        ref, _ = prob.residual(with_field=False)
        ud = torch.tensor(u, device="cuda")
        out = ctypes.c_double(-1.0)
        st = lib.petto_residual_norm_static(ctypes.byref(grid), spec.nu, ctypes.c_void_p(ud.data_ptr()),
                                            ctypes.c_void_p(E.data_ptr()), ctypes.c_void_p(F.data_ptr()),
                                            ctypes.c_void_p(fixed.data_ptr()), ctypes.byref(out),
                                            ctypes.c_void_p(stream))
        assert st == C.PETTO_OK
        assert abs(out.value - ref) <= 1e-5 * ref, (call, out.value, ref)
    big = C.petto_grid(3, 200, 200, 200, 1.0)
    out = ctypes.c_double(0.0)
    assert lib.petto_residual_norm_static(ctypes.byref(big), 0.3, ctypes.c_void_p(ud.data_ptr()),
                                          ctypes.c_void_p(E.data_ptr()), None, None, ctypes.byref(out),
                                          None) == C.PETTO_EINVAL
    prob.close()
