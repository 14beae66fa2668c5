"""Host stand-in for a slab's context, for the multi-rank slab tests on CPU: the oracle's
FP64 APT/PT sweep over the slab's own grid.  The GPU sweeps write the owned node planes
only, so after each oracle sweep the ghost planes (u and w) are put back, and the residual
sums cover the owned planes."""
import numpy as np

from tests._util import oracle_materials, oracle_problem


class OracleSlab:
    np_dtype = np.float64

    def __init__(self, spec):
        self.spec = spec
        self.nrhs, self.ncomp = 1, spec.ncomp
        self.op, self.om = oracle_problem(spec), oracle_materials(spec)
        self.F, self.fixed = self.op.load_vector(), self.op.fixed_mask()
        self.E = self.om.modulus(np.asarray(spec.phi0, np.float64))
        self.u = np.zeros(self.op.ndof)
        self.w = np.zeros(self.op.ndof)
        self.zlo, self.zhi = 0, spec.nz

    # [ncomp][planes][ny+1][nx+1] views of the oracle's interleaved [nodes][ncomp] vectors
    def _grid(self, v):
        s = self.spec
        return v.reshape(s.nz + 1, s.ny + 1, s.nx + 1, self.ncomp)

    def set_owned_planes(self, zlo, zhi, z_global=0):
        self.zlo, self.zhi = zlo, zhi

    def select_kernel(self, name):
        pass

    def plane_shape(self):
        return (self.ncomp, self.spec.ny + 1, self.spec.nx + 1)

    def get_plane(self, k, out):
        out.numpy()[:] = np.moveaxis(self._grid(self.u)[k], -1, 0)
        return out

    def set_plane(self, k, src):
        self._grid(self.u)[k] = np.moveaxis(src.numpy(), 0, -1)

    def set_design(self, phi):
        self.E = self.om.modulus(np.asarray(phi, np.float64))

    def set_state(self, u, w=None):
        self.u = np.ascontiguousarray(np.asarray(u, np.float64).T.reshape(-1))
        self.w = np.zeros_like(self.u) if w is None else np.ascontiguousarray(np.asarray(w, np.float64).T.reshape(-1))

    def get_state(self, dtype=np.float64):
        return np.ascontiguousarray(self.u.reshape(-1, self.ncomp).T).astype(dtype)

    def _owned_r2(self, u):
        R, _ = self.op.residual(self.E, self.F, self.fixed, u)
        return float((self._grid(R)[self.zlo:self.zhi + 1] ** 2).sum())

    def residual(self, with_field=False):
        return self._owned_r2(self.u), None

    def sweep(self, kind, n, a, b, s1, local_dt, want_res=True):
        r2 = 0.0
        for _ in range(n):
            r2 = self._owned_r2(self.u)
            keep_u, keep_w = self.u.copy(), self.w.copy()
            if kind == 0:
                self.op.apt_sweep(self.E, self.F, self.fixed, a, b, self.u, self.w, local_dt=local_dt)
            else:
                self.op.pt_sweep(self.E, self.F, self.fixed, s1, self.u, local_dt=local_dt)
            for v, k in ((self.u, keep_u), (self.w, keep_w)):
                g, gk = self._grid(v), self._grid(k)
                g[:self.zlo] = gk[:self.zlo]
                g[self.zhi + 1:] = gk[self.zhi + 1:]
        return r2

    def slab_solve(self, exchange, allreduce, mode=1, tol=1e-6, a=None, b=None, s1=None, local_dt=None,
                   check_every=50, max_sweeps=200000, momentum=0, refine=False, **_):
        """The hook protocol of petto_slab_solve for the host stand-in: an exchange before every
        sweep, the whole grid's ||F|| and check residuals through allreduce.  Fixed momentum
        (0) or PT only (2)."""
        if momentum not in (0, 2) or mode != 1:
            raise NotImplementedError("the host stand-in runs fixed-momentum APT or PT to a tolerance")
        sp = self.spec  # the constants left out are the workload's, as Problem.solve_opts takes them
        a = sp.apt_a if a is None else a
        b = sp.apt_b if b is None else b
        s1 = sp.pt_s1 if s1 is None else s1
        local_dt = sp.local_dt if local_dt is None else local_dt
        free = self._grid(np.where(self.fixed == 0, self.F, 0.0))[self.zlo:self.zhi + 1]
        fn = float(np.sqrt(allreduce([float((free ** 2).sum())])[0]))
        kind = 0 if momentum == 0 else 1
        sweeps, rn = 0, float("nan")
        while sweeps < max_sweeps:
            exchange()
            check = check_every > 0 and (sweeps + 1) % check_every == 0
            r2 = self.sweep(kind, 1, a, b, s1, local_dt)
            sweeps += 1
            if check or sweeps == max_sweeps:
                rn = float(np.sqrt(allreduce([r2])[0]))
                if not np.isfinite(rn) or rn <= tol * fn:
                    break
        conv = bool(np.isfinite(rn) and rn <= tol * fn)
        return {"sweeps": sweeps, "rel_res": rn / fn if fn else float("nan"), "converged": conv,
                "fell_back_to_pt": False}
