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
        self.set_design(spec.phi0)
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

    # ---------------------------------------------------------------- decomposed design step
    # The hook protocol of petto_slab_design_step on the host stand-in, from the oracle's
    # pieces: cell energies, sensitivity, the update written with the slabs' sums, and the
    # Cahn-Hilliard half steps with the oracle's no-flux cell Laplacian on the held layers
    # plus the copy of the layer above.

    def set_design(self, phi):
        self.phi = np.array(phi, dtype=np.float64).reshape(self.om.n_phases, -1)
        self.E = self.om.modulus(self.phi)
        s = self.spec
        self.mu = np.zeros(self.phi.shape[1])
        self.phi_hi = np.zeros((self.phi.shape[0], s.nx * s.ny))
        self.mu_hi = np.zeros(s.nx * s.ny)

    def get_design(self, dtype=np.float64):
        return self.phi.astype(dtype)

    def layer_bytes(self, field):
        return self.spec.nx * self.spec.ny * 8 if field in (0, 1) else 0

    def _layer(self, field, phase, k):
        s, pl = self.spec, self.spec.nx * self.spec.ny
        if k == s.nz:
            return self.phi_hi[phase] if field == 0 else self.mu_hi
        arr = self.phi[phase] if field == 0 else self.mu
        return arr[k * pl:(k + 1) * pl]

    def get_layer(self, field, phase, k, out):
        out.numpy().view(np.float64)[:] = self._layer(field, phase, k)
        return out

    def set_layer(self, field, phase, k, src):
        self._layer(field, phase, k)[:] = src.numpy().view(np.float64)

    def _lap(self, v, hi):
        """No-flux cell Laplacian of v over the held layers, with the layer above (hi) when the
        slab has an upper neighbour."""
        from oracle import oracle as O
        s = self.spec
        if hi is None:
            return O.OracleProblem(3, s.nx, s.ny, s.nz).cell_laplacian(v)
        ext = np.concatenate([v, hi])
        return O.OracleProblem(3, s.nx, s.ny, s.nz + 1).cell_laplacian(ext)[:v.size]

    def slab_design_step(self, exchange, exchange_layer, allreduce, allreduce_max, solve_kw=None, pf_kw=None):
        from oracle import oracle as O
        s = self.spec
        sk = dict(solve_kw or {})
        rep = self.slab_solve(exchange, allreduce, **sk)
        exchange()
        pl = s.nx * s.ny
        c0, c1 = self.zlo * pl, min(self.zhi + 1, s.nz) * pl  # own cell layers
        ncount = allreduce([float(c1 - c0)])[0]
        e = self.op.cell_energy(self.u)
        sens, _ = self.om.sensitivity(self.phi, self.E, e)
        C = allreduce([float((self.E * e)[c0:c1].sum())])[0]
        own_nodes = self._grid(np.ones_like(self.u))
        own_nodes[:self.zlo] = 0
        own_nodes[self.zhi + 1:] = 0
        W = allreduce([float((self.F * self.u * own_nodes.reshape(-1)).sum())])[0]
        smax = allreduce_max([float(np.abs(sens[p]).max()) for p in range(self.phi.shape[0])])
        pf = dict(alpha_h=s.alpha_h, kappa_v=s.kappa_v, kappa_1=s.kappa_1, gamma_g=s.gamma_g, tau=s.tau,
                  vol_mode=s.vol_mode, n_bisect=s.n_bisect)
        pf.update(pf_kw or {})
        P = self.phi.shape[0]
        g = np.stack([pf["alpha_h"] * sens[p] / smax[p] if smax[p] > 0 else 0 * sens[p] for p in range(P)])
        dv = self.phi - g - pf["kappa_1"] * (self.phi.sum(axis=0) - 1.0)
        lam = np.zeros(P)
        if pf["vol_mode"] == O.PROJECTED:
            lo, hi = np.full(P, -2.0), np.full(P, 2.0)
            for _ in range(pf["n_bisect"]):
                mid = 0.5 * (lo + hi)
                sums = allreduce([float(np.clip(dv[p, c0:c1] - mid[p], 0, 1).sum()) for p in range(P)])
                for p in range(P):
                    if sums[p] / ncount > s.vol_frac[p]:
                        lo[p] = mid[p]
                    else:
                        hi[p] = mid[p]
            lam = 0.5 * (lo + hi)
            self.phi = np.clip(dv - lam[:, None], 0.0, 1.0)
        else:
            mean = np.array(allreduce([float(self.phi[p, c0:c1].sum()) for p in range(P)])) / ncount
            lam = mean
            self.phi = dv - (pf["kappa_v"] * (mean - np.asarray(s.vol_frac)))[:, None]
        upper = self.zhi < s.nz  # the slab has an upper neighbour
        for p in range(P):
            exchange_layer(0, p)
            self.mu[:] = [O.double_well_deriv(x) for x in self.phi[p]] - pf["gamma_g"] * self._lap(
                self.phi[p], self.phi_hi[p] if upper else None)
            exchange_layer(1, p)
            self.phi[p] += pf["tau"] * self._lap(self.mu, self.mu_hi if upper else None)
        for p in range(P):
            exchange_layer(0, p)
        self.E = self.om.modulus(self.phi)
        mean0 = allreduce([float(self.phi[0, c0:c1].sum())])[0] / ncount
        return {"step": 1, "compliance": C, "work": W, "rel_res": rep["rel_res"], "sweeps": rep["sweeps"],
                "seconds": 0.0, "mean_phi0": mean0, "lambda0": float(lam[0]), "converged": rep["converged"]}
