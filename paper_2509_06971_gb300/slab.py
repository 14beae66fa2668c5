"""Decomposition of one 3D grid into z slabs: the exchange step of a state solve spread over
several contexts (GPUs).

The sweep of Sec. 2.2 updates each node from its 3 x 3 x 3 node neighbourhood and its eight
cells, so cutting the grid along z needs, per interface and sweep, one node plane of u from
each side.  Slab s owns node planes k0..k1 of the whole grid; its context holds those planes
plus one ghost plane on each interior side, and the cell layers between them, with the
loads of its own planes and the supports clipped to its range.  Before every sweep each
interface plane goes from its owner into the neighbour's ghost plane; the sweep writes the
owned planes only (``petto_set_owned_planes``), so the owned planes follow the whole grid's
sweeps, and the residual sums of the slabs add up to the whole grid's.  The modulus of the
ghost cell layers comes from the design, which every slab holds for its own range.

Two drivers share this host logic:

* ``SlabGrid`` keeps every slab in this process (several contexts on one GPU; planes copied
  device to device on the shared stream);
* ``DistributedSlabs`` gives each rank of a ``torch.distributed`` group one slab and moves
  the planes with point-to-point messages (NCCL between GPUs, gloo between host processes)
  and the residual with an all-reduce.

The state solve is decomposed: sweeps, residuals, and the solve loop itself, which runs in
the library (``petto_slab_solve``) with this module's exchange and all-reduce as its hooks
(fixed or adaptive-restart momentum, PT, and the FP64 refinement of FP32 states: each slab
keeps the FP64 state of its planes and ghost planes, its own planes' defect, the whole
grid's defect norm and the whole grid's scale of the FP16 right-hand side).  So is the
design loop (``petto_slab_design_step``): a slab owns the cell layers whose lower node plane
it owns, holds the layer below its first one (its ghost layer) and keeps a copy of the layer
above its top one; the sensitivity, the update and the modulus are computed on every held
layer (a ghost layer gets its owner's bits), the compliance, the means and the bisection's
sums over the owned ones (all-reduced), and the Cahn-Hilliard step exchanges phi's and mu's
interface layers around each half step.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def slab_ranges(nz: int, n: int) -> list[tuple[int, int]]:
    """Owned node planes (k0, k1), inclusive, of n slabs over the nz + 1 node planes of a
    grid with nz cell layers: contiguous, in order, sizes differing by at most one."""
    planes = nz + 1
    if not 1 <= n <= planes:
        raise ValueError(f"cannot cut {planes} node planes into {n} slabs")
    base, extra = divmod(planes, n)
    out, k = [], 0
    for s in range(n):
        m = base + (1 if s < extra else 0)
        out.append((k, k + m - 1))
        k += m
    return out


@dataclass(frozen=True)
class SlabGeom:
    """Node planes of one slab in whole-grid indices: owned k0..k1, held g0..g1 (owned plus
    the ghost planes).  Local plane index = global - g0."""
    k0: int
    k1: int
    g0: int
    g1: int

    @property
    def zlo(self) -> int:
        return self.k0 - self.g0

    @property
    def zhi(self) -> int:
        return self.k1 - self.g0

    @property
    def nz(self) -> int:
        """cell layers of the slab's grid"""
        return self.g1 - self.g0


def slab_geometry(nz: int, n: int) -> list[SlabGeom]:
    return [SlabGeom(k0, k1, max(k0 - 1, 0), min(k1 + 1, nz)) for k0, k1 in slab_ranges(nz, n)]


def slab_loads(loads, g: SlabGeom):
    """Point loads on the slab's owned planes, in its local indices."""
    return [((i, j, k - g.g0), c, v) for (i, j, k), c, v in loads if g.k0 <= k <= g.k1]


def slab_boxes(boxes, g: SlabGeom):
    """Support boxes clipped to the planes the slab holds, in its local indices."""
    out = []
    for lo, hi, mask in boxes:
        klo, khi = max(lo[2], g.g0), min(hi[2], g.g1)
        if klo <= khi:
            out.append(((lo[0], lo[1], klo - g.g0), (hi[0], hi[1], khi - g.g0), mask))
    return out


def slab_cells(field, spec, g: SlabGeom) -> np.ndarray:
    """[P][cells] of the whole grid -> the slab's cell layers g0..g1-1."""
    f = np.asarray(field)
    return np.ascontiguousarray(f.reshape(f.shape[0], spec.nz, spec.ny, spec.nx)[:, g.g0:g.g1].reshape(f.shape[0], -1))


def slab_nodes(u, spec, g: SlabGeom) -> np.ndarray:
    """[C][nodes] of the whole grid -> the slab's node planes g0..g1."""
    a = np.asarray(u)
    return np.ascontiguousarray(
        a.reshape(a.shape[0], spec.nz + 1, spec.ny + 1, spec.nx + 1)[:, g.g0:g.g1 + 1].reshape(a.shape[0], -1))


def slab_spec(spec, g: SlabGeom):
    """The problem a slab's context solves: its planes, loads, supports and design."""
    if spec.dim != 3:
        raise ValueError("slabs cut a 3D grid along z")
    phi0 = None if spec.phi0 is None else slab_cells(spec.phi0, spec, g)
    return spec.with_(name=f"{spec.name}_z{g.k0}-{g.k1}", nz=g.nz, loads=slab_loads(spec.loads, g),
                      boxes=slab_boxes(spec.boxes, g), phi0=phi0, keepout=None)


def interface_copies(geom: list[SlabGeom]):
    """The plane copies of one exchange, (src slab, src local plane, dst slab, dst local
    plane): each interface's two owned boundary planes into the neighbours' ghost planes."""
    out = []
    for s in range(len(geom) - 1):
        lo, hi = geom[s], geom[s + 1]
        out.append((s, lo.zhi, s + 1, 0))          # lo's top owned plane -> hi's lower ghost
        out.append((s + 1, hi.zlo, s, lo.nz))      # hi's bottom owned plane -> lo's upper ghost
    return out


def owned_layers(g: SlabGeom, nz: int) -> tuple[int, int]:
    """The cell layers a slab owns, whole-grid indices [c0, c1): those whose lower node plane
    it owns."""
    return g.k0, min(g.k1 + 1, nz)


def design_step_ok(geom: list[SlabGeom]) -> bool:
    """The decomposed design step needs every slab to own two node planes or more: then
    every slab owns a cell layer, and a slab's top layer has the grid's next layer above it
    exactly when the slab has an upper neighbour."""
    return all(g.k1 > g.k0 for g in geom)


def interface_layer_copies(geom: list[SlabGeom]):
    """The cell-layer copies of one design-field exchange, (src slab, src local layer, dst
    slab, dst local layer): the lower slab's top layer into the upper slab's ghost layer 0,
    and the upper slab's first own layer (1) into the lower slab's copy of the layer above
    its top (local index nz)."""
    out = []
    for s in range(len(geom) - 1):
        lo = geom[s]
        out.append((s, lo.nz - 1, s + 1, 0))
        out.append((s + 1, 1, s, lo.nz))
    return out


def _torch():
    import torch
    return torch


class _SlabDriver:
    """What both drivers do around their slabs' contexts."""

    def _gather_owned(self, parts, ncomp):
        spec = self.spec
        out = np.empty((ncomp, spec.nz + 1, spec.ny + 1, spec.nx + 1), dtype=parts[0][1].dtype)
        for g, u in parts:
            ul = u.reshape(ncomp, g.nz + 1, spec.ny + 1, spec.nx + 1)
            out[:, g.k0:g.k1 + 1] = ul[:, g.zlo:g.zhi + 1]
        return out.reshape(ncomp, -1)

    def solve(self, tol: float = 1e-6, kind: int = 0, a: float | None = None, b: float | None = None,
              s1: float | None = None, local_dt: bool | None = None, check_every: int = 50,
              max_sweeps: int = 200000, momentum: int | None = None, refine: bool = True) -> dict:
        """The state solve over the slabs, one petto_slab_solve per slab (the loop runs in the
        library; this driver supplies its exchange and all-reduce hooks): APT with fixed
        momentum (kind 0, momentum 0), PT only (kind 1, momentum 2) or the adaptive-restart
        momentum (momentum 1), until ||R|| <= tol ||F|| of the whole grid at a check (every
        check_every sweeps) or max_sweeps; FP32 grids below tol 1e-3 with the FP64 refinement
        (refine, as Problem.solve)."""
        if momentum is None:
            momentum = 0 if kind == 0 else 2
        kw = dict(mode=1, tol=tol, check_every=check_every, max_sweeps=max_sweeps, momentum=momentum, refine=refine)
        # constants left out take the problem's defaults (Problem.solve_opts), as a whole-grid solve does
        kw.update({k: v for k, v in dict(a=a, b=b, s1=s1, local_dt=local_dt).items() if v is not None})
        rep = self._slab_solve(kw)
        return {"sweeps": rep["sweeps"], "rel_res": rep["rel_res"], "converged": rep["converged"],
                "fell_back_to_pt": rep["fell_back_to_pt"]}

    def design_step(self, solve_kw: dict | None = None, pf_kw: dict | None = None) -> dict:
        """One design loop over the slabs (petto_slab_design_step on every slab, this driver
        supplying the plane and cell-layer exchanges and the sums and maxima): the whole
        grid's metrics.  The state solve as solve()."""
        if not design_step_ok(self.geom):
            raise ValueError("the decomposed design step needs two node planes or more per slab")
        kw = dict(mode=1)
        kw.update(solve_kw or {})
        return self._slab_design_step(kw, dict(pf_kw or {}))

    def _gather_design(self, parts):
        spec = self.spec
        out = None
        for g, phi in parts:
            phi = np.asarray(phi)
            if out is None:
                out = np.empty((phi.shape[0], spec.nz, spec.ny, spec.nx), dtype=phi.dtype)
            c0, c1 = owned_layers(g, spec.nz)
            out[:, c0:c1] = phi.reshape(phi.shape[0], g.nz, spec.ny, spec.nx)[:, c0 - g.g0:c1 - g.g0]
        return out.reshape(out.shape[0], -1)


class SlabGrid(_SlabDriver):
    """Every slab of the grid in this process: n contexts on the current GPU, exchanged by
    device-to-device plane copies on the shared stream."""

    def __init__(self, spec, n_slabs: int, *, kernel: str | None = None, nrhs: int = 1, load_cases=None,
                 **problem_kw):
        from .problem import Problem
        torch = _torch()
        self.spec = spec
        self.geom = slab_geometry(spec.nz, n_slabs)
        self.probs = []
        if problem_kw.get("stream") is None:
            # one stream for every slab's context: the plane copies between contexts and the
            # sweeps are then ordered without host synchronisation
            self._stream = torch.cuda.Stream()
            problem_kw["stream"] = self._stream.cuda_stream
        try:
            for g in self.geom:
                cases = None if load_cases is None else [slab_loads(c, g) for c in load_cases]
                p = Problem(slab_spec(spec, g), nrhs=nrhs, load_cases=cases, **problem_kw)
                self.probs.append(p)
                if kernel:
                    p.select_kernel(kernel)
                p.set_owned_planes(g.zlo, g.zhi, g.g0)
        except Exception:
            self.close()  # the contexts made so far
            raise
        p0 = self.probs[0]
        self.ncomp = p0.nrhs * p0.ncomp
        dt = torch.float64 if p0.np_dtype == np.float64 else torch.float32
        self._buf = torch.empty(p0.plane_shape(), dtype=dt, device="cuda")
        self._lbuf = None  # cell-layer copies of the design step
        # ||F|| over the free DOFs: the residual of the zero state, summed over the slabs
        self.f_norm = float(np.sqrt(sum(p.residual(with_field=False)[0] for p in self.probs)))

    def close(self):
        for p in self.probs:
            p.synchronize()  # the plane buffer is torch's again only once its copies are done
        for p in self.probs:
            p.close()
        self.probs = []

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_design(self, phi):
        for g, p in zip(self.geom, self.probs):
            p.set_design(slab_cells(phi, self.spec, g))

    def set_state(self, u, w=None):
        for g, p in zip(self.geom, self.probs):
            p.set_state(slab_nodes(u, self.spec, g), None if w is None else slab_nodes(w, self.spec, g))

    def get_state(self, with_w: bool = False, dtype=np.float64):
        parts = [(g, p.get_state(with_w=with_w, dtype=dtype)) for g, p in zip(self.geom, self.probs)]
        if not with_w:
            return self._gather_owned(parts, self.ncomp)
        return (self._gather_owned([(g, uw[0]) for g, uw in parts], self.ncomp),
                self._gather_owned([(g, uw[1]) for g, uw in parts], self.ncomp))

    def exchange(self):
        """Each interface plane from its owner into the neighbour's ghost plane."""
        for src, ks, dst, kd in interface_copies(self.geom):
            self.probs[src].get_plane(ks, self._buf)
            self.probs[dst].set_plane(kd, self._buf)

    def sweep(self, kind: int, n: int, a: float = 0.0, b: float = 0.0, s1: float = 0.0,
              local_dt: bool = False) -> float:
        """n sweeps of every slab, an exchange before each; ||R||^2 of the last over the grid."""
        r2 = 0.0
        for t in range(n):
            self.exchange()
            last = t == n - 1
            vals = [p.sweep(kind, 1, a, b, s1, local_dt, want_res=last) for p in self.probs]
            if last:
                r2 = float(sum(vals))
        return r2

    def residual(self) -> float:
        """||R||^2 of the current state over the whole grid."""
        self.exchange()
        return float(sum(p.residual(with_field=False)[0] for p in self.probs))

    def get_design(self, dtype=np.float64):
        """The whole grid's design, each cell layer from the slab that owns it."""
        return self._gather_design([(g, p.get_design(dtype=dtype)) for g, p in zip(self.geom, self.probs)])

    def exchange_layer(self, field: int, phase: int):
        """Each interface's cell layers of phi's phase (field 0) or mu (field 1), from their
        owners into the neighbours' ghost layer and copy of the layer above."""
        torch = _torch()
        nb = self.probs[0].layer_bytes(field)
        if self._lbuf is None or self._lbuf.numel() < nb:
            self._lbuf = torch.empty(nb, dtype=torch.uint8, device="cuda")
        buf = self._lbuf[:nb]
        for src, ks, dst, kd in interface_layer_copies(self.geom):
            self.probs[src].get_layer(field, phase, ks, buf)
            self.probs[dst].set_layer(field, phase, kd, buf)

    def _threads(self, call):
        """One host thread per slab runs call(slab, hooks); the hooks meet at a barrier: the
        first slab's thread makes every interface copy (all contexts share one stream, so the
        copies fall between the slabs' kernels), and the sums and maxima are taken in slab
        order in every thread, so all slabs take the same decisions."""
        import threading
        n = len(self.probs)
        bar = threading.Barrier(n, timeout=600)
        vals = [None] * n
        out, errs = [None] * n, []

        def hooks(s):
            def copies(fn):
                def run(*args):
                    bar.wait()
                    if s == 0:
                        fn(*args)
                    bar.wait()
                return run

            def reducer(op):
                def run(v):
                    vals[s] = list(v)
                    bar.wait()
                    res = [op(vals[q][i] for q in range(n)) for i in range(len(v))]
                    bar.wait()
                    return res
                return run
            return {"exchange": copies(self.exchange), "exchange_layer": copies(self.exchange_layer),
                    "allreduce": reducer(sum), "allreduce_max": reducer(max)}

        def run(s):
            try:
                out[s] = call(s, hooks(s))
            except BaseException as e:  # noqa: BLE001 -- re-raised below
                errs.append(e)
                bar.abort()

        threads = [threading.Thread(target=run, args=(s,)) for s in range(n)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        if errs:
            raise errs[0]
        return out[0]

    def _slab_solve(self, kw):
        return self._threads(lambda s, h: self.probs[s].slab_solve(h["exchange"], h["allreduce"],
                                                                   allreduce_max=h["allreduce_max"], **kw))

    def _slab_design_step(self, solve_kw, pf_kw):
        return self._threads(lambda s, h: self.probs[s].slab_design_step(
            h["exchange"], h["exchange_layer"], h["allreduce"], h["allreduce_max"], solve_kw=solve_kw, pf_kw=pf_kw))


class DistributedSlabs(_SlabDriver):
    """One slab per rank of a torch.distributed group (rank r holds slab r).  Planes move
    between neighbouring ranks as point-to-point messages; residuals are all-reduced.
    ``make_problem(local_spec)`` builds the rank's context (default: a Problem on the
    current GPU, so each rank selects its GPU with torch.cuda.set_device first); plane
    buffers live where the backend moves data (CUDA for NCCL).  Every rank constructs its
    driver and calls the same methods in the same order (they contain collectives)."""

    def __init__(self, spec, *, group=None, make_problem=None, kernel: str | None = None, device=None):
        torch = _torch()
        import torch.distributed as dist
        self.dist, self.group = dist, group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.spec = spec
        self.geom = slab_geometry(spec.nz, self.world)
        self.g = self.geom[self.rank]
        local = slab_spec(spec, self.g)
        if make_problem is None:
            from .problem import Problem
            make_problem = Problem
        self.prob = make_problem(local)
        if kernel:
            self.prob.select_kernel(kernel)
        self.prob.set_owned_planes(self.g.zlo, self.g.zhi, self.g.g0)
        self.ncomp = self.prob.nrhs * self.prob.ncomp
        if device is None:
            device = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
        self.device = torch.device(device)
        dt = torch.float64 if self.prob.np_dtype == np.float64 else torch.float32
        shape = self.prob.plane_shape()
        self._send = [torch.empty(shape, dtype=dt, device=self.device) for _ in range(2)]
        self._recv = [torch.empty(shape, dtype=dt, device=self.device) for _ in range(2)]
        self.f_norm = float(np.sqrt(self._allreduce(self.prob.residual(with_field=False)[0])))

    def _global_rank(self, r):
        return r if self.group is None else self.dist.get_global_rank(self.group, r)

    def _allreduce(self, x: float) -> float:
        t = _torch().tensor([x], dtype=_torch().float64, device=self.device)
        self.dist.all_reduce(t, group=self.group)
        return float(t.item())

    def exchange(self):
        """Send the owned boundary planes to the neighbours, receive their planes into the
        ghost planes."""
        dist, r, g = self.dist, self.rank, self.g
        ops = []
        if r + 1 < self.world:  # upper neighbour
            self.prob.get_plane(g.zhi, self._send[1])
            ops.append(dist.P2POp(dist.isend, self._send[1], self._global_rank(r + 1), self.group))
            ops.append(dist.P2POp(dist.irecv, self._recv[1], self._global_rank(r + 1), self.group))
        if r > 0:               # lower neighbour
            self.prob.get_plane(g.zlo, self._send[0])
            ops.append(dist.P2POp(dist.isend, self._send[0], self._global_rank(r - 1), self.group))
            ops.append(dist.P2POp(dist.irecv, self._recv[0], self._global_rank(r - 1), self.group))
        if not ops:
            return
        cuda = self.device.type == "cuda"
        if cuda:
            self.prob.synchronize()  # the planes are packed on the context's stream
        for req in dist.batch_isend_irecv(ops):
            req.wait()
        if cuda:
            _torch().cuda.current_stream().synchronize()  # received before the context reads them
        if r + 1 < self.world:
            self.prob.set_plane(g.nz, self._recv[1])
        if r > 0:
            self.prob.set_plane(0, self._recv[0])

    def sweep(self, kind: int, n: int, a: float = 0.0, b: float = 0.0, s1: float = 0.0,
              local_dt: bool = False) -> float:
        r2 = 0.0
        for t in range(n):
            self.exchange()
            last = t == n - 1
            v = self.prob.sweep(kind, 1, a, b, s1, local_dt, want_res=last)
            if last:
                r2 = self._allreduce(v)
        return r2

    def _allreduce_list(self, values):
        t = _torch().tensor(list(values), dtype=_torch().float64, device=self.device)
        self.dist.all_reduce(t, group=self.group)
        return t.tolist()

    def _slab_solve(self, kw):
        return self.prob.slab_solve(self.exchange, self._allreduce_list, allreduce_max=self._allreduce_max_list, **kw)

    def _allreduce_max_list(self, values):
        t = _torch().tensor(list(values), dtype=_torch().float64, device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX, group=self.group)
        return t.tolist()

    def exchange_layer(self, field: int, phase: int):
        """The design-field layers at this rank's interfaces: its top layer up (into the upper
        neighbour's ghost layer), its first own layer down (into the lower neighbour's copy of
        the layer above)."""
        torch, dist, r, g = _torch(), self.dist, self.rank, self.g
        nb = self.prob.layer_bytes(field)
        bufs = [torch.empty(nb, dtype=torch.uint8, device=self.device) for _ in range(4)]
        ops = []
        if r + 1 < self.world:  # upper neighbour: send the top layer, receive its first own layer
            self.prob.get_layer(field, phase, g.nz - 1, bufs[0])
            ops.append(dist.P2POp(dist.isend, bufs[0], self._global_rank(r + 1), self.group))
            ops.append(dist.P2POp(dist.irecv, bufs[1], self._global_rank(r + 1), self.group))
        if r > 0:               # lower neighbour: send the first own layer, receive the ghost layer
            self.prob.get_layer(field, phase, 1, bufs[2])
            ops.append(dist.P2POp(dist.isend, bufs[2], self._global_rank(r - 1), self.group))
            ops.append(dist.P2POp(dist.irecv, bufs[3], self._global_rank(r - 1), self.group))
        if not ops:
            return
        cuda = self.device.type == "cuda"
        if cuda:
            self.prob.synchronize()
        for req in dist.batch_isend_irecv(ops):
            req.wait()
        if cuda:
            torch.cuda.current_stream().synchronize()
        if r + 1 < self.world:
            self.prob.set_layer(field, phase, g.nz, bufs[1])
        if r > 0:
            self.prob.set_layer(field, phase, 0, bufs[3])

    def _slab_design_step(self, solve_kw, pf_kw):
        return self.prob.slab_design_step(self.exchange, self.exchange_layer, self._allreduce_list,
                                          self._allreduce_max_list, solve_kw=solve_kw, pf_kw=pf_kw)

    def get_design(self, dtype=np.float64):
        """The whole grid's design, assembled on every rank."""
        mine = np.asarray(self.prob.get_design(dtype=np.float64))
        parts = [None] * self.world
        self.dist.all_gather_object(parts, (self.rank, mine), group=self.group)
        return self._gather_design([(self.geom[r], phi) for r, phi in parts]).astype(dtype)

    def set_design(self, phi):
        self.prob.set_design(slab_cells(phi, self.spec, self.g))

    def set_state(self, u, w=None):
        self.prob.set_state(slab_nodes(u, self.spec, self.g), None if w is None else slab_nodes(w, self.spec, self.g))

    def get_state(self, dtype=np.float64):
        """The whole grid's state, assembled on every rank."""
        mine = np.asarray(self.prob.get_state(dtype=np.float64))
        parts = [None] * self.world
        self.dist.all_gather_object(parts, (self.rank, mine), group=self.group)
        return self._gather_owned([(self.geom[r], u) for r, u in parts], self.ncomp).astype(dtype)
