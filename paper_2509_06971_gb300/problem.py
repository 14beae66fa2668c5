"""Thin Python layer over the C ABI: a ``Problem`` owning one ``petto_ctx``.

All numerics run in libpetto's CUDA kernels; this module only marshals arrays and
structs.  Arrays may be numpy arrays (host) or CUDA torch tensors (device, read and
written on the context's stream).  Layouts are the natural ones of include/petto.h:
design [P, cells] with cell (i,j,k) -> i + nx(j + ny k); state [C, nodes] with node
(i,j,k) -> i + (nx+1)(j + (ny+1)k).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import capi as C

_DT = {np.dtype(np.float32): C.PETTO_F32, np.dtype(np.float64): C.PETTO_F64}
_STORAGE = {"f32": C.PETTO_F32, "f64": C.PETTO_F64, "bf16": C.PETTO_BF16, "f16": C.PETTO_F16}


def _torch():
    import torch
    return torch


def _is_cuda_tensor(x) -> bool:
    try:
        torch = _torch()
    except ImportError:
        return False
    return isinstance(x, torch.Tensor) and x.is_cuda


def _tensor_dtype(t) -> int:
    torch = _torch()
    m = {torch.float32: C.PETTO_F32, torch.float64: C.PETTO_F64, torch.bfloat16: C.PETTO_BF16,
         torch.float16: C.PETTO_F16}
    if t.dtype not in m:
        raise TypeError(f"unsupported tensor dtype {t.dtype}")
    return m[t.dtype]


class Problem:
    """One PeTTO instance on the GPU (grid, materials, loads, supports, design, state)."""

    def __init__(self, spec, *, nrhs: int = 1, load_cases=None, stream=None, precision: str | None = None,
                 storage: str | None = None):
        self.spec = spec
        self.lib = C.load()
        prec = precision or spec.precision
        stor = storage or spec.storage
        self.precision = C.PETTO_F64 if prec == "f64" else C.PETTO_F32
        self.np_dtype = np.float64 if prec == "f64" else np.float32
        self.storage = _STORAGE[stor]
        self.nrhs = nrhs
        self.ncomp = spec.ncomp
        self.P = spec.n_phases
        self.ncells = spec.ncells
        self.nnodes = spec.nnodes
        if stream is None:
            try:
                torch = _torch()
                stream = torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else None
            except ImportError:
                stream = None
        self.stream = stream
        cases = load_cases if load_cases is not None else [spec.loads]
        if len(cases) != nrhs:
            raise ValueError("need one load list per load case")
        nodes, comps, vals, rhs = [], [], [], []
        for r, case in enumerate(cases):
            for node, comp, val in case:
                node = list(node) + [0] * (3 - len(node))
                nodes.extend(node[:3])
                comps.append(comp)
                vals.append(val)
                rhs.append(r)
        self._keep = []
        n = len(vals)
        node_a = (ctypes.c_int64 * max(1, len(nodes)))(*nodes)
        comp_a = (ctypes.c_int32 * max(1, n))(*comps)
        val_a = (ctypes.c_double * max(1, n))(*vals)
        rhs_a = (ctypes.c_int32 * max(1, n))(*rhs)
        loads = C.petto_loads(n, node_a, comp_a, val_a, rhs_a, float(spec.body_source))
        boxes = []
        masks = []
        for lo, hi, mask in spec.boxes:
            lo = list(lo) + [0] * (3 - len(lo))
            hi = list(hi) + [0] * (3 - len(hi))
            boxes.extend(lo[:3] + hi[:3])
            masks.append(mask)
        box_a = (ctypes.c_int64 * max(1, len(boxes)))(*boxes)
        mask_a = (ctypes.c_uint32 * max(1, len(masks)))(*masks)
        bcs = C.petto_bcs(len(masks), box_a, mask_a)
        mod = (ctypes.c_double * len(spec.moduli))(*spec.moduli)
        mat = C.petto_materials(spec.physics, self.P, mod, spec.e_min, spec.nu, spec.penal, spec.interp)
        grid = C.petto_grid(spec.dim, spec.nx, spec.ny, spec.nz if spec.dim == 3 else 0, spec.h)
        vol = (ctypes.c_double * self.P)(*spec.vol_frac)
        opt = C.petto_options(self.precision, self.storage, nrhs, ctypes.c_void_p(stream) if stream else None)
        ctx = ctypes.c_void_p()
        st = self.lib.petto_create(ctypes.byref(grid), ctypes.byref(mat), ctypes.byref(loads), ctypes.byref(bcs),
                                   vol, ctypes.byref(opt), ctypes.byref(ctx))
        if st != C.PETTO_OK:
            raise C.PettoError(st, "petto_create failed")
        self.ctx = ctx
        if spec.phi0 is not None:
            self.set_design(np.asarray(spec.phi0, dtype=np.float64))
        if spec.keepout is not None:
            self.set_keepout(spec.keepout, spec.keepout_target, spec.kappa_b)

    # --------------------------------------------------------------- lifecycle
    def close(self):
        if getattr(self, "ctx", None):
            self.lib.petto_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _ck(self, st, allow=(C.PETTO_OK,)):
        return C.check(self.ctx, st, allow)

    @property
    def launches(self) -> int:
        return int(self.lib.petto_launch_count(self.ctx))

    def profile(self, enable: bool = True):
        self._ck(self.lib.petto_profile(self.ctx, int(bool(enable))))

    def profile_read(self, with_rhs: bool = False):
        """(summed sweep device milliseconds, sweeps timed[, sweeps with a dense RHS]) since
        the last read."""
        ms, n, nr = ctypes.c_double(0.0), ctypes.c_int64(0), ctypes.c_int64(0)
        self._ck(self.lib.petto_profile_read(self.ctx, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(nr)))
        return (ms.value, n.value, nr.value) if with_rhs else (ms.value, n.value)

    def autotune(self, sweeps: int = 20) -> dict:
        """Time the applicable sweep kernels / tile shapes and keep the fastest."""
        import json
        buf = ctypes.create_string_buffer(4096)
        self._ck(self.lib.petto_autotune(self.ctx, int(sweeps), buf, len(buf)))
        return json.loads(buf.value.decode() or "{}")

    def set_keepout(self, box, target, kappa_b: float):
        """Keep-out region of the update (petto_set_keepout): box ((lo), (hi)) inclusive cell
        ranges, target per phase; box None removes it."""
        if box is None:
            self._ck(self.lib.petto_set_keepout(self.ctx, None, None, 0.0))
            return
        lo, hi = (list(box[0]) + [0, 0])[:3], (list(box[1]) + [0, 0])[:3]
        b = (ctypes.c_int64 * 6)(*(lo + hi))
        t = (ctypes.c_double * self.P)(*[float(x) for x in target])
        self._ck(self.lib.petto_set_keepout(self.ctx, b, t, float(kappa_b)))

    def select_kernel(self, name: str):
        """Pick the sweep kernel by autotuner name ("march2d", "gather/32x8", "tma2/zs16", ...)."""
        self._ck(self.lib.petto_select_kernel(self.ctx, name.encode()))

    def kernel_info(self):
        """(name of the sweep kernel in use, bytes per node and component of the right-hand
        side its refinement sweeps read)."""
        buf = ctypes.create_string_buffer(64)
        rb = ctypes.c_int(0)
        self._ck(self.lib.petto_kernel_info(self.ctx, buf, 64, ctypes.byref(rb)))
        return buf.value.decode(), rb.value

    def synchronize(self):
        self._ck(self.lib.petto_synchronize(self.ctx))

    # --------------------------------------------------------------- fields
    def _in(self, x, allowed=(C.PETTO_F32, C.PETTO_F64)):
        if _is_cuda_tensor(x):
            x = x.contiguous()
            dt = _tensor_dtype(x)
            if dt not in allowed:
                raise TypeError("dtype not accepted here")
            return x, ctypes.c_void_p(x.data_ptr()), dt, 1
        a = np.ascontiguousarray(x)
        if a.dtype not in _DT:
            a = a.astype(np.float64)
        return a, a.ctypes.data_as(ctypes.c_void_p), _DT[a.dtype], 0

    def set_design(self, phi):
        keep, ptr, dt, dev = self._in(phi, (C.PETTO_F32, C.PETTO_F64, C.PETTO_BF16, C.PETTO_F16))
        self._ck(self.lib.petto_set_design(self.ctx, ptr, dt, dev))

    def get_design(self, dtype=np.float64) -> np.ndarray:
        out = np.empty((self.P, self.ncells), dtype=dtype)
        self._ck(self.lib.petto_get_design(self.ctx, out.ctypes.data_as(ctypes.c_void_p), _DT[out.dtype], 0))
        return out

    def set_state(self, u, w=None):
        ku, pu, dt, dev = self._in(u)
        if w is not None:
            kw, pw, dtw, devw = self._in(w)
            assert dtw == dt and devw == dev
        else:
            pw = None
        self._ck(self.lib.petto_set_state(self.ctx, pu, pw, dt, dev))

    def get_state(self, with_w: bool = False, dtype=np.float64):
        shape = (self.nrhs * self.ncomp, self.nnodes)
        u = np.empty(shape, dtype=dtype)
        w = np.empty(shape, dtype=dtype) if with_w else None
        self._ck(self.lib.petto_get_state(self.ctx, u.ctypes.data_as(ctypes.c_void_p),
                                          w.ctypes.data_as(ctypes.c_void_p) if with_w else None, _DT[u.dtype], 0))
        return (u, w) if with_w else u

    def get_modulus(self, dtype=np.float64) -> np.ndarray:
        E = np.empty(self.ncells, dtype=dtype)
        self._ck(self.lib.petto_get_modulus(self.ctx, E.ctypes.data_as(ctypes.c_void_p), _DT[E.dtype], 0))
        return E

    # --------------------------------------------------------------- slabs
    def set_owned_planes(self, zlo: int, zhi: int, z_global: int = 0):
        """Sweeps write node planes zlo..zhi only (a slab of a decomposed 3D grid whose local
        plane 0 is plane z_global of the whole grid)."""
        self._ck(self.lib.petto_set_owned_planes(self.ctx, int(zlo), int(zhi), int(z_global)))

    def plane_shape(self):
        s = self.spec
        return (self.nrhs * self.ncomp, s.ny + 1, s.nx + 1)

    def get_plane(self, k: int, out=None):
        """Node plane k of the current state as [components][ny+1][nx+1] in the sweep
        precision, into `out` (a CUDA tensor: stream-ordered device copy) or a new array."""
        if out is None:
            out = np.empty(self.plane_shape(), dtype=self.np_dtype)
        if _is_cuda_tensor(out):
            ptr, dev = out.data_ptr(), 1
        else:
            arr = out.numpy() if hasattr(out, "numpy") else out  # host tensors through their array view
            if arr.dtype != self.np_dtype or not arr.flags.c_contiguous:
                raise ValueError("plane buffers are contiguous and in the sweep precision")
            ptr, dev = arr.ctypes.data, 0
        self._ck(self.lib.petto_get_plane(self.ctx, int(k), ctypes.c_void_p(ptr), self.precision, dev))
        return out

    def set_plane(self, k: int, src):
        """Write node plane k of the current state from [components][ny+1][nx+1]."""
        if _is_cuda_tensor(src):
            src = src.contiguous()
            ptr, dev = src.data_ptr(), 1
        else:
            src = np.ascontiguousarray(src.numpy() if hasattr(src, "numpy") else src, dtype=self.np_dtype)
            ptr, dev = src.ctypes.data, 0
        self._ck(self.lib.petto_set_plane(self.ctx, int(k), ctypes.c_void_p(ptr), self.precision, dev))

    # --------------------------------------------------------------- solver
    def sweep(self, kind: int, n: int, a: float = 0.0, b: float = 0.0, s1: float = 0.0, local_dt: bool = False,
              want_res: bool = True):
        r = ctypes.c_double(0.0)
        self._ck(self.lib.petto_sweep(self.ctx, kind, int(n), float(a), float(b), float(s1), int(bool(local_dt)),
                                      ctypes.byref(r) if want_res else None))
        return r.value if want_res else None

    def set_wait_limit(self, tries: int = -1):
        """Attempts of each bounded ring wait of the TMA sweeps (-1: the default)."""
        self._ck(self.lib.petto_set_wait_limit(self.ctx, int(tries)))

    def sweep_rhs(self, kind: int, n: int, r, a: float = 0.0, b: float = 0.0, s1: float = 0.0,
                  local_dt: bool = False, want_res: bool = True):
        """n sweeps with the dense right-hand side r [C, nodes] (FP64, host array or CUDA
        tensor) in place of the loads: the correction sweeps of the FP64 refinement."""
        ptr, on_dev, keep = self._rhs_in(r)
        res = ctypes.c_double(0.0)
        self._ck(self.lib.petto_sweep_rhs(self.ctx, kind, int(n), float(a), float(b), float(s1),
                                          int(bool(local_dt)), ptr, on_dev, ctypes.byref(res) if want_res else None))
        del keep
        return res.value if want_res else None

    def _rhs_in(self, r):
        if _is_cuda_tensor(r):
            t = r.contiguous()
            if t.dtype != _torch().float64:
                raise TypeError("the right-hand side is FP64")
            return ctypes.c_void_p(t.data_ptr()), 1, t
        a = np.ascontiguousarray(np.asarray(r, dtype=np.float64).reshape(self.nrhs * self.ncomp, self.nnodes))
        return a.ctypes.data_as(ctypes.c_void_p), 0, a

    def residual(self, with_field: bool = True, dtype=np.float64):
        r = ctypes.c_double(0.0)
        R = np.empty((self.nrhs * self.ncomp, self.nnodes), dtype=dtype) if with_field else None
        self._ck(self.lib.petto_residual(self.ctx, ctypes.byref(r),
                                         R.ctypes.data_as(ctypes.c_void_p) if with_field else None,
                                         _DT[np.dtype(dtype)], 0))
        return r.value, R

    def residual64(self, u, with_field: bool = True):
        """The FP64 defect F - K(E) u of an FP64 state u [C][nodes] (petto_residual64: the
        refinement's defect kernel; FP32 contexts).  Returns (sum R^2, R or None)."""
        u = np.ascontiguousarray(np.asarray(u, np.float64).reshape(self.nrhs * self.ncomp, self.nnodes))
        r = ctypes.c_double(0.0)
        R = np.empty_like(u) if with_field else None
        self._ck(self.lib.petto_residual64(self.ctx, u.ctypes.data_as(ctypes.c_void_p), 0, ctypes.byref(r),
                                           R.ctypes.data_as(ctypes.c_void_p) if with_field else None))
        return r.value, R

    def solve_opts(self, mode=None, **kw) -> C.petto_solve_opts:
        """Defaults: the workload's constants and schedule (tolerance mode unless the
        workload is the paper's fixed-count loop); momentum from the workload (adaptive
        restart with the momentum cap a = 1 unless given), refine = 1 (FP64 refinement
        for FP32 states)."""
        s = self.spec
        mode = int(kw.pop("mode", s.solve_mode if mode is None else mode))
        momentum = int(kw.get("momentum", s.momentum))
        a = float(kw.get("a", 1.0 if momentum else s.apt_a))
        return C.petto_solve_opts(mode, int(kw.get("n_apt", s.n_apt)), int(kw.get("n_pt", s.n_pt)), a,
                                  float(kw.get("b", s.apt_b)), float(kw.get("s1", s.pt_s1)),
                                  float(kw.get("tol", s.tol)), int(kw.get("max_sweeps", s.max_sweeps)),
                                  int(kw.get("check_every", s.check_every)),
                                  int(bool(kw.get("local_dt", s.local_dt))), momentum,
                                  int(bool(kw.get("refine", True))))

    def slab_solve(self, exchange, allreduce, allreduce_max=None, mode=None, **kw) -> dict:
        """The state solve of one slab of a decomposed grid (petto_slab_solve): exchange()
        fills the ghost planes before every sweep, allreduce / allreduce_max (list of floats)
        return their sums / maxima over the slabs.  Options as solve(); the FP64 refinement of
        an FP32 solve (refine, the default) needs allreduce_max."""
        o = self.solve_opts(mode, **kw)
        errors = []

        def _ex(ctx, user):
            try:
                exchange()
                return C.PETTO_OK
            except BaseException as e:  # noqa: BLE001 -- handed back to the caller below
                errors.append(e)
                return C.PETTO_EINVAL

        def reducer(fn):
            def call(values, n, user):
                try:
                    out = fn([values[i] for i in range(n)])
                    for i in range(n):
                        values[i] = float(out[i])
                    return C.PETTO_OK
                except BaseException as e:  # noqa: BLE001
                    errors.append(e)
                    return C.PETTO_EINVAL
            return C.petto_allreduce_fn(call)

        ex, ar = C.petto_exchange_fn(_ex), reducer(allreduce)
        am = reducer(allreduce_max) if allreduce_max is not None else C.petto_allreduce_fn()
        rep = C.petto_solve_report()
        st = self.lib.petto_slab_solve(self.ctx, ctypes.byref(o), ex, ar, am, None, ctypes.byref(rep))
        if errors:
            raise errors[0]
        self._ck(st, allow=(C.PETTO_OK, C.PETTO_ENOTCONV))
        return _report(rep, st)

    def slab_design_step(self, exchange, exchange_layer, allreduce, allreduce_max, solve_kw=None, pf_kw=None) -> dict:
        """One design loop of one slab of a decomposed grid (petto_slab_design_step):
        exchange() fills the ghost planes, exchange_layer(field, phase) the cell layers next to
        each interface, allreduce / allreduce_max (list of floats) return the sums / maxima
        over the slabs.  Returns the whole grid's metrics of the step."""
        so = self.solve_opts(**(solve_kw or {}))
        po = self.pf_opts(**(pf_kw or {}))
        errors = []

        def guard(fn):
            def call(*args):
                try:
                    fn(*args)
                    return C.PETTO_OK
                except BaseException as e:  # noqa: BLE001 -- handed back to the caller below
                    errors.append(e)
                    return C.PETTO_EINVAL
            return call

        def reducer(fn):
            def call(values, n, user):
                out = fn([values[i] for i in range(n)])
                for i in range(n):
                    values[i] = float(out[i])
            return guard(call)

        ex = C.petto_exchange_fn(guard(lambda ctx, user: exchange()))
        exl = C.petto_layer_exchange_fn(guard(lambda ctx, field, phase, user: exchange_layer(field, phase)))
        ar, am = C.petto_allreduce_fn(reducer(allreduce)), C.petto_allreduce_fn(reducer(allreduce_max))
        m = (ctypes.c_double * 8)()
        st = self.lib.petto_slab_design_step(self.ctx, ctypes.byref(so), ctypes.byref(po), ex, exl, ar, am, None, m)
        if errors:
            raise errors[0]
        self._ck(st, allow=(C.PETTO_OK, C.PETTO_ENOTCONV))
        return {"step": int(m[0]), "compliance": m[1], "work": m[2], "rel_res": m[3], "sweeps": int(m[4]),
                "seconds": m[5], "mean_phi0": m[6], "lambda0": m[7], "converged": st == C.PETTO_OK}

    def layer_bytes(self, field: int) -> int:
        return int(self.lib.petto_layer_bytes(self.ctx, int(field)))

    def _layer_buf(self, field, buf):
        """(pointer, on_device) of a layer buffer of petto_layer_bytes bytes: a contiguous CUDA
        tensor (stream-ordered copy) or a host array / tensor."""
        nb = self.layer_bytes(field)  # 0 for a field the library rejects (it reports the error)
        if _is_cuda_tensor(buf):
            if not buf.is_contiguous() or (nb and buf.numel() * buf.element_size() != nb):
                raise ValueError("layer buffers are contiguous, petto_layer_bytes long")
            return buf.data_ptr(), 1
        arr = buf.numpy() if hasattr(buf, "numpy") else buf
        if not arr.flags.c_contiguous or (nb and arr.nbytes != nb):
            raise ValueError("layer buffers are contiguous, petto_layer_bytes long")
        return arr.ctypes.data, 0

    def get_layer(self, field: int, phase: int, k: int, out):
        """Cell layer k (k = nz: the copy of the layer above) of phi's phase (field 0, storage
        type) or mu (field 1, sweep precision) into out, raw bytes."""
        ptr, dev = self._layer_buf(field, out)
        self._ck(self.lib.petto_get_layer(self.ctx, int(field), int(phase), int(k), ctypes.c_void_p(ptr), dev))
        return out

    def set_layer(self, field: int, phase: int, k: int, src):
        ptr, dev = self._layer_buf(field, src)
        self._ck(self.lib.petto_set_layer(self.ctx, int(field), int(phase), int(k), ctypes.c_void_p(ptr), dev))

    def solve(self, mode=None, **kw) -> dict:
        o = self.solve_opts(mode, **kw)
        rep = C.petto_solve_report()
        st = self._ck(self.lib.petto_pt_solve(self.ctx, ctypes.byref(o), ctypes.byref(rep)),
                      allow=(C.PETTO_OK, C.PETTO_ENOTCONV))
        return _report(rep, st)

    # --------------------------------------------------------------- design
    def sensitivity(self, out=None, want_field: bool = True):
        """(compliance, work, dC/dphi) -- out may be a CUDA tensor [P, cells] (f32/f64)."""
        Cv, Wv = ctypes.c_double(0.0), ctypes.c_double(0.0)
        if out is not None and _is_cuda_tensor(out):
            self._ck(self.lib.petto_sensitivity(self.ctx, ctypes.byref(Cv), ctypes.byref(Wv),
                                                ctypes.c_void_p(out.data_ptr()), _tensor_dtype(out), 1))
            return Cv.value, Wv.value, out
        s = np.empty((self.P, self.ncells), dtype=np.float64) if want_field else None
        self._ck(self.lib.petto_sensitivity(self.ctx, ctypes.byref(Cv), ctypes.byref(Wv),
                                            s.ctypes.data_as(ctypes.c_void_p) if want_field else None,
                                            C.PETTO_F64, 0))
        return Cv.value, Wv.value, s

    def pf_opts(self, **kw) -> C.petto_pf_opts:
        s = self.spec
        return C.petto_pf_opts(int(kw.get("vol_mode", s.vol_mode)), float(kw.get("alpha_h", s.alpha_h)),
                               float(kw.get("kappa_v", s.kappa_v)), float(kw.get("kappa_1", s.kappa_1)),
                               float(kw.get("gamma_g", s.gamma_g)), float(kw.get("tau", s.tau)),
                               int(kw.get("ch_steps", 1)), int(kw.get("n_bisect", s.n_bisect)))

    def design_update(self, **kw) -> np.ndarray:
        o = self.pf_opts(**kw)
        lam = (ctypes.c_double * self.P)()
        self._ck(self.lib.petto_design_update(self.ctx, ctypes.byref(o), lam))
        return np.array(lam[:])

    def cahn_hilliard(self, **kw):
        o = self.pf_opts(**kw)
        self._ck(self.lib.petto_cahn_hilliard(self.ctx, ctypes.byref(o)))

    def phase_field_step(self, **kw) -> np.ndarray:
        o = self.pf_opts(**kw)
        vol = (ctypes.c_double * self.P)()
        self._ck(self.lib.petto_phase_field_step(self.ctx, ctypes.byref(o), vol))
        return np.array(vol[:])

    def optimize(self, n_steps: int, solve_kw: dict | None = None, pf_kw: dict | None = None, log=None):
        so = self.solve_opts(**(solve_kw or {}))
        po = self.pf_opts(**(pf_kw or {}))
        hist = []

        def _cb(m, user):
            row = {"step": int(m[0]), "compliance": m[1], "work": m[2], "rel_res": m[3], "sweeps": int(m[4]),
                   "seconds": m[5], "mean_phi0": m[6], "lambda0": m[7]}
            hist.append(row)
            if log:
                log(row)

        cb = C.petto_step_cb(_cb)
        st = self._ck(self.lib.petto_optimize(self.ctx, int(n_steps), ctypes.byref(so), ctypes.byref(po), cb, None),
                      allow=(C.PETTO_OK, C.PETTO_ENOTCONV))
        return hist, st

    def save(self, path: str):
        self._ck(self.lib.petto_save(self.ctx, path.encode()))

    def load(self, path: str):
        self._ck(self.lib.petto_load(self.ctx, path.encode()))


def _report(rep, st) -> dict:
    return {"sweeps": rep.sweeps, "apt_sweeps": rep.apt_sweeps, "pt_sweeps": rep.pt_sweeps,
            "res_norm": rep.res_norm, "f_norm": rep.f_norm, "rel_res": rep.rel_res, "r_pde": rep.r_pde,
            "converged": bool(rep.converged), "fell_back_to_pt": bool(rep.fell_back_to_pt), "status": st}


class Batch:
    """Many 2D problems advanced together by the batched sweep (petto_batch_* in
    include/petto.h): one kernel launch per sweep over every problem still iterating.
    The problems stay usable on their own (design, state, sensitivity); the batch borrows
    their contexts, so close the batch before the problems."""

    def __init__(self, problems):
        self.problems = list(problems)
        self.lib = C.load()
        n = len(self.problems)
        arr = (ctypes.c_void_p * n)(*[p.ctx.value for p in self.problems])
        out = ctypes.c_void_p()
        st = self.lib.petto_batch_create(n, arr, ctypes.byref(out))
        if st != C.PETTO_OK:
            raise C.PettoError(st, "petto_batch_create failed")
        self.batch = out

    def close(self):
        if getattr(self, "batch", None):
            self.lib.petto_batch_destroy(self.batch)
            self.batch = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _ck(self, st, allow=(C.PETTO_OK,)):
        return C.check_batch(self.batch, st, allow)

    def __len__(self):
        return len(self.problems)

    @property
    def launches(self) -> int:
        return int(self.lib.petto_batch_launch_count(self.batch))

    def solve_opts(self, mode=None, **kw):
        n = len(self.problems)
        arr = (C.petto_solve_opts * n)()
        for i, p in enumerate(self.problems):
            arr[i] = p.solve_opts(mode, **kw)
        return arr

    def solve(self, mode=None, **kw) -> list:
        """Solve every problem; one report dict per problem (as Problem.solve)."""
        n = len(self.problems)
        opts = self.solve_opts(mode, **kw)
        reps = (C.petto_solve_report * n)()
        st = self._ck(self.lib.petto_batch_pt_solve(self.batch, opts, reps), allow=(C.PETTO_OK, C.PETTO_ENOTCONV))
        return [_report(reps[i], st) for i in range(n)]

    def optimize(self, n_steps: int, solve_kw: dict | None = None, pf_kw: dict | None = None):
        """n_steps PeTTO loops on every problem.  Returns (metrics [n_steps, n, 8] as in
        Problem.optimize's rows, status)."""
        n = len(self.problems)
        so = self.solve_opts(**(solve_kw or {}))
        po = (C.petto_pf_opts * n)()
        for i, p in enumerate(self.problems):
            po[i] = p.pf_opts(**(pf_kw or {}))
        m = np.zeros((max(1, n_steps), n, 8), dtype=np.float64)
        st = self._ck(self.lib.petto_batch_optimize(self.batch, int(n_steps), so, po,
                                                    m.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
                      allow=(C.PETTO_OK, C.PETTO_ENOTCONV))
        return m[:n_steps], st

    def profile(self, enable: bool = True):
        self._ck(self.lib.petto_batch_profile(self.batch, int(bool(enable))))

    def profile_read(self):
        """(milliseconds, batch sweeps) of the timed sweep chunks since the last read."""
        ms = ctypes.c_double(0.0)
        n = ctypes.c_int64(0)
        self._ck(self.lib.petto_batch_profile_read(self.batch, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value


class PettoCompliance:
    """torch.autograd.Function factory: C(phi) = F.u(phi) with u solved on the GPU, and
    dC/dphi from the hand-written adjoint kernel (the compliance is self-adjoint, so the
    adjoint state is u itself; Sec. 2.3 computes this derivative by AD instead)."""

    @staticmethod
    def apply(phi, problem: Problem, **solve_kw):
        torch = _torch()

        class _Fn(torch.autograd.Function):
            @staticmethod
            def forward(ctx, x):
                problem.set_design(x.detach())
                problem.solve(**solve_kw)
                grad = torch.empty_like(x, dtype=torch.float64 if problem.precision == C.PETTO_F64 else torch.float32)
                Cv, _, _ = problem.sensitivity(out=grad)
                ctx.save_for_backward(grad)
                return torch.tensor(Cv, dtype=torch.float64, device=x.device)

            @staticmethod
            def backward(ctx, g):
                (grad,) = ctx.saved_tensors
                return (g * grad).to(phi.dtype), None

        return _Fn.apply(phi)
