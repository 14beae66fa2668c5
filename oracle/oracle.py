"""FP64 CPU oracle of the PeTTO hot path -- Python shim over ``petto_oracle.c``.

TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and the CPU-baseline leg
of the benchmark may import this module.  It shares no code with the GPU path and
imports nothing from the product package; callers hand it plain numbers and numpy
arrays.

Every function names the passage of the paper (PeTTO, arXiv 2509.06971) it follows;
the arithmetic itself lives in ``petto_oracle.c`` and is a literal restatement of
the definitions (cell loop over corners, scatter of element forces).

Conventions (oracle only): node (i, j, k) -> n = i + (nx+1)(j + (ny+1)k), DOFs
interleaved as n*ncomp + a; cell (i, j, k) -> i + nx(j + ny k); design fields [P, cells].
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "petto_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

ELASTIC, THERMAL = 0, 1
SIMP_MODIFIED, SIMP_PAPER = 0, 1
PROJECTED, PENALTY = 0, 1


_SO_OMP = os.path.join(_BUILD, "liboracle_omp.so")


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (plain C99, -O2, no fast-math), and the
    same source with OpenMP for the all-core CPU baseline (skipped when the compiler has no
    OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    flags = ["-O2", "-std=gnu99", "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off"]
    for so, extra in ((_SO, []), (_SO_OMP, ["-fopenmp"])):
        if force or not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(_SRC):
            tmp = so + f".{os.getpid()}.tmp"
            try:
                subprocess.check_call(["gcc", *flags, *extra, _SRC, "-o", tmp, "-lm"])
            except (subprocess.CalledProcessError, OSError):
                if so == _SO:
                    raise
                continue
            os.replace(tmp, so)
    return _SO


def openmp_available() -> bool:
    build()
    return os.path.exists(_SO_OMP)


class _Grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("h", ctypes.c_double), ("physics", ctypes.c_int), ("nu", ctypes.c_double)]


_P = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int
_L = ctypes.c_int64


_lib_omp = None


def _load(openmp: bool = False):
    """The oracle library; openmp=True: its OpenMP build (all-core CPU baseline only)."""
    global _lib, _lib_omp
    with _lock:
        if (_lib_omp if openmp else _lib) is None:
            path = build()
            if openmp:
                if not os.path.exists(_SO_OMP):
                    raise RuntimeError("the oracle's OpenMP build is not available")
                path = _SO_OMP
            lib = ctypes.CDLL(path)
            g = ctypes.POINTER(_Grid)
            sig = {
                "or_ncomp": (_I, [g]), "or_nnodes": (_L, [g]), "or_ncells": (_L, [g]), "or_ndof": (_L, [g]),
                "or_apply_K": (None, [g, _P, _P, _P]),
                "or_cell_energy": (None, [g, _P, _P]),
                "or_assemble_K": (_L, [g, _P, _P, _P, _P]),
                "or_body_load": (None, [g, _D, _P]),
                "or_residual": (_D, [g, _P, _P, _P, _P, _P]),
                "or_diag_K": (None, [g, _P, _P]),
                "or_pt_sweep": (_D, [g, _P, _P, _P, _D, _P, _P, _P]),
                "or_apt_sweep": (_D, [g, _P, _P, _P, _D, _D, _P, _P, _P, _P, _P]),
                "or_solve": (None, [g, _P, _P, _P, _I, _L, _L, _D, _D, _D, _D, _L, _I, _I, _I, _P, _P, _P]),
                "or_material": (None, [_L, _I, _P, _P, _D, _D, _I, _P]),
                "or_sensitivity": (_D, [_L, _I, _P, _P, _D, _D, _I, _P, _P, _P]),
                "or_update": (None, [_L, _I, _P, _P, _P, _I, _D, _D, _D, _I, _P]),
                "or_update_b": (None, [_L, _I, _P, _P, _P, _I, _D, _D, _D, _I, _P, _P, _D, _P]),
                "or_double_well": (_D, [_D]), "or_double_well_deriv": (_D, [_D]),
                "or_cell_laplacian": (None, [g, _P, _P]),
                "or_ch_step": (None, [g, _I, _D, _D, _P]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            if openmp:
                _lib_omp = lib
            else:
                _lib = lib
    return _lib_omp if openmp else _lib


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"], "oracle arrays must be C-contiguous"
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


@dataclass
class OracleProblem:
    """A PDE instance for the oracle: grid, physics, loads and Dirichlet boxes.

    loads:  list of ((i, j, k), comp, value) nodal forces (external force, Sec. 3.2).
    body_source: uniform source f (Sec. 2.2 Poisson equation; f = 0.01 in Sec. 3.1).
    boxes:  list of ((lo_i, lo_j, lo_k), (hi_i, hi_j, hi_k), comp_mask): nodes in the
            inclusive box have u_a = 0 for every component a whose bit is set.
    """
    dim: int
    nx: int
    ny: int
    nz: int = 0
    h: float = 1.0
    physics: int = ELASTIC
    nu: float = 0.3
    loads: list = field(default_factory=list)
    body_source: float = 0.0
    boxes: list = field(default_factory=list)
    openmp: bool = False  # run on the OpenMP build (the all-core CPU baseline only)

    def __post_init__(self):
        if self.dim == 2:
            self.nz = 0
        self._g = _Grid(self.dim, self.nx, self.ny, self.nz, float(self.h), self.physics, float(self.nu))

    # sizes ---------------------------------------------------------------
    @property
    def ncomp(self) -> int:
        return self.dim if self.physics == ELASTIC else 1

    @property
    def node_shape(self):
        return (self.nx + 1, self.ny + 1, self.nz + 1 if self.dim == 3 else 1)

    @property
    def nnodes(self) -> int:
        a, b, c = self.node_shape
        return a * b * c

    @property
    def ncells(self) -> int:
        return self.nx * self.ny * (self.nz if self.dim == 3 else 1)

    @property
    def ndof(self) -> int:
        return self.nnodes * self.ncomp

    def node_id(self, i, j, k=0) -> int:
        return i + (self.nx + 1) * (j + (self.ny + 1) * k)

    # problem data ----------------------------------------------------------
    def fixed_mask(self) -> np.ndarray:
        """uint8 per DOF: 1 where a Dirichlet box fixes that component."""
        nx1, ny1, nz1 = self.node_shape
        m = np.zeros((nz1, ny1, nx1, self.ncomp), dtype=np.uint8)
        for lo, hi, mask in self.boxes:
            lo = list(lo) + [0] * (3 - len(lo))
            hi = list(hi) + [0] * (3 - len(hi))
            for a in range(self.ncomp):
                if (mask >> a) & 1:
                    m[lo[2]:hi[2] + 1, lo[1]:hi[1] + 1, lo[0]:hi[0] + 1, a] = 1
        return np.ascontiguousarray(m.reshape(-1))

    def load_vector(self) -> np.ndarray:
        F = np.zeros(self.ndof)
        for node, comp, val in self.loads:
            node = list(node) + [0] * (3 - len(node))
            F[self.node_id(*node) * self.ncomp + comp] += val
        if self.body_source != 0.0:
            assert self.ncomp == 1, "a body source is a scalar heat source (Sec. 2.2)"
            _load(self.openmp).or_body_load(ctypes.byref(self._g), float(self.body_source), _ptr(F))
        return F

    # operator ---------------------------------------------------------------
    def apply_K(self, E, u) -> np.ndarray:
        E, u = _f64(E), _f64(u)
        out = np.empty(self.ndof)
        _load(self.openmp).or_apply_K(ctypes.byref(self._g), _ptr(E), _ptr(u), _ptr(out))
        return out

    def cell_energy(self, u) -> np.ndarray:
        u = _f64(u)
        e = np.empty(self.ncells)
        _load(self.openmp).or_cell_energy(ctypes.byref(self._g), _ptr(u), _ptr(e))
        return e

    def assemble_K(self, E):
        """scipy.sparse CSR matrix of K(E), assembled from element matrices."""
        import scipy.sparse as sp
        E = _f64(E)
        nl = (1 << self.dim) * self.ncomp
        nt = self.ncells * nl * nl
        rows = np.empty(nt, dtype=np.int64)
        cols = np.empty(nt, dtype=np.int64)
        vals = np.empty(nt)
        _load(self.openmp).or_assemble_K(ctypes.byref(self._g), _ptr(E), _ptr(rows), _ptr(cols), _ptr(vals))
        return sp.csr_matrix((vals, (rows, cols)), shape=(self.ndof, self.ndof))

    def residual(self, E, F, fixed, u):
        E, F, u = _f64(E), _f64(F), _f64(u)
        R = np.empty(self.ndof)
        r2 = _load(self.openmp).or_residual(ctypes.byref(self._g), _ptr(E), _ptr(F), _ptr(fixed), _ptr(u), _ptr(R))
        return R, r2

    def direct_solve(self, E, F, fixed) -> np.ndarray:
        """u with K_ff u_f = F_f and u = 0 on fixed DOFs (sparse LU via scipy)."""
        import scipy.sparse.linalg as spla
        K = self.assemble_K(E)
        free = np.flatnonzero(fixed == 0)
        u = np.zeros(self.ndof)
        u[free] = spla.spsolve(K[free][:, free].tocsc(), _f64(F)[free])
        return u

    def diag_K(self, E) -> np.ndarray:
        E = _f64(E)
        out = np.empty(self.ndof)
        _load(self.openmp).or_diag_K(ctypes.byref(self._g), _ptr(E), _ptr(out))
        return out

    # sweeps -----------------------------------------------------------------
    def inverse_diag(self, E) -> np.ndarray:
        """1/diag(K(E)) per DOF (0 where the diagonal is 0): the local pseudo-time step scale."""
        return self._dinv(E, True)

    def _dinv(self, E, local_dt):
        if not local_dt:
            return None
        d = self.diag_K(E)
        return np.where(d > 0, 1.0 / np.where(d > 0, d, 1.0), 0.0)

    def pt_sweep(self, E, F, fixed, s1, u, local_dt=False, dinv=None) -> float:
        """In place on u (float64, contiguous).  Returns sum R^2 of the input state.
        dinv: 1/diag(K) from an earlier ``inverse_diag`` call on the same E (saves the
        recomputation of diag(K) on large grids)."""
        E, F = _f64(E), _f64(F)
        R = np.empty(self.ndof)
        dinv = self._dinv(E, local_dt) if dinv is None or not local_dt else _f64(dinv)
        return _load(self.openmp).or_pt_sweep(ctypes.byref(self._g), _ptr(E), _ptr(F), _ptr(fixed), float(s1),
                                   None if dinv is None else _ptr(dinv), _ptr(u), _ptr(R))

    def apt_sweep(self, E, F, fixed, a, b, u, w, local_dt=False, dinv=None) -> float:
        """In place on u and w.  Returns sum R^2 of the input state.  dinv as in pt_sweep."""
        E, F = _f64(E), _f64(F)
        R = np.empty(self.ndof)
        dinv = self._dinv(E, local_dt) if dinv is None or not local_dt else _f64(dinv)
        return _load(self.openmp).or_apt_sweep(ctypes.byref(self._g), _ptr(E), _ptr(F), _ptr(fixed), float(a), float(b),
                                    None if dinv is None else _ptr(dinv), _ptr(u), _ptr(w), _ptr(R), None)

    def solve(self, E, F, fixed, u, *, mode=1, n_apt=0, n_pt=0, a=0.9, b=0.25, s1=0.25, tol=1e-8,
              max_sweeps=100000, check_every=50, local_dt=False, momentum=0) -> dict:
        """Hybrid APT -> PT schedule (Sec. 2.2).  In place on u; returns the report.
        momentum=1 selects the adaptive-restart momentum (see or_solve)."""
        E, F = _f64(E), _f64(F)
        w = np.zeros(self.ndof)
        rep = np.zeros(8)
        _load(self.openmp).or_solve(ctypes.byref(self._g), _ptr(E), _ptr(F), _ptr(fixed), int(mode), int(n_apt), int(n_pt),
                         float(a), float(b), float(s1), float(tol), int(max_sweeps), int(check_every),
                         int(bool(local_dt)), int(momentum), _ptr(u), _ptr(w), _ptr(rep))
        return {"sweeps": int(rep[0]), "apt_sweeps": int(rep[1]), "pt_sweeps": int(rep[2]),
                "res_norm": rep[3], "f_norm": rep[4],
                "rel_res": rep[3] / rep[4] if rep[4] > 0 else float("nan"),
                "converged": bool(rep[5]), "fell_back_to_pt": bool(rep[6]), "w": w}

    def cell_laplacian(self, v) -> np.ndarray:
        v = _f64(v)
        out = np.empty(self.ncells)
        _load(self.openmp).or_cell_laplacian(ctypes.byref(self._g), _ptr(v), _ptr(out))
        return out

    def ch_step(self, phi, gamma_g, tau) -> None:
        """In place on phi [P, cells] (Sec. 2.4, forward Euler)."""
        P = phi.shape[0] if phi.ndim == 2 else 1
        _load(self.openmp).or_ch_step(ctypes.byref(self._g), int(P), float(gamma_g), float(tau), _ptr(phi))


@dataclass
class OracleMaterials:
    """Material interpolation (Sec. 3.1 overall conductivity, Sec. 3.2 overall modulus)."""
    moduli: list
    e_min: float = 1e-9
    penal: float = 3.0
    interp: int = SIMP_MODIFIED

    @property
    def n_phases(self) -> int:
        return 1 if self.interp == SIMP_MODIFIED else len(self.moduli)

    def modulus(self, phi) -> np.ndarray:
        phi = _f64(phi)
        ncell = phi.shape[-1]
        E = np.empty(ncell)
        mod = _f64(self.moduli)
        _load().or_material(ncell, self.n_phases, _ptr(phi), _ptr(mod), float(self.e_min), float(self.penal),
                            int(self.interp), _ptr(E))
        return E

    def sensitivity(self, phi, E, e):
        """(s [P, cells], C) with s = dC/dphi = -(dE/dphi) e (total derivative)."""
        phi, E, e = _f64(phi), _f64(E), _f64(e)
        ncell = E.shape[0]
        s = np.empty((self.n_phases, ncell))
        mod = _f64(self.moduli)
        C = _load().or_sensitivity(ncell, self.n_phases, _ptr(phi), _ptr(mod), float(self.e_min),
                                   float(self.penal), int(self.interp), _ptr(E), _ptr(e), _ptr(s))
        return s, C


def update(phi, s, V, *, vol_mode=PROJECTED, alpha_h=0.1, kappa_v=0.0, kappa_1=0.0, n_bisect=60,
           keepout=None, Vb=None, kappa_b=0.0):
    """Design update (Sec. 2.3 combined objective; Sec. 3.1 normalised step; Sec. 3.4
    keep-out term when ``keepout`` (bool per cell), ``Vb`` (per phase) and ``kappa_b`` are
    given).  In place on phi [P, cells]; returns lambda per phase (projected) or the
    pre-step mean (penalty)."""
    P, ncell = phi.shape
    s = _f64(s).reshape(P, ncell)
    Vv = _f64(V).reshape(P)
    lam = np.empty(P)
    if keepout is None:
        _load().or_update(ncell, P, _ptr(phi), _ptr(s), _ptr(Vv), int(vol_mode), float(alpha_h), float(kappa_v),
                          float(kappa_1), int(n_bisect), _ptr(lam))
    else:
        keep = np.ascontiguousarray(np.asarray(keepout, dtype=np.uint8).reshape(ncell))
        Vbv = _f64(Vb).reshape(P)
        _load().or_update_b(ncell, P, _ptr(phi), _ptr(s), _ptr(Vv), int(vol_mode), float(alpha_h),
                            float(kappa_v), float(kappa_1), int(n_bisect), keep.ctypes.data_as(ctypes.c_void_p),
                            _ptr(Vbv), float(kappa_b), _ptr(lam))
    return lam


def double_well(x: float) -> float:
    return _load().or_double_well(float(x))


def double_well_deriv(x: float) -> float:
    return _load().or_double_well_deriv(float(x))


def design_step(prob: OracleProblem, mat: OracleMaterials, phi, u, F, fixed, V, solve_kw: dict, pf_kw: dict,
                ch_steps: int = 1) -> dict:
    """One PeTTO optimisation loop (Fig. 5): state solve (APT then PT), sensitivity
    update, Cahn-Hilliard step.  phi and u are updated in place; returns the metrics."""
    E = mat.modulus(phi)
    rep = prob.solve(E, F, fixed, u, **solve_kw)
    e = prob.cell_energy(u)
    s, C = mat.sensitivity(phi, E, e)
    lam = update(phi, s, V, vol_mode=pf_kw.get("vol_mode", PROJECTED), alpha_h=pf_kw.get("alpha_h", 0.1),
                 kappa_v=pf_kw.get("kappa_v", 0.0), kappa_1=pf_kw.get("kappa_1", 0.0),
                 n_bisect=pf_kw.get("n_bisect", 60), keepout=pf_kw.get("keepout"), Vb=pf_kw.get("Vb"),
                 kappa_b=pf_kw.get("kappa_b", 0.0))
    for _ in range(ch_steps):
        prob.ch_step(phi, pf_kw.get("gamma_g", 0.0), pf_kw.get("tau", 0.0))
    return {"compliance": C, "work": float(np.dot(F, u)), "lambda": lam, "sweeps": rep["sweeps"],
            "rel_res": rep["rel_res"], "mean_phi": phi.mean(axis=1)}
