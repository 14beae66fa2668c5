"""Slab decomposition of a 3D grid, host side (no GPU): the slab geometry and restriction
logic, and the multi-rank driver over gloo with each rank's slab swept by the oracle."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2509_06971_gb300 import slab as S
from paper_2509_06971_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("nz", [1, 2, 7, 20])
@pytest.mark.parametrize("n", [1, 2, 3, 5])
def test_slab_ranges_partition_the_node_planes(nz, n):
    if n > nz + 1:
        with pytest.raises(ValueError):
            S.slab_ranges(nz, n)
        return
    r = S.slab_ranges(nz, n)
    planes = [k for k0, k1 in r for k in range(k0, k1 + 1)]
    assert planes == list(range(nz + 1))
    sizes = [k1 - k0 + 1 for k0, k1 in r]
    assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 1


@pytest.mark.parametrize("nz,n", [(1, 2), (7, 3), (20, 5), (9, 10)])
def test_interface_copies_fill_every_ghost_plane_from_its_owner(nz, n):
    geom = S.slab_geometry(nz, n)
    filled = {s: set() for s in range(n)}
    for src, ks, dst, kd in S.interface_copies(geom):
        gs, gd = geom[src], geom[dst]
        k = gs.g0 + ks
        assert gd.g0 + kd == k                      # the same plane of the whole grid
        assert gs.k0 <= k <= gs.k1                  # sent by its owner
        assert not gd.k0 <= k <= gd.k1              # into a plane the receiver does not own
        filled[dst].add(kd)
    for s, g in enumerate(geom):
        ghosts = {kl for kl in range(g.nz + 1) if not g.zlo <= kl <= g.zhi}
        assert filled[s] == ghosts                  # every ghost plane, once
        assert g.g0 >= 0 and g.g1 <= nz and g.g1 - g.g0 <= g.k1 - g.k0 + 2


@pytest.mark.parametrize("nz,n", [(3, 2), (7, 3), (20, 5), (17, 9)])
def test_cell_layers_are_owned_once_and_every_copy_comes_from_its_owner(nz, n):
    """The decomposed design step: the owned cell layers partition the grid's; each slab
    holds its own layers, plus the layer below (ghost, filled from its owner) where it has a
    lower neighbour; each slab with an upper neighbour gets that neighbour's first own layer
    as its copy of the layer above (local index nz).  Every slab owns two node planes or more
    (so every slab owns a cell layer), which the design step requires."""
    geom = S.slab_geometry(nz, n)
    assert S.design_step_ok(geom)
    owner = {}
    for s, g in enumerate(geom):
        c0, c1 = S.owned_layers(g, nz)
        assert g.g0 <= c0 <= c1 <= g.g0 + g.nz  # held by the slab
        for c in range(c0, c1):
            assert c not in owner
            owner[c] = s
    assert sorted(owner) == list(range(nz))
    filled = {s: set() for s in range(n)}
    for src, ks, dst, kd in S.interface_layer_copies(geom):
        gs, gd = geom[src], geom[dst]
        c = gs.g0 + ks
        assert owner[c] == src                  # sent by its owner
        assert gd.g0 + kd == c                  # the same layer of the whole grid
        assert owner.get(c) != dst
        filled[dst].add(kd)
    for s, g in enumerate(geom):
        c0, c1 = S.owned_layers(g, nz)
        held_not_owned = {c - g.g0 for c in range(g.g0, g.g0 + g.nz) if not c0 <= c < c1}
        above = {g.nz} if s + 1 < n else set()
        assert filled[s] == held_not_owned | above


def test_design_step_needs_two_planes_per_slab():
    assert not S.design_step_ok(S.slab_geometry(2, 2))   # the top slab would own no cell layer
    assert S.design_step_ok(S.slab_geometry(3, 2))


def test_slab_spec_restricts_loads_boxes_and_design():
    base = W.cantilever3d(12, 6, 9)
    loads = base.loads + [((3, 2, 4), 0, 0.5), ((5, 5, 5), 1, -0.25), ((0, 0, 9), 2, 1.0)]
    boxes = base.boxes + [((12, 0, 2), (12, 6, 6), 0b010)]
    spec = base.with_(loads=loads, boxes=boxes, phi0=W.random_design(base, seed=3))
    geom = S.slab_geometry(spec.nz, 3)
    back = []
    for g in geom:
        ls = S.slab_spec(spec, g)
        assert ls.nz == g.nz and ls.nx == spec.nx and ls.keepout is None
        back += [((i, j, k + g.g0), c, v) for (i, j, k), c, v in ls.loads]
        for (lo, hi, m) in ls.boxes:
            assert 0 <= lo[2] <= hi[2] <= g.nz
        # the design of the cell layers the slab holds
        full = np.asarray(spec.phi0).reshape(1, spec.nz, spec.ny, spec.nx)
        assert np.array_equal(np.asarray(ls.phi0).reshape(1, g.nz, spec.ny, spec.nx), full[:, g.g0:g.g1])
    assert sorted(back) == sorted(loads)  # every load on exactly one slab
    # the clamped face x = 0 spans every slab; the roller box only the slabs holding planes 2..6
    assert all(any(lo[0] == 0 and hi[0] == 0 for lo, hi, _ in S.slab_boxes(boxes, g)) for g in geom)


def test_owned_planes_reassemble_the_state():
    spec = W.cantilever3d(6, 4, 10)
    u = W.random_state(spec, seed=4)
    d = S._SlabDriver()
    d.spec = spec
    for n in (1, 2, 4, 11):
        geom = S.slab_geometry(spec.nz, n)
        parts = [(g, S.slab_nodes(u, spec, g)) for g in geom]
        assert np.array_equal(d._gather_owned(parts, 3), u)


WORKER = r"""
import json, os, sys
sys.path.insert(0, {root!r})
import numpy as np
import torch.distributed as dist
from paper_2509_06971_gb300 import slab as S, workloads as W
from tests._slab_fake import OracleSlab
from tests._util import nodes_to_oracle, oracle_materials, oracle_problem, oracle_to_nodes

dist.init_process_group("gloo")
rank, world = dist.get_rank(), dist.get_world_size()
base = W.cantilever3d(10, 6, 9)
loads = base.loads + [((4, 3, 4), 0, 0.7), ((6, 2, 5), 1, -0.4), ((2, 5, 3), 2, 0.25)]
boxes = base.boxes + [((10, 0, 3), (10, 6, 7), 0b010)]
spec = base.with_(loads=loads, boxes=boxes, phi0=W.random_design(base, seed=11))
u0 = W.random_state(spec, seed=12)
w0 = W.random_state(spec, seed=13, scale=0.1)
d = S.DistributedSlabs(spec, make_problem=OracleSlab)
d.set_state(u0, w0)
r2a = d.sweep(0, 3, 0.9, 0.8, 0.0, True)
r2p = d.sweep(1, 2, 0.0, 0.0, 0.15, True)
u = d.get_state()
out = {{"rank": rank, "f_norm": d.f_norm, "r2a": r2a, "r2p": r2p}}
if rank == 0:
    op, om = oracle_problem(spec), oracle_materials(spec)
    E, F, fixed = om.modulus(spec.phi0), op.load_vector(), op.fixed_mask()
    uo, wo = nodes_to_oracle(u0), nodes_to_oracle(w0)
    for _ in range(3):
        r2a_o = op.apt_sweep(E, F, fixed, 0.9, 0.8, uo, wo, local_dt=True)
    for _ in range(2):
        r2p_o = op.pt_sweep(E, F, fixed, 0.15, uo, local_dt=True)
    un = oracle_to_nodes(uo, 3)
    out.update(err=float(np.abs(u - un).max() / np.abs(un).max()), r2a_o=r2a_o, r2p_o=r2p_o,
               f_o=float(np.sqrt((F[~fixed.astype(bool)] ** 2).sum())))
print(json.dumps(out))
dist.destroy_process_group()
"""


def _free_port():
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


@pytest.mark.parametrize("world", [2, 3])
def test_distributed_slabs_follow_the_whole_grid(world):
    """world gloo ranks, one slab each, the oracle's sweep on every slab: three APT and two
    PT sweeps with a plane exchange before each leave the state of the same sweeps on the
    whole grid, and the all-reduced residual sums are the whole grid's."""
    port = _free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE=str(world), LOCAL_RANK=str(r), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER.format(root=ROOT)], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=300) for p in procs]
    res = []
    for p, (o, e) in zip(procs, outs):
        assert p.returncode == 0, e
        res.append(json.loads(o.strip().splitlines()[-1]))
    r0 = res[0]
    assert r0["err"] < 1e-13
    assert abs(r0["r2a"] - r0["r2a_o"]) <= 1e-12 * r0["r2a_o"]
    assert abs(r0["r2p"] - r0["r2p_o"]) <= 1e-12 * r0["r2p_o"]
    assert abs(r0["f_norm"] - r0["f_o"]) <= 1e-12 * r0["f_o"]
    for r in res[1:]:
        assert r["r2a"] == r0["r2a"] and r["r2p"] == r0["r2p"]


SOLVE_WORKER = r"""
import json, os, sys
sys.path.insert(0, {root!r})
import numpy as np
import torch.distributed as dist
from paper_2509_06971_gb300 import slab as S, workloads as W
from tests._slab_fake import OracleSlab
from tests._util import nodes_to_oracle, oracle_materials, oracle_problem

dist.init_process_group("gloo")
base = W.cantilever3d(8, 4, 6, precision="f64")
spec = base.with_(phi0=W.random_design(base, seed=14, lo=0.4, hi=0.9))
d = S.DistributedSlabs(spec, make_problem=OracleSlab)
rep = d.solve(tol=1e-8, check_every=25, max_sweeps=20000)
u = d.get_state()
out = {{"rank": dist.get_rank(), "rep": {{k: float(v) for k, v in rep.items()}}}}
if dist.get_rank() == 0:
    op, om = oracle_problem(spec), oracle_materials(spec)
    F = op.load_vector()
    ud = op.direct_solve(om.modulus(spec.phi0), F, op.fixed_mask())
    out["C"], out["Cd"] = float(F @ nodes_to_oracle(u)), float(F @ ud)
print(json.dumps(out))
dist.destroy_process_group()
"""


def test_distributed_slab_solve_reaches_the_direct_solution():
    """Two gloo ranks, oracle slabs: the fixed-momentum APT solve with a plane exchange
    before every sweep and all-reduced check residuals converges to 1e-8, and the assembled
    state's compliance equals the oracle's direct solve to 1e-6."""
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE="2", LOCAL_RANK=str(r), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", SOLVE_WORKER.format(root=ROOT)], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=600) for p in procs]
    res = []
    for p, (o, e) in zip(procs, outs):
        assert p.returncode == 0, e
        res.append(json.loads(o.strip().splitlines()[-1]))
    r0 = res[0]
    assert r0["rep"]["converged"] == 1.0 and r0["rep"]["rel_res"] <= 1e-8
    assert res[1]["rep"] == r0["rep"]
    assert abs(r0["C"] - r0["Cd"]) <= 1e-6 * abs(r0["Cd"])


def test_one_slab_is_the_whole_grid():
    spec = W.cantilever3d(8, 4, 5)
    (g,) = S.slab_geometry(spec.nz, 1)
    assert (g.k0, g.k1, g.g0, g.g1, g.zlo, g.zhi, g.nz) == (0, 5, 0, 5, 0, 5, 5)
    assert S.interface_copies([g]) == []
    ls = S.slab_spec(spec, g)
    assert ls.loads == spec.loads and ls.boxes == [tuple(b) for b in spec.boxes] and ls.nz == spec.nz


def test_slab_geometry_rejects_2d():
    spec = W.mbb_halfbeam(12, 4)
    with pytest.raises(ValueError):
        S.slab_spec(spec, S.SlabGeom(0, 0, 0, 1))


DESIGN_WORKER = r"""
import json, os, sys
sys.path.insert(0, {root!r})
import numpy as np
import torch.distributed as dist
from oracle import oracle as O
from paper_2509_06971_gb300 import slab as S, workloads as W
from tests._slab_fake import OracleSlab
from tests._util import oracle_materials, oracle_problem

dist.init_process_group("gloo")
base = W.cantilever3d(8, 4, 6, precision="f64")
spec = base.with_(phi0=W.random_design(base, seed=15, lo=0.2, hi=0.6), vol_mode={vol_mode},
                  kappa_v=0.5 if {vol_mode} == 1 else base.kappa_v)
d = S.DistributedSlabs(spec, make_problem=OracleSlab)
solve_kw = dict(tol=1e-11, check_every=25, max_sweeps=60000, momentum=0)
row = d.design_step(solve_kw=solve_kw)
phi = d.get_design()
out = {{"rank": dist.get_rank(), "row": row}}
if dist.get_rank() == 0:
    op, om = oracle_problem(spec), oracle_materials(spec)
    F, fixed = op.load_vector(), op.fixed_mask()
    ph, u = spec.phi0.copy(), np.zeros(op.ndof)
    m = O.design_step(op, om, ph, u, F, fixed, spec.vol_frac,
                      dict(mode=1, a=spec.apt_a, b=spec.apt_b, s1=spec.pt_s1, tol=1e-12, max_sweeps=400000,
                           check_every=25, local_dt=spec.local_dt, momentum=0),
                      dict(alpha_h=spec.alpha_h, gamma_g=spec.gamma_g, tau=spec.tau, vol_mode=spec.vol_mode,
                           kappa_v=spec.kappa_v, kappa_1=spec.kappa_1, n_bisect=spec.n_bisect))
    out["C"], out["dphi"] = m["compliance"], float(np.abs(phi - ph).max())
print(json.dumps(out))
dist.destroy_process_group()
"""


@pytest.mark.parametrize("vol_mode", [0, 1])
def test_distributed_design_step_matches_the_oracle_loop(vol_mode):
    """Two gloo ranks, oracle slabs: one design loop through DistributedSlabs.design_step --
    plane exchanges, the cell-layer exchanges of the Cahn-Hilliard half steps (point to
    point), sums and maxima all-reduced -- against the oracle's loop on the whole grid:
    compliance within 1e-8, design within 1e-8 (projected and penalty update)."""
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE="2", LOCAL_RANK=str(r), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", DESIGN_WORKER.format(root=ROOT, vol_mode=vol_mode)],
                                      env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=600) for p in procs]
    res = []
    for p, (o, e) in zip(procs, outs):
        assert p.returncode == 0, e
        res.append(json.loads(o.strip().splitlines()[-1]))
    r0 = res[0]
    assert res[1]["row"] == r0["row"]  # every rank reports the whole grid's metrics
    assert abs(r0["row"]["compliance"] - r0["C"]) <= 1e-8 * abs(r0["C"])
    assert r0["dphi"] <= 1e-8
