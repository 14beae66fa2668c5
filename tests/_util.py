"""Test helpers: turn a workload spec into oracle inputs (test infrastructure only)."""
import numpy as np

from oracle import oracle as O


def oracle_problem(spec, loads=None):
    return O.OracleProblem(spec.dim, spec.nx, spec.ny, spec.nz, h=spec.h, physics=spec.physics, nu=spec.nu,
                           loads=spec.loads if loads is None else loads, body_source=spec.body_source,
                           boxes=spec.boxes)


def oracle_materials(spec):
    return O.OracleMaterials(list(spec.moduli), spec.e_min, spec.penal, spec.interp)


def nodes_to_oracle(field_cn):
    """[ncomp, nodes] -> oracle interleaved [nodes*ncomp]."""
    return np.ascontiguousarray(np.asarray(field_cn, dtype=np.float64).T.reshape(-1))


def oracle_to_nodes(u, ncomp):
    """oracle interleaved [nodes*ncomp] -> [ncomp, nodes]."""
    return np.ascontiguousarray(np.asarray(u).reshape(-1, ncomp).T)


def node_coords(prob):
    nx1, ny1, nz1 = prob.node_shape
    k, j, i = np.meshgrid(np.arange(nz1), np.arange(ny1), np.arange(nx1), indexing="ij")
    return np.stack([i.reshape(-1), j.reshape(-1), k.reshape(-1)], 1).astype(float) * prob.h
