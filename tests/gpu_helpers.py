"""Shared helpers for the GPU parity tests: build a library mesh and the FP64
oracle from the same seeded workload."""
import numpy as np


def f32(a):
    """Round to FP32 and back: the library stores materials in FP32, so the
    oracle is given the identical values."""
    return np.asarray(a, np.float32).astype(np.float64)


def make_pair(w, precision="fp32", refine=0, use_graphs=True, factor_oracle=True):
    from oracle.pd_oracle import PDOracle
    from paper_2405_12484_gb300.sim import Mesh

    m = Mesh(w.rest, w.tets, w.pinned, w.tet_domain, w.n_domains, w.density)
    m.set_materials(w.gamma_s, w.gamma_v)
    m.prefactor(w.dt, precision=precision, refine_steps=refine, use_graphs=use_graphs)
    o = PDOracle(w.rest, w.tets, w.pinned, f32(w.gamma_s), f32(w.gamma_v), w.density, w.dt, factor=factor_oracle)
    return m, o


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))
