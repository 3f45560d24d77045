"""Synthetic workload generators: sizes, orientation and conformity."""
import numpy as np
import pytest

from workloads.meshes import adjoint_slab, parity_slab, request_workload, serving_requests, slab, sweater_shell


def _faces(tets):
    f = np.concatenate([tets[:, [1, 2, 3]], tets[:, [0, 2, 3]], tets[:, [0, 1, 3]], tets[:, [0, 1, 2]]])
    f = np.sort(f, axis=1)
    _, counts = np.unique(f, axis=0, return_counts=True)
    return counts


def _signed_vol(rest, tets):
    a = rest[tets[:, 1]] - rest[tets[:, 0]]
    b = rest[tets[:, 2]] - rest[tets[:, 0]]
    c = rest[tets[:, 3]] - rest[tets[:, 0]]
    return np.einsum("ij,ij->i", a, np.cross(b, c)) / 6


def test_parity_slab_sizes():
    w = parity_slab()
    assert (w.n_v, w.n_t, int(w.pinned.sum()), w.n_domains) == (1323, 4800, 63, 8)
    assert np.all(np.bincount(w.tet_domain) == 600)
    assert np.all(_signed_vol(w.rest, w.tets) > 0)
    assert w.gamma_s.min() >= 1e3 and w.gamma_s.max() <= 1e5
    assert np.allclose(w.gamma_v, 10 * w.gamma_s)


@pytest.mark.parametrize("tpc", [5, 6])
def test_slab_is_conforming(tpc):
    nx, ny, nz = 3, 4, 2
    rest, tets, _ = slab(nx, ny, nz, 0.01, tpc)
    c = _faces(tets)
    assert c.max() == 2
    assert int((c == 1).sum()) == 2 * 2 * (nx * ny + ny * nz + nx * nz)
    assert np.all(_signed_vol(rest, tets) > 0)


def test_shell_sizes_and_conformity():
    w = sweater_shell()
    assert (w.n_v, w.n_t, int(w.pinned.sum()), w.n_domains) == (98475, 390000, 975, 200)
    cnt = np.bincount(w.tet_domain)
    assert cnt.min() == 1872 and cnt.max() == 2028
    small = sweater_shell(n_theta=30, n_z=5, n_r=2, dom_theta=3, dom_z=2)
    c = _faces(small.tets)
    assert c.max() == 2
    # open cylinder: boundary = inner + outer walls + bottom + top annuli
    assert int((c == 1).sum()) == 2 * (2 * 30 * 5 + 2 * 30 * 2)
    assert np.all(_signed_vol(small.rest, small.tets) > 0)


def test_adjoint_slab_sizes():
    w = adjoint_slab()
    assert (w.n_v, w.n_t, w.n_domains) == (13005, 50000, 25)
    assert np.all(_signed_vol(w.rest, w.tets) > 0)


def test_serving_stream_is_seeded():
    a = serving_requests()
    b = serving_requests()
    assert a == b and len(a) == 64
    sizes = np.array([r[2] for r in a])
    assert sizes.min() >= 5000 and sizes.max() <= 200000
    w = request_workload(a[0][1], a[0][2], a[0][3])
    assert 0.5 * a[0][2] < w.n_t < 2.0 * a[0][2]
