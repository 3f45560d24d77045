"""Pins of the harmonic-initialization oracle (oracle/harmonic.py; Sec. 6
"Harmonic Initialization", Eq. q2gamma): the element Laplacian against the
closed-form spectrum of a path graph, eigen-identities on a slab, the chain
rule of the reduced coordinates against finite differences, the full basis
reproducing the un-reduced Gauss-Newton direction, and rank 1 recovering a
constant material."""
import numpy as np
import pytest

from oracle.adjoint import AdjointOracle
from oracle.gauss_newton import GaussNewtonOracle
from oracle.harmonic import (ReducedGN, basis_matrix, dual_laplacian, face_adjacency, fit_reduced,
                             harmonic_basis)
from oracle.pd_oracle import PDOracle
from workloads.meshes import slab_workload


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def test_tet_chain_has_the_path_graph_spectrum():
    # Boerdijk-Coxeter chain: tet j = (j, j+1, j+2, j+3); consecutive tets share
    # a face, tets two apart only an edge -> the face-adjacency graph is a path
    n = 25
    tets = np.array([[j, j + 1, j + 2, j + 3] for j in range(n)])
    assert len(face_adjacency(tets)) == n - 1
    lam, H = harmonic_basis(tets, n)
    k = np.arange(n)
    assert np.allclose(lam, 2.0 - 2.0 * np.cos(np.pi * k / n), atol=1e-12)
    # eigenvectors cos(pi k (j + 1/2) / n), up to sign
    j = np.arange(n)
    for kk in (1, 2, 7):
        ref = np.cos(np.pi * kk * (j + 0.5) / n)
        ref /= np.linalg.norm(ref)
        assert abs(abs(H[:, kk] @ ref) - 1.0) < 1e-10


@pytest.fixture(scope="module")
def slab():
    return slab_workload(4, 4, 2, 0.01, 5, (2, 2), seed=3, n_iter=10, name="harm-pins")


def test_slab_basis_identities(slab):
    w = slab
    L = dual_laplacian(w.tets).toarray()
    assert np.allclose(L.sum(axis=1), 0)
    # every interior tet of the 5-tet cube split has 4 face neighbours at most
    assert L.diagonal().max() <= 4
    lam, H = harmonic_basis(w.tets, 12)
    assert abs(lam[0]) < 1e-12 and lam[1] > 1e-6                  # connected mesh
    assert np.allclose(np.abs(H[:, 0]), 1.0 / np.sqrt(w.n_t))     # h_1 constant
    assert np.allclose(H.T @ H, np.eye(12), atol=1e-12)
    assert np.linalg.norm(L @ H - H * lam) < 1e-10
    rng = np.random.default_rng(2)
    z = rng.standard_normal((w.n_t, 100))
    z -= H @ (H.T @ z)
    rq = np.einsum("ij,ij->j", z, L @ z) / np.einsum("ij,ij->j", z, z)
    assert rq.min() >= lam[-1] * (1 - 1e-9)


def _gn(w, gs, gv):
    return GaussNewtonOracle(AdjointOracle(PDOracle(w.rest, w.tets, w.pinned, gs, gv, w.density, w.dt)))


def test_reduced_gradient_is_the_chain_rule(slab):
    w = slab
    _, H = harmonic_basis(w.tets, 10)
    D = basis_matrix(H)
    gamma = np.concatenate([w.gamma_s, w.gamma_v])
    q = D.T @ gamma
    g0 = D @ q
    x0, v0, pins = w.rest, np.zeros_like(w.rest), w.pin_targets(0)
    rng = np.random.default_rng(3)
    target = _gn(w, g0[:w.n_t] * 1.2, g0[w.n_t:] * 1.2).equilibrium(x0, v0, pins)
    gn = _gn(w, g0[:w.n_t], g0[w.n_t:])
    x = gn.equilibrium(x0, v0, pins)
    gq = ReducedGN(gn, H).gradient(x, target)
    v = rng.standard_normal(q.size) * np.abs(q).max()
    h = 1e-5                      # moves the softest element by about 0.4 %

    def loss(qq):
        gm = D @ qq
        g2 = _gn(w, gm[:w.n_t], gm[w.n_t:])
        return g2.loss(g2.equilibrium(x0, v0, pins), target)

    fd = (loss(q + h * v) - loss(q - h * v)) / (2 * h)
    assert abs(gq @ v - fd) < 1e-4 * abs(fd)


def test_full_basis_reproduces_the_unreduced_direction(slab):
    w = slab
    _, H = harmonic_basis(w.tets, w.n_t)
    D = basis_matrix(H)
    gn = _gn(w, w.gamma_s, w.gamma_v)
    x0, v0, pins = w.rest, np.zeros_like(w.rest), w.pin_targets(0)
    x = gn.equilibrium(x0, v0, pins)
    target = x + 1e-4 * np.random.default_rng(4).standard_normal(x.shape)
    g = gn.gradient(x, target)
    red = ReducedGN(gn, H)
    dq, kq = red.direction(x, D.T @ g, 1e-2)
    d = gn.direction(x, g, gn.kappa(x, g, 1e-2))
    assert abs(kq - gn.kappa(x, g, 1e-2)) < 1e-8 * kq
    assert rel(D @ dq, d) < 1e-8


def test_rank_one_recovers_a_constant_material(slab):
    w = slab
    x0, v0, pins = w.rest, np.zeros_like(w.rest), w.pin_targets(0)
    ones = np.ones(w.n_t)
    target = _gn(w, 2e4 * ones, 2e5 * ones).equilibrium(x0, v0, pins)
    _, H = harmonic_basis(w.tets, 1)
    gamma0 = np.concatenate([1.5e4 * ones, 1.2e5 * ones])
    g, losses = fit_reduced(w.rest, w.tets, w.pinned, w.density, w.dt, x0, v0, pins, target, gamma0, H,
                            n_gn=6, kappa_rel=1e-6)
    assert losses[-1] < 1e-6 * losses[0]
    assert rel(g, np.concatenate([2e4 * ones, 2e5 * ones])) < 1e-2
    assert np.ptp(g[:w.n_t]) < 1e-6 * g[0] and np.ptp(g[w.n_t:]) < 1e-6 * g[-1]   # stays constant


def test_planted_mistake_edge_adjacency_breaks_the_path_pin(monkeypatch):
    """Counting tets that share only an edge as neighbours must fail the
    closed-form path spectrum."""
    import oracle.harmonic as Hm
    n = 25
    tets = np.array([[j, j + 1, j + 2, j + 3] for j in range(n)])

    def edge_pairs(t):
        t = np.asarray(t)
        return np.array([(a, b) for a in range(len(t)) for b in range(a + 1, len(t))
                         if len(set(t[a]) & set(t[b])) >= 2], np.int64).reshape(-1, 2)

    monkeypatch.setattr(Hm, "face_adjacency", edge_pairs)
    lam, _ = Hm.harmonic_basis(tets, n)
    assert not np.allclose(lam, 2.0 - 2.0 * np.cos(np.pi * np.arange(n) / n), atol=1e-6)
