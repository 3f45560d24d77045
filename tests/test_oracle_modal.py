"""Pins of the modal (paper-faithful) global-solve oracle (oracle/modal.py,
Sec. 7.2): identities the construction must satisfy and convergence facts,
none of which re-types the oracle's formulas."""
import numpy as np
import pytest

from oracle.modal import ModalDD, classify
from oracle.pd_oracle import PDOracle
from workloads.meshes import slab_workload


@pytest.fixture(scope="module")
def setup():
    w = slab_workload(8, 8, 2, 0.01, 6, (2, 2), seed=5, n_iter=10, name="modal-pins")
    o = PDOracle(w.rest, w.tets, w.pinned, w.gamma_s, w.gamma_v, w.density, w.dt)
    rng = np.random.default_rng(3)
    b = rng.standard_normal((o.free.size, 3))
    exact = o.chol.solve(b)
    return w, o, b, exact


def _dd(w, o, modes):
    return ModalDD(o.K_ff, o.free, w.n_v, w.tets, w.tet_domain, w.n_domains, w.pinned, modes=modes)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_all_modes_is_the_direct_solve(setup):
    # with every internal mode the subspace is the whole space: the Galerkin
    # solve is the exact solve of K x = b
    w, o, b, exact = setup
    dd = _dd(w, o, modes=10 ** 6)
    assert rel(dd.reduced_solve(b), exact) < 1e-10


def test_interface_values_are_exact_with_any_number_of_modes(setup):
    # Phi^T (K_ii Psi + K_ib) = 0 decouples x_b from the truncation
    w, o, b, exact = setup
    dd = _dd(w, o, modes=5)
    x = dd.reduced_solve(b)
    assert rel(x[dd.B], exact[dd.B]) < 1e-10
    assert rel(x, exact) > 1e-6          # but the internal response is truncated


def test_normal_modes_are_the_lowest_eigenpairs(setup):
    w, o, _, _ = setup
    dd = _dd(w, o, modes=12)
    rng = np.random.default_rng(8)
    Kd = o.K_ff.toarray()
    for d in dd.domains:
        Kii = Kd[np.ix_(d["I"], d["I"])]
        Phi, lam = d["Phi"], d["lam"]
        assert np.allclose(Phi.T @ Phi, np.eye(Phi.shape[1]), atol=1e-10)
        assert np.linalg.norm(Kii @ Phi - Phi * lam) < 1e-9 * np.linalg.norm(Kii)
        # Courant-Fischer: no direction orthogonal to the modes has a lower
        # Rayleigh quotient than the largest kept eigenvalue
        z = rng.standard_normal((Kii.shape[0], 200))
        z -= Phi @ (Phi.T @ z)
        rq = np.einsum("ij,ij->j", z, Kii @ z) / np.einsum("ij,ij->j", z, z)
        assert rq.min() >= lam.max() * (1 - 1e-9)


def test_more_modes_never_hurt(setup):
    w, o, b, exact = setup
    errs = [rel(_dd(w, o, modes=m).reduced_solve(b), exact) for m in (2, 8, 20, 40)]
    assert all(errs[k + 1] <= errs[k] + 1e-12 for k in range(len(errs) - 1)), errs


def test_chebyshev_jacobi_converges_to_the_direct_solve(setup):
    w, o, b, exact = setup
    dd = _dd(w, o, modes=20)
    rho = dd.jacobi_rho()
    assert 0 < rho < 1
    x0 = dd.reduced_solve(b)
    e = [rel(dd.chebyshev_jacobi(b, x0, s, rho), exact) for s in (0, 10, 40, 400)]
    assert e[1] < e[0] and e[2] < e[1]
    assert e[3] < 1e-9
    # Chebyshev weights beat plain Jacobi (rho = 0 gives omega = 1 throughout)
    assert rel(dd.chebyshev_jacobi(b, x0, 40, rho), exact) < rel(dd.chebyshev_jacobi(b, x0, 40, 0.0), exact)


def test_planted_mistake_largest_modes_is_worse(setup):
    # keeping the largest instead of the smallest eigenvalues must lose accuracy
    w, o, b, exact = setup
    dd = _dd(w, o, modes=12)
    good = rel(dd.reduced_solve(b), exact)
    Kd = o.K_ff.toarray()
    for d in dd.domains:
        lam, vec = np.linalg.eigh(Kd[np.ix_(d["I"], d["I"])])
        d["lam"], d["Phi"] = lam[-12:], vec[:, -12:]
    assert rel(dd.reduced_solve(b), exact) > 2 * good


def test_classify_counts_match_the_mesh(setup):
    w, o, _, _ = setup
    iface, vdom = classify(w.n_v, w.tets, w.tet_domain, w.pinned)
    assert not np.any(iface & w.pinned.astype(bool))
    free = ~w.pinned.astype(bool)
    assert np.all((vdom >= 0) == (free & ~iface))
