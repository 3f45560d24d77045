"""Pins of the FP64 adjoint oracle (Sec. 6.1: Eq. g, Eq. pxpgamma,
Eq. adjoint_state, Eq. adjoint_state_solve).

Projection derivatives and the Hessian are checked against central finite
differences of the oracle's own projections/residual; the adjoint gradient
against central finite differences of the loss through the whole
equilibrium forward simulation.
"""
import numpy as np
import pytest

from oracle.adjoint import AdjointOracle, ProjectionDerivative
from oracle.pd_oracle import PDOracle
from oracle.projections import project_both
from workloads.meshes import slab_workload

rng = np.random.default_rng(21)


def test_projection_derivatives_match_finite_differences():
    F = np.eye(3) + 0.4 * rng.standard_normal((300, 3, 3))
    F = F[np.linalg.det(F) > 0.1]
    # include inverted elements away from sigma_2 + sigma_3 = 0
    G = np.eye(3) + 0.3 * rng.standard_normal((100, 3, 3))
    G[:, :, 2] *= -1
    sv = np.linalg.svd(G, compute_uv=False)
    F = np.concatenate([F, G[(sv[:, 1] - sv[:, 2]) > 0.2]])
    D = ProjectionDerivative(F)
    dF = rng.standard_normal(F.shape)
    h = 1e-6
    Rp, Vp, *_ = project_both(F + h * dF)
    Rm, Vm, *_ = project_both(F - h * dF)
    assert np.abs((Rp - Rm) / (2 * h) - D.dR(dF)).max() < 1e-7
    assert np.abs((Vp - Vm) / (2 * h) - D.dV(dF)).max() < 1e-6 * max(1.0, np.abs(D.dV(dF)).max())


@pytest.fixture(scope="module")
def small():
    w = slab_workload(4, 4, 2, 0.01, 5, (2, 2), seed=3, n_iter=10, name="adj")
    o = PDOracle(w.rest, w.tets, w.pinned, w.gamma_s, w.gamma_v, w.density, w.dt)
    return w, o, AdjointOracle(o)


def test_hessian_matches_finite_differences_of_the_residual(small):
    w, o, A = small
    x = w.rest + 1e-3 * rng.standard_normal(w.rest.shape)
    y = x + 1e-4 * rng.standard_normal(x.shape)
    H = A.hessian(x)
    v = np.zeros_like(x)
    v[o.free] = rng.standard_normal((len(o.free), 3))
    h = 1e-7
    fd = (A.residual(x + h * v, y) - A.residual(x - h * v, y)) / (2 * h)
    Hv = H @ v[o.free].ravel()
    assert np.abs(fd[o.free].ravel() - Hv).max() < 1e-5 * np.abs(Hv).max()


def test_equilibrium_satisfies_the_constraint(small):
    w, o, A = small
    xs, vs = A.forward(w.rest, np.zeros_like(w.rest), w.pin_targets, 3)
    for n in range(1, 4):
        y = o.inertial_target(xs[n - 1], vs[n - 1], A.g)
        r = A.residual(xs[n], y)[o.free]
        assert np.linalg.norm(r) < 1e-10 * np.linalg.norm(o.mass[o.free] * 9.81)


def test_adjoint_gradient_matches_finite_differences(small):
    w, o, A = small
    n_steps = 5
    w2 = slab_workload(4, 4, 2, 0.01, 5, (2, 2), seed=4, n_iter=10, name="adj-target")
    At = AdjointOracle(PDOracle(w.rest, w.tets, w.pinned, w2.gamma_s, w2.gamma_v, w.density, w.dt))
    targets, _ = At.forward(w.rest, np.zeros_like(w.rest), w.pin_targets, n_steps)
    xs, _ = A.forward(w.rest, np.zeros_like(w.rest), w.pin_targets, n_steps)
    gs, gv = A.gradient(xs, targets)
    theta = w.gamma_s.copy()

    def loss_at(th):
        oo = PDOracle(w.rest, w.tets, w.pinned, th, 10 * th, w.density, w.dt)
        AA = AdjointOracle(oo)
        xx, _ = AA.forward(w.rest, np.zeros_like(w.rest), w.pin_targets, n_steps)
        return AA.loss(xx, targets, o.free)

    for e in rng.choice(o.n_t, 6, replace=False):
        h = 1e-4 * theta[e]
        tp, tm = theta.copy(), theta.copy()
        tp[e] += h
        tm[e] -= h
        fd = (loss_at(tp) - loss_at(tm)) / (2 * h)
        ad = gs[e] + 10.0 * gv[e]          # tied parameter: gamma_s = theta, gamma_v = 10 theta
        assert abs(fd - ad) <= 1e-5 * abs(fd), (e, fd, ad)


def test_gradient_vanishes_on_its_own_trajectory(small):
    w, o, A = small
    xs, _ = A.forward(w.rest, np.zeros_like(w.rest), w.pin_targets, 3)
    gs, gv = A.gradient(xs, [x.copy() for x in xs])
    assert np.abs(gs).max() == 0.0 and np.abs(gv).max() == 0.0


def test_checkpointed_recomputation_is_bitwise_identical(small):
    w, o, A = small
    xs, vs = A.forward(w.rest, np.zeros_like(w.rest), w.pin_targets, 6)
    # recompute steps 3..6 from the checkpoint at step 3
    xr, vr = A.forward(xs[3], vs[3], lambda n: w.pin_targets(n + 3), 3)
    for k in range(4):
        assert np.array_equal(xr[k], xs[3 + k])
