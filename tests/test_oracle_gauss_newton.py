"""Pins of the adjoint Gauss-Newton oracle (oracle/gauss_newton.py; Sec. 6.2
Eq. gn, Eq. agn and the Levenberg-Marquardt shift; Sec. 6.3 line search and
non-negativity).

The pins do not re-type the oracle's formulas: the paper's sparse block
system is solved as printed and compared with the dense normal equations;
the sensitivity dx/dgamma and the loss gradient are compared with central
finite differences through the whole equilibrium solve; Gauss-Newton must
behave as a second-order method on a zero-residual pose and reduce to a
scaled gradient step for a large shift; a planted mistake in dg/dgamma must
be caught by the finite-difference pin.
"""
import numpy as np
import pytest

from oracle.adjoint import AdjointOracle
from oracle.gauss_newton import (FLOOR, GaussNewtonOracle, clamp_direction, fit_pose, pick_pivot,
                                 project)
from oracle.pd_oracle import PDOracle
from workloads.meshes import slab_workload


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def _gn(w, gs, gv):
    return GaussNewtonOracle(AdjointOracle(PDOracle(w.rest, w.tets, w.pinned, gs, gv, w.density, w.dt)))


@pytest.fixture(scope="module")
def pose():
    w = slab_workload(4, 4, 2, 0.01, 5, (2, 2), seed=3, n_iter=10, name="gn-pins")
    x0, v0, pins = w.rest, np.zeros_like(w.rest), w.pin_targets(0)
    rng = np.random.default_rng(1)
    gs_star = w.gamma_s * np.exp(0.05 * rng.standard_normal(w.n_t))
    target = _gn(w, gs_star, 10 * gs_star).equilibrium(x0, v0, pins)
    gn = _gn(w, w.gamma_s, w.gamma_v)
    x = gn.equilibrium(x0, v0, pins)
    return w, gn, x, target


def _x_of(w, gamma, pins):
    n_t = w.n_t
    return _gn(w, gamma[:n_t], gamma[n_t:]).equilibrium(w.rest, np.zeros_like(w.rest), pins)


def test_block_system_is_the_negated_normal_equations(pose):
    w, gn, x, target = pose
    g = gn.gradient(x, target)
    kappa = gn.kappa(x, g, 1e-2)
    _, _, d_block = gn.block_solve(x, g, kappa)
    d = gn.direction(x, g, kappa)
    assert rel(-d_block, d) < 1e-8
    # with a fifth of the parameters pivoted (rows and columns removed)
    active = np.random.default_rng(4).random(2 * w.n_t) > 0.2
    _, _, d_block = gn.block_solve(x, g, kappa, active)
    d = gn.direction(x, g, kappa, active)
    assert np.all(d[~active] == 0) and np.all(d_block[~active] == 0)
    assert rel(-d_block, d) < 1e-8


def test_sensitivity_and_gn_form_match_finite_differences(pose):
    w, gn, x, _ = pose
    gamma = np.concatenate([w.gamma_s, w.gamma_v])
    rng = np.random.default_rng(7)
    pins = w.pin_targets(0)
    J = gn.sensitivity(x)
    P = gn.gn_matrix(x)
    f = gn.o.free
    jv = []
    for _ in range(2):
        v = gamma * rng.standard_normal(gamma.size)           # relative directions
        h = 1e-4
        fd = (_x_of(w, gamma + h * v, pins) - _x_of(w, gamma - h * v, pins)) / (2 * h)
        fd = fd[f].ravel()
        assert rel(J @ v, fd) < 1e-4
        jv.append((v, fd))
    (v1, j1), (v2, j2) = jv
    # P is the Gauss-Newton form 2 (J v1).(J v2)
    assert abs(v1 @ P @ v2 - 2.0 * j1 @ j2) < 1e-4 * abs(2.0 * j1 @ j1) ** 0.5 * abs(2.0 * j2 @ j2) ** 0.5
    # the two-solve product is the dense matrix's
    assert rel(gn.gn_product(x, v1), P @ v1) < 1e-9


def test_gradient_matches_finite_differences_of_the_pose_loss(pose):
    w, gn, x, target = pose
    gamma = np.concatenate([w.gamma_s, w.gamma_v])
    g = gn.gradient(x, target)
    rng = np.random.default_rng(9)
    v = gamma * rng.standard_normal(gamma.size)
    h = 1e-4
    pins = w.pin_targets(0)
    lp = gn.loss(_x_of(w, gamma + h * v, pins), target)
    lm = gn.loss(_x_of(w, gamma - h * v, pins), target)
    fd = (lp - lm) / (2 * h)
    assert abs(g @ v - fd) < 1e-4 * abs(fd)


def test_gn_step_is_second_order_on_a_zero_residual_pose(pose):
    w, gn, x, target = pose
    g = gn.gradient(x, target)
    e0 = gn.loss(x, target)
    gamma = np.concatenate([w.gamma_s, w.gamma_v])
    pins = w.pin_targets(0)
    d = gn.direction(x, g, gn.kappa(x, g, 1e-5))
    assert d @ g < 0
    e_gn = gn.loss(_x_of(w, np.maximum(gamma + d, FLOOR), pins), target)
    assert e_gn < 1e-2 * e0
    # steepest descent, at its best over a range of step lengths (the largest
    # moves the most sensitive parameter by 30 % of its value), stays far behind
    unit = np.min(gamma / np.abs(g))
    e_gd = min(gn.loss(_x_of(w, np.maximum(gamma - a * unit * g, FLOOR), pins), target)
               for a in (0.3, 0.1, 0.03, 0.01))
    assert e_gd > 0.5 * e0
    assert e_gn < 0.02 * e_gd


def test_large_shift_gives_the_scaled_gradient(pose):
    w, gn, x, target = pose
    g = gn.gradient(x, target)
    kappa = gn.kappa(x, g, 1e8)
    d = gn.direction(x, g, kappa)
    assert rel(d, -g / kappa) < 1e-6


def test_projection_clamp_and_pivot_helpers():
    trial, neg = project(np.array([1.0, -2.0, 0.5, -1e-9]), FLOOR)
    assert np.array_equal(neg, [False, True, False, True])
    assert np.array_equal(trial, [1.0, FLOOR, 0.5, FLOOR])
    d = clamp_direction(np.array([-1.0, -1.0, 2.0, -3.0]), np.array([True, False, True, False]))
    assert np.array_equal(d, [0.0, -1.0, 2.0, -3.0])
    gamma = np.array([FLOOR, FLOOR, 5.0, FLOOR, FLOOR])
    raw = np.array([-1.0, -4.0, -9.0, 3.0, -7.0])
    clamped = np.array([True, True, True, True, True])
    pivot = np.array([False, False, False, False, True])
    # index 2 is above the floor, 3 would rise, 4 is already pivoted
    assert pick_pivot(gamma, raw, clamped, pivot, FLOOR) == 1
    assert pick_pivot(gamma, raw, np.zeros(5, bool), pivot, FLOOR) is None


def test_fit_keeps_gamma_feasible_and_the_loss_decreasing():
    w = slab_workload(4, 4, 2, 0.01, 5, (2, 2), seed=3, n_iter=10, name="gn-fit")
    x0, v0, pins = w.rest, np.zeros_like(w.rest), w.pin_targets(0)
    rng = np.random.default_rng(1)
    gs_star = w.gamma_s.copy()
    gs_star[rng.choice(w.n_t, 12, replace=False)] /= 50.0      # a few much softer elements
    target = _gn(w, gs_star, 10 * gs_star).equilibrium(x0, v0, pins)
    gs, gv, losses, recs = fit_pose(w.rest, w.tets, w.pinned, w.density, w.dt, x0, v0, pins, target,
                                    w.gamma_s, w.gamma_v, n_gd=1, n_gn=2, kappa_rel=1e-2)
    assert [r["kind"] for r in recs] == ["gd", "gn", "gn"]
    assert all(losses[k + 1] < losses[k] for k in range(len(losses) - 1))
    assert losses[-1] < 0.5 * losses[0]
    gamma = np.concatenate([gs, gv])
    assert gamma.min() >= FLOOR
    # the softened elements drive some parameters through zero: they sit at the floor
    assert recs[-1]["clamped"] > 0 and np.any(gamma == FLOOR)


def test_planted_mistake_in_dg_dgamma_is_caught(pose, monkeypatch):
    """Using F - R(F) for the volume parameters as well must break the
    finite-difference pin of the sensitivity."""
    import oracle.gauss_newton as G
    w, gn, x, _ = pose
    gamma = np.concatenate([w.gamma_s, w.gamma_v])
    real = G.project_both

    def wrong(F):
        R, V, *rest = real(F)
        return (R, R, *rest)

    monkeypatch.setattr(G, "project_both", wrong)
    J = gn.sensitivity(x)
    monkeypatch.setattr(G, "project_both", real)
    v = np.zeros_like(gamma)
    v[w.n_t:] = w.gamma_v                                        # move only the volume parameters
    h = 1e-4
    pins = w.pin_targets(0)
    fd = (_x_of(w, gamma + h * v, pins) - _x_of(w, gamma - h * v, pins)) / (2 * h)
    assert rel(J @ v, fd[gn.o.free].ravel()) > 1e-2


def test_pivoting_keeps_the_direction_a_descent_direction():
    """With a tiny shift the clamped Gauss-Newton direction stops being a
    descent direction on the softened pose; pivoting removes cached
    parameters at the floor until it is one again (Sec. 6.3)."""
    w = slab_workload(4, 4, 2, 0.01, 5, (2, 2), seed=3, n_iter=10, name="gn-pivot")
    x0, v0, pins = w.rest, np.zeros_like(w.rest), w.pin_targets(0)
    rng = np.random.default_rng(1)
    gs_star = w.gamma_s.copy()
    gs_star[rng.choice(w.n_t, 12, replace=False)] /= 50.0
    target = _gn(w, gs_star, 10 * gs_star).equilibrium(x0, v0, pins)
    gs, gv, losses, recs = fit_pose(w.rest, w.tets, w.pinned, w.density, w.dt, x0, v0, pins, target,
                                    w.gamma_s, w.gamma_v, n_gd=1, n_gn=3, kappa_rel=1e-6)
    assert recs[-1]["pivots"] > 0
    assert all(losses[k + 1] < losses[k] for k in range(len(losses) - 1))
    gamma = np.concatenate([gs, gv])
    assert gamma.min() >= FLOOR
    # after the pivots every direction taken is a descent direction
    assert all(r["descent"] < 0 for r in recs)
