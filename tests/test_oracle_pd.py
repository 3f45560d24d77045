"""Pins of the FP64 projective-dynamics oracle (Sec. 7, Sec. 7.1).

The oracle's matrix, right-hand side, solver and stepper are checked
against closed forms (volumes, mass, the quadratic form of K), invariants
(rest state, translation invariance, momentum, monotone PD energy) and a
direct minimisation of the implicit-Euler objective on tiny meshes.
"""
import numpy as np
import pytest
import scipy.optimize as so

from oracle.pd_oracle import (PDOracle, deformation_gradient, lumped_mass, rest_shape,
                              stiffness_scalar)
from oracle.projections import project_both
from workloads.meshes import parity_slab, slab, sweater_shell

rng = np.random.default_rng(5)


@pytest.fixture(scope="module")
def slab_w():
    return parity_slab()


@pytest.fixture(scope="module")
def slab_o(slab_w):
    w = slab_w
    return PDOracle(w.rest, w.tets, w.pinned, w.gamma_s, w.gamma_v, w.density, w.dt)


def test_volume_and_mass_closed_form(slab_w, slab_o):
    assert np.all(slab_o.vol > 0)
    assert abs(slab_o.vol.sum() - 0.2 * 0.2 * 0.02) < 1e-15
    assert abs(slab_o.mass.sum() - 300.0 * 0.2 * 0.2 * 0.02) < 1e-13
    # faceted shell: annulus between two regular N-gons times the height
    s = sweater_shell(n_theta=40, n_z=6, n_r=2, dom_theta=4, dom_z=2)
    _, vol, _ = rest_shape(s.rest, s.tets)
    N, ro, ri = 40, 0.305, 0.295
    exact = 0.5 * N * np.sin(2 * np.pi / N) * (ro ** 2 - ri ** 2) * 0.6
    assert abs(vol.sum() - exact) < 1e-14
    assert np.all(vol > 0)


def test_stiffness_quadratic_form_matches_gradient_energy(slab_w, slab_o):
    # x^T K_s x = sum_v m_v/dt^2 x_v^2 + sum_e V_e (gs+gv) |grad phi_e|^2 where
    # phi_e is the linear interpolant of the scalar field x on tet e
    o = slab_o
    x = rng.standard_normal(o.n_v)
    lhs = x @ (o.K @ x)
    X = o.rest[o.tets]
    E = np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]], axis=1)   # rows
    dv = np.stack([x[o.tets[:, k]] - x[o.tets[:, 0]] for k in (1, 2, 3)], axis=1)
    grad = np.linalg.solve(E, dv[..., None])[..., 0]
    rhs = np.sum(o.mass / o.dt ** 2 * x * x) + np.sum(o.vol * (o.gamma_s + o.gamma_v) * np.sum(grad ** 2, 1))
    assert abs(lhs - rhs) < 1e-11 * abs(rhs)


def test_rest_state_is_a_fixed_point(slab_w, slab_o):
    x, v = slab_o.step(slab_w.rest, np.zeros_like(slab_w.rest), None, gravity=(0, 0, 0), n_iter=5)
    assert np.abs(x - slab_w.rest).max() < 1e-14
    assert np.abs(v).max() < 1e-11


def test_corner_forces_sum_to_zero(slab_w, slab_o):
    x = slab_w.rest + 0.002 * rng.standard_normal(slab_w.rest.shape)
    R, V = slab_o.local(x)
    P = slab_o.ws[:, None, None] * R + slab_o.wv[:, None, None] * V
    f = np.einsum("eij,ecj->eci", P, slab_o.g)
    assert np.abs(f.sum(axis=1)).max() < 1e-12 * np.abs(f).max()


def test_pd_energy_never_increases(slab_w, slab_o):
    x, v = slab_w.rest.copy(), np.zeros_like(slab_w.rest)
    for n in range(8):
        rec = []
        x, v = slab_o.step(x, v, slab_w.pin_targets(n), n_iter=6, record=rec)
        q = np.array([r[1] for r in rec])
        assert np.all(np.diff(q) <= 1e-12 * np.abs(q[:-1]))


def test_global_step_solves_the_linear_system_exactly(slab_w, slab_o):
    o = slab_o
    x = slab_w.rest + 0.003 * rng.standard_normal(slab_w.rest.shape)
    y = x + 0.001 * rng.standard_normal(x.shape)
    R, V = o.local(x)
    b = o.rhs(y, R, V)
    xp = slab_w.rest[o.pin_ids]
    xf = o.global_solve(b, xp)
    res = o.K_ff @ xf - (b[o.free] - o.K_fp @ xp)
    assert np.abs(res).max() < 1e-12 * np.abs(b).max()


def _energy_and_grad(o, x, y):
    """Implicit-Euler objective E(x) = Q(x; R(x), V(x)) and its gradient from
    per-element forces (no assembled matrix)."""
    F = deformation_gradient(x, o.tets, o.g)
    R, V, *_ = project_both(F)
    E = 0.5 / o.dt ** 2 * np.sum(o.mass[:, None] * (x - y) ** 2) + 0.5 * np.sum(
        o.ws * np.sum((F - R) ** 2, axis=(1, 2)) + o.wv * np.sum((F - V) ** 2, axis=(1, 2)))
    P = o.ws[:, None, None] * (F - R) + o.wv[:, None, None] * (F - V)
    grad = (o.mass / o.dt ** 2)[:, None] * (x - y)
    np.add.at(grad, o.tets.ravel(), np.einsum("eij,ecj->eci", P, o.g).reshape(-1, 3))
    return E, grad


def test_energy_gradient_matches_finite_differences_and_k_minus_b(slab_w, slab_o):
    o = slab_o
    x = slab_w.rest + 0.002 * rng.standard_normal(slab_w.rest.shape)
    y = x + 0.001 * rng.standard_normal(x.shape)
    E, grad = _energy_and_grad(o, x, y)
    h = 1e-7
    for _ in range(12):
        v, c = rng.integers(o.n_v), rng.integers(3)
        xp, xm = x.copy(), x.copy()
        xp[v, c] += h
        xm[v, c] -= h
        fd = (_energy_and_grad(o, xp, y)[0] - _energy_and_grad(o, xm, y)[0]) / (2 * h)
        assert abs(fd - grad[v, c]) < 2e-5 * max(1.0, abs(grad[v, c]))
    # the PD system is the stationarity condition: K x - b = grad E
    R, V = o.local(x)
    kxb = (o.K @ x) - o.rhs(y, R, V)
    assert np.abs(kxb - grad).max() < 1e-9 * np.abs(grad).max()


def _tiny(kind):
    if kind == "tet":
        rest = np.array([[0, 0, 0], [0.01, 0, 0], [0, 0.01, 0], [0, 0, 0.01]], float)
        tets = np.array([[0, 1, 2, 3]], np.int32)
        pinned = np.array([1, 1, 0, 0], np.uint8)
    else:
        rest, tets, _ = slab(1, 1, 1, 0.01, 6)
        pinned = (rest[:, 0] < 1e-12).astype(np.uint8)
    gs = np.full(tets.shape[0], 2e3)
    return rest, tets, pinned, gs


@pytest.mark.parametrize("kind", ["tet", "cube"])
def test_converged_pd_is_the_implicit_euler_minimiser(kind):
    rest, tets, pinned, gs = _tiny(kind)
    o = PDOracle(rest, tets, pinned, gs, 10 * gs, 300.0, 1.0 / 30.0)
    v0 = np.zeros_like(rest)
    v0[:, 2] = -0.3
    x_pd, _ = o.step(rest, v0, None, n_iter=4000)
    y = o.inertial_target(rest, v0)
    free = o.free

    def fun(z):
        x = rest.copy()
        x[free] = z.reshape(-1, 3)
        E, g = _energy_and_grad(o, x, y)
        return E, g[free].ravel()

    x0 = y[free].ravel()
    res = so.minimize(fun, x0, jac=True, method="BFGS", options={"gtol": 1e-13, "maxiter": 20000})
    x_min = rest.copy()
    x_min[free] = res.x.reshape(-1, 3)
    disp = np.abs(x_min - rest).max()
    assert disp > 1e-4                       # the test actually moves the mesh
    assert np.abs(x_pd - x_min).max() < 1e-7 * max(disp, 1e-3)
    assert np.abs(_energy_and_grad(o, x_pd, y)[1][free]).max() < 1e-8


def test_momentum_is_conserved_without_pins_or_gravity():
    rest, tets, _ = slab(3, 3, 1, 0.01, 6)
    gs = np.exp(rng.uniform(np.log(1e3), np.log(1e5), tets.shape[0]))
    o = PDOracle(rest, tets, np.zeros(rest.shape[0], np.uint8), gs, 10 * gs)
    x = rest.copy()
    v = 0.5 * rng.standard_normal(rest.shape)
    p0 = (o.mass[:, None] * v).sum(0)
    for _ in range(5):
        x, v = o.step(x, v, None, gravity=(0, 0, 0), n_iter=7)
        p = (o.mass[:, None] * v).sum(0)
        assert np.abs(p - p0).max() < 1e-11 * np.abs(p0).max()


class _WrongSignOracle(PDOracle):
    """Planted mistake: the volume target enters b with the wrong sign."""

    def rhs(self, y, R, V):
        return super().rhs(y, R, -V)


def test_planted_mistake_breaks_the_rest_state_pin(slab_w):
    w = slab_w
    bad = _WrongSignOracle(w.rest, w.tets, w.pinned, w.gamma_s, w.gamma_v, w.density, w.dt)
    x, _ = bad.step(w.rest, np.zeros_like(w.rest), None, gravity=(0, 0, 0), n_iter=3)
    assert np.abs(x - w.rest).max() > 1e-4


def test_lumped_mass_counts_each_tet_once():
    rest, tets, _ = slab(2, 2, 2, 0.01, 5)
    _, vol, _ = rest_shape(rest, tets)
    m = lumped_mass(rest.shape[0], tets, vol, 300.0)
    assert abs(m.sum() - 300.0 * 0.02 ** 3) < 1e-15
    K = stiffness_scalar(rest.shape[0], tets, vol, rest_shape(rest, tets)[2], np.ones(len(tets)),
                         np.ones(len(tets)), m, 0.01)
    # elastic part annihilates constants: K 1 = m / dt^2
    assert np.abs(K @ np.ones(rest.shape[0]) - m / 1e-4).max() < 1e-9 * (m / 1e-4).max()
