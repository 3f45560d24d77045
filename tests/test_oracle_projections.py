"""Pins of the oracle's local-step projections (Sec. 7.1, Eq. pd_local, Eq. vol_pre).

Each check compares the oracle with something other than itself: closed
forms, group invariances, an independent library polar decomposition, and a
brute-force 2-D search of the volume problem.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle.projections import (CLAMP, project_both, project_rotation, project_volume,
                                project_volume_sigma, svd_rotation_variant)

rng = np.random.default_rng(1234)


def random_rotations(n, rng):
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)], -1),
        np.stack([2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)], -1),
        np.stack([2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)], -1),
    ], 1)


def test_identity_gives_identity():
    R, V, *_ = project_both(np.eye(3)[None])
    assert np.allclose(R[0], np.eye(3), atol=1e-14)
    assert np.allclose(V[0], np.eye(3), atol=1e-14)


def test_rotation_is_its_own_projection():
    Q = random_rotations(200, rng)
    R, V, *_ = project_both(Q)
    assert np.abs(R - Q).max() < 1e-12
    assert np.abs(V - Q).max() < 1e-12


def test_unit_determinant_is_its_own_volume_projection():
    A = np.eye(3) + 0.3 * rng.standard_normal((300, 3, 3))
    det = np.linalg.det(A)
    A = A[det > 0.05]
    A = A / np.cbrt(np.linalg.det(A))[:, None, None]
    V = project_volume(A)
    assert np.abs(V - A).max() < 1e-10


@pytest.mark.parametrize("s", [0.3, 0.7, 1.0, 1.4])
def test_isotropic_scaling(s):
    # F = s I: R = I, and V = I when s is moderate (the all-r+ root is the minimum)
    R, V, *_ = project_both((s * np.eye(3))[None])
    assert np.allclose(R[0], np.eye(3), atol=1e-13)
    assert np.allclose(V[0], np.eye(3), atol=1e-12)


def test_orthonormal_det_plus_one_and_unit_det():
    F = np.eye(3) + 0.8 * rng.standard_normal((2000, 3, 3))
    R, V, U, s, W, d = project_both(F)
    RtR = np.einsum("eki,ekj->eij", R, R)
    assert np.abs(RtR - np.eye(3)).max() < 1e-12
    assert np.abs(np.linalg.det(R) - 1).max() < 1e-12
    assert np.abs(np.linalg.det(V) - 1).max() < 1e-11
    assert np.all(d >= CLAMP * (1 - 1e-12))
    # rotation-variant SVD reconstructs F with U, W in SO(3)
    Frec = (U * s[:, None, :]) @ np.swapaxes(W, 1, 2)
    assert np.abs(Frec - F).max() < 1e-12
    assert np.abs(np.linalg.det(U) - 1).max() < 1e-12
    assert np.abs(np.linalg.det(W) - 1).max() < 1e-12
    assert np.all(np.sign(s[:, 2]) == np.sign(np.linalg.det(F)))


def test_rotation_matches_library_polar_for_positive_det():
    F = np.eye(3) + 0.5 * rng.standard_normal((200, 3, 3))
    F = F[np.linalg.det(F) > 0.05]
    R = project_rotation(F)
    for i in range(F.shape[0]):
        u, _ = sla.polar(F[i])
        assert np.abs(u - R[i]).max() < 1e-10


def test_rotation_equivariance_and_invariance():
    F = np.eye(3) + 0.7 * rng.standard_normal((300, 3, 3))
    Q = random_rotations(300, rng)
    P = random_rotations(300, rng)
    R, V, *_ = project_both(F)
    R2, V2, *_ = project_both(Q @ F @ P)
    assert np.abs(R2 - Q @ R @ P).max() < 1e-10
    assert np.abs(V2 - Q @ V @ P).max() < 1e-8


def test_rotation_is_nearest_among_perturbed_rotations():
    F = np.eye(3) + 0.6 * rng.standard_normal((50, 3, 3))
    R = project_rotation(F)
    base = np.sum((F - R) ** 2, axis=(1, 2))
    for _ in range(20):
        Qp = random_rotations(50, rng)
        # small rotation: interpolate toward identity via a few Gram-Schmidt steps
        A = R @ (np.eye(3) + 0.05 * (Qp - np.swapaxes(Qp, 1, 2)))
        U, _, Vh = np.linalg.svd(A)
        Qn = U @ Vh
        Qn[np.linalg.det(Qn) < 0] *= -1
        assert np.all(np.sum((F - Qn) ** 2, axis=(1, 2)) >= base - 1e-12)


def test_volume_is_nearest_among_perturbed_unit_det():
    F = np.eye(3) + 0.5 * rng.standard_normal((60, 3, 3))
    V = project_volume(F)
    base = np.sum((F - V) ** 2, axis=(1, 2))
    for _ in range(30):
        A = V + 0.02 * rng.standard_normal(V.shape)
        det = np.linalg.det(A)
        ok = det > 0
        A = A[ok] / np.cbrt(det[ok])[:, None, None]
        # stay inside the clamp region
        sv = np.linalg.svd(A, compute_uv=False)
        keep = sv.min(axis=1) >= CLAMP
        cost = np.sum((F[ok][keep] - A[keep]) ** 2, axis=(1, 2))
        assert np.all(cost >= base[ok][keep] - 1e-12)


def test_diagonal_kkt_structure():
    # F = diag(sigma): V diagonal; free targets share mu = (d - sigma) d
    s = np.array([[1.3, 1.0, 0.8], [1.1, 0.95, 0.9], [0.9, 0.8, 0.7]])
    V = project_volume(np.stack([np.diag(r) for r in s]))
    for i in range(s.shape[0]):
        d = np.diag(V[i])
        assert np.abs(V[i] - np.diag(d)).max() < 1e-12
        mu = (d - s[i]) * d
        assert np.ptp(mu) < 1e-12
        assert abs(np.prod(d) - 1) < 1e-13


def _brute_force_volume(s, lo=CLAMP, n=1201, rounds=9):
    """min over u in R^2 of sum (d - s)^2, d = (e^u1, e^u2, e^(-u1-u2)), d >= lo."""
    a, b = np.log(lo), -2 * np.log(lo)

    def cost(u1, u2):
        d1, d2 = np.exp(u1), np.exp(u2)
        d3 = np.exp(-u1 - u2)
        c = (d1 - s[0]) ** 2 + (d2 - s[1]) ** 2 + (d3 - s[2]) ** 2
        bad = (d1 < lo) | (d2 < lo) | (d3 < lo * (1 - 1e-15))
        return np.where(bad, np.inf, c)

    g = np.linspace(a, b, n)
    U1, U2 = np.meshgrid(g, g, indexing="ij")
    C = cost(U1, U2)
    # refine around the best few grid minima (several basins may compete)
    flat = np.argsort(C, axis=None)[:40]
    best_c, best_u = np.inf, None
    for f in flat:
        i, j = np.unravel_index(f, C.shape)
        u1, u2 = U1[i, j], U2[i, j]
        h = (b - a) / (n - 1)
        for _ in range(rounds):
            gg = np.linspace(-2 * h, 2 * h, 41)
            A1, A2 = np.meshgrid(u1 + gg, u2 + gg, indexing="ij")
            CC = cost(A1, A2)
            k = np.unravel_index(np.argmin(CC), CC.shape)
            u1, u2 = A1[k], A2[k]
            h /= 10
        c = cost(np.array(u1), np.array(u2))
        if c < best_c:
            best_c, best_u = float(c), (u1, u2)
    u1, u2 = best_u
    return best_c, np.array([np.exp(u1), np.exp(u2), np.exp(-u1 - u2)])


ADVERSARIAL = [
    (1, 1, 1), (2, 2, 1), (100, 1, 1), (3, 1, 0.2), (1.1, 0.9, -0.3), (0.5, 0.5, 0.5),
    (5, 5, 5), (1.5, 1.5, 1.5), (1.0001, 1.0, 0.9999), (2, 1e-3, 1e-3), (1, 1, 0.0),
    (1, 1, -1), (0.02, 0.02, 0.02), (50, 50, 1e-4), (1.9, 1.8, 1.7), (3, 3, 0.5),
    (10, 0.5, 0.5), (0.3, 0.2, -0.1), (2.5, 0.4, 0.05), (8, 8, 8), (1.2, 1.2, -2.0),
]


@pytest.mark.parametrize("s", ADVERSARIAL)
def test_volume_projection_matches_brute_force_adversarial(s):
    s = np.array(s, float)
    d = project_volume_sigma(s[None])[0]
    c_or = np.sum((d - s) ** 2)
    c_bf, d_bf = _brute_force_volume(s)
    assert abs(np.prod(d) - 1) < 1e-12
    assert np.all(d >= CLAMP * (1 - 1e-12))
    assert c_or <= c_bf + 1e-12 * max(1.0, c_bf)
    assert c_bf <= c_or + 1e-8 * max(1.0, c_or)


def test_volume_projection_matches_brute_force_random():
    r = np.random.default_rng(77)
    for _ in range(40):
        s = np.sort(np.exp(r.uniform(np.log(0.05), np.log(20.0), 3)))[::-1].copy()
        if r.uniform() < 0.25:
            s[2] = -s[2]
        d = project_volume_sigma(s[None])[0]
        c_or = np.sum((d - s) ** 2)
        c_bf, d_bf = _brute_force_volume(s)
        assert c_or <= c_bf + 1e-12 * max(1.0, c_bf), (s, d, d_bf)
        assert c_bf <= c_or + 1e-8 * max(1.0, c_or), (s, d, d_bf)
        # unique minimiser here unless costs of distinct points tie
        if np.abs(d - d_bf).max() > 1e-4:
            assert abs(c_bf - c_or) < 1e-9 * max(1.0, c_or)


def test_planted_mistake_is_caught():
    # a projection that forgets the clamp / uses the naive all-r+ root fails
    # the brute-force comparison on a large-stretch case
    s = np.array([2.0, 2.0, 1.0])
    naive = np.cbrt(1.0 / np.prod(s)) * s      # uniform rescaling to det 1
    c_bf, _ = _brute_force_volume(s)
    assert np.sum((naive - s) ** 2) > c_bf + 1e-3
    d = project_volume_sigma(s[None])[0]
    assert abs(np.sum((d - s) ** 2) - c_bf) < 1e-8
