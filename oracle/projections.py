"""FP64 oracle for the per-element projections of the local step.

TEST INFRASTRUCTURE ONLY: imported by tests/, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of bench.py.  The CUDA library never imports or calls it.

Paper passages followed (Sec. 7.1, Projective Dynamics, and Eq. pd_local):

* the rotation target R(F) = argmin over SO(3) of ||F - A||_F, obtained by
  polar decomposition through the SVD F = U Sigma W^T;
* the volume target V(F) = argmin over SL(3) of ||F - A||_F.  The paper
  reduces it to three singular values (Eq. vol_pre): minimise
  sum_i dsigma_i^2 subject to prod_i (sigma_i + dsigma_i) = 1 and
  sigma_i + dsigma_i > 0, solved through the KKT system of the equality
  constraint with any violating target clamped to [0.01, inf) and frozen.

Readings taken here (the paper is terse):

* SVD convention: rotation-variant, U and W in SO(3); the last singular value
  carries the sign of det F.  Then R = U W^T and V = U diag(d) W^T.  Sharing
  U, W between F and V is exact for this problem: the Frobenius-nearest point
  of a set invariant under left/right rotations keeps the singular vectors
  (von Neumann's trace inequality).
* The clamp acts on the target singular value d_i = sigma_i + dsigma_i and
  keeps d_i >= 0.01, so the problem solved is
      min sum_i (d_i - sigma_i)^2   s.t.  prod_i d_i = 1,  d_i >= 0.01,
  and the answer is its GLOBAL minimiser (the KKT system has several
  stationary points; the paper's "very few iterations" is read as "to
  convergence").

Method (written for checking by eye, not for speed): every local minimiser
lies in the relative interior of one face of the feasible set (no, one or
two targets held at the clamp), where it is a KKT point:
(d_i - sigma_i) d_i = mu for the free i, so each free d_i is a root
r+(mu) = (sigma_i + sqrt(sigma_i^2 + 4 mu))/2 or r-(mu) = (sigma_i -
sqrt(...))/2.  In log coordinates u_i = ln d_i the constraint is linear and
the objective's Hessian is diag(2 d_i (2 d_i - sigma_i)); an r- root has
d_i < sigma_i/2, so two r- roots give negative curvature along
e_j - e_k and cannot be a minimum.  Hence the candidates are: all r+ (the
product is increasing in mu: one root, bisection), exactly one r- (found by
scanning that component's value and bisecting every sign change), and the
three corners with two clamped targets.  The answer is the cheapest
feasible candidate.
"""
from __future__ import annotations

import numpy as np

CLAMP = 0.01          # lower bound on a target singular value (Sec. 7.1)
_SCAN = 192           # grid points of the one-r- scan
_BISECT = 90            # bisection steps: the bracket reaches FP64 rounding in < 80


def svd_rotation_variant(F: np.ndarray):
    """F = U diag(s) W^T with U, W in SO(3); s[..., 2] has the sign of det F.

    Uses LAPACK's SVD (numpy) and flips the last column of U or W when its
    determinant is negative, moving the sign onto the smallest singular value.
    """
    F = np.asarray(F, dtype=np.float64)
    U, s, Vh = np.linalg.svd(F)
    U = U.copy()
    s = s.copy()
    W = np.swapaxes(Vh, -1, -2).copy()
    du = np.linalg.det(U) < 0
    U[du, :, 2] *= -1.0
    s[du, 2] *= -1.0
    dw = np.linalg.det(W) < 0
    W[dw, :, 2] *= -1.0
    s[dw, 2] *= -1.0
    return U, s, W


def project_rotation(F: np.ndarray) -> np.ndarray:
    """R(F) = U W^T: the nearest rotation (polar factor with det +1)."""
    U, _, W = svd_rotation_variant(F)
    return U @ np.swapaxes(W, -1, -2)


def _rp(s, mu):
    return 0.5 * (s + np.sqrt(np.maximum(s * s + 4.0 * mu, 0.0)))


def _rm(s, mu):
    return 0.5 * (s - np.sqrt(np.maximum(s * s + 4.0 * mu, 0.0)))


def _all_plus(s: np.ndarray, logp: float, lo: float):
    """Free targets all on r+, prod = exp(logp), each >= lo.  s: (n, k).

    Returns d (n, k) with NaN rows where this face holds no KKT point.
    """
    n, k = s.shape
    # smallest mu with every r+ real and >= lo: r+ >= lo always holds when
    # sigma >= 2 lo (r+ >= sigma/2); otherwise it needs mu >= lo^2 - sigma lo
    mu_lo = np.max(np.where(s >= 2.0 * lo, -0.25 * s * s, lo * lo - s * lo), axis=1)
    c = max(np.exp(logp / k), lo)
    mu_hi = np.max(c * c - s * c, axis=1)              # every r+ >= c: product >= p
    mu_hi = np.maximum(mu_hi, mu_lo)

    def psi(mu):
        return np.sum(np.log(_rp(s, mu[:, None])), axis=1) - logp

    ok = psi(mu_lo) <= 0.0
    a, b = mu_lo.copy(), mu_hi.copy()
    for _ in range(_BISECT):
        m = 0.5 * (a + b)
        neg = psi(m) <= 0.0
        a = np.where(neg, m, a)
        b = np.where(neg, b, m)
    mu = 0.5 * (a + b)
    d = _rp(s, mu[:, None])
    d[~ok] = np.nan
    return d


def _one_minus(s: np.ndarray, m: int, logp: float, lo: float):
    """Free target m on r-, the others on r+; prod = exp(logp); all >= lo.

    The r- value t of component m parameterises the branch:
    mu = t^2 - s_m t for t in [lo, s_m/2].  Returns a list of (n, k) arrays,
    one per root found (NaN where a row has fewer roots).
    """
    n, k = s.shape
    sm = s[:, m]
    others = [i for i in range(k) if i != m]
    so = s[:, others]
    out = []
    valid_rows = sm / 2.0 > lo
    if not np.any(valid_rows):
        return out
    # upper bound of psi over the branch: t <= s_m/2 and mu <= lo^2 - s_m lo
    mu_top = lo * lo - sm * lo
    bound = np.log(np.maximum(sm / 2.0, lo)) + np.sum(
        np.log(np.maximum(_rp(so, mu_top[:, None]), 1e-300)), axis=1) - logp
    rows = np.nonzero(valid_rows & (bound >= 0.0))[0]
    if rows.size == 0:
        return out
    sr, sor = sm[rows], so[rows]
    g = np.linspace(0.0, 1.0, _SCAN)[None, :]
    t = lo * np.exp(g * np.log(sr[:, None] / 2.0 / lo))   # geometric grid on [lo, s_m/2]

    def psi(tt):
        mu = tt * tt - sr[:, None] * tt if tt.ndim == 2 else tt * tt - sr * tt
        if tt.ndim == 2:
            disc = sor[:, None, :] ** 2 + 4.0 * mu[:, :, None]
            dp = 0.5 * (sor[:, None, :] + np.sqrt(np.maximum(disc, 0.0)))
            val = np.log(tt) + np.sum(np.log(np.maximum(dp, 1e-300)), axis=2) - logp
            bad = np.any(disc < 0.0, axis=2) | np.any(dp < lo, axis=2)
        else:
            disc = sor ** 2 + 4.0 * mu[:, None]
            dp = 0.5 * (sor + np.sqrt(np.maximum(disc, 0.0)))
            val = np.log(tt) + np.sum(np.log(np.maximum(dp, 1e-300)), axis=1) - logp
            bad = np.any(disc < 0.0, axis=1) | np.any(dp < lo, axis=1)
        return np.where(bad, np.nan, val)

    v = psi(t)
    sc = (v[:, :-1] * v[:, 1:] <= 0.0) & np.isfinite(v[:, :-1]) & np.isfinite(v[:, 1:])
    ri, gi = np.nonzero(sc)
    if ri.size == 0:
        return out
    a, b = t[ri, gi], t[ri, gi + 1]
    fa = v[ri, gi]
    srr, sorr = sr[ri], sor[ri]
    for _ in range(_BISECT):
        mid = 0.5 * (a + b)
        mu = mid * mid - srr * mid
        dp = _rp(sorr, mu[:, None])
        fm = np.log(mid) + np.sum(np.log(np.maximum(dp, 1e-300)), axis=1) - logp
        same = (fm * fa) > 0.0
        a = np.where(same, mid, a)
        fa = np.where(same, fm, fa)
        b = np.where(same, b, mid)
    tt = 0.5 * (a + b)
    mu = tt * tt - srr * tt
    dp = _rp(sorr, mu[:, None])
    # group roots by row: each root becomes its own candidate array
    order = np.argsort(ri, kind="stable")
    ri_s = ri[order]
    rank = np.arange(ri_s.size) - np.searchsorted(ri_s, ri_s, side="left")
    for r in range(int(rank.max()) + 1 if rank.size else 0):
        sel = order[rank == r]
        cand = np.full((n, k), np.nan)
        rr = rows[ri[sel]]
        cand[rr, m] = tt[sel]
        for j, oi in enumerate(others):
            cand[rr, oi] = dp[sel, j]
        out.append(cand)
    return out


def project_volume_sigma(sig: np.ndarray, lo: float = CLAMP) -> np.ndarray:
    """Global minimiser d of sum (d_i - sig_i)^2 s.t. prod d = 1, d_i >= lo.

    sig: (..., 3) signed singular values.  Returns d with the same shape.
    """
    sig = np.asarray(sig, dtype=np.float64)
    shp = sig.shape
    s = sig.reshape(-1, 3)
    n = s.shape[0]
    best = np.full((n, 3), np.nan)
    best_cost = np.full(n, np.inf)

    def consider(d):
        cost = np.sum((d - s) ** 2, axis=1)
        better = np.isfinite(cost) & (cost < best_cost)
        best[better] = d[better]
        best_cost[better] = cost[better]

    for clamped in ([], [0], [1], [2], [0, 1], [0, 2], [1, 2]):
        free = [i for i in range(3) if i not in clamped]
        logp = -len(clamped) * np.log(lo)
        if len(free) == 1:
            d = np.full((n, 3), lo)
            d[:, free[0]] = np.exp(logp)
            consider(d)
            continue
        sf = s[:, free]
        cands = [_all_plus(sf, logp, lo)]
        for m in range(len(free)):
            cands.extend(_one_minus(sf, m, logp, lo))
        for c in cands:
            d = np.full((n, 3), lo)
            d[:, free] = c
            consider(d)
    return best.reshape(shp)


def project_volume(F: np.ndarray) -> np.ndarray:
    """V(F) = U diag(d) W^T with d from `project_volume_sigma`."""
    U, s, W = svd_rotation_variant(F)
    d = project_volume_sigma(s)
    return (U * d[..., None, :]) @ np.swapaxes(W, -1, -2)


def project_both(F: np.ndarray):
    """(R, V, U, s, W, d) for a batch of deformation gradients."""
    U, s, W = svd_rotation_variant(F)
    d = project_volume_sigma(s)
    Wt = np.swapaxes(W, -1, -2)
    R = U @ Wt
    V = (U * d[..., None, :]) @ Wt
    return R, V, U, s, W, d
