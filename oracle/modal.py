"""FP64 oracle of the paper's own global step (Sec. 7.2 and the solver set-up
of Sec. 8): the component-mode subspace with a truncated set of fixed-interface
normal modes per domain, followed by full-space Jacobi sweeps with Chebyshev
weights.

TEST INFRASTRUCTURE ONLY: imported by tests/ (and nothing on the product
path).  It shares no code with the CUDA library.

Per domain d (internal vertices i, boundary vertices b of the domain):
  * boundary modes Psi_d = -K_ii^-1 K_ib                (Eq. cms_boundary)
  * normal modes Phi_d: eigenvectors of K_ii for its `modes` smallest
    eigenvalues, Phi^T K_ii Phi = Lambda                 (the eigenproblem after
    Eq. cms_boundary), Phi orthonormal
  * subspace x_i = Phi_d p_d + Psi_d x_b                  (Eq. global_subspace)
Galerkin projection of K x = b onto that subspace: Phi^T (K_ii Psi + K_ib) = 0,
so the reduced matrix is block diagonal, [Lambda_d ...; S], with the interface
Schur complement S = K_BB + sum_d K_bi Psi_d, and
  p_d = Lambda_d^-1 Phi_d^T b_i,
  x_b = S^-1 (b_B + sum_d Psi_d^T b_i),
  x_i = Phi_d p_d + Psi_d x_b.
The reduced result is then refined in the full space ("A-Jacobi" of the
paper's set-up: Jacobi iterations, combined in the paper two or three per GPU
pass -- the same iterates) with the Chebyshev semi-iterative weights of
Wang 2015: with rho the spectral radius of the Jacobi iteration matrix
I - D^-1 K,
  x_hat = x_k + D^-1 (b - K x_k),
  omega_1 = 1, omega_2 = 2 / (2 - rho^2), omega_{k+1} = 4 / (4 - rho^2 omega_k),
  x_{k+1} = omega_{k+1} (x_hat - x_{k-1}) + x_{k-1}.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp


def classify(n_v, tets, tet_domain, pinned):
    """Interface vertices: not pinned and touched by tets of two or more domains.
    Returns (is_interface bool[n_v], domain of each non-interface free vertex or -1)."""
    tets = np.asarray(tets, np.int64)
    tet_domain = np.asarray(tet_domain, np.int64)
    first = np.full(n_v, -1, np.int64)
    multi = np.zeros(n_v, bool)
    for t in range(tets.shape[0]):
        d = tet_domain[t]
        for v in tets[t]:
            if first[v] < 0:
                first[v] = d
            elif first[v] != d:
                multi[v] = True
    pinned = np.asarray(pinned, bool)
    iface = multi & ~pinned
    vdom = np.where(iface | pinned, -1, first)
    return iface, vdom


class ModalDD:
    """The paper's subspace global solve on the free block K_ff (scalar matrix,
    the same for x, y and z)."""

    def __init__(self, K_ff, free_ids, n_v, tets, tet_domain, n_domains, pinned, modes=20):
        K = sp.csr_matrix(K_ff)
        self.K = K
        self.n = K.shape[0]
        free_ids = np.asarray(free_ids, np.int64)
        iface, vdom = classify(n_v, tets, tet_domain, pinned)
        row_of = np.full(n_v, -1, np.int64)
        row_of[free_ids] = np.arange(free_ids.size)
        self.B = row_of[np.nonzero(iface)[0]]                          # interface rows of K_ff
        self.B.sort()
        bpos = np.full(self.n, -1, np.int64)
        bpos[self.B] = np.arange(self.B.size)
        self.domains = []
        Kd = K.tocsr()
        for d in range(n_domains):
            I = row_of[np.nonzero(vdom == d)[0]]
            I = np.sort(I[I >= 0])
            if I.size == 0:
                continue
            # the domain's boundary: interface rows coupled to its internal rows
            cols = np.unique(Kd[I].indices)
            bd = np.sort(cols[bpos[cols] >= 0])
            Kii = Kd[I][:, I].toarray()
            Kib = Kd[I][:, bd].toarray()
            lam, vec = np.linalg.eigh(Kii)                                # ascending
            r = min(modes, I.size)
            Psi = -np.linalg.solve(Kii, Kib)
            self.domains.append(dict(I=I, bd=bd, bpos=bpos[bd], Kib=Kib, Psi=Psi, lam=lam[:r], Phi=vec[:, :r]))
        nB = self.B.size
        S = Kd[self.B][:, self.B].toarray()
        for dd in self.domains:
            S[np.ix_(dd["bpos"], dd["bpos"])] += dd["Kib"].T @ dd["Psi"]
        self.S = S
        self.S_cho = sla.cho_factor(S) if nB else None
        self.Dinv = 1.0 / K.diagonal()

    # -- the reduced (subspace) solve ------------------------------------------
    def reduced_solve(self, b):
        b = np.asarray(b, np.float64)
        x = np.zeros_like(b)
        c = b[self.B].copy()
        for dd in self.domains:
            c[dd["bpos"]] += dd["Psi"].T @ b[dd["I"]]
        xb = sla.cho_solve(self.S_cho, c) if self.B.size else c
        x[self.B] = xb
        for dd in self.domains:
            p = (dd["Phi"].T @ b[dd["I"]]) / dd["lam"][:, None]
            x[dd["I"]] = dd["Phi"] @ p + dd["Psi"] @ xb[dd["bpos"]]
        return x

    # -- full-space Chebyshev-weighted Jacobi --------------------------------
    def jacobi_rho(self):
        """Spectral radius of the Jacobi iteration matrix I - D^-1 K (dense
        eigenvalues of the similar symmetric matrix I - D^-1/2 K D^-1/2)."""
        d = np.sqrt(self.Dinv)
        A = np.eye(self.n) - (d[:, None] * self.K.toarray() * d[None, :])
        return float(np.max(np.abs(np.linalg.eigvalsh(A))))

    def chebyshev_jacobi(self, b, x0, sweeps, rho):
        b = np.asarray(b, np.float64)
        x_prev = np.array(x0, np.float64)
        x = x_prev.copy()
        omega = 1.0
        for k in range(1, sweeps + 1):
            x_hat = x + self.Dinv[:, None] * (b - self.K @ x)
            if k == 1:
                omega = 1.0
            elif k == 2:
                omega = 2.0 / (2.0 - rho * rho)
            else:
                omega = 4.0 / (4.0 - rho * rho * omega)
            x_new = omega * (x_hat - x_prev) + x_prev
            x_prev, x = x, x_new
        return x

    def solve(self, b, sweeps=0, rho=None):
        x = self.reduced_solve(b)
        if sweeps > 0:
            x = self.chebyshev_jacobi(b, x, sweeps, self.jacobi_rho() if rho is None else rho)
        return x
