"""The block preconditioner's design, checked on the oracle's matrix (CPU).

The CUDA path replaces the zero p_ff block (Sec. 4) by a Schur approximation
S^-1 = (mu / (gamma h^2)) I + (1/dt) L_p^-1 and solves V and D' by multigrid.
Here V and D' are solved exactly (sparse LU), so that only the block
structure and the Schur approximation act: block upper-triangular on
(v, p_ff), then the Darcy block with the C'_1 coupling, inside a right-
preconditioned GMRES to 1e-10 on the oracle's assembled system.  The
iteration counts show what each reading of the Schur block buys.
"""
import numpy as np
import pytest

import oracle as O
from paper_2108_13229_gb300 import inputs as I

sp = pytest.importorskip("scipy.sparse.linalg")


def _cell_laplacian(n, traction):
    L = np.zeros((n * n, n * n))
    for j in range(n):
        for i in range(n):
            k = j * n + i
            for ii, jj in ((i + 1, j), (i - 1, j), (i, j + 1), (i, j - 1)):
                if 0 <= ii < n and 0 <= jj < n:
                    L[k, k] += 1.0
                    L[k, jj * n + ii] -= 1.0
            if j == 0:
                L[k, k] += 2.0
            if traction and i in (0, n - 1):
                L[k, k] += 2.0
    return L


def _gmres_iterations(n, mu, K, dt, bc, gamma=0.5, side_terms=True, mass_term=True, visc_term=True,
                      darcy_first=False, maxit=60):
    o = O.Oracle(n, mu, 1.0, dt, K, bc=bc, dp=1.0, t_end=25 * dt)
    A = o.scipy_csr().tocsc()
    nv, npf = 2 * n * (n + 1), n * n
    V, B, B1 = A[:nv, :nv], A[:nv, nv:nv + npf], A[:nv, nv + npf:]
    Cp, D = A[nv + npf:, :nv], A[nv + npf:, nv + npf:]
    Vlu, Dlu = sp.splu(V.tocsc()), sp.splu(D.tocsc())
    Linv = np.linalg.inv(_cell_laplacian(n, bc != 0 and side_terms))
    h = 1.0 / n

    def prec(r):
        rv, rp, rm = r[:nv], r[nv:nv + npf], r[nv + npf:]
        zp = ((mu / (gamma * h * h)) * rp if visc_term else 0.0) + ((1.0 / dt) * (Linv @ rp) if mass_term else 0.0)
        if darcy_first:  # D' first, its result in the velocity block through B'_1
            zm = Dlu.solve(rm)
            return np.concatenate([Vlu.solve(rv - B @ zp - B1 @ zm), zp, zm])
        zv = Vlu.solve(rv - B @ zp)
        return np.concatenate([zv, zp, Dlu.solve(rm - Cp @ zv)])

    b = o.rhs(np.zeros(o.ndof), dt)
    nb = np.linalg.norm(b)
    Q, Z = [b / nb], []
    H = np.zeros((maxit + 1, maxit))
    for k in range(maxit):
        Z.append(prec(Q[k]))
        w = A @ Z[k]
        for i in range(k + 1):
            H[i, k] = Q[i] @ w
            w = w - H[i, k] * Q[i]
        H[k + 1, k] = np.linalg.norm(w)
        Q.append(w / H[k + 1, k])
        e1 = np.zeros(k + 2)
        e1[0] = nb
        y = np.linalg.lstsq(H[:k + 2, :k + 1], e1, rcond=None)[0]
        if np.linalg.norm(b - A @ (np.array(Z).T @ y)) <= 1e-10 * nb:
            return k + 1
    return maxit + 1


def test_schur_side_terms_with_traction_sides():
    # the pressure-driven problem (Sec. 5) on the log-normal workload's
    # parameters at 32^2: the side terms of L_p (the half-volume side faces)
    # cut the iterations from 27 to 11; on the Dirichlet-sided problem the
    # same block structure needs 9
    n = 32
    K = I.lognormal_K(n, -4.0, 1.0, 16.0, seed=0)
    with_sides = _gmres_iterations(n, 1e-3, K, 0.05, 2)
    without = _gmres_iterations(n, 1e-3, K, 0.05, 2, side_terms=False)
    assert with_sides <= 12 and without >= 2 * with_sides, (with_sides, without)
    assert _gmres_iterations(n, 1e-3, K, 0.05, 0) <= 10


def test_schur_terms_each_matter():
    # the log-normal workload (mu = 1e-3, dt = 0.05) at 32^2, where the mass
    # h^2/dt ~ 2e-2 outweighs mu = 1e-3 on the velocity diagonal: 9 iterations
    # with both halves of S^-1, 11 with the mass half alone, more than 60 with
    # the viscous half alone; gamma = 1/2 (the full-stress value) beats 1 and 1/4
    n = 32
    K = I.lognormal_K(n, -4.0, 1.0, 16.0, seed=0)
    both = _gmres_iterations(n, 1e-3, K, 0.05, 0)
    assert both <= 10
    assert _gmres_iterations(n, 1e-3, K, 0.05, 0, visc_term=False) > both
    assert _gmres_iterations(n, 1e-3, K, 0.05, 0, mass_term=False) > 60
    assert _gmres_iterations(n, 1e-3, K, 0.05, 0, gamma=1.0) > both
    assert _gmres_iterations(n, 1e-3, K, 0.05, 0, gamma=0.25) > both


def test_quasi_steady_paper_parameters():
    # the paper's parameters (K = 1e-6, dt = 2e5 s, mu = 1e-3): only the
    # viscous half of S^-1 acts, and the steady Schur spectrum (0.09-0.68
    # h^2/mu) leaves 23-27 iterations from a zero guess in either block order,
    # against 9-11 on the log-normal workload
    n = 32
    K = np.full((n, n), 1e-6)
    for bc in (0, 2):
        a = _gmres_iterations(n, 1e-3, K, 2e5, bc)
        b = _gmres_iterations(n, 1e-3, K, 2e5, bc, darcy_first=True)
        assert 20 <= a <= 30 and abs(a - b) <= 2, (bc, a, b)
