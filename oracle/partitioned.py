"""Partitioned Dirichlet-Neumann coupling with IQN-ILS post-processing (Sec. 3), FP64 CPU oracle.

TEST INFRASTRUCTURE ONLY: the tests use this module; the product library
never imports it.  It works on the oracle's assembled CSR matrix of Eq. (9)
(``oracle.Oracle``) with direct sparse subdomain solves (scipy's SuperLU):
no blocking, no inexact solver, so the coupling iteration can be checked
against the monolithic solution directly.

The two subdomain solvers of Sec. 3, on the discretisation of the monolithic
system (the interface rows of Eqs. (5)-(7)), exchange the interface normal
velocity and the porous-medium pressure at the interface:

* S_pm takes the normal velocity v_Gamma through the interface as flux data
  (the outflow h v_Gamma of the top Darcy cells, Eq. (7)) and solves the
  Darcy rows for p_pm; it passes on the pressure of the cells below Gamma,
  p_top (Eq. (5) reconstructs the interface pressure from it and v_Gamma).
* S_ff takes p_top as data of the normal-stress balance of the v_Gamma half
  control volumes (Eq. (5), block B'_1) and solves the free-flow rows for
  u, v (v_Gamma included, BJS slip of Eq. (6) inside) and p_ff; it passes on
  the new interface velocity v~ = v_Gamma.

With traction free-flow sides (the paper's channel, bc 1 and 2) the order of
Sec. 3 is also available (order="paper"): S_ff takes v_Gamma as Dirichlet
data (identity v_Gamma rows) and returns the interface pressure p_Gamma, the
normal stress that balances the v_Gamma half control volumes (their row of
Eq. (5) with the TPFA reconstruction term mu h^2/(2K) v_Gamma and the -h p_pm
coupling left out, divided by h); S_pm takes p_Gamma as Dirichlet pressure on
its top boundary over the half cell below Gamma (transmissibility 2K/mu) and
returns the Darcy velocity v~ = (2K/(mu h)) (p_c - p_Gamma) through Gamma.

R(v) = S_ff(S_pm(v)) - v (order "pm") or S_pm(S_ff(v)) - v (order "paper") is
the fixed-point residual of Sec. 3.  Each
subdomain solve is the monolithic system's own rows with the other
subdomain's unknowns held fixed, so at a root of R both subdomain states
together satisfy every row of Eq. (9): the coupled iteration reproduces the
monolithic solution.  (Sec. 3 solves the free flow first, with the interface
velocity as its data.  That order needs a pressure boundary in the free
flow, which the paper's channel has; with the velocity prescribed on the
whole remaining free-flow boundary, as in the test problems here, the
free-flow block with a prescribed v_Gamma is singular (the pressure constant)
and the data must balance its mass, so the two solvers run in the other
order; `paper_order_ff_operator` exposes that block for the test that
shows the singularity.)

IQN-ILS (the interface quasi-Newton method with an inverse Jacobian from a
least-squares model that Sec. 3 uses as post-processing): with x~_k = H(x_k)
and r_k = x~_k - x_k, the differences dr = r_k - r_{k-1} and dx~ = x~_k -
x~_{k-1} of all earlier iterations of the time step are kept as the columns
of V and W; alpha = argmin ||V alpha + r_k||_2 and x_{k+1} = x~_k + W alpha.
The first iteration of a time step is a relaxed Picard step x_1 = x_0 +
omega0 r_0.  Stopping test of Sec. 3 on the exchanged pressure and velocity:
||p_{k+1} - p_k||_2 < eps ||p_{k+1}||_2 and ||v~_{k+1} - v_k||_2 <
eps ||v~_{k+1}||_2.
"""
from __future__ import annotations

import numpy as np

from . import Oracle, offsets


class DNOracle:
    """Subdomain solvers S_pm, S_ff and the coupled iteration for one implicit-Euler step."""

    def __init__(self, o: Oracle, K, flux_scale: float = 1.0, order: str = "pm"):
        import scipy.sparse as sp
        import scipy.sparse.linalg as spl
        n = o.n
        self.o, self.n = o, n
        self.h, self.mu = 1.0 / n, o.mu
        off = offsets(n)
        A = o.scipy_csr().tocsr()
        self.A = A
        self.nF = off["p_pm"]
        self.G = off["v"] + np.arange(n)                      # v_Gamma faces (v row 0)
        self.T = (n - 1) * n + np.arange(n)                   # pm cells below Gamma, inside the pm block
        F = slice(0, self.nF)
        P = slice(self.nF, A.shape[0])
        self.AFF, self.AFP = A[F, F].tocsc(), A[F, P].tocsr()
        self.APF, self.APP = A[P, F].tocsr(), A[P, P].tocsc()
        # flux_scale != 1 lets a test plant a wrong interface flux in S_pm
        self.flux_scale = flux_scale
        self.order = order
        if order == "paper":
            Kt = np.asarray(K, dtype=np.float64).reshape(n, n)[n - 1]
            self.rg = self.mu * self.h * self.h / (2.0 * Kt)   # reconstruction term of the v_Gamma rows
            self.Ttop = 2.0 * Kt / self.mu                      # half-cell transmissibility below Gamma
            self.Arow_G = A[self.G, :][:, F].tocsr()
            self._ff = spl.splu(self.paper_order_ff_operator().tocsc())
            app = self.APP.tocsr() + sp.diags(np.bincount(self.T, weights=self.Ttop, minlength=n * n))
            self._pm = spl.splu(app.tocsc())
        else:
            self._ff = spl.splu(self.AFF)
            self._pm = spl.splu(self.APP)

    def paper_order_ff_operator(self):
        """Free-flow rows with v_Gamma prescribed (identity rows): the first solver of Sec. 3's order."""
        M = self.AFF.tolil()
        for g in self.G:
            M.rows[g] = [g]
            M.data[g] = [1.0]
        return M.tocsr()

    # --- subdomain solvers -------------------------------------------------
    def s_pm(self, v, b):
        """Darcy rows with the interface flux h v given; returns (x_P, p_top)."""
        xF = np.zeros(self.nF)
        xF[self.G] = self.flux_scale * v
        xP = self._pm.solve(b[self.nF:] - self.APF @ xF)
        return xP, xP[self.T].copy()

    def s_ff(self, p_top, b):
        """Free-flow rows with the pm pressure below Gamma given; returns (x_F, v~)."""
        xP = np.zeros(self.A.shape[0] - self.nF)
        xP[self.T] = p_top
        xF = self._ff.solve(b[: self.nF] - self.AFP @ xP)
        return xF, xF[self.G].copy()

    # --- the order of Sec. 3 (free flow first; traction sides only) --------
    def s_ff_paper(self, v, b):
        """Free-flow solve with v_Gamma = v prescribed; returns (x_F, p_Gamma)."""
        bF = b[: self.nF].copy()
        bF[self.G] = v
        xF = self._ff.solve(bF)
        pG = (self.Arow_G @ xF - self.rg * xF[self.G] - b[self.G]) / self.h
        return xF, pG

    def s_pm_paper(self, pG, b):
        """Darcy solve with p_Gamma prescribed on top (half cell); returns (x_P, v~)."""
        bP = b[self.nF:].copy()
        bP[self.T] += self.Ttop * pG
        xP = self._pm.solve(bP)
        return xP, self.Ttop / self.h * (xP[self.T] - pG)

    def H(self, v, b):
        if self.order == "paper":
            xF, p = self.s_ff_paper(v, b)
            xP, vt = self.s_pm_paper(p, b)
            return vt, p, xF, xP
        xP, p = self.s_pm(v, b)
        xF, vt = self.s_ff(p, b)
        return vt, p, xF, xP

    # --- coupled iteration --------------------------------------------------
    def solve(self, b, v0, eps: float = 1e-10, omega0: float = 0.1, max_iter: int = 200, qmax: int = 30,
              accelerate: bool = True):
        """IQN-ILS (or, accelerate=False, relaxed Picard) iteration; returns (x, evaluations of H)."""
        v = np.asarray(v0, dtype=np.float64).copy()
        p_prev = r_prev = vt_prev = None
        Vc, Wc = [], []
        for k in range(1, max_iter + 1):
            vt, p, xF, xP = self.H(v, b)
            if p_prev is not None:
                if (np.linalg.norm(p - p_prev) < eps * np.linalg.norm(p)
                        and np.linalg.norm(vt - v) < eps * np.linalg.norm(vt)):
                    return np.concatenate([xF, xP]), k
            r = vt - v
            if r_prev is None or not accelerate:
                vn = v + omega0 * r
            else:
                Vc.append(r - r_prev)
                Wc.append(vt - vt_prev)
                if len(Vc) > qmax:
                    Vc.pop(0)
                    Wc.pop(0)
                Vm, Wm = np.stack(Vc, 1), np.stack(Wc, 1)
                alpha = np.linalg.lstsq(Vm, -r, rcond=None)[0]
                vn = vt + Wm @ alpha
            p_prev, r_prev, vt_prev = p, r, vt
            v = vn
        raise RuntimeError("coupling iteration did not converge in %d evaluations" % max_iter)
