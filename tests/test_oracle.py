"""Pins of the FP64 oracle against things other than itself (CPU only).

* the manufactured solution, re-derived symbolically from its stream function
  and the PDE (Eqs. (1)-(7)) with sympy;
* Table 1 (Sec. 1): DoF counts exactly, matrix entries per DoF;
* brute force: the banded LU against numpy's dense LAPACK solve;
* structure: S*A symmetric (S = -1 on the pressure rows), identity
  Dirichlet rows, B * const = 0 away from Gamma, Darcy row sums;
* invariants of a solution: discrete divergence, global mass balance through
  Gamma (Eq. (7)) on both sides;
* second-order convergence to the manufactured solution, and loss of it when
  a coupling parameter is planted inconsistently;
* the Schur complement of the (v, p_ff) block at its viscous and mass limits,
  the two terms of the preconditioner's Schur block;
* definiteness of the viscous and Darcy blocks, the half-volume mass rows, and
  decay of the kinetic energy without data.
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_2108_13229_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _table1():
    rows = []
    with open(os.path.join(GOLDEN, "table1.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                n, dof, dens = line.split()
                rows.append((int(n), int(dof), float(dens)))
    return rows


# ---------------------------------------------------------------------------
# manufactured solution
# ---------------------------------------------------------------------------
def test_mms_symbolic():
    sp = pytest.importorskip("sympy")
    x, y, t, mu = sp.symbols("x y t mu", real=True)
    A = sp.pi ** 2 + 2
    phi = 1 + A * (y - 1) + (y - 1) ** 2
    psi = sp.sin(sp.pi * x) * phi
    s = 1 + t
    u = sp.diff(psi, y) * s
    v = -sp.diff(psi, x) * s
    ppm = sp.cos(sp.pi * x) * sp.exp(sp.pi * (y - 1)) * s
    # Eq. (5) on y = 1 fixes p_ff (taken constant in y): p - 2 mu dv/dy = p_pm
    pff = sp.simplify((ppm + 2 * mu * sp.diff(v, y)).subs(y, 1))
    # Eq. (2) and Darcy (Eqs. (3), (4) with K = mu = 1): div v = 0, lap p_pm = 0
    assert sp.simplify(sp.diff(u, x) + sp.diff(v, y)) == 0
    assert sp.simplify(sp.diff(ppm, x, 2) + sp.diff(ppm, y, 2)) == 0
    # Eq. (6) with K = alpha = 1, n = (0,-1), t = (1,0): u = du/dy + dv/dx on y = 1
    assert sp.simplify((u - (sp.diff(u, y) + sp.diff(v, x))).subs(y, 1)) == 0
    # Eq. (7) with K = mu = 1: v_ff(y=1) = -dp_pm/dy(y=1)
    assert sp.simplify((v + sp.diff(ppm, y)).subs(y, 1)) == 0
    # no flow through the pm sides
    assert sp.simplify(sp.diff(ppm, x).subs(x, 0)) == 0
    assert sp.simplify(sp.diff(ppm, x).subs(x, 1)) == 0
    # forcing of Eq. (1) from the full symmetric stress (rho = 1)
    txx, tyy = 2 * mu * sp.diff(u, x), 2 * mu * sp.diff(v, y)
    txy = mu * (sp.diff(u, y) + sp.diff(v, x))
    fx = sp.diff(u, t) + sp.diff(-txx + pff, x) + sp.diff(-txy, y)
    fy = sp.diff(v, t) + sp.diff(-txy, x) + sp.diff(-tyy + pff, y)
    exprs = {"u": u, "v": v, "ppm": ppm}
    exprs_mu = {"pff": pff, "fx": fx, "fy": fy}
    rng = np.random.default_rng(1)
    for name, e in exprs.items():
        f = sp.lambdify((x, y, t), e, "math")
        for _ in range(5):
            px, py, pt = rng.uniform(0, 1), rng.uniform(0, 2), rng.uniform(0, 2)
            assert O.mms(name, px, py, pt) == pytest.approx(f(px, py, pt), rel=1e-13, abs=1e-13)
    for name, e in exprs_mu.items():
        f = sp.lambdify((x, y, t, mu), e, "math")
        for m in (1.0, 1e-3):
            for _ in range(5):
                px, py, pt = rng.uniform(0, 1), rng.uniform(0, 2), rng.uniform(0, 2)
                assert O.mms(name, px, py, pt, m) == pytest.approx(f(px, py, pt, m), rel=1e-12, abs=1e-12)


# ---------------------------------------------------------------------------
# Table 1
# ---------------------------------------------------------------------------
def test_table1_dof_counts():
    for n, dof, _ in _table1():
        assert O.dof_count(n) == dof
    for n, dof, _ in _table1()[:3]:
        assert O.Oracle(n, 1.0, 1.0, 0.1, I.constant_K(n)).ndof == dof


def test_table1_entries_per_dof():
    # Table 1 prints one decimal; on the two finest grids the boundary rows no
    # longer matter and the interior stencils (11-point momentum with the full
    # stress, 4-point continuity, 5-point TPFA) fix the ratio.
    for n, dof, dens in _table1():
        if n < 160:
            continue
        o = O.Oracle(n, 1.0, 1.0, 0.1, I.constant_K(n))
        assert round(o.nnz / o.ndof, 1) == dens
    # the interior-only limit (2*11 + 4 + 5)/4 = 7.75 bounds the ratio from above
    assert O.Oracle(500, 1.0, 1.0, 0.1, I.constant_K(500)).nnz / O.dof_count(500) < 7.75


def test_table1_entries_per_dof_pressure_driven():
    # the matrix of the paper's own problem (Sec. 5: pressure on the free-flow
    # sides, no slip on top) reproduces every column of Table 1's density row,
    # the coarse ones included, with the printed decimal cut off rather than
    # rounded (6x6: 6.756 -> 6.7).  Its side u faces are momentum rows of half
    # control volumes; with Dirichlet sides (the manufactured problem) they are
    # identity rows and the small grids fall short (6x6: 6.04).
    for n, dof, dens in _table1():
        o = O.Oracle(n, 1.0, 1.0, 0.1, I.constant_K(n), bc=2)
        assert o.ndof == dof
        assert int(10.0 * o.nnz / o.ndof) == round(10.0 * dens), (n, o.nnz / o.ndof, dens)
    o = O.Oracle(6, 1.0, 1.0, 0.1, I.constant_K(6), bc=0)
    assert int(10.0 * o.nnz / o.ndof) < 67


# ---------------------------------------------------------------------------
# brute force: banded LU vs dense LAPACK
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n", [4, 5, 8])
def test_banded_lu_vs_dense(n):
    K = I.lognormal_K(n, -4.0, 1.5, 2.0, seed=n)
    o = O.Oracle(n, 1e-3, 0.7, 0.05, K)
    A = o.scipy_csr().toarray()
    rng = np.random.default_rng(n)
    b = rng.standard_normal(o.ndof)
    x_band = o.solve(b)
    x_dense = np.linalg.solve(A, b)
    assert np.linalg.norm(x_band - x_dense) <= 1e-10 * np.linalg.norm(x_dense)
    assert np.linalg.norm(A @ x_band - b) <= 1e-12 * np.linalg.norm(b) * max(1.0, np.abs(A).max())
    kl, ku = o.bandwidth()
    assert kl <= 3 * n + 2 and ku <= 3 * n + 2


# ---------------------------------------------------------------------------
# structure of A (Eq. (9))
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n", [5, 8])
def test_structure(n):
    K = I.lognormal_K(n, -4.0, 1.0, 3.0, seed=3)
    mu = 1e-3
    o = O.Oracle(n, mu, 1.3, 0.05, K)
    A = o.scipy_csr().toarray()
    off = O.offsets(n)
    S = np.ones(o.ndof)
    S[off["p_ff"]:] = -1.0
    SA = S[:, None] * A
    # symmetric saddle-point form: V = V^T, C = -B^T, C'_1 = -B'_1^T, D' = D'^T
    assert np.abs(SA - SA.T).max() <= 1e-14 * np.abs(A).max()
    # Dirichlet velocity faces: identity rows, eliminated from every other row
    dirichlet = []
    for j in range(n):
        dirichlet += [off["u"] + j * (n + 1), off["u"] + j * (n + 1) + n]
    dirichlet += [off["v"] + n * n + i for i in range(n)]
    for k in dirichlet:
        e = np.zeros(o.ndof)
        e[k] = 1.0
        assert np.array_equal(A[k], e) and np.array_equal(A[:, k], e)
    # continuity rows have no diagonal; no pressure-pressure coupling in ff
    assert np.all(A[off["p_ff"]:off["p_pm"], off["p_ff"]:off["p_pm"]] == 0)
    # gradient of a constant ff pressure vanishes except on the v_Gamma rows
    one = np.zeros(o.ndof)
    one[off["p_ff"]:off["p_pm"]] = 1.0
    y = A @ one
    vg = slice(off["v"], off["v"] + n)
    assert np.allclose(y[vg], 1.0 / n, rtol=1e-14)
    y[vg] = 0.0
    assert np.abs(y).max() == 0.0
    # Darcy row sums: fluxes between cells cancel, only the Dirichlet bottom remains
    onep = np.zeros(o.ndof)
    onep[off["p_pm"]:] = 1.0
    yp = (A @ onep)[off["p_pm"]:].reshape(n, n)
    assert np.allclose(yp[0], 2.0 * K[0] / mu, rtol=1e-13)
    assert np.abs(yp[1:]).max() <= 1e-12 * np.abs(yp[0]).max()


# ---------------------------------------------------------------------------
# invariants of a solution
# ---------------------------------------------------------------------------
def test_divergence_and_interface_mass_balance():
    n, mu = 16, 1e-3
    K = I.lognormal_K(n, -4.0, 1.0, 4.0, seed=7)
    o = O.Oracle(n, mu, 1.0, 0.05, K)
    x0 = O.exact(n, 0.0, mu)
    x = o.run(x0, 0.0, 3)
    f = O.split(x, n)
    h = 1.0 / n
    u, v, ppm = f["u"], f["v"], f["p_pm"]
    div = h * (u[:, 1:] - u[:, :-1] + v[1:, :] - v[:-1, :])
    assert np.abs(div).max() <= 1e-12 * h * np.abs(u).max()
    # flux into the Darcy domain through Gamma (Eq. (7)) = flux leaving ff through Gamma
    #   ff side: h*sum(v_Gamma) = h*sum(u_right - u_left) + h*sum(v_top)
    q_gamma = h * v[0].sum()
    q_ff = h * (u[:, n] - u[:, 0]).sum() + h * v[n].sum()
    assert abs(q_gamma - q_ff) <= 1e-12 * h * np.abs(v).sum()
    #   pm side: what enters through Gamma leaves through the Dirichlet bottom
    t_end = 3 * 0.05
    g = np.array([O.mms("ppm", (i + 0.5) * h, 0.0, t_end) for i in range(n)])
    q_bottom = (2.0 * K[0] / mu * (ppm[0] - g)).sum()
    assert abs(q_gamma + q_bottom) <= 1e-10 * abs(q_bottom) + 1e-13


# ---------------------------------------------------------------------------
# convergence to the manufactured solution
# ---------------------------------------------------------------------------
def _mms_errors(n, alpha=1.0, kval=1.0, steps=10, dt=0.1):
    o = O.Oracle(n, 1.0, alpha, dt, I.constant_K(n, kval))
    x = o.run(O.exact(n, 0.0, 1.0), 0.0, steps)
    xe = O.exact(n, steps * dt, 1.0)
    h = 1.0 / n
    fs, fe = O.split(x, n), O.split(xe, n)
    return {k: float(np.sqrt(h * h * np.sum((fs[k] - fe[k]) ** 2))) for k in fs}


def test_mms_second_order():
    ns = [16, 32, 64, 128]
    errs = [_mms_errors(n) for n in ns]
    orders = [{k: np.log2(a[k] / b[k]) for k in a} for a, b in zip(errs, errs[1:])]
    for od in orders:
        for k in ("u", "v", "p_pm"):
            assert od[k] >= 1.9, (k, orders)
    # the ff pressure carries a first-order error in the two top corner cells;
    # its L2 order rises towards two
    pf = [od["p_ff"] for od in orders]
    assert pf[0] >= 1.5 and pf[-1] >= 1.8 and pf[0] < pf[1] < pf[2], orders


@pytest.mark.parametrize("alpha,kval", [(2.0, 1.0), (1.0, 2.0)])
def test_mms_detects_planted_inconsistency(alpha, kval):
    # the manufactured solution needs alpha_BJ = 1 and K = mu = 1; planting
    # another value in the oracle must stop convergence
    e1, e2 = _mms_errors(32, alpha, kval), _mms_errors(64, alpha, kval)
    assert max(np.log2(e1[k] / e2[k]) for k in e1) < 1.0


# ---------------------------------------------------------------------------
# traction free-flow sides (bc 1: manufactured data; bc 2: the paper's
# pressure-driven problem)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("bc", [1, 2])
def test_traction_sides_structure(bc):
    # the half-control-volume rows of the side u faces keep the symmetric
    # saddle-point form (V = V^T, C = -B^T); no identity rows remain on the sides
    n = 6
    K = I.lognormal_K(n, -4.0, 1.0, 3.0, seed=4)
    o = O.Oracle(n, 1e-3, 0.8, 0.05, K, bc=bc)
    A = o.scipy_csr().toarray()
    off = O.offsets(n)
    S = np.ones(o.ndof)
    S[off["p_ff"]:] = -1.0
    SA = S[:, None] * A
    assert np.abs(SA - SA.T).max() <= 1e-14 * np.abs(A).max()
    for j in range(n):
        for i in (0, n):
            k = off["u"] + j * (n + 1) + i
            assert np.count_nonzero(A[k]) >= 5  # a momentum row, not an identity
    # the same DoF count (Table 1)
    assert o.ndof == 4 * n * n + 2 * n
    # the gradient of a constant ff pressure now also acts on the side faces
    one = np.zeros(o.ndof)
    one[off["p_ff"]:off["p_pm"]] = 1.0
    y = (A @ one)[off["u"]:off["v"]].reshape(n, n + 1)
    assert np.allclose(y[:, 0], 1.0 / n) and np.allclose(y[:, n], -1.0 / n)
    assert np.abs(y[:, 1:n]).max() == 0.0


def test_traction_sides_second_order():
    # manufactured solution with traction sides (P_b = p - 2 mu du/dx, V_b = v)
    def errs(n, steps=10, dt=0.1):
        o = O.Oracle(n, 1.0, 1.0, dt, I.constant_K(n), bc=1)
        x = o.run(O.exact(n, 0.0, 1.0), 0.0, steps)
        xe = O.exact(n, steps * dt, 1.0)
        h = 1.0 / n
        fs, fe = O.split(x, n), O.split(xe, n)
        return {k: float(np.sqrt(h * h * np.sum((fs[k] - fe[k]) ** 2))) for k in fs}
    e = [errs(n) for n in (16, 32, 64, 128)]
    orders = [{k: np.log2(a[k] / b[k]) for k in a} for a, b in zip(e, e[1:])]
    for k in ("u", "v", "p_pm", "p_ff"):
        assert orders[-1][k] >= 1.8, (k, orders)


def test_inflow_pressure_half_cosine():
    assert O.p_in(2.0, 10.0, 0.0) == 0.0
    assert abs(O.p_in(2.0, 10.0, 5.0) - 1.0) <= 1e-15
    assert abs(O.p_in(2.0, 10.0, 10.0) - 2.0) <= 1e-15
    assert O.p_in(2.0, 10.0, 30.0) == O.p_in(2.0, 10.0, 10.0)
    assert O.p_in(2.0, 10.0, 2.5) < O.p_in(2.0, 10.0, 7.5)


def test_pressure_driven_problem_mass_balance():
    # the paper's problem: flow enters on the left, leaves on the right and
    # through the porous medium; every cell conserves mass, the interface flux
    # is the same on both sides, and the pm passes it on to its bottom
    n, mu, dt, t_end = 16, 1e-3, 0.2, 2.0
    K = I.lognormal_K(n, -4.0, 1.0, 4.0, seed=5)
    o = O.Oracle(n, mu, 1.0, dt, K, bc=2, dp=1.0, t_end=t_end)
    x = o.run(np.zeros(o.ndof), 0.0, 5)
    f = O.split(x, n)
    h = 1.0 / n
    u, v, ppm = f["u"], f["v"], f["p_pm"]
    div = h * (u[:, 1:] - u[:, :-1] + v[1:, :] - v[:-1, :])
    assert np.abs(div).max() <= 1e-12 * h * np.abs(u).max()
    assert np.abs(v[n]).max() == 0.0  # no slip on the top
    q_in, q_out = h * u[:, 0].sum(), h * u[:, n].sum()
    q_gamma = -h * v[0].sum()  # downward into the porous medium
    assert q_in > 0 and q_out > 0 and q_gamma > 0
    assert abs(q_in - q_out - q_gamma) <= 1e-12 * q_in
    q_bottom = (2.0 * K[0] / mu * ppm[0]).sum()  # out through p = 0 at y = 0
    assert abs(q_gamma - q_bottom) <= 1e-10 * q_gamma
    # with the pressure drop still rising the flow accelerates
    x1 = o.run(x, 5 * dt, 1)
    assert h * O.split(x1, n)["u"][:, 0].sum() > q_in


# ---------------------------------------------------------------------------
# the Schur complement of the (v, p_ff) block at its two limits: the readings
# the Cahouet-Chabard block of the preconditioner rests on (Sec. 4 replaces
# the zero block; its scale is not printed)
# ---------------------------------------------------------------------------
def _stokes_blocks(n, mu, dt, K, bc=0):
    A = O.Oracle(n, mu, 1.0, dt, K, bc=bc).scipy_csr().toarray()
    nu = n * (n + 1)
    vel, pff = np.arange(2 * nu), np.arange(2 * nu, 2 * nu + n * n)
    return A[np.ix_(vel, vel)], A[np.ix_(vel, pff)], A[np.ix_(pff, vel)]


def _cell_laplacian_interface2(n, traction=False):
    # 5-point cell Laplacian with unit transmissibilities, no flow through the
    # free-flow walls, and 2 on the diagonal of the cells above the interface
    # (their v_Gamma face carries half a control volume of mass); with traction
    # sides also 2 on the cells beside them (half-volume side u faces)
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


@pytest.mark.parametrize("n", [8, 12])
@pytest.mark.parametrize("bc", [0, 2])
def test_schur_viscous_limit_is_half(n, bc):
    # dt -> infinity: S = -C V^-1 B of the full-stress operator equals
    # h^2 / (2 mu) exactly on the (n-2)^2 interior pressure modes (n (n-2) with
    # traction sides), the rest of its spectrum lies below h^2 / mu; so
    # S^-1 ~ mu / (gamma h^2) with gamma = 1/2 (a Laplacian momentum operator
    # would give gamma = 1)
    h = 1.0 / n
    for mu, K in [(1.0, np.ones((n, n))), (1e-3, I.lognormal_K(n, -4.0, 1.0, 4.0, seed=n))]:
        V, B, C = _stokes_blocks(n, mu, 1e12, K, bc)
        ev = np.sort(np.linalg.eigvals(-C @ np.linalg.solve(V, B)).real) * mu / h**2
        assert np.sum(np.abs(ev - 0.5) < 1e-8) == (n - 2) * (n - 2 if bc == 0 else n), (mu, ev)
        assert 0.05 < ev[0] and ev[-1] < 1.0


@pytest.mark.parametrize("n", [8, 12])
@pytest.mark.parametrize("bc", [0, 1, 2])
def test_schur_mass_limit_is_cell_laplacian(n, bc):
    # dt -> 0: V -> (h^2/dt) M with M = 1, and 1/2 on the half-volume faces,
    # so S -> dt B^T M^-1 B / h^2 = dt L_p, L_p the cell Laplacian with 2 on
    # the interface cells (and on the side cells with traction sides); the gap
    # closes linearly in dt, and without the side terms it stays O(1)
    K = I.lognormal_K(n, -4.0, 1.0, 4.0, seed=n)
    L = _cell_laplacian_interface2(n, traction=bc != 0)
    gaps = []
    for dt in (1e-6, 1e-8):
        V, B, C = _stokes_blocks(n, 1e-3, dt, K, bc)
        S = -C @ np.linalg.solve(V, B)
        gaps.append(np.linalg.norm(S - dt * L) / np.linalg.norm(dt * L))
    assert gaps[0] < 1e-5 and gaps[1] < 1e-7
    assert 50 < gaps[0] / gaps[1] < 200
    if bc != 0:
        L0 = _cell_laplacian_interface2(n)
        assert np.linalg.norm(S - 1e-8 * L0) / np.linalg.norm(1e-8 * L0) > 0.1


# ---------------------------------------------------------------------------
# definiteness and energy: what the symmetry pin cannot see (a sign slip in a
# symmetric term, e.g. the wall shear or the eliminated BJS slip, keeps S*A
# symmetric but makes the viscous block indefinite)
# ---------------------------------------------------------------------------
def _mass_weights(n, K, bc):
    # the implicit-Euler mass of each velocity row, h^2 m_k / dt, read off the
    # diagonal at two time steps: 1 on full control volumes, 1/2 on half ones,
    # 0 on identity (Dirichlet) rows
    h, nv = 1.0 / n, 2 * n * (n + 1)
    A1 = O.Oracle(n, 1e-3, 1.0, 0.1, K, bc=bc).scipy_csr().toarray()
    A2 = O.Oracle(n, 1e-3, 1.0, 0.2, K, bc=bc).scipy_csr().toarray()
    m = (np.diag(A1)[:nv] - np.diag(A2)[:nv]) / (h * h * (1 / 0.1 - 1 / 0.2))
    return A1, m


@pytest.mark.parametrize("bc", [0, 1, 2])
def test_viscous_and_darcy_blocks_are_spd(bc):
    n = 8
    h, nv = 1.0 / n, 2 * n * (n + 1)
    K = I.lognormal_K(n, -4.0, 1.0, 4.0, seed=3)
    A, m = _mass_weights(n, K, bc)
    # half control volumes: the v_Gamma faces, and the side u faces with traction sides
    assert np.sum(np.isclose(m, 0.5)) == (n if bc == 0 else 3 * n)
    assert np.sum(np.isclose(m, 0.0)) == (3 * n if bc == 0 else n)
    assert np.all(np.isclose(m, 0.0) | np.isclose(m, 0.5) | np.isclose(m, 1.0))
    free = ~np.isclose(m, 0.0)
    Vs = (A[:nv, :nv] - np.diag(h * h * m / 0.1))[np.ix_(free, free)]
    assert np.abs(Vs - Vs.T).max() <= 1e-15 * np.abs(Vs).max()
    # positive definite on the scale of mu = 1e-3 (smallest eigenvalue 0.1-0.3 mu here)
    assert np.linalg.eigvalsh(Vs)[0] / 1e-3 > 0.05
    D = A[nv + n * n:, nv + n * n:]
    assert np.abs(D - D.T).max() == 0.0 and np.linalg.eigvalsh(D)[0] > 0


def test_kinetic_energy_decays_without_data():
    # the pressure-driven problem with zero pressure drop has no data: from any
    # velocity, the M-norm of the velocity must not grow over a backward-Euler
    # step (the pressure terms cancel, the viscous and Darcy blocks dissipate)
    n = 8
    nv = 2 * n * (n + 1)
    K = I.lognormal_K(n, -4.0, 1.0, 4.0, seed=4)
    _, m = _mass_weights(n, K, 2)
    o = O.Oracle(n, 1e-3, 1.0, 0.1, K, bc=2, dp=0.0)
    x = np.random.default_rng(5).standard_normal(o.ndof)
    x[:nv][np.isclose(m, 0.0)] = 0.0
    E = [float(np.sum(m * x[:nv] ** 2))]
    x = o.run(x, 0.0, 1)
    for s in range(1, 8):
        E.append(float(np.sum(m * x[:nv] ** 2)))
        x = o.run(x, 0.1 * s, 1)
    assert all(b < a for a, b in zip(E, E[1:])), E


def test_paper_parameters_linear_and_quasi_steady():
    # the physical parameters of Sec. 5 (K = 1e-6 m^2, alpha_BJ = 1, dt = 2e5 s,
    # t_end = 50e5 s, a half-cosine pressure difference of at most 1e-9 Pa; the
    # viscosity, not printed, is taken as water's 1e-3 Pa s) on 16^2 cells:
    # * the solution is linear in the pressure difference, so the build's
    #   unit amplitude gives the same fields scaled by 1e9;
    # * the mass term h^2/dt is some 1e-5 of the viscous one: every step is
    #   the steady solution of its own inflow pressure, to 5e-4 at the first
    #   step and closer at every later one, 2e-6 at t_end, where the pressure
    #   stops rising
    n, mu, dt, t_end, dp = 16, 1e-3, 2e5, 50e5, 1e-9
    K = np.full((n, n), 1e-6)
    o = O.Oracle(n, mu, 1.0, dt, K, bc=2, dp=dp, t_end=t_end)
    o1 = O.Oracle(n, mu, 1.0, dt, K, bc=2, dp=1.0, t_end=t_end)
    steady = O.Oracle(n, mu, 1.0, 1e20, K, bc=2, dp=dp, t_end=t_end)
    x, x1 = np.zeros(o.ndof), np.zeros(o.ndof)
    lag = []
    for s in range(25):
        x, x1 = o.run(x, s * dt, 1), o1.run(x1, s * dt, 1)
        assert np.linalg.norm(1e-9 * x1 - x) <= 1e-14 * np.linalg.norm(x)
        xs = steady.solve(steady.rhs(np.zeros(o.ndof), (s + 1) * dt))
        f, fs = O.split(x, n), O.split(xs, n)
        lag.append(max(np.linalg.norm(f[k] - fs[k]) / np.linalg.norm(fs[k]) for k in f))
    assert lag[0] < 1e-3 and all(b < a for a, b in zip(lag, lag[1:])) and lag[-1] < 3e-6, lag
    h = 1.0 / n
    q_in, q_out, q_gamma = h * f["u"][:, 0].sum(), h * f["u"][:, n].sum(), -h * f["v"][0].sum()
    assert q_in > 0 and abs(q_in - q_out - q_gamma) <= 1e-12 * q_in


# ---------------------------------------------------------------------------
# the product and residual routines the GPU tests use as checkers
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n", [4, 16, 128])
@pytest.mark.parametrize("bc", [0, 2])
def test_apply_and_residual_match_scipy(n, bc):
    # or_apply and or_residual walk the CSR themselves; scipy's sparse product
    # over the exported arrays is an independent walk.  A wrong row range,
    # a skipped last row or a norm of the wrong vector fails here.
    rng = np.random.default_rng(100 + n + bc)
    K = I.lognormal_K(n, -4.0, 1.0, 4.0, seed=n + bc)
    o = O.Oracle(n, 1e-3, 1.3, 0.05, K, bc=bc, dp=1.0, t_end=1.0)
    A = o.scipy_csr()
    assert A.shape == (O.dof_count(n),) * 2
    x = rng.standard_normal(o.ndof)
    b = rng.standard_normal(o.ndof)
    Ax = A @ x
    y = o.apply(x)
    assert np.linalg.norm(y - Ax) <= 1e-14 * np.linalg.norm(Ax)
    r, nrm = o.residual(x, b)
    rr = b - Ax
    assert np.linalg.norm(r - rr) <= 1e-14 * np.linalg.norm(rr)
    assert abs(nrm - np.linalg.norm(rr)) <= 1e-14 * np.linalg.norm(rr)
    # the norm is that of b - A x, not of b or of A x
    assert abs(nrm - np.linalg.norm(b)) > 1e-3 * np.linalg.norm(b)
    # a solved system has (almost) no residual
    o2 = O.Oracle(n, 1e-3, 1.3, 0.05, K, bc=bc) if n <= 16 else None
    if o2 is not None:
        xs = o2.solve(b)
        _, nrm2 = o2.residual(xs, b)
        assert nrm2 <= 1e-10 * np.linalg.norm(b)


def test_interface_row_written_out():
    # The v_Gamma rows at n = 4, written from the half-control-volume balance
    # of Eq. (5) over [x_i, x_{i+1}] x [1, 1 + h/2]:
    #   mass      h^2/(2 dt) v_G
    #   top       h p_ff(i,0) - 2 mu (v(i,1) - v_G)            (normal stress at the cell centre)
    #   bottom    -h p_G,  p_G = p_pm(i,n-1) - mu h/(2 K) v_G    (TPFA reconstruction, Eq. (7))
    #   sides     -(h/2) tau(x_{i+1}) + (h/2) tau(x_i),  tau at a Gamma corner from the
    #             eliminated BJS slip of Eq. (6): tau = w (2 u(.,0) + dv), w = mu/(h + 2 beta),
    #             beta = mean sqrt(K) of the two cells below / alpha, dv the jump of v_G;
    #             at the wall x = 0: tau = mu v_G / (h/2) (wall velocity is data).
    n, mu, alpha, dt = 4, 0.7, 1.9, 0.3
    h = 1.0 / n
    K = np.exp(np.random.default_rng(3).normal(-1.0, 0.8, (n, n)))
    o = O.Oracle(n, mu, alpha, dt, K.ravel())
    A = o.scipy_csr().tocsr()
    off = O.offsets(n)

    def iu(i, j):
        return off["u"] + j * (n + 1) + i

    def iv(i, j):
        return off["v"] + j * n + i

    def ipf(i, j):
        return off["p_ff"] + j * n + i

    def ipm(i, j):
        return off["p_pm"] + j * n + i

    def w(i):  # BJS shear coefficient of the interface corner at x_i, 1 <= i <= n-1
        beta = 0.5 * (np.sqrt(K[n - 1, i - 1]) + np.sqrt(K[n - 1, i])) / alpha
        return mu / (h + 2 * beta)

    def row(r):
        a = A.getrow(r)
        return dict(zip(a.indices.tolist(), a.data.tolist()))

    # interior face i = 1 (both corners on Gamma)
    i = 1
    want = {
        iv(i, 0): h * h / (2 * dt) + 2 * mu + mu * h * h / (2 * K[n - 1, i]) + 0.5 * h * (w(i) + w(i + 1)),
        iv(i, 1): -2 * mu,
        ipf(i, 0): h,
        ipm(i, n - 1): -h,
        iu(i, 0): h * w(i),
        iu(i + 1, 0): -h * w(i + 1),
        iv(i - 1, 0): -0.5 * h * w(i),
        iv(i + 1, 0): -0.5 * h * w(i + 1),
    }
    got = row(iv(i, 0))
    assert set(got) == set(want)
    for k in want:
        assert abs(got[k] - want[k]) <= 1e-15 * max(1.0, abs(want[k])), (k, got[k], want[k])
    # wall face i = 0: the left corner is the Dirichlet side at half distance
    i = 0
    want = {
        iv(i, 0): h * h / (2 * dt) + 2 * mu + mu * h * h / (2 * K[n - 1, i]) + mu + 0.5 * h * w(i + 1),
        iv(i, 1): -2 * mu,
        ipf(i, 0): h,
        ipm(i, n - 1): -h,
        iu(i + 1, 0): -h * w(i + 1),
        iv(i + 1, 0): -0.5 * h * w(i + 1),
    }
    got = row(iv(i, 0))
    assert set(got) == set(want)
    for k in want:
        assert abs(got[k] - want[k]) <= 1e-15 * max(1.0, abs(want[k])), (k, got[k], want[k])
    # the Darcy cell below face 1 sees h v_G (Eq. (7), block C'_1)
    assert abs(row(ipm(1, n - 1))[iv(1, 0)] - h) <= 1e-16
