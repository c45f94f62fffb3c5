"""Pins of the FP64 oracle on the channel geometry of the paper's model
problem (Sec. 5 and its figure: a free flow three times as wide as the porous
medium, the interface the middle third of the channel's floor, walls beside
it), CPU only.

* the DoF count 10n^2 + 4n and the identity rows of the Dirichlet faces (the
  floor faces beside the interface among them, none on it);
* structure: S*A symmetric on the non-identity rows (S = -1 on the pressure
  rows), so the discrete operator keeps the saddle-point form of Eq. (9);
* second-order convergence to the manufactured solution continued over
  x in [-1, 2], with Dirichlet and with traction ends, and the loss of it when
  the BJS coefficient of Eq. (6) is planted inconsistently (the slip rows on
  the interface are used);
* the pressure-driven problem: per-cell mass balance, no flow through the
  walls, inflow = outflow + flux into the porous medium, that flux leaving
  through the pm bottom; and decay of the kinetic energy without data.
"""
import numpy as np
import pytest

import oracle as O
from paper_2108_13229_gb300 import inputs as I

GEO = 1


def _csr(n, bc=0, mu=1.0, alpha=1.0, dt=0.1, K=None):
    K = np.ones((n, n)) if K is None else K
    return O.Oracle(n, mu, alpha, dt, K, bc=bc, geo=GEO).scipy_csr().toarray()


def _identity_rows(A):
    return [r for r in range(A.shape[0]) if A[r, r] == 1.0 and np.count_nonzero(A[r]) == 1]


@pytest.mark.parametrize("n", [4, 6, 8])
def test_channel_dof_count_and_layout(n):
    nx = 3 * n
    assert O.dof_count(n, GEO) == 10 * n * n + 4 * n
    off = O.offsets(n, GEO)
    assert off["v"] == n * (nx + 1) and off["p_ff"] - off["v"] == nx * (n + 1)
    assert off["p_pm"] - off["p_ff"] == nx * n and off["end"] - off["p_pm"] == n * n
    x = O.exact(n, 0.0, 1.0, GEO)
    assert x.size == O.dof_count(n, GEO)
    f = O.split(x, n, GEO)
    assert f["u"].shape == (n, nx + 1) and f["v"].shape == (n + 1, nx) and f["p_ff"].shape == (n, nx)


@pytest.mark.parametrize("bc", [0, 2])
def test_channel_identity_rows(bc):
    n = 6
    nx = 3 * n
    A = _csr(n, bc)
    off = O.offsets(n, GEO)
    ident = set(_identity_rows(A))
    floor = [off["v"] + i for i in range(nx)]
    on_gamma = set(range(n, 2 * n))
    for i in range(nx):
        assert (floor[i] in ident) == (i not in on_gamma), i
    lid = {off["v"] + n * nx + i for i in range(nx)}
    assert lid <= ident
    ends = {off["u"] + j * (nx + 1) + i for j in range(n) for i in (0, nx)}
    assert (ends <= ident) == (bc == 0)
    want = len(lid) + (nx - n) + (len(ends) if bc == 0 else 0)
    assert len(ident) == want
    # an identity row's unknown enters no other row (its value is data)
    for r in ident:
        col = A[:, r].copy()
        col[r] = 0.0
        assert not np.any(col), r


@pytest.mark.parametrize("bc", [0, 1, 2])
def test_channel_saddle_point_symmetry(bc):
    n = 6
    K = I.lognormal_K(n, -1.0, 1.0, 2.0, seed=3)
    A = _csr(n, bc, mu=0.7, alpha=1.4, dt=0.3, K=K)
    off = O.offsets(n, GEO)
    S = np.ones(A.shape[0])
    S[off["p_ff"]:] = -1.0
    keep = np.setdiff1d(np.arange(A.shape[0]), _identity_rows(A))
    M = (S[:, None] * A)[np.ix_(keep, keep)]
    assert np.abs(M - M.T).max() <= 1e-14 * np.abs(M).max()
    # the coupling blocks live on the interface alone: p_pm reaches only the
    # v faces on Gamma, and v reaches the Darcy rows only there
    nx = 3 * n
    gam = [off["v"] + i for i in range(n, 2 * n)]
    pm = np.arange(off["p_pm"], off["end"])
    vel = np.arange(0, off["p_ff"])
    rows_pm_in_vel = set(np.nonzero(np.any(A[np.ix_(vel, pm)] != 0.0, axis=1))[0])
    assert rows_pm_in_vel == set(gam)
    cols = set(np.nonzero(np.any(A[np.ix_(pm, vel)] != 0.0, axis=0))[0])
    assert cols == set(gam)
    assert nx == 3 * n


def _mms_errors(n, bc=0, alpha=1.0, steps=10, dt=0.1):
    o = O.Oracle(n, 1.0, alpha, dt, I.constant_K(n, 1.0), bc=bc, geo=GEO)
    x = o.run(O.exact(n, 0.0, 1.0, GEO), 0.0, steps)
    xe = O.exact(n, steps * dt, 1.0, GEO)
    h = 1.0 / n
    fs, fe = O.split(x, n, GEO), O.split(xe, n, GEO)
    return {k: float(np.sqrt(h * h * np.sum((fs[k] - fe[k]) ** 2))) for k in fs}


@pytest.mark.parametrize("bc", [0, 1])
def test_channel_mms_second_order(bc):
    # the manufactured solution solves Eqs. (1)-(7) for every x, so its values
    # on the walls beside the interface are consistent Dirichlet data; bc 1
    # prescribes the normal stress and tangential velocity at x = -1, 2
    ns = [8, 16, 32]
    errs = [_mms_errors(n, bc) for n in ns]
    orders = [{k: np.log2(a[k] / b[k]) for k in a} for a, b in zip(errs, errs[1:])]
    for od in orders:
        for k in ("u", "p_pm"):
            assert od[k] >= 1.9, (k, orders)
        assert od["v"] >= 1.85, orders
        assert od["p_ff"] >= 1.55, orders
    assert orders[0]["p_ff"] < orders[1]["p_ff"], orders


def test_channel_mms_sees_the_slip_rows():
    # alpha_BJ = 2 is inconsistent with the manufactured solution (it needs 1):
    # the interface rows of Eq. (6) enter, so the error stops decreasing
    e16 = _mms_errors(16, alpha=2.0)
    e32 = _mms_errors(32, alpha=2.0)
    assert np.log2(e16["u"] / e32["u"]) < 1.0


def test_channel_pressure_driven_mass_balance():
    n, mu, dt, t_end = 12, 1e-3, 0.2, 2.0
    nx = 3 * n
    K = I.lognormal_K(n, -4.0, 1.0, 4.0, seed=5)
    o = O.Oracle(n, mu, 1.0, dt, K, bc=2, dp=1.0, t_end=t_end, geo=GEO)
    x = o.run(np.zeros(o.ndof), 0.0, 5)
    f = O.split(x, n, GEO)
    h = 1.0 / n
    u, v, ppm = f["u"], f["v"], f["p_pm"]
    div = h * (u[:, 1:] - u[:, :-1] + v[1:, :] - v[:-1, :])
    assert np.abs(div).max() <= 1e-12 * h * np.abs(u).max()
    assert np.abs(v[n]).max() == 0.0  # no slip on the lid
    wall = np.r_[0:n, 2 * n:nx]
    assert np.abs(v[0, wall]).max() == 0.0  # nothing crosses the floor beside the interface
    q_in, q_out = h * u[:, 0].sum(), h * u[:, nx].sum()
    q_gamma = -h * v[0, n:2 * n].sum()  # downward into the porous medium
    assert q_in > 0 and q_out > 0 and q_gamma > 0
    assert abs(q_in - q_out - q_gamma) <= 1e-12 * q_in
    q_bottom = (2.0 * K[0] / mu * ppm[0]).sum()
    assert abs(q_gamma - q_bottom) <= 1e-10 * q_gamma


def test_channel_kinetic_energy_decays_without_data():
    n = 6
    nx = 3 * n
    K = I.lognormal_K(n, -4.0, 1.0, 4.0, seed=4)
    o = O.Oracle(n, 1e-3, 1.0, 0.1, K, bc=2, dp=0.0, geo=GEO)
    A = o.scipy_csr().toarray()
    off = O.offsets(n, GEO)
    nv = off["p_ff"]
    # mass of each velocity row: the backward-Euler diagonal part, h^2/dt on full
    # control volumes and half of it on v_Gamma and the traction end faces
    m = np.zeros(nv)
    m[:] = 1.0
    ident = set(_identity_rows(A))
    for r in range(nv):
        if r in ident:
            m[r] = 0.0
    j_u = np.arange(off["v"]) // (nx + 1)
    i_u = np.arange(off["v"]) % (nx + 1)
    m[:off["v"]][(i_u == 0) | (i_u == nx)] *= 0.5
    m[off["v"] + n:off["v"] + 2 * n] *= 0.5
    x = np.random.default_rng(5).standard_normal(o.ndof)
    x[:nv][m == 0.0] = 0.0
    E = [float(np.sum(m * x[:nv] ** 2))]
    for s in range(6):
        x = o.run(x, 0.1 * s, 1)
        E.append(float(np.sum(m * x[:nv] ** 2)))
    assert all(b < a for a, b in zip(E, E[1:])), E
    assert j_u.max() == n - 1
