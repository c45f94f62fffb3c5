"""Pins of the partitioned-coupling oracle (Sec. 3) against the monolithic system.

The partitioned scheme has no printed worked example; it is pinned by what
the mathematics fixes: the coupling blocks of Eq. (9) are exactly the
interface rows the split acts on, the monolithic solution is a fixed point
of S_ff o S_pm, the accelerated iteration converges to the monolithic
solution and (R being affine) terminates within the interface dimension,
relaxed Picard alone is slower, and the order of Sec. 3 (free flow first,
velocity prescribed) leaves a singular free-flow block on these boundary
conditions.  A planted wrong interface flux moves the fixed point.  The
linearised maps show why the porous-medium-first order is the default: it
contracts, while Sec. 3's order amplifies by about 2K/(mu h).
"""
import numpy as np
import pytest

import oracle as O
from oracle.partitioned import DNOracle
from paper_2108_13229_gb300 import inputs as I


def setup(n, seed, mu=1e-3, alpha=1.0, dt=0.05, sigma=1.0):
    K = I.lognormal_K(n, -4.0, sigma, 4.0, seed=seed)
    o = O.Oracle(n, mu, alpha, dt, K)
    x0 = O.exact(n, 0.0, mu)
    b = o.rhs(x0, dt)
    return o, K, b


def test_coupling_blocks_are_the_interface_rows():
    # A[F, P] lives only on the v_Gamma rows (-h, block B'_1) and A[P, F] only on the
    # top Darcy rows (+h, block C'_1)
    n = 8
    o, K, b = setup(n, 1)
    d = DNOracle(o, K)
    AFP = d.AFP.tocoo()
    assert set(AFP.row.tolist()) == set(d.G.tolist())
    assert np.allclose(AFP.data, -d.h)
    APF = d.APF.tocoo()
    assert set(APF.row.tolist()) == set(d.T.tolist()) and set(APF.col.tolist()) == set(d.G.tolist())
    assert np.allclose(APF.data, d.h)


@pytest.mark.parametrize("n,seed", [(8, 2), (12, 3)])
def test_monolithic_solution_is_fixed_point(n, seed):
    o, K, b = setup(n, seed)
    x = o.solve(b)
    d = DNOracle(o, K)
    f = O.split(x, n)
    v = f["v"][0].copy()
    vt, p, xF, xP = d.H(v, b)
    assert np.abs(vt - v).max() <= 1e-10 * np.abs(v).max()
    assert np.abs(p - f["p_pm"][n - 1]).max() <= 1e-10 * np.abs(f["p_pm"]).max()
    assert np.abs(np.concatenate([xF, xP]) - x).max() <= 1e-10 * np.abs(x).max()


def test_paper_order_free_flow_block_is_singular_here():
    # with the velocity prescribed on the rest of the free-flow boundary, the free-flow
    # rows with a prescribed v_Gamma leave the pressure constant undetermined: the
    # constant p_ff vector is in the null space
    n = 8
    o, K, b = setup(n, 9)
    d = DNOracle(o, K)
    M = d.paper_order_ff_operator()
    off = O.offsets(n)
    z = np.zeros(d.nF)
    z[off["p_ff"]:off["p_pm"]] = 1.0
    assert np.abs(M @ z).max() <= 1e-12 * abs(M).max()
    # while the free-flow block of this order (v_Gamma an unknown) is not
    assert np.abs(d.AFF @ z).max() > 1e-3


@pytest.mark.parametrize("n,seed,mu", [(8, 4, 1e-3), (16, 5, 1e-3), (8, 6, 1.0)])
def test_iqn_ils_reaches_monolithic_solution(n, seed, mu):
    o, K, b = setup(n, seed, mu=mu)
    x = o.solve(b)
    d = DNOracle(o, K)
    xd, evals = d.solve(b, np.zeros(n), eps=1e-12)
    for k, e in O.split(xd, n).items():
        ref = O.split(x, n)[k]
        assert np.linalg.norm(e - ref) <= 1e-8 * np.linalg.norm(ref), k
    # R is affine in v: the least-squares model spans the n-dimensional
    # interface space after at most n differences
    assert evals <= n + 3


def test_acceleration_beats_picard():
    n = 8
    o, K, b = setup(n, 7)
    d = DNOracle(o, K)
    _, e_iqn = d.solve(b, np.zeros(n), eps=1e-10)
    with pytest.raises(RuntimeError):
        d.solve(b, np.zeros(n), eps=1e-10, accelerate=False, max_iter=e_iqn)


def test_planted_interface_flux_moves_fixed_point():
    n = 8
    o, K, b = setup(n, 8)
    x = o.solve(b)
    d = DNOracle(o, K, flux_scale=0.5)  # half the interface flux into the Darcy solve
    xd, _ = d.solve(b, np.zeros(n), eps=1e-12)
    assert np.linalg.norm(xd - x) > 1e-4 * np.linalg.norm(x)


def test_paper_order_well_posed_with_pressure_sides():
    # on the paper's pressure-driven problem (traction sides) the free-flow block
    # with a prescribed v_Gamma is regular: the order of Sec. 3 is well posed there
    import scipy.sparse.linalg as spl
    n = 8
    K = I.lognormal_K(n, -4.0, 1.0, 4.0, seed=10)
    o = O.Oracle(n, 1e-3, 1.0, 0.05, K, bc=2)
    d = DNOracle(o, K)
    M = d.paper_order_ff_operator().tocsc()
    off = O.offsets(n)
    z = np.zeros(d.nF)
    z[off["p_ff"]:off["p_pm"]] = 1.0
    assert np.abs(M @ z).max() > 1e-3
    lu = spl.splu(M)
    rng = np.random.default_rng(0)
    r = rng.standard_normal(d.nF)
    x = lu.solve(r)
    assert np.linalg.norm(M @ x - r) <= 1e-10 * np.linalg.norm(r)
    # and the coupled iteration still reproduces the monolithic step
    b = o.rhs(np.zeros(o.ndof), 0.05)
    xd, _ = d.solve(b, np.zeros(n), eps=1e-12)
    x_mono = o.solve(b)
    assert np.linalg.norm(xd - x_mono) <= 1e-9 * np.linalg.norm(x_mono)


@pytest.mark.parametrize("bc,n", [(1, 8), (2, 8), (2, 16)])
def test_paper_order_reaches_monolithic_solution(bc, n):
    # Sec. 3's order (free flow first with the velocity, then the porous medium
    # with the interface pressure) on problems with traction sides: the
    # monolithic solution is its fixed point (the interface pressure there is the
    # TPFA reconstruction of Eq. (5)) and IQN-ILS reaches it
    K = I.lognormal_K(n, -4.0, 1.0, 4.0, seed=11 + n)
    mu = 1e-3
    o = O.Oracle(n, mu, 1.0, 0.05, K, bc=bc)
    x0 = O.exact(n, 0.0, mu) if bc == 1 else np.zeros(o.ndof)
    b = o.rhs(x0, 0.05)
    x = o.solve(b)
    d = DNOracle(o, K, order="paper")
    f = O.split(x, n)
    v = f["v"][0].copy()
    vt, p, xF, xP = d.H(v, b)
    assert np.abs(vt - v).max() <= 1e-9 * np.abs(v).max()
    recon = f["p_pm"][n - 1] - mu / n / (2.0 * K.reshape(n, n)[n - 1]) * v
    assert np.abs(p - recon).max() <= 1e-9 * np.abs(recon).max()
    xd, evals = d.solve(b, np.zeros(n), eps=1e-12)
    assert np.linalg.norm(xd - x) <= 1e-8 * np.linalg.norm(x)
    # relaxed first step, n difference columns, the step onto the fixed point,
    # and the evaluations the stopping test needs to see the change vanish
    assert evals <= n + 4


@pytest.mark.parametrize("n,seed", [(24, 40), (32, 5)])
def test_order_amplification(n, seed):
    # the linearised coupling maps on the pressure-driven problem (traction
    # sides, log-normal K, mu = 1e-3): Sec. 3's order passes the interface
    # pressure through the half cell below Gamma, so an error in the free-flow
    # solve's pressure reaches the returned velocity multiplied by about the
    # transmissibility over h, 2K/(mu h) (between its mean and its maximum over
    # the interface); the whole map dH/dv amplifies by hundreds.  The
    # porous-medium-first map contracts (norm below 0.1), so no subdomain
    # error is amplified
    K = I.lognormal_K(n, -4.0, 1.0, 16.0, seed=seed)
    mu = 1e-3
    o = O.Oracle(n, mu, 1.0, 0.05, K, bc=2)
    b = np.zeros(o.ndof)  # the maps are affine: their linear parts
    paper, pm = DNOracle(o, K, order="paper"), DNOracle(o, K, order="pm")
    E = np.eye(n)
    J_pm_solve = np.stack([paper.s_pm_paper(e, b)[1] for e in E], 1)
    fac = 2.0 * K[n - 1] / (mu / n)
    assert fac.mean() <= np.linalg.norm(J_pm_solve, 2) <= fac.max()
    assert np.linalg.norm(np.stack([paper.H(e, b)[0] for e in E], 1), 2) > 100.0
    assert np.linalg.norm(np.stack([pm.H(e, b)[0] for e in E], 1), 2) < 0.1
