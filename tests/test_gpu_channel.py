"""Parity of the CUDA path with the FP64 oracle on the channel geometry of
the model problem (Sec. 5): free flow 3n x n cells over the n x n porous
medium, the interface the middle third of the channel's floor, walls beside
it (sd_options.geometry = SD_GEO_CHANNEL).

Tolerances as in test_gpu_parity: operator and right-hand side relative L2
<= 1e-13 (the same FP64 rows summed in another order), every column of the
4 x 4 operator to 1e-14 of the largest entry; solves at rtol = 1e-12 per
field <= 1e-8 against the oracle's direct solve.  Grids: n = 5 and 12
(ragged: 16 and 37 u faces per row), 40 (121 faces, four 32-wide tiles and a
tail, the blocks beside the porous medium take the free-flow-only interior
rows) and 64 (coarsening 64 -> 8).
"""
import numpy as np
import pytest

import oracle as O
from paper_2108_13229_gb300 import inputs as I

pytestmark = pytest.mark.gpu

GEO = 1


@pytest.fixture(scope="module")
def sd():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_13229_gb300 import sd as S
    S._load()
    return S


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def fields_rel(x, xr, n):
    fs, fr = O.split(x, n, GEO), O.split(xr, n, GEO)
    return {k: rel(fs[k], fr[k]) for k in fs}


def make(sd, n, mu, K, alpha, dt, precision=1, rtol=1e-10, **kw):
    o = sd.sd_options_default()
    o.precision = precision
    o.rtol = rtol
    o.geometry = sd.SD_GEO_CHANNEL
    for k, v in kw.items():
        setattr(o, k, v)
    return sd.sd_create(n, mu, K, alpha, dt, o)


def test_channel_dof_and_fields(sd):
    n = 12
    assert sd.sd_dof_count_geometry(n, sd.SD_GEO_CHANNEL) == O.dof_count(n, GEO)
    K = I.lognormal_K(n, -4.0, 1.0, 4.0, seed=1)
    h = make(sd, n, 1e-3, K, 1.0, 0.05)
    assert h.dof == O.dof_count(n, GEO)
    # the initial state is the manufactured solution continued over x in [-1, 2]
    _, _, x = sd.sd_get_state(h)
    assert rel(x, O.exact(n, 0.0, 1e-3, GEO)) <= 1e-15
    f = sd.sd_get_fields(h)
    fo = O.split(x, n, GEO)
    for k in fo:
        assert f[k].shape == fo[k].shape and np.array_equal(f[k], fo[k]), k


@pytest.mark.parametrize("bc", [0, 1, 2])
def test_channel_operator_columns(sd, bc):
    # every unit vector of a 4 x 4 porous medium under a 12 x 4 channel
    n = 4
    K = I.lognormal_K(n, -4.0, 1.0, 2.0, seed=2 + bc)
    o = O.Oracle(n, 0.7, 0.9, 0.2, K, bc=bc, geo=GEO)
    A = o.scipy_csr().toarray()
    h = make(sd, n, 0.7, K, 0.9, 0.2, bc=bc)
    scale = np.abs(A).max()
    for k in range(o.ndof):
        e = np.zeros(o.ndof)
        e[k] = 1.0
        assert np.abs(sd.sd_apply(h, e) - A[:, k]).max() <= 1e-14 * scale, k


@pytest.mark.parametrize("bc", [0, 1, 2])
@pytest.mark.parametrize("n", [5, 12, 40, 64])
def test_channel_operator_parity(sd, n, bc):
    K = I.lognormal_K(n, -4.0, 1.5, 4.0, seed=n + 7 * bc)
    o = O.Oracle(n, 1e-3, 1.3, 0.05, K, bc=bc, geo=GEO)
    h = make(sd, n, 1e-3, K, 1.3, 0.05, bc=bc)
    rng = np.random.default_rng(n)
    for _ in range(3):
        x = rng.standard_normal(o.ndof)
        assert rel(sd.sd_apply(h, x), o.apply(x)) <= 1e-13


@pytest.mark.parametrize("bc", [0, 1, 2])
def test_channel_rhs_parity(sd, bc):
    n = 12
    K = I.lognormal_K(n, -4.0, 1.0, 4.0, seed=3)
    o = O.Oracle(n, 1e-3, 0.9, 0.05, K, bc=bc, dp=2.0, t_end=0.5, geo=GEO)
    h = make(sd, n, 1e-3, K, 0.9, 0.05, bc=bc, bc_dp=2.0, bc_tend=0.5)
    rng = np.random.default_rng(4)
    for t in (0.05, 0.3, 0.73):
        xp = rng.standard_normal(o.ndof)
        assert rel(sd.sd_rhs(h, xp, t), o.rhs(xp, t)) <= 1e-13


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("n", [8, 12, 40])
def test_channel_solve_parity(sd, n, precision):
    K = I.lognormal_K(n, -4.0, 1.0, 4.0, seed=n)
    o = O.Oracle(n, 1e-3, 1.3, 0.05, K, geo=GEO)
    h = make(sd, n, 1e-3, K, 1.3, 0.05, precision, rtol=1e-12)
    rng = np.random.default_rng(10 + n)
    b = rng.standard_normal(o.ndof)
    x = np.zeros(o.ndof)
    info = sd.sd_solve(h, b, x)
    assert info["status"] == 0 and info["relres"] <= 1e-12
    for k, e in fields_rel(x, o.solve(b), n).items():
        assert e <= 1e-8, (k, e)


@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("precision", [0, 1])
def test_channel_mms_time_stepping(sd, precision, bc):
    # the manufactured solution on the channel: 16 x 16 pm cells, mu = K = alpha = 1, dt = 0.1
    n = 16
    K = np.ones((n, n))
    o = O.Oracle(n, 1.0, 1.0, 0.1, K, bc=bc, geo=GEO)
    xr = o.run(O.exact(n, 0.0, 1.0, GEO), 0.0, 6)
    h = make(sd, n, 1.0, K, 1.0, 0.1, precision, rtol=1e-12, bc=bc)
    infos = sd.sd_step(h, 6)
    assert all(i["status"] == 0 for i in infos)
    for k, e in fields_rel(sd.sd_get_state(h)[2], xr, n).items():
        assert e <= 1e-8, (k, e)


@pytest.mark.parametrize("precision,n", [(0, 24), (1, 32), (1, 64)])
def test_channel_pressure_driven_problem(sd, precision, n):
    # the model problem of Sec. 5: from rest, the inflow pressure rising over 10 steps, lognormal K
    K = I.lognormal_K(n, -4.0, 1.0, 16.0, seed=34)
    dt = 0.05
    o = O.Oracle(n, 1e-3, 1.0, dt, K, bc=2, dp=1.0, t_end=10 * dt, geo=GEO)
    xr = o.run(np.zeros(o.ndof), 0.0, 6)
    h = make(sd, n, 1e-3, K, 1.0, dt, precision, rtol=1e-12, bc=2, bc_dp=1.0, bc_tend=10 * dt)
    infos = sd.sd_step(h, 6)
    assert all(i["status"] == 0 for i in infos)
    for k, e in fields_rel(sd.sd_get_state(h)[2], xr, n).items():
        assert e <= 1e-8, (k, e)


def test_channel_pressure_driven_balance_at_512(sd):
    # 512 x 512 pm cells under a 1536 x 512 channel (2.6 M unknowns), the bench's
    # physics: the oracle recomputes the residual of the GPU state with its own
    # CSR matrix, and the flow obeys the balances that hold at any size
    n = 512
    K = I.lognormal_K(n, -4.0, 1.0, 16.0, seed=0)
    dt = 0.05
    h = make(sd, n, 1e-3, K, 1.0, dt, 1, bc=2, bc_dp=1.0, bc_tend=10 * dt)
    infos = sd.sd_step(h, 4)
    assert all(i["status"] == 0 and i["relres"] <= 1e-10 for i in infos)
    _, _, x1, x0 = sd.sd_get_state(h, with_prev=True)
    o = O.Oracle(n, 1e-3, 1.0, dt, K, bc=2, dp=1.0, t_end=10 * dt, geo=GEO)
    b = o.rhs(x0, 4 * dt)
    _, r = o.residual(x1, b)
    assert r / np.linalg.norm(b) <= 1.05e-10
    f = O.split(x1, n, GEO)
    hh = 1.0 / n
    nx = 3 * n
    u, v = f["u"], f["v"]
    assert np.abs(v[n]).max() == 0.0 and np.abs(v[0, np.r_[0:n, 2 * n:nx]]).max() == 0.0
    q_in, q_out = hh * u[:, 0].sum(), hh * u[:, nx].sum()
    q_gamma = -hh * v[0, n:2 * n].sum()
    assert q_in > 0 and q_out > 0
    # the continuity rows hold to the solve's tolerance
    assert abs(q_in - q_out - q_gamma) <= 1e-6 * q_in


def test_channel_lockstep_batch_bitwise(sd):
    n = 32
    Ks = [I.lognormal_K(n, -4.0, 1.0, 8.0, seed=40 + k) for k in range(3)]
    alone = []
    for K in Ks:
        h = make(sd, n, 1e-3, K, 1.0, 0.05, bc=2, bc_dp=1.0)
        sd.sd_step(h, 3)
        alone.append(sd.sd_get_state(h)[2])
    for flags in (sd.SD_BATCH_LOCKSTEP, sd.SD_BATCH_LOCKSTEP | sd.SD_BATCH_GRAPH):
        hs = [make(sd, n, 1e-3, K, 1.0, 0.05, bc=2, bc_dp=1.0) for K in Ks]
        sd.sd_solve_batch_ex(hs, [3, 3, 3], flags=flags)
        for h, xa in zip(hs, alone):
            assert np.array_equal(sd.sd_get_state(h)[2], xa)


def test_channel_options(sd):
    n = 16
    K = np.ones((n, n))
    # the partitioned coupling serves the square geometry only
    with pytest.raises(sd.SdError):
        make(sd, n, 1.0, K, 1.0, 0.1, coupling=sd.SD_PARTITIONED)
    # n = 9 * 2^k cannot coarsen to 8 x 8 or below
    with pytest.raises(sd.SdError):
        make(sd, 18, 1.0, np.ones((18, 18)), 1.0, 0.1)


@pytest.mark.parametrize("n,bc", [(64, 0), (64, 2), (256, 0), (256, 2), (512, 0), (512, 2), (1024, 2)])
def test_channel_tiled_smoothing_bitwise(sd, n, bc):
    # the shared-memory tiles (with the residual and restriction fused into the
    # pre-smoothing on levels up to 256 cells per side) and, with tile 2 from
    # 1024 cells per side, the register-column tiles of the Darcy block, against
    # one launch per Chebyshev step: the same bits, over tile heights 4, 8 and 16
    K = I.lognormal_K(n, -4.0, 1.0, 16.0, seed=5)
    xs = []
    for tile, rows in ((0, 0), (1, 4), (1, 8), (2, 16), (2, 0)):
        h = make(sd, n, 1e-3, K, 1.0, 0.05, bc=bc, bc_dp=1.0, tile=tile, tile_rows=rows)
        infos = sd.sd_step(h, 3)
        assert all(i["status"] == 0 for i in infos)
        xs.append(sd.sd_get_state(h)[2])
    for x in xs[1:]:
        assert np.array_equal(x, xs[0])
