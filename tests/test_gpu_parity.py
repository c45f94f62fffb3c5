"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances:
 * operator and right-hand side: the same FP64 rows summed in another order,
   relative L2 <= 1e-13 (a few ulps times the row length);
 * solves at rtol = 1e-12: per-field relative L2 <= 1e-8 against the
   oracle's direct solve (forward error <= cond * 1e-12 with cond <~ 1e4);
 * at the workload size the oracle cannot factor; there it recomputes the
   residual of the GPU solution with its own CSR matrix.
Grids span several 32 x 8 thread tiles with ragged tails (n = 40: 41 faces
per row) and odd coarsest grids (n = 5, 12, 40).
"""
import numpy as np
import pytest

import oracle as O
from paper_2108_13229_gb300 import inputs as I

pytestmark = pytest.mark.gpu


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
    fs, fr = O.split(x, n), O.split(xr, n)
    return {k: rel(fs[k], fr[k]) for k in fs}


def make(sd, n, mu, K, alpha, dt, precision=1, rtol=1e-10, **kw):
    o = sd.sd_options_default()
    o.precision = precision
    o.rtol = rtol
    for k, v in kw.items():
        setattr(o, k, v)
    return sd.sd_create(n, mu, K, alpha, dt, o)


@pytest.mark.parametrize("n", [4, 5, 12, 40, 72])
def test_operator_parity(sd, n):
    K = I.lognormal_K(n, -4.0, 1.5, 4.0, seed=n)
    o = O.Oracle(n, 1e-3, 1.3, 0.05, K)
    h = make(sd, n, 1e-3, K, 1.3, 0.05)
    rng = np.random.default_rng(n)
    for _ in range(3):
        x = rng.standard_normal(o.ndof)
        assert rel(sd.sd_apply(h, x), o.apply(x)) <= 1e-13


def test_operator_columns(sd):
    # apply to every unit vector of a 4 x 4 grid: each column of the CSR matrix
    n = 4
    K = I.lognormal_K(n, -4.0, 1.0, 2.0, seed=1)
    o = O.Oracle(n, 0.7, 0.9, 0.2, K)
    A = o.scipy_csr().toarray()
    h = make(sd, n, 0.7, K, 0.9, 0.2)
    scale = np.abs(A).max()
    for k in range(o.ndof):
        e = np.zeros(o.ndof)
        e[k] = 1.0
        assert np.abs(sd.sd_apply(h, e) - A[:, k]).max() <= 1e-14 * scale


@pytest.mark.parametrize("n", [5, 40])
def test_rhs_parity(sd, n):
    K = I.lognormal_K(n, -4.0, 1.0, 4.0, seed=2)
    o = O.Oracle(n, 1e-3, 1.0, 0.05, K)
    h = make(sd, n, 1e-3, K, 1.0, 0.05)
    rng = np.random.default_rng(3)
    for t in (0.05, 0.73):
        xp = rng.standard_normal(o.ndof)
        assert rel(sd.sd_rhs(h, xp, t), o.rhs(xp, t)) <= 1e-13


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("n", [4, 8, 12, 40])
def test_solve_parity(sd, n, precision):
    K = I.lognormal_K(n, -4.0, 1.0, 4.0, seed=n)
    o = O.Oracle(n, 1e-3, 1.3, 0.05, K)
    h = make(sd, n, 1e-3, K, 1.3, 0.05, precision, rtol=1e-12)
    rng = np.random.default_rng(10 + n)
    b = rng.standard_normal(o.ndof)
    x = np.zeros(o.ndof)
    info = sd.sd_solve(h, b, x)
    assert info["status"] == 0 and info["relres"] <= 1e-12
    for k, e in fields_rel(x, o.solve(b), n).items():
        assert e <= 1e-8, (k, e)


@pytest.mark.parametrize("precision", [0, 1])
def test_mms_time_stepping(sd, precision):
    # manufactured-solution case: 32 x 32 cells, mu = K = alpha = 1, dt = 0.1, 10 steps
    n = 32
    K = np.ones((n, n))
    o = O.Oracle(n, 1.0, 1.0, 0.1, K)
    xr = o.run(O.exact(n, 0.0, 1.0), 0.0, 10)
    h = make(sd, n, 1.0, K, 1.0, 0.1, precision, rtol=1e-12)
    infos = sd.sd_step(h, 10)
    assert all(i["status"] == 0 for i in infos)
    t, step, x = sd.sd_get_state(h)
    assert step == 10 and abs(t - 1.0) < 1e-12
    for k, e in fields_rel(x, xr, n).items():
        assert e <= 1e-8, (k, e)
    # at the default rtol = 1e-10 the result stays within the forward-error bound
    h2 = make(sd, n, 1.0, K, 1.0, 0.1, precision)
    infos = sd.sd_step(h2, 10)
    assert max(i["relres"] for i in infos) <= 1e-10
    _, _, x2 = sd.sd_get_state(h2)
    for k, e in fields_rel(x2, xr, n).items():
        assert e <= 1e-6, (k, e)


@pytest.mark.parametrize("coarsest", [16, 4])
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("n", [64, 128])
def test_lognormal_time_stepping(sd, n, precision, coarsest):
    # the workload's physics (mu = 1e-3, ln K ~ N(-4, 1), corr. 16 cells) on grids the oracle factors;
    # coarsest 16: the dense 16 x 16 solve spread over all SMs, 4: the fused single-CTA coarse cycle;
    # five steps, so that the default quadratic extrapolation starts (step 4)
    K = I.lognormal_K(n, -4.0, 1.0, 16.0, seed=0)
    o = O.Oracle(n, 1e-3, 1.0, 0.05, K)
    xr = o.run(O.exact(n, 0.0, 1e-3), 0.0, 5)
    h = make(sd, n, 1e-3, K, 1.0, 0.05, precision, rtol=1e-12, coarsest=coarsest)
    infos = sd.sd_step(h, 5)
    assert all(i["status"] == 0 for i in infos)
    _, _, x = sd.sd_get_state(h)
    for k, e in fields_rel(x, xr, n).items():
        assert e <= 1e-8, (k, e)


@pytest.mark.parametrize("n", [1024, 2048])
def test_workload_size_residual(sd, n):
    # 1024 x 1024 cells, the benchmark's launch configuration (mixed precision, rtol 1e-10),
    # and the 2048 x 2048 workload: the oracle recomputes ||b - A x|| / ||b|| of the GPU state
    # with its own CSR matrix
    K = I.lognormal_K(n, -4.0, 1.0, 16.0, seed=0)
    o = O.Oracle(n, 1e-3, 1.0, 0.05, K)
    h = make(sd, n, 1e-3, K, 1.0, 0.05, 1)
    sd.sd_step(h, 1)
    _, _, x1 = sd.sd_get_state(h)
    info = sd.sd_step(h, 1)[0]
    _, _, x2 = sd.sd_get_state(h)
    b = o.rhs(x1, 0.1)
    _, r = o.residual(x2, b)
    assert r / np.linalg.norm(b) <= 1.05e-10 and info["relres"] <= 1e-10
    # operator parity at full size on a random vector
    rng = np.random.default_rng(0)
    xv = rng.standard_normal(o.ndof)
    assert rel(sd.sd_apply(h, xv), o.apply(xv)) <= 1e-13


def test_extrapolation_orders_reach_the_same_states(sd):
    # the initial guess only moves the iteration count: the states of 8 steps
    # with linear, quadratic and cubic extrapolation agree to the tolerance
    n = 64
    K = I.lognormal_K(n, -4.0, 1.0, 16.0, seed=14)
    xs, its = [], []
    for ex in (1, 2, 3):
        h = make(sd, n, 1e-3, K, 1.0, 0.05, rtol=1e-11, extrapolate=ex)
        infos = sd.sd_step(h, 8)
        assert all(i["status"] == 0 and i["relres"] <= 1e-11 for i in infos)
        xs.append(sd.sd_get_state(h)[2])
        its.append(sum(i["iters"] for i in infos[3:]))
    for x in xs[1:]:
        assert rel(x, xs[0]) <= 1e-8
    assert its[1] < its[0]


@pytest.mark.parametrize("extrapolate", [2, 1])
def test_determinism_and_state_roundtrip(sd, extrapolate):
    # resume from (t, step, x^n, x^{n-1}) and, for the quadratic extrapolation,
    # x^{n-2}: bitwise the uninterrupted run
    n = 64
    K = I.lognormal_K(n, -4.0, 1.0, 16.0, seed=4)
    h1 = make(sd, n, 1e-3, K, 1.0, 0.05, extrapolate=extrapolate)
    h2 = make(sd, n, 1e-3, K, 1.0, 0.05, extrapolate=extrapolate)
    sd.sd_step(h1, 5)
    sd.sd_step(h2, 3)
    t, st, x, xp = sd.sd_get_state(h2, with_prev=True)
    xpp = sd.sd_get_history(h2)
    assert (xpp is not None) == (extrapolate == 2)
    h3 = make(sd, n, 1e-3, K, 1.0, 0.05, extrapolate=extrapolate)
    sd.sd_set_state(h3, t, st, x, xp)
    if xpp is not None:
        assert sd.sd_get_history(h3) is None  # cleared by sd_set_state
        sd.sd_set_history(h3, xpp)
    sd.sd_step(h2, 2)
    sd.sd_step(h3, 2)
    a, b, c = sd.sd_get_state(h1)[2], sd.sd_get_state(h2)[2], sd.sd_get_state(h3)[2]
    assert np.array_equal(a, b) and np.array_equal(a, c)


def test_batch_alone_vs_mixed(sd):
    cases = [(32, 1), (64, 2), (128, 3), (64, 4)]
    alone = []
    for n, seed in cases:
        h = make(sd, n, 1e-3, I.lognormal_K(n, -4.0, 1.5, 16.0, seed=seed), 0.5 + seed, 0.1)
        sd.sd_step(h, 3)
        alone.append(sd.sd_get_state(h)[2])
    hs = [make(sd, n, 1e-3, I.lognormal_K(n, -4.0, 1.5, 16.0, seed=seed), 0.5 + seed, 0.1) for n, seed in cases]
    infos = sd.sd_solve_batch(hs, [3] * len(cases))
    assert all(i["status"] == 0 for inf in infos for i in inf)
    for h, xa in zip(hs, alone):
        assert np.array_equal(sd.sd_get_state(h)[2], xa)


@pytest.mark.parametrize("precision", [1, 0])
def test_lockstep_batch_bitwise(sd, precision):
    # lockstep groups (same n): instances with their own K field, alpha_BJ
    # and iteration counts share every launch; converged instances sit idle.
    # Each result equals its solo run bit for bit, as does the
    # one-stream-per-instance mode.  n = 48 (one group of three, 49 faces per
    # row; dense 12 x 12 coarsest solve), n = 16 with coarsest 4 (fused coarse
    # cycle from the fine level), one n = 40 alone.
    cases = [(48, 1, 0.1), (48, 2, 3.0), (48, 3, 10.0), (16, 4, 0.3), (16, 5, 7.0), (40, 6, 1.0)]
    def mk(n, seed, alpha):
        K = I.lognormal_K(n, -4.0, 0.5 + 0.3 * seed, 16.0, seed=seed)
        return make(sd, n, 1e-3, K, alpha, 0.1, precision, coarsest=4 if n == 16 else 16)
    alone, its_alone = [], []
    for n, seed, alpha in cases:
        h = mk(n, seed, alpha)
        infos = sd.sd_step(h, 4)
        alone.append(sd.sd_get_state(h)[2])
        its_alone.append([i["iters"] for i in infos])
    for lockstep in (True, False):
        hs = [mk(n, seed, alpha) for n, seed, alpha in cases]
        l0 = sd.sd_launch_count()
        infos = sd.sd_solve_batch(hs, [4] * len(cases), lockstep=lockstep)
        launches = sd.sd_launch_count() - l0
        for h, xa, inf, ia in zip(hs, alone, infos, its_alone):
            assert [i["iters"] for i in inf] == ia
            assert all(i["status"] == 0 for i in inf)
            assert np.array_equal(sd.sd_get_state(h)[2], xa)
        if lockstep:
            launches_lockstep = launches
        else:
            assert launches_lockstep < launches  # the groups share their launches


@pytest.mark.parametrize("precision", [1, 0])
def test_graph_batch_bitwise(sd, precision):
    # SD_BATCH_GRAPH: all groups of a step (uneven grids: a group of three 48^2, a
    # group of two 16^2 with the fused coarse cycle, one 40^2 alone) in one graph
    # launch, the solves decided on the device; every state, iteration and
    # restart count equals the solo run's (restart 4 and max_iters 9 bring in
    # restarts and the iteration cap), and equals the host-driven groups'
    cases = [(48, 1, 0.1), (48, 2, 3.0), (48, 3, 10.0), (16, 4, 0.3), (16, 5, 7.0), (40, 6, 1.0)]
    def mk(n, seed, alpha, **kw):
        K = I.lognormal_K(n, -4.0, 0.5 + 0.3 * seed, 16.0, seed=seed)
        return make(sd, n, 1e-3, K, alpha, 0.1, precision, coarsest=4 if n == 16 else 16, **kw)
    for kw in ({}, {"restart": 4, "max_iters": 9}):
        alone, inf_alone = [], []
        for n, seed, alpha in cases:
            h = mk(n, seed, alpha, **kw)
            inf = sd.sd_step(h, 4, raise_on_error=False)
            alone.append(sd.sd_get_state(h)[2])
            inf_alone.append(inf)
        for flags in (sd.SD_BATCH_LOCKSTEP | sd.SD_BATCH_GRAPH, sd.SD_BATCH_LOCKSTEP):
            hs = [mk(n, seed, alpha, **kw) for n, seed, alpha in cases]
            infos = sd.sd_solve_batch_ex(hs, [4] * len(cases), flags=flags, raise_on_error=False)
            for h, xa, inf, ia in zip(hs, alone, infos, inf_alone):
                for a, b in zip(inf, ia):
                    for key in ("iters", "restarts", "status", "reorths", "relres", "relres_v", "relres_pff",
                                "relres_pm"):
                        assert a[key] == b[key], (flags, key, a[key], b[key])
                assert np.array_equal(sd.sd_get_state(h)[2], xa)
        if kw:  # the cap was reached somewhere: the NOCONV path ran on the device
            assert any(i["status"] == sd.SD_E_NOCONV for inf in inf_alone for i in inf)


def test_graph_batch_uneven_steps(sd):
    # groups with different step counts: the graph is rebuilt when a group
    # stops; a second call on the same handles reuses the cached graph, and
    # destroying a member drops it (the next batch builds its own)
    cases = [(32, 1, 4), (32, 2, 4), (24, 3, 2), (24, 4, 2)]
    flags = sd.SD_BATCH_LOCKSTEP | sd.SD_BATCH_GRAPH
    def mk(n, seed):
        return make(sd, n, 1e-3, I.lognormal_K(n, -4.0, 1.0, 8.0, seed=seed), 1.0, 0.1, 1)
    alone = []
    for n, seed, steps in cases:
        h = mk(n, seed)
        sd.sd_step(h, steps + 3)
        alone.append(sd.sd_get_state(h))
    hs = [mk(n, seed) for n, seed, _ in cases]
    sd.sd_solve_batch_ex(hs, [c[2] for c in cases], flags=flags)
    sd.sd_solve_batch_ex(hs, [3] * len(cases), flags=flags)
    sd.sd_solve_batch_ex(hs[2:], [0, 0], flags=flags)  # another batch: the cache changes hands
    for h, (t, step, xa) in zip(hs, alone):
        t2, step2, x2 = sd.sd_get_state(h)
        assert step2 == step and t2 == t and np.array_equal(x2, xa)
    del hs
    hs = [mk(n, seed) for n, seed, _ in cases[:2]]
    sd.sd_solve_batch_ex(hs, [c[2] + 3 for c in cases[:2]], flags=flags)
    for h, (t, step, xa) in zip(hs, alone[:2]):
        assert np.array_equal(sd.sd_get_state(h)[2], xa)


@pytest.mark.parametrize("lockstep", [True, False])
def test_server_results_match_alone(sd, lockstep):
    # lockstep: runs of one size class step together, joining and leaving
    # between ticks (n = 32 and n = 64 have two runs each of different lengths).
    # A server made without options picks the multigrid depth per run: runs
    # under 40 steps coarsen to 4 x 4, longer ones stop at 16 x 16.
    reqs = [(32, 5, 1), (64, 7, 2), (128, 4, 3), (32, 9, 4), (96, 6, 5), (64, 5, 6), (32, 41, 7)]
    srv = sd.sd_server_create(8 << 30, 3, lockstep=lockstep)
    tickets = []
    for n, steps, seed in reqs:
        K = I.lognormal_K(n, -4.0, 1.0, 16.0, seed=seed)
        tickets.append(sd.sd_submit(srv, n, 1e-3, K, 1.0, 0.1, steps, keep_fields=True))
    sd.sd_server_drain(srv)
    for (n, steps, seed), tk in zip(reqs, tickets):
        rc, res, x = sd.sd_poll(srv, tk, want_x=True)
        assert rc == 0 and res["steps_done"] == steps and res["latency_ms"] >= res["run_ms"] > 0
        K = I.lognormal_K(n, -4.0, 1.0, 16.0, seed=seed)
        h = make(sd, n, 1e-3, K, 1.0, 0.1, coarsest=4 if steps < 40 else 16)
        sd.sd_step(h, steps)
        assert np.array_equal(sd.sd_get_state(h)[2], x)
    sd.sd_server_destroy(srv)


def test_error_paths(sd):
    n = 32
    K = np.ones((n, n))
    h = make(sd, n, 1.0, K, 1.0, 0.1, max_iters=2)
    infos = sd.sd_step(h, 1, raise_on_error=False)
    assert infos[0]["status"] == sd.SD_E_NOCONV
    t, st, _ = sd.sd_get_state(h)
    assert st == 1 and abs(t - 0.1) < 1e-15
    srv = sd.sd_server_create(1 << 20, 1)
    with pytest.raises(sd.SdError) as e:
        sd.sd_submit(srv, 256, 1e-3, np.ones((256, 256)), 1.0, 0.1, 2)
    assert e.value.code == sd.SD_E_NOMEM
    assert sd.sd_poll(srv, 12345)[0] == sd.SD_E_STATE
    sd.sd_server_destroy(srv)


def test_numeric_error_from_nan_rhs(sd):
    # a NaN planted in b on the host: the first residual norm is NaN, the
    # solve returns SD_E_NUMERIC before any update, and x keeps the guess
    n = 32
    K = I.lognormal_K(n, -4.0, 1.0, 4.0, seed=4)
    h = make(sd, n, 1e-3, K, 1.0, 0.05)
    rng = np.random.default_rng(4)
    b = rng.standard_normal(sd.sd_dof_count(n))
    b[7] = np.nan
    x0 = rng.standard_normal(b.size)
    x = x0.copy()
    info = sd.sd_solve(h, b, x, raise_on_error=False)
    assert info["status"] == sd.SD_E_NUMERIC
    assert np.array_equal(x, x0)
    # the handle stays usable: a finite right-hand side solves afterwards
    b[7] = 0.0
    info = sd.sd_solve(h, b, x)
    assert info["status"] == 0 and info["relres"] <= 1e-10


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("n", [40, 64])
def test_schur_mass_only_parity(sd, n, precision):
    # the Schur block as the viscosity-scaled pressure mass matrix alone,
    # S^-1 = (mu/(gamma h^2)) I (schur_mass = 0), on the log-normal physics:
    # the same states as the oracle, three steps.  The residual test bounds
    # the error only through the condition number, and this weaker Schur block
    # leaves iterates whose p_ff error (1.7e-8 at rtol 1e-12, n = 40) sits
    # above the per-field bound, so the solve runs to rtol 1e-13.
    K = I.lognormal_K(n, -4.0, 1.0, 16.0, seed=1)
    o = O.Oracle(n, 1e-3, 1.0, 0.05, K)
    xr = o.run(O.exact(n, 0.0, 1e-3), 0.0, 3)
    h = make(sd, n, 1e-3, K, 1.0, 0.05, precision, rtol=1e-13, schur_mass=0, max_iters=3000)
    infos = sd.sd_step(h, 3)
    assert all(i["status"] == 0 for i in infos), infos
    print("schur_mass=0 n=%d precision=%d iterations per step:" % (n, precision), [i["iters"] for i in infos])
    _, _, x = sd.sd_get_state(h)
    for k, e in fields_rel(x, xr, n).items():
        assert e <= 1e-8, (k, e)


@pytest.mark.parametrize("mode", [1, 2])
def test_paper_block_preconditioners(sd, mode):
    # P^pv_BJ and P^pv_BGS with the identity on the p_ff block (Sec. 4) on the
    # manufactured-solution case: same solution as the oracle
    n = 16
    K = np.ones((n, n))
    o = O.Oracle(n, 1.0, 1.0, 0.1, K)
    xr = o.run(O.exact(n, 0.0, 1.0), 0.0, 1)
    h = make(sd, n, 1.0, K, 1.0, 0.1, 0, rtol=1e-12, precond=mode, max_iters=3000)
    info = sd.sd_step(h, 1)[0]
    assert info["status"] == 0
    _, _, x = sd.sd_get_state(h)
    for k, e in fields_rel(x, xr, n).items():
        assert e <= 1e-8, (k, e)


def test_graph_replay_bitwise(sd):
    # the captured Arnoldi step launches exactly the kernels of the direct path
    n = 64
    K = I.lognormal_K(n, -4.0, 1.0, 16.0, seed=9)
    xs = []
    for graph in (0, 1):
        h = make(sd, n, 1e-3, K, 1.0, 0.05, graph=graph)
        sd.sd_step(h, 4)
        xs.append(sd.sd_get_state(h)[2])
    assert np.array_equal(xs[0], xs[1])


@pytest.mark.parametrize("restart,max_iters,precision", [(30, 600, 1), (4, 600, 1), (4, 600, 0), (4, 6, 1)])
def test_solve_graph_bitwise(sd, restart, max_iters, precision):
    # graph option 2 (a whole solve as one graph, its loop decided on the
    # device) runs the iterations of the step-by-step path: the same iterates
    # bit for bit and the same counters; the kernel count grows by exactly the
    # control kernels (2 per solve, 2 per restart cycle, 1 per iteration)
    n = 64
    K = I.lognormal_K(n, -4.0, 1.0, 16.0, seed=9)
    res = []
    for graph in (1, 2):
        h = make(sd, n, 1e-3, K, 1.0, 0.05, precision, graph=graph, restart=restart, max_iters=max_iters)
        l0 = sd.sd_launch_count()
        infos = sd.sd_step(h, 3, raise_on_error=False)
        res.append((infos, sd.sd_launch_count() - l0, sd.sd_get_state(h)[2]))
    (i1, c1, x1), (i2, c2, x2) = res
    assert np.array_equal(x1, x2)
    keys = ["iters", "restarts", "status", "relres", "reorths", "relres_v", "relres_pff", "relres_pm"]
    for a, b in zip(i1, i2):
        assert [a[k] for k in keys] == [b[k] for k in keys]
    if max_iters < 600:
        assert all(i["status"] == -3 for i in i2)
    else:
        assert all(i["status"] == 0 for i in i2)
        assert max(i["restarts"] for i in i2) >= (2 if restart == 4 else 1)
    extra = sum(2 + 2 * i["restarts"] + i["iters"] for i in i2)
    assert c2 == c1 + extra


def test_solve_graph_partitioned_and_solve(sd):
    # the subdomain solves of the partitioned coupling and sd_solve (another
    # iterate buffer: the graph is rebuilt for it) through graph option 2
    n = 64
    K = I.lognormal_K(n, -4.0, 1.0, 16.0, seed=12)
    out = []
    for graph in (1, 2):
        h = make(sd, n, 1e-3, K, 1.0, 0.05, graph=graph, coupling=1)
        infos = sd.sd_step(h, 2)
        hm = make(sd, n, 1e-3, K, 1.0, 0.05, graph=graph)
        sd.sd_step(hm, 1)
        b = sd.sd_rhs(hm, sd.sd_get_state(hm)[2], 0.1)
        x = np.zeros_like(b)
        si = sd.sd_solve(hm, b, x)
        sd.sd_step(hm, 1)
        out.append((infos, sd.sd_get_state(h)[2], x, si, sd.sd_get_state(hm)[2]))
    (ia, xa, sa, ka, ya), (ib, xb, sb, kb, yb) = out
    assert [(i["iters"], i["coupling_iters"]) for i in ia] == [(i["iters"], i["coupling_iters"]) for i in ib]
    assert np.array_equal(xa, xb)
    assert np.array_equal(sa, sb) and ka["iters"] == kb["iters"]
    assert np.array_equal(ya, yb)


@pytest.mark.parametrize("precision", [0, 1])
def test_darcy_overlap_parity(sd, precision):
    # block-diagonal Darcy part on a second stream: same solution as the oracle
    n = 64
    K = I.lognormal_K(n, -4.0, 1.0, 16.0, seed=0)
    o = O.Oracle(n, 1e-3, 1.0, 0.05, K)
    xr = o.run(O.exact(n, 0.0, 1e-3), 0.0, 3)
    h = make(sd, n, 1e-3, K, 1.0, 0.05, precision, rtol=1e-12, darcy_coupled=0)
    infos = sd.sd_step(h, 3)
    assert all(i["status"] == 0 for i in infos)
    _, _, x = sd.sd_get_state(h)
    for k, e in fields_rel(x, xr, n).items():
        assert e <= 1e-8, (k, e)


@pytest.mark.parametrize("precision", [0, 1])
def test_darcy_first_parity(sd, precision):
    # Darcy block first (B'_1 kept), concurrent with the pressure block: same solution
    n = 64
    K = I.lognormal_K(n, -4.0, 1.0, 16.0, seed=0)
    o = O.Oracle(n, 1e-3, 1.0, 0.05, K)
    xr = o.run(O.exact(n, 0.0, 1e-3), 0.0, 3)
    h = make(sd, n, 1e-3, K, 1.0, 0.05, precision, rtol=1e-12, darcy_coupled=2)
    infos = sd.sd_step(h, 3)
    assert all(i["status"] == 0 for i in infos)
    _, _, x = sd.sd_get_state(h)
    for k, e in fields_rel(x, xr, n).items():
        assert e <= 1e-8, (k, e)


def test_pdl_bitwise(sd):
    # programmatic dependent launch only changes when grids start, not what they compute
    n = 64
    K = I.lognormal_K(n, -4.0, 1.0, 16.0, seed=10)
    xs = []
    for pdl in (0, 1):
        h = make(sd, n, 1e-3, K, 1.0, 0.05, pdl=pdl)
        sd.sd_step(h, 3)
        xs.append(sd.sd_get_state(h)[2])
    assert np.array_equal(xs[0], xs[1])


@pytest.mark.parametrize("n,bc", [(64, 0), (96, 0), (256, 0), (1024, 0), (1024, 2)])
def test_tiled_smoothing_bitwise(sd, n, bc):
    # all Chebyshev steps of a smoothing in one tiled kernel, prolongation folded
    # in, with 16-, 8- or 4-row tiles (0: by level size), and with tile 2 in
    # register-column tiles (cell blocks from 1024 cells per side): the same
    # arithmetic per point as the per-step kernels (n = 96: 97 faces per row, a
    # one-face ragged tile column; 97 = 3 * 26 + 19, a ragged register strip;
    # bc 2: the traction sides' rows)
    K = I.lognormal_K(n, -4.0, 1.0, 16.0, seed=11)
    xs = []
    for tile, rows in ((0, 16), (1, 16), (1, 8), (1, 4), (1, 0), (2, 16), (2, 8), (2, 4), (2, 0)):
        h = make(sd, n, 1e-3, K, 1.0, 0.05, 1, tile=tile, tile_rows=rows, bc=bc, bc_dp=1.0)
        sd.sd_step(h, 3)
        xs.append(sd.sd_get_state(h)[2])
    for x in xs[1:]:
        assert np.array_equal(xs[0], x)


def test_autotune(sd, tmp_path):
    # the tuner returns a candidate of its grid, caches it, and the tuned
    # solver still matches the oracle's direct solves
    n = 48
    K = I.lognormal_K(n, -4.0, 1.0, 16.0, seed=12)
    base = sd.sd_options_default()
    base.rtol = 1e-12
    cache = str(tmp_path / "tune.txt")
    best, ms = sd.sd_autotune(n, 1e-3, K, 1.0, 0.05, base, 1, cache)
    assert ms > 0
    assert best.tile_rows in (0, 8, 16) and best.coarsest in (4, 8, 16) and best.cheb_degree in (2, 3, 4)
    assert best.rtol == base.rtol and best.restart == base.restart
    lines = open(cache).read().splitlines()
    assert len(lines) == 1 and lines[0].startswith("sdtune2 ")
    again, ms2 = sd.sd_autotune(n, 1e-3, K, 1.0, 0.05, base, 1, cache)
    assert (again.tile_rows, again.coarsest, again.cheb_degree) == (best.tile_rows, best.coarsest, best.cheb_degree)
    assert abs(ms2 - ms) <= 1e-6 * ms and len(open(cache).read().splitlines()) == 1
    o = O.Oracle(n, 1e-3, 1.0, 0.05, K)
    xr = o.run(O.exact(n, 0.0, 1e-3), 0.0, 2)
    h = sd.sd_create(n, 1e-3, K, 1.0, 0.05, best)
    sd.sd_step(h, 2)
    for k, e in fields_rel(sd.sd_get_state(h)[2], xr, n).items():
        assert e <= 1e-8, (k, e)


@pytest.mark.parametrize("n,precision", [(24, 1), (40, 0), (64, 1)])
def test_partitioned_coupling_parity(sd, n, precision):
    # Sec. 3 coupling (Darcy solve with the interface flux, free-flow solve with the
    # pressure below, IQN-ILS on the interface velocity) against the oracle's
    # monolithic direct solves: the coupled state is the monolithic solution, to the
    # coupling tolerance; the number of coupling iterations matches the oracle's own
    # partitioned iteration with exact subdomain solves within one
    from oracle.partitioned import DNOracle
    K = I.lognormal_K(n, -4.0, 1.0, 16.0, seed=20 + n)
    o = O.Oracle(n, 1e-3, 1.0, 0.05, K)
    x0 = O.exact(n, 0.0, 1e-3)
    xr = o.run(x0, 0.0, 2)
    h = make(sd, n, 1e-3, K, 1.0, 0.05, precision, rtol=1e-12, coupling=sd.SD_PARTITIONED, coupling_eps=1e-10)
    infos = sd.sd_step(h, 2)
    assert all(i["status"] == 0 and i["coupling_iters"] >= 2 for i in infos)
    assert all(i["relres"] <= 1e-9 for i in infos)
    for k, e in fields_rel(sd.sd_get_state(h)[2], xr, n).items():
        assert e <= 1e-7, (k, e)
    # first step from the same initial state: coupling iterations vs the oracle's
    d = DNOracle(o, K)
    b = o.rhs(x0, 0.05)
    _, evals = d.solve(b, O.split(x0, n)["v"][0].copy(), eps=1e-10)
    assert abs(infos[0]["coupling_iters"] - evals) <= 1, (infos[0]["coupling_iters"], evals)


@pytest.mark.parametrize("bc", [0, 2])
def test_partitioned_long_run_does_not_stall(sd, bc):
    # default options over many steps of the lognormal workload: the subdomain
    # solves run three decades below the coupling test, so every step's
    # coupling converges in a few iterations (with the solves at rtol = 1e-10
    # the iteration stalled at coupling_max on some steps); on the
    # pressure-driven problem the Darcy solves reach their rounding floor above
    # that tolerance and stop there (stagnation accepted at rtol)
    wl = I.lognormal_at_scale(256)
    o = sd.sd_options_default()
    o.coupling = sd.SD_PARTITIONED
    o.bc = bc
    h = sd.sd_create(256, wl.mu, wl.K(), wl.alpha, wl.dt, o)
    infos = sd.sd_step(h, 30, raise_on_error=False)
    assert all(i["status"] == 0 for i in infos), [i["status"] for i in infos]
    assert max(i["coupling_iters"] for i in infos) <= 10
    assert max(i["relres"] for i in infos) <= 1e-10


def test_partitioned_manufactured_solution(sd):
    # the manufactured case through the partitioned coupling matches the oracle's
    # monolithic run (mu = K = alpha = 1, dt = 0.1)
    n = 32
    K = np.ones(n * n)
    o = O.Oracle(n, 1.0, 1.0, 0.1, K)
    xr = o.run(O.exact(n, 0.0, 1.0), 0.0, 3)
    h = make(sd, n, 1.0, K, 1.0, 0.1, 0, rtol=1e-12, coupling=sd.SD_PARTITIONED, coupling_eps=1e-10)
    infos = sd.sd_step(h, 3)
    assert all(i["status"] == 0 for i in infos)
    for k, e in fields_rel(sd.sd_get_state(h)[2], xr, n).items():
        assert e <= 1e-7, (k, e)


# --------------------------------------------------------------- traction sides
# bc 1: manufactured solution with traction free-flow sides; bc 2: the paper's
# pressure-driven problem (Sec. 5)
@pytest.mark.parametrize("bc", [1, 2])
@pytest.mark.parametrize("n", [4, 5, 12, 40])
def test_traction_operator_parity(sd, n, bc):
    K = I.lognormal_K(n, -4.0, 1.5, 4.0, seed=30 + n)
    o = O.Oracle(n, 1e-3, 1.3, 0.05, K, bc=bc)
    h = make(sd, n, 1e-3, K, 1.3, 0.05, bc=bc)
    rng = np.random.default_rng(n)
    for _ in range(3):
        x = rng.standard_normal(o.ndof)
        assert rel(sd.sd_apply(h, x), o.apply(x)) <= 1e-13
    if n == 4:  # every column
        A = o.scipy_csr().toarray()
        scale = np.abs(A).max()
        for k in range(o.ndof):
            e = np.zeros(o.ndof)
            e[k] = 1.0
            assert np.abs(sd.sd_apply(h, e) - A[:, k]).max() <= 1e-14 * scale


@pytest.mark.parametrize("bc", [1, 2])
def test_traction_rhs_parity(sd, bc):
    n = 24
    K = I.lognormal_K(n, -4.0, 1.0, 4.0, seed=33)
    o = O.Oracle(n, 1e-3, 0.9, 0.05, K, bc=bc, dp=2.0, t_end=0.5)
    h = make(sd, n, 1e-3, K, 0.9, 0.05, bc=bc, bc_dp=2.0, bc_tend=0.5)
    rng = np.random.default_rng(4)
    for t in (0.05, 0.3, 0.73):
        xp = rng.standard_normal(o.ndof)
        assert rel(sd.sd_rhs(h, xp, t), o.rhs(xp, t)) <= 1e-13


@pytest.mark.parametrize("precision", [0, 1])
def test_traction_mms_time_stepping(sd, precision):
    n = 32
    K = np.ones((n, n))
    o = O.Oracle(n, 1.0, 1.0, 0.1, K, bc=1)
    xr = o.run(O.exact(n, 0.0, 1.0), 0.0, 5)
    h = make(sd, n, 1.0, K, 1.0, 0.1, precision, rtol=1e-12, bc=1)
    infos = sd.sd_step(h, 5)
    assert all(i["status"] == 0 for i in infos)
    for k, e in fields_rel(sd.sd_get_state(h)[2], xr, n).items():
        assert e <= 1e-8, (k, e)


@pytest.mark.parametrize("precision,n", [(0, 24), (1, 40), (1, 64)])
def test_pressure_driven_problem(sd, precision, n):
    # from rest, the inflow pressure rising over 10 steps; lognormal K
    K = I.lognormal_K(n, -4.0, 1.0, 16.0, seed=34)
    dt = 0.05
    o = O.Oracle(n, 1e-3, 1.0, dt, K, bc=2, dp=1.0, t_end=10 * dt)
    xr = o.run(np.zeros(o.ndof), 0.0, 6)
    h = make(sd, n, 1e-3, K, 1.0, dt, precision, rtol=1e-12, bc=2, bc_dp=1.0, bc_tend=10 * dt)
    infos = sd.sd_step(h, 6)
    assert all(i["status"] == 0 for i in infos)
    for k, e in fields_rel(sd.sd_get_state(h)[2], xr, n).items():
        assert e <= 1e-8, (k, e)


@pytest.mark.parametrize("geometry", [0, 1])
def test_darcy_schur_block_at_paper_parameters(sd, geometry):
    # the paper's own parameters (Sec. 5: K = 1e-6, mu = 1e-3, dt = 2e5, quasi-steady): the preconditioner's
    # Darcy block with the interface's Schur correction (darcy_schur = 1, the default) and without it reach
    # the oracle's states alike (the operator is the same), and the correction cuts the iterations
    n, dt = 32, 2e5
    K = np.full((n, n), 1e-6)
    o = O.Oracle(n, 1e-3, 1.0, dt, K, bc=2, dp=1e-9, t_end=50e5, geo=geometry)
    xr = o.run(np.zeros(o.ndof), 0.0, 4)
    its = {}
    for ds in (1, 0):
        h = make(sd, n, 1e-3, K, 1.0, dt, 1, rtol=1e-12, bc=2, bc_dp=1e-9, bc_tend=50e5, darcy_schur=ds,
                 geometry=geometry)
        infos = sd.sd_step(h, 4)
        assert all(i["status"] == 0 for i in infos)
        its[ds] = sum(i["iters"] for i in infos)
        fs, fr = O.split(sd.sd_get_state(h)[2], n, geometry), O.split(xr, n, geometry)
        for k in fs:
            assert rel(fs[k], fr[k]) <= 1e-8, (ds, k)
    assert its[1] <= 0.7 * its[0], its


def test_pressure_driven_partitioned(sd):
    # the partitioned coupling of Sec. 3 on the paper's problem
    n = 32
    K = I.lognormal_K(n, -4.0, 1.0, 16.0, seed=35)
    dt = 0.05
    o = O.Oracle(n, 1e-3, 1.0, dt, K, bc=2, dp=1.0, t_end=10 * dt)
    xr = o.run(np.zeros(o.ndof), 0.0, 4)
    h = make(sd, n, 1e-3, K, 1.0, dt, 1, rtol=1e-12, bc=2, bc_dp=1.0, bc_tend=10 * dt,
             coupling=sd.SD_PARTITIONED, coupling_eps=1e-10)
    infos = sd.sd_step(h, 4)
    assert all(i["status"] == 0 for i in infos)
    for k, e in fields_rel(sd.sd_get_state(h)[2], xr, n).items():
        assert e <= 1e-7, (k, e)


@pytest.mark.parametrize("bc,order", [(1, 1), (2, 1), (2, 2)])
def test_partitioned_orders_with_traction_sides(sd, bc, order):
    # both orders of the subdomain solves (2: Sec. 3's, free flow first with the
    # velocity prescribed; 1: porous medium first) on traction-side problems:
    # the coupled state matches the oracle's monolithic step.  Porous medium
    # first: the coupling iteration count matches the oracle's own iteration
    # within one.  Free flow first: its map multiplies the free-flow solve's
    # error by 2K/(mu h) (about 900 here) and its free-flow solves are slow (the
    # velocity V-cycle treats the prescribed interface velocity as unknown), so
    # the coupling tolerance is 1e-8 and the count may exceed the oracle's
    # (exact subdomain solves) by a few.  Its convergence is erratic in the
    # preconditioner: measured here, it converges with the hierarchy coarsened
    # to 4 cells (25 coupling iterations) but not with the coarsest grid at 8
    # (FP32 V-cycles) or at 12 (FP64), where the porous-medium-first order
    # takes 6 at every depth; this case therefore pins coarsest = 4.
    from oracle.partitioned import DNOracle
    n, dt, mu = 24, 0.05, 1e-3
    eps = 1e-10 if order == 1 else 1e-8
    K = I.lognormal_K(n, -4.0, 1.0, 16.0, seed=40 + bc)
    o = O.Oracle(n, mu, 1.0, dt, K, bc=bc, dp=1.0, t_end=10 * dt)
    x0 = O.exact(n, 0.0, mu) if bc == 1 else np.zeros(o.ndof)
    b = o.rhs(x0, dt)
    xr = o.solve(b)
    h = make(sd, n, mu, K, 1.0, dt, 0, rtol=1e-12, bc=bc, bc_dp=1.0, bc_tend=10 * dt,
             coupling=sd.SD_PARTITIONED, coupling_eps=eps, coupling_order=order,
             coarsest=16 if order == 1 else 4)
    info = sd.sd_step(h, 1)[0]
    assert info["status"] == 0
    for k, e in fields_rel(sd.sd_get_state(h)[2], xr, n).items():
        assert e <= (1e-7 if order == 1 else 1e-5), (k, e)
    d = DNOracle(o, K, order="paper" if order == 2 else "pm")
    _, evals = d.solve(b, O.split(x0, n)["v"][0].copy(), eps=eps)
    if order == 1:
        assert abs(info["coupling_iters"] - evals) <= 1, (info["coupling_iters"], evals)
    else:
        assert info["coupling_iters"] <= evals + 6, (info["coupling_iters"], evals)


@pytest.mark.parametrize("coupling", [0, 1])
def test_block_residuals(sd, coupling):
    # the per-block residuals split the reported relative residual:
    # relres^2 = relres_v^2 + relres_pff^2 + relres_pm^2; also in a lockstep batch
    n = 32
    K = I.lognormal_K(n, -4.0, 1.0, 16.0, seed=50)
    h = make(sd, n, 1e-3, K, 1.0, 0.05, 1, coupling=coupling)
    for info in sd.sd_step(h, 3):
        parts = np.array([info["relres_v"], info["relres_pff"], info["relres_pm"]])
        assert np.all(parts >= 0)
        assert abs(np.sqrt((parts ** 2).sum()) - info["relres"]) <= 1e-6 * info["relres"] + 1e-300
    if coupling == 0:
        hs = [make(sd, n, 1e-3, I.lognormal_K(n, -4.0, 1.0, 16.0, seed=51 + q), 1.0, 0.05, 1) for q in range(3)]
        for inf in sd.sd_solve_batch(hs, [2, 2, 2]):
            for info in inf:
                parts = np.array([info["relres_v"], info["relres_pff"], info["relres_pm"]])
                assert abs(np.sqrt((parts ** 2).sum()) - info["relres"]) <= 1e-6 * info["relres"]
