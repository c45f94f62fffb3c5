"""The C ABI without a GPU: the library builds, loads and exports every entry
point include/sd.h declares; host-side validation and sizes."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_functions():
    src = open(os.path.join(ROOT, "include", "sd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sd_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def sd():
    from paper_2108_13229_gb300 import build as B
    from paper_2108_13229_gb300 import sd as S
    if not os.path.exists(S.lib_path()):
        B.build_library()
    S._load()
    return S


def test_exports_every_declared_function(sd):
    import ctypes
    lib = ctypes.CDLL(sd.lib_path())
    names = _header_functions()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name
    # the binding wraps every declared function under the same name
    for name in names:
        assert hasattr(sd, name), name


def test_dof_count_table1(sd):
    for line in open(os.path.join(ROOT, "tests", "golden", "table1.txt")):
        if line.strip() and not line.startswith("#"):
            n, dof, _ = line.split()
            assert sd.sd_dof_count(int(n)) == int(dof)


def test_dof_count_geometry(sd):
    # the channel's count is the oracle's (a different library, the same layout)
    import oracle as O
    for n in (2, 4, 5, 64, 1024):
        assert sd.sd_dof_count_geometry(n, sd.SD_GEO_SQUARE) == sd.sd_dof_count(n)
        assert sd.sd_dof_count_geometry(n, sd.SD_GEO_CHANNEL) == O.dof_count(n, 1) == 10 * n * n + 4 * n
    assert sd.sd_dof_count_geometry(4, 7) == -1
    assert sd.sd_options_default().geometry == sd.SD_GEO_SQUARE


def test_options_default(sd):
    o = sd.sd_options_default()
    assert o.restart == 30 and o.rtol == 1e-10 and o.precision == sd.SD_MIXED
    assert o.precond == sd.SD_TRI_SCHUR and o.cheb_degree >= 1 and o.schur_gamma == 0.5 and o.schur_mass == 1


def test_memory_estimate(sd):
    e = [sd.sd_memory_estimate(n) for n in (32, 64, 128, 1024)]
    assert all(v > 0 for v in e) and e == sorted(e)
    o = sd.sd_options_default()
    o.precision = sd.SD_FP64
    assert sd.sd_memory_estimate(1024, o) > sd.sd_memory_estimate(1024)
    # grids that cannot coarsen to <= 16 cells are rejected
    assert sd.sd_memory_estimate(34) == -1


def test_validation_without_gpu(sd):
    n = 8
    K = np.ones((n, n))
    for args in [(n, -1.0, K, 1.0, 0.1), (n, 1.0, K, 0.0, 0.1), (n, 1.0, K, 1.0, 0.0), (34, 1.0, np.ones((34, 34)), 1.0, 0.1)]:
        with pytest.raises(sd.SdError) as e:
            sd.sd_create(*args)
        assert e.value.code == sd.SD_E_INVAL
    Kb = K.copy()
    Kb[3, 4] = np.nan
    with pytest.raises(sd.SdError) as e:
        sd.sd_create(n, 1.0, Kb, 1.0, 0.1)
    assert e.value.code == sd.SD_E_INVAL
    Kb[3, 4] = -1.0
    with pytest.raises(sd.SdError) as e:
        sd.sd_create(n, 1.0, Kb, 1.0, 0.1)
    assert e.value.code == sd.SD_E_INVAL
    o = sd.sd_options_default()
    o.restart = 31
    with pytest.raises(sd.SdError):
        sd.sd_create(n, 1.0, K, 1.0, 0.1, o)
    assert sd.sd_strerror(sd.SD_E_NOCONV).startswith("FGMRES")


def test_struct_layout_matches_binding(sd):
    import ctypes
    for k, cls in enumerate([sd.sd_grid, sd.sd_options, sd.sd_step_info, sd.sd_request, sd.sd_result]):
        assert sd.sd_struct_size(k) == ctypes.sizeof(cls), cls.__name__


def test_option_validation_without_gpu(sd):
    # every option is checked on the host before any device work
    n = 8
    K = np.ones((n, n))
    g = sd.sd_grid(n, n)
    bad = [("bc", 3), ("bc", -1), ("coupling", 2), ("coupling_order", 3), ("tile_rows", 12),
           ("cheb_degree", 0), ("cheb_degree", 9), ("coarsest", 1), ("darcy_coupled", 3), ("orth", 2),
           ("bc_tend", -1.0), ("bc_dp", float("nan")), ("graph", 3), ("graph", -1)]
    for field, value in bad:
        o = sd.sd_options_default()
        setattr(o, field, value)
        assert sd._load().sd_memory_estimate(ctypes.byref(g), ctypes.byref(o)) == -1, field
        with pytest.raises(sd.SdError) as e:
            sd.sd_create(n, 1.0, K, 1.0, 0.1, o)
        assert e.value.code == sd.SD_E_INVAL, field
    # partitioned coupling: its parameters, and Sec. 3's order needs traction sides
    for field, value in [("coupling_columns", 0), ("coupling_columns", 31), ("coupling_eps", 0.0),
                         ("coupling_omega", 0.0), ("coupling_max", 0), ("coupling_rtol", -1e-12),
                         ("coupling_rtol", 1.0)]:
        o = sd.sd_options_default()
        o.coupling = sd.SD_PARTITIONED
        setattr(o, field, value)
        assert sd._load().sd_memory_estimate(ctypes.byref(g), ctypes.byref(o)) == -1, field
    o = sd.sd_options_default()
    o.coupling = sd.SD_PARTITIONED
    o.coupling_order = sd.SD_ORDER_FF_FIRST
    assert sd._load().sd_memory_estimate(ctypes.byref(g), ctypes.byref(o)) == -1
    o.bc = sd.SD_BC_PAPER
    assert sd._load().sd_memory_estimate(ctypes.byref(g), ctypes.byref(o)) > 0
    # the partitioned state adds the subdomain right-hand side and the IQN-ILS columns
    base = sd.sd_options_default()
    assert sd._load().sd_memory_estimate(ctypes.byref(g), ctypes.byref(o)) > \
        sd._load().sd_memory_estimate(ctypes.byref(g), ctypes.byref(base))
    # valid boundary modes
    for bc in (sd.SD_BC_MMS, sd.SD_BC_MMS_TRACTION, sd.SD_BC_PAPER):
        o = sd.sd_options_default()
        o.bc = bc
        assert sd._load().sd_memory_estimate(ctypes.byref(g), ctypes.byref(o)) > 0


def test_batch_validation_without_gpu(sd):
    # rejected before any handle is read: NULL handles, negative step counts,
    # a handle listed twice (the stand-in handles point at zeroed host memory)
    lib = sd._load()
    blob = ctypes.create_string_buffer(1 << 16)
    a, b = ctypes.addressof(blob), ctypes.addressof(blob) + 4096
    for hs, ns in [([a, None], [1, 1]), ([a, b], [1, -1]), ([a, a], [1, 1]), ([a, b, a], [2, 2, 2])]:
        arr = (ctypes.c_void_p * len(hs))(*hs)
        steps = (ctypes.c_int32 * len(ns))(*ns)
        for flags in (0, sd.SD_BATCH_LOCKSTEP, sd.SD_BATCH_LOCKSTEP | sd.SD_BATCH_GRAPH):
            assert lib.sd_solve_batch_ex(arr, len(hs), steps, None, 0, flags) == sd.SD_E_INVAL, (hs, ns)
    assert lib.sd_solve_batch_ex(None, 0, None, None, 0, 0) == sd.SD_OK
    assert lib.sd_solve_batch_ex(None, 1, None, None, 0, 0) == sd.SD_E_INVAL


def test_server_admission_without_gpu(sd):
    # the server checks every request on the host at submission: bad sizes and
    # step counts, and runs whose device memory exceeds the whole budget
    with pytest.raises(sd.SdError) as e:
        sd.sd_server_create(0, 2)
    assert e.value.code == sd.SD_E_INVAL
    srv = sd.sd_server_create(int(sd.sd_memory_estimate(32) * 1.5), 2)
    for n, steps, code in [(64, 5, sd.SD_E_NOMEM), (34, 5, sd.SD_E_INVAL), (32, -1, sd.SD_E_INVAL)]:
        with pytest.raises(sd.SdError) as e:
            sd.sd_submit(srv, n, 1e-3, np.ones((n, n)), 1.0, 0.1, steps)
        assert e.value.code == code, (n, steps)
    assert sd.sd_poll(srv, 12345)[0] == sd.SD_E_STATE
    sd.sd_server_drain(srv)  # nothing queued: returns at once
    del srv


def test_autotune_cache_without_gpu(sd, tmp_path):
    # a cache hit returns the stored choice with no device work; lines for
    # another key, or with options sd_create would reject, are skipped
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("the cache key names the device; this test writes the no-device key")
    n = 32
    K = np.ones((n, n))
    o = sd.sd_options_default()
    key = "sdtune2 unknown %d %d %d %d %d %d %d %.17g" % (n, o.precision, o.precond, o.darcy_coupled, o.restart,
                                                         o.bc, o.coupling, o.rtol)
    path = tmp_path / "tune.txt"
    path.write_text("\n".join([
        "garbage line",
        key + " 8 4 2 1.5",
        key.replace(" %d " % n, " 64 ", 1) + " 16 16 3 0.5",   # another grid size
        key.replace("%.17g" % o.rtol, "1e-08") + " 16 8 4 0.25",  # another rtol
        key + " 12 4 2 0.1",                                     # tile_rows 12 is invalid
        key + " 8 1 2 0.1",                                      # coarsest 1 is invalid
    ]) + "\n")
    best, ms = sd.sd_autotune(n, 1.0, K, 1.0, 0.1, None, 3, str(path))
    assert (best.tile_rows, best.coarsest, best.cheb_degree, ms) == (8, 4, 2, 1.5)
    assert best.rtol == o.rtol and best.restart == o.restart
    path.write_text(key + " 8 4 2 1.5\n" + key + " 16 8 3 0.75\n")
    best, ms = sd.sd_autotune(n, 1.0, K, 1.0, 0.1, None, 3, str(path))
    assert (best.tile_rows, best.coarsest, best.cheb_degree, ms) == (16, 8, 3, 0.75)  # the last line wins
    with pytest.raises(sd.SdError) as e:
        sd.sd_autotune(n, 1.0, K, 1.0, 0.1, None, 0, str(path))
    assert e.value.code == sd.SD_E_INVAL
    # only invalid matching lines: the tuner times candidates, which cannot
    # run without a device, so none converges and nothing is appended
    path.write_text(key + " 12 4 2 0.1\n")
    with pytest.raises(sd.SdError) as e:
        sd.sd_autotune(n, 1.0, K, 1.0, 0.1, None, 3, str(path))
    assert e.value.code == sd.SD_E_NOCONV
    assert path.read_text() == key + " 12 4 2 0.1\n"


def test_apply_noalloc_validation_without_gpu(sd):
    # checked on the host before any device work: the fixed capacity, the
    # physical parameters, and device memory for every array
    for n, mu, dt in [(sd.SD_NOALLOC_MAX_N * 2, 1.0, 0.1), (8, -1.0, 0.1), (8, 1.0, 0.0), (8, 1.0, 0.1)]:
        d = 4 * n * n + 2 * n
        with pytest.raises(sd.SdError) as e:
            sd.sd_apply_noalloc(n, mu, np.ones(n * n), 1.0, dt, np.zeros(d), np.zeros(d))
        assert e.value.code == sd.SD_E_INVAL, (n, mu, dt)
    # arrays shorter than the layout are refused by the binding itself
    n = 8
    d = 4 * n * n + 2 * n
    with pytest.raises(ValueError):
        sd.sd_apply_noalloc(n, 1.0, np.ones(n * n), 1.0, 0.1, np.zeros(d - 1), np.zeros(d))
    with pytest.raises(ValueError):
        sd.sd_apply_noalloc(n, 1.0, np.ones(n * n), 1.0, 0.1, np.zeros(d), np.zeros(d - 1))


def test_server_reserves_each_runs_own_depth(sd):
    # a server made without options runs short requests (under 40 steps) with
    # a 4 x 4 coarsest grid and long ones with 16 x 16; it reserves for each
    # the memory of the run it will create, so a budget between the two fits
    # the short request and refuses the long one
    import ctypes
    n = 64
    est = {}
    for co in (4, 16):
        o = sd.sd_options_default()
        o.coarsest = co
        g = sd.sd_grid(n, n)
        est[co] = sd._load().sd_memory_estimate(ctypes.byref(g), ctypes.byref(o))
    slack = 4 << 20  # setup temporaries reserved with every run
    assert est[4] < est[16]
    srv = sd.sd_server_create((est[4] + est[16]) // 2 + slack, 1)
    with pytest.raises(sd.SdError) as e:
        sd.sd_submit(srv, n, 1e-3, np.ones((n, n)), 1.0, 0.1, 50)
    assert e.value.code == sd.SD_E_NOMEM
    ticket = sd.sd_submit(srv, n, 1e-3, np.ones((n, n)), 1.0, 0.1, 5)
    sd.sd_server_drain(srv)  # without a device the run ends with SD_E_CUDA; with one it completes
    assert sd.sd_poll(srv, ticket)[0] in (sd.SD_OK, sd.SD_E_CUDA)
    del srv


@pytest.mark.parametrize("lockstep", [False, True])
def test_server_lifecycle_without_gpu(sd, lockstep):
    # drain returns once every request has ended (without a device each run
    # ends with SD_E_CUDA at its setup), a ticket is answered once, and a
    # server destroyed with requests still queued or running shuts down
    srv = sd.sd_server_create(1 << 30, 2, lockstep=lockstep)
    tickets = [sd.sd_submit(srv, 32, 1e-3, np.ones((32, 32)), 1.0, 0.1, 5) for _ in range(4)]
    sd.sd_server_drain(srv)
    for t in tickets:
        rc, res, _ = sd.sd_poll(srv, t)
        assert rc in (sd.SD_OK, sd.SD_E_CUDA) and res["status"] == rc
        assert sd.sd_poll(srv, t)[0] == sd.SD_E_STATE
    busy = sd.sd_server_create(1 << 30, 2, lockstep=lockstep)
    for _ in range(6):
        sd.sd_submit(busy, 32, 1e-3, np.ones((32, 32)), 1.0, 0.1, 5)
    del busy
    del srv
