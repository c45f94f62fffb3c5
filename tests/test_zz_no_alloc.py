"""sd_apply_noalloc: the coupled operator y = A x for callers that cannot
allocate device memory (fixed memory pools, real-time loops, code that may
not create a handle).  Its result must equal the handle-based sd_apply, call
after call, although every call reuses the same fixed device array."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_apply_noalloc_matches_sd_apply():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_13229_gb300 import inputs as I
    from paper_2108_13229_gb300 import sd
    dev = torch.device("cuda", 0)
    # calls in a row on the shared array: a small grid, the largest allowed
    # grid, then the small grid again with other inputs (stale contents of the
    # larger call must not leak into the result)
    nmax = sd.SD_NOALLOC_MAX_N
    cases = [(40, 1e-3, 1.3, 0.05, 11), (nmax, 1e-3, 1.0, 0.05, 12), (40, 0.7, 0.4, 0.2, 13)]
    for n, mu, alpha, dt, seed in cases:
        K = I.lognormal_K(n, -4.0, 1.0, 16.0, seed=seed)
        x = np.random.default_rng(seed).standard_normal(4 * n * n + 2 * n)
        h = sd.sd_create(n, mu, K, alpha, dt)
        y_ref = sd.sd_apply(h, x)
        sd.sd_destroy(h)
        Kd = torch.from_numpy(np.ascontiguousarray(K)).to(dev)
        xd = torch.from_numpy(x).to(dev)
        yd = torch.full_like(xd, float("nan"))
        sd.sd_apply_noalloc(n, mu, Kd, alpha, dt, xd, yd)
        torch.cuda.synchronize()
        assert _rel(yd.cpu().numpy(), y_ref) <= 1e-13, (n, seed)


def test_apply_noalloc_rejects():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_13229_gb300 import sd
    dev = torch.device("cuda", 0)
    n = 512  # beyond the fixed capacity
    K = torch.ones(n * n, dtype=torch.float64, device=dev)
    x = torch.zeros(4 * n * n + 2 * n, dtype=torch.float64, device=dev)
    with pytest.raises(sd.SdError) as e:
        sd.sd_apply_noalloc(n, 1.0, K, 1.0, 0.1, x, torch.empty_like(x))
    assert e.value.code == sd.SD_E_INVAL
    n = 8  # tensors shorter than 4n^2+2n are refused before any device work
    K = torch.ones(n * n, dtype=torch.float64, device=dev)
    x = torch.zeros(4 * n * n + 2 * n, dtype=torch.float64, device=dev)
    with pytest.raises(ValueError):
        sd.sd_apply_noalloc(n, 1.0, K, 1.0, 0.1, x[:-1], torch.empty_like(x))
    with pytest.raises(ValueError):
        sd.sd_apply_noalloc(n, 1.0, K, 1.0, 0.1, x, torch.empty_like(x)[:-1])
    # host memory is not accepted
    with pytest.raises(sd.SdError) as e:
        sd.sd_apply_noalloc(n, 1.0, np.ones(n * n), 1.0, 0.1, np.zeros(4 * n * n + 2 * n), np.zeros(4 * n * n + 2 * n))
    assert e.value.code == sd.SD_E_INVAL
