"""The allocation-free C^H entry point against the regular one.

shl_chom_noalloc serves callers that cannot allocate device memory (code
inside another framework's memory pool, or a latency-critical loop where
cudaMalloc may stall); its scratch is a fixed array inside the library.  This
file runs last so that, if it fails, a stop-at-first-failure run has already
run every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_2511_04025_b300 import shl  # noqa: E402

DEV = "cuda:0"


def _case(r, seed):
    rng = np.random.default_rng(seed)
    m = (rng.uniform(size=r ** 3) < 0.35).astype(np.uint8)
    u = rng.standard_normal((6, r ** 3, 3)) * 0.01
    return torch.tensor(m, device=DEV), torch.tensor(oracle.aos_to_soa(u), device=DEV)


def test_chom_noalloc_matches_chom_on_two_calls_in_a_row():
    if not torch.cuda.is_available():
        pytest.fail("no CUDA device: GPU tests need a B300")
    with shl.Context(0) as c:
        for r, seed in ((24, 1), (17, 2)):
            mask, u = _case(r, seed)
            ref = shl.shl_chom(c.handle, r, u, mask=mask)
            C_dev = torch.full((36,), float("nan"), dtype=torch.float64, device=DEV)
            shl.shl_chom_noalloc(r, u, C_dev, mask=mask)
            torch.cuda.synchronize()
            C = C_dev.cpu().numpy().reshape(6, 6)
            assert np.abs(C - ref).max() <= 1e-13 * np.abs(ref).max()


def test_chom_noalloc_rejects_oversized_grid():
    C_dev = torch.empty(36, dtype=torch.float64, device=DEV)
    u = torch.empty(18, dtype=torch.float64, device=DEV)
    with pytest.raises(shl.ShlError) as e:
        shl.shl_chom_noalloc(513, u, C_dev, mask=torch.empty(1, dtype=torch.uint8, device=DEV))
    assert e.value.status == shl.SHL_EINVAL and "512" in str(e.value)


def test_chom_noalloc_smoothed_density_matches_oracle_on_a_side_stream():
    """Smoothed density rho at r = 16 on a non-blocking stream (only that
    stream is synchronised), against the oracle's energy sum on the same u."""
    r = 16
    rng = np.random.default_rng(5)
    rho = rng.uniform(0.0, 1.0, r ** 3)
    u = rng.standard_normal((6, r ** 3, 3)) * 0.02
    ref, _ = oracle.chom(r, rho, u)
    s = torch.cuda.Stream(device=DEV)
    with torch.cuda.stream(s):
        rho_d = torch.tensor(rho, device=DEV)
        u_d = torch.tensor(oracle.aos_to_soa(u), device=DEV)
        C_dev = torch.full((36,), float("nan"), dtype=torch.float64, device=DEV)
    for _ in range(2):
        shl.shl_chom_noalloc(r, u_d, C_dev, rho=rho_d, stream=s)
        s.synchronize()
        C = C_dev.cpu().numpy().reshape(6, 6)
        assert np.abs(C - ref).max() <= 1e-12 * np.abs(ref).max()


def test_chom_noalloc_rejects_wrong_device_dtype_and_size():
    C_dev = torch.empty(36, dtype=torch.float64, device=DEV)
    u = torch.zeros(18 * 8 ** 3, dtype=torch.float64, device=DEV)
    m = torch.zeros(8 ** 3, dtype=torch.uint8, device=DEV)
    with pytest.raises(ValueError):
        shl.shl_chom_noalloc(8, u.cpu(), C_dev, mask=m)
    with pytest.raises(ValueError):
        shl.shl_chom_noalloc(8, u.float(), C_dev, mask=m)
    with pytest.raises(ValueError):
        shl.shl_chom_noalloc(9, u, C_dev, mask=m)
