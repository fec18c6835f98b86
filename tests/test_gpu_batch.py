"""The concurrent batch entry point (shl_homogenize_batch): each design's
C^H is the one shl_homogenize returns for it alone, grids and charge counts
may differ within a batch, the caller's stream orders the batch, and an
invalid member rejects the whole batch before anything runs."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2511_04025_b300 import inputs, shl  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.fail("no CUDA device: GPU tests need a B300")
    c = shl.Context(0, max_batch=4)
    yield c.handle
    c.close()


def _mix():
    ds = [inputs.random_design(40 + i, n, vf) for i, (n, vf) in enumerate([(8, 0.15), (24, 0.08), (12, 0.2),
                                                                             (64, 0.05), (8, 0.1), (16, 0.12)])]
    rs = [24, 32, 16, 32, 24, 20]
    return ds, rs


@pytest.mark.parametrize("prec", [shl.SHL_FP32_REFINE, shl.SHL_FP64])
def test_batch_matches_designs_alone(ctx, prec):
    ds, rs = _mix()
    o = shl.default_solve_opts(precision=prec, tol=1e-9)
    Cb, stb = shl.shl_homogenize_batch(ctx, ds, rs, o)
    assert Cb.shape == (len(ds), 6, 6)
    for d, r, C, st in zip(ds, rs, Cb, stb):
        Ca, sta = shl.shl_homogenize(ctx, d, r, o)
        assert st["status"] == shl.SHL_OK
        assert np.abs(C - Ca).max() <= 1e-12 * np.abs(Ca).max()
        assert st["iters"] == sta["iters"]
        assert st["n_solid"] == sta["n_solid"]


def test_batch_waits_for_the_callers_stream(ctx):
    """A batch queued behind a long device sleep on the caller's stream
    cannot finish before the sleep does."""
    ds, rs = _mix()
    o = shl.default_solve_opts(precision=shl.SHL_FP32_REFINE, tol=1e-7)
    shl.shl_homogenize_batch(ctx, ds[:3], rs[:3], o)  # warm: graphs and workspaces
    s = torch.cuda.Stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(s):
        e0.record(s)
        torch.cuda._sleep(200_000_000)
        e1.record(s)
    s.synchronize()
    sleep_s = e0.elapsed_time(e1) / 1e3
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        t0 = time.perf_counter()
        torch.cuda._sleep(200_000_000)
        shl.shl_homogenize_batch(ctx, ds[:3], rs[:3], o, stream=s)
        wall = time.perf_counter() - t0
    assert wall >= 0.8 * sleep_s, (wall, sleep_s)
    s.synchronize()


def test_batch_rejects_an_invalid_member_before_running(ctx):
    ds, rs = _mix()
    before = shl.shl_get_counters(ctx)["kernel_launches"]
    bad = ds[2].copy(vf=None, t=None)  # neither a thickness nor a volume fraction
    o = shl.default_solve_opts(precision=shl.SHL_FP32_REFINE, tol=1e-7)
    with pytest.raises(shl.ShlError) as e:
        shl.shl_homogenize_batch(ctx, ds[:2] + [bad] + ds[3:], rs, o)
    assert e.value.status == shl.SHL_EINVAL
    assert shl.shl_get_counters(ctx)["kernel_launches"] == before
    C, st = shl.shl_homogenize_batch(ctx, [], [], o)
    assert C.shape == (0, 6, 6) and st == []
