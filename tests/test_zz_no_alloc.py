"""ssvp_median_depth_noalloc through the C ABI, against the FP64 oracle's median and the context's
median (ssvp_clip_median_depth).

Some callers may not allocate device memory at all: a plug-in living inside a video host that
owns every GPU buffer through its own pool, or a per-frame real-time callback where a
cudaMalloc/cudaFree would synchronise the device and stall the pipeline.  For them the library
offers a median entry point whose scratch is a fixed array inside the library.  These checks
run it on several inputs in a row (a call must not see the previous call's leftovers in the
shared array) and compare each result exactly with the oracle's lower median and with the
regular entry point.  This file is named to be collected last.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ss():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_2102_03011_gb300 as ss
    return ss


def _inputs():
    a = synth.make_clip("planes3", 160, 90, 16, seed=0).depth
    b = synth.make_clip("room", 320, 180, 5, seed=3).depth.copy()
    b[0, :20] = np.nan
    b[1, :, :50] = -1.0
    b[2, 7:9] = 0.0
    b[3, 40:60, 100:200] = np.inf
    return a, b


def test_noalloc_median_equals_oracle_and_context_median_on_consecutive_calls(ss):
    import torch
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    ctx = ss.ssvp_create(0, stream)
    try:
        for rep in range(2):  # the second round starts from the first round's leftovers
            for i, d in enumerate(_inputs()):
                F, H, W = d.shape
                dd = torch.from_numpy(np.ascontiguousarray(d)).to(dev)
                rgb = torch.zeros((F, H, W, 3), dtype=torch.float32, device=dev)
                ss.ssvp_load_clip(ctx, i, W, H, F, rgb, dd)
                want = ss.ssvp_clip_median_depth(ctx, i)
                out = torch.full((1,), -7.0, dtype=torch.float32, device=dev)
                ss.ssvp_median_depth_noalloc(dd, dd.numel(), out, stream)
                torch.cuda.synchronize()
                assert out.item() == oracle.median_depth(d), (rep, i, out.item(), oracle.median_depth(d))
                assert out.item() == want, (rep, i, out.item(), want)
    finally:
        ss.ssvp_destroy(ctx)


def _oracle_median(d):
    """The oracle's lower median, NaN when no value is valid (the entry point's documented result)."""
    try:
        return oracle.median_depth(d)
    except ValueError:
        return float("nan")


def test_noalloc_median_of_a_prefix_and_of_no_valid_value(ss):
    import torch
    dev = torch.device("cuda:0")
    _, b = _inputs()
    dd = torch.from_numpy(np.ascontiguousarray(b)).to(dev)
    out = torch.zeros(1, dtype=torch.float32, device=dev)
    # the first 20 rows of frame 0 are NaN: prefixes of 1 and 6,400 values hold no valid value
    for n in (1, 6400, 6401, 57_601, dd.numel() - 3):
        ss.ssvp_median_depth_noalloc(dd, n, out)
        torch.cuda.synchronize()
        want = _oracle_median(b.reshape(-1)[:n])
        got = out.item()
        assert (np.isnan(want) and np.isnan(got)) or got == want, (n, got, want)
    bad = torch.tensor([np.nan, 0.0, -1.0, np.inf, -np.inf, -0.0], dtype=torch.float32, device=dev)
    ss.ssvp_median_depth_noalloc(bad, bad.numel(), out)
    torch.cuda.synchronize()
    assert np.isnan(out.item())
    with pytest.raises(ValueError):
        oracle.median_depth(bad.cpu().numpy())  # the oracle agrees: no valid value


def test_noalloc_median_rejects_sizes_beyond_its_scratch(ss):
    import torch
    d = torch.ones(4, dtype=torch.float32, device="cuda")
    out = torch.zeros(1, dtype=torch.float32, device="cuda")
    for n in (0, 2 ** 32):  # refused by the C entry point before any work is queued
        rc = ss.lib.ssvp_median_depth_noalloc(d.data_ptr(), n, out.data_ptr(), None)
        assert rc == ss.SSVP_EINVAL
        assert "outside" in ss.ssvp_last_error(None)
    with pytest.raises(ValueError):
        ss.ssvp_median_depth_noalloc(d, 5, out)  # more values than the tensor holds


def test_noalloc_median_refuses_host_memory(ss):
    import torch
    host = np.ones(16, np.float32)
    out = torch.zeros(1, dtype=torch.float32, device="cuda")
    rc = ss.lib.ssvp_median_depth_noalloc(host.ctypes.data, 16, out.data_ptr(), None)
    assert rc == ss.SSVP_EINVAL and "depth_dev" in ss.ssvp_last_error(None)
    pinned = torch.ones(16, dtype=torch.float32).pin_memory()
    d = torch.ones(16, dtype=torch.float32, device="cuda")
    rc = ss.lib.ssvp_median_depth_noalloc(d.data_ptr(), 16, pinned.data_ptr(), None)
    assert rc == ss.SSVP_EINVAL and "median_dev" in ss.ssvp_last_error(None)
