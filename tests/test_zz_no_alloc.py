"""ssvp_median_depth_noalloc against the context's median (ssvp_clip_median_depth), via the C ABI.

Some callers may not allocate device memory at all: a plug-in living inside a video host that
owns every GPU buffer through its own pool, or a per-frame real-time callback where a
cudaMalloc/cudaFree would synchronise the device and stall the pipeline.  For them the library
offers a median entry point whose scratch is a fixed array inside the library.  These checks
run it twice in a row (the second call must not see the first call's leftovers) and compare
with the regular entry point, exactly, as the other median tests do.  This file is named to be
collected last.
"""
import numpy as np
import pytest

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


def test_noalloc_median_equals_context_median_on_consecutive_calls(ss):
    import torch
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    a = synth.make_clip("planes3", 160, 90, 16, seed=0).depth
    b = synth.make_clip("room", 320, 180, 5, seed=3).depth.copy()
    b[0, :20] = np.nan
    b[1, :, :50] = -1.0
    b[2, 7:9] = 0.0
    b[3, 40:60, 100:200] = np.inf
    ctx = ss.ssvp_create(0, stream)
    try:
        for i, d in enumerate((a, b)):
            F, H, W = d.shape
            dd = torch.from_numpy(np.ascontiguousarray(d)).to(dev)
            rgb = torch.zeros((F, H, W, 3), dtype=torch.float32, device=dev)
            ss.ssvp_load_clip(ctx, i, W, H, F, rgb, dd)
            want = ss.ssvp_clip_median_depth(ctx, i)
            out = torch.full((1,), float("nan"), dtype=torch.float32, device=dev)
            ss.ssvp_median_depth_noalloc(dd, dd.numel(), out, stream)
            torch.cuda.synchronize()
            assert out.item() == want, (i, out.item(), want)
    finally:
        ss.ssvp_destroy(ctx)


def test_noalloc_median_rejects_sizes_beyond_its_scratch(ss):
    import torch
    d = torch.ones(4, dtype=torch.float32, device="cuda")
    out = torch.zeros(1, dtype=torch.float32, device="cuda")
    for n in (0, 2 ** 32):
        with pytest.raises(ss.SsvpError) as e:
            ss.ssvp_median_depth_noalloc(d, n, out)
        assert e.value.code == ss.SSVP_EINVAL
        assert "outside" in str(e.value)
