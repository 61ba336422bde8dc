"""Helpers for the GPU parity tests: run the C-ABI path on a clip and compare with the oracle."""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

import oracle

COLOUR_TOL = 1e-3  # max abs colour difference in FP32 against the FP64 oracle


@dataclass
class GpuResult:
    rgb: np.ndarray                 # (ch, cw, 3)
    nacc: np.ndarray | None = None
    nexam: np.ndarray | None = None
    sumw: np.ndarray | None = None
    status: np.ndarray | None = None  # (ch, cw, ns)
    centre: np.ndarray | None = None  # (ch, cw, ns, 2)
    bits: np.ndarray | None = None    # (ch, cw, ns, k, k) bool (aperture: cap x cap from the box origin)
    box: np.ndarray | None = None     # (ch, cw, ns, 4) aperture box x0, y0, x1, y1
    count: np.ndarray | None = None   # (ch, cw, ns) frustum gather: samples per window frame
    hash: np.ndarray | None = None    # (ch, cw, ns) uint64 frustum membership checksum


class Session:
    """One library context with clips loaded from synth.Clip objects (device buffers)."""

    def __init__(self):
        import torch
        import paper_2102_03011_gb300 as ss
        self.ss, self.torch = ss, torch
        self.dev = torch.device("cuda:0")
        self.stream = torch.cuda.current_stream(self.dev)
        self.ctx = ss.ssvp_create(0, self.stream)
        self.clips = {}

    def close(self):
        self.ss.ssvp_destroy(self.ctx)

    def load(self, cid, clip, colour_fmt=0, rgb=None, depth=None, K=None, w2c=None, host=False):
        t = self.torch
        rgb = clip.rgb if rgb is None else rgb
        depth = clip.depth if depth is None else depth
        F, H, W = depth.shape
        if host:
            r, d = np.ascontiguousarray(rgb), np.ascontiguousarray(depth)
        else:
            r, d = t.from_numpy(np.ascontiguousarray(rgb)).to(self.dev), t.from_numpy(np.ascontiguousarray(depth)).to(self.dev)
        self.ss.ssvp_load_clip(self.ctx, cid, W, H, F, r, d, None, colour_fmt)
        self.ss.ssvp_set_cameras(self.ctx, cid, clip.K if K is None else K, 1, clip.w2c if w2c is None else w2c)
        self.ss.ssvp_sync(self.ctx)
        self.clips[cid] = (W, H, F)

    def params(self, **kw):
        p = self.ss.ssvp_params_default()
        for k, v in kw.items():
            setattr(p, k, v)
        return p

    def run(self, cid, O, crop=None, membership=False, **kw) -> GpuResult:
        t, ss = self.torch, self.ss
        W, H, F = self.clips[cid]
        x0, y0, cw, ch = crop if crop is not None else (0, 0, W, H)
        p = self.params(frame_begin=O, frame_end=O + 1, crop_x=x0, crop_y=y0, crop_w=cw, crop_h=ch, **kw)
        ns = 2 * p.half_window + 1
        aperture = p.mode == ss.SSVP_MODE_APERTURE
        k = p.cap if aperture else p.k
        head = 5 if aperture else 3
        recw = head + (k * k + 31) // 32
        mem = stats = None
        if membership:
            mem = t.zeros((ch, cw, ns, recw), dtype=t.int32, device=self.dev)
            stats = t.zeros((ch, cw, 3), dtype=t.int32, device=self.dev)
            p.membership_out = mem.data_ptr()
            p.pixel_stats_out = stats.data_ptr()
        ss.ssvp_gather_filter(self.ctx, p, [cid])
        out = t.empty((1, H, W, 3), dtype=t.float32, device=self.dev)
        ss.ssvp_read_output(self.ctx, cid, O, O + 1, out)
        ss.ssvp_sync(self.ctx)
        rgb = out[0, y0:y0 + ch, x0:x0 + cw].cpu().numpy()
        res = GpuResult(rgb)
        if membership:
            m = mem.cpu().numpy()
            s = stats.cpu().numpy()
            res.nacc, res.nexam = s[..., 0].astype(np.int64), s[..., 1].astype(np.int64)
            res.sumw = s[..., 2].view(np.float32).astype(np.float64)
            res.status = m[..., 0]
            if aperture:
                res.box = m[..., 1:5]
            else:
                res.centre = m[..., 1:3]
            words = m[..., head:].view(np.uint32)
            b = np.arange(k * k)
            bits = (words[..., b >> 5] >> (b & 31).astype(np.uint32)) & 1
            res.bits = bits.reshape(ch, cw, ns, k, k).astype(bool)
        return res


def oracle_params(median, k, T, mode=oracle.MODE_DENOISE, radius_rel=0.005, **kw):
    return oracle.Params(mode=mode, k=k, T=T, radius=radius_rel * median, **kw)


def compare(g: GpuResult, o: oracle.Result, k: int):
    """Membership must match exactly except (a) windows whose centre lies within the tie band of a
    rounding tie (the oracle's `amb` flag), where the GPU may pick the neighbouring centre, and
    (b) candidates within 1e-5 relative of the radius (the oracle's band flag).  Pixels where such
    an allowed difference actually occurred are excluded from the colour and count comparison;
    every other pixel must match colour within COLOUR_TOL and counts exactly.  Returns a summary."""
    ch, cw, ns = o.status.shape
    amb = (o.amb == 1) & (o.status == 1)
    band = (o.codes & oracle.CODE_BAND) != 0
    o_acc = (o.codes & 7) == oracle.CODE_ACCEPT
    # GPU status 2 (window entirely outside the image) is oracle status 1 with no pixel inside
    o_none = (o.status == 1) & np.all((o.codes & 7) == oracle.CODE_OUT, axis=(-1, -2))
    g_stat = np.where(g.status == 2, 1, g.status)
    st_diff = o.status != g_stat
    assert not (st_diff & ~amb).any(), f"status mismatch at {np.argwhere(st_diff & ~amb)[:5]}"
    both = (o.status == 1) & (g.status == 1) & ~o_none
    cen_diff = both & np.any(o.centre != g.centre, axis=-1)
    assert not (cen_diff & ~amb).any(), f"window centre mismatch at {np.argwhere(cen_diff & ~amb)[:5]}"
    win_diff = st_diff | cen_diff
    cmp = both & ~cen_diff
    bit_diff = (o_acc != g.bits) & cmp[..., None, None]
    assert not (bit_diff & ~band).any(), \
        f"{int((bit_diff & ~band).sum())} membership differences, first {np.argwhere(bit_diff & ~band)[:5]}"
    excl = win_diff.any(-1) | bit_diff.any(axis=(-1, -2, -3))
    ok = ~excl
    cerr = np.abs(g.rgb.astype(np.float64) - o.rgb).max(-1)
    assert cerr[ok].max(initial=0.0) <= COLOUR_TOL, f"colour max abs {cerr[ok].max()} > {COLOUR_TOL}"
    np.testing.assert_array_equal(g.nacc[ok], o.nacc[ok])
    np.testing.assert_array_equal(g.nexam[ok], o.nexam[ok])
    np.testing.assert_allclose(g.sumw[ok], o.sumw[ok], rtol=1e-4)
    return dict(pixels=ch * cw, excluded=int(excl.sum()), members=int((o_acc & cmp[..., None, None]).sum()),
                max_colour_err=float(cerr[ok].max(initial=0.0)), max_colour_err_all=float(cerr.max()),
                band_candidates=int((band & (o.status == 1)[..., None, None]).sum()),
                band_flips=int(bit_diff.sum()), ambiguous_windows=int(amb.sum()), centre_flips=int(win_diff.sum()))


def compare_aperture(g: GpuResult, o: oracle.Result, cap: int):
    """Aperture membership: the scanned box must match except at flagged rounding ties of the
    seed projections; accepted bits must match except within 1e-5 of the cone radius; colour
    and counts are compared wherever no such allowed difference occurred."""
    amb = (o.amb == 1) & (o.status == 1)
    band = (o.codes & oracle.CODE_BAND) != 0
    o_acc = (o.codes & 7) == oracle.CODE_ACCEPT
    o_none = (o.status == 1) & np.all((o.codes & 7) == oracle.CODE_OUT, axis=(-1, -2))
    g_stat = np.where(g.status == 2, 1, g.status)
    st_diff = o.status != g_stat
    assert not (st_diff & ~amb).any(), f"status mismatch at {np.argwhere(st_diff & ~amb)[:5]}"
    both = (o.status == 1) & (g.status == 1) & ~o_none
    box_diff = both & np.any(o.box != g.box, axis=-1)
    assert not (box_diff & ~amb).any(), f"box mismatch at {np.argwhere(box_diff & ~amb)[:5]}"
    cmp = both & ~box_diff
    bit_diff = (o_acc != g.bits) & cmp[..., None, None]
    assert not (bit_diff & ~band).any(), \
        f"{int((bit_diff & ~band).sum())} membership differences, first {np.argwhere(bit_diff & ~band)[:5]}"
    excl = (st_diff | box_diff).any(-1) | bit_diff.any(axis=(-1, -2, -3))
    ok = ~excl
    cerr = np.abs(g.rgb.astype(np.float64) - o.rgb).max(-1)
    assert cerr[ok].max(initial=0.0) <= COLOUR_TOL, f"colour max abs {cerr[ok].max()} > {COLOUR_TOL}"
    np.testing.assert_array_equal(g.nacc[ok], o.nacc[ok])
    np.testing.assert_array_equal(g.nexam[ok], o.nexam[ok])
    np.testing.assert_allclose(g.sumw[ok], o.sumw[ok], rtol=1e-4)
    ch, cw, ns = o.status.shape
    return dict(pixels=ch * cw, excluded=int(excl.sum()), members=int((o_acc & cmp[..., None, None]).sum()),
                max_colour_err=float(cerr[ok].max(initial=0.0)), band_flips=int(bit_diff.sum()),
                box_flips=int(box_diff.sum()), ambiguous_windows=int(amb.sum()))


def run_frustum(sess: Session, cid, O, crop=None, membership=False, **kw) -> GpuResult:
    """Frustum gather (Eq. 1-2) through the C ABI; with membership, status (ch, cw, ns), the
    per-slot sample counts in `nexam`'s place (`count`) and the 64-bit checksums (`hash`)."""
    t, ss = sess.torch, sess.ss
    W, H, F = sess.clips[cid]
    x0, y0, cw, ch = crop if crop is not None else (0, 0, W, H)
    p = sess.params(frame_begin=O, frame_end=O + 1, crop_x=x0, crop_y=y0, crop_w=cw, crop_h=ch,
                    gather=ss.SSVP_GATHER_FRUSTUM, **kw)
    ns = 2 * p.half_window + 1
    mem = stats = None
    if membership:
        mem = t.zeros((ch, cw, ns, 4), dtype=t.int32, device=sess.dev)
        stats = t.zeros((ch, cw, 3), dtype=t.int32, device=sess.dev)
        p.membership_out = mem.data_ptr()
        p.pixel_stats_out = stats.data_ptr()
    ss.ssvp_gather_filter(sess.ctx, p, [cid])
    out = t.empty((1, H, W, 3), dtype=t.float32, device=sess.dev)
    ss.ssvp_read_output(sess.ctx, cid, O, O + 1, out)
    ss.ssvp_sync(sess.ctx)
    res = GpuResult(out[0, y0:y0 + ch, x0:x0 + cw].cpu().numpy())
    if membership:
        m = mem.cpu().numpy()
        s = stats.cpu().numpy()
        res.nacc, res.nexam = s[..., 0].astype(np.int64), s[..., 1].astype(np.int64)
        res.sumw = s[..., 2].view(np.float32).astype(np.float64)
        res.status = m[..., 0]
        res.count = m[..., 1]
        res.hash = m[..., 2].view(np.uint32).astype(np.uint64) | (m[..., 3].view(np.uint32).astype(np.uint64) << np.uint64(32))
    return res


def compare_frustum(g: GpuResult, o: oracle.FrustumResult, ref_valid: np.ndarray):
    """Per (pixel, window frame): sample counts and membership checksums must match exactly
    except where the oracle saw a candidate within the tie band of Eq. 2's bound (or of near /
    far).  Pixels where such an allowed difference occurred are excluded from the colour and
    count comparison; every other pixel must match colour within COLOUR_TOL."""
    band = o.band != 0
    # the GPU marks an invalid reference depth with -2 and frames outside the clip with -1
    assert (g.status[~ref_valid] == -2).all()
    diff = (g.count != o.count) | (g.hash != o.hash)
    diff &= ref_valid[..., None]
    assert not (diff & ~band).any(), \
        f"{int((diff & ~band).sum())} membership differences, first {np.argwhere(diff & ~band)[:5]}"
    excl = diff.any(-1)
    ok = ~excl
    cerr = np.abs(g.rgb.astype(np.float64) - o.rgb).max(-1)
    assert cerr[ok].max(initial=0.0) <= COLOUR_TOL, f"colour max abs {cerr[ok].max()} > {COLOUR_TOL}"
    np.testing.assert_array_equal(g.nacc[ok], o.nacc[ok])
    # the GPU reports sum w in FP32: Gaussian-tail weights carry relative error growing with their
    # exponent, and sums below its range read 0 (Eq. 3 itself is rescaled)
    np.testing.assert_allclose(g.sumw[ok], o.sumw[ok], rtol=1e-4, atol=1e-6)
    return dict(pixels=int(ok.size), excluded=int(excl.sum()), members=int(o.count.sum()),
                band_slots=int(band.sum()), max_colour_err=float(cerr[ok].max(initial=0.0)),
                max_colour_err_all=float(cerr.max()))


def run_superres(sess: Session, cid, O, scale, crop=None, membership=False, **kw) -> GpuResult:
    """Super-resolution (Eq. 6-7) through the C ABI; crop in output-grid pixels."""
    t, ss = sess.torch, sess.ss
    W, H, F = sess.clips[cid]
    Wo, Ho = W * scale, H * scale
    x0, y0, cw, ch = crop if crop is not None else (0, 0, Wo, Ho)
    p = sess.params(frame_begin=O, frame_end=O + 1, crop_x=x0, crop_y=y0, crop_w=cw, crop_h=ch, **kw)
    ns = 2 * p.half_window + 1
    mem = stats = None
    if membership:
        mem = t.zeros((ch, cw, ns, 4), dtype=t.int32, device=sess.dev)
        stats = t.zeros((ch, cw, 3), dtype=t.int32, device=sess.dev)
        p.membership_out = mem.data_ptr()
        p.pixel_stats_out = stats.data_ptr()
    out = t.zeros((1, Ho, Wo, 3), dtype=t.float32, device=sess.dev)
    ss.ssvp_superres(sess.ctx, p, cid, scale, out)
    ss.ssvp_sync(sess.ctx)
    res = GpuResult(out[0, y0:y0 + ch, x0:x0 + cw].cpu().numpy())
    if membership:
        m = mem.cpu().numpy()
        s = stats.cpu().numpy()
        res.nacc, res.nexam = s[..., 0].astype(np.int64), s[..., 1].astype(np.int64)
        res.sumw = s[..., 2].view(np.float32).astype(np.float64)
        res.status = m[..., 0]
        res.count = m[..., 1]
        res.hash = m[..., 2].view(np.uint32).astype(np.uint64) | (m[..., 3].view(np.uint32).astype(np.uint64) << np.uint64(32))
    return res


def compare_flagged(rgb: np.ndarray, o: oracle.Result):
    """Colour parity where no GPU membership record exists (the batched plan): every pixel must
    match within COLOUR_TOL except pixels the oracle flags (a candidate within 1e-5 relative of
    the radius or a window centre within the tie band), where membership may legitimately differ.
    Returns the number of flagged pixels, how many of them actually differ by more than
    COLOUR_TOL, and the largest error at unflagged pixels."""
    band = ((o.codes & oracle.CODE_BAND) != 0).any(axis=(-1, -2, -3))
    amb = ((o.amb == 1) & (o.status == 1)).any(-1)
    ok = ~(band | amb)
    cerr = np.abs(rgb.astype(np.float64) - o.rgb).max(-1)
    assert cerr[ok].max(initial=0.0) <= COLOUR_TOL, \
        f"colour max abs {cerr[ok].max()} > {COLOUR_TOL} at {np.argwhere(ok & (cerr > COLOUR_TOL))[:5]}"
    return dict(pixels=int(ok.size), flagged=int((~ok).sum()), differing=int((cerr > COLOUR_TOL).sum()),
                max_colour_err=float(cerr[ok].max(initial=0.0)), max_colour_err_all=float(cerr.max()))


def superres_ref_valid(c, O, scale, crop):
    """Validity of super-resolution's bilinear reference depth per output-grid pixel of the crop:
    all four input pixels valid (coordinates clamped to the image)."""
    Wo, Ho = c.W * scale, c.H * scale
    x0, y0, cw, ch = crop if crop is not None else (0, 0, Wo, Ho)
    U = np.clip((np.arange(x0, x0 + cw) + 0.5) / scale - 0.5, 0, c.W - 1)
    V = np.clip((np.arange(y0, y0 + ch) + 0.5) / scale - 0.5, 0, c.H - 1)
    ux0, vy0 = np.floor(U).astype(int), np.floor(V).astype(int)
    ux1, vy1 = np.minimum(ux0 + 1, c.W - 1), np.minimum(vy0 + 1, c.H - 1)
    d = c.depth[O]
    ok = np.isfinite(d) & (d > 0)
    return ok[vy0][:, ux0] & ok[vy0][:, ux1] & ok[vy1][:, ux0] & ok[vy1][:, ux1]
