"""GPU parity of the forward path against the FP64 oracle, through the C ABI.

Bit-exact: bin edges, bin map, window counts (Eq. 1 numerator), integral
images and integral histograms. Floating point: the tone-mapped output within
|gpu - ref| <= 1e-4 * max(|ref|, 1e-3); the window variance within the bound
set by the 2^-Q quantisation of the normalised log (see _sigma2_tol).
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2102_01289_gb300 as tm  # noqa: E402

REL = 1e-4
FLOOR = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _built():
    tm.build()


def f32(v):
    return float(np.float32(v))


def params_pair(orc, n, radii, eps=0.1, alpha=1.0, ld_min=0.0, ld_max=1.0, sat=0.6, flags=0):
    """The same parameters for the library (float) and the oracle (the float
    values widened to double). The sRGB output bit has no oracle counterpart:
    the oracle's float output is encoded by the test."""
    gp = tm.make_params(n, radii, eps, alpha, ld_min, ld_max, sat, flags=flags)
    s = len(radii)
    op = orc.make_params(n, radii, eps=[float(gp.eps[f]) for f in range(s)],
                         alpha=[float(gp.alpha[f]) for f in range(s)], ld_min=float(gp.ld_min),
                         ld_max=float(gp.ld_max), sat=float(gp.sat), flags=flags & ~tm.TM_FLAG_SRGB_U8)
    return gp, op


def run_gpu(img, gp, out_dtype=None, debug=True, path=0):
    x = torch.from_numpy(np.ascontiguousarray(img)).cuda()
    ctx = tm.tm_create(gp)
    try:
        tm.tm_set_debug(ctx, debug)
        tm.tm_set_option(ctx, tm.TM_OPT_HIST_PATH, path)
        out = torch.empty(x.shape, dtype=out_dtype or torch.float32, device="cuda")
        tm.tm_forward(ctx, x, out)
        d = {}
        if debug:
            H, W = img.shape[:2]
            s = gp.n_fields
            d["range"] = tm.tm_debug_export(ctx, tm.TM_DBG_RANGE).cpu().numpy()
            d["thr"] = tm.tm_debug_export(ctx, tm.TM_DBG_THRESHOLDS).cpu().numpy() if gp.n_bins > 1 else np.zeros(0, np.float32)
            d["bins"] = tm.tm_debug_export(ctx, tm.TM_DBG_BINS).cpu().numpy().reshape(H, W)
            d["cnt"] = tm.tm_debug_export(ctx, tm.TM_DBG_COUNTS).cpu().numpy().view(np.uint32).reshape(s, H, W)
            d["sigma2"] = tm.tm_debug_export(ctx, tm.TM_DBG_SIGMA2).cpu().numpy().reshape(s, H, W)
            d["weight"] = tm.tm_debug_export(ctx, tm.TM_DBG_WEIGHT).cpu().numpy().reshape(s, H, W)
            d["lf"] = tm.tm_debug_export(ctx, tm.TM_DBG_LF).cpu().numpy().reshape(s, H, W)
            d["l"] = tm.tm_debug_export(ctx, tm.TM_DBG_L).cpu().numpy().reshape(H, W)
            d["qbits"] = int(tm.tm_debug_export(ctx, tm.TM_DBG_QSHIFT).cpu().numpy()[0])
        torch.cuda.synchronize()
        return out.cpu().numpy(), d
    finally:
        tm.tm_destroy(ctx)


def _sigma2_tol(ref, qbits):
    # q carries at most ~1 unit of 2^-Q error per pixel (rounding + log2f);
    # var(l + e) - var(l) <= 2 sigma |e| + |e|^2
    d = 2.0 ** -qbits
    return 2.5 * np.sqrt(np.maximum(ref, 0)) * d + 3 * d * d + 2e-6 * ref


def assert_out_close(got, ref, rel=REL, floor=FLOOR):
    err = np.abs(got.astype(np.float64) - ref)
    tol = rel * np.maximum(np.abs(ref), floor)
    bad = err > tol
    assert not bad.any(), (f"{bad.sum()} of {bad.size} outside tolerance; worst err {err.max():.3e} "
                           f"at ref {ref.ravel()[np.argmax(err)]:.4e}")


CASES = [
    # (H, W, n, radii, seed)
    (384, 512, 32, [4, 16, 64], 0),      # 512x384, 32 bins, radii 4/16/64
    (61, 97, 16, [1, 5, 40], 1),         # ragged, last window larger than the image
    (45, 70, 64, [(3, 1), (0, 7), 12], 2),  # rectangular fields, r = 0 width
    (33, 40, 256, [2, 9], 3),            # maximum bin count
    (20, 30, 1, [3], 4),                 # one bin: every count is zero
]


PATHS = [1, 2]  # fused sweep, materialised integral histogram


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("H,W,n,radii,seed", CASES)
def test_forward_matches_oracle(orc, H, W, n, radii, seed, path):
    img = synth.wdr_image(H, W, seed=seed)
    gp, op = params_pair(orc, n, radii, eps=[0.1, 0.05, 0.2][: len(radii)],
                         alpha=[1.0, 0.7, 1.3][: len(radii)], ld_min=0.02, ld_max=0.98)
    out, d = run_gpu(img, gp, path=path)
    ref, fl = orc.forward(img, op)
    pre = orc.prepare(img, n)
    assert d["range"][0] == pre["imin"] and d["range"][1] == pre["imax"]
    assert np.array_equal(d["thr"], pre["thr"])                 # bin edges, bitwise
    assert np.array_equal(d["bins"], pre["bins"])               # bin map (Section II-A)
    assert np.array_equal(d["cnt"], fl.cnt)                     # Eq. 1 numerators
    tol = _sigma2_tol(fl.sigma2, d["qbits"])
    assert np.all(np.abs(d["sigma2"] - fl.sigma2) <= tol)        # Eq. 10
    assert np.allclose(d["lf"], fl.lf, rtol=1e-6, atol=1e-7)     # Eq. 2
    assert_out_close(d["l"], fl.l)                               # Eq. 3
    assert_out_close(out, ref)                                   # Eq. 12


@pytest.mark.parametrize("path", PATHS)
def test_degenerate_images(orc, path):
    gp, op = params_pair(orc, 8, [1, 3], ld_min=0.3)
    for shape in [(1, 1), (1, 17), (23, 1), (2, 2)]:
        img = synth.wdr_image(*shape, seed=7)
        out, d = run_gpu(img, gp, path=path)
        ref, fl = orc.forward(img, op)
        assert np.array_equal(d["cnt"], fl.cnt)
        assert_out_close(out, ref)
    const = np.full((9, 13, 3), 2.5, np.float32)
    out, d = run_gpu(const, gp, path=path)
    ref, _ = orc.forward(const, op)
    assert np.all(d["bins"] == 0) and np.all(d["sigma2"] == 0)
    assert_out_close(out, ref)


def test_half_input_and_outputs(orc):
    img16 = synth.wdr_image(70, 90, seed=5, dtype=np.float16)
    gp, op = params_pair(orc, 32, [2, 8, 30])
    ref, _ = orc.forward(img16.astype(np.float32), op)
    out, _ = run_gpu(img16, gp, out_dtype=torch.float32, debug=False)
    assert_out_close(out, ref)
    out16, _ = run_gpu(img16, gp, out_dtype=torch.float16, debug=False)
    # half output: the rounding to half adds up to half a half-ulp
    err = np.abs(out16.astype(np.float64) - ref)
    ulp = np.spacing(np.abs(ref).astype(np.float16)).astype(np.float64)
    assert np.all(err <= REL * np.maximum(np.abs(ref), FLOOR) + 0.5 * ulp)
    out8, _ = run_gpu(img16, gp, out_dtype=torch.uint8, debug=False)
    ref8 = np.floor(255.0 * np.clip(ref, 0, 1) + 0.5)
    diff = np.abs(out8.astype(np.int64) - ref8)
    assert diff.max() <= 1 and (diff > 0).mean() <= 1e-4


def test_pitched_input_and_repeat_calls(orc):
    img = synth.wdr_image(40, 50, seed=6)
    gp, op = params_pair(orc, 16, [2, 6])
    big = torch.zeros((40, 64, 3), dtype=torch.float32, device="cuda")
    big[:, :50] = torch.from_numpy(img).cuda()
    view = big[:, :50]
    ctx = tm.tm_create(gp)
    try:
        outs = []
        for _ in range(3):  # the range accumulators re-arm between calls
            o = torch.empty((40, 50, 3), device="cuda")
            tm.tm_forward(ctx, view, o)
            outs.append(o.cpu().numpy())
        img2 = synth.wdr_image(40, 50, seed=60)
        o2 = torch.empty((40, 50, 3), device="cuda")
        tm.tm_forward(ctx, torch.from_numpy(img2).cuda(), o2)
        torch.cuda.synchronize()
    finally:
        tm.tm_destroy(ctx)
    ref, _ = orc.forward(img, op)
    for o in outs:
        assert np.array_equal(o, outs[0])
        assert_out_close(o, ref)
    ref2, _ = orc.forward(img2, op)
    assert_out_close(o2.cpu().numpy(), ref2)


def test_host_buffers_match_device(orc):
    img = synth.wdr_image(64, 80, seed=8)
    gp, op = params_pair(orc, 32, [3, 10])
    out_dev, _ = run_gpu(img, gp, debug=False)
    ctx = tm.tm_create(gp)
    try:
        out_host = np.empty_like(img)
        tm.tm_forward_host(ctx, img, out_host)
    finally:
        tm.tm_destroy(ctx)
    assert np.array_equal(out_host, out_dev)


def test_pinned_host_output_written_directly(orc):
    """A page-locked output buffer is written by the last kernel itself; the
    result equals the device path, for float32 and float16 outputs, and for a
    pitched (row-padded) pinned buffer."""
    img = synth.wdr_image(300, 410, seed=9)
    gp, op = params_pair(orc, 32, [3, 10, 60])
    out_dev, _ = run_gpu(img, gp, debug=False)
    ctx = tm.tm_create(gp)
    try:
        hin = torch.from_numpy(img).pin_memory()
        hout = torch.empty_like(hin).pin_memory()
        for _ in range(2):  # a second call reuses the context's staging
            hout.zero_()
            tm.tm_forward_host(ctx, hin.numpy(), hout.numpy())
            assert np.array_equal(hout.numpy(), out_dev)
        # float16 output through a pinned buffer
        h16 = torch.empty(img.shape, dtype=torch.float16).pin_memory()
        tm.tm_forward_host(ctx, hin.numpy(), h16.numpy())
        x = torch.from_numpy(img).cuda()
        y16 = torch.empty(img.shape, dtype=torch.float16, device="cuda")
        tm.tm_forward(ctx, x, y16)
        torch.cuda.synchronize()
        assert torch.equal(h16, y16.cpu())
        # pitched pinned output: rows padded by 7 pixels
        H, W = img.shape[:2]
        big = torch.zeros((H, W + 7, 3), dtype=torch.float32).pin_memory()
        view = big.numpy()[:, :W, :]
        tm.tm_forward_host(ctx, hin.numpy(), view)
        assert np.array_equal(view, out_dev)
        assert not big.numpy()[:, W:, :].any()
    finally:
        tm.tm_destroy(ctx)


def test_async_host_stream_matches_device(orc):
    """tm_forward_host_async over a stream of page-locked frames, with two
    sizes interleaved (slot reuse and a slot regrow) and no synchronisation
    between calls: every output equals the device path's. Pageable buffers
    are rejected with TM_EINVAL."""
    gp, op = params_pair(orc, 32, [3, 10, 60])
    frames = [synth.wdr_image(*hw, seed=20 + k) for k, hw in enumerate([(120, 160)] * 3 + [(200, 150)] * 2 + [(120, 160)])]
    refs = [run_gpu(f, gp, debug=False)[0] for f in frames]
    ctx = tm.tm_create(gp)
    try:
        hins = [torch.from_numpy(f).pin_memory() for f in frames]
        houts = [torch.zeros_like(h).pin_memory() for h in hins]
        stream = torch.cuda.current_stream()
        for hi, ho in zip(hins, houts):
            tm.tm_forward_host_async(ctx, hi.numpy(), ho.numpy(), stream)
        stream.synchronize()
        for ho, ref in zip(houts, refs):
            assert np.array_equal(ho.numpy(), ref)
        with pytest.raises(tm.TmError) as ei:
            tm.tm_forward_host_async(ctx, frames[0], np.empty_like(frames[0]), stream)
        assert ei.value.status == tm.TM_EINVAL
    finally:
        tm.tm_destroy(ctx)


def test_async_host_interleaved_with_caller_stream_calls(orc):
    """Device-path calls on the same context between asynchronous host calls
    (a forward of another size, a backward, a debug export) share its
    workspace with the forwards in flight on the internal forward stream; a
    second caller stream and a uint8 output slot are mixed in. Every result
    equals the one from a fresh context."""
    gp, op = params_pair(orc, 32, [3, 10, 60])
    frames = [synth.wdr_image(120, 160, seed=40 + k) for k in range(4)]
    other = synth.wdr_image(90, 210, seed=50)
    refs = [run_gpu(f, gp, debug=False)[0] for f in frames]
    ref_u8 = run_gpu(frames[3], gp, out_dtype=torch.uint8, debug=False)[0]
    ref_other, d_other = run_gpu(other, gp, debug=True)
    xo = torch.from_numpy(other).cuda()
    g = torch.from_numpy(synth.wdr_image(90, 210, seed=51)).cuda()
    fresh = tm.tm_create(gp)
    try:
        gin_ref = torch.empty_like(xo)
        tm.tm_forward(fresh, xo, torch.empty_like(xo))
        tm.tm_backward(fresh, xo, g, gin_ref)
        torch.cuda.synchronize()
    finally:
        tm.tm_destroy(fresh)
    ctx = tm.tm_create(gp)
    try:
        hins = [torch.from_numpy(f).pin_memory() for f in frames]
        houts = [torch.zeros_like(h).pin_memory() for h in hins]
        hu8 = torch.zeros(hins[3].shape, dtype=torch.uint8).pin_memory()
        s1, s2 = torch.cuda.current_stream(), torch.cuda.Stream()
        yo = torch.empty_like(xo)
        gin = torch.empty_like(xo)
        tm.tm_forward_host_async(ctx, hins[0].numpy(), houts[0].numpy(), s1)
        tm.tm_forward_host_async(ctx, hins[1].numpy(), houts[1].numpy(), s1)
        tm.tm_forward(ctx, xo, yo, s1)
        bins = tm.tm_debug_export(ctx, tm.TM_DBG_BINS, s1)
        tm.tm_forward_host_async(ctx, hins[2].numpy(), houts[2].numpy(), s2)
        tm.tm_backward(ctx, xo, g, gin, stream=s2)
        tm.tm_forward_host_async(ctx, hins[3].numpy(), houts[3].numpy(), s2)
        tm.tm_forward_host_async(ctx, hins[3].numpy(), hu8.numpy(), s2)
        s1.synchronize()
        s2.synchronize()
        for ho, ref in zip(houts, refs):
            assert np.array_equal(ho.numpy(), ref)
        assert np.array_equal(hu8.numpy(), ref_u8)
        assert np.array_equal(yo.cpu().numpy(), ref_other)
        assert np.array_equal(bins.cpu().numpy().reshape(90, 210), d_other["bins"])
        assert torch.equal(gin.cpu(), gin_ref.cpu())
    finally:
        tm.tm_destroy(ctx)


def test_integral_image_entry_point_exact(orc):
    rng = np.random.default_rng(0)
    # up to a full-size ragged plane (several row segments of the column pass)
    for H, W in [(1, 1), (7, 3000), (300, 257), (2500, 5), (33, 129), (3001, 4003)]:
        q = rng.integers(-(2 ** 23), 2 ** 23 + 1, size=(H, W)).astype(np.int32)
        qt = torch.from_numpy(q).cuda()
        s1 = torch.empty((H + 1, W + 1), dtype=torch.int64, device="cuda")
        s2 = torch.empty_like(s1)
        tm.tm_integral_image(qt, s1, s2)
        torch.cuda.synchronize()
        r1 = orc.integral_i64(q)
        r2 = orc.integral_i64(q.astype(np.int64) ** 2)
        assert np.array_equal(s1.cpu().numpy().view(np.uint64), r1)
        assert np.array_equal(s2.cpu().numpy().view(np.uint64), r2)


def test_integral_histogram_entry_point_exact(orc):
    rng = np.random.default_rng(1)
    for H, W, n in [(1, 1, 1), (37, 2100, 5), (129, 64, 64), (9, 11, 256)]:
        b = rng.integers(0, n, size=(H, W)).astype(np.uint8)
        bt = torch.from_numpy(b).cuda()
        hk = torch.empty((n, H + 1, W + 1), dtype=torch.int32, device="cuda")
        tm.tm_integral_histogram(bt, n, hk)
        torch.cuda.synchronize()
        assert np.array_equal(hk.cpu().numpy().view(np.uint32), orc.integral_histogram(b, n))


def test_big_window_wide_counts_and_tile_edges(orc):
    """Windows over 2^16 pixels take uint32 count planes; tiles leave ragged
    edges. 600 x 700, radii 5/40/150 (301 x 301 > 2^16), 24 bins."""
    img = synth.wdr_image(600, 700, seed=13)
    gp, op = params_pair(orc, 24, [5, 40, (150, 150)])
    out, d = run_gpu(img, gp, path=1)
    ref, fl = orc.forward(img, op)
    assert np.array_equal(d["cnt"], fl.cnt)
    assert_out_close(out, ref)


def test_full_size_12mp_sampled(orc):
    """4000 x 3000, 64 bins, radii 8/32/128: edges and the whole bin map
    bit-exact; outputs at sampled pixels (corners, borders, interior) against
    the oracle's direct per-pixel evaluation."""
    H, W = 3000, 4000
    img = synth.wdr_image(H, W, seed=1, decades=(-3.0, 5.0))
    gp, op = params_pair(orc, 64, [8, 32, 128])
    out, d = run_gpu(img, gp)
    pre = orc.prepare(img, 64)
    assert np.array_equal(d["thr"], pre["thr"])
    assert np.array_equal(d["bins"], pre["bins"])
    rng = np.random.default_rng(2)
    ys = np.concatenate([[0, 0, H - 1, H - 1, 127, 128, 129, H - 129], rng.integers(0, H, 120)])
    xs = np.concatenate([[0, W - 1, 0, W - 1, 4000 - 129, 128, 3, 2000], rng.integers(0, W, 120)])
    ref, dd = orc.forward_pixels(img, op, xs, ys)
    assert np.array_equal(d["cnt"][:, ys, xs].T, dd["cnt"])
    assert_out_close(out[ys, xs], ref)


@pytest.mark.parametrize("path", PATHS)
def test_full_size_12mp_every_count(orc, path):
    """4000 x 3000, 64 bins, radii 8/32/128 on both histogram paths: the Eq. 1
    numerator of every pixel and every field equals the oracle's (bin map,
    then the box sums of the integral image of [b < b(p)], Eq. 7-9), bit for
    bit; the bin map itself too."""
    H, W = 3000, 4000
    img = synth.wdr_image(H, W, seed=7, decades=(-3.0, 5.0))
    gp, op = params_pair(orc, 64, [8, 32, 128])
    x = torch.from_numpy(img).cuda()
    y = torch.empty_like(x)
    ctx = tm.tm_create(gp)
    try:
        tm.tm_set_debug(ctx, True)
        tm.tm_set_option(ctx, tm.TM_OPT_HIST_PATH, path)
        tm.tm_forward(ctx, x, y)
        bins = tm.tm_debug_export(ctx, tm.TM_DBG_BINS).cpu().numpy().reshape(H, W)
        cnt = tm.tm_debug_export(ctx, tm.TM_DBG_COUNTS).cpu().numpy().view(np.uint32).reshape(3, H, W)
        torch.cuda.synchronize()
    finally:
        tm.tm_destroy(ctx)
    pre = orc.prepare(img, 64)
    assert np.array_equal(bins, pre["bins"])
    ref = orc.window_counts(pre["bins"], op)
    bad = cnt != ref
    assert not bad.any(), f"{int(bad.sum())} counts differ, first at {np.argwhere(bad)[0]}"


def _pyramid_pair(orc, W, H, s=5, n=5):
    """The paper's preset (Section IV): s fields halving from the whole
    image (rectangular windows), n bins, eps 0.1, sat 0.6."""
    gp = tm.tm_params_pyramid(W, H, s, n)
    radii = [(int(gp.rx[f]), int(gp.ry[f])) for f in range(s)]
    op = orc.make_params(n, radii, eps=[float(gp.eps[f]) for f in range(s)],
                         alpha=[float(gp.alpha[f]) for f in range(s)], ld_min=float(gp.ld_min),
                         ld_max=float(gp.ld_max), sat=float(gp.sat))
    return gp, op


@pytest.mark.parametrize("path", PATHS)
def test_paper_preset_matches_oracle(orc, path):
    """s = 5 fields from the whole image down by halves, n = 5: windows larger
    than the image (clipped areas), rectangular fields, few bins."""
    H, W = 150, 220
    img = synth.wdr_image(H, W, seed=31)
    gp, op = _pyramid_pair(orc, W, H)
    out, d = run_gpu(img, gp, path=path)
    ref, fl = orc.forward(img, op)
    assert np.array_equal(d["cnt"], fl.cnt)
    assert_out_close(out, ref)


def test_paper_preset_12mp_sampled(orc):
    """The preset at 4000 x 3000: the largest window is the whole image, wider
    than the 32 chunks of a swept row, so the context takes the materialised
    integral histogram (4 cumulative planes at n = 5). Bin map bit-exact,
    outputs at sampled pixels against direct per-pixel evaluation."""
    H, W = 3000, 4000
    img = synth.wdr_image(H, W, seed=3, decades=(-3.0, 5.0))
    gp, op = _pyramid_pair(orc, W, H)
    out, d = run_gpu(img, gp)
    pre = orc.prepare(img, 5)
    assert np.array_equal(d["bins"], pre["bins"])
    ys = np.array([0, H - 1, 0, H - 1, 1500, 777, 2999, 1])
    xs = np.array([0, W - 1, W - 1, 0, 2000, 3333, 17, 3998])
    ref, dd = orc.forward_pixels(img, op, xs, ys)
    assert np.array_equal(d["cnt"][:, ys, xs].T, dd["cnt"])
    assert_out_close(out[ys, xs], ref)


FLAG_SETS = [tm.TM_FLAG_CDF_INCLUSIVE, tm.TM_FLAG_AREA_LITERAL, tm.TM_FLAG_VAR_LINEAR,
             tm.TM_FLAG_CDF_INCLUSIVE | tm.TM_FLAG_AREA_LITERAL | tm.TM_FLAG_VAR_LINEAR]


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("flags", FLAG_SETS)
def test_reading_variants_match_oracle(orc, flags, path):
    """Each reading variant (Eq. 1 with <=, Algorithm 1's unclipped area,
    Eq. 10 on i / imax) against the oracle's: counts bit-exact, variances
    within the quantisation bound, outputs within the float tolerance. The
    last field is larger than the image (clipping and padding matter)."""
    H, W = 61, 97
    img = synth.wdr_image(H, W, seed=41)
    gp, op = params_pair(orc, 16, [1, (6, 3), 40], eps=[0.1, 0.05, 0.2], flags=flags)
    out, d = run_gpu(img, gp, path=path)
    ref, fl = orc.forward(img, op)
    assert np.array_equal(d["cnt"], fl.cnt)
    assert np.all(np.abs(d["sigma2"] - fl.sigma2) <= _sigma2_tol(fl.sigma2, d["qbits"]))
    assert_out_close(d["l"], fl.l)
    assert_out_close(out, ref)


def test_inclusive_cdf_on_the_sweep_at_full_bin_range(orc):
    """Eq. 1 with <= reads threshold b + 1, one past the highest bin of a
    tile; 256 bins and a region spanning all of them."""
    img = synth.wdr_image(40, 60, seed=42, decades=(-4.0, 6.0))
    gp, op = params_pair(orc, 256, [2, 9], flags=tm.TM_FLAG_CDF_INCLUSIVE)
    out, d = run_gpu(img, gp, path=1)
    ref, fl = orc.forward(img, op)
    assert np.array_equal(d["cnt"], fl.cnt)
    assert_out_close(out, ref)


@pytest.mark.parametrize("width", [256, 512])
@pytest.mark.parametrize("segments", [0, 12, 200])
def test_sweep_segments_and_threshold_passes(orc, segments, width):
    """The sweep's segments run on over the bands they claim; CTAs that finish
    early take the rest. A 1500-column image with 256 bins over ten decades
    has tiles whose bins span more thresholds than the shared memory holds
    (several passes: such a segment claims its group's bands up front).
    Counts bit-exact and output within tolerance at every tiling (0: the
    automatic one; 12 and 200 segments: long and short bands) and at both
    strip widths (256: six strips, the last ragged; 512: three)."""
    img = synth.wdr_image(240, 1500, seed=7, decades=(-4.0, 6.0))
    gp, op = params_pair(orc, 256, [3, 20])
    x = torch.from_numpy(np.ascontiguousarray(img)).cuda()
    ctx = tm.tm_create(gp)
    try:
        tm.tm_set_debug(ctx, 1)
        tm.tm_set_option(ctx, tm.TM_OPT_HIST_PATH, 1)
        tm.tm_set_option(ctx, tm.TM_OPT_SWEEP_TILES, segments)
        tm.tm_set_option(ctx, tm.TM_OPT_SWEEP_WIDTH, width)
        out = torch.empty_like(x)
        for _ in range(2):  # the claims are cleared for every call
            tm.tm_forward(ctx, x, out)
        cnt = tm.tm_debug_export(ctx, tm.TM_DBG_COUNTS).cpu().numpy().view(np.uint32).reshape(2, 240, 1500)
        torch.cuda.synchronize()
    finally:
        tm.tm_destroy(ctx)
    ref, fl = orc.forward(img, op)
    assert np.array_equal(cnt, fl.cnt)
    assert_out_close(out.cpu().numpy(), ref)


@pytest.mark.parametrize("width", [0, 512])
def test_sweep_wide_fields_take_narrow_strips(orc, width):
    """A half-width of 300 does not fit a 512-column strip's swept row (32
    chunks of 32 columns), so the sweep runs on 256-column strips whatever
    width is asked for; counts bit-exact, output within tolerance."""
    img = synth.wdr_image(200, 1400, seed=71)
    gp, op = params_pair(orc, 32, [5, 300])
    x = torch.from_numpy(np.ascontiguousarray(img)).cuda()
    ctx = tm.tm_create(gp)
    try:
        tm.tm_set_debug(ctx, 1)
        tm.tm_set_option(ctx, tm.TM_OPT_HIST_PATH, 1)
        tm.tm_set_option(ctx, tm.TM_OPT_SWEEP_WIDTH, width)
        out = torch.empty_like(x)
        tm.tm_forward(ctx, x, out)
        cnt = tm.tm_debug_export(ctx, tm.TM_DBG_COUNTS).cpu().numpy().view(np.uint32).reshape(2, 200, 1400)
        torch.cuda.synchronize()
    finally:
        tm.tm_destroy(ctx)
    ref, fl = orc.forward(img, op)
    assert np.array_equal(cnt, fl.cnt)
    assert_out_close(out.cpu().numpy(), ref)


def test_srgb_uint8_output(orc):
    """TM_FLAG_SRGB_U8: uint8 output is floor(255 srgb(clamp(c)) + 0.5) of
    the oracle's float result, within 1 LSB on at most 0.01% of the values."""
    img = synth.wdr_image(70, 90, seed=43)
    gp, op = params_pair(orc, 32, [2, 8, 30], flags=tm.TM_FLAG_SRGB_U8)
    ref, _ = orc.forward(img, op)
    out8, _ = run_gpu(img, gp, out_dtype=torch.uint8, debug=False)
    ref8 = orc.to_u8(ref, srgb=True).astype(np.int64)
    diff = np.abs(out8.astype(np.int64) - ref8)
    assert diff.max() <= 1 and (diff > 0).mean() <= 1e-4
    # float outputs are not encoded
    outf, _ = run_gpu(img, gp, debug=False)
    assert_out_close(outf, ref)


@pytest.mark.parametrize("path", PATHS)
def test_streaming_range_reuse(orc, path):
    """TM_OPT_REUSE_RANGE: each frame is binned and normalised over the
    previous frame's range (pixels outside it clamp to the end bins and to
    lhat 0 / 1), and the bin pass takes the frame's own range for the next
    one. The first frame, a frame of another size, and any frame after the
    option is switched off use their own range."""
    H, W = 90, 120
    frames = [synth.wdr_image(H, W, seed=50), 3.0 * synth.wdr_image(H, W, seed=51),
              0.5 * synth.wdr_image(H, W, seed=52)]
    frames = [f.astype(np.float32) for f in frames]
    gp, op = params_pair(orc, 32, [2, 8, 30])
    ranges = [tuple(float(v) for v in (orc.prepare(f, 32)["imin"], orc.prepare(f, 32)["imax"])) for f in frames]
    ctx = tm.tm_create(gp)
    try:
        tm.tm_set_debug(ctx, True)
        tm.tm_set_option(ctx, tm.TM_OPT_HIST_PATH, path)
        tm.tm_set_option(ctx, tm.TM_OPT_REUSE_RANGE, 1)

        def fwd(img):
            x = torch.from_numpy(np.ascontiguousarray(img)).cuda()
            y = torch.empty_like(x)
            tm.tm_forward(ctx, x, y)
            cnt = tm.tm_debug_export(ctx, tm.TM_DBG_COUNTS).cpu().numpy().view(np.uint32)
            rng = tm.tm_debug_export(ctx, tm.TM_DBG_RANGE).cpu().numpy()
            torch.cuda.synchronize()
            return y.cpu().numpy(), cnt.reshape(3, *img.shape[:2]), (float(rng[0]), float(rng[1]))

        used = [None, ranges[0], ranges[1]]
        for k, img in enumerate(frames):
            out, cnt, rng = fwd(img)
            ref, fl = orc.forward(img, op, range_=used[k])
            assert rng == (used[k] or ranges[0])
            assert np.array_equal(cnt, fl.cnt)
            assert_out_close(out, ref)
        # another size: its own range
        small = synth.wdr_image(40, 50, seed=53)
        out, cnt, rng = fwd(small)
        ref, fl = orc.forward(small, op)
        assert np.array_equal(cnt, fl.cnt)
        assert_out_close(out, ref)
        # option off: own range again
        tm.tm_set_option(ctx, tm.TM_OPT_REUSE_RANGE, 0)
        out, cnt, rng = fwd(frames[1])
        ref, fl = orc.forward(frames[1], op)
        assert rng == ranges[1]
        assert_out_close(out, ref)
    finally:
        tm.tm_destroy(ctx)


@pytest.mark.parametrize("n", [5, 48])
def test_automatic_path_matches_forced_paths(orc, n):
    """TM_OPT_HIST_PATH = 0 times both histogram paths on the first image of a
    size and keeps the faster; every call, first and later, agrees with both
    forced paths and with the oracle."""
    img = synth.wdr_image(200, 300, seed=60)
    gp, op = params_pair(orc, n, [3, 12, 40])
    ref, _ = orc.forward(img, op)
    outs = {}
    for path in (1, 2):
        outs[path], _ = run_gpu(img, gp, debug=False, path=path)
    x = torch.from_numpy(img).cuda()
    ctx = tm.tm_create(gp)
    try:
        for _ in range(3):  # the first call measures, the later ones reuse the choice
            y = torch.empty_like(x)
            tm.tm_forward(ctx, x, y)
            torch.cuda.synchronize()
            got = y.cpu().numpy()
            assert_out_close(got, ref)
            assert np.allclose(got, outs[1], rtol=1e-6, atol=1e-7) and np.allclose(got, outs[2], rtol=1e-6, atol=1e-7)
    finally:
        tm.tm_destroy(ctx)


MAX_FIELDS_RADII = [0, 1, 3, (7, 2), 15, (40, 0), (32767, 5), 32767]
MAX_FIELDS_EPS = [0.1, 0.05, 0.2, 0.08, 0.3, 0.1, 0.02, 0.15]
MAX_FIELDS_ALPHA = [1.0, 0.7, 1.3, 0.9, 1.1, 0.5, 1.0, 0.8]


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("flags", [0, tm.TM_FLAG_CDF_INCLUSIVE | tm.TM_FLAG_AREA_LITERAL])
def test_eight_fields_and_maximum_radius(orc, flags, path):
    """TM_MAX_FIELDS fields with half-sizes from 0 to TM_MAX_RADIUS: the last
    two windows span the image in one or both directions (the sweep clips
    their half-sizes to the image); under Algorithm 1's area the largest window
    is 65535 x 65535 pixels, an Eq. 1 denominator just under 2^32. Counts
    bit-exact, variances within the quantisation bound, outputs within the
    float tolerance, on a 70 x 90 and a 37 x 300 image."""
    for H, W, seed in [(70, 90, 70), (37, 300, 71)]:
        img = synth.wdr_image(H, W, seed=seed)
        gp, op = params_pair(orc, 16, MAX_FIELDS_RADII, eps=MAX_FIELDS_EPS, alpha=MAX_FIELDS_ALPHA,
                             ld_min=0.02, ld_max=0.98, flags=flags)
        out, d = run_gpu(img, gp, path=path)
        ref, fl = orc.forward(img, op)
        assert np.array_equal(d["cnt"], fl.cnt)
        assert np.all(np.abs(d["sigma2"] - fl.sigma2) <= _sigma2_tol(fl.sigma2, d["qbits"]))
        assert np.allclose(d["lf"], fl.lf, rtol=1e-6, atol=1e-7)
        assert_out_close(d["l"], fl.l)
        assert_out_close(out, ref)


def _mem_available_gb():
    try:
        with open("/proc/meminfo") as fh:
            for line in fh:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) / 2 ** 20
    except OSError:
        pass
    return 0.0


LARGE_RADII = [(150, 150), (140, 150), (150, 120), 130, (110, 150), (150, 110), 145, (120, 140)]


@pytest.mark.parametrize("path", PATHS)
def test_large_image_64bit_offsets_sampled(orc, path):
    """16384 x 12288 (201 MP) with 8 fields whose windows each hold more than
    2^16 pixels: 8 uint32 count planes, byte offsets past 2^31 on the fused
    path; 16 bins, 15 cumulative planes of
    805 MB on the materialised one. Range, bin edges and bin map exact;
    counts, variances and outputs at sampled pixels (corners, edges, tile
    seams, random) against the oracle's direct per-pixel evaluation."""
    H, W = 12288, 16384
    if _mem_available_gb() < 24 or torch.cuda.mem_get_info()[0] < 80 * 2 ** 30:
        pytest.skip("needs 24 GB of host and 80 GB of device memory")
    img = synth.wdr_mosaic(H, W, seed=80)
    gp, op = params_pair(orc, 16, LARGE_RADII, eps=MAX_FIELDS_EPS, alpha=MAX_FIELDS_ALPHA)
    rng = np.random.default_rng(81)
    ys = np.concatenate([[0, 0, H - 1, H - 1, 3071, 3072, 6143, 6144, 150, H - 151],
                         rng.integers(0, H, 110)])
    xs = np.concatenate([[0, W - 1, 0, W - 1, 4095, 4096, 8191, 8192, W - 151, 150],
                         rng.integers(0, W, 110)])
    x = torch.from_numpy(img).cuda()
    y = torch.empty_like(x)
    yi, xi = torch.from_numpy(ys).cuda(), torch.from_numpy(xs).cuda()
    ctx = tm.tm_create(gp)
    try:
        tm.tm_set_debug(ctx, True)
        tm.tm_set_option(ctx, tm.TM_OPT_HIST_PATH, path)
        tm.tm_forward(ctx, x, y)
        rng_dev = tm.tm_debug_export(ctx, tm.TM_DBG_RANGE).cpu().numpy()
        thr = tm.tm_debug_export(ctx, tm.TM_DBG_THRESHOLDS).cpu().numpy()
        bins = tm.tm_debug_export(ctx, tm.TM_DBG_BINS).view(H, W).cpu().numpy()
        qbits = int(tm.tm_debug_export(ctx, tm.TM_DBG_QSHIFT).cpu().numpy()[0])
        sampled = {}
        for key, what in (("cnt", tm.TM_DBG_COUNTS), ("sigma2", tm.TM_DBG_SIGMA2)):
            plane = tm.tm_debug_export(ctx, what).view(gp.n_fields, H, W)
            sampled[key] = plane[:, yi, xi].T.cpu().numpy()
            del plane
        out = y[yi, xi].cpu().numpy()
        torch.cuda.synchronize()
    finally:
        tm.tm_destroy(ctx)
    del x, y
    pre = orc.prepare(img, 16)
    assert rng_dev[0] == pre["imin"] and rng_dev[1] == pre["imax"]
    assert np.array_equal(thr, pre["thr"])
    assert np.array_equal(bins, pre["bins"])
    del pre, bins
    ref, dd = orc.forward_pixels(img, op, xs, ys)
    assert np.array_equal(sampled["cnt"].view(np.uint32), dd["cnt"])
    assert np.all(np.abs(sampled["sigma2"] - dd["sigma2"]) <= _sigma2_tol(dd["sigma2"], qbits))
    assert_out_close(out, ref)
