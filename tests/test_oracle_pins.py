"""Pins of the FP64 oracle against what the paper and mathematics fix.

Nothing here retypes the oracle's formulas: each check is a brute-force count
on a tiny image, a library routine standing in for a textbook special case
(numpy cumsum / var / bincount), a closed form, an invariant the paper states,
or a finite difference. Each is chosen so that a plausible slip in the oracle
(swapped weight, wrong corner index, dropped term, wrong sign) fails here.
"""
import json
import math
import os

import numpy as np
import pytest

import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _grey(vals):
    v = np.asarray(vals, np.float32)
    return np.repeat(v[..., None], 3, axis=-1)


# ---------------------------------------------------------------- Eq. 11 --
def test_luminance_weights_match_eq11(orc):
    g = json.load(open(os.path.join(GOLDEN, "paper_constants.json")))
    wr, wg, wb = g["luminance_weights"]["value"]
    assert orc.luminance(1.0, 0.0, 0.0) == np.float32(wr)
    assert orc.luminance(0.0, 1.0, 0.0) == np.float32(wg)
    assert orc.luminance(0.0, 0.0, 1.0) == np.float32(wb)
    # weights sum to one (up to float rounding), so grey in -> same luminance
    assert abs(orc.luminance(3.0, 3.0, 3.0) - 3.0) < 3.0 * 2e-7


def test_luminance_float_order_and_floor(orc):
    rng = np.random.default_rng(1)
    f = np.float32
    for r, g, b in rng.uniform(0, 1e4, size=(200, 3)).astype(np.float32):
        expect = (f(0.2126) * r + f(0.7152) * g) + f(0.0722) * b  # numpy float32 ops
        assert orc.luminance(r, g, b) == expect
    assert orc.luminance(0.0, 0.0, 0.0) == np.float32(1e-30)


# ------------------------------------------------ Section II-A binning --
@pytest.mark.parametrize("n", [1, 2, 5, 32, 64, 256])
def test_bins_equal_width_in_log(orc, n):
    img = synth.wdr_image(37, 53, seed=n)
    d = orc.prepare(img, n)
    lum = d["lum"].astype(np.float64)
    lo, hi = math.log(d["imin"]), math.log(d["imax"])
    u = n * (np.log(lum) - lo) / (hi - lo)
    expect = np.minimum(np.floor(u), n - 1).astype(np.int64)
    near_edge = np.abs(u - np.round(u)) < 1e-9
    assert np.array_equal(d["bins"][~near_edge], expect[~near_edge])
    assert d["bins"].min() == 0 and d["bins"].max() == n - 1
    assert d["bins"].ravel()[np.argmin(lum)] == 0
    assert d["bins"].ravel()[np.argmax(lum)] == n - 1
    thr = d["thr"]
    assert thr.shape == (n - 1,)
    assert np.all(np.diff(thr.astype(np.float64)) > 0)
    # edges round up: the float just below each edge lies below the exact edge
    for k in range(1, n):
        exact_u = k  # edge k sits at u == k
        below = np.nextafter(thr[k - 1], np.float32(0))
        assert n * (math.log(float(below)) - lo) / (hi - lo) < exact_u + 1e-9


def test_degenerate_range_all_bin_zero(orc):
    d = orc.prepare(_grey(np.full((4, 6), 7.0)), 16)
    assert np.all(d["bins"] == 0) and np.all(d["lhat"] == 0)


def test_lhat_normalised_log(orc):
    img = _grey([[1.0, 10.0, 100.0, 1000.0]])
    d = orc.prepare(img, 4)
    lum = d["lum"].astype(np.float64).ravel()
    lh = d["lhat"].ravel()
    assert lh[0] == 0.0 and abs(lh[-1] - 1.0) < 1e-15
    # log base does not matter: compare with log10 ratio
    ref = (np.log10(lum) - np.log10(lum[0])) / (np.log10(lum[-1]) - np.log10(lum[0]))
    assert np.allclose(lh, ref, atol=1e-14)


# ------------------------------------------------------------- Eq. 5 ----
def test_integral_image_matches_cumsum(orc):
    rng = np.random.default_rng(0)
    v = rng.integers(-(2 ** 40), 2 ** 40, size=(19, 23))
    S = orc.integral_i64(v)
    ref = np.zeros((20, 24), np.uint64)
    ref[1:, 1:] = np.cumsum(np.cumsum(v.astype(np.uint64), 0), 1)  # wraps mod 2^64
    assert np.array_equal(S, ref)
    vf = rng.standard_normal((7, 9))
    Sf = orc.integral_f64(vf)
    assert np.allclose(Sf[1:, 1:], np.cumsum(np.cumsum(vf, 0), 1), atol=1e-12)
    assert np.all(Sf[0] == 0) and np.all(Sf[:, 0] == 0)


def test_integral_image_wraps_mod_2_64(orc):
    v = np.full((3, 3), 2 ** 62, np.int64)
    S = orc.integral_i64(v)
    assert int(S[3, 3]) == (9 * 2 ** 62) % (2 ** 64)


# --------------------------------------------------------- Eq. 7-9 ------
def test_integral_histogram_matches_onehot_cumsum(orc):
    rng = np.random.default_rng(3)
    n = 7
    b = rng.integers(0, n, size=(11, 13)).astype(np.uint8)
    Hk = orc.integral_histogram(b, n)
    for k in range(n):
        ref = np.zeros((12, 14), np.int64)
        ref[1:, 1:] = np.cumsum(np.cumsum((b == k).astype(np.int64), 0), 1)
        assert np.array_equal(Hk[k].astype(np.int64), ref)
    # Eq. 9 with Algorithm 1's corners (x - r - 1, x + r) on interior windows
    r, x, y = 2, 6, 5
    for k in range(n):
        box = (int(Hk[k, y + r + 1, x + r + 1]) - int(Hk[k, y + r + 1, x - r])
               - int(Hk[k, y - r, x + r + 1]) + int(Hk[k, y - r, x - r]))
        assert box == int(np.sum(b[y - r:y + r + 1, x - r:x + r + 1] == k))
    # histogram counts of every window sum to the window area (Eq. 1's T)
    tot = sum(int(Hk[k, -1, -1]) for k in range(n))
    assert tot == b.size


# -------------------------------------------- Eq. 1, 2, 4, 10 by brute force
RADII_SETS = [
    [0],
    [1],
    [(2, 1), (0, 3)],
    [1, 3, 40],  # last window larger than the image
]


@pytest.mark.parametrize("radii", RADII_SETS)
def test_forward_fields_against_brute_force(orc, radii):
    img = synth.wdr_image(9, 12, seed=len(radii) + 5)
    n = 6
    p = orc.make_params(n, radii, eps=[0.1, 0.02, 0.3, 0.05][: len(radii)])
    out, fl = orc.forward(img, p)
    d = orc.prepare(img, n)
    b, lh = d["bins"].astype(np.int64), d["lhat"]
    H, W = b.shape
    for f, r in enumerate(radii):
        rx, ry = (r, r) if np.isscalar(r) else r
        for y in range(H):
            for x in range(W):
                ys = slice(max(y - ry, 0), min(y + ry, H - 1) + 1)
                xs = slice(max(x - rx, 0), min(x + rx, W - 1) + 1)
                win_b, win_l = b[ys, xs], lh[ys, xs]
                assert fl.area[f, y, x] == win_b.size
                assert fl.cnt[f, y, x] == int(np.sum(win_b < b[y, x]))  # strict (Eq. 1)
                v = float(np.var(win_l))
                assert abs(fl.sigma2[f, y, x] - v) <= 1e-12 + 1e-9 * v
                assert abs(fl.mu[f, y, x] - float(np.mean(win_l))) <= 1e-12
    # convex combination (Eq. 3) and weight range (Eq. 4)
    lo = fl.lf.min(axis=0) - 1e-12
    hi = fl.lf.max(axis=0) + 1e-12
    assert np.all((fl.l >= lo) & (fl.l <= hi))
    alpha = np.array([p.alpha[f] for f in range(len(radii))])[:, None, None]
    assert np.all(fl.weight >= 0) and np.all(fl.weight < alpha)


def test_forward_matches_direct_pixel_path(orc):
    img = synth.wdr_image(23, 31, seed=11)
    p = orc.make_params(16, [1, 4, 12])
    out, fl = orc.forward(img, p)
    yy, xx = np.meshgrid(np.arange(23), np.arange(31), indexing="ij")
    o2, d = orc.forward_pixels(img, p, xx.ravel(), yy.ravel())
    assert np.array_equal(d["cnt"].T.reshape(3, 23, 31), fl.cnt)
    assert np.allclose(o2, out.reshape(-1, 3), rtol=1e-12, atol=1e-15)


# ------------------------------------------------------ special cases ----
def test_constant_image_maps_to_ld_min(orc):
    img = _grey(np.full((6, 8), 3.5))
    p = orc.make_params(8, [1, 2], ld_min=0.25, ld_max=0.9)
    out, fl = orc.forward(img, p)
    assert np.all(fl.sigma2 == 0) and np.all(fl.weight == 0)
    assert np.allclose(out, 0.25, atol=1e-15)  # grey: (C/i)^sat == 1 up to rounding


def test_zero_radius_maps_to_ld_min(orc):
    img = synth.wdr_image(8, 8, seed=2)
    p = orc.make_params(8, [0], ld_min=0.1)
    out, fl = orc.forward(img, p)
    assert np.all(fl.cnt == 0) and np.all(fl.sigma2 == 0)
    assert np.allclose(fl.l, 0.1)


def test_single_global_field_is_histogram_equalisation(orc):
    """s = 1 with a window covering the image: P is the global strict-below
    histogram CDF (Section II-B: the mapping becomes global and monotone)."""
    img = synth.wdr_image(14, 17, seed=4)
    n = 10
    p = orc.make_params(n, [100], ld_min=0.0, ld_max=1.0)
    out, fl = orc.forward(img, p)
    b = orc.prepare(img, n)["bins"]
    hist = np.bincount(b.ravel(), minlength=n)
    cdf_below = np.concatenate([[0], np.cumsum(hist)[:-1]]) / b.size
    assert np.allclose(fl.lf[0], cdf_below[b], atol=1e-15)
    assert np.allclose(fl.l, cdf_below[b], atol=1e-15)
    lum = orc.prepare(img, n)["lum"].ravel()
    order = np.argsort(lum, kind="stable")
    assert np.all(np.diff(fl.l.ravel()[order]) >= -1e-15)  # monotone in luminance


def test_two_level_step_counts_closed_form(orc):
    img, (y0, y1, x0, x1) = synth.box_image(20, 24, seed=5)
    r = 3
    p = orc.make_params(4, [r])
    out, fl = orc.forward(img, p)
    H, W = 20, 24

    def overlap(a0, a1, b0, b1):  # |[a0,a1] cap [b0,b1-1]|
        return max(0, min(a1, b1 - 1) - max(a0, b0) + 1)

    for y in range(H):
        for x in range(W):
            wy0, wy1 = max(y - r, 0), min(y + r, H - 1)
            wx0, wx1 = max(x - r, 0), min(x + r, W - 1)
            area = (wy1 - wy0 + 1) * (wx1 - wx0 + 1)
            bright = overlap(wy0, wy1, y0, y1) * overlap(wx0, wx1, x0, x1)
            inside = (y0 <= y < y1) and (x0 <= x < x1)
            assert fl.cnt[0, y, x] == (area - bright if inside else 0)


def test_colour_restoration_closed_form(orc):
    # one pixel with C/i = 2 in red: out_r / L = 2^0.6 (Eq. 12, sat = 0.6)
    img = synth.wdr_image(6, 6, seed=9)
    p = orc.make_params(8, [1, 2])
    out, fl = orc.forward(img, p)
    lum = orc.prepare(img, 8)["lum"].astype(np.float64)
    ratio = img.astype(np.float64) / lum[..., None]
    assert np.allclose(out, ratio ** 0.6 * fl.l[..., None], rtol=1e-13)
    assert abs(2.0 ** 0.6 - 1.5157165665103982) < 1e-15
    grey = _grey(synth.wdr_image(5, 5, seed=1)[..., 1])
    og, fg = orc.forward(grey, p)
    assert np.allclose(og[..., 0], og[..., 2]) and np.allclose(og[..., 0], fg.l, rtol=1e-6)


# ------------------------------------------------------------ invariants --
def test_scale_invariance(orc):
    img = synth.wdr_image(16, 21, seed=8)
    p = orc.make_params(12, [1, 5])
    out, fl = orc.forward(img, p)
    out2, fl2 = orc.forward(img * np.float32(8.0), p)
    assert np.array_equal(orc.prepare(img, 12)["bins"], orc.prepare(img * np.float32(8.0), 12)["bins"])
    assert np.array_equal(fl.cnt, fl2.cnt)
    assert np.allclose(out2, out, rtol=1e-12, atol=1e-15)


def test_power_law_invariance_of_tone_mapped_luminance(orc):
    # lhat and the bins only see ln i up to an affine map: i -> i^gamma leaves L
    base = synth.wdr_image(12, 12, seed=3)[..., 0].astype(np.float64)
    img1 = _grey(base)
    img2 = _grey(base ** 1.7)
    p = orc.make_params(6, [1, 3])
    _, f1 = orc.forward(img1, p)
    _, f2 = orc.forward(img2, p)
    b1, b2 = orc.prepare(img1, 6)["bins"], orc.prepare(img2, 6)["bins"]
    if not np.array_equal(b1, b2):
        pytest.skip("a pixel sits within float rounding of a bin edge")
    assert np.allclose(f1.l, f2.l, rtol=1e-5, atol=1e-9)


def test_tone_curve_monotone_in_centre_bin(orc):
    # raising only the centre pixel (same window otherwise) never lowers L_w
    base = _grey(np.full((7, 7), 1.0))
    base[0, 0] = 0.01
    base[6, 6] = 1000.0
    p = orc.make_params(8, [3])
    vals = np.geomspace(0.02, 900, 25)
    lfs = []
    for v in vals:
        im = base.copy()
        im[3, 3] = v
        _, fl = orc.forward(im, p)
        lfs.append(fl.lf[0, 3, 3])
    assert np.all(np.diff(lfs) >= 0) and lfs[-1] > lfs[0]


def test_weight_limits(orc):
    # W -> alpha when sigma^2 >> eps, W -> 0 when sigma^2 << eps (Section II-B)
    img = synth.wdr_image(20, 20, seed=12)
    _, big = orc.forward(img, orc.make_params(8, [4], eps=1e-9, alpha=0.7))
    _, small = orc.forward(img, orc.make_params(8, [4], eps=1e9))
    m = big.sigma2[0] > 1e-4
    assert np.allclose(big.weight[0][m], 0.7, rtol=1e-3)
    assert np.all(small.weight < 1e-9)


# --------------------------------------------------------------- adjoint --
def _fd_setup(orc, seed=0, H=6, W=7, radii=(1, 2, 9), flags=0):
    rng = np.random.default_rng(seed)
    img = synth.wdr_image(H, W, seed=seed).astype(np.float64)
    p = orc.make_params(5, list(radii), eps=[0.05, 0.1, 0.2][: len(radii)],
                        alpha=[1.0, 0.8, 1.2][: len(radii)], ld_min=0.05, ld_max=0.95, sat=0.6,
                        flags=flags)
    bins = orc.prepare(img.astype(np.float32), 5)["bins"]
    g = rng.standard_normal(img.shape)
    return img, p, bins, g


@pytest.mark.parametrize("flags", [0, 3])  # defaults; inclusive CDF + Algorithm 1's area
def test_adjoint_matches_central_differences_input(orc, flags):
    img, p, bins, g = _fd_setup(orc, flags=flags)
    gin, _ = orc.backward(img, p, g, lum_f64=True, bins=bins)
    rng = np.random.default_rng(1)
    idx = [tuple(rng.integers(0, s) for s in img.shape) for _ in range(12)]
    lum = img @ np.array([0.2126, 0.7152, 0.0722])
    idx += [np.unravel_index(np.argmin(lum), lum.shape) + (1,),
            np.unravel_index(np.argmax(lum), lum.shape) + (0,)]  # range terms
    for ix in idx:
        h = 1e-6 * max(abs(img[ix]), 1e-3)
        ip, im = img.copy(), img.copy()
        ip[ix] += h
        im[ix] -= h
        fd = (np.sum(g * orc.forward_fixed_bins(ip, p, bins))
              - np.sum(g * orc.forward_fixed_bins(im, p, bins))) / (2 * h)
        assert abs(fd - gin[ix]) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(gin).max()), (ix, fd, gin[ix])


@pytest.mark.parametrize("flags", [0, 3])
def test_adjoint_matches_central_differences_params(orc, flags):
    img, p, bins, g = _fd_setup(orc, seed=3, flags=flags)
    _, gp = orc.backward(img, p, g, lum_f64=True, bins=bins)

    def loss(q):
        return float(np.sum(g * orc.forward_fixed_bins(img, q, bins)))

    def bumped(attr, f, delta):
        q = orc.Params.from_buffer_copy(p)
        if f is None:
            setattr(q, attr, getattr(q, attr) + delta)
        else:
            getattr(q, attr)[f] += delta
        return q

    h = 1e-6
    checks = [("ld_min", None, gp["ld_min"]), ("ld_max", None, gp["ld_max"]), ("sat", None, gp["sat"])]
    checks += [("eps", f, gp["eps"][f]) for f in range(p.n_fields)]
    checks += [("alpha", f, gp["alpha"][f]) for f in range(p.n_fields)]
    for attr, f, an in checks:
        fd = (loss(bumped(attr, f, h)) - loss(bumped(attr, f, -h))) / (2 * h)
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (attr, f, fd, an)


def test_value_on_bin_edge_goes_to_upper_bin(orc):
    """Reading R3: a luminance equal to an edge belongs to the upper bin."""
    n = 8
    img = _grey(np.geomspace(0.01, 100.0, 40).reshape(5, 8))
    d = orc.prepare(img, n)
    k = 3
    edge = d["thr"][k - 1]
    hit = None
    for v in (edge, np.nextafter(edge, np.float32(0)), np.nextafter(edge, np.float32(np.inf))):
        for w in np.float32(v) * (1 + np.arange(-8, 9, dtype=np.float32) * np.float32(6e-8)):
            if orc.luminance(w, w, w) == edge:
                hit = w
                break
        if hit is not None:
            break
    assert hit is not None
    img[2, 3] = hit
    d2 = orc.prepare(img, n)
    assert d2["imin"] == d["imin"] and d2["imax"] == d["imax"]
    assert d2["lum"][2, 3] == edge and d2["bins"][2, 3] == k


# ------------------------------------------- reading variants (flags) -----
@pytest.mark.parametrize("radii", [[0], [(2, 1), 3], [1, 40]])
def test_variant_flags_against_brute_force(orc, radii):
    """Eq. 1 with <= (inclusive), Algorithm 1's unclipped area with zero
    padding, and Eq. 10 on i / imax, each against explicit numpy windows."""
    img = synth.wdr_image(9, 11, seed=21)
    n = 7
    d = orc.prepare(img, n)
    b, lh, lum = d["bins"].astype(np.int64), d["lhat"], d["lum"].astype(np.float64)
    H, W = b.shape
    lin = lum / lum.max()
    for flags in (orc.CDF_INCLUSIVE, orc.AREA_LITERAL, orc.VAR_LINEAR,
                  orc.CDF_INCLUSIVE | orc.AREA_LITERAL | orc.VAR_LINEAR):
        p = orc.make_params(n, radii, flags=flags)
        _, fl = orc.forward(img, p)
        _, dd = orc.forward_pixels(img, p, np.arange(W).repeat(H), np.tile(np.arange(H), W))
        vals = lin if flags & orc.VAR_LINEAR else lh
        for f, r in enumerate(radii):
            rx, ry = (r, r) if np.isscalar(r) else r
            padded = np.pad(vals, ((ry, ry), (rx, rx)))  # zeros outside the image
            for y in range(H):
                for x in range(W):
                    ys = slice(max(y - ry, 0), min(y + ry, H - 1) + 1)
                    xs = slice(max(x - rx, 0), min(x + rx, W - 1) + 1)
                    wb = b[ys, xs]
                    cnt = int(np.sum(wb <= b[y, x])) if flags & orc.CDF_INCLUSIVE else int(np.sum(wb < b[y, x]))
                    if flags & orc.AREA_LITERAL:
                        area = (2 * rx + 1) * (2 * ry + 1)
                        v = float(np.var(padded[y:y + 2 * ry + 1, x:x + 2 * rx + 1]))
                    else:
                        area = wb.size
                        v = float(np.var(vals[ys, xs]))
                    assert fl.cnt[f, y, x] == cnt and fl.area[f, y, x] == area
                    assert abs(fl.sigma2[f, y, x] - v) <= 1e-12 + 1e-9 * v
                    k = x * H + y  # the direct per-pixel path agrees
                    assert dd["cnt"][k, f] == cnt
                    assert abs(dd["sigma2"][k, f] - v) <= 1e-12 + 1e-9 * v


def test_inclusive_single_global_field_is_inclusive_histogram_cdf(orc):
    """s = 1 covering the image with Eq. 1 read as <=: P is the inclusive
    histogram CDF, so the brightest bin maps to ld_max."""
    img = synth.wdr_image(14, 17, seed=4)
    n = 10
    p = orc.make_params(n, [100], ld_min=0.0, ld_max=1.0, flags=orc.CDF_INCLUSIVE)
    _, fl = orc.forward(img, p)
    b = orc.prepare(img, n)["bins"]
    cdf = np.cumsum(np.bincount(b.ravel(), minlength=n)) / b.size
    assert np.allclose(fl.lf[0], cdf[b], atol=1e-15)
    assert np.isclose(fl.lf[0][b == b.max()].min(), 1.0)


def test_literal_area_constant_image(orc):
    """A constant image under Algorithm 1's area: P = 0 everywhere (nothing is
    strictly below), and near the border the zero padding gives a positive
    variance of the normalised log only if the value differs from 0; for the
    darkest possible constant image (lhat = 0 everywhere) it stays 0."""
    img = _grey(np.full((6, 8), 3.5))
    p = orc.make_params(8, [2], flags=orc.AREA_LITERAL)
    _, fl = orc.forward(img, p)
    assert np.all(fl.cnt == 0) and np.all(fl.area == 25)
    assert np.all(fl.sigma2 == 0)


def test_srgb_encode_published_values(orc):
    """IEC 61966-2-1 transfer function at published points: linear 0.5 ->
    0.7353569830524495 (8-bit 188), 0.18 -> 0.4613561295004773, the knee
    0.0031308 -> 0.040449936, 0 -> 0, 1 -> 1; 8-bit 128 decodes to linear
    0.21586050011389926 and encodes back."""
    enc = orc.srgb_encode([0.5, 0.18, 0.0031308, 0.0, 1.0, 0.21586050011389926])
    ref = [0.7353569830524495, 0.4613561295004773, 0.040449936, 0.0, 1.0, 128 / 255]
    assert np.allclose(enc, ref, rtol=0, atol=2e-9)
    assert orc.to_u8([0.5], srgb=True)[0] == 188 and orc.to_u8([0.5])[0] == 128


def test_forward_with_a_given_range(orc):
    """Streaming reuse reads an earlier frame's range: with the image's own
    range it is the plain forward; with a narrower range the bins come from
    that range's edges (numpy searchsorted on exp-spaced edges) and the
    normalised log is clamped to [0, 1]."""
    img = synth.wdr_image(12, 15, seed=6)
    n = 8
    p = orc.make_params(n, [1, 4])
    d = orc.prepare(img, n)
    own = (float(d["imin"]), float(d["imax"]))
    o1, f1 = orc.forward(img, p)
    o2, f2 = orc.forward(img, p, range_=own)
    assert np.array_equal(o1, o2) and np.array_equal(f1.cnt, f2.cnt)
    lum = d["lum"].astype(np.float64)
    lo, hi = np.quantile(lum, [0.2, 0.8]).astype(np.float32)
    _, f3 = orc.forward(img, p, range_=(lo, hi))
    k = np.arange(1, n)
    edges = np.exp(np.log(float(lo)) + (np.log(float(hi)) - np.log(float(lo))) * k / n)
    b = np.searchsorted(edges, lum, side="right")  # edge value -> upper bin
    lhat = np.clip((np.log(lum) - np.log(float(lo))) / (np.log(float(hi)) - np.log(float(lo))), 0, 1)
    H, W = b.shape
    for y in range(H):
        for x in range(W):
            w = (slice(max(y - 1, 0), min(y + 1, H - 1) + 1), slice(max(x - 1, 0), min(x + 1, W - 1) + 1))
            assert f3.cnt[0, y, x] == int(np.sum(b[w] < b[y, x]))
            v = float(np.var(lhat[w]))
            assert abs(f3.sigma2[0, y, x] - v) <= 1e-12 + 1e-9 * v


# ------------------------------------------ Eq. 1 numerators, counts only --
@pytest.mark.parametrize("flags", [0, 1])
@pytest.mark.parametrize("radii", [[0, 1, (3, 2)], [(7, 0), 40]])
def test_window_counts_against_brute_force(orc, flags, radii):
    """Counts alone (integral image of [b < k] per threshold) equal a direct
    count over every clipped window of a tiny image, for < and <=."""
    img = synth.wdr_image(13, 17, seed=len(radii) + flags)
    n = 6
    bins = orc.prepare(img, n)["bins"].astype(np.int64)
    p = orc.make_params(n, radii, flags=flags)
    got = orc.window_counts(bins, p)
    H, W = bins.shape
    for f, r in enumerate(radii):
        rx, ry = (r, r) if np.isscalar(r) else r
        for y in range(H):
            for x in range(W):
                win = bins[max(0, y - ry): y + ry + 1, max(0, x - rx): x + rx + 1]
                k = bins[y, x] + (1 if flags & 1 else 0)
                assert got[f, y, x] == np.count_nonzero(win < k)


def test_window_counts_equal_forward_counts(orc):
    """The counts-only path and the forward's per-bin box sums (Eq. 9 summed
    over the bins below) agree everywhere, on every reading variant."""
    img = synth.wdr_image(40, 57, seed=11)
    for flags in (0, 1, 2, 3):
        p = orc.make_params(32, [2, (9, 4), 30], flags=flags)
        _, fl = orc.forward(img, p)
        bins = orc.prepare(img, 32)["bins"]
        assert np.array_equal(orc.window_counts(bins, p), fl.cnt)


def test_threads_do_not_change_results(orc):
    """The per-pixel loops over host threads give the single-thread forward
    bit for bit, and the adjoint up to FP64 summation order."""
    img = synth.wdr_image(31, 45, seed=4)
    p = orc.make_params(16, [3, 11])
    rng = np.random.default_rng(0)
    gout = rng.standard_normal(img.shape)
    try:
        orc.set_threads(1)
        ref, fl = orc.forward(img, p)
        gi1, gp1 = orc.backward(img.astype(np.float64), p, gout)
        orc.set_threads(4)
        out, fl4 = orc.forward(img, p)
        gi4, gp4 = orc.backward(img.astype(np.float64), p, gout)
    finally:
        orc.set_threads(1)
    assert np.array_equal(out, ref) and np.array_equal(fl4.sigma2, fl.sigma2)
    assert np.allclose(gi4, gi1, rtol=1e-12, atol=1e-15 * np.abs(gi1).max())
    for k in gp1:
        assert np.allclose(gp4[k], gp1[k], rtol=1e-12, atol=1e-12)


# ------------------------------------- Section III capture front-end --
def _ln_err_bound(ldr):
    """|ln E_merged - ln E| for a linear camera: each exposure's estimate is
    off by at most ln(1 + 0.5/z) <= 0.5/z, and w(z) <= z, so the hat-weighted
    mean is off by at most 0.5 (contributing exposures) / sum of weights."""
    z = np.stack([a.astype(np.float64) for a in ldr])
    w = np.where(z <= 127, z, 255 - z)
    return 0.5 * (w > 0).sum(axis=0) / np.maximum(w.sum(axis=0), 1e-300), w.sum(axis=0)


def test_merge_linear_camera_recovers_radiance(orc):
    """Under a linear response the merged radiance equals the scene radiance
    within the quantisation bound wherever some exposure is unclipped."""
    img = synth.wdr_image(24, 31, seed=5).astype(np.float64)
    times = [5e-5, 5e-4, 5e-3, 5e-2, 5e-1, 5.0]  # six exposures a decade apart cover the image's range
    ldr = synth.camera_exposures(img, times, gamma=1.0, xsat=1.0)
    g = synth.camera_log_response(gamma=1.0, xsat=1.0)
    E = orc.merge_exposures(ldr, times, g)
    bound, wsum = _ln_err_bound(ldr)
    ok = wsum > 0
    assert ok.mean() > 0.99
    err = np.abs(np.log(E) - np.log(img))
    assert np.all(err[ok] <= bound[ok] + 1e-12)


def test_merge_single_exposure_inverts_the_response(orc):
    rng = np.random.default_rng(3)
    z = rng.integers(1, 255, size=(7, 9, 3)).astype(np.uint8)
    g = synth.camera_log_response(gamma=2.2, xsat=3.0)
    E = orc.merge_exposures([z], [0.25], g)
    expect = np.exp(g[np.arange(3)[None, None, :], z] - np.log(0.25))
    assert np.allclose(E, expect, rtol=1e-14)


def test_merge_time_scaling_and_order(orc):
    """Scaling every exposure time by c divides the radiance by c; the order
    of the exposures does not matter."""
    img = synth.wdr_image(11, 13, seed=6).astype(np.float64)
    times = np.array([2e-4, 3e-3, 2e-2, 5e-1])
    ldr = synth.camera_exposures(img, times)
    g = synth.camera_log_response()
    E = orc.merge_exposures(ldr, times, g)
    E2 = orc.merge_exposures(ldr, times * 8.0, g)
    assert np.allclose(E2 * 8.0, E, rtol=1e-12)
    perm = [2, 0, 3, 1]
    E3 = orc.merge_exposures([ldr[i] for i in perm], times[perm], g)
    assert np.allclose(E3, E, rtol=1e-12)


def test_merge_hat_weights_and_clipped_fallback(orc):
    """Values 0 and 255 carry no weight: a pixel at 200 in one exposure and 255
    in the other takes the first alone; a pixel clipped everywhere takes the
    shortest exposure when saturated and the longest when black."""
    g = synth.camera_log_response(gamma=1.0)
    a = np.array([[[200, 0, 255]]], np.uint8)
    b = np.array([[[255, 0, 255]]], np.uint8)
    times = [0.5, 2.0]
    E = orc.merge_exposures([a, b], times, g)[0, 0]
    assert np.isclose(E[0], np.exp(g[0, 200] - np.log(0.5)), rtol=1e-14)
    assert np.isclose(E[1], np.exp(g[1, 0] - np.log(2.0)), rtol=1e-14)    # black: longest
    assert np.isclose(E[2], np.exp(g[2, 255] - np.log(0.5)), rtol=1e-14)  # saturated: shortest
