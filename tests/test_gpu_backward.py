"""GPU parity of the hand-written adjoint (tm_backward / TMFunction).

Against the FP64 oracle adjoint (bins fixed, float luminance as in the
forward): input and parameter gradients within 1e-3 relative, with a floor of
1e-3 of the largest input gradient. Against central finite differences of the
GPU forward itself at pixels away from bin edges and from the range extremes.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2102_01289_gb300 as tm  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    tm.build()


def _pair(orc, n, radii, eps, alpha, ld_min=0.05, ld_max=0.95, sat=0.6, flags=0):
    gp = tm.make_params(n, radii, eps, alpha, ld_min, ld_max, sat, flags=flags)
    s = len(radii)
    op = orc.make_params(n, radii, eps=[float(gp.eps[f]) for f in range(s)],
                         alpha=[float(gp.alpha[f]) for f in range(s)], ld_min=float(gp.ld_min),
                         ld_max=float(gp.ld_max), sat=float(gp.sat), flags=flags)
    return gp, op


def _gpu_backward(img, gp, gout):
    x = torch.from_numpy(img).cuda()
    g = torch.from_numpy(gout.astype(np.float32)).cuda()
    gin = torch.empty_like(x)
    gpar = torch.empty(3 + 2 * gp.n_fields, dtype=torch.float32, device="cuda")
    ctx = tm.tm_create(gp)
    try:
        tm.tm_backward(ctx, x, g, gin, gpar)
        torch.cuda.synchronize()
    finally:
        tm.tm_destroy(ctx)
    return gin.cpu().numpy().astype(np.float64), gpar.cpu().numpy().astype(np.float64)


# The last two cases (added below): 300 x 320 with the radii 8/32/128 (r = 128
# windows lie wholly inside the image; the fixed-point integral pass spans
# several row segments), and 40 x 2200, whose rows span three 1024-column
# chunks of the integral tiles (row and tile totals carried across chunks).
CASES = [
    (40, 56, 16, [2, 7, 30]),
    (33, 47, 32, [(3, 1), 9]),
    (64, 64, 8, [4, 16, 64]),  # last window larger than the image
    (37, 53, 16, [0, 1, 3, (7, 2), 12, 25, (32767, 4), 32767]),  # 8 fields up to the largest radius
]


@pytest.mark.parametrize("flags", [0, 3])  # defaults; inclusive CDF + Algorithm 1's area
@pytest.mark.parametrize("H,W,n,radii", CASES + [(300, 320, 32, [8, 32, 128]), (40, 2200, 16, [3, 12, 40])])
def test_backward_matches_oracle_adjoint(orc, H, W, n, radii, flags):
    rng = np.random.default_rng(H + W)
    img = synth.wdr_image(H, W, seed=H * 7 + W)
    s = len(radii)
    gp, op = _pair(orc, n, radii, eps=[(0.1, 0.03, 0.2)[f % 3] for f in range(s)],
                   alpha=[(1.0, 0.8, 1.2)[f % 3] for f in range(s)], flags=flags)
    gout = rng.standard_normal(img.shape)
    gin, gpar = _gpu_backward(img, gp, gout)
    orc.set_threads(orc.num_procs())  # windows of up to 257 x 257 pixels: the oracle loops are long
    try:
        ref_in, ref_p = orc.backward(img.astype(np.float64), op, gout, lum_f64=False)
    finally:
        orc.set_threads(1)
    floor = 1e-3 * np.abs(ref_in).max()
    err = np.abs(gin - ref_in)
    assert np.all(err <= 1e-3 * np.abs(ref_in) + floor), (err.max(), np.abs(ref_in).max())
    ref_vec = np.concatenate([[ref_p["ld_min"], ref_p["ld_max"], ref_p["sat"]], ref_p["eps"], ref_p["alpha"]])
    assert np.allclose(gpar, ref_vec, rtol=1e-3, atol=1e-3 * np.abs(ref_vec).max())


def test_backward_reuses_forward_intermediates():
    """TM_OPT_BACKWARD_REUSE: right after a forward of the same images the
    backward takes the forward's intermediates (fewer launches) with results
    identical to the recomputation; other images, or a forward of other
    images in between, are recomputed."""
    n, H, W = 3, 60, 80
    xs = [torch.from_numpy(synth.wdr_image(H, W, seed=70 + k)).cuda() for k in range(n)]
    ys = [torch.empty_like(x) for x in xs]
    gs = [torch.randn_like(x) for x in xs]
    p = tm.make_params(16, [2, 8, 30])

    def run(reuse, between=None):
        ctx = tm.tm_create(p)
        try:
            tm.tm_set_option(ctx, tm.TM_OPT_BACKWARD_REUSE, reuse)
            gins = [torch.empty_like(x) for x in xs]
            gp = torch.empty(9, device="cuda")
            tm.tm_forward_batch(ctx, xs, ys)
            if between is not None:
                tm.tm_forward(ctx, between, torch.empty_like(between))
            tm.tm_backward_batch(ctx, xs, gs, gins, gp)
            launches = tm.tm_last_launch_count(ctx)
            gin1 = torch.empty_like(xs[0])
            gp1 = torch.empty(9, device="cuda")
            tm.tm_forward(ctx, xs[0], ys[0])
            tm.tm_backward(ctx, xs[0], gs[0], gin1, gp1)
            torch.cuda.synchronize()
            return [g.cpu() for g in gins], gp.cpu(), gin1.cpu(), gp1.cpu(), launches
        finally:
            tm.tm_destroy(ctx)

    ref = run(0)
    got = run(1)
    for a, b in zip(ref[0], got[0]):
        assert torch.equal(a, b)
    assert torch.equal(ref[1], got[1]) and torch.equal(ref[2], got[2]) and torch.equal(ref[3], got[3])
    assert got[4] < ref[4]  # the recomputation's launches were skipped
    other = torch.from_numpy(synth.wdr_image(50, 50, seed=99)).cuda()
    mixed = run(1, between=other)
    for a, b in zip(ref[0], mixed[0]):
        assert torch.equal(a, b)
    assert mixed[4] == ref[4]


def test_backward_matches_gpu_finite_differences(orc):
    """Central differences of the GPU forward (h = 1e-3 relative) at pixels
    whose normalised log sits at least a quarter bin from any edge."""
    H, W, n = 48, 48, 16
    img = synth.wdr_image(H, W, seed=3)
    gp, _ = _pair(orc, n, [2, 6, 20], eps=[0.1, 0.05, 0.2], alpha=[1.0, 1.0, 1.0])
    rng = np.random.default_rng(0)
    gout = rng.standard_normal(img.shape)
    gin, _ = _gpu_backward(img, gp, gout)
    pre = orc.prepare(img, n)
    u = n * pre["lhat"]
    frac = u - np.floor(u)
    ok = (frac > 0.25) & (frac < 0.75)
    lum = pre["lum"]
    ok &= (lum != lum.min()) & (lum != lum.max())
    ys, xs = np.nonzero(ok)
    pick = rng.choice(len(ys), 6, replace=False)
    ctx = tm.tm_create(gp)
    g = torch.from_numpy(gout).cuda()

    def loss(im):
        x = torch.from_numpy(im).cuda()
        y = torch.empty_like(x)
        tm.tm_forward(ctx, x, y)
        return float((y.double() * g).sum())

    try:
        for k in pick:
            y0, x0, c = ys[k], xs[k], int(rng.integers(0, 3))
            h = 1e-3 * float(img[y0, x0, c])
            ip, im = img.copy(), img.copy()
            ip[y0, x0, c] += h
            im[y0, x0, c] -= h
            hp = float(ip[y0, x0, c]) - float(img[y0, x0, c])
            hm = float(img[y0, x0, c]) - float(im[y0, x0, c])
            fd = (loss(ip) - loss(im)) / (hp + hm)
            an = gin[y0, x0, c]
            assert abs(fd - an) <= 2e-2 * abs(an) + 1e-3 * np.abs(gin).max(), (y0, x0, c, fd, an)
    finally:
        tm.tm_destroy(ctx)


def test_autograd_function_batch():
    H, W = 40, 52
    imgs = np.stack([synth.wdr_image(H, W, seed=s) for s in range(3)])
    p = tm.make_params(16, [2, 8, 30])
    theta = tm.params_tensor(p).requires_grad_(True)
    cache = tm._CtxCache(p)
    x = torch.from_numpy(imgs).cuda().requires_grad_(True)
    out = tm.TMFunction.apply(x, theta, cache)
    g = torch.randn_like(out)
    (out * g).sum().backward()
    # the same gradients through the C ABI, image by image
    ctx = tm.tm_create(p)
    try:
        gp_sum = torch.zeros(theta.numel(), device="cuda")
        for b in range(3):
            gin = torch.empty_like(x[b])
            gpar = torch.empty(theta.numel(), device="cuda")
            tm.tm_backward(ctx, x[b].detach().contiguous(), g[b].contiguous(), gin, gpar)
            gp_sum += gpar
            # equal but for the order of floating-point atomics in the range terms
            assert torch.allclose(x.grad[b], gin, rtol=1e-6, atol=1e-7 * float(gin.abs().max()))
        torch.cuda.synchronize()
        assert torch.allclose(theta.grad, gp_sum.cpu(), rtol=1e-5, atol=1e-6)
    finally:
        tm.tm_destroy(ctx)
        cache.close()


def test_backward_batch_matches_per_image():
    """tm_backward_batch over images of different sizes (one batched forward
    recompute, then the adjoint per image) equals tm_backward image by image;
    grad_params is the sum over the images."""
    sizes = [(40, 52), (97, 61), (128, 128), (33, 200)]
    p = tm.make_params(16, [2, 8, 30], eps=[0.1, 0.05, 0.2], alpha=[1.0, 0.8, 1.2])
    rng = np.random.default_rng(5)
    xs = [torch.from_numpy(synth.wdr_image(h, w, seed=20 + i)).cuda() for i, (w, h) in enumerate(sizes)]
    gs = [torch.from_numpy(rng.standard_normal((h, w, 3)).astype(np.float32)).cuda() for (w, h) in sizes]
    ctx = tm.tm_create(p)
    try:
        ref_in, ref_p = [], torch.zeros(3 + 2 * 3, device="cuda")
        for x, g in zip(xs, gs):
            gi = torch.empty_like(x)
            gp = torch.empty(3 + 2 * 3, device="cuda")
            tm.tm_backward(ctx, x, g, gi, gp)
            ref_in.append(gi)
            ref_p += gp
        gins = [torch.empty_like(x) for x in xs]
        gp_b = torch.empty(3 + 2 * 3, device="cuda")
        tm.tm_backward_batch(ctx, xs, gs, gins, gp_b)
        torch.cuda.synchronize()
        for a, b in zip(gins, ref_in):
            assert torch.allclose(a, b, rtol=1e-6, atol=1e-7 * float(b.abs().max()))
        assert torch.allclose(gp_b, ref_p, rtol=1e-5, atol=1e-6 * float(ref_p.abs().max()))
        # without grad_in, and an empty batch (zero parameter gradient)
        tm.tm_backward_batch(ctx, xs, gs, None, gp_b)
        torch.cuda.synchronize()
        assert torch.allclose(gp_b, ref_p, rtol=1e-5, atol=1e-6 * float(ref_p.abs().max()))
        tm.tm_backward_batch(ctx, [], [], None, gp_b)
        torch.cuda.synchronize()
        assert float(gp_b.abs().max()) == 0.0
    finally:
        tm.tm_destroy(ctx)


def test_backward_rejects_linear_variance():
    p = tm.make_params(8, [1, 3], flags=tm.TM_FLAG_VAR_LINEAR)
    x = torch.from_numpy(synth.wdr_image(16, 16, seed=1)).cuda()
    ctx = tm.tm_create(p)
    try:
        with pytest.raises(tm.TmError) as e:
            tm.tm_backward(ctx, x, torch.ones_like(x), torch.empty_like(x))
        assert e.value.status == tm.TM_EUNSUPPORTED
    finally:
        tm.tm_destroy(ctx)
