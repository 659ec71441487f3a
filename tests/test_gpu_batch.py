"""Batched forward (one launch per stage for the whole batch, the sweep as a
persistent kernel over an (image, tile) queue, captured in a CUDA graph):
every image must equal its own single-image forward bit for bit, graph
replays must track the current input contents, and one image of the batch is
checked against the FP64 oracle."""
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


SIZES = [(97, 61), (640, 480), (333, 257), (1, 1), (1280, 720), (45, 900), (200, 3)]


def _single(ctx, x):
    y = torch.empty_like(x) if x.dtype != torch.float16 else torch.empty_like(x)
    tm.tm_forward(ctx, x, y)
    return y


@pytest.mark.parametrize("dtype", [np.float32, np.float16])
def test_batch_equals_per_image(dtype):
    p = tm.make_params(32, [4, 16, 64])
    imgs = [synth.wdr_image(h, w, seed=i, dtype=dtype) for i, (w, h) in enumerate(SIZES)]
    xs = [torch.from_numpy(a).cuda() for a in imgs]
    ys = [torch.empty_like(x) for x in xs]
    ctx = tm.tm_create(p)
    try:
        tm.tm_forward_batch(ctx, xs, ys)
        torch.cuda.synchronize()
        for x, y in zip(xs, ys):
            ref = _single(ctx, x)
            torch.cuda.synchronize()
            assert torch.equal(y, ref)
    finally:
        tm.tm_destroy(ctx)


def test_batch_of_more_images_than_one_descriptor_launch():
    """The job descriptors reach the device as kernel parameters, 32 per
    launch: batches of 33 and 70 images take two and three such launches,
    first as a captured graph and then as its replay; every image equals its
    own call."""
    p = tm.make_params(16, [2, 9])
    rng = np.random.default_rng(5)
    ctx = tm.tm_create(p)
    try:
        for n in (33, 70):
            sizes = [(int(rng.integers(8, 90)), int(rng.integers(8, 90))) for _ in range(n)]
            xs = [torch.from_numpy(synth.wdr_image(h, w, seed=100 + i)).cuda() for i, (w, h) in enumerate(sizes)]
            ys = [torch.empty_like(x) for x in xs]
            refs = [_single(ctx, x) for x in xs]
            for _ in range(2):  # capture, then replay
                for y in ys:
                    y.zero_()
                tm.tm_forward_batch(ctx, xs, ys)
                torch.cuda.synchronize()
                for y, ref in zip(ys, refs):
                    assert torch.equal(y, ref)
    finally:
        tm.tm_destroy(ctx)


def test_graph_replay_tracks_inputs():
    p = tm.make_params(16, [2, 9, 40])
    sizes = [(300, 200), (128, 96), (257, 255)]
    xs = [torch.from_numpy(synth.wdr_image(h, w, seed=10 + i)).cuda() for i, (w, h) in enumerate(sizes)]
    ys = [torch.empty_like(x) for x in xs]
    ctx = tm.tm_create(p)
    try:
        tm.tm_forward_batch(ctx, xs, ys)  # captures
        first = [y.clone() for y in ys]
        tm.tm_forward_batch(ctx, xs, ys)  # replays
        torch.cuda.synchronize()
        for a, b in zip(first, ys):
            assert torch.equal(a, b)
        # new contents in the same buffers: the replay must see them
        for i, (w, h) in enumerate(sizes):
            xs[i].copy_(torch.from_numpy(synth.wdr_image(h, w, seed=50 + i)).cuda())
        tm.tm_forward_batch(ctx, xs, ys)
        torch.cuda.synchronize()
        for x, y in zip(xs, ys):
            assert torch.equal(y, _single(ctx, x))
        # a single forward in between invalidates nothing visible to the caller
        _single(ctx, xs[0])
        tm.tm_forward_batch(ctx, xs, ys)
        torch.cuda.synchronize()
        for x, y in zip(xs, ys):
            assert torch.equal(y, _single(ctx, x))
    finally:
        tm.tm_destroy(ctx)


def test_single_image_graph_cache():
    """Single-image forwards replay a cached CUDA graph per (input, output)
    pair once the pair comes back (a pair seen once runs its launches
    directly). Three images cycled three times (captured on their second
    call, replayed on the third), then eight images of several sizes cycled
    twice (more pairs than graph slots; the workspace grows on the way, which
    drops the cache), a batch in between and new contents in a cached input.
    Every output equals the same forward without graphs (stage timing on),
    bit for bit."""
    p = tm.make_params(16, [2, 9, 40])
    sizes = [(300, 200), (128, 96), (257, 255), (64, 64), (520, 130), (96, 300), (200, 200), (33, 47)]
    xs = [torch.from_numpy(synth.wdr_image(h, w, seed=20 + i)).cuda() for i, (w, h) in enumerate(sizes)]
    ys = [torch.empty_like(x) for x in xs]
    ref_ctx = tm.tm_create(p)
    ctx = tm.tm_create(p)
    try:
        tm.tm_set_option(ref_ctx, tm.TM_OPT_HIST_PATH, 1)
        tm.tm_set_option(ref_ctx, tm.TM_OPT_STAGE_TIMING, 1)  # no graphs
        tm.tm_set_option(ctx, tm.TM_OPT_HIST_PATH, 1)

        def ref(x):
            y = torch.empty_like(x)
            tm.tm_forward(ref_ctx, x, y)
            return y

        def check(k, tag):
            tm.tm_forward(ctx, xs[k], ys[k])
            torch.cuda.synchronize()
            assert torch.equal(ys[k], ref(xs[k])), (tag, k)

        for rnd in range(3):
            for k in range(3):
                check(k, ("three", rnd))
        for rnd in range(2):
            for k in range(len(xs)):
                check(k, ("eight", rnd))
            if rnd == 0:
                zs = [torch.empty_like(x) for x in xs[:3]]
                tm.tm_forward_batch(ctx, xs[:3], zs)
                torch.cuda.synchronize()
                for x, z in zip(xs[:3], zs):
                    assert torch.equal(z, ref(x))
        # new contents in a cached input: the replay sees them
        xs[0].copy_(torch.from_numpy(synth.wdr_image(200, 300, seed=99)).cuda())
        check(0, "new contents")
        check(0, "new contents, again")
    finally:
        tm.tm_destroy(ctx)
        tm.tm_destroy(ref_ctx)


def test_batch_image_matches_oracle(orc):
    p = tm.make_params(32, [4, 16, 64])
    op = orc.make_params(32, [4, 16, 64], eps=float(np.float32(0.1)), sat=float(np.float32(0.6)))
    imgs = [synth.wdr_image(h, w, seed=i) for i, (w, h) in enumerate([(90, 70), (160, 120), (50, 40)])]
    xs = [torch.from_numpy(a).cuda() for a in imgs]
    ys = [torch.empty_like(x) for x in xs]
    ctx = tm.tm_create(p)
    try:
        tm.tm_forward_batch(ctx, xs, ys)
        torch.cuda.synchronize()
    finally:
        tm.tm_destroy(ctx)
    for a, y in zip(imgs, ys):
        ref, _ = orc.forward(a, op)
        got = y.cpu().numpy().astype(np.float64)
        assert np.all(np.abs(got - ref) <= 1e-4 * np.maximum(np.abs(ref), 1e-3))


def test_empty_batch_is_noop():
    ctx = tm.tm_create(tm.make_params(8, [1]))
    try:
        tm.tm_forward_batch(ctx, [], [])
        assert tm.tm_last_launch_count(ctx) == 0
    finally:
        tm.tm_destroy(ctx)


def test_unsynchronised_calls_of_different_sizes():
    """Calls issued back to back without synchronisation, on images whose sizes
    (and so job layouts, sweep plans and tile queues) all differ, interleaved
    with batch captures and replays: the per-call descriptor staging must not
    be rewritten while an earlier call's copy is still pending."""
    p = tm.make_params(32, [4, 16, 64])
    sizes = [(1500, 1000), (97, 61), (1200, 900), (333, 257), (1024, 1024), (45, 900), (800, 600)]
    xs = [torch.from_numpy(synth.wdr_image(h, w, seed=70 + i)).cuda() for i, (w, h) in enumerate(sizes)]
    ctx = tm.tm_create(p)
    try:
        refs = []
        for x in xs:
            refs.append(_single(ctx, x))
            torch.cuda.synchronize()
        ys = [torch.empty_like(x) for x in xs]
        for rep in range(3):
            for x, y in zip(xs, ys):
                tm.tm_forward(ctx, x, y)
            yb = [torch.empty_like(x) for x in xs[:3]]
            tm.tm_forward_batch(ctx, xs[:3], yb)  # capture, then replays
            for x, y in zip(reversed(xs), reversed(ys)):
                tm.tm_forward(ctx, x, y)
            tm.tm_forward_batch(ctx, xs[:3], yb)
        torch.cuda.synchronize()
        for y, r in zip(ys, refs):
            assert torch.equal(y, r)
        for y, r in zip(yb, refs[:3]):
            assert torch.equal(y, r)
    finally:
        tm.tm_destroy(ctx)


def test_uneven_batch_c4_shapes(orc):
    """An uneven batch shaped like the 64-image workload (64 bins, radii
    8/32/128): 4096 x 3072, 640 x 480, 1920 x 1080, a 16:9 and a 4:3 image.
    Every image equals its own single-image forward bit for bit (the largest
    holds whole-wave tiles over 16 strips), and the largest matches the
    oracle's direct per-pixel evaluation at sampled pixels (corners, borders,
    strip seams, random)."""
    sizes = [(4096, 3072), (640, 480), (1920, 1080), (1280, 720), (2048, 1536)]
    p = tm.make_params(64, [8, 32, 128])
    op = orc.make_params(64, [8, 32, 128], eps=float(np.float32(0.1)), sat=float(np.float32(0.6)))
    imgs = [synth.wdr_image(h, w, seed=200 + i) for i, (w, h) in enumerate(sizes)]
    xs = [torch.from_numpy(a).cuda() for a in imgs]
    ys = [torch.empty_like(x) for x in xs]
    ctx = tm.tm_create(p)
    try:
        tm.tm_set_option(ctx, tm.TM_OPT_HIST_PATH, 1)
        tm.tm_forward_batch(ctx, xs, ys)
        torch.cuda.synchronize()
        for x, y in zip(xs, ys):
            ref = _single(ctx, x)
            torch.cuda.synchronize()
            assert torch.equal(y, ref)
        big = ys[0].cpu().numpy()
    finally:
        tm.tm_destroy(ctx)
    W, H = sizes[0]
    rng = np.random.default_rng(9)
    yy = np.concatenate([[0, 0, H - 1, H - 1, 128, H - 129, 1500, 7], rng.integers(0, H, 80)])
    xx = np.concatenate([[0, W - 1, 0, W - 1, 255, 256, 3839, 3840], rng.integers(0, W, 80)])
    orc.set_threads(orc.num_procs())
    try:
        ref, _ = orc.forward_pixels(imgs[0], op, xx, yy)
    finally:
        orc.set_threads(1)
    got = big[yy, xx].astype(np.float64)
    assert np.all(np.abs(got - ref) <= 1e-4 * np.maximum(np.abs(ref), 1e-3))


def _batch_stages(ctx, xs, ys):
    tm.tm_set_option(ctx, tm.TM_OPT_STAGE_TIMING, 1)
    tm.tm_stage_times(ctx)
    tm.tm_forward_batch(ctx, xs, ys)
    names = set(tm.tm_stage_times(ctx))
    tm.tm_set_option(ctx, tm.TM_OPT_STAGE_TIMING, 0)
    return names


def test_paper_preset_batch_takes_the_batched_materialised_path():
    """The paper's preset (s = 5 fields halving from a 2000 x 1500 image, n = 5)
    is too wide for the sweep at these sizes: the batch runs as one batched
    materialised pass (no per-image fallback) and equals per-image calls bit
    for bit, first captured and then replayed."""
    p = tm.tm_params_pyramid(2000, 1500, 5, 5)
    sizes = [(2000, 1500), (1024, 768), (640, 480)]
    xs = [torch.from_numpy(synth.wdr_image(h, w, seed=300 + i)).cuda() for i, (w, h) in enumerate(sizes)]
    ys = [torch.empty_like(x) for x in xs]
    ctx = tm.tm_create(p)
    try:
        for rep in range(2):
            for y in ys:
                y.zero_()
            names = _batch_stages(ctx, xs, ys)
            assert "batch_materialised" in names and "batch" not in names, names
            torch.cuda.synchronize()
            for x, y in zip(xs, ys):
                assert torch.equal(y, _single(ctx, x))
    finally:
        tm.tm_destroy(ctx)


def test_mixed_batch_splits_by_path():
    """Fields that fit the sweep on a small image but not on a large one: the
    batch splits into a fused pass and a materialised pass, each image equal
    to its own call."""
    p = tm.make_params(16, [4, (700, 600)])
    sizes = [(2400, 1800), (300, 200), (1600, 1200), (97, 61)]
    xs = [torch.from_numpy(synth.wdr_image(h, w, seed=400 + i)).cuda() for i, (w, h) in enumerate(sizes)]
    ys = [torch.empty_like(x) for x in xs]
    ctx = tm.tm_create(p)
    try:
        tm.tm_set_option(ctx, tm.TM_OPT_HIST_PATH, 1)
        with pytest.raises(tm.TmError):  # forcing the sweep: the large images do not fit
            tm.tm_forward_batch(ctx, xs, ys)
        tm.tm_set_option(ctx, tm.TM_OPT_HIST_PATH, 0)
        names = _batch_stages(ctx, xs, ys)
        assert "batch_materialised" in names, names
        torch.cuda.synchronize()
        for x, y in zip(xs, ys):
            assert torch.equal(y, _single(ctx, x))
    finally:
        tm.tm_destroy(ctx)
