"""GPU parity of the Section III capture front-end (tm_merge_exposures:
Debevec and Malik's radiance map from several exposures) against the FP64
oracle, alone and followed by the tone-mapping forward."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2102_01289_gb300 as tm  # noqa: E402

TIMES = [5e-5, 5e-4, 5e-3, 5e-2]  # four exposures, a decade apart (the paper captures four)


def _merge_gpu(ldr, times, g, dtype=torch.float32):
    xs = [torch.from_numpy(a).cuda() for a in ldr]
    H, W = ldr[0].shape[:2]
    out = torch.empty((H, W, 3), dtype=dtype, device="cuda")
    tm.tm_merge_exposures(xs, times, g, out)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("H,W,gamma", [(97, 61, 2.2), (480, 640, 1.0), (1, 1, 2.2), (33, 1000, 1.8)])
def test_merge_matches_oracle(orc, H, W, gamma):
    img = synth.wdr_image(H, W, seed=H + W).astype(np.float64)
    ldr = synth.camera_exposures(img, TIMES, gamma=gamma)
    g = synth.camera_log_response(gamma=gamma)
    ref = orc.merge_exposures(ldr, TIMES, g)
    got = _merge_gpu(ldr, [float(np.float32(t)) for t in TIMES], g)
    assert np.all(np.abs(got - ref) <= 2e-5 * ref), np.abs(got / ref - 1).max()
    half = _merge_gpu(ldr, TIMES, g, torch.float16)
    assert np.all(np.abs(half - ref) <= 1e-3 * ref + 1e-7)


def test_merge_clipped_and_extreme_pixels(orc):
    """Pixels black or saturated in every exposure, and single-exposure and
    eight-exposure merges, against the oracle's readings."""
    rng = np.random.default_rng(2)
    ldr = [rng.integers(0, 256, size=(50, 70, 3)).astype(np.uint8) for _ in range(8)]
    ldr[0][:5] = 255
    for a in ldr:
        a[:5] = 255
        a[5:10] = 0
    times = [float(np.float32(t)) for t in np.geomspace(1e-4, 1.0, 8)]
    g = synth.camera_log_response(gamma=2.2, xsat=2.0)
    for n in (1, 4, 8):
        ref = orc.merge_exposures(ldr[:n], times[:n], g)
        got = _merge_gpu(ldr[:n], times[:n], g)
        assert np.all(np.abs(got - ref) <= 2e-5 * ref)


def test_merge_then_tone_map_matches_oracle(orc):
    """The paper's application: four exposures merged into a WDR image, then
    tone-mapped (32 bins, radii 4/16/64), against the oracle doing the same."""
    H, W = 200, 300
    img = synth.wdr_image(H, W, seed=77).astype(np.float64)
    g = synth.camera_log_response()
    ldr = synth.camera_exposures(img, TIMES)
    times = [float(np.float32(t)) for t in TIMES]
    xs = [torch.from_numpy(a).cuda() for a in ldr]
    wdr = torch.empty((H, W, 3), dtype=torch.float32, device="cuda")
    tm.tm_merge_exposures(xs, times, g, wdr)
    out = torch.empty_like(wdr)
    p = tm.make_params(32, [4, 16, 64])
    ctx = tm.tm_create(p)
    try:
        tm.tm_forward(ctx, wdr, out)
        torch.cuda.synchronize()
    finally:
        tm.tm_destroy(ctx)
    # the two merges agree within 2e-5; the tone-mapping comparison then takes
    # the GPU's merged image as the common input (a last-bit difference in the
    # input could move a pixel across a bin edge)
    merged = orc.merge_exposures(ldr, times, g).astype(np.float32)
    gpu_merged = wdr.cpu().numpy()
    assert np.all(np.abs(gpu_merged.astype(np.float64) - merged) <= 2e-5 * merged)
    op = orc.make_params(32, [4, 16, 64], eps=float(np.float32(0.1)), sat=float(np.float32(0.6)))
    ref, _ = orc.forward(gpu_merged, op)  # the forward on the GPU's own WDR image
    got = out.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got - ref) <= 1e-4 * np.maximum(np.abs(ref), 1e-3))
