"""Seeded synthetic wide-dynamic-range inputs.

This module only draws inputs; it holds none of the tone-mapping arithmetic
(no luminance weights, no logarithmic binning, no windows) so that both the
CUDA path's tests/benchmark and the CPU oracle can take their inputs from it.

Recipe (one image):
  1. log10 luminance is a linear ramp along a random direction spanning the
     requested decades [lo, hi];
  2. ``n_rects`` axis-aligned rectangles (position uniform, each side 3-30 % of
     the image side) add +-U(0.5, 2) decades (sign with probability 1/2);
  3. the result is clipped to [lo, hi] decades;
  4. luminance is multiplied per pixel by (1 + noise * N(0, 1));
  5. chroma (c_r, c_g, c_b) ~ U(0.2, 0.8), drawn once for the background and
     once per rectangle; RGB = c * Y / mean(c).
The wide-dynamic-range photographs the paper evaluates on are not available;
these images stand in for them with the same value range and structure (a
smooth global trend, large bright/dark regions, sensor-like noise).
"""
from __future__ import annotations

import numpy as np

__all__ = ["wdr_image", "wdr_mosaic", "wdr_video_frame", "uneven_sizes", "box_image", "wdr_device",
           "camera_exposures", "camera_log_response"]


def _draw_scene(rng: np.random.Generator, H: int, W: int, n_rects: int):
    theta = rng.uniform(0.0, 2.0 * np.pi)
    rects = []
    for _ in range(n_rects):
        rh = int(max(1, round(rng.uniform(0.03, 0.30) * H)))
        rw = int(max(1, round(rng.uniform(0.03, 0.30) * W)))
        y0 = float(rng.uniform(0, max(H - rh, 1)))
        x0 = float(rng.uniform(0, max(W - rw, 1)))
        amp = rng.uniform(0.5, 2.0) * (1.0 if rng.uniform() < 0.5 else -1.0)
        chroma = rng.uniform(0.2, 0.8, size=3)
        vy, vx = rng.uniform(-3.0, 3.0, size=2)  # pixels per frame (video only)
        rects.append((y0, x0, rh, rw, amp, chroma, vy, vx))
    bg_chroma = rng.uniform(0.2, 0.8, size=3)
    return theta, rects, bg_chroma


def _render(H, W, lo, hi, theta, rects, bg_chroma, noise_rng, noise, shift=0.0,
            t=0.0, dtype=np.float32):
    yy = np.linspace(-0.5, 0.5, H, dtype=np.float64)[:, None]
    xx = np.linspace(-0.5, 0.5, W, dtype=np.float64)[None, :]
    ramp = np.cos(theta) * xx + np.sin(theta) * yy  # in [-0.71, 0.71]
    ramp = (ramp - ramp.min()) / max(ramp.max() - ramp.min(), 1e-12)
    dec = lo + (hi - lo) * ramp + shift
    chroma = np.empty((H, W, 3), np.float64)
    chroma[...] = bg_chroma
    for (y0, x0, rh, rw, amp, c, vy, vx) in rects:
        ys = int(round(y0 + vy * t)) % max(H, 1)
        xs = int(round(x0 + vx * t)) % max(W, 1)
        ye, xe = min(ys + rh, H), min(xs + rw, W)
        dec[ys:ye, xs:xe] += amp
        chroma[ys:ye, xs:xe] = c
    np.clip(dec, lo, hi, out=dec)
    Y = np.power(10.0, dec)
    Y *= 1.0 + noise * noise_rng.standard_normal((H, W))
    np.maximum(Y, 10.0 ** lo * 1e-3, out=Y)
    rgb = chroma * (Y / chroma.mean(axis=2))[..., None]
    return rgb.astype(dtype)


def wdr_image(H: int, W: int, seed: int, decades=(-2.0, 4.0), n_rects: int = 20,
              noise: float = 0.02, dtype=np.float32) -> np.ndarray:
    """One synthetic WDR image, (H, W, 3) HWC."""
    rng = np.random.default_rng(seed)
    theta, rects, bg = _draw_scene(rng, H, W, n_rects)
    return _render(H, W, decades[0], decades[1], theta, rects, bg, rng, noise, dtype=dtype)


def wdr_mosaic(H: int, W: int, seed: int, tile=(3072, 4096), dtype=np.float32) -> np.ndarray:
    """A large (H, W, 3) image without a full-size float64 render: one
    ``tile``-sized scene (``wdr_image``) repeated over the frame, each copy
    flipped by its grid position and scaled by 10^U(-1, 1) of its own, so the
    copies differ in range and orientation. Memory stays near 2x the output."""
    th, tw = min(tile[0], H), min(tile[1], W)
    base = wdr_image(th, tw, seed=seed, dtype=dtype)
    rng = np.random.default_rng(seed + 1)
    out = np.empty((H, W, 3), dtype)
    for i, y0 in enumerate(range(0, H, th)):
        for j, x0 in enumerate(range(0, W, tw)):
            t = base[:: (-1 if i % 2 else 1), :: (-1 if j % 2 else 1)]
            h, w = min(th, H - y0), min(tw, W - x0)
            np.multiply(t[:h, :w], dtype(10.0 ** rng.uniform(-1.0, 1.0)), out=out[y0:y0 + h, x0:x0 + w])
    return out


def wdr_video_frame(H: int, W: int, seed: int, frame: int, decades=(-2.0, 4.0),
                    n_rects: int = 20, noise: float = 0.02, drift: float = 0.01,
                    dtype=np.float16) -> np.ndarray:
    """Frame ``frame`` of a synthetic WDR video: rectangles move at constant
    seeded velocities over a ramp drifting ``drift`` decades per frame; the
    per-frame noise uses seed ``seed + frame``."""
    rng = np.random.default_rng(seed)
    theta, rects, bg = _draw_scene(rng, H, W, n_rects)
    nrng = np.random.default_rng(seed + 1 + frame)
    return _render(H, W, decades[0], decades[1], theta, rects, bg, nrng, noise,
                   shift=drift * frame, t=float(frame), dtype=dtype)


def uneven_sizes(n: int, seed: int, wmin: int = 640, wmax: int = 4096,
                 hmin: int = 480, hmax: int = 3072):
    """(W, H) pairs: W ~ U{wmin..wmax}, aspect 4:3 or 16:9, H in [hmin, hmax]."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        w = int(rng.integers(wmin, wmax + 1))
        a = (4.0 / 3.0) if rng.uniform() < 0.5 else (16.0 / 9.0)
        h = int(round(w / a))
        if hmin <= h <= hmax:
            out.append((w, h))
    return out


def box_image(H: int, W: int, seed: int, levels=(0.01, 100.0), dtype=np.float32):
    """Grey two-level test image: a random rectangle at ``levels[1]`` on a
    background at ``levels[0]`` (closed-form window counts near its edges)."""
    rng = np.random.default_rng(seed)
    img = np.full((H, W, 3), levels[0], dtype=np.float64)
    y0, x0 = int(rng.integers(0, max(H // 2, 1))), int(rng.integers(0, max(W // 2, 1)))
    y1, x1 = int(rng.integers(y0 + 1, H + 1)), int(rng.integers(x0 + 1, W + 1))
    img[y0:y1, x0:x1] = levels[1]
    return img.astype(dtype), (y0, y1, x0, x1)


def wdr_device(H: int, W: int, seed: int, device, decades=(-2.0, 4.0), n_rects: int = 20,
               noise: float = 0.02, frame=None, drift: float = 0.01, dtype=None):
    """The same recipe rendered with torch on ``device`` (for benchmarks that
    need hundreds of megapixels of input quickly). The scene (ramp direction,
    rectangles, chroma) is drawn from ``seed`` exactly as by ``wdr_image``;
    ``frame`` (optional) moves the rectangles and drifts the ramp as
    ``wdr_video_frame`` does. The per-pixel noise comes from a torch generator
    seeded with ``seed + 1 + frame``, so pixel values differ from the numpy
    renderers'. Returns an (H, W, 3) tensor (float32 unless ``dtype``)."""
    import torch

    rng = np.random.default_rng(seed)
    theta, rects, bg = _draw_scene(rng, H, W, n_rects)
    t = 0.0 if frame is None else float(frame)
    shift = 0.0 if frame is None else drift * frame
    lo, hi = decades
    f64 = torch.float64
    yy = torch.linspace(-0.5, 0.5, H, dtype=f64, device=device)[:, None]
    xx = torch.linspace(-0.5, 0.5, W, dtype=f64, device=device)[None, :]
    ramp = float(np.cos(theta)) * xx + float(np.sin(theta)) * yy
    ramp = (ramp - ramp.min()) / torch.clamp(ramp.max() - ramp.min(), min=1e-12)
    dec = lo + (hi - lo) * ramp + shift
    chroma = torch.empty((H, W, 3), dtype=f64, device=device)
    chroma[...] = torch.as_tensor(bg, dtype=f64, device=device)
    for (y0, x0, rh, rw, amp, c, vy, vx) in rects:
        ys = int(round(y0 + vy * t)) % max(H, 1)
        xs = int(round(x0 + vx * t)) % max(W, 1)
        ye, xe = min(ys + rh, H), min(xs + rw, W)
        dec[ys:ye, xs:xe] += amp
        chroma[ys:ye, xs:xe] = torch.as_tensor(c, dtype=f64, device=device)
    dec.clamp_(lo, hi)
    Y = torch.pow(10.0, dec)
    g = torch.Generator(device=device)
    g.manual_seed(int(seed) + 1 + (0 if frame is None else int(frame)))
    Y *= 1.0 + noise * torch.randn((H, W), generator=g, dtype=f64, device=device)
    Y.clamp_(min=10.0 ** lo * 1e-3)
    rgb = chroma * (Y / chroma.mean(dim=2))[..., None]
    return rgb.to(dtype or torch.float32).contiguous()


# An assumed camera for the exposure front-end (the paper's capture data and
# recovered response are not available): sensor exposure X = radiance x time,
# pixel value z = round(255 (min(X, xsat) / xsat)^(1/gamma)) per channel.
def camera_exposures(radiance, times, gamma: float = 2.2, xsat: float = 1.0):
    """uint8 (H, W, 3) exposures of a linear radiance image, one per time."""
    E = np.asarray(radiance, dtype=np.float64)
    out = []
    for t in times:
        X = np.clip(E * float(t) / xsat, 0.0, 1.0)
        out.append(np.rint(255.0 * np.power(X, 1.0 / gamma)).astype(np.uint8))
    return out


def camera_log_response(gamma: float = 2.2, xsat: float = 1.0) -> np.ndarray:
    """(3, 256) log inverse response of that camera: g(z) = ln(xsat (z/255)^gamma)
    (the value for z = 0 repeats z = 1's; it only enters through zero weight or
    the all-dark fallback)."""
    z = np.arange(256, dtype=np.float64)
    z[0] = 1.0
    g = np.log(xsat) + gamma * np.log(z / 255.0)
    return np.repeat(g[None, :], 3, axis=0)
