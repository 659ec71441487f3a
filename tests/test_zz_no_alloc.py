"""The allocation-free integral image (tm_integral_image_noalloc).

Some callers cannot allocate device memory while they run (a per-frame
deadline that forbids allocator calls after start-up, code inside another
framework's allocator callbacks, a process that reserved all device memory up
front). The entry point they call keeps its scratch in a static device array
of the library instead of calling cudaMalloc. These tests call it through the
C ABI: a small plane against the oracle's Eq. 5 integral image, and planes
whose scratch only fits the array once the row segments are made taller
(4000 x 3000, and 3001 x 4100 with a partial last segment) against
tm_integral_image, each on two calls in a row that share the static
scratch."""
import ctypes

import numpy as np
import pytest

import paper_2102_01289_gb300 as tm


@pytest.fixture(scope="module", autouse=True)
def _built():
    tm.build()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    # 600000 x 1 needs 16 * 600000 bytes of column sums: more than 8 MiB
    L = tm.lib()
    fake = ctypes.c_void_p(0x1000)
    assert L.tm_integral_image_noalloc(fake, 600000, 1, ctypes.c_void_p(0x2000),
                                       ctypes.c_void_p(0x3000), None) == tm.TM_EINVAL
    assert b"8 MiB" in L.tm_last_error(None)
    assert L.tm_integral_image_noalloc(None, 4, 4, fake, fake, None) == tm.TM_EINVAL
    assert b"null" in L.tm_last_error(None)


def _q(rng, H, W):
    return rng.integers(-(2 ** 23), 2 ** 23 + 1, size=(H, W)).astype(np.int32)


@pytest.mark.gpu
def test_noalloc_matches_oracle_twice(orc):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rng = np.random.default_rng(7)
    for H, W in [(257, 300), (2000, 77)]:  # two calls in a row on the shared scratch
        qh = _q(rng, H, W)
        q = torch.from_numpy(qh).cuda()
        b1 = torch.full((H + 1, W + 1), -1, dtype=torch.int64, device="cuda")
        b2 = torch.full_like(b1, -1)
        tm.tm_integral_image_noalloc(q, b1, b2)
        torch.cuda.synchronize()
        assert np.array_equal(b1.cpu().numpy().view(np.uint64), orc.integral_i64(qh))
        assert np.array_equal(b2.cpu().numpy().view(np.uint64), orc.integral_i64(qh.astype(np.int64) ** 2))


@pytest.mark.gpu
def test_noalloc_tall_segments_match_allocating_entry_point_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rng = np.random.default_rng(8)
    for H, W in [(3000, 4000), (4100, 3001)]:
        q = torch.from_numpy(_q(rng, H, W)).cuda()
        a1 = torch.empty((H + 1, W + 1), dtype=torch.int64, device="cuda")
        a2 = torch.empty_like(a1)
        tm.tm_integral_image(q, a1, a2)
        for _ in range(2):
            b1 = torch.full_like(a1, -1)
            b2 = torch.full_like(a1, -1)
            tm.tm_integral_image_noalloc(q, b1, b2)
            torch.cuda.synchronize()
            assert torch.equal(a1, b1) and torch.equal(a2, b2)
