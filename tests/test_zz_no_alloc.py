"""The allocation-free integral image (tm_integral_image_noalloc).

Some callers cannot allocate device memory while they run (a per-frame
deadline that forbids allocator calls after start-up, code inside another
framework's allocator callbacks, a process that reserved all device memory up
front). The entry point they call keeps its scratch in a static device array
of the library instead of calling cudaMalloc. These tests call it through the
C ABI and require the same integers as tm_integral_image, on two calls in a
row that share the static scratch."""
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
    assert L.tm_integral_image_noalloc(None, 4, 4, fake, fake, None) == tm.TM_EINVAL


@pytest.mark.gpu
def test_noalloc_matches_allocating_entry_point_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rng = np.random.default_rng(7)
    for H, W in [(257, 300), (2000, 77)]:  # two calls in a row on the shared scratch
        q = torch.from_numpy(rng.integers(-(2 ** 23), 2 ** 23 + 1, size=(H, W)).astype(np.int32)).cuda()
        a1 = torch.empty((H + 1, W + 1), dtype=torch.int64, device="cuda")
        a2 = torch.empty_like(a1)
        b1 = torch.full_like(a1, -1)
        b2 = torch.full_like(a1, -1)
        tm.tm_integral_image(q, a1, a2)
        tm.tm_integral_image_noalloc(q, b1, b2)
        torch.cuda.synchronize()
        assert torch.equal(a1, b1) and torch.equal(a2, b2)
