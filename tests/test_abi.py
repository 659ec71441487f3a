"""C-ABI library checks that need no GPU: it builds for sm_103a, loads, exports
every symbol include/tm.h declares, and rejects invalid arguments on the host
before any launch."""
import ctypes
import json
import os
import re

import numpy as np
import pytest

import paper_2102_01289_gb300 as tm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built():
    tm.build()
    return tm.lib()


def _declared():
    src = open(os.path.join(ROOT, "include", "tm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tm_[a-z_0-9]+)\s*\(", src)))


def test_header_declarations_match_binding():
    assert _declared() == sorted(tm.EXPORTS)


def test_library_exports_every_declared_symbol(built):
    out = os.popen(f"nm -D --defined-only {tm.LIB_PATH}").read()
    names = set(re.findall(r"\b(tm_[a-z_0-9]+)\b", out))
    missing = [n for n in _declared() if n not in names]
    assert not missing, missing
    for n in _declared():
        assert getattr(built, n) is not None


def test_library_targets_sm_103a(built):
    out = os.popen(f"cuobjdump --list-elf {tm.LIB_PATH} 2>&1").read()
    assert "sm_103a" in out


def test_defaults_are_the_papers(built):
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_constants.json")))
    p = tm.tm_params_default()
    q = g["quality_setting"]["value"]
    assert (p.n_bins, p.n_fields) == (q["n"], q["s"])
    assert np.isclose(p.sat, g["sat"]["value"]) and np.isclose(p.eps[0], g["eps"]["value"])
    ex = g["pyramid_example"]["value"]
    sizes = [2 * p.rx[f] for f in range(p.n_fields)]
    assert sizes[0] == ex["largest"] and sizes[-1] == ex["smallest"]
    assert all(sizes[f] == ex["ratio"] * sizes[f + 1] for f in range(p.n_fields - 1))
    pp = tm.tm_params_pyramid(2048, 2048, 5, 5)
    assert [2 * pp.rx[f] for f in range(5)] == sizes


@pytest.mark.parametrize("field,value", [
    ("n_bins", 0), ("n_bins", 257), ("n_fields", 0), ("n_fields", 9), ("sat", -1.0),
    ("ld_min", 2.0), ("flags", 16), ("flags", -1),
])
def test_create_rejects_bad_params(built, field, value):
    p = tm.make_params(8, [1, 2])
    setattr(p, field, value)
    with pytest.raises(tm.TmError) as e:
        tm.tm_create(p)
    assert e.value.status == tm.TM_EINVAL
    assert tm.tm_last_error(None)


def test_create_rejects_bad_field_values(built):
    for attr, val in (("eps", 0.0), ("eps", float("nan")), ("alpha", -0.5), ("rx", -1), ("ry", 40000)):
        p = tm.make_params(8, [1, 2])
        getattr(p, attr)[1] = val
        with pytest.raises(tm.TmError):
            tm.tm_create(p)


def test_forward_rejects_bad_descriptors_without_launch(built):
    ctx = tm.tm_create(tm.make_params(8, [1]))
    L = tm.lib()
    try:
        good = tm.TmImage(0x1000, 4, 4, 12, tm.TM_F32)
        cases = [
            tm.TmImage(None, 4, 4, 12, tm.TM_F32),       # null data
            tm.TmImage(0x1000, 0, 4, 12, tm.TM_F32),     # empty width
            tm.TmImage(0x1000, 4, 0, 12, tm.TM_F32),     # empty height
            tm.TmImage(0x1000, 4, 4, 11, tm.TM_F32),     # pitch < 3W
            tm.TmImage(0x1000, 4, 4, 12, 7),             # unknown dtype
            tm.TmImage(0x1002, 4, 4, 12, tm.TM_F32),     # misaligned
        ]
        for bad in cases:
            s = L.tm_forward(ctx, ctypes.byref(bad), ctypes.byref(tm.TmImage(0x9000, 4, 4, 12, 0)), None)
            assert s == tm.TM_EINVAL, (bad.width, bad.height, bad.pitch, bad.dtype)
        s = L.tm_forward(ctx, ctypes.byref(tm.TmImage(0x1000, 4, 4, 12, tm.TM_U8)),
                         ctypes.byref(tm.TmImage(0x9000, 4, 4, 12, 0)), None)
        assert s == tm.TM_EUNSUPPORTED
        s = L.tm_forward(ctx, ctypes.byref(good), ctypes.byref(tm.TmImage(0x9000, 5, 4, 15, 0)), None)
        assert s == tm.TM_EINVAL  # size mismatch
        s = L.tm_forward(ctx, ctypes.byref(good), ctypes.byref(tm.TmImage(0x1010, 4, 4, 12, 0)), None)
        assert s == tm.TM_EINVAL and "overlap" in tm.tm_last_error(ctx)
        assert L.tm_forward(None, ctypes.byref(good), ctypes.byref(good), None) == tm.TM_EINVAL
        assert L.tm_forward_batch(ctx, -1, None, None, None) == tm.TM_EINVAL
        assert L.tm_forward_batch(ctx, 0, None, None, None) == tm.TM_OK  # empty batch
        assert L.tm_integral_histogram(None, 4, 4, 8, None, None) == tm.TM_EINVAL
        assert L.tm_integral_image(None, 4, 4, None, None, None) == tm.TM_EINVAL
        assert L.tm_set_option(ctx, tm.TM_OPT_HIST_PATH, 9) == tm.TM_EINVAL
        assert L.tm_set_option(ctx, tm.TM_OPT_SWEEP_WIDTH, 300) == tm.TM_EINVAL
        assert L.tm_set_option(ctx, tm.TM_OPT_SWEEP_WIDTH, 512) == tm.TM_OK
        n = ctypes.c_size_t()
        assert L.tm_debug_size(ctx, tm.TM_DBG_BINS, ctypes.byref(n)) == tm.TM_ESTATE
    finally:
        tm.tm_destroy(ctx)
    tm.tm_destroy(None)


def test_missing_library_fails_loudly(monkeypatch):
    monkeypatch.setattr(tm, "_lib", None)
    monkeypatch.setattr(tm, "LIB_PATH", "/nonexistent/libtm.so")
    with pytest.raises(RuntimeError, match="missing"):
        tm.tm_create(tm.TmParams())


def test_defined_flags_accepted(built):
    for flags in (tm.TM_FLAG_CDF_INCLUSIVE, tm.TM_FLAG_AREA_LITERAL, tm.TM_FLAG_VAR_LINEAR,
                  tm.TM_FLAG_SRGB_U8, 15):
        p = tm.make_params(8, [1, 2])
        p.flags = flags
        tm.tm_destroy(tm.tm_create(p))


def test_merge_exposures_rejects_bad_arguments(built):
    """Host validation of the capture front-end: no launch for a bad count,
    time, size or response table (TM_EINVAL with a message)."""
    import ctypes

    L = built
    fake = (ctypes.c_void_p * 9)(*([0x1000] * 9))
    times = (ctypes.c_float * 9)(*([0.01] * 9))
    g = (ctypes.c_float * 768)(*([0.0] * 768))
    out = tm.TmImage()
    out.data, out.width, out.height, out.pitch, out.dtype = 0x2000, 4, 3, 12, tm.TM_F32
    args = lambda n, t=times, gg=g, w=4: (n, ctypes.cast(fake, ctypes.c_void_p), ctypes.cast(t, ctypes.c_void_p),  # noqa: E731
                                          w, 3, 12, ctypes.cast(gg, ctypes.c_void_p), ctypes.byref(out), None)
    assert L.tm_merge_exposures(*args(0)) == tm.TM_EINVAL
    assert L.tm_merge_exposures(*args(9)) == tm.TM_EINVAL
    bad_t = (ctypes.c_float * 9)(*([0.01] * 8 + [0.0]))
    assert L.tm_merge_exposures(*args(9, bad_t)) == tm.TM_EINVAL
    bad_t4 = (ctypes.c_float * 4)(0.01, -1.0, 0.1, 1.0)
    assert L.tm_merge_exposures(*args(4, bad_t4)) == tm.TM_EINVAL
    assert b"times" in L.tm_last_error(None)
    bad_g = (ctypes.c_float * 768)(*([0.0] * 767 + [float("inf")]))
    assert L.tm_merge_exposures(*args(4, times, bad_g)) == tm.TM_EINVAL
    assert L.tm_merge_exposures(*args(4, times, g, 5)) == tm.TM_EINVAL  # out size differs
