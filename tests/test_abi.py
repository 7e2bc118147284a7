"""The C-ABI library loads, exports every symbol its header declares, and
validates arguments on the host (no GPU needed, no compute calls)."""

import ctypes
import os
import re

import pytest

from paper_2408_06513_gb300 import build as dc_build
from paper_2408_06513_gb300 import declutter as dc

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "declutter.h")


@pytest.fixture(scope="module")
def lib():
    dc_build.build()
    return dc.load_library()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\**\s*(\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("declutter_create", "splat_density", "integral_images", "displacement_field",
                     "advect_samples", "regularize"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert names
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(dc.exported_symbols()) == names


def test_status_strings(lib):
    assert dc.declutter_status_string(0) == "ok"
    for s in range(1, 8):
        assert dc.declutter_status_string(s) not in ("ok", "unknown status")
    assert dc.declutter_kernel_name(0) == "splat"
    assert dc.declutter_kernel_name(99) is None


def _params(**kw):
    p = dc.dc_params()
    p.log2_res = kw.get("log2_res", 9)
    p.kernel_r = kw.get("kernel_r", -1)
    p.sigma = kw.get("sigma", 0.0)
    p.d0 = kw.get("d0", -1.0)
    p.pixel_center = kw.get("pixel_center", 0)
    p.clamp_positions = kw.get("clamp_positions", 1)
    p.carry_mode = kw.get("carry_mode", 0)
    p.band_rows = kw.get("band_rows", 0)
    p.keep_order = kw.get("keep_order", 0)
    return p


@pytest.mark.parametrize("kw,status", [
    (dict(log2_res=3), 2),
    (dict(log2_res=14), 2),
    (dict(kernel_r=65), 1),
    (dict(log2_res=4, kernel_r=16), 1),
    (dict(pixel_center=2), 1),
    (dict(carry_mode=5), 1),
    (dict(band_rows=-1), 1),
    (dict(band_rows=65), 1),
    (dict(band_rows=128), 1),
    (dict(keep_order=2), 1),
])
def test_create_rejects_bad_parameters(lib, kw, status):
    h = ctypes.c_void_p()
    p = _params(**kw)
    st = lib.declutter_create(ctypes.byref(p), 0, None, ctypes.byref(h))
    assert st == status
    assert not h.value
    assert dc.declutter_last_error()


def test_calls_on_null_context_fail_cleanly(lib):
    assert lib.regularize(None, None, 0, 1, None) == 1
    assert lib.declutter_sync(None) == 1
    assert lib.declutter_destroy(None) == 0


def test_every_kernel_kind_has_algorithmic_bytes(lib):
    # bench.py divides each kernel kind's algorithmic bytes by its time: every
    # kind the library reports needs a formula, and no name is left over
    import bench

    names = [dc.declutter_kernel_name(k) for k in range(dc.KERNEL_KINDS)]
    assert all(names) and dc.declutter_kernel_name(dc.KERNEL_KINDS) is None
    info = type("Info", (), {"band_rows": 2})()
    for name in names:
        assert bench.algorithmic_bytes(name, 1_000_000, 512, info) > 0, name
    assert set(bench.KERNELS_PER_UNIT) <= set(names)


def test_surrogate_flop_count():
    # the network of surrogate_create(8, 4, 32, in_channels=3): 8 encoder, 6
    # decoder and one head convolution, 3x3; per 256^2 sample, counted by hand:
    # 113.2M (3 -> 32) + seven c -> c convolutions of 1208.0M + three of
    # 604.0M (c -> 2c encoder) + three of 2416.0M (2c -> c decoder, upsampled
    # input) + 75.5M (head) = 17,704,157,184 FLOP
    import bench

    layers = bench.surrogate_layer_flops()
    assert len(layers) == 15
    assert sum(layers) == 17_704_157_184
    assert layers[0] == 2 * 65536 * 32 * 27 and layers[-1] == 2 * 65536 * 2 * 288


def test_autotune_cache_file_round_trip(tmp_path):
    # the autotuner's cache file (host only, no device needed): a file
    # written by hand loads, saves back with the same entries, and a
    # malformed file is refused without changing the cache
    from paper_2408_06513_gb300 import declutter as dc
    dc.declutter_autotune_clear()
    good = tmp_path / "tune.txt"
    good.write_text("declutter-autotune 1\nNVIDIA_GB300 152 9 4 0 0 19 1 2 0\nNVIDIA_GB300 152 11 16 0 0 23 0 14 1\n")
    dc.declutter_autotune_load(str(good))
    out = tmp_path / "out.txt"
    dc.declutter_autotune_save(str(out))
    lines = out.read_text().splitlines()
    assert lines[0] == "declutter-autotune 1"
    assert sorted(lines[1:]) == sorted(good.read_text().splitlines()[1:])
    bad = tmp_path / "bad.txt"
    bad.write_text("declutter-autotune 1\nNVIDIA_GB300 152 9 4 0 0 19 1 99 0\n")  # band rows out of range
    with pytest.raises(dc.DeclutterError):
        dc.declutter_autotune_load(str(bad))
    with pytest.raises(dc.DeclutterError):
        dc.declutter_autotune_load(str(tmp_path / "missing.txt"))
    dc.declutter_autotune_save(str(out))
    assert len(out.read_text().splitlines()) == 3
    dc.declutter_autotune_clear()
    dc.declutter_autotune_save(str(out))
    assert out.read_text().splitlines() == ["declutter-autotune 1"]
