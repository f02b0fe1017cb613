"""Host-side checks of the C ABI (no GPU): the library builds, loads and
exports every function include/*.h declares, and argument errors
come back as status codes before anything touches a device."""
import ctypes
import os
import re

import pytest

import paper_2507_19926_gb300 as mf
from paper_2507_19926_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()  # incremental: recompiles only what changed
    return mf.load_library()


def declared_functions():
    inc = os.path.join(ROOT, "include")
    src = "".join(open(os.path.join(inc, n)).read() for n in sorted(os.listdir(inc)) if n.endswith(".h"))
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mf_[a-z0-9_]+)\s*\(", src)))


def test_header_declarations_exported(lib):
    names = declared_functions()
    assert "mf_median_filter" in names and len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(mf.EXPORTS)


def test_status_strings(lib):
    assert mf.mf_version().startswith("medianfilter")
    for code in range(0, -10, -1):
        assert lib.mf_status_string(code)


@pytest.mark.parametrize("k", [0, 2, 4, 77, -3])
def test_rejects_bad_k(lib, k):
    rc = lib.mf_median_filter(ctypes.c_void_p(0x10000), ctypes.c_void_p(0x90000), 8, 8, 8, 1, 0, k, 0, None)
    assert rc == -1
    assert b"k must be odd" in lib.mf_last_error()


def test_rejects_bad_pitch_alias_dtype_shape(lib):
    a, b = ctypes.c_void_p(0x100000), ctypes.c_void_p(0x900000)
    assert lib.mf_median_filter(a, b, 8, 8, 7, 1, 0, 3, 0, None) == -3
    assert lib.mf_median_filter(a, b, 8, 8, 18, 1, 2, 3, 0, None) == -3   # u32 pitch not multiple of 4
    assert lib.mf_median_filter(a, a, 8, 8, 8, 1, 0, 3, 0, None) == -4    # alias
    assert lib.mf_median_filter(a, b, 8, 8, 8, 1, 7, 3, 0, None) == -2    # dtype
    assert lib.mf_median_filter(a, b, 0, 8, 8, 1, 0, 3, 0, None) == -1    # H
    assert lib.mf_median_filter(a, b, 8, 8, 8, 0, 0, 3, 0, None) == -1    # channels
    assert lib.mf_median_filter(a, b, 8, 8, 8, 1, 0, 3, 1, None) == -1    # border
    assert lib.mf_median_filter(None, b, 8, 8, 8, 1, 0, 3, 0, None) == -1  # null
    assert lib.mf_median_filter_bwd(a, b, a, 8, 8, 32, 32, 1, 3, 0, None) == -4  # grad_in aliases
    assert lib.mf_median_filter_bwd(a, b, ctypes.c_void_p(0x5000000), 8, 8, 32, 32, 1, 3, 9, None) == -1
    # a plane whose linear indices do not fit int32
    far = ctypes.c_void_p(1 << 45)
    assert lib.mf_median_filter_bwd(a, b, far, 65536, 65536, 1 << 18, 1 << 18, 1, 3, 1, None) == -1
    # config entry: k = 1 and configurations past the last one are refused before any launch
    assert lib.mf_median_filter_config(a, b, 8, 8, 8, 1, 0, 1, 0, None) == -9
    assert lib.mf_median_filter_config(a, b, 8, 8, 8, 1, 0, 3, 99, None) == -9
    assert lib.mf_median_filter_config(a, b, 8, 8, 8, 1, 0, 3, -1, None) == -9


def test_describe_dispatch(lib):
    d = mf.mf_describe(480, 640, 1, mf.MF_U8, 5)
    assert "oblivious" in d and "k=5" in d
    assert mf.mf_describe(10, 10, 1, mf.MF_F32, 1) == "identity copy"


def test_size_aware_default_for_lone_small_images(lib):
    """Untuned, a lone 8/16-bit image at k = 3, 5 runs the configuration
    without a wide run below 2^20 pixels, the 2-tile run up to 2^22 pixels
    and the 4-tile run above (host dispatch only; no GPU)."""
    import os
    if os.environ.get("MF_TUNE_CACHE"):
        pytest.skip("a tuning cache decides the configuration")
    for k in (3, 5):
        for dt in (mf.MF_U8, mf.MF_U16):
            runs = [mf.mf_describe(H, W, 1, dt, k, mf.MF_AUTO).split("run=")[1].split()[0]
                    for H, W in ((480, 640), (1080, 1920), (4096, 4096))]
            assert runs == ["1", "2", "4"], (k, dt, runs)
    # 32-bit keys keep their default at every size
    small = mf.mf_describe(480, 640, 1, mf.MF_F32, 5, mf.MF_AUTO)
    big = mf.mf_describe(4096, 4096, 1, mf.MF_F32, 5, mf.MF_AUTO)
    assert small.split("kernel=")[1] == big.split("kernel=")[1]


def test_batch_rejects_bad_descriptors(lib):
    d = mf.ImageDesc(0x1000, 0x900000, 8, 8, 8, 1, mf.MF_U8, 33)  # k > 31
    with pytest.raises(mf.MedianFilterError):
        mf.mf_batch_plan_create([d])
    d = mf.ImageDesc(0x1000, 0x1000, 8, 8, 8, 1, mf.MF_U8, 3)  # aliasing
    with pytest.raises(mf.MedianFilterError):
        mf.mf_batch_plan_create([d])
    d = mf.ImageDesc(0x1000, 0x900000, 8, 8, 4, 1, mf.MF_U8, 3)  # pitch < W
    with pytest.raises(mf.MedianFilterError):
        mf.mf_batch_plan_create([d])


def test_volume_rejects_bad_arguments(lib):
    a, b = ctypes.c_void_p(0x100000), ctypes.c_void_p(0x900000)
    f = lib.mf_median_filter_3d
    assert f(a, b, 4, 8, 8, 8, 1, 0, 4, None) == -1      # even k
    assert f(a, b, 4, 8, 8, 8, 1, 0, 21, None) == -1     # k beyond 19
    assert f(a, b, 0, 8, 8, 8, 1, 0, 3, None) == -1      # D
    assert f(a, b, 4, 8, 8, 8, 0, 0, 3, None) == -1      # volumes
    assert f(a, b, 4, 8, 8, 7, 1, 0, 3, None) == -3      # pitch < W
    assert f(a, b, 4, 8, 8, 18, 1, 2, 3, None) == -3     # u32 pitch not a multiple of 4
    assert f(a, a, 4, 8, 8, 8, 1, 0, 3, None) == -4      # alias
    assert f(a, b, 4, 8, 8, 8, 1, 9, 3, None) == -2      # dtype
    assert f(None, b, 4, 8, 8, 8, 1, 0, 3, None) == -1   # null
    g = lib.mf_median_filter_3d_ex
    assert g(a, b, 4, 8, 8, 8, 1, 0, 3, 7, None) == -1   # variant
    assert g(a, b, 4, 8, 8, 8, 1, 0, 7, 1, None) == -9   # no network built for k = 7
    assert "volumetric" in mf.mf_median_filter_3d_describe(7, mf.MF_U8)
    assert "oblivious" in mf.mf_median_filter_3d_describe(3, mf.MF_U8)


def test_volume_describe_carries_the_work_counts(lib):
    """bench.py reads the per-voxel work of a volume plan from these lines
    (roofline fractions): the network form gives its min/max per voxel, the
    data-aware form its merged and sorted elements per voxel."""
    import re
    net = mf.mf_median_filter_3d_describe(5, mf.MF_U8)
    assert re.search(r"min/max per voxel=([\d.]+)", net) and "oblivious" in net
    plan = mf.mf_median_filter_3d_describe(9, mf.MF_F32)
    m = re.search(r"merged/vox=([\d.]+) sorted/vox=([\d.]+)", plan)
    assert m and float(m.group(1)) > 0 and "data-aware" in plan
