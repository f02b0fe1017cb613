"""Volumetric k x k x k median (hierarchical tiling in 3D, Sec. 7.2) on the
GPU against the CPU oracle, bit for bit."""
import numpy as np
import pytest

import oracle
from paper_2507_19926_gb300 import synth
from gpu_util import ensure_lib, same_bits, to_dev, to_host, f32_specials

pytestmark = pytest.mark.gpu

DTYPES = ["u8", "u16", "u32", "f32"]


def gpu_filter_3d(x, k, variant="auto"):
    import torch
    import paper_2507_19926_gb300 as mf
    ensure_lib()
    xd = to_dev(x)
    y = mf.median_filter_3d(xd, k, variant=variant)
    torch.cuda.synchronize()
    return to_host(y, None)


@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("k", [3, 5, 7, 9, 11, 13, 15, 17, 19])
def test_volume_parity_ragged(dt, k):
    # 13 x 19 x 23 spans several root tiles on every axis with ragged tails
    shape = (2, 13, 19, 23) if k <= 11 else (1, 9, 14, 17)
    for j, gen in enumerate((synth.uniform, synth.levels16)):
        x = gen(shape, dt, 5000 + 10 * k + j)
        assert same_bits(gpu_filter_3d(x, k), oracle.median_filter_3d(x, k)), (dt, k, gen.__name__)


@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 1, 40), (1, 30, 1), (25, 1, 1), (2, 3, 4), (1, 17, 33)])
def test_volume_thin_shapes(shape):
    for k in (3, 5, 9):
        x = synth.uniform(shape, "u8", 17 + k)
        assert same_bits(gpu_filter_3d(x, k), oracle.median_filter_3d(x, k)), (shape, k)


def test_volume_f32_special_values():
    x = f32_specials((6, 20, 30), 77).reshape(6, 20, 30)
    for k in (3, 7):
        assert same_bits(gpu_filter_3d(x, k), oracle.median_filter_3d(x, k))


def test_volume_k1_and_padded_pitch():
    import torch
    import paper_2507_19926_gb300 as mf
    ensure_lib()
    x = synth.uniform((5, 11, 30), "u16", 9)
    assert same_bits(gpu_filter_3d(x, 1), x)
    big = to_dev(np.pad(x, ((0, 0), (0, 0), (0, 10))))  # row pitch 40 elements
    out = torch.zeros_like(big)
    mf.mf_median_filter_3d(big.data_ptr(), out.data_ptr(), 5, 11, 30, 80, 1, mf.MF_U16, 5,
                           torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    got = to_host(out, np.uint16)
    assert np.array_equal(got[:, :, :30], oracle.median_filter_3d(x, 5))
    assert (got[:, :, 30:] == 0).all()


def test_volume_256_cube_sampled_slices():
    """A 256^3 u8 volume, k = 7: slices near both faces and random ones
    against the oracle evaluated on the same slices' windows."""
    x = synth.uniform((256, 256, 256), "u8", 6000)
    got = gpu_filter_3d(x, 7)
    for z in (0, 1, 2, 3, 127, 252, 253, 254, 255):
        lo, hi = max(0, z - 3), min(256, z + 4)
        want = oracle.median_filter_3d(x[lo:hi], 7)[z - lo]
        assert np.array_equal(got[z], want), z


@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("variant", ["oblivious", "data_aware"])
@pytest.mark.parametrize("k", [3, 5])
def test_volume_both_variants(k, dt, variant):
    """k = 3, 5: the register network (data-oblivious) and the shared-memory
    plan (data-aware) on volumes with ragged tails on every axis."""
    for j, gen in enumerate((synth.uniform, synth.levels16)):
        x = gen((3, 11, 37, 70), dt, 7000 + 10 * k + j)
        assert same_bits(gpu_filter_3d(x, k, variant), oracle.median_filter_3d(x, k)), (dt, variant, j)
    xs = f32_specials((7, 9, 40), 71) if dt == "f32" else synth.uniform((1, 1, 5), dt, 72)
    assert same_bits(gpu_filter_3d(xs, k, variant), oracle.median_filter_3d(xs, k))


def test_volume_oblivious_unbuilt_k_is_refused():
    import paper_2507_19926_gb300 as mf
    with pytest.raises(mf.MedianFilterError) as e:
        gpu_filter_3d(synth.uniform((4, 5, 6), "u8", 1), 7, "oblivious")
    assert e.value.status == mf.MF_ERR_UNSUPPORTED
