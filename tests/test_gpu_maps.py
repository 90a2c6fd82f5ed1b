"""GPU parity of the block-space maps: decode tables bit-exact against the
oracle's recursive construction, coverage counts and idle threads equal to
the oracle's thread-level enumeration (Sec. III-A, III-C, III-D)."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mp", ["lambda", "bbox", "linear", "rb"])
@pytest.mark.parametrize("nb", [1, 2, 3, 5, 8, 13, 64, 100, 1024, 4096])
def test_map2_table_device(gpu, oracle, mp, nb):
    if mp != "lambda" and nb > 1024:
        pytest.skip("large box/linear tables add nothing")
    t = gpu.map_blocks(2, nb, mp).cpu().numpy()
    assert np.array_equal(t, oracle.table2(nb, mp))


@pytest.mark.parametrize("mp", ["lambda", "bbox", "linear"])
@pytest.mark.parametrize("nb", [1, 2, 3, 4, 7, 16, 33, 64, 256])
def test_map3_table_device(gpu, oracle, mp, nb):
    if mp != "lambda" and nb > 64:
        pytest.skip("large box/linear tables add nothing")
    t = gpu.map_blocks(3, nb, mp).cpu().numpy()
    assert np.array_equal(t, oracle.table3(nb, mp))


@pytest.mark.parametrize("mp", ["lambda", "bbox", "linear", "rb"])
@pytest.mark.parametrize("n,rho", [(1, 16), (2, 1), (5, 2), (16, 4), (33, 8), (100, 16),
                                   (257, 16), (300, 32), (1000, 7)])
def test_cover2_device(gpu, oracle, mp, n, rho):
    count, idle = gpu.map2(n, rho, mp)
    ref_count, ref_idle = oracle.cover2(n, rho, mp)
    assert np.array_equal(count.cpu().numpy(), ref_count)
    assert int(idle.item()) == ref_idle


@pytest.mark.parametrize("mp", ["lambda", "bbox", "linear"])
@pytest.mark.parametrize("n,rho", [(1, 8), (3, 2), (17, 4), (40, 8), (64, 8), (100, 5), (130, 10)])
def test_cover3_device(gpu, oracle, mp, n, rho):
    count, idle = gpu.map3(n, rho, mp)
    ref_count, ref_idle = oracle.cover3(n, rho, mp)
    assert np.array_equal(count.cpu().numpy(), ref_count)
    assert int(idle.item()) == ref_idle


def test_cover2_full_size_rb(gpu, oracle):
    """The rectangular box (2-simplex only) at n = 1024: every pair once."""
    c2, i2 = gpu.map2(1024, 16, "rb")
    assert c2.numel() == 524800 and bool((c2 == 1).all())
    assert int(i2.item()) == oracle.cover2(1024, 16, "rb")[1]


def test_rb_has_no_3_simplex_form(gpu):
    with pytest.raises(gpu.SimplexError):
        gpu.map3(40, 4, "rb")


@pytest.mark.parametrize("mp", ["lambda", "bbox", "linear"])
def test_cover_full_size(gpu, oracle, mp):
    """n = 1024 points: every one of the n(n+1)/2 = 524,800 pairs and of the
    n(n+1)(n+2)/6 = 179,481,600 triples is reached exactly once."""
    n = 1024
    c2, i2 = gpu.map2(n, 16, mp)
    assert c2.numel() == 524800 and bool((c2 == 1).all())
    assert int(i2.item()) == oracle.cover2(n, 16, mp)[1]
    c3, i3 = gpu.map3(n, 8, mp)
    assert c3.numel() == 179481600
    assert int(c3.min()) == 1 and int(c3.max()) == 1
    del c3
    torch.cuda.empty_cache()
    _, ref_idle = oracle.cover3(n, 8, mp)
    assert int(i3.item()) == ref_idle


@pytest.mark.parametrize("mp", ["lambda", "bbox"])
@pytest.mark.parametrize("nb", [1, 2, 3, 8, 13, 32, 64])
def test_map4_table_device(gpu, oracle, mp, nb):
    if mp != "lambda" and nb > 32:
        pytest.skip("large box tables add nothing")
    t = gpu.map_blocks(4, nb, mp).cpu().numpy()
    assert np.array_equal(t, oracle.table4(nb, mp))


@pytest.mark.parametrize("mp", ["lambda", "bbox"])
@pytest.mark.parametrize("n,rho", [(1, 4), (2, 1), (5, 2), (17, 4), (33, 4), (40, 5), (64, 3)])
def test_cover4_device(gpu, oracle, mp, n, rho):
    count, idle = gpu.map4(n, rho, mp)
    ref_count, ref_idle = oracle.cover4(n, rho, mp)
    assert np.array_equal(count.cpu().numpy(), ref_count)
    assert int(idle.item()) == ref_idle


@pytest.mark.parametrize("mp", ["lambda", "bbox"])
def test_cover4_n128(gpu, oracle, mp):
    """n = 128 points, 4^4 threads per block: every one of the C(131, 4) =
    11,716,640 quadruples is reached exactly once."""
    count, idle = gpu.map4(128, 4, mp)
    assert count.numel() == 11716640
    assert int(count.min()) == 1 and int(count.max()) == 1
    assert int(idle.item()) == oracle.cover4(128, 4, mp)[1]
