"""GPU parity of the packed EDM (Sec. I: the EDM is a 2-simplex problem)
against the FP64 oracle: relative error <= 1e-5 per entry, diagonal exactly 0.
Full comparison where the oracle runs in seconds; seeded sampled pairs plus
every diagonal-tile pair at the full configuration sizes."""
import numpy as np
import pytest
import torch

import synth
from helpers import gather, packed_index, rel_err, to_gpu

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.mark.parametrize("mp", ["lambda", "bbox", "linear", "rb"])
@pytest.mark.parametrize("n,d", [(1, 3), (2, 1), (31, 3), (33, 7), (100, 3), (257, 33),
                                 (600, 64), (1000, 5)])
def test_edm_small(gpu, oracle, mp, n, d):
    x = synth.normal(n, d, seed=100 + n + d)
    out = gpu.edm_packed(to_gpu(x), mp, "fp32").cpu().numpy()
    ref = oracle.edm_packed(x)
    i = np.arange(n)
    assert (out[packed_index(i, i)] == 0).all()
    off = ref > 0
    if off.any():
        assert rel_err(out[off], ref[off]).max() <= TOL
    assert out.shape == ref.shape


@pytest.mark.parametrize("mp", ["lambda", "bbox", "linear"])
def test_edm_config_n1024_d3(gpu, oracle, mp):
    """2-simplex plain: n = 1024, d = 3, U[0,1)^3 seed 0, all 524,800 entries."""
    x = synth.make_points("edm_n1024_d3")
    out = gpu.edm_packed(to_gpu(x), mp, "fp32").cpu().numpy()
    ref = oracle.edm_packed(x)
    assert out.shape == (524800,)
    diag = packed_index(np.arange(1024), np.arange(1024))
    assert (out[diag] == 0).all()
    off = np.ones(out.size, bool)
    off[diag] = False
    assert rel_err(out[off], ref[off]).max() <= TOL


def sampled_check(out, x, oracle, seed, nb_rho=32, count=200000):
    n = x.shape[0]
    pr = synth.sample_pairs(count, n, seed)
    # every pair of the first and last diagonal tiles too
    for t0 in (0, (n // nb_rho - 1) * nb_rho):
        ii, jj = np.tril_indices(nb_rho)
        pr = np.concatenate([pr, np.stack([ii + t0, jj + t0], axis=1)])
    got = gather(out, packed_index(pr[:, 0], pr[:, 1]))
    ref = oracle.edm_pairs(x, pr)
    diag = pr[:, 0] == pr[:, 1]
    assert (got[diag] == 0).all()
    return rel_err(got[~diag], ref[~diag]).max()


@pytest.mark.parametrize("name,prec", [("edm_n32768_d256", "fp32")])
def test_edm_precision_config_sampled(gpu, oracle, name, prec):
    x = synth.make_points(name)
    out = gpu.edm_packed(to_gpu(x), "lambda", prec)
    assert out.numel() == 32768 * 32769 // 2
    assert sampled_check(out, x, oracle, seed=21) <= TOL


def test_edm_scale_config_sampled(gpu, oracle):
    """n = 65536 (2,147,516,416 entries, 64-bit packed indices), d = 64."""
    w = synth.WORKLOADS["stress_n65536_d64"]
    x = synth.normal(w["n"], w["d"], w["seed"])
    out = gpu.edm_packed(to_gpu(x), "lambda", "fp32")
    assert out.numel() == 2147516416
    assert sampled_check(out, x, oracle, seed=22) <= TOL
    del out
    torch.cuda.empty_cache()


def test_edm_maps_agree_bitwise(gpu):
    """The maps run the same tile body, so their outputs are identical."""
    x = to_gpu(synth.normal(3000, 16, seed=23))
    a = gpu.edm_packed(x, "lambda")
    assert torch.equal(a, gpu.edm_packed(x, "bbox"))
    assert torch.equal(a, gpu.edm_packed(x, "linear"))
    assert torch.equal(a, gpu.edm_packed(x, "rb"))


# ---------------------------------------------------------------- tensor cores

BF_TOL = 1e-5


@pytest.mark.parametrize("mp", ["lambda", "bbox", "linear", "rb"])
@pytest.mark.parametrize("n,d", [(1, 64), (128, 64), (129, 64), (200, 128), (300, 256), (1000, 64),
                                 (700, 192)])
def test_edm_bf16x3_small(gpu, oracle, mp, n, d):
    """Gram term on tensor cores (BF16 hi+lo split, FP32 accumulation),
    every entry against the FP64 oracle."""
    x = synth.normal(n, d, seed=600 + n + d)
    out = gpu.edm_packed(to_gpu(x), mp, "bf16x3")
    gpu.simplex_device_errors()
    out = out.cpu().numpy()
    ref = oracle.edm_packed(x)
    i = np.arange(n)
    assert (out[packed_index(i, i)] == 0).all()
    off = ref > 0
    if off.any():
        assert rel_err(out[off], ref[off]).max() <= BF_TOL


def test_edm_bf16x3_near_duplicates(gpu, oracle):
    """Points that nearly coincide make the Gram form cancel; those entries
    are recomputed in FP32 and still meet the tolerance."""
    base = synth.normal(150, 64, seed=31)
    x = np.concatenate([base, base + 1e-3 * synth.normal(150, 64, seed=32)]).astype(np.float32)
    out = gpu.edm_packed(to_gpu(x), "lambda", "bf16x3")
    gpu.simplex_device_errors()
    out = out.cpu().numpy()
    ref = oracle.edm_packed(x)
    off = ref > 0
    assert rel_err(out[off], ref[off]).max() <= BF_TOL


def test_edm_bf16x3_precision_config(gpu, oracle):
    """n = 32768, d = 256, N(0,1) seed 2 (536,887,296 entries): sampled pairs
    plus two whole diagonal tiles against the FP64 oracle."""
    x = synth.make_points("edm_n32768_d256")
    out = gpu.edm_packed(to_gpu(x), "lambda", "bf16x3")
    gpu.simplex_device_errors()
    assert sampled_check(out, x, oracle, seed=21, nb_rho=128) <= BF_TOL


def test_edm_bf16x3_scale_config(gpu, oracle):
    """n = 65536, d = 64 (2,147,516,416 entries) with the library's choice
    (AUTO selects the tensor-core path for d = 64)."""
    w = synth.WORKLOADS["stress_n65536_d64"]
    x = synth.normal(w["n"], w["d"], w["seed"])
    out = gpu.edm_packed(to_gpu(x), "lambda", "auto")
    gpu.simplex_device_errors()
    assert sampled_check(out, x, oracle, seed=22, nb_rho=128) <= BF_TOL
    del out
    torch.cuda.empty_cache()


@pytest.mark.parametrize("n,d", [(1500, 128), (1501, 64)])
def test_edm_bf16x3_maps_agree(gpu, n, d):
    """Both tensor-core kernels (two-CTA clusters for d >= 128, rows of 256
    columns below) write the same entries under every map."""
    x = to_gpu(synth.normal(n, d, seed=33))
    a = gpu.edm_packed(x, "lambda", "bf16x3")
    assert torch.equal(a, gpu.edm_packed(x, "bbox", "bf16x3"))
    assert torch.equal(a, gpu.edm_packed(x, "linear", "bf16x3"))
    assert torch.equal(a, gpu.edm_packed(x, "rb", "bf16x3"))
    gpu.simplex_device_errors()
