"""GPU parity of the tile-packed EDM (simplex_edm_tiles): every 128 x 128
tile of the squared-distance matrix one contiguous block, tiles in packed
lower order; diagonal tiles whole (upper entries are the mirrored pairs),
diagonal and padding exactly 0.  Against the oracle's own construction of
the layout (FP64): relative error <= 1e-5 per nonzero entry, exact zeros where
the oracle has them.  The lower entries must also equal, bit for bit, what
simplex_edm_packed writes for the same pairs (the same kernel arithmetic,
only the store layout differs)."""
import numpy as np
import pytest
import torch

import synth
from helpers import gather, rel_err, to_gpu

pytestmark = pytest.mark.gpu
TOL = 1e-5
MAPS = ["lambda", "bbox", "linear", "rb"]


def tiles_index(i, j):
    """Layout position of (i, j) (j <= i, or a mirrored pair of a diagonal
    tile), written from the header's formula."""
    i = np.asarray(i, np.int64)
    j = np.asarray(j, np.int64)
    I, J = i // 128, j // 128
    return (I * (I + 1) // 2 + J) * 16384 + (i % 128) * 128 + j % 128


def check_against_oracle(out, ref):
    zero = ref == 0
    assert (out[zero] == 0).all()
    if (~zero).any():
        assert rel_err(out[~zero], ref[~zero]).max() <= TOL


def lower_equals_packed(tiles, packed, n):
    """The lower triangle gathered from the tiles equals the packed rows."""
    i, j = np.tril_indices(n)
    assert torch.equal(tiles[torch.from_numpy(tiles_index(i, j)).to(tiles.device)], packed)


@pytest.mark.parametrize("mp", MAPS)
@pytest.mark.parametrize("n,d", [(1, 3), (2, 1), (127, 3), (129, 5), (300, 33), (1000, 5)])
def test_tiles_fp32_small(gpu, oracle, mp, n, d):
    x = synth.normal(n, d, seed=1100 + n + d)
    xt = to_gpu(x)
    out = gpu.edm_tiles(xt, mp, "fp32")
    assert out.numel() == gpu.simplex_edm_tiles_len(n) == oracle.edm_tiles(x).size
    check_against_oracle(out.cpu().numpy(), oracle.edm_tiles(x))
    lower_equals_packed(out, gpu.edm_packed(xt, mp, "fp32"), n)


@pytest.mark.parametrize("mp", MAPS)
@pytest.mark.parametrize("n,d", [(1, 64), (128, 64), (129, 64), (300, 256), (1000, 64), (700, 192),
                                 (2000, 64)])
def test_tiles_bf16x3_small(gpu, oracle, mp, n, d):
    """Both tensor-core kernels (d < 128: steps of two tiles, one CTA per SM;
    d >= 128: two-CTA clusters), stores by TMA tensor boxes."""
    x = synth.normal(n, d, seed=1200 + n + d)
    xt = to_gpu(x)
    out = gpu.edm_tiles(xt, mp, "bf16x3")
    gpu.simplex_device_errors()
    check_against_oracle(out.cpu().numpy(), oracle.edm_tiles(x))
    lower_equals_packed(out, gpu.edm_packed(xt, mp, "bf16x3"), n)
    gpu.simplex_device_errors()


def test_tiles_overwrite_every_float(gpu, oracle):
    """Every float of the output is written: a buffer pre-filled with NaN
    comes back equal to the oracle's layout (padding included), on both
    paths and a ragged n."""
    for prec, d in (("fp32", 3), ("bf16x3", 64), ("bf16x3", 128)):
        x = synth.normal(333, d, seed=77)
        out = torch.full((gpu.simplex_edm_tiles_len(333),), float("nan"), device="cuda")
        gpu.simplex_edm_tiles(to_gpu(x), out, "lambda", prec, gpu.workspace("edm", 333, d, "lambda", prec))
        gpu.simplex_device_errors()
        check_against_oracle(out.cpu().numpy(), oracle.edm_tiles(x))


def test_tiles_near_duplicates(gpu, oracle):
    base = synth.normal(150, 64, seed=31)
    x = np.concatenate([base, base + 1e-3 * synth.normal(150, 64, seed=32)]).astype(np.float32)
    out = gpu.edm_tiles(to_gpu(x), "lambda", "bf16x3")
    gpu.simplex_device_errors()
    check_against_oracle(out.cpu().numpy(), oracle.edm_tiles(x))


def test_tiles_scale_config(gpu, oracle):
    """n = 65536, d = 64 (N(0,1), seed 4): 131,328 tiles, 8.6 GB.  Seeded
    pairs over the triangle, two whole diagonal tiles (both triangles) and
    one off-diagonal tile against the oracle; the lower entries of a sample
    equal the packed-row layout's."""
    w = synth.WORKLOADS["stress_n65536_d64"]
    x = synth.normal(w["n"], w["d"], w["seed"])
    xt = to_gpu(x)
    n = w["n"]
    out = gpu.edm_tiles(xt, "lambda", "bf16x3")
    gpu.simplex_device_errors()
    assert out.numel() == 512 * 513 // 2 * 16384
    pr = synth.sample_pairs(200000, n, seed=23)
    sq = []
    for t0 in (0, n - 128):
        a, b = np.meshgrid(np.arange(128), np.arange(128), indexing="ij")
        sq.append(np.stack([a.ravel() + t0, b.ravel() + t0], axis=1))   # whole square
    a, b = np.meshgrid(np.arange(128), np.arange(128), indexing="ij")
    sq.append(np.stack([a.ravel() + 40960, b.ravel() + 1280], axis=1))  # tile (320, 10)
    pr_all = np.concatenate([pr] + sq)
    got = gather(out, tiles_index(pr_all[:, 0], pr_all[:, 1]))
    ref = oracle.edm_pairs(x, pr_all)
    diag = pr_all[:, 0] == pr_all[:, 1]
    assert (got[diag] == 0).all()
    assert rel_err(got[~diag], ref[~diag]).max() <= TOL
    packed = gpu.edm_packed(xt, "lambda", "bf16x3")
    assert np.array_equal(got[:len(pr)], gather(packed, pr[:, 0] * (pr[:, 0] + 1) // 2 + pr[:, 1]))
    del out, packed
    torch.cuda.empty_cache()
