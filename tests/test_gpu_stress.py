"""GPU parity of the stress loss over the packed EDM and its gradient
against the FP64 oracle: loss within 1e-5 relative, gradient within 1e-4
relative per row (and against FP64 central differences)."""
import numpy as np
import pytest
import torch

import synth
from helpers import gather, packed_index, rel_err, stress_moments, to_gpu

pytestmark = pytest.mark.gpu
L_TOL = 1e-5
G_TOL = 1e-4


def row_err(g, G):
    return np.linalg.norm(g - G, axis=1) / np.linalg.norm(G, axis=1)


@pytest.mark.parametrize("mp", ["lambda", "bbox", "linear", "rb"])
@pytest.mark.parametrize("n,d", [(2, 1), (33, 3), (100, 8), (257, 64), (700, 33)])
def test_stress_small(gpu, oracle, mp, n, d):
    x = synth.normal(n, d, seed=400 + n)
    y = synth.perturbed(x, 0.1, seed=500 + n)
    xt, yt = to_gpu(x), to_gpu(y)
    loss, D = gpu.stress_fwd(xt, yt, mp, store_d=True)
    ref = oracle.stress_loss(x, y)
    err = abs(loss.item() - ref) / ref
    print(f"stress loss {mp} n={n} d={d}: rel err {err:.2e}")
    assert err <= L_TOL
    ref_D = oracle.edm_packed(x)
    off = ref_D > 0
    assert rel_err(D.cpu().numpy()[off], ref_D[off]).max() <= 1e-5
    g = gpu.stress_bwd(xt, yt, 1.0, mp).double().cpu().numpy()
    G = oracle.stress_grad_rows(x, y, range(n))
    assert row_err(g, G).max() <= G_TOL


def test_autograd_and_fd(gpu, oracle):
    x = synth.normal(150, 6, seed=31)
    y = synth.perturbed(x, 0.2, seed=32)
    xt = to_gpu(x).requires_grad_(True)
    L = gpu.stress_loss(xt, to_gpu(y))
    (2.5 * L).backward()
    g = xt.grad.double().cpu().numpy()
    G = 2.5 * oracle.stress_grad_rows(x, y, range(150))
    assert row_err(g, G).max() <= G_TOL
    xd, yd = x.astype(np.float64), y.astype(np.float64)
    h = 1e-5
    for a in (0, 77):
        for t in range(6):
            xp, xm = xd.copy(), xd.copy()
            xp[a, t] += h
            xm[a, t] -= h
            fd = 2.5 * (oracle.stress_loss(xp, yd) - oracle.stress_loss(xm, yd)) / (2 * h)
            assert g[a, t] == pytest.approx(fd, rel=G_TOL, abs=1e-6 * np.abs(G).max())


def test_zero_at_reference(gpu):
    x = to_gpu(synth.normal(300, 5, seed=33))
    loss, _ = gpu.stress_fwd(x, x)
    assert loss.item() == 0.0
    assert bool((gpu.stress_bwd(x, x) == 0).all())


def test_scale_config_sampled(gpu, oracle):
    """n = 65536, d = 64, N(0,1) seed 4, y = x + 0.1 N(0,1) seed 5: gradient
    rows of 16 sampled atoms and 100k sampled entries of the stored D against
    the oracle; sum of the gradient ~ 0."""
    w = synth.WORKLOADS["stress_n65536_d64"]
    x = synth.normal(w["n"], w["d"], w["seed"])
    y = synth.perturbed(x, w["sigma"], w["y_seed"])
    xt, yt = to_gpu(x), to_gpu(y)
    loss, D = gpu.stress_fwd(xt, yt, "lambda", store_d=True)
    pr = synth.sample_pairs(100000, w["n"], seed=41)
    got = gather(D, packed_index(pr[:, 0], pr[:, 1]))
    ref = oracle.edm_pairs(x, pr)
    m = pr[:, 0] != pr[:, 1]
    assert rel_err(got[m], ref[m]).max() <= 1e-5
    del D
    torch.cuda.empty_cache()
    g = gpu.stress_bwd(xt, yt)
    rows = synth.sample_indices(16, w["n"], seed=42)
    G = oracle.stress_grad_rows(x, y, rows)
    assert row_err(g[torch.from_numpy(rows).cuda()].double().cpu().numpy(), G).max() <= G_TOL
    gs = g.double().sum(0).abs().max().item()
    assert gs <= 1e-4 * g.double().abs().sum(0).max().item()
    L_ref, G_all = stress_moments(x, y)
    assert abs(loss.item() - L_ref) <= L_TOL * L_ref
    assert row_err(g.double().cpu().numpy(), G_all).max() <= G_TOL


# ---------------------------------------------------------------- tensor cores
#
# prec="bf16x3": every pair product on the tensor cores from BF16 hi + lo
# splits (|v - hi - lo| <= 2^-16 |v|, products hi.hi + hi.lo + lo.hi, FP32
# accumulation).  Per residual that is a relative error of a few 2^-16 of
# sum_t |S_it Delta_jt| + |Delta_it S_jt| in the worst case and ~1e-6 of r
# typically; the loss, a sum of 2e9 squares with independent errors, and the
# gradient rows keep the FP32 path's tolerances.
TC_L_TOL = 1e-5
TC_G_TOL = 1e-4


@pytest.mark.parametrize("mp", ["lambda", "bbox", "linear", "rb"])
@pytest.mark.parametrize("n,d", [(1, 32), (2, 64), (129, 32), (300, 64), (513, 96), (1000, 64)])
def test_stress_tensor_small(gpu, oracle, mp, n, d):
    x = synth.normal(n, d, seed=600 + n)
    y = synth.perturbed(x, 0.1, seed=700 + n)
    xt, yt = to_gpu(x), to_gpu(y)
    loss, D = gpu.stress_fwd(xt, yt, mp, "bf16x3", store_d=True)
    ref = oracle.stress_loss(x, y)
    assert abs(loss.item() - ref) <= TC_L_TOL * ref
    ref_D = oracle.edm_packed(x)
    off = ref_D > 0
    if off.any():
        assert rel_err(D.cpu().numpy()[off], ref_D[off]).max() <= 1e-5
    g = gpu.stress_bwd(xt, yt, 1.0, mp, "bf16x3").double().cpu().numpy()
    G = oracle.stress_grad_rows(x, y, range(n))
    if n == 1:
        assert (g == 0).all()
    else:
        assert row_err(g, G).max() <= TC_G_TOL


def test_stress_tensor_maps_agree(gpu):
    """The maps visit the same tiles: identical loss, gradient equal up
    to the order of the FP32 atomic flushes."""
    x = synth.normal(1100, 64, seed=81)
    y = synth.perturbed(x, 0.1, seed=82)
    xt, yt = to_gpu(x), to_gpu(y)
    L = [gpu.stress_fwd(xt, yt, mp, "bf16x3")[0].item() for mp in ("lambda", "bbox", "linear", "rb")]
    for v in L[1:]:
        assert v == pytest.approx(L[0], rel=1e-12)
    g = [gpu.stress_bwd(xt, yt, 1.0, mp, "bf16x3").double() for mp in ("lambda", "bbox", "linear", "rb")]
    for h in g[1:]:
        assert (h - g[0]).abs().max().item() <= 1e-5 * g[0].abs().max().item()


def test_stress_tensor_zero_autograd_fd(gpu, oracle):
    x = synth.normal(260, 32, seed=83)
    xt = to_gpu(x)
    loss, _ = gpu.stress_fwd(xt, xt, "lambda", "bf16x3")
    assert loss.item() == 0.0
    assert bool((gpu.stress_bwd(xt, xt, 1.0, "lambda", "bf16x3") == 0).all())
    y = synth.perturbed(x, 0.2, seed=84)
    xg = to_gpu(x).requires_grad_(True)
    (1.5 * gpu.stress_loss(xg, to_gpu(y), "lambda", "bf16x3")).backward()
    g = xg.grad.double().cpu().numpy()
    G = 1.5 * oracle.stress_grad_rows(x, y, range(260))
    assert row_err(g, G).max() <= TC_G_TOL
    xd, yd = x.astype(np.float64), y.astype(np.float64)
    h = 1e-5
    for a, t in ((0, 0), (131, 17), (259, 31)):
        xp, xm = xd.copy(), xd.copy()
        xp[a, t] += h
        xm[a, t] -= h
        fd = 1.5 * (oracle.stress_loss(xp, yd) - oracle.stress_loss(xm, yd)) / (2 * h)
        assert g[a, t] == pytest.approx(fd, rel=TC_G_TOL, abs=1e-6 * np.abs(G).max())


def test_stress_tensor_scale_config(gpu, oracle):
    """n = 65536, d = 64 (the benchmark configuration and launch): the loss
    and every gradient row against the FP64 moment identity, 16 rows against
    the oracle's pairwise sums, 100k entries of the stored D."""
    w = synth.WORKLOADS["stress_n65536_d64"]
    x = synth.normal(w["n"], w["d"], w["seed"])
    y = synth.perturbed(x, w["sigma"], w["y_seed"])
    xt, yt = to_gpu(x), to_gpu(y)
    loss, D = gpu.stress_fwd(xt, yt, "lambda", "bf16x3", store_d=True)
    pr = synth.sample_pairs(100000, w["n"], seed=43)
    got = gather(D, packed_index(pr[:, 0], pr[:, 1]))
    ref = oracle.edm_pairs(x, pr)
    m = pr[:, 0] != pr[:, 1]
    assert rel_err(got[m], ref[m]).max() <= 1e-5
    del D
    torch.cuda.empty_cache()
    L_ref, G_all = stress_moments(x, y)
    assert abs(loss.item() - L_ref) <= TC_L_TOL * L_ref
    g = gpu.stress_bwd(xt, yt, 1.0, "lambda", "bf16x3").double().cpu().numpy()
    assert row_err(g, G_all).max() <= TC_G_TOL
    rows = synth.sample_indices(16, w["n"], seed=44)
    assert row_err(g[rows], oracle.stress_grad_rows(x, y, rows)).max() <= TC_G_TOL
    # loss and gradient in one pass, at the same size
    lf, gf = gpu.stress_fwd_bwd(xt, yt, 1.0, "lambda", "bf16x3")
    assert abs(lf.item() - L_ref) <= TC_L_TOL * L_ref
    assert row_err(gf.double().cpu().numpy(), G_all).max() <= TC_G_TOL


@pytest.mark.parametrize("mp", ["lambda", "bbox"])
def test_stress_tensor_bwd_padded_grid(gpu, oracle, mp):
    """n = 49153, d = 64: nb = 385 tile rows, so the lambda map pads its grid
    to 512 (idle grid blocks among the tiles) and the walk's prologue scans
    128 blocks of 1024 grid blocks; the tiles are cut into equal chunks
    across that sequence.  Every gradient row against the FP64 moment
    identity, 8 rows against the oracle's pairwise sums."""
    n, d = 49153, 64
    x = synth.normal(n, d, seed=61)
    y = synth.perturbed(x, 0.1, seed=62)
    g = gpu.stress_bwd(to_gpu(x), to_gpu(y), 1.0, mp, "bf16x3").double().cpu().numpy()
    gpu.simplex_device_errors()
    _, G_all = stress_moments(x, y)
    assert row_err(g, G_all).max() <= TC_G_TOL
    rows = synth.sample_indices(8, n, seed=63)
    assert row_err(g[rows], oracle.stress_grad_rows(x, y, rows)).max() <= TC_G_TOL
    torch.cuda.empty_cache()


@pytest.mark.parametrize("mp", ["lambda", "bbox", "linear", "rb"])
@pytest.mark.parametrize("prec,n,d", [("fp32", 1, 4), ("fp32", 2, 1), ("fp32", 100, 8), ("fp32", 257, 64),
                                      ("bf16x3", 1, 32), ("bf16x3", 300, 64), ("bf16x3", 513, 96)])
def test_stress_fwd_bwd_one_pass(gpu, oracle, mp, prec, n, d):
    """simplex_stress_fwd_bwd: the oracle's loss (unscaled) and gradient
    (times gscale) within each precision's tolerances, and the gradient of
    simplex_stress_bwd up to the order of the FP32 atomic flushes."""
    x = synth.normal(n, d, seed=900 + n)
    y = synth.perturbed(x, 0.1, seed=901 + n)
    xt, yt = to_gpu(x), to_gpu(y)
    loss, g = gpu.stress_fwd_bwd(xt, yt, 2.5, mp, prec)
    ref = oracle.stress_loss(x, y)
    if n == 1:
        assert loss.item() == 0.0 and bool((g == 0).all())
        return
    err = abs(loss.item() - ref) / ref
    print(f"stress fwd_bwd loss {mp} {prec} n={n} d={d}: rel err {err:.2e}")
    assert err <= (TC_L_TOL if prec == "bf16x3" else L_TOL)
    G = 2.5 * oracle.stress_grad_rows(x, y, range(n))
    gd = g.double().cpu().numpy()
    assert row_err(gd, G).max() <= (TC_G_TOL if prec == "bf16x3" else G_TOL)
    gs = gpu.stress_bwd(xt, yt, 2.5, mp, prec).double()
    assert (g.double() - gs).abs().max().item() <= 1e-5 * gs.abs().max().item()
