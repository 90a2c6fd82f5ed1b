"""The no-allocation ATM energy entry point.

Some callers cannot allocate device memory: plug-ins that are handed only a
stream and their tensors by a host framework whose caching allocator owns
the GPU's memory, or latency-critical loops that must avoid cudaMalloc and
cudaFree because those can synchronise the device.
``simplex_atm_energy_noalloc`` serves them from a fixed scratch array inside
the library.  These tests call it through the C ABI (ctypes, raw pointers)
and compare it with the FP64 oracle where the oracle finishes in seconds,
and with ``simplex_atm_energy`` (caller-provided workspace) at the sizes
where it does not, always on two calls in a row and within the 1e-6
relative tolerance of the energy tests.  The largest accepted sizes and the
first rejected ones pin the scratch limit (grid blocks + 1024 reduction
slots <= 524,288 doubles); the lambda map at n = 4096 (401,408 grid blocks)
also runs the two-stage reduction, whose chunk sums sit in the same array.
This file is named so that pytest collects it last.
"""
import ctypes

import pytest
import torch

import synth

pytestmark = pytest.mark.gpu
E_TOL = 1e-6
ESCRATCH = 7
MAPS = ["lambda", "bbox", "linear"]


def call_noalloc(L, x, e, mp, nu=1.0, eps=1e-4):
    n, d = x.shape
    return L.simplex_atm_energy_noalloc(n, d, ctypes.c_void_p(x.data_ptr()), nu, eps,
                                        ctypes.c_void_p(e.data_ptr()), MAPS.index(mp),
                                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def noalloc_energy(L, pts, mp):
    x = torch.from_numpy(pts).cuda()
    got = torch.full((), float("nan"), dtype=torch.float64, device="cuda")
    assert call_noalloc(L, x, got, mp) == 0
    return got.item()


def test_noalloc_matches_oracle_twice(gpu, oracle):
    """Two calls in a row (different sizes and maps) against the oracle."""
    L = gpu.lib()
    cases = [(synth.make_points("atm_n1024"), "lambda"),
             (synth.uniform_cube(333, 3, 5.0, seed=77), "bbox")]
    for pts, mp in cases:
        assert noalloc_energy(L, pts, mp) == pytest.approx(oracle.atm_energy(pts), rel=E_TOL)


@pytest.mark.parametrize("mp,n_max", [("lambda", 4096), ("bbox", 2560), ("linear", 4640)])
def test_noalloc_largest_accepted_size(gpu, mp, n_max):
    """The largest n each map accepts, twice in a row, against the workspace
    entry point (the oracle's O(n^3) sum would take minutes here)."""
    L = gpu.lib()
    blocks = gpu.simplex_grid_blocks(3, (n_max + 31) // 32, mp)
    assert blocks + 1024 <= 1 << 19
    pts = synth.uniform_cube(n_max, 3, 20.0, seed=5 + n_max)
    ref = gpu.atm_energy_raw(torch.from_numpy(pts).cuda(), 1.0, 1e-4, mp).item()
    for _ in range(2):
        assert noalloc_energy(L, pts, mp) == pytest.approx(ref, rel=E_TOL)


@pytest.mark.parametrize("mp,n_first", [("lambda", 4097), ("bbox", 2561), ("linear", 4641)])
def test_noalloc_rejects_sizes_beyond_its_scratch(gpu, mp, n_first):
    L = gpu.lib()
    assert gpu.simplex_grid_blocks(3, (n_first + 31) // 32, mp) + 1024 > 1 << 19
    x = torch.zeros((n_first, 3), dtype=torch.float32, device="cuda")
    e = torch.zeros((), dtype=torch.float64, device="cuda")
    assert call_noalloc(L, x, e, mp) == ESCRATCH
    assert L.simplex_strerror(ESCRATCH)
    torch.cuda.synchronize()
    assert e.item() == 0.0
