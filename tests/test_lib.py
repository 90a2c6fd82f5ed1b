"""Host-side checks of libsimplex (no GPU needed).

* the library builds and exports every entry point ``include/simplex.h``
  declares;
* the map decode, compiled for the host from the same header the kernels
  use, equals the oracle's independent recursive construction bit for bit;
* argument validation returns status codes before any GPU work.
"""
import ctypes
import os
import re

import numpy as np
import pytest
import torch

import paper_1610_07394_gb300 as sx
from paper_1610_07394_gb300 import build as sxbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    sxbuild.build()
    return sx.lib()


def header_symbols():
    with open(os.path.join(ROOT, "include", "simplex.h")) as f:
        text = f.read()
    return sorted(set(re.findall(r"\b(simplex_\w+)\s*\(", text)))


def test_exports_every_declared_symbol(L):
    syms = header_symbols()
    assert len(syms) >= 15
    for s in syms:
        assert hasattr(L, s), s
    assert sorted(sx.EXPORTS) == syms


def test_abi_and_strerror(L):
    assert sx.simplex_abi_version() == 5
    for st in range(7):
        assert L.simplex_strerror(st)
    assert L.simplex_last_cuda_error() == 0


def host_table(m, nb, mp):
    g = sx.simplex_grid_blocks(m, nb, mp)
    t = torch.empty((g, 2 * m), dtype=torch.int32)
    sx.simplex_map_blocks_host(m, nb, mp, t)
    return t.numpy()


@pytest.mark.parametrize("mp", ["lambda", "bbox", "linear", "rb"])
@pytest.mark.parametrize("nb", [1, 2, 3, 4, 5, 7, 8, 16, 31, 64, 100, 256, 1024, 4096])
def test_decode2_host_equals_oracle(oracle, mp, nb):
    if mp != "lambda" and nb > 1024:
        pytest.skip("box/linear tables of this size add nothing")
    assert sx.simplex_grid_blocks(2, nb, mp) == np.prod(oracle.grid2(nb, mp))
    assert np.array_equal(host_table(2, nb, mp), oracle.table2(nb, mp))


@pytest.mark.parametrize("mp", ["lambda", "bbox", "linear"])
@pytest.mark.parametrize("nb", [1, 2, 3, 4, 5, 6, 8, 9, 16, 20, 32, 64, 128, 256])
def test_decode3_host_equals_oracle(oracle, mp, nb):
    if mp != "lambda" and nb > 128:
        pytest.skip("box/linear tables of this size add nothing")
    assert sx.simplex_grid_blocks(3, nb, mp) == np.prod(oracle.grid3(nb, mp))
    assert np.array_equal(host_table(3, nb, mp), oracle.table3(nb, mp))


@pytest.mark.parametrize("mp", ["lambda", "bbox"])
@pytest.mark.parametrize("nb", [1, 2, 3, 4, 5, 7, 8, 9, 16, 17, 31, 32, 33, 64])
def test_decode4_host_equals_oracle(oracle, mp, nb):
    """The library's closed-form m = 4 decode equals the oracle's table, which
    places each cross term of each level at its orthotope point (the inverse
    direction) and recurses."""
    if mp != "lambda" and nb > 32:
        pytest.skip("box tables of this size add nothing")
    assert sx.simplex_grid_blocks(4, nb, mp) == np.prod(oracle.grid4(nb, mp))
    assert np.array_equal(host_table(4, nb, mp), oracle.table4(nb, mp))


def test_linear_decode_large_indices(oracle):
    """The root-based inverse with its integer fix-up stays exact where FP32
    roots alone are off (8l+1 and 6l beyond 2^24): whole tables of a large
    triangle and tetrahedron against the oracle's enumeration."""
    nb = 4100
    assert np.array_equal(host_table(2, nb, "linear"), oracle.table2(nb, "linear"))
    nb = 300
    assert np.array_equal(host_table(3, nb, "linear"), oracle.table3(nb, "linear"))


def test_grid_and_workspace_sizes(L):
    assert sx.simplex_grid_blocks(2, 64, "lambda") == 32 * 64
    assert sx.simplex_grid_blocks(3, 32, "lambda") == 16 * 16 * (16 + 8 + 2)
    assert sx.simplex_grid_blocks(3, 32, "bbox") == 32 ** 3
    assert sx.simplex_grid_blocks(3, 32, "linear") == 32 * 33 * 34 // 6
    # m = 4: (p/2)^3 x (p/2 + p/8) for lambda (the plane K = L is the m = 3
    # grid's), nb^4 for the box, no linear or RB form
    assert sx.simplex_grid_blocks(4, 32, "lambda") == 16 ** 3 * (16 + 4)
    assert sx.simplex_grid_blocks(4, 4, "lambda") == 2 ** 3 * (2 + 1)
    assert sx.simplex_grid_blocks(4, 2, "lambda") == 1
    assert sx.simplex_grid_blocks(4, 32, "bbox") == 32 ** 4
    assert sx.simplex_grid_blocks(4, 32, "linear") == -1
    assert sx.simplex_grid_blocks(4, 32, "rb") == -1
    assert sx.simplex_grid_blocks(5, 32, "lambda") == -1
    # the rectangular box: 2-simplex only, exactly the triangle's blocks
    assert sx.simplex_grid_blocks(2, 32, "rb") == 32 * 33 // 2
    assert sx.simplex_grid_blocks(2, 33, "rb") == 33 * 34 // 2
    assert sx.simplex_grid_blocks(3, 32, "rb") == -1
    assert sx.simplex_workspace_bytes("atm_energy", 1024, 3, "rb") == -1
    assert sx.simplex_workspace_bytes("edm", 1024, 3, "rb") == 0
    rho = sx.simplex_block_rho("atm_energy")
    nb = -(-1024 // rho)
    # pair tables (16 KB per block pair of the 2-simplex of blocks), then one
    # FP64 partial per grid block and 1024 reduction slots
    assert sx.simplex_workspace_bytes("atm_energy", 1024, 3, "lambda") == nb * (nb + 1) // 2 * 16384 + 8 * (
        sx.simplex_grid_blocks(3, nb, "lambda") + 1024)
    # forces: their own pair tables (72 KB per block pair), the 16-byte tile
    # counter of the persistent kernel, then the partials
    assert sx.simplex_workspace_bytes("atm_forces", 1024, 3, "lambda") == nb * (nb + 1) // 2 * 73728 + 16 + 8 * (
        sx.simplex_grid_blocks(3, nb, "lambda") + 1024)
    assert sx.simplex_workspace_bytes("map2", 10, 1) == 0
    # loss and gradient in one pass: FP32 tiles need one FP64 partial per grid
    # block (64-point blocks); the tensor-core path the backward's workspace
    nb64 = -(-1000 // sx.simplex_block_rho("stress_fwd_bwd", 8, "fp32"))
    assert sx.simplex_workspace_bytes("stress_fwd_bwd", 1000, 8, "lambda", "fp32") == 8 * (
        sx.simplex_grid_blocks(2, nb64, "lambda") + 1024)
    assert sx.simplex_workspace_bytes("stress_fwd_bwd", 1000, 64, "lambda", "bf16x3") == \
        sx.simplex_workspace_bytes("stress_bwd", 1000, 64, "lambda", "bf16x3") > 0
    assert sx.simplex_workspace_bytes("atm_energy", 0, 3) == -1
    # tile-packed EDM: nt(nt+1)/2 tiles of 128 x 128, nt = ceil(n / 128)
    assert [sx.simplex_edm_tiles_len(n) for n in (1, 128, 129, 256, 65536)] == \
        [16384, 16384, 3 * 16384, 3 * 16384, 512 * 513 // 2 * 16384]
    assert sx.simplex_edm_tiles_len(0) == -1 and sx.simplex_edm_tiles_len((1 << 31) + 1) == -1


def test_validation_before_gpu_work(L):
    """Bad arguments come back as status codes; nothing reaches the GPU."""
    null = None
    assert L.simplex_edm_packed(0, 3, 16, 16, 0, 0, null, 0, null) == 1          # n < 1
    assert L.simplex_edm_packed(4, 3, null, 16, 0, 0, null, 0, null) == 1        # NULL x
    assert L.simplex_edm_packed(4, 3, 16, 16, 7, 0, null, 0, null) == 1          # bad map
    assert L.simplex_edm_packed(4, 3, 17, 16, 0, 0, null, 0, null) == 2          # misaligned x
    assert L.simplex_atm_energy(8, 2, 16, 1.0, 1e-4, 16, 0, null, 0, null) == 4   # d != 3
    assert L.simplex_atm_energy(8, 3, 16, 1.0, 1e-4, 16, 0, null, 0, null) == 6   # no workspace
    assert L.simplex_atm_energy(8, 3, 16, 1.0, 1e-4, 16, 0, 256, 16, null) == 6  # too small
    assert L.simplex_map2(10, 33, 0, 16, 16, null) == 1                          # rho > 32
    assert L.simplex_map3(10, 11, 0, 16, 16, null) == 1                          # rho^3 > 1024
    assert L.simplex_map4(10, 6, 0, 16, 16, null) == 1                           # rho^4 > 1024
    assert L.simplex_map4(10, 4, 2, 16, 16, null) == 1                           # no m = 4 linear map
    assert L.simplex_map4(10, 4, 3, 16, 16, null) == 1                           # no m = 4 RB
    assert L.simplex_map4(65537, 4, 0, 16, 16, null) == 3                        # index overflow
    # size limits, reported before any device work
    assert L.simplex_map2((1 << 31) + 1, 16, 0, 16, 16, null) == 3               # n > 2^31
    assert L.simplex_map3(3000001, 8, 0, 16, 16, null) == 3                      # 64-bit index bound
    assert L.simplex_edm_packed((1 << 31) + 1, 3, 16, 16, 0, 0, null, 0, null) == 3   # n > 2^31
    assert L.simplex_edm_packed(1 << 20, (1 << 24) + 1, 16, 16, 0, 0, null, 0, null) == 3  # d > 2^24
    assert L.simplex_atm_energy((1 << 22) + 1, 3, 16, 1.0, 1e-4, 16, 0, null, 0, null) == 3  # n > 2^22
    assert L.simplex_atm_energy(0, 3, 16, 1.0, 1e-4, 16, 0, null, 0, null) == 1               # empty
    assert L.simplex_map2(0, 16, 0, 16, 16, null) == 1                                         # empty
    assert L.simplex_map4(0, 4, 0, 16, 16, null) == 1                                          # empty
    assert L.simplex_stress_bwd(8, 4, 16, 16, 1.0, 20, 0, 0, null, 0, null) == 2  # grad not 16B
    assert L.simplex_stress_fwd_bwd(8, 4, 16, 16, 1.0, 16, null, 0, 0, null, 0, null) == 1  # NULL loss
    assert L.simplex_stress_fwd_bwd(8, 4, 16, 16, 1.0, null, 16, 0, 0, null, 0, null) == 1  # NULL grad
    assert L.simplex_stress_fwd_bwd(8, 4, 16, 16, 1.0, 16, 12, 0, 0, null, 0, null) == 2    # loss not 8B
    assert L.simplex_stress_fwd_bwd(8, 4, 16, 16, 1.0, 16, 16, 0, 0, null, 0, null) == 6    # no workspace
    assert L.simplex_edm_tiles(0, 3, 16, 16, 0, 0, null, 0, null) == 1           # n < 1
    assert L.simplex_edm_tiles(4, 3, 16, 16, 4, 0, null, 0, null) == 1           # bad map
    assert L.simplex_edm_tiles((1 << 31) + 1, 3, 16, 16, 0, 0, null, 0, null) == 3   # n > 2^31
    assert L.simplex_edm_tiles(8, 64, 16, 16, 0, 1, null, 0, null) == 6          # no workspace
    assert L.simplex_edm_tiles(8, 64, 16, 20, 0, 1, 256, 1 << 20, null) == 2     # TMA stores need 16 B
    assert L.simplex_map_blocks_host(2, 4, 0, null) == 1
    assert L.simplex_map3(10, 4, 3, 16, 16, null) == 1                           # no 3-simplex RB
    assert L.simplex_atm_energy(8, 3, 16, 1.0, 1e-4, 16, 3, 256, 1 << 20, null) == 1  # RB for m = 3


def test_binding_requires_cuda_tensors(L):
    x = torch.zeros(8, 3)
    with pytest.raises(TypeError):
        sx.simplex_atm_energy(x, 1.0, 1e-4, torch.zeros((), dtype=torch.float64))
