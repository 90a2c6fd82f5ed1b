"""Pins for the CPU oracle: facts fixed by the paper and by mathematics.

Nothing here calls the CUDA library.  Each test checks the oracle against
something other than itself: closed forms the paper prints, brute force on
tiny inputs written differently from the oracle, invariants, and finite
differences.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")


def paper():
    with open(GOLDEN) as f:
        return json.load(f)


# ---------------------------------------------------------------- helpers

def lambda2_closed_form(nb):
    """Eq. (map2d): lambda(w) = (w_x + q b, w_y + 2 q b), b = 2^floor(log2 w_y),
    q = floor(w_x / b), for grid rows w_y >= 1 of the (nb/2) x nb grid."""
    out = {}
    for wy in range(1, nb):
        b = 1 << (wy.bit_length() - 1)
        for wx in range(nb // 2):
            q = wx // b
            out[(wx, wy)] = (wx + q * b, wy + 2 * q * b)
    return out


def lambda3_closed_form(p):
    """The two-case 3-simplex map read with the shared parameters b, q
    (Sec. III-C), written as a direct formula (no recursion)."""
    h0 = p // 2
    out = {}
    for wz in range(h0 + p // 4):
        for wy in range(h0):
            for wx in range(h0):
                if wz < h0:
                    h, off, s, u, v = h0, 0, wx, wy, wz
                else:
                    if wy == 0:
                        continue
                    b = 1 << (wy.bit_length() - 1)
                    z = wz - h0
                    if z >= b:
                        continue
                    q = wx // b
                    h, off, s, u, v = b, 2 * q * b, wx - q * b, wy - b, z
                if u <= s:
                    out[(wx, wy, wz)] = (off + u, off + s, off + h + v)
                else:
                    out[(wx, wy, wz)] = (off + v, off + h + s, off + h + u)
    return out


def blocks_of(tab, width):
    """All data blocks listed in a table, as tuples."""
    res = []
    for row in tab:
        for s in range(2):
            e = row[width * s: width * (s + 1)]
            if e[0] >= 0:
                res.append(tuple(int(v) for v in e))
    return res


# ---------------------------------------------------------------- volumes

def test_general_volume_formula_reduces_to_m2_m3_m4():
    """Sec. III-D, eq. (generic-m) with r = 1/2, beta = 2 gives eq. (m2), the
    two-branch eq. (m3), and (n^4 - n)/14 for m = 4."""
    for k in range(1, 12):
        n = 2 ** k
        for m, denom in ((2, 2), (3, 6), (4, 14)):
            generic = (n ** m - 2 ** k) / (2 ** m - 2)
            assert generic == (n ** m - n) / denom
        # recursion V(S_n) = (n/2)^m + 2 V(S_{n/2}), V(S_1) = 0
        for m in (2, 3, 4):
            v = 0
            for j in range(1, k + 1):
                v = (2 ** j // 2) ** m + 2 * v
            assert v * (2 ** m - 2) == n ** m - n


def test_general_m_limits_match_paper():
    g = paper()
    for m, want in ((4, g["general_m_r_half_beta_2"]["m4_extra_limit"]),
                    (5, g["general_m_extra_limit"]["m5"]),
                    (7, g["general_m_extra_limit"]["m7"])):
        assert math.factorial(m) / (2 ** m - 2) - 1 == pytest.approx(want, rel=1e-12)
    assert (1 / 5) == pytest.approx(g["three_branch_extra_volume_limit"]["value"])


# ---------------------------------------------------------------- 2-simplex maps

@pytest.mark.parametrize("k", range(1, 13))
def test_lambda2_recursive_equals_closed_form(oracle, k):
    """The recursive construction of S_n^2 (Sec. III-A) and the O(1) formula of
    eq. (map2d) give the same block for every grid block with w_y >= 1."""
    nb = 2 ** k
    tab = oracle.table2(nb, "lambda")
    gx, gy = oracle.grid2(nb, "lambda")
    assert (gx, gy) == (nb // 2, nb)
    got = tab.reshape(gy, gx, 4)
    if nb <= 256:
        ref = lambda2_closed_form(nb)
        for (wx, wy), (X, Y) in ref.items():
            assert tuple(got[wy, wx]) == (X, Y, -1, -1), (nb, wx, wy)
    else:  # vectorised form of the same closed form
        wy, wx = np.meshgrid(np.arange(1, nb), np.arange(nb // 2), indexing="ij")
        b = 2 ** np.floor(np.log2(wy)).astype(np.int64)
        q = wx // b
        assert np.array_equal(got[1:, :, 0], wx + q * b)
        assert np.array_equal(got[1:, :, 1], wy + 2 * q * b)
    # grid row 0: the diagonal block pair (the reading used throughout)
    assert np.array_equal(got[0, :, 0], 2 * np.arange(gx))
    assert np.array_equal(got[0, :, 2], 2 * np.arange(gx) + 1)


@pytest.mark.parametrize("nb", [1, 2, 3, 5, 8, 13, 64, 100, 256])
@pytest.mark.parametrize("m", ["lambda", "bbox", "linear", "rb"])
def test_table2_is_bijection(oracle, nb, m):
    """Every block of the lower block triangle {X <= Y < nb} is listed once."""
    blocks = blocks_of(oracle.table2(nb, m), 2)
    want = [(x, y) for y in range(nb) for x in range(y + 1)]
    assert sorted(blocks) == sorted(want)
    assert len(blocks) == nb * (nb + 1) // 2


@pytest.mark.parametrize("nb", range(1, 41))
def test_rb_rows_fold(oracle, nb):
    """Rectangular box: a grid of exactly nb(nb+1)/2 blocks for every nb (no
    idle block, unlike lambda off powers of two), grid row k holding only
    triangle rows floor(nb/2) + k and floor(nb/2) - 1 - k, the longer one
    first and each row's blocks in column order."""
    gx, gy = oracle.grid2(nb, "rb")
    assert gx * gy == nb * (nb + 1) // 2
    tab = oracle.table2(nb, "rb").reshape(gy, gx, 4)
    h = nb // 2
    for k in range(gy):
        row = [tuple(e[:2]) for e in tab[k]]
        lo = [(x, h + k) for x in range(h + k + 1)]
        hi = [(x, h - 1 - k) for x in range(h - k)] if h - 1 - k >= 0 else []
        assert row == lo + hi
    assert (tab[:, :, 2] == -1).all()


@pytest.mark.parametrize("k", range(1, 11))
def test_lambda2_volume_is_S_n(oracle, k):
    """Off-diagonal blocks of the lambda grid = V(S_n^2) = n(n-1)/2 (eq. m2),
    and V(S_{n+1}) = V(S_n) + n = V(Delta_n^2)."""
    nb = 2 ** k
    tab = oracle.table2(nb, "lambda")
    gx, _ = oracle.grid2(nb, "lambda")
    off_diag = int((tab[gx:, 0] >= 0).sum())
    assert off_diag == nb * (nb - 1) // 2
    assert off_diag + nb == nb * (nb + 1) // 2


def test_bbox2_extra_volume(oracle):
    """Sec. I, Eq. 3: the bounding box grid is ~2x Delta^2 (alpha -> 1)."""
    g = paper()
    nb = 4096
    gx, gy = oracle.grid2(nb, "bbox")
    alpha = gx * gy / (nb * (nb + 1) / 2) - 1
    assert alpha == pytest.approx(g["bbox_extra_volume_limit"]["m2"], abs=1e-3)
    lgx, lgy = oracle.grid2(nb, "lambda")
    assert gx * gy / (lgx * lgy) == pytest.approx(g["lambda2_space_improvement_vs_bbox"]["value"])


# ---------------------------------------------------------------- 3-simplex maps

@pytest.mark.parametrize("k", range(1, 8))
def test_lambda3_recursive_equals_closed_form(oracle, k):
    """The recursive two-branch construction (Sec. III-C) equals the direct
    formula with b = 2^floor(log2 w_y), q = floor(w_x / b)."""
    p = 2 ** k
    gx, gy, gz = oracle.grid3(p, "lambda")
    assert (gx, gy, gz) == (p // 2, p // 2, p // 2 + p // 4 + 2)
    tab = oracle.table3(p, "lambda").reshape(gz, gy, gx, 6)
    ref = lambda3_closed_form(p)
    for wz in range(gz - 2):
        for wy in range(gy):
            for wx in range(gx):
                e = tuple(int(v) for v in tab[wz, wy, wx])
                if (wx, wy, wz) in ref:
                    assert e == ref[(wx, wy, wz)] + (-1, -1, -1)
                else:
                    assert e == (-1,) * 6


@pytest.mark.parametrize("nb", [1, 2, 3, 4, 5, 8, 11, 16, 32, 64])
@pytest.mark.parametrize("m", ["lambda", "bbox", "linear"])
def test_table3_is_bijection(oracle, nb, m):
    """Every block of {I <= J <= K < nb} is listed exactly once."""
    blocks = blocks_of(oracle.table3(nb, m), 3)
    want = [(i, j, k) for k in range(nb) for j in range(k + 1) for i in range(j + 1)]
    assert len(blocks) == len(want) == nb * (nb + 1) * (nb + 2) // 6
    assert sorted(blocks) == sorted(want)


@pytest.mark.parametrize("k", range(1, 9))
def test_lambda3_volume_and_extra(oracle, k):
    """The cube part lists V(S_n^3) = (n^3 - n)/6 blocks (two-branch eq. m3),
    i.e. {I <= J < K}; its grid is (n/2)(n/2)(3n/4) and the extra volume
    tends to 2/16 (Sec. III-C)."""
    p = 2 ** k
    gx, gy, gz = oracle.grid3(p, "lambda")
    tab = oracle.table3(p, "lambda").reshape(gz, gy * gx, 6)
    cube = blocks_of(tab[: gz - 2].reshape(-1, 6), 3)
    assert len(cube) == (p ** 3 - p) // 6
    assert all(i <= j < kk for i, j, kk in cube)
    grid_cube = gx * gy * (gz - 2)
    if p >= 4:
        assert grid_cube == 3 * p ** 3 // 16
        alpha = grid_cube / ((p ** 3 - p) / 6) - 1
        assert alpha == pytest.approx(9 * p * p / (8 * (p * p - 1)) - 1, rel=1e-12)
    if p == 256:
        assert alpha == pytest.approx(paper()["lambda3_extra_volume"]["value"], abs=1e-4)


# ---------------------------------------------------------------- 4-simplex maps

@pytest.mark.parametrize("nb", [1, 2, 3, 4, 5, 7, 8, 9, 13, 16, 24])
@pytest.mark.parametrize("m", ["lambda", "bbox"])
def test_table4_is_bijection(oracle, nb, m):
    """lambda lists every block of {I <= J <= K < L < nb} exactly once (the
    plane K = L is left to the 3-simplex map) and no grid point twice (the
    construction raises on a collision); the box lists every block of
    {I <= J <= K <= L}."""
    blocks = blocks_of(oracle.table4(nb, m), 4)
    strict = m == "lambda"
    want = [(i, j, k, l) for l in range(nb) for k in range(l if strict else l + 1)
            for j in range(k + 1) for i in range(j + 1)]
    assert len(blocks) == len(want) == math.comb(nb + (2 if strict else 3), 4)
    assert sorted(blocks) == sorted(want)


@pytest.mark.parametrize("k", range(1, 7))
def test_lambda4_volume_and_extra(oracle, k):
    """The recursive set S_n^4 (r = 1/2, beta = 2) holds (n^4 - n)/14 grid
    points (Sec. III-D), at least the C(n+2, 4) blocks I <= J <= K < L it
    covers (the paper's strict inequality holds from n = 4; at n = 2 both
    are 1), inside a grid of (n/2)^3 (n/2 + n/8) blocks."""
    p = 2 ** k
    V = oracle.volume4(p)
    assert V * 14 == p ** 4 - p
    D = math.comb(p + 2, 4)
    assert V >= D and (V > D or p == 2)
    assert len(blocks_of(oracle.table4(p, "lambda"), 4)) == D
    assert int(np.prod(oracle.grid4(p, "lambda"))) >= V


def test_lambda4_extra_volume_limit(oracle):
    """Sec. III-D: the extra volume of the r = 1/2, beta = 2 set tends to
    m!/(2^m - 2) - 1 = 5/7 for m = 4."""
    p = 2 ** 13
    V = oracle.volume4(p)
    assert V / math.comb(p + 2, 4) - 1 == pytest.approx(
        paper()["general_m_r_half_beta_2"]["m4_extra_limit"], abs=1e-3)


def test_bbox3_extra_volume(oracle):
    g = paper()
    nb = 1024
    gx, gy, gz = oracle.grid3(nb, "bbox")
    alpha = gx * gy * gz / (nb * (nb + 1) * (nb + 2) / 6) - 1
    assert alpha == pytest.approx(g["bbox_extra_volume_limit"]["m3"], abs=0.02)
    # lambda grid vs box: 6 / (1 + 1/8) in the limit
    lg = np.prod(oracle.grid3(nb, "lambda"))
    assert gx * gy * gz / lg == pytest.approx(g["lambda3_space_improvement_vs_bbox"]["value"] / 1.125, rel=0.01)


# ---------------------------------------------------------------- coverage

def brute_idle2(n, rho, m, nb, table):
    """Idle threads by direct enumeration of the thread rule."""
    idle = 0
    gx = len(table) if m != "lambda" else None
    for w, e in enumerate(table):
        for r in range(rho):
            for c in range(rho):
                took = False
                if m == "lambda" and w < nb_pow2(nb) // 2:
                    cells = [(r, c)] + ([(r, rho)] if c == 0 else [])
                    for (rr, cc) in cells:
                        if cc <= rr:
                            i = 2 * w * rho + rr
                        else:
                            i = (2 * w + 1) * rho + (rho - 1 - rr)
                        took |= i < n
                elif e[0] >= 0:
                    i, j = e[1] * rho + r, e[0] * rho + c
                    took = j <= i < n
                idle += not took
    return idle


def nb_pow2(nb):
    p = 2
    while p < nb:
        p *= 2
    return p


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 16, 33, 64, 100])
@pytest.mark.parametrize("rho", [1, 2, 4, 8])
@pytest.mark.parametrize("m", ["lambda", "bbox", "linear", "rb"])
def test_cover2(oracle, n, rho, m):
    """Every element of Delta_n^2 (n(n+1)/2 of them) is hit exactly once."""
    counts, idle = oracle.cover2(n, rho, m)
    assert counts.size == n * (n + 1) // 2
    assert (counts == 1).all()
    nb = -(-n // rho)
    assert idle == brute_idle2(n, rho, m, nb, oracle.table2(nb, m))
    if n % rho == 0:
        if m == "bbox":
            assert idle == nb * (nb - 1) // 2 * rho * rho + nb * rho * (rho - 1) // 2
        if m in ("linear", "rb"):
            assert idle == nb * rho * (rho - 1) // 2
        if m == "lambda" and nb == nb_pow2(nb):
            assert idle == 0  # the diagonal pairing leaves no thread idle


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 17, 32])
@pytest.mark.parametrize("rho", [1, 2, 4])
@pytest.mark.parametrize("m", ["lambda", "bbox", "linear"])
def test_cover3(oracle, n, rho, m):
    counts, idle = oracle.cover3(n, rho, m)
    assert counts.size == n * (n + 1) * (n + 2) // 6
    assert (counts == 1).all()
    nb = -(-n // rho)
    if n % rho == 0:
        V = n * (n + 1) * (n + 2) // 6
        g = int(np.prod(oracle.grid3(nb, m)))
        busy_pair = math.comb(rho + 2, 3)  # threads busy in both blocks of a diagonal pair
        pairs = 0
        if m == "lambda":
            tab = oracle.table3(nb, m)
            pairs = int((tab[:, 3] >= 0).sum())
        assert idle == g * rho ** 3 - V + pairs * busy_pair


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 13, 17])
@pytest.mark.parametrize("rho", [1, 2, 4])
@pytest.mark.parametrize("m", ["lambda", "bbox"])
def test_cover4(oracle, n, rho, m):
    """Every element of Delta_n^4 (C(n+3, 4) of them) is reached once; with
    n a multiple of rho the idle threads are the launched threads less the
    elements, plus the threads that take an element in both blocks of a
    diagonal pair of the m = 3 grid that carries the plane K = L."""
    counts, idle = oracle.cover4(n, rho, m)
    assert counts.size == math.comb(n + 3, 4)
    assert (counts == 1).all()
    nb = -(-n // rho)
    if n % rho == 0:
        g = int(np.prod(oracle.grid4(nb, m)))
        pairs = 0
        if m == "lambda":
            g += int(np.prod(oracle.grid3(nb, "lambda")))
            pairs = int((oracle.table3(nb, "lambda")[:, 3] >= 0).sum())
        assert idle == g * rho ** 4 - math.comb(n + 3, 4) + pairs * math.comb(rho + 3, 4)


# ---------------------------------------------------------------- EDM

def test_edm_line_closed_form(oracle):
    """Points on a line at spacing s: D_ij = ((i - j) s)^2."""
    n, s = 40, 0.75
    x = np.zeros((n, 3))
    x[:, 1] = s * np.arange(n)
    D = oracle.edm_packed(x)
    for i in range(n):
        for j in range(i + 1):
            assert D[i * (i + 1) // 2 + j] == ((i - j) * s) ** 2


def test_edm_integer_lattice_matches_gram_form(oracle):
    """On integer coordinates every step is exact, so the difference form of
    the oracle equals the Gram form |x|^2 + |y|^2 - 2 x.y bit for bit."""
    rng = np.random.default_rng(7)
    x = rng.integers(-50, 50, size=(61, 9)).astype(np.float64)
    D = oracle.edm_packed(x)
    G = x @ x.T
    nrm = np.diag(G)
    full = nrm[:, None] + nrm[None, :] - 2 * G
    i, j = np.tril_indices(len(x))
    assert np.array_equal(D, full[i, j])


def test_edm_invariances(oracle):
    x = synth.normal(50, 7, seed=11).astype(np.float64)
    D = oracle.edm_packed(x)
    assert np.allclose(oracle.edm_packed(x + 3.25), D, rtol=1e-12, atol=1e-12)
    assert np.allclose(oracle.edm_packed(2.0 * x), 4.0 * D, rtol=1e-15)
    perm = synth.sample_indices(50, 50, seed=3)
    Dp = oracle.edm_packed(x[perm])
    for a in range(50):
        for b in range(a + 1):
            i, j = max(perm[a], perm[b]), min(perm[a], perm[b])
            assert Dp[a * (a + 1) // 2 + b] == pytest.approx(D[i * (i + 1) // 2 + j], rel=1e-14)
    i = np.arange(50)
    assert (D[i * (i + 1) // 2 + i] == 0).all()


@pytest.mark.parametrize("n", [1, 127, 128, 129, 300])
def test_edm_tiles_layout(oracle, n):
    """Tile-packed layout on points of a line (x_i = i, so D_ij = (i - j)^2
    names the pair): walking the tile triangle row by row with nested loops,
    each 128 x 128 block is the corresponding block of the full square matrix
    (numpy broadcasting), the padding past n is 0, every float is accounted
    for, and the lower entries of the tiles are exactly the packed rows."""
    x = np.zeros((n, 2))
    x[:, 0] = np.arange(n)
    T = oracle.edm_tiles(x)
    nt = -(-n // 128)
    full = np.zeros((nt * 128, nt * 128))
    idx = np.arange(n, dtype=np.float64)
    full[:n, :n] = (idx[:, None] - idx[None, :]) ** 2
    off, lower = 0, []
    for I in range(nt):
        for J in range(I + 1):
            blk = T[off:off + 128 * 128].reshape(128, 128)
            assert np.array_equal(blk, full[128 * I:128 * I + 128, 128 * J:128 * J + 128])
            off += 128 * 128
    assert off == len(T)
    # gather the lower triangle back from the tiles, row by row
    for i in range(n):
        I = i // 128
        row = [T[(I * (I + 1) // 2 + j // 128) * 16384 + (i % 128) * 128 + j % 128] for j in range(i + 1)]
        lower.extend(row)
    assert np.array_equal(np.array(lower), oracle.edm_packed(x))


def test_edm_pairs_matches_packed(oracle):
    x = synth.normal(80, 5, seed=2)
    D = oracle.edm_packed(x)
    pr = synth.sample_pairs(500, 80, seed=9)
    got = oracle.edm_pairs(x, pr)
    assert np.array_equal(got, D[pr[:, 0] * (pr[:, 0] + 1) // 2 + pr[:, 1]])


# ---------------------------------------------------------------- ATM

def test_atm_equilateral(oracle):
    """Equilateral side L: every angle is 60 deg, each vertex dot product is
    L^2/2; softened: e = nu (1 + 3 (L^2/2 / s)^3) / s^{9/2}, s = L^2 + eps.
    At eps = 0 this is 11 / (8 L^9)."""
    L = 1.3
    x = np.array([[0, 0, 0], [L, 0, 0], [L / 2, L * math.sqrt(3) / 2, 0]])
    assert oracle.atm_energy(x, 1.0, 0.0) == pytest.approx(11 / (8 * L ** 9), rel=1e-13)
    eps, nu = 1e-2, 0.7
    s = L * L + eps
    want = nu * (1 + 3 * (L * L / 2 / s) ** 3) / s ** 4.5
    assert oracle.atm_energy(x, nu, eps) == pytest.approx(want, rel=1e-13)


def test_atm_collinear(oracle):
    """Equally spaced on a line (a, a, 2a): cosines 1, -1, 1, so
    e = -2 / (a a 2a)^3 = -1 / (4 a^9)."""
    a = 0.9
    x = np.array([[0, 0, 0], [0, a, 0], [0, 2 * a, 0]])
    assert oracle.atm_energy(x, 1.0, 0.0) == pytest.approx(-1 / (4 * a ** 9), rel=1e-12)


def test_atm_right_angle(oracle):
    """A right angle makes the cosine product 0: e = P^{-3/2} exactly, also
    with softening."""
    L, eps = 1.1, 3e-3
    x = np.array([[0, 0, 0], [L, 0, 0], [0, L, 0]])
    P = (L * L + eps) * (L * L + eps) * (2 * L * L + eps)
    assert oracle.atm_energy(x, 1.0, eps) == pytest.approx(P ** -1.5, rel=1e-13)


def test_atm_bruteforce_law_of_cosines(oracle):
    """Pure-Python brute force at eps = 0, with the cosines from side lengths
    (law of cosines) instead of the oracle's dot products."""
    x = synth.uniform_cube(9, 3, 2.0, seed=5).astype(np.float64)
    tot = 0.0
    for i, j, k in itertools.combinations(range(9), 3):
        rij = math.dist(x[i], x[j]); rjk = math.dist(x[j], x[k]); rki = math.dist(x[k], x[i])
        ci = (rij ** 2 + rki ** 2 - rjk ** 2) / (2 * rij * rki)
        cj = (rij ** 2 + rjk ** 2 - rki ** 2) / (2 * rij * rjk)
        ck = (rjk ** 2 + rki ** 2 - rij ** 2) / (2 * rjk * rki)
        tot += (1 + 3 * ci * cj * ck) / (rij * rjk * rki) ** 3
    assert oracle.atm_energy(x, 1.0, 0.0) == pytest.approx(tot, rel=1e-11)


def test_atm_grad_abs(oracle):
    """The per-atom sum of the magnitudes of the gradient's per-side parts.
    Equilateral triangle: at each atom two parts of equal length at 60
    degrees, so the sum is 2/sqrt(3) times the gradient's norm, whatever the
    side derivative is.  Right isosceles triangle: at the right-angle vertex
    two equal parts at 90 degrees, ratio sqrt(2).  Additive over the four
    triples of four atoms; at least the gradient's norm on a cloud;
    homogeneous of degree -10 without softening (the gradient of a degree -9
    energy)."""
    L = 1.3
    tri = np.array([[0, 0, 0], [L, 0, 0], [L / 2, L * np.sqrt(3) / 2, 0]])
    for eps in (0.0, 1e-4):
        k = oracle.atm_grad_abs(tri, 1.0, eps)
        g = np.linalg.norm(oracle.atm_grad(tri, 1.0, eps), axis=1)
        assert np.allclose(k / g, 2 / np.sqrt(3), rtol=1e-12)
    ri = np.array([[0.4, 0.0, 0.0], [0.0, 0.0, 0.0], [0.0, 0.4, 0.0]])   # right angle at atom 1
    k = oracle.atm_grad_abs(ri, 1.0, 1e-4)
    g = np.linalg.norm(oracle.atm_grad(ri, 1.0, 1e-4), axis=1)
    assert k[1] / g[1] == pytest.approx(np.sqrt(2), rel=1e-12)
    four = synth.uniform_cube(4, 3, 2.0, seed=91).astype(np.float64)
    total = np.zeros(4)
    for drop in range(4):
        keep = [a for a in range(4) if a != drop]
        total[keep] += oracle.atm_grad_abs(four[keep], 1.0, 1e-4)
    assert np.allclose(oracle.atm_grad_abs(four, 1.0, 1e-4), total, rtol=1e-12)
    cloud = synth.uniform_cube(40, 3, 3.0, seed=92)
    k = oracle.atm_grad_abs(cloud, 1.0, 1e-4)
    g = np.linalg.norm(oracle.atm_grad(cloud, 1.0, 1e-4), axis=1)
    assert (k >= g * (1 - 1e-12)).all() and (k > 1.5 * g).any()
    c = cloud.astype(np.float64)
    assert np.allclose(oracle.atm_grad_abs(2.0 * c, 1.0, 0.0), 2.0 ** -10 * oracle.atm_grad_abs(c, 1.0, 0.0),
                       rtol=1e-10)


def test_atm_abs_energy(oracle):
    """Sum of |e| over the triples: on one triangle it is |E| of the closed
    forms (equilateral e > 0, collinear e < 0); on a cloud it matches a
    pure-Python brute force of sum |e| with law-of-cosines cosines at
    eps = 0, exceeds |E| when the terms have both signs, and equals E on a
    set whose terms are all positive (acute triangles only: a regular
    tetrahedron)."""
    L, a = 1.3, 0.9
    tri = np.array([[0, 0, 0], [L, 0, 0], [L / 2, L * math.sqrt(3) / 2, 0]])
    line = np.array([[0, 0, 0], [0, a, 0], [0, 2 * a, 0]])
    assert oracle.atm_abs_energy(tri, 1.0, 0.0) == pytest.approx(11 / (8 * L ** 9), rel=1e-13)
    assert oracle.atm_abs_energy(line, 1.0, 0.0) == pytest.approx(1 / (4 * a ** 9), rel=1e-12)
    x = synth.uniform_cube(9, 3, 2.0, seed=5).astype(np.float64)
    tot, signs = 0.0, set()
    for i, j, k in itertools.combinations(range(9), 3):
        rij = math.dist(x[i], x[j]); rjk = math.dist(x[j], x[k]); rki = math.dist(x[k], x[i])
        ci = (rij ** 2 + rki ** 2 - rjk ** 2) / (2 * rij * rki)
        cj = (rij ** 2 + rjk ** 2 - rki ** 2) / (2 * rij * rjk)
        ck = (rjk ** 2 + rki ** 2 - rij ** 2) / (2 * rjk * rki)
        e = (1 + 3 * ci * cj * ck) / (rij * rjk * rki) ** 3
        signs.add(e > 0)
        tot += abs(e)
    assert signs == {True, False}
    A = oracle.atm_abs_energy(x, 1.0, 0.0)
    assert A == pytest.approx(tot, rel=1e-11)
    assert A > abs(oracle.atm_energy(x, 1.0, 0.0)) * (1 + 1e-9)
    tet = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], np.float64)
    assert oracle.atm_abs_energy(tet, 0.5, 1e-3) == pytest.approx(oracle.atm_energy(tet, 0.5, 1e-3), rel=1e-14)


def random_rotation(seed):
    q, r = np.linalg.qr(synth.normal(3, 3, seed=seed).astype(np.float64))
    return q * np.sign(np.diag(r))


def test_atm_invariances(oracle):
    x = synth.uniform_cube(24, 3, 3.0, seed=8).astype(np.float64)
    E = oracle.atm_energy(x)
    assert oracle.atm_energy(x + np.array([1.5, -2.0, 0.25])) == pytest.approx(E, rel=1e-11)
    assert oracle.atm_energy(x @ random_rotation(4).T) == pytest.approx(E, rel=1e-11)
    perm = synth.sample_indices(24, 24, seed=12)
    assert oracle.atm_energy(x[perm]) == pytest.approx(E, rel=1e-12)


def test_atm_grad_finite_differences(oracle):
    """Central differences of the FP64 energy match the analytic gradient."""
    x = synth.uniform_cube(8, 3, 2.0, seed=13).astype(np.float64)
    g = oracle.atm_grad(x)
    h = 1e-5
    fd = np.zeros_like(x)
    for a in range(len(x)):
        for t in range(3):
            xp, xm = x.copy(), x.copy()
            xp[a, t] += h
            xm[a, t] -= h
            fd[a, t] = (oracle.atm_energy(xp) - oracle.atm_energy(xm)) / (2 * h)
    assert np.allclose(g, fd, rtol=1e-6, atol=1e-9 * np.abs(g).max())


def test_atm_atom_energy_and_grad_rows(oracle):
    x = synth.uniform_cube(20, 3, 3.0, seed=14).astype(np.float64)
    E = oracle.atm_energy(x)
    parts = [oracle.atm_atom_energy(x, a) for a in range(20)]
    assert sum(parts) == pytest.approx(3 * E, rel=1e-12)
    g = oracle.atm_grad(x)
    atoms = [0, 7, 19, 3]
    assert np.allclose(oracle.atm_grad_atoms(x, atoms), g[atoms], rtol=1e-12, atol=1e-14 * np.abs(g).max())
    # FD through the partial energy of one atom (what the full-size checks use)
    h = 1e-5
    for a in atoms[:2]:
        for t in range(3):
            xp, xm = x.copy(), x.copy()
            xp[a, t] += h
            xm[a, t] -= h
            fd = (oracle.atm_atom_energy(xp, a) - oracle.atm_atom_energy(xm, a)) / (2 * h)
            assert fd == pytest.approx(g[a, t], rel=1e-6, abs=1e-9 * np.abs(g).max())
    assert oracle.atm_energy_slice(x, 0, 20) == pytest.approx(E, rel=1e-15)
    assert oracle.atm_energy_slice(x, 0, 7) + oracle.atm_energy_slice(x, 7, 20) == pytest.approx(E, rel=1e-13)


def test_atm_force_balance_and_euler(oracle):
    """Translation invariance: sum of gradients is 0; rotation invariance:
    total torque is 0; at eps = 0 the energy is homogeneous of degree -9, so
    sum_i x_i . grad_i E = -9 E (Euler's theorem)."""
    x = synth.uniform_cube(16, 3, 3.0, seed=15).astype(np.float64)
    g = oracle.atm_grad(x)
    scale = np.abs(g).sum()
    assert np.abs(g.sum(axis=0)).max() < 1e-12 * scale
    assert np.abs(np.cross(x, g).sum(axis=0)).max() < 1e-11 * scale * np.abs(x).max()
    g0 = oracle.atm_grad(x, 1.0, 0.0)
    E0 = oracle.atm_energy(x, 1.0, 0.0)
    assert (x * g0).sum() == pytest.approx(-9 * E0, rel=1e-10)


# ---------------------------------------------------------------- stress

def test_stress_two_points(oracle):
    x = np.array([[0.0, 1.0], [2.0, -1.0]])
    y = np.array([[0.5, 0.0], [1.0, 1.0]])
    D, delta = 8.0, 1.25
    assert oracle.stress_loss(x, y) == (D - delta) ** 2
    g = oracle.stress_grad_rows(x, y, [0, 1])
    assert np.allclose(g[0], 4 * (D - delta) * (x[0] - x[1]), rtol=1e-15)
    assert np.allclose(g[1], -g[0], rtol=1e-15)


def test_stress_zero_at_reference(oracle):
    x = synth.normal(30, 4, seed=16)
    assert oracle.stress_loss(x, x) == 0.0
    assert (oracle.stress_grad_rows(x, x, range(30)) == 0).all()


def test_stress_fd_and_balance(oracle):
    x = synth.normal(12, 5, seed=17).astype(np.float64)
    y = synth.perturbed(x.astype(np.float32), 0.3, seed=18).astype(np.float64)
    g = oracle.stress_grad_rows(x, y, range(12))
    assert np.abs(g.sum(axis=0)).max() < 1e-11 * np.abs(g).sum()
    h = 1e-6
    for a in (0, 5, 11):
        for t in range(5):
            xp, xm = x.copy(), x.copy()
            xp[a, t] += h
            xm[a, t] -= h
            fd = (oracle.stress_loss(xp, y) - oracle.stress_loss(xm, y)) / (2 * h)
            assert fd == pytest.approx(g[a, t], rel=1e-6, abs=1e-8 * np.abs(g).max())


# ---------------------------------------------------------------- inputs

def test_synth_recipes():
    """The generator is SplitMix64: check its first published outputs for
    seed 0 and the ranges of the recipes."""
    z = synth.splitmix64(0, 3)
    assert [int(v) for v in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    u = synth.uniform_cube(1000, 3, 10.0, seed=1)
    assert u.dtype == np.float32 and u.min() >= 0 and u.max() < 10.0
    g = synth.normal(4096, 4, seed=2).astype(np.float64)
    assert abs(g.mean()) < 0.02 and abs(g.std() - 1) < 0.02
    assert len(set(synth.sample_indices(64, 4096, seed=3).tolist())) == 64


def test_stress_moment_identity(oracle):
    """Squared distances are quadratic in the coordinates, so the stress loss
    and its gradient have closed forms over moment matrices: with S = x + y,
    Delta = x - y, a_i = S_i . Delta_i and r_ij = a_i + a_j - S_i.Delta_j -
    Delta_i.S_j,  sum_j r_ij = n a_i + sum a - S_i.sum(Delta) - Delta_i.sum(S)
    and sum_j r_ij x_j = a_i sum(x) + a^T x - S_i (Delta^T x) - Delta_i (S^T x);
    L = (1/2) sum_ij r_ij^2 expands the same way.  None of this is the
    oracle's pairwise loop."""
    x = synth.normal(70, 5, seed=51).astype(np.float64)
    y = synth.perturbed(x.astype(np.float32), 0.2, seed=52).astype(np.float64)
    n = len(x)
    S, De = x + y, x - y
    a = (S * De).sum(1)
    rs = n * a + a.sum() - S @ De.sum(0) - De @ S.sum(0)
    rx = np.outer(a, x.sum(0)) + a @ x - S @ (De.T @ x) - De @ (S.T @ x)
    grad = 4 * (x * rs[:, None] - rx)
    assert np.allclose(oracle.stress_grad_rows(x, y, range(n)), grad, rtol=1e-9, atol=1e-9 * np.abs(grad).max())
    # L via the Gram matrices of the stacked factors U = [a, 1, S, Delta], V = [1, a, -Delta, -S]
    U = np.hstack([a[:, None], np.ones((n, 1)), S, De])
    V = np.hstack([np.ones((n, 1)), a[:, None], -De, -S])
    L = 0.5 * np.sum((U.T @ U) * (V.T @ V))   # sum_ij (U_i . V_j)^2
    assert oracle.stress_loss(x, y) == pytest.approx(L, rel=1e-10)
    # the helper the GPU tests use at full size is this same identity
    from helpers import stress_moments
    Lh, gh = stress_moments(x, y)
    assert Lh == pytest.approx(L, rel=1e-12)
    assert np.allclose(gh, grad, rtol=1e-12, atol=1e-12 * np.abs(grad).max())


def test_atm_energy_grad_slice(oracle):
    """The slice [i_lo, i_hi) of the outer loop: its gradient is the FD
    gradient of its own energy (a different function of x than the total),
    and slices partition the total energy and gradient."""
    x = synth.uniform_cube(14, 3, 2.5, seed=16).astype(np.float64)
    e, g = oracle.atm_energy_grad_slice(x, 3, 9)
    h = 1e-5
    for a in (0, 3, 8, 13):
        for t in range(3):
            xp, xm = x.copy(), x.copy()
            xp[a, t] += h
            xm[a, t] -= h
            fd = (oracle.atm_energy_grad_slice(xp, 3, 9)[0] - oracle.atm_energy_grad_slice(xm, 3, 9)[0]) / (2 * h)
            assert fd == pytest.approx(g[a, t], rel=1e-6, abs=1e-9 * np.abs(g).max())
    e0, g0 = oracle.atm_energy_grad_slice(x, 0, 3)
    e2, g2 = oracle.atm_energy_grad_slice(x, 9, 14)
    assert e0 + e + e2 == pytest.approx(oracle.atm_energy(x), rel=1e-12)
    assert np.allclose(g0 + g + g2, oracle.atm_grad(x), rtol=1e-11, atol=1e-13 * np.abs(g).max())


def test_stress_loss_rows(oracle):
    """Row slices of the loss: the two-point closed form on the one row that
    holds a pair, and slices that add up to the moment-matrix form of L
    (O(n d^2), no pairwise loop)."""
    from helpers import stress_moments
    x = np.array([[0.0, 1.0], [2.0, -1.0]])
    y = np.array([[0.5, 0.0], [1.0, 1.0]])
    assert oracle.stress_loss_rows(x, y, 0, 1) == 0.0
    assert oracle.stress_loss_rows(x, y, 1, 2) == (8.0 - 1.25) ** 2
    a = synth.normal(90, 5, seed=17).astype(np.float64)
    b = synth.perturbed(a, 0.2, seed=18).astype(np.float64)
    parts = oracle.stress_loss_rows(a, b, 0, 31) + oracle.stress_loss_rows(a, b, 31, 90)
    assert parts == pytest.approx(stress_moments(a, b)[0], rel=1e-11)
