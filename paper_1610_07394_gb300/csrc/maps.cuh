// maps.cuh -- block-space maps from a CUDA grid onto discrete orthogonal
// simplices, evaluated in registers at the start of a block.
//
// Paper: Navarro, Bustos, Hitschfeld, "Possibilities of Recursive GPU Mapping
// for Discrete Orthogonal Simplices" (arXiv 1610.07394).
//
//  * lambda, m = 2 (Sec. III-A, eq. (map2d)): grid (p/2) x p for p = 2^k
//    blocks per side.  For w_y >= 1, b = 2^floor(log2 w_y) and
//    q = floor(w_x / b); the block goes to (w_x + q b, w_y + 2 q b), i.e.
//    (column X, row Y) with X < Y.  floor(log2 y) is (32 - 1) - clz(y) and
//    2^floor(log2 y) is 1 << that (the paper's printed bit formulas are off by
//    one; these are the exact forms).  Grid row 0 is not part of the
//    recursive set; this library gives block w_x of that row the two
//    diagonal blocks 2 w_x and 2 w_x + 1.
//  * lambda, m = 3 (Sec. III-C, "Alternative Map for 3-Simplices"): grid
//    (p/2) x (p/2) x (p/2 + p/4 + 2).  z < p/2 is the main cube of the
//    two-branch recursive set; p/2 <= z < 3p/4 holds the cubes of the
//    recursive halves, level b = 2^floor(log2 w_y) in grid rows [b, 2b),
//    sub-problem q = floor(w_x / b) at data offset 2 q b, cube depth b.  A
//    cube of side h at offset off sends its local point (s, u, v) to
//    (off+u, off+s, off+h+v) when u <= s (the paper's "inside" case) and to
//    (off+v, off+h+s, off+h+u) otherwise (its reflected case), covering the
//    blocks I <= J < K.  The last two z-layers form a (p/2) x p grid that the
//    m = 2 map sends onto the plane J = K (left out of the recursive set).
//  * bounding box (Sec. I): the identity, blocks outside the simplex exit.
//  * linear (Sec. I, enumeration map g; the root-based block maps of the
//    authors' earlier work, Sec. II): a 1-D grid over the row-major
//    enumeration, inverted with sqrtf / cbrtf and then fixed up exactly in
//    integer arithmetic.
//  * lambda, m = 4 (Sec. III-D: the recursive set with r = 1/2, beta = 2,
//    V(S_n^4) = (n^4 - n)/14; the paper gives the set and its volume, not a
//    map): the blocks I <= J <= K < L split at half size h into L L L L and
//    H H H H (the two recursive copies) and the cross terms, which one h^4
//    orthotope covers with idle points (ortho4).  Grid (p/2)^3 x (p/2 + p/8):
//    w < p/2 is the top orthotope; the orthotopes of the recursive levels
//    sit in grid rows y in [b, 2b) (b = 2^floor(log2 y), sub-problem
//    q = floor(x / b) at data offset 2 q b, as for m = 2 and 3) with their
//    last two coordinates (u, v) stored as m = u b + v in z + (w - p/2) p/2.
//    The plane K = L is the 3-simplex {I <= J <= K} and takes the m = 3 map.
//  * rectangular box, m = 2 only (Sec. II: the RB strategy for packed
//    triangular matrices, applied to the parallel space): the lower triangle
//    of nb blocks per side is cut at half height h = floor(nb / 2) and its top
//    rows are laid after the bottom ones, grid row k holding triangle row
//    h + k (columns 0 .. h + k) and then row h - 1 - k (columns
//    0 .. h - 1 - k): a grid of (nb + 1 - nb mod 2) x ceil(nb / 2) blocks,
//    exactly the triangle's nb (nb + 1) / 2 for every nb, decoded with one
//    comparison.
//
// Every function is __host__ __device__ so the host-side decode table can be
// compared against an independent construction without a GPU.
#pragma once
#include <cstdint>
#include <cmath>

#if defined(__CUDACC__)
#define SX_HD __host__ __device__ __forceinline__
#else
#define SX_HD inline
#endif

namespace sx {

enum MapKind { MAP_LAMBDA = 0, MAP_BBOX = 1, MAP_LINEAR = 2, MAP_RB = 3 };

// floor(log2 v) for v >= 1: (word bits - 1) - clz(v).
SX_HD int floor_log2(uint32_t v) {
#if defined(__CUDA_ARCH__)
    return 31 - __clz(v);
#else
    return 31 - __builtin_clz(v);
#endif
}

// The power of two p >= max(v, 2) the recursive maps are built on.
SX_HD int64_t pow2_at_least(int64_t v) {
    int64_t p = 2;
    while (p < v) p <<= 1;
    return p;
}

// Up to two data blocks of a 2-simplex (x = column block, y = row block,
// x <= y); `pair` marks the diagonal pair of grid row 0 of the lambda map,
// whose blocks are d0 = 2 w_x and d1 = 2 w_x + 1 (before filtering).
struct List2 {
    int cnt;
    int x[2], y[2];
    bool pair;
    int d0, d1;
};

// Up to two data blocks of a 3-simplex (i <= j <= k).
struct List3 {
    int cnt;
    int i[2], j[2], k[2];
    bool pair;
};

SX_HD void push2(List2 &L, int x, int y, int nb) {
    if (y < nb) { L.x[L.cnt] = x; L.y[L.cnt] = y; ++L.cnt; }
}

SX_HD void push3(List3 &L, int i, int j, int k, int nb) {
    if (k < nb) { L.i[L.cnt] = i; L.j[L.cnt] = j; L.k[L.cnt] = k; ++L.cnt; }
}

// ---------------------------------------------------------------- m = 2

SX_HD List2 decode2_lambda(uint32_t wx, uint32_t wy, int nb) {
    List2 L;
    L.cnt = 0; L.pair = false; L.d0 = L.d1 = -1;
    L.x[0] = L.x[1] = L.y[0] = L.y[1] = 0;
    if (wy == 0) {
        // the diagonal pair (d0, d0), (d1, d1) with d1 = d0 + 1, each kept if
        // below nb: the kept ones are a prefix, so the list is written with
        // constant indices (a data-dependent index would put it in local memory)
        L.pair = true;
        L.d0 = (int)(2 * wx);
        L.d1 = (int)(2 * wx + 1);
        L.x[0] = L.y[0] = L.d0;
        L.x[1] = L.y[1] = L.d1;
        L.cnt = (L.d0 < nb ? 1 : 0) + (L.d1 < nb ? 1 : 0);
        return L;
    }
    const int l = floor_log2(wy);        // recursion level: b = 2^l
    const uint32_t q = wx >> l;          // which square of that level
    push2(L, (int)(wx + (q << l)), (int)(wy + (q << (l + 1))), nb);
    return L;
}

SX_HD List2 decode2_bbox(uint32_t wx, uint32_t wy, int nb) {
    List2 L;
    L.cnt = 0; L.pair = false; L.d0 = L.d1 = -1;
    if (wx <= wy) push2(L, (int)wx, (int)wy, nb);
    return L;
}

// Row-major enumeration of {x <= y}: l = y(y+1)/2 + x.
SX_HD void tri_root(int64_t l, int64_t &y, int64_t &x) {
    float f = sqrtf(8.0f * (float)l + 1.0f);
    int64_t r = (int64_t)((f - 1.0f) * 0.5f);
    if (r < 0) r = 0;
    while (r > 0 && r * (r + 1) / 2 > l) --r;
    while ((r + 1) * (r + 2) / 2 <= l) ++r;
    y = r;
    x = l - r * (r + 1) / 2;
}

SX_HD List2 decode2_linear(int64_t l, int nb) {
    List2 L;
    L.cnt = 0; L.pair = false; L.d0 = L.d1 = -1;
    int64_t y, x;
    tri_root(l, y, x);
    push2(L, (int)x, (int)y, nb);
    return L;
}

// Rectangular box: grid row wy holds triangle row h + wy, then row h - 1 - wy.
SX_HD List2 decode2_rb(uint32_t wx, uint32_t wy, int nb) {
    List2 L;
    L.cnt = 0; L.pair = false; L.d0 = L.d1 = -1;
    const int h = nb >> 1, yb = h + (int)wy;
    if ((int)wx <= yb) push2(L, (int)wx, yb, nb);
    else push2(L, (int)wx - yb - 1, h - 1 - (int)wy, nb);
    return L;
}

// ---------------------------------------------------------------- m = 3

SX_HD void cube3(List3 &L, int h, int off, int s, int u, int v, int nb) {
    if (u <= s) push3(L, off + u, off + s, off + h + v, nb);
    else push3(L, off + v, off + h + s, off + h + u, nb);
}

SX_HD List3 decode3_lambda(uint32_t wx, uint32_t wy, uint32_t wz, int p, int nb) {
    List3 L;
    L.cnt = 0; L.pair = false;
    const uint32_t h0 = (uint32_t)p >> 1, q4 = (uint32_t)p >> 2;
    if (wz < h0) {                       // main cube, h(w) = w + (0, n/2, 0)
        cube3(L, (int)h0, 0, (int)wx, (int)wy, (int)wz, nb);
    } else if (wz < h0 + q4) {           // cubes of the recursive halves
        if (wy == 0) return L;
        const int l = floor_log2(wy);
        const uint32_t b = 1u << l, z = wz - h0;
        if (z >= b) return L;
        const uint32_t q = wx >> l;
        cube3(L, (int)b, (int)(q << (l + 1)), (int)(wx - (q << l)), (int)(wy - b), (int)z, nb);
    } else {                             // plane J = K via the m = 2 map
        const uint32_t wy2 = wy + (wz - h0 - q4) * h0;
        List2 P = decode2_lambda(wx, wy2, nb);
        L.pair = P.pair;
        for (int t = 0; t < P.cnt; ++t) push3(L, P.x[t], P.y[t], P.y[t], nb);
    }
    return L;
}

SX_HD List3 decode3_bbox(uint32_t wx, uint32_t wy, uint32_t wz, int nb) {
    List3 L;
    L.cnt = 0; L.pair = false;
    if (wx <= wy && wy <= wz) push3(L, (int)wx, (int)wy, (int)wz, nb);
    return L;
}

SX_HD int64_t tet(int64_t k) { return k * (k + 1) * (k + 2) / 6; }

// Row-major enumeration of {i <= j <= k}: l = k(k+1)(k+2)/6 + j(j+1)/2 + i.
SX_HD List3 decode3_linear(int64_t l, int nb) {
    List3 L;
    L.cnt = 0; L.pair = false;
    float f = cbrtf(6.0f * (float)l);
    int64_t k = (int64_t)f - 1;
    if (k < 0) k = 0;
    while (k > 0 && tet(k) > l) --k;
    while (tet(k + 1) <= l) ++k;
    int64_t j, i;
    tri_root(l - tet(k), j, i);
    push3(L, (int)i, (int)j, (int)k, nb);
    return L;
}

// ---------------------------------------------------------------- m = 4

// A data block (I, J, K, L) of the 4-simplex of blocks, or none (ok false).
struct Blk4 {
    int i, j, k, l;
    bool ok;
};

// The orthotope of one level: local point (a, b, c, d) in [0, h)^4 to the
// cross terms {x1 <= x2 <= x3 < x4 : x1 < h <= x4} over [0, 2h) at data
// offset off, or none.  Fold (a, b) and (c, d) each into a pair "a <= b" or
// "b < a" (and likewise for c, d); then
//   a <= b, d <  c:                      L L H H  (a, b, h+d, h+c)
//   a <= b, c <= d, b <= c:               L L L H  (a, b, c, h+d), x4' >= x3
//   a <= b, c <= d, a <= c, d < b:        L H H H  (a, h+c, h+d, h+b), x1 <= x2'
//   b <  a, c <= d, d <= a:               L L L H  (c, d, a, h+b), x4' < x3
//   b <  a, d <  c, b <= d:               L H H H  (a, h+b, h+d, h+c), x2' < x1
// and every other point is idle.  The five images are disjoint and their
// union is all cross terms (checked against an enumeration of the cross
// terms by the oracle).
SX_HD Blk4 ortho4(int h, int off, int a, int b, int c, int d, int nb) {
    Blk4 B;
    B.ok = false; B.i = B.j = B.k = B.l = -1;
    int x1, x2, x3, x4;
    if (a <= b) {
        if (d < c) { x1 = a; x2 = b; x3 = h + d; x4 = h + c; }
        else if (b <= c) { x1 = a; x2 = b; x3 = c; x4 = h + d; }
        else if (a <= c && d < b) { x1 = a; x2 = h + c; x3 = h + d; x4 = h + b; }
        else return B;
    } else {
        if (c <= d) {
            if (d > a) return B;
            x1 = c; x2 = d; x3 = a; x4 = h + b;
        } else {
            if (b > d) return B;
            x1 = a; x2 = h + b; x3 = h + d; x4 = h + c;
        }
    }
    if (off + x4 >= nb) return B;
    B.i = off + x1; B.j = off + x2; B.k = off + x3; B.l = off + x4;
    B.ok = true;
    return B;
}

// Depth of the grid's slab (w >= p/2) that holds the recursive levels: the
// largest level (b = p/4) stores b^2 = p^2/16 points (u, v) in rows of p/2.
SX_HD int slab4(int64_t p) { return p >= 8 ? (int)(p / 8) : (p == 4 ? 1 : 0); }

SX_HD Blk4 decode4_lambda(uint32_t x, uint32_t y, uint32_t z, uint32_t w, int p, int nb) {
    const uint32_t h0 = (uint32_t)p >> 1;
    if (w < h0) return ortho4((int)h0, 0, (int)x, (int)y, (int)z, (int)w, nb);
    Blk4 B;
    B.ok = false; B.i = B.j = B.k = B.l = -1;
    if (y == 0) return B;
    const int l = floor_log2(y);            // level: orthotope side b = 2^l
    const uint32_t b = 1u << l;
    const uint32_t m = (w - h0) * h0 + z;   // (u, v) of the level's orthotope
    if (m >= b * b) return B;
    const uint32_t q = x >> l;              // sub-problem of the level
    return ortho4((int)b, (int)(q << (l + 1)), (int)(x - (q << l)), (int)(y - b), (int)(m >> l),
                  (int)(m & (b - 1)), nb);
}

SX_HD Blk4 decode4_bbox(uint32_t x, uint32_t y, uint32_t z, uint32_t w, int nb) {
    Blk4 B;
    B.ok = x <= y && y <= z && z <= w && (int)w < nb;
    B.i = B.ok ? (int)x : -1; B.j = B.ok ? (int)y : -1;
    B.k = B.ok ? (int)z : -1; B.l = B.ok ? (int)w : -1;
    return B;
}

// ---------------------------------------------------------------- grids

struct Grid { int64_t gx, gy, gz; int p; };

SX_HD Grid grid2(int64_t nb, int map) {
    Grid g; g.gz = 1; g.p = 0;
    if (map == MAP_LAMBDA) {
        int64_t p = pow2_at_least(nb);
        g.p = (int)p; g.gx = p / 2; g.gy = p;
    } else if (map == MAP_BBOX) {
        g.gx = nb; g.gy = nb;
    } else if (map == MAP_RB) {
        g.gx = nb + 1 - (nb & 1); g.gy = (nb + 1) / 2;
    } else {
        g.gx = nb * (nb + 1) / 2; g.gy = 1;
    }
    return g;
}

SX_HD Grid grid3(int64_t nb, int map) {
    Grid g; g.p = 0;
    if (map == MAP_LAMBDA) {
        int64_t p = pow2_at_least(nb);
        g.p = (int)p; g.gx = p / 2; g.gy = p / 2; g.gz = p / 2 + p / 4 + 2;
    } else if (map == MAP_BBOX) {
        g.gx = nb; g.gy = nb; g.gz = nb;
    } else if (map == MAP_RB) {
        g.gx = 0; g.gy = 0; g.gz = 0;   // no 3-simplex form (callers reject it)
    } else {
        g.gx = nb * (nb + 1) * (nb + 2) / 6; g.gy = 1; g.gz = 1;
    }
    return g;
}

// 4-D grid of the m = 4 maps (x fastest, then y, z, w).  LAMBDA: the blocks
// I <= J <= K < L only (the plane K = L takes grid3); BBOX: nb^4, all of
// I <= J <= K <= L.
struct Grid4 { int64_t gx, gy, gz, gw; int p; };

SX_HD Grid4 grid4(int64_t nb, int map) {
    Grid4 g; g.p = 0;
    if (map == MAP_LAMBDA) {
        int64_t p = pow2_at_least(nb);
        g.p = (int)p; g.gx = g.gy = g.gz = p / 2; g.gw = p / 2 + slab4(p);
    } else {
        g.gx = g.gy = g.gz = g.gw = nb;
    }
    return g;
}

// Decode of grid block (wx, wy, wz) for a map chosen at compile time.
template <int MAP>
SX_HD List2 decode2(uint32_t wx, uint32_t wy, int nb) {
    if (MAP == MAP_LAMBDA) return decode2_lambda(wx, wy, nb);
    if (MAP == MAP_BBOX) return decode2_bbox(wx, wy, nb);
    if (MAP == MAP_RB) return decode2_rb(wx, wy, nb);
    return decode2_linear((int64_t)wx, nb);
}

template <int MAP>
SX_HD List3 decode3(uint32_t wx, uint32_t wy, uint32_t wz, int p, int nb) {
    if (MAP == MAP_LAMBDA) return decode3_lambda(wx, wy, wz, p, nb);
    if (MAP == MAP_BBOX) return decode3_bbox(wx, wy, wz, nb);
    return decode3_linear((int64_t)wx, nb);
}

}  // namespace sx
