/*
 * oracle.c -- plain, slow, FP64 CPU oracle for the simplex-domain hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant with the CUDA library; neither includes the other.
 *
 * Paper: C. A. Navarro, B. Bustos, N. Hitschfeld, "Possibilities of Recursive
 * GPU Mapping for Discrete Orthogonal Simplices" (arXiv 1610.07394).
 *
 * What is here, each written from its definition:
 *   - block-space map tables built by *recursive construction* of the sets
 *     S_n^2 (Sec. III-A, Eq. 5-9) and the two-branch S_n^3 (Sec. III-C,
 *     "Alternative Map for 3-Simplices"), the r = 1/2, beta = 2 set S_n^4
 *     (Sec. III-D, built from its cross terms), the bounding box (Sec. I, f(x)=x),
 *     the linear enumeration g (Sec. I, Eq. 2 expanded) and, for m = 2, the
 *     rectangular box (Sec. II: the RB strategy for packed triangular
 *     matrices, applied to the parallel space) laid out row by row;
 *   - thread-level coverage counts over the discrete orthogonal simplices
 *     Delta_n^2, Delta_n^3 and Delta_n^4 (Eq. 1-2, volumes of Sec. III-A /
 *     III-B / III-D);
 *   - the packed Euclidean distance matrix (Sec. I: EDM as a 2-simplex
 *     problem), the Axilrod-Teller-Muto triple-dipole energy and its
 *     gradient (Sec. I: triple-interaction n-body as a 3-simplex problem),
 *     and a stress loss over the packed EDM with its gradient.
 *
 * Conventions (the readings the library documents as well):
 *   - n points; a block is a tile of rho consecutive points; nb = ceil(n/rho).
 *   - 2-simplex: pairs (i, j) with j <= i < n ("row i, column j"), packed
 *     row-major lower: idx = i(i+1)/2 + j.  Blocks (X, Y) = (column, row).
 *   - 3-simplex: triples i <= j <= k < n, packed
 *     idx = k(k+1)(k+2)/6 + j(j+1)/2 + i.  Blocks (I, J, K).
 *   - Map tables: for every grid block w, a list of up to two data blocks;
 *     m=2 entries are (X0,Y0,X1,Y1), m=3 entries (I0,J0,K0,I1,J1,K1), m=4
 *     entries (I,J,K,L,-1,-1,-1,-1); unused
 *     slots are -1; a data block with any coordinate >= nb is dropped.
 * All floating point is double; the build disables FP contraction so the
 * results are the same on every host.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { MAP_LAMBDA = 0, MAP_BBOX = 1, MAP_LINEAR = 2, MAP_RB = 3 };

static int64_t pow2_at_least(int64_t v)
{
    int64_t p = 2;
    while (p < v) p *= 2;
    return p;
}

/* ======================= 2-simplex tables ======================= */

/* Grid shape of each 2-simplex map, in blocks. */
int64_t oracle_grid2(int64_t nb, int map, int64_t *gx, int64_t *gy)
{
    if (map == MAP_LAMBDA) {
        int64_t p = pow2_at_least(nb);
        *gx = p / 2; *gy = p;
    } else if (map == MAP_BBOX) {
        *gx = nb; *gy = nb;
    } else if (map == MAP_RB) {
        /* one pair of triangle rows per grid row, each pair nb + 1 (nb
         * even) or nb (nb odd) blocks long */
        *gy = (nb + 1) / 2;
        *gx = (nb % 2 == 0) ? nb + 1 : nb;
    } else {
        *gx = nb * (nb + 1) / 2; *gy = 1;
    }
    return (*gx) * (*gy);
}

static void put2(int32_t *e, int slot, int64_t x, int64_t y, int64_t nb)
{
    if (x >= nb || y >= nb) return;
    /* keep valid blocks first */
    if (slot == 1 && e[0] < 0) slot = 0;
    e[2 * slot] = (int32_t)x;
    e[2 * slot + 1] = (int32_t)y;
}

/*
 * Recursive set S_s^2 (Sec. III-A, Eq. 5): a square of (s/2)^2 blocks plus two
 * copies of S_{s/2}.  S_s placed at data offset `off` covers the blocks
 * {off <= X < Y < off + s}; its square holds rows [off+s/2, off+s) and
 * columns [off, off+s/2).  In the grid, S_s occupies rows [1, s) and the
 * s/2 columns starting at `gc`; its square sits in grid rows [s/2, s), the
 * first child in the left half of the columns, the second in the right half.
 */
static void lam2_place(int64_t s, int64_t gc, int64_t off, int64_t gx,
                       int64_t nb, int32_t *tab)
{
    if (s < 2) return;
    int64_t h = s / 2;
    for (int64_t wy = h; wy < s; ++wy)
        for (int64_t wx = gc; wx < gc + h; ++wx)
            put2(tab + 4 * (wy * gx + wx), 0, off + (wx - gc), off + h + (wy - h), nb);
    lam2_place(h, gc, off, gx, nb, tab);
    lam2_place(h, gc + h / 2, off + h, gx, nb, tab);
}

/* Map table of a 2-simplex map over nb blocks; tab has grid*4 int32. */
int64_t oracle_table2(int64_t nb, int map, int32_t *tab)
{
    int64_t gx, gy;
    int64_t g = oracle_grid2(nb, map, &gx, &gy);
    for (int64_t t = 0; t < 4 * g; ++t) tab[t] = -1;
    if (map == MAP_LAMBDA) {
        lam2_place(gy, 0, 0, gx, nb, tab);
        /* grid row 0 is not part of S (Sec. III-A: the diagonal is left out);
         * the reading used here gives block wx of that row the diagonal
         * blocks 2wx and 2wx+1. */
        for (int64_t wx = 0; wx < gx; ++wx) {
            put2(tab + 4 * wx, 0, 2 * wx, 2 * wx, nb);
            put2(tab + 4 * wx, 1, 2 * wx + 1, 2 * wx + 1, nb);
        }
    } else if (map == MAP_BBOX) {
        for (int64_t wy = 0; wy < gy; ++wy)
            for (int64_t wx = 0; wx <= wy; ++wx)
                put2(tab + 4 * (wy * gx + wx), 0, wx, wy, nb);
    } else if (map == MAP_RB) {
        /* Rectangular box: cut the block triangle (rows y = 0 .. nb-1, row y
         * holding columns 0 .. y) at half height, h = floor(nb/2).  Grid row
         * k is filled left to right with the blocks of triangle row h + k and
         * then, where that row is shorter than the grid, with the blocks of
         * triangle row h - 1 - k. */
        int64_t h = nb / 2;
        for (int64_t k = 0; k < gy; ++k) {
            int64_t w = k * gx;
            for (int64_t x = 0; x <= h + k; ++x) put2(tab + 4 * (w++), 0, x, h + k, nb);
            if (h - 1 - k >= 0)
                for (int64_t x = 0; x <= h - 1 - k; ++x) put2(tab + 4 * (w++), 0, x, h - 1 - k, nb);
        }
    } else {
        /* linear enumeration of the lower block triangle, row by row */
        int64_t l = 0;
        for (int64_t y = 0; y < nb; ++y)
            for (int64_t x = 0; x <= y; ++x)
                put2(tab + 4 * (l++), 0, x, y, nb);
    }
    return g;
}

/* ======================= 3-simplex tables ======================= */

int64_t oracle_grid3(int64_t nb, int map, int64_t *gx, int64_t *gy, int64_t *gz)
{
    if (map == MAP_LAMBDA) {
        int64_t p = pow2_at_least(nb);
        *gx = p / 2; *gy = p / 2; *gz = p / 2 + p / 4 + 2;
    } else if (map == MAP_BBOX) {
        *gx = nb; *gy = nb; *gz = nb;
    } else {
        *gx = nb * (nb + 1) * (nb + 2) / 6; *gy = 1; *gz = 1;
    }
    return (*gx) * (*gy) * (*gz);
}

static void put3(int32_t *e, int slot, int64_t i, int64_t j, int64_t k, int64_t nb)
{
    if (i >= nb || j >= nb || k >= nb) return;
    if (slot == 1 && e[0] < 0) slot = 0;
    e[3 * slot] = (int32_t)i;
    e[3 * slot + 1] = (int32_t)j;
    e[3 * slot + 2] = (int32_t)k;
}

/*
 * Two-branch recursive set S_s^3 (Sec. III-C): V(S_s) = (s/2)^3 + 2 V(S_{s/2}),
 * = V(Delta_{s-1}^3), so S_s covers the blocks {off <= I <= J < K < off+s}
 * (the plane J = K is left out, as the paper states).  Split the index range
 * into a low half L and a high half H (each h = s/2 blocks): the triples
 * with I, J, K in L L L and H H H are the two recursive copies; the rest,
 * L L H and L H H, hold h^2(h+1)/2 + h^2(h-1)/2 = h^3 blocks and are the
 * main cube.  The cube's local point (x, u, v) goes to L L H when u <= x
 * ("inside" in the paper) and to L H H otherwise (the paper's reflected
 * "diagonal or outside" case).
 *
 * Placement in the grid (Sec. III-C, h(w) = w + (0, n/2, 0) and the shared
 * parameters b, q of the 2-simplex map): the top cube fills grid z in
 * [0, p/2); the cube of a sub-problem of size s < p at offset off fills
 * grid x in [off/2, off/2 + s/2), y in [s/2, s), z in [p/2, p/2 + s/2).
 */
static void lam3_place(int64_t s, int64_t off, int64_t p, int64_t nb, int32_t *tab)
{
    if (s < 2) return;
    int64_t h = s / 2, gx = p / 2, gy = p / 2;
    for (int64_t v = 0; v < h; ++v)
        for (int64_t u = 0; u < h; ++u)
            for (int64_t x = 0; x < h; ++x) {
                int64_t wx, wy, wz;
                if (s == p) { wx = x; wy = u; wz = v; }
                else { wx = off / 2 + x; wy = h + u; wz = p / 2 + v; }
                int32_t *e = tab + 6 * ((wz * gy + wy) * gx + wx);
                if (u <= x) put3(e, 0, off + u, off + x, off + h + v, nb);
                else put3(e, 0, off + v, off + h + x, off + h + u, nb);
            }
    lam3_place(h, off, p, nb, tab);
    lam3_place(h, off + h, p, nb, tab);
}

/* Map table of a 3-simplex map over nb blocks; tab has grid*6 int32. */
int64_t oracle_table3(int64_t nb, int map, int32_t *tab)
{
    int64_t gx, gy, gz;
    int64_t g = oracle_grid3(nb, map, &gx, &gy, &gz);
    for (int64_t t = 0; t < 6 * g; ++t) tab[t] = -1;
    if (map == MAP_LAMBDA) {
        int64_t p = pow2_at_least(nb);
        lam3_place(p, 0, p, nb, tab);
        /* The plane J = K (left out of S) is a 2-simplex of blocks {I <= J};
         * the last two grid z-layers together have (p/2) x p blocks, the
         * shape of the 2-simplex grid, and take the 2-simplex map. */
        int64_t g2x, g2y;
        oracle_grid2(nb, MAP_LAMBDA, &g2x, &g2y);
        int32_t *t2 = (int32_t *)malloc(sizeof(int32_t) * 4 * g2x * g2y);
        oracle_table2(nb, MAP_LAMBDA, t2);
        for (int64_t z = 0; z < 2; ++z)
            for (int64_t wy = 0; wy < gy; ++wy)
                for (int64_t wx = 0; wx < gx; ++wx) {
                    int64_t w2 = (wy + z * gy) * g2x + wx;
                    int32_t *e = tab + 6 * (((gz - 2 + z) * gy + wy) * gx + wx);
                    for (int s = 0; s < 2; ++s)
                        if (t2[4 * w2 + 2 * s] >= 0)
                            put3(e, s, t2[4 * w2 + 2 * s], t2[4 * w2 + 2 * s + 1],
                                 t2[4 * w2 + 2 * s + 1], nb);
                }
        free(t2);
    } else if (map == MAP_BBOX) {
        for (int64_t wz = 0; wz < gz; ++wz)
            for (int64_t wy = 0; wy <= wz; ++wy)
                for (int64_t wx = 0; wx <= wy; ++wx)
                    put3(tab + 6 * ((wz * gy + wy) * gx + wx), 0, wx, wy, wz, nb);
    } else {
        int64_t l = 0;
        for (int64_t k = 0; k < nb; ++k)
            for (int64_t j = 0; j <= k; ++j)
                for (int64_t i = 0; i <= j; ++i)
                    put3(tab + 6 * (l++), 0, i, j, k, nb);
    }
    return g;
}

/* ======================= 4-simplex tables ======================= */

/*
 * Recursive set S_s^4 with r = 1/2, beta = 2 (Sec. III-D): V(S_s) =
 * (s/2)^4 + 2 V(S_{s/2}) = (s^4 - s)/14.  It holds the blocks
 * {off <= I <= J <= K < L < off+s} (the hyperplane K = L is a 3-simplex of
 * blocks, covered by the m = 3 set).  Split the index range into halves L
 * and H of h = s/2 blocks: L L L L and H H H H are the two recursive copies;
 * the cross terms (I < off+h <= L) go into one h^4 orthotope, which has room
 * to spare (the paper gives the volume, not the assignment; this is the
 * library's reading, written here in the other direction: from each cross
 * term to its orthotope point).  With local indices x1 <= x2 <= x3 < x4
 * and x' = x - h for an index in H:
 *   L L L H, x4' >= x3: point (x1, x2, x3, x4');
 *   L L L H, x4' <  x3: point (x3, x4', x1, x2);
 *   L L H H:            point (x1, x2, x4', x3');
 *   L H H H, x1 <= x2': point (x1, x4', x2', x3');
 *   L H H H, x1 >  x2': point (x1, x2', x4', x3').
 * Placement in the 4-D grid (x, y, z, w) of shape (p/2)^3 x (p/2 + slab):
 * the top orthotope (s = p) fills w < p/2 with (x, y, z, w) = the point;
 * the orthotope (a, b, c, d) of a sub-problem of size s < p at offset off
 * goes to x = off/2 + a, y = s/2 + b, and m = c s/2 + d to z = m mod p/2,
 * w = p/2 + floor(m / (p/2)) (the shared b, q of the 2-simplex map).
 * Returns 0, or -1 when two cross terms land on one grid point.
 */
static int64_t slab4(int64_t p) { return p >= 8 ? p / 8 : (p == 4 ? 1 : 0); }

int64_t oracle_grid4(int64_t nb, int map, int64_t *gx, int64_t *gy, int64_t *gz, int64_t *gw)
{
    if (map == MAP_LAMBDA) {
        int64_t p = pow2_at_least(nb);
        *gx = p / 2; *gy = p / 2; *gz = p / 2; *gw = p / 2 + slab4(p);
    } else {
        *gx = nb; *gy = nb; *gz = nb; *gw = nb;
    }
    return (*gx) * (*gy) * (*gz) * (*gw);
}

static int lam4_place(int64_t s, int64_t off, int64_t p, int64_t nb, int32_t *tab)
{
    if (s < 2) return 0;
    int64_t h = s / 2, g = p / 2;
    for (int64_t x4 = h; x4 < s; ++x4)
        for (int64_t x3 = 0; x3 < x4; ++x3)
            for (int64_t x2 = 0; x2 <= x3; ++x2)
                for (int64_t x1 = 0; x1 <= x2 && x1 < h; ++x1) {
                    int64_t a, b, c, d;
                    if (x3 < h) {                       /* L L L H */
                        if (x4 - h >= x3) { a = x1; b = x2; c = x3; d = x4 - h; }
                        else { a = x3; b = x4 - h; c = x1; d = x2; }
                    } else if (x2 < h) {                /* L L H H */
                        a = x1; b = x2; c = x4 - h; d = x3 - h;
                    } else if (x1 <= x2 - h) {          /* L H H H */
                        a = x1; b = x4 - h; c = x2 - h; d = x3 - h;
                    } else {
                        a = x1; b = x2 - h; c = x4 - h; d = x3 - h;
                    }
                    int64_t wx, wy, wz, ww;
                    if (s == p) { wx = a; wy = b; wz = c; ww = d; }
                    else {
                        int64_t m = c * h + d;
                        wx = off / 2 + a; wy = h + b; wz = m % g; ww = g + m / g;
                    }
                    int32_t *e = tab + 8 * (((ww * g + wz) * g + wy) * g + wx);
                    if (off + x4 >= nb) continue;    /* past the last block: dropped */
                    if (e[0] >= 0) return -1;
                    e[0] = (int32_t)(off + x1); e[1] = (int32_t)(off + x2);
                    e[2] = (int32_t)(off + x3); e[3] = (int32_t)(off + x4);
                }
    if (lam4_place(h, off, p, nb, tab)) return -1;
    return lam4_place(h, off + h, p, nb, tab);
}

/* Map table of a 4-simplex map over nb blocks; tab has grid*8 int32
 * (I, J, K, L, then four unused -1).  LAMBDA: the blocks I <= J <= K < L
 * (the plane K = L takes the 3-simplex map); BBOX: every I <= J <= K <= L.
 * Returns the grid size, or -1 if the lambda placement collides. */
int64_t oracle_table4(int64_t nb, int map, int32_t *tab)
{
    int64_t gx, gy, gz, gw;
    int64_t g = oracle_grid4(nb, map, &gx, &gy, &gz, &gw);
    for (int64_t t = 0; t < 8 * g; ++t) tab[t] = -1;
    if (map == MAP_LAMBDA) {
        int64_t p = pow2_at_least(nb);
        if (lam4_place(p, 0, p, nb, tab)) return -1;
    } else {
        for (int64_t l = 0; l < nb; ++l)
            for (int64_t k = 0; k <= l; ++k)
                for (int64_t j = 0; j <= k; ++j)
                    for (int64_t i = 0; i <= j; ++i) {
                        int32_t *e = tab + 8 * (((l * gz + k) * gy + j) * gx + i);
                        e[0] = (int32_t)i; e[1] = (int32_t)j; e[2] = (int32_t)k; e[3] = (int32_t)l;
                    }
    }
    return g;
}

/* Volume of the recursive set S_s^4: the orthotope points of every level
 * (mapped or idle), summed over the recursion. */
int64_t oracle_volume4(int64_t s)
{
    if (s < 2) return 0;
    int64_t h = s / 2;
    return h * h * h * h + 2 * oracle_volume4(h);
}

/* ======================= coverage ======================= */

/*
 * Thread-level coverage of Delta_n^2 = {(i, j): 0 <= j <= i < n}.
 * Each grid block has rho*rho threads (r, c).  For a grid block whose list
 * is a single block (X, Y), thread (r, c) takes element (Y*rho + r,
 * X*rho + c), kept when column <= row < n.  For a 2-simplex-map block of grid
 * row 0 (two diagonal blocks D0, D1), the two triangles of rho(rho+1)/2
 * elements are read as one rho x (rho+1) rectangle: cell (r, c) is element
 * (r, c) of D0 when c <= r, else element (rho-1-r, c-r-1) of D1; thread
 * (r, c) takes cell (r, c) and, when c == 0, also cell (r, rho).
 * count[] (n(n+1)/2 int32) must be zeroed by the caller; returns the number
 * of threads that took no element.
 */
int64_t oracle_cover2(int64_t n, int64_t rho, int map, int32_t *count)
{
    int64_t nb = (n + rho - 1) / rho, gx, gy;
    int64_t g = oracle_grid2(nb, map, &gx, &gy);
    int32_t *tab = (int32_t *)malloc(sizeof(int32_t) * 4 * g);
    oracle_table2(nb, map, tab);
    int64_t idle = 0;
    for (int64_t w = 0; w < g; ++w) {
        int32_t *e = tab + 4 * w;
        int diag_pair = (map == MAP_LAMBDA && w < gx);
        for (int64_t r = 0; r < rho; ++r)
            for (int64_t c = 0; c < rho; ++c) {
                int took = 0;
                if (diag_pair) {
                    int64_t d0 = 2 * w, d1 = 2 * w + 1;
                    for (int extra = 0; extra < 2; ++extra) {
                        if (extra && c != 0) break;
                        int64_t cc = extra ? rho : c, i, j;
                        if (cc <= r) { i = d0 * rho + r; j = d0 * rho + cc; }
                        else { i = d1 * rho + (rho - 1 - r); j = d1 * rho + (cc - r - 1); }
                        if (i < n) { count[i * (i + 1) / 2 + j]++; took = 1; }
                    }
                } else if (e[0] >= 0) {
                    int64_t i = (int64_t)e[1] * rho + r, j = (int64_t)e[0] * rho + c;
                    if (j <= i && i < n) { count[i * (i + 1) / 2 + j]++; took = 1; }
                }
                if (!took) ++idle;
            }
    }
    free(tab);
    return idle;
}

/*
 * Thread-level coverage of Delta_n^3 = {(i, j, k): 0 <= i <= j <= k < n}.
 * Each grid block has rho^3 threads (a, b, c); it walks its list of data
 * blocks in order and thread (a, b, c) takes element (I*rho+a, J*rho+b,
 * K*rho+c) of each, kept when i <= j <= k < n.  count[] has
 * n(n+1)(n+2)/6 int32, zeroed by the caller; returns the idle threads.
 */
int64_t oracle_cover3(int64_t n, int64_t rho, int map, int32_t *count)
{
    int64_t nb = (n + rho - 1) / rho, gx, gy, gz;
    int64_t g = oracle_grid3(nb, map, &gx, &gy, &gz);
    int32_t *tab = (int32_t *)malloc(sizeof(int32_t) * 6 * g);
    oracle_table3(nb, map, tab);
    int64_t idle = 0;
    for (int64_t w = 0; w < g; ++w) {
        int32_t *e = tab + 6 * w;
        for (int64_t c = 0; c < rho; ++c)
            for (int64_t b = 0; b < rho; ++b)
                for (int64_t a = 0; a < rho; ++a) {
                    int took = 0;
                    for (int s = 0; s < 2; ++s) {
                        if (e[3 * s] < 0) continue;
                        int64_t i = (int64_t)e[3 * s] * rho + a;
                        int64_t j = (int64_t)e[3 * s + 1] * rho + b;
                        int64_t k = (int64_t)e[3 * s + 2] * rho + c;
                        if (i <= j && j <= k && k < n) {
                            count[k * (k + 1) * (k + 2) / 6 + j * (j + 1) / 2 + i]++;
                            took = 1;
                        }
                    }
                    if (!took) ++idle;
                }
    }
    free(tab);
    return idle;
}

/*
 * Thread-level coverage of Delta_n^4 = {(i, j, k, l): i <= j <= k <= l < n},
 * packed idx = l(l+1)(l+2)(l+3)/24 + k(k+1)(k+2)/6 + j(j+1)/2 + i.  Each
 * grid block has rho^4 threads (a, b, c, d) and takes element (I rho + a,
 * J rho + b, K rho + c, L rho + d), kept when i <= j <= k <= l < n.  LAMBDA
 * walks the 4-simplex table (K < L) and then the 3-simplex lambda table
 * with each block (I, J, K) read as (I, J, K, K); BBOX the nb^4 table.
 * count[] zeroed by the caller; returns the idle threads (-1 on a
 * placement collision).
 */
int64_t oracle_cover4(int64_t n, int64_t rho, int map, int32_t *count)
{
    int64_t nb = (n + rho - 1) / rho, gx, gy, gz, gw;
    int64_t g = oracle_grid4(nb, map, &gx, &gy, &gz, &gw);
    int32_t *tab = (int32_t *)malloc(sizeof(int32_t) * 8 * g);
    if (oracle_table4(nb, map, tab) < 0) { free(tab); return -1; }
    int64_t g3 = 0, hx, hy, hz;
    int32_t *tab3 = NULL;
    if (map == MAP_LAMBDA) {
        g3 = oracle_grid3(nb, MAP_LAMBDA, &hx, &hy, &hz);
        tab3 = (int32_t *)malloc(sizeof(int32_t) * 6 * g3);
        oracle_table3(nb, MAP_LAMBDA, tab3);
    }
    int64_t idle = 0;
    for (int64_t w = 0; w < g + g3; ++w) {
        int64_t blk[2][4];
        int nblk = 0;
        if (w < g) {
            int32_t *e = tab + 8 * w;
            if (e[0] >= 0) { for (int t = 0; t < 4; ++t) blk[0][t] = e[t]; nblk = 1; }
        } else {
            int32_t *e = tab3 + 6 * (w - g);
            for (int s = 0; s < 2; ++s)
                if (e[3 * s] >= 0) {
                    blk[nblk][0] = e[3 * s]; blk[nblk][1] = e[3 * s + 1];
                    blk[nblk][2] = e[3 * s + 2]; blk[nblk][3] = e[3 * s + 2];
                    ++nblk;
                }
        }
        for (int64_t d = 0; d < rho; ++d)
            for (int64_t c = 0; c < rho; ++c)
                for (int64_t b = 0; b < rho; ++b)
                    for (int64_t a = 0; a < rho; ++a) {
                        int took = 0;
                        for (int s = 0; s < nblk; ++s) {
                            int64_t i = blk[s][0] * rho + a, j = blk[s][1] * rho + b;
                            int64_t k = blk[s][2] * rho + c, l = blk[s][3] * rho + d;
                            if (i <= j && j <= k && k <= l && l < n) {
                                count[l * (l + 1) * (l + 2) * (l + 3) / 24 + k * (k + 1) * (k + 2) / 6
                                      + j * (j + 1) / 2 + i]++;
                                took = 1;
                            }
                        }
                        if (!took) ++idle;
                    }
    }
    free(tab);
    free(tab3);
    return idle;
}

/* ======================= EDM ======================= */

/* Squared Euclidean distance of points p and q in d dimensions. */
static double sqdist(const double *p, const double *q, int64_t d)
{
    double s = 0.0;
    for (int64_t t = 0; t < d; ++t) {
        double diff = p[t] - q[t];
        s += diff * diff;
    }
    return s;
}

/* Packed lower EDM of squared distances, out[i(i+1)/2 + j] for j <= i. */
void oracle_edm_packed(int64_t n, int64_t d, const double *x, double *out)
{
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j <= i; ++j)
            out[i * (i + 1) / 2 + j] = sqdist(x + i * d, x + j * d, d);
}

/*
 * The same distances in the tile-packed layout (each 128 x 128 tile of the
 * matrix one contiguous block; the data-side counterpart of the RB packing of
 * Sec. II).  Tiles (I, J), J <= I, follow one another in packed lower order;
 * inside a tile, row a and column b are at a * 128 + b.  A diagonal tile
 * holds its whole square, and rows or columns >= n are 0.
 */
void oracle_edm_tiles(int64_t n, int64_t d, const double *x, double *out)
{
    const int64_t T = 128, nt = (n + T - 1) / T;
    double *tile = out;
    for (int64_t I = 0; I < nt; ++I)
        for (int64_t J = 0; J <= I; ++J) {
            for (int64_t a = 0; a < T; ++a)
                for (int64_t b = 0; b < T; ++b) {
                    int64_t i = I * T + a, j = J * T + b;
                    tile[a * T + b] = (i < n && j < n) ? sqdist(x + i * d, x + j * d, d) : 0.0;
                }
            tile += T * T;
        }
}

/* Squared distances of the listed pairs (i, j). */
void oracle_edm_pairs(int64_t d, const double *x, const int64_t *pairs,
                      int64_t count, double *out)
{
    for (int64_t t = 0; t < count; ++t)
        out[t] = sqdist(x + pairs[2 * t] * d, x + pairs[2 * t + 1] * d, d);
}

/* ======================= ATM triple-dipole ======================= */

/*
 * Axilrod-Teller-Muto term of one triangle (i, j, k):
 *   e = nu (1 + 3 cos g_i cos g_j cos g_k) / (r_ij r_jk r_ki)^3
 * with every squared side softened, r^2 -> r^2 + eps, both in the cosines'
 * norms and in the denominator.  The cosines come from dot products of the
 * edge vectors at each vertex.
 */
static double atm_term(const double *xi, const double *xj, const double *xk,
                       double nu, double eps)
{
    double eij[3], eik[3], ejk[3];
    for (int t = 0; t < 3; ++t) {
        eij[t] = xj[t] - xi[t];
        eik[t] = xk[t] - xi[t];
        ejk[t] = xk[t] - xj[t];
    }
    double sij = eij[0] * eij[0] + eij[1] * eij[1] + eij[2] * eij[2] + eps;
    double sik = eik[0] * eik[0] + eik[1] * eik[1] + eik[2] * eik[2] + eps;
    double sjk = ejk[0] * ejk[0] + ejk[1] * ejk[1] + ejk[2] * ejk[2] + eps;
    double rij = sqrt(sij), rik = sqrt(sik), rjk = sqrt(sjk);
    /* vertex i: edges i->j, i->k; vertex j: j->i, j->k; vertex k: k->i, k->j */
    double ci = (eij[0] * eik[0] + eij[1] * eik[1] + eij[2] * eik[2]) / (rij * rik);
    double cj = (-eij[0] * ejk[0] - eij[1] * ejk[1] - eij[2] * ejk[2]) / (rij * rjk);
    double ck = (eik[0] * ejk[0] + eik[1] * ejk[1] + eik[2] * ejk[2]) / (rik * rjk);
    double r3 = rij * rjk * rik;
    return nu * (1.0 + 3.0 * ci * cj * ck) / (r3 * r3 * r3);
}

/* Total energy: sum over 0 <= i < j < k < n (points are n x 3, row-major). */
double oracle_atm_energy(int64_t n, const double *x, double nu, double eps)
{
    double e = 0.0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j)
            for (int64_t k = j + 1; k < n; ++k)
                e += atm_term(x + 3 * i, x + 3 * j, x + 3 * k, nu, eps);
    return e;
}

/* Energy restricted to triples with i in [i_lo, i_hi) (a slice of the outer
 * loop; used to time a bounded sample of the full sum). */
double oracle_atm_energy_slice(int64_t n, const double *x, double nu, double eps,
                               int64_t i_lo, int64_t i_hi)
{
    double e = 0.0;
    for (int64_t i = i_lo; i < i_hi && i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j)
            for (int64_t k = j + 1; k < n; ++k)
                e += atm_term(x + 3 * i, x + 3 * j, x + 3 * k, nu, eps);
    return e;
}

/* Sum of |e| over all triples (the scale against which rounding of a signed
 * sum is measured). */
double oracle_atm_abs_energy(int64_t n, const double *x, double nu, double eps)
{
    double e = 0.0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j)
            for (int64_t k = j + 1; k < n; ++k)
                e += fabs(atm_term(x + 3 * i, x + 3 * j, x + 3 * k, nu, eps));
    return e;
}

/* Energy of the triples that contain atom `a` (a function of x_a alone when
 * the other atoms are held fixed; its gradient in x_a is dE/dx_a). */
double oracle_atm_atom_energy(int64_t n, const double *x, int64_t a,
                              double nu, double eps)
{
    double e = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        if (j == a) continue;
        for (int64_t k = j + 1; k < n; ++k) {
            if (k == a) continue;
            e += atm_term(x + 3 * a, x + 3 * j, x + 3 * k, nu, eps);
        }
    }
    return e;
}

/*
 * Partial derivatives of one term with respect to its three squared sides.
 * Write A = |x_i-x_j|^2, B = |x_j-x_k|^2, C = |x_k-x_i|^2 (unsoftened) and
 * sA = A + eps etc.  The dot products at the vertices are
 *   Di = (A + C - B)/2,  Dj = (A + B - C)/2,  Dk = (B + C - A)/2,
 * P = sA sB sC, and e = nu (P^{-3/2} + 3 Di Dj Dk P^{-5/2}).  Then
 *   de/dA = nu [ -3/2 P^{-3/2}/sA + 3 (dD/dA) P^{-5/2} - 15/2 D P^{-5/2}/sA ]
 * with D = Di Dj Dk and dD/dA = (Dj Dk + Di Dk - Di Dj)/2; B and C follow
 * by the symmetric rules dD/dB = (Di Dk + Di Dj - Dj Dk)/2,
 * dD/dC = (Dj Dk + Di Dj - Di Dk)/2.
 */
static void atm_sides_grad(const double *xi, const double *xj, const double *xk,
                           double nu, double eps, double *gA, double *gB, double *gC)
{
    double A = sqdist(xi, xj, 3), B = sqdist(xj, xk, 3), C = sqdist(xk, xi, 3);
    double sA = A + eps, sB = B + eps, sC = C + eps;
    double Di = 0.5 * (A + C - B), Dj = 0.5 * (A + B - C), Dk = 0.5 * (B + C - A);
    double P = sA * sB * sC;
    double D = Di * Dj * Dk;
    double p32 = 1.0 / (P * sqrt(P));
    double p52 = p32 / P;
    double dA = 0.5 * (Dj * Dk + Di * Dk - Di * Dj);
    double dB = 0.5 * (Di * Dk + Di * Dj - Dj * Dk);
    double dC = 0.5 * (Dj * Dk + Di * Dj - Di * Dk);
    *gA = nu * (-1.5 * p32 / sA + 3.0 * dA * p52 - 7.5 * D * p52 / sA);
    *gB = nu * (-1.5 * p32 / sB + 3.0 * dB * p52 - 7.5 * D * p52 / sB);
    *gC = nu * (-1.5 * p32 / sC + 3.0 * dC * p52 - 7.5 * D * p52 / sC);
}

/* Full gradient dE/dx (n x 3), O(n^3): the chain rule through the sides,
 * dA/dx_i = 2(x_i - x_j), dA/dx_j = -2(x_i - x_j), and so on. */
void oracle_atm_grad(int64_t n, const double *x, double nu, double eps, double *grad)
{
    memset(grad, 0, sizeof(double) * 3 * n);
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j)
            for (int64_t k = j + 1; k < n; ++k) {
                const double *xi = x + 3 * i, *xj = x + 3 * j, *xk = x + 3 * k;
                double gA, gB, gC;
                atm_sides_grad(xi, xj, xk, nu, eps, &gA, &gB, &gC);
                for (int t = 0; t < 3; ++t) {
                    double ij = xi[t] - xj[t], jk = xj[t] - xk[t], ki = xk[t] - xi[t];
                    grad[3 * i + t] += 2.0 * gA * ij - 2.0 * gC * ki;
                    grad[3 * j + t] += -2.0 * gA * ij + 2.0 * gB * jk;
                    grad[3 * k + t] += -2.0 * gB * jk + 2.0 * gC * ki;
                }
            }
}

/* Conditioning of the gradient: for every atom, the sum over the triples
 * that hold it of the magnitudes of the two parts its gradient gets from
 * the triple's two sides at that atom, 2 |de/ds| |x_a - x_b| each (the
 * gradient itself sums the same parts as vectors).  An FP32 evaluation
 * that rounds each side derivative independently errs in an atom's gradient
 * by a small multiple of the FP32 unit roundoff times this sum, however
 * much the parts cancel (a pair of atoms much closer than the rest makes
 * the parts at a third atom large and nearly opposite). */
void oracle_atm_grad_abs(int64_t n, const double *x, double nu, double eps, double *out)
{
    memset(out, 0, sizeof(double) * n);
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j)
            for (int64_t k = j + 1; k < n; ++k) {
                const double *xi = x + 3 * i, *xj = x + 3 * j, *xk = x + 3 * k;
                double gA, gB, gC;
                atm_sides_grad(xi, xj, xk, nu, eps, &gA, &gB, &gC);
                const double a = 2.0 * fabs(gA) * sqrt(sqdist(xi, xj, 3));
                const double b = 2.0 * fabs(gB) * sqrt(sqdist(xj, xk, 3));
                const double c = 2.0 * fabs(gC) * sqrt(sqdist(xk, xi, 3));
                out[i] += a + c;
                out[j] += a + b;
                out[k] += b + c;
            }
}

/* Energy of the triples i < j < k with i in [i_lo, i_hi), and their
 * contribution to the gradient added into grad (n x 3): a slice of the outer
 * loop of the total energy and gradient, used to time a bounded sample of the
 * energy-and-forces workload (slices partition the sum). */
double oracle_atm_energy_grad_slice(int64_t n, const double *x, double nu, double eps,
                                    int64_t i_lo, int64_t i_hi, double *grad)
{
    double e = 0.0;
    for (int64_t i = i_lo; i < i_hi && i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j)
            for (int64_t k = j + 1; k < n; ++k) {
                const double *xi = x + 3 * i, *xj = x + 3 * j, *xk = x + 3 * k;
                double gA, gB, gC;
                e += atm_term(xi, xj, xk, nu, eps);
                atm_sides_grad(xi, xj, xk, nu, eps, &gA, &gB, &gC);
                for (int t = 0; t < 3; ++t) {
                    double ij = xi[t] - xj[t], jk = xj[t] - xk[t], ki = xk[t] - xi[t];
                    grad[3 * i + t] += 2.0 * gA * ij - 2.0 * gC * ki;
                    grad[3 * j + t] += -2.0 * gA * ij + 2.0 * gB * jk;
                    grad[3 * k + t] += -2.0 * gB * jk + 2.0 * gC * ki;
                }
            }
    return e;
}

/* Gradient rows of the listed atoms only, O(n^2) each. */
void oracle_atm_grad_atoms(int64_t n, const double *x, double nu, double eps,
                           const int64_t *atoms, int64_t count, double *out)
{
    for (int64_t t = 0; t < count; ++t) {
        int64_t a = atoms[t];
        double g[3] = {0.0, 0.0, 0.0};
        for (int64_t j = 0; j < n; ++j) {
            if (j == a) continue;
            for (int64_t k = j + 1; k < n; ++k) {
                if (k == a) continue;
                /* triangle (a, j, k): A = |x_a - x_j|^2, C = |x_k - x_a|^2 */
                const double *xa = x + 3 * a, *xj = x + 3 * j, *xk = x + 3 * k;
                double gA, gB, gC;
                atm_sides_grad(xa, xj, xk, nu, eps, &gA, &gB, &gC);
                for (int s = 0; s < 3; ++s)
                    g[s] += 2.0 * gA * (xa[s] - xj[s]) - 2.0 * gC * (xk[s] - xa[s]);
            }
        }
        out[3 * t] = g[0]; out[3 * t + 1] = g[1]; out[3 * t + 2] = g[2];
    }
}

/* ======================= stress loss ======================= */

/*
 * Stress of a configuration x against reference squared distances taken
 * from y:  L = sum_{i<j} (D_ij - delta_ij)^2,  D_ij = |x_i - x_j|^2,
 * delta_ij = |y_i - y_j|^2.
 */
double oracle_stress_loss(int64_t n, int64_t d, const double *x, const double *y)
{
    double L = 0.0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < i; ++j) {
            double r = sqdist(x + i * d, x + j * d, d) - sqdist(y + i * d, y + j * d, d);
            L += r * r;
        }
    return L;
}

/* The loss terms of rows i in [i_lo, i_hi): sum over j < i of (D_ij -
 * delta_ij)^2 (slices partition L; used to time a bounded sample). */
double oracle_stress_loss_rows(int64_t n, int64_t d, const double *x, const double *y,
                               int64_t i_lo, int64_t i_hi)
{
    double L = 0.0;
    for (int64_t i = i_lo; i < i_hi && i < n; ++i)
        for (int64_t j = 0; j < i; ++j) {
            double r = sqdist(x + i * d, x + j * d, d) - sqdist(y + i * d, y + j * d, d);
            L += r * r;
        }
    return L;
}

/* dL/dx_i = sum_{j != i} 2 (D_ij - delta_ij) * 2 (x_i - x_j), for listed rows. */
void oracle_stress_grad_rows(int64_t n, int64_t d, const double *x, const double *y,
                             const int64_t *rows, int64_t count, double *out)
{
    for (int64_t t = 0; t < count; ++t) {
        int64_t i = rows[t];
        double *g = out + t * d;
        for (int64_t s = 0; s < d; ++s) g[s] = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double r = sqdist(x + i * d, x + j * d, d) - sqdist(y + i * d, y + j * d, d);
            for (int64_t s = 0; s < d; ++s)
                g[s] += 4.0 * r * (x[i * d + s] - x[j * d + s]);
        }
    }
}
