// edm.cu -- packed lower-triangular Euclidean distance matrix over the
// 2-simplex {j <= i} (Sec. I names the EDM as a 2-simplex problem), one
// 32 x 32 tile per data block, the block chosen by a block-space map
// (Sec. III-A eq. (map2d), bounding box, or linear enumeration).
#include "common.cuh"
#include "kernels.h"
#include "tile.cuh"

namespace sx {

// Position of pair (i, j) in the tile-packed layout: tile (i / 128, j / 128)
// of the tile triangle in packed lower order, 128 x 128 floats row-major.
// For j <= i, and for the mirror (j, i) of a pair inside a diagonal tile.
__device__ __forceinline__ int64_t tiles_index(int64_t i, int64_t j) {
    const int64_t I = i >> 7, J = j >> 7;
    return ((I * (I + 1) / 2 + J) << 14) + ((i & 127) << 7) + (j & 127);
}

// Stores D_ij (j <= i < n) in the chosen layout; in the tile layout a pair
// inside a diagonal tile also fills its mirror entry (j, i).
template <bool TILES>
__device__ __forceinline__ void put_pair(float *__restrict__ out, int64_t i, int64_t j, float v) {
    if constexpr (TILES) {
        out[tiles_index(i, j)] = v;
        if ((i >> 7) == (j >> 7) && j != i) out[tiles_index(j, i)] = v;
    } else {
        out[i * (i + 1) / 2 + j] = v;
    }
}

// FP32 difference form: out[i(i+1)/2 + j] = sum_t (x_it - x_jt)^2 (or the
// tile-packed position of (i, j)).
template <int MAP, bool TILES>
__global__ void __launch_bounds__(256) k_edm_simt(int64_t n, int d, const float *__restrict__ x,
                                                  float *__restrict__ out, int nb) {
    __shared__ TileSmem sm;
    const List2 L = decode2<MAP>(blockIdx.x, blockIdx.y, nb);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (L.pair && L.cnt == 2) {
        // the two diagonal blocks of lambda's grid row 0 in one packed pass
        const int64_t b0 = (int64_t)L.d0 * kEdmRho, b1 = (int64_t)L.d1 * kEdmRho;
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        pair_sqdist(x, n, d, b0, b1, sm, acc);
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int r = w + 8 * m;
            const bool first = lane <= r;
            const int64_t i = first ? b0 + r : b1 + 31 - r;
            const int64_t j = first ? b0 + lane : b1 + lane - r - 1;
            if (i < n) put_pair<TILES>(out, i, j, acc[m]);
        }
        if (w == 0 && b1 + lane < n) {
            const int64_t i = b1 + lane;
            put_pair<TILES>(out, i, i, 0.0f);   // the second block's diagonal
        }
        return;
    }
    for (int t = 0; t < L.cnt; ++t) {
        const int64_t row0 = (int64_t)(t ? L.y[1] : L.y[0]) * kEdmRho, col0 = (int64_t)(t ? L.x[1] : L.x[0]) * kEdmRho;
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        tile_sqdist(x, n, d, row0, col0, sm, acc);
        const int64_t j = col0 + lane;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int64_t i = row0 + w + 8 * m;
            if (j <= i && i < n) put_pair<TILES>(out, i, j, acc[m]);
        }
    }
}

// Whether a request runs on the tensor-core path.
static bool use_umma(int64_t d, int prec) {
    return prec == SIMPLEX_PREC_BF16X3 || (prec == SIMPLEX_PREC_AUTO && d >= 64 && d % 64 == 0);
}

int edm_rho(int64_t d, int prec) { return use_umma(d, prec) ? kEdmUmmaRho : kEdmRho; }

int64_t edm_workspace_bytes(int64_t n, int64_t d, int map, int prec) {
    (void)map;
    return use_umma(d, prec) ? edm_umma_workspace_bytes(n, d) : 0;
}

}  // namespace sx

using namespace sx;

namespace sx {

template <bool TILES>
static void launch_simt(int map, const Grid &g, cudaStream_t s, int64_t n, int d, const float *x, float *out,
                        int nb) {
    if (map == MAP_LAMBDA) k_edm_simt<MAP_LAMBDA, TILES><<<dim_of(g), 256, 0, s>>>(n, d, x, out, nb);
    else if (map == MAP_BBOX) k_edm_simt<MAP_BBOX, TILES><<<dim_of(g), 256, 0, s>>>(n, d, x, out, nb);
    else if (map == MAP_RB) k_edm_simt<MAP_RB, TILES><<<dim_of(g), 256, 0, s>>>(n, d, x, out, nb);
    else k_edm_simt<MAP_LINEAR, TILES><<<dim_of(g), 256, 0, s>>>(n, d, x, out, nb);
}

// Both layouts: argument checks, then the tensor-core or the SIMT path.
static int edm_run(int64_t n, int64_t d, const float *x, float *out, int map, int prec, bool tiles,
                   void *workspace, int64_t ws_bytes, void *stream) {
    if (n < 1 || d < 1 || !x || !out || map < MAP_LAMBDA || map > MAP_RB) return SIMPLEX_EINVAL;
    if (prec < SIMPLEX_PREC_FP32 || prec > SIMPLEX_PREC_AUTO) return SIMPLEX_EINVAL;
    if (!aligned(x, 4) || !aligned(out, 4)) return SIMPLEX_EALIGN;
    if (d > (1 << 24) || n > ((int64_t)1 << 31) || n * d > ((int64_t)1 << 40)) return SIMPLEX_EOVERFLOW;
    cudaStream_t s = (cudaStream_t)stream;
    if (use_umma(d, prec)) return edm_umma_run(n, d, x, out, map, tiles, workspace, ws_bytes, s);
    const int64_t nb = (n + kEdmRho - 1) / kEdmRho;
    const Grid g = grid2(nb, map);
    if (!grid_fits(g)) return SIMPLEX_EOVERFLOW;
    if (tiles && n % 128 != 0) {
        // the padding of the last tile row is 0 (its other entries are written
        // again by the kernel, later on the same stream)
        const int64_t nt = (n + 127) / 128;
        int st = cuda_status(cudaMemsetAsync(out + ((nt - 1) * nt / 2 << 14), 0, sizeof(float) * (size_t)(nt << 14), s));
        if (st) return st;
    }
    prof_begin(s);
    if (tiles) launch_simt<true>(map, g, s, n, (int)d, x, out, (int)nb);
    else launch_simt<false>(map, g, s, n, (int)d, x, out, (int)nb);
    prof_end(s);
    note_launches(1);
    return launch_status();
}

}  // namespace sx

extern "C" int simplex_edm_packed(int64_t n, int64_t d, const float *x, float *out, int map,
                                  int prec, void *workspace, int64_t ws_bytes, void *stream) {
    return edm_run(n, d, x, out, map, prec, false, workspace, ws_bytes, stream);
}

extern "C" int64_t simplex_edm_tiles_len(int64_t n) {
    if (n < 1 || n > ((int64_t)1 << 31)) return -1;
    const int64_t nt = (n + 127) / 128;
    return (nt * (nt + 1) / 2) << 14;
}

extern "C" int simplex_edm_tiles(int64_t n, int64_t d, const float *x, float *out, int map,
                                 int prec, void *workspace, int64_t ws_bytes, void *stream) {
    return edm_run(n, d, x, out, map, prec, true, workspace, ws_bytes, stream);
}
