// tile.cuh -- a 32 x 32 tile of squared distances on SIMT cores (FP32,
// difference form), shared by the packed EDM and the stress kernels.
//
// 256 threads: warp w owns tile rows w, w+8, w+16, w+24; lane c owns column c.
// Points are staged in shared memory 32 coordinates at a time (row pitch 33
// floats, so the column reads of a warp hit 32 different banks).
#pragma once
#include "common.cuh"

namespace sx {

struct TileSmem {
    float rows[32][33];
    float cols[32][33];
};

// Loads coordinates [c0, c0 + dc) of points p0 .. p0+31 (zero past n).
__device__ __forceinline__ void load_chunk(const float *__restrict__ x, int64_t n, int d,
                                           int64_t p0, int c0, int dc, float (*dst)[33]) {
    for (int e = threadIdx.x; e < 32 * dc; e += 256) {
        const int rr = e / dc, cc = e - rr * dc;
        const int64_t p = p0 + rr;
        dst[rr][cc] = p < n ? __ldg(x + p * d + c0 + cc) : 0.0f;
    }
}

// acc[m] += |x_{row0+w+8m} - x_{col0+lane}|^2 over all d coordinates.
__device__ __forceinline__ void tile_sqdist(const float *__restrict__ x, int64_t n, int d,
                                            int64_t row0, int64_t col0, TileSmem &sm,
                                            float acc[4]) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int c0 = 0; c0 < d; c0 += 32) {
        const int dc = d - c0 < 32 ? d - c0 : 32;
        __syncthreads();
        load_chunk(x, n, d, row0, c0, dc, sm.rows);
        load_chunk(x, n, d, col0, c0, dc, sm.cols);
        __syncthreads();
        for (int cc = 0; cc < dc; ++cc) {
            const float xj = sm.cols[lane][cc];
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const float diff = sm.rows[w + 8 * m][cc] - xj;
                acc[m] = fmaf(diff, diff, acc[m]);
            }
        }
    }
}

// A diagonal block pair (blocks at b0 and b1, b0 < b1) packed into one
// 32 x 33 rectangle, as the 2-simplex map pairs them in its grid row 0:
// element (r, c), c <= r, is (i, j) = (b0 + r, b0 + c) of the first block's
// lower triangle; c > r is (b1 + 31 - r, b1 + c - r - 1) of the second's
// strictly lower triangle (its diagonal, column 32, is zero).  acc[m] +=
// |x_i - x_j|^2 for rows r = w + 8m and column c = lane; the first block's
// points are staged in sm.rows, the second's in sm.cols.
__device__ __forceinline__ void pair_sqdist(const float *__restrict__ x, int64_t n, int d,
                                            int64_t b0, int64_t b1, TileSmem &sm, float acc[4]) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int c0 = 0; c0 < d; c0 += 32) {
        const int dc = d - c0 < 32 ? d - c0 : 32;
        __syncthreads();
        load_chunk(x, n, d, b0, c0, dc, sm.rows);
        load_chunk(x, n, d, b1, c0, dc, sm.cols);
        __syncthreads();
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int r = w + 8 * m;
            const bool first = lane <= r;
            const float *pi = first ? &sm.rows[r][0] : &sm.cols[31 - r][0];
            const float *pj = first ? &sm.rows[lane][0] : &sm.cols[lane - r - 1][0];
            float a = acc[m];
            for (int cc = 0; cc < dc; ++cc) {
                const float diff = pi[cc] - pj[cc];
                a = fmaf(diff, diff, a);
            }
            acc[m] = a;
        }
    }
}

}  // namespace sx
