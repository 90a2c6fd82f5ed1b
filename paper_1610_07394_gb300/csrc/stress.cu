// stress.cu -- stress loss over the packed EDM and its gradient, on the
// 2-simplex of pairs {j < i} (Sec. I: the EDM is a 2-simplex problem), one
// 32 x 32 tile per data block chosen by a block-space map (Sec. III-A).
//
//   L = sum_{i<j} (D_ij - delta_ij)^2,  D_ij = |x_i - x_j|^2,
//   delta_ij = |y_i - y_j|^2,
//   dL/dx_i = 4 sum_{j != i} (D_ij - delta_ij)(x_i - x_j).
// Both passes recompute the residual r_ij = D_ij - delta_ij from the points
// (never stored), as a sum of per-coordinate differences of squares (see
// tile_resid); the forward pass can also write the packed D.  Pair
// arithmetic is FP32; the loss is reduced in FP64; the gradient accumulates
// in FP32 global atomics.
#include "common.cuh"
#include "kernels.h"
#include "tile.cuh"

namespace sx {

template <int MAP>
__global__ void __launch_bounds__(256) k_stress_fwd(int64_t n, int d, const float *__restrict__ x,
                                                    const float *__restrict__ y,
                                                    float *__restrict__ d_out, int nb,
                                                    double *__restrict__ partials) {
    __shared__ TileSmem sm;
    __shared__ ResidSmem rs;
    __shared__ double red[8];
    const List2 L = decode2<MAP>(blockIdx.x, blockIdx.y, nb);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double total = 0.0;
    for (int t = 0; t < L.cnt; ++t) {
        const int64_t row0 = (int64_t)L.y[t] * kStressRho, col0 = (int64_t)L.x[t] * kStressRho;
        float D[4] = {0.f, 0.f, 0.f, 0.f}, r[4] = {0.f, 0.f, 0.f, 0.f};
        if (d_out) tile_sqdist(x, n, d, row0, col0, sm, D);
        tile_resid(x, y, n, d, row0, col0, rs, r);
        const int64_t j = col0 + lane;
        float loc = 0.f;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int64_t i = row0 + w + 8 * m;
            if (j < i && i < n) loc = fmaf(r[m], r[m], loc);
            if (d_out && j <= i && i < n) d_out[i * (i + 1) / 2 + j] = D[m];
        }
        total += (double)loc;
    }
    const double s = block_sum_f64<256>(total, red);
    if (threadIdx.x == 0) partials[blockIdx.x + (int64_t)gridDim.x * blockIdx.y] = s;
}

template <int MAP>
__global__ void __launch_bounds__(256) k_stress_bwd(int64_t n, int d, const float *__restrict__ x,
                                                    const float *__restrict__ y, float scale4,
                                                    int nb, float *__restrict__ grad) {
    __shared__ TileSmem sm;
    __shared__ ResidSmem rs;
    __shared__ float C[32][33];
    __shared__ float rsum[32], csum[32];
    const List2 L = decode2<MAP>(blockIdx.x, blockIdx.y, nb);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int t = 0; t < L.cnt; ++t) {
        const int64_t row0 = (int64_t)L.y[t] * kStressRho, col0 = (int64_t)L.x[t] * kStressRho;
        float r[4] = {0.f, 0.f, 0.f, 0.f};
        tile_resid(x, y, n, d, row0, col0, rs, r);
        const int64_t j = col0 + lane;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int64_t i = row0 + w + 8 * m;
            C[w + 8 * m][lane] = (j < i && i < n) ? r[m] : 0.0f;
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            float s = 0.f;
            for (int c = 0; c < 32; ++c) s += C[lane][c];
            rsum[lane] = s;
        } else if (threadIdx.x < 64) {
            float s = 0.f;
            for (int r = 0; r < 32; ++r) s += C[r][lane];
            csum[lane] = s;
        }
        // grad_i += 4 (x_i rowsum_i - sum_j C_ij x_j), grad_j += 4 (x_j colsum_j - sum_i C_ij x_i)
        for (int c0 = 0; c0 < d; c0 += 32) {
            const int dc = d - c0 < 32 ? d - c0 : 32;
            __syncthreads();
            load_chunk(x, n, d, row0, c0, dc, sm.rows);
            load_chunk(x, n, d, col0, c0, dc, sm.cols);
            __syncthreads();
            if (lane < dc) {
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    const int r = w + 8 * m;
                    float gr = 0.f, gc = 0.f;
                    for (int q = 0; q < 32; ++q) {
                        gr = fmaf(C[r][q], sm.cols[q][lane], gr);
                        gc = fmaf(C[q][r], sm.rows[q][lane], gc);
                    }
                    const int64_t i = row0 + r, jj = col0 + r;
                    if (i < n) atomicAdd(grad + i * d + c0 + lane, scale4 * fmaf(sm.rows[r][lane], rsum[r], -gr));
                    if (jj < n) atomicAdd(grad + jj * d + c0 + lane, scale4 * fmaf(sm.cols[r][lane], csum[r], -gc));
                }
            }
        }
        __syncthreads();
    }
}

static int stress_check(int64_t n, int64_t d, const float *x, const float *y, int map, int prec,
                        Grid &g, int64_t &nb) {
    if (n < 1 || d < 1 || !x || !y || map < MAP_LAMBDA || map > MAP_LINEAR) return SIMPLEX_EINVAL;
    if (prec < SIMPLEX_PREC_FP32 || prec > SIMPLEX_PREC_AUTO) return SIMPLEX_EINVAL;
    if (prec == SIMPLEX_PREC_BF16X3) return SIMPLEX_EUNSUPPORTED;
    if (!aligned(x, 4) || !aligned(y, 4)) return SIMPLEX_EALIGN;
    if (d > (1 << 24) || n > ((int64_t)1 << 31) || n * d > ((int64_t)1 << 40)) return SIMPLEX_EOVERFLOW;
    nb = (n + kStressRho - 1) / kStressRho;
    g = grid2(nb, map);
    if (!grid_fits(g)) return SIMPLEX_EOVERFLOW;
    return SIMPLEX_OK;
}

}  // namespace sx

using namespace sx;

extern "C" int simplex_stress_fwd(int64_t n, int64_t d, const float *x, const float *y,
                                  float *d_out, double *loss, int map, int prec, void *workspace,
                                  int64_t ws_bytes, void *stream) {
    if (!loss) return SIMPLEX_EINVAL;
    Grid g;
    int64_t nb;
    int st = stress_check(n, d, x, y, map, prec, g, nb);
    if (st) return st;
    if (!aligned(loss, 8) || (d_out && !aligned(d_out, 4))) return SIMPLEX_EALIGN;
    const int64_t blocks = g.gx * g.gy;
    if (!workspace || ws_bytes < 8 * (blocks + kReduceSlots) || !aligned(workspace, 256))
        return SIMPLEX_EWORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    double *partials = (double *)workspace;
    prof_begin(s);
    if (map == MAP_LAMBDA) k_stress_fwd<MAP_LAMBDA><<<dim_of(g), 256, 0, s>>>(n, (int)d, x, y, d_out, (int)nb, partials);
    else if (map == MAP_BBOX) k_stress_fwd<MAP_BBOX><<<dim_of(g), 256, 0, s>>>(n, (int)d, x, y, d_out, (int)nb, partials);
    else k_stress_fwd<MAP_LINEAR><<<dim_of(g), 256, 0, s>>>(n, (int)d, x, y, d_out, (int)nb, partials);
    prof_end(s);
    note_launches(1);
    if ((st = launch_status())) return st;
    return reduce_partials(partials, blocks, partials + blocks, loss, s);
}

extern "C" int simplex_stress_bwd(int64_t n, int64_t d, const float *x, const float *y,
                                  double gscale, float *grad, int map, int prec, void *workspace,
                                  int64_t ws_bytes, void *stream) {
    (void)workspace; (void)ws_bytes;
    if (!grad) return SIMPLEX_EINVAL;
    Grid g;
    int64_t nb;
    int st = stress_check(n, d, x, y, map, prec, g, nb);
    if (st) return st;
    if (!aligned(grad, 16)) return SIMPLEX_EALIGN;
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = cuda_status(cudaMemsetAsync(grad, 0, sizeof(float) * (size_t)(n * d), s)))) return st;
    const float scale4 = (float)(4.0 * gscale);
    prof_begin(s);
    if (map == MAP_LAMBDA) k_stress_bwd<MAP_LAMBDA><<<dim_of(g), 256, 0, s>>>(n, (int)d, x, y, scale4, (int)nb, grad);
    else if (map == MAP_BBOX) k_stress_bwd<MAP_BBOX><<<dim_of(g), 256, 0, s>>>(n, (int)d, x, y, scale4, (int)nb, grad);
    else k_stress_bwd<MAP_LINEAR><<<dim_of(g), 256, 0, s>>>(n, (int)d, x, y, scale4, (int)nb, grad);
    prof_end(s);
    note_launches(1);
    return launch_status();
}
