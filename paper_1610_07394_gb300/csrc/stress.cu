// stress.cu -- stress loss over the packed EDM and its gradient, on the
// 2-simplex of pairs {j < i} (Sec. I: the EDM is a 2-simplex problem), one
// 64 x 64 tile per data block chosen by a block-space map (Sec. III-A).
//
//   L = sum_{i<j} (D_ij - delta_ij)^2,  D_ij = |x_i - x_j|^2,
//   delta_ij = |y_i - y_j|^2,
//   dL/dx_i = 4 sum_{j != i} (D_ij - delta_ij)(x_i - x_j).
//
// The residual is recomputed per pair, never stored.  With S = x + y,
// Delta = x - y and a_i = S_i . Delta_i = |x_i|^2 - |y_i|^2,
//   r_ij = D_ij - delta_ij = a_i + a_j - (S_i . Delta_j + Delta_i . S_j),
// a sum of products of the same size as r itself for configurations that
// y perturbs (no cancellation between two large squared distances), so the
// tile is a register-blocked FP32 product: each thread owns 4 x 4 pairs and
// does 32 FMAs per coordinate from four 16-byte shared loads.  The backward
// pass turns the residual tile C (C_ij = r_ij for j < i) into both sides'
// contributions, grad_I += 4 (rowsum(C) x_I - C x_J) and
// grad_J += 4 (colsum(C) x_J - C^T x_I), as two register-blocked tile
// products, flushed with FP32 (vector) atomics.  The loss is reduced per
// block with compensated FP32 sums and across blocks in FP64.  The optional
// packed D of the forward pass is the FP32 difference form of the EDM.
#include "common.cuh"
#include "kernels.h"
#include "tile.cuh"

namespace sx {

constexpr int SR = kStressRho;   // 64 points per tile side
constexpr int SC = 32;           // coordinates staged per chunk

// Shared memory of one tile: coordinates transposed ([t][point]) so that a
// thread's four consecutive points are one 16-byte load.  Point p of
// coordinate t sits at column sw(t, p) = p ^ (4 (t & 7)): the staging writes
// (32 consecutive t, one p per warp) spread over 8 bank groups instead of 1,
// and groups of four points stay contiguous.
struct StressSmem {
    float sr[SC][SR], dr[SC][SR];     // S and Delta of the row tile (points i)
    float sc[SC][SR], dc[SC][SR];     // S and Delta of the column tile (points j)
    float ar[SR], ac[SR];             // a = S . Delta of row / column points
    float C[SR][SR + 4];              // residual tile (backward), [j][i]
    float rsum[SR], csum[SR];
};

__device__ __forceinline__ int sw(int t, int p) { return p ^ ((t & 7) << 2); }

// Stages coordinates [c0, c0 + dc) of the row and column tiles as S, Delta.
__device__ __forceinline__ void stage_sd(const float *__restrict__ x, const float *__restrict__ y,
                                         int64_t n, int d, int64_t row0, int64_t col0, int c0,
                                         int dc, StressSmem &sm) {
    for (int e = threadIdx.x; e < 2 * SR * SC; e += 256) {
        const int side = e / (SR * SC), rem = e - side * SR * SC;
        const int p = rem / SC, t = rem - p * SC;   // t fastest: coalesced global reads
        const int64_t g = (side ? col0 : row0) + p;
        float xv = 0.f, yv = 0.f;
        if (t < dc && g < n) {
            xv = __ldg(x + g * d + c0 + t);
            yv = __ldg(y + g * d + c0 + t);
        }
        const int q = sw(t, p);
        if (side) { sm.sc[t][q] = xv + yv; sm.dc[t][q] = xv - yv; }
        else { sm.sr[t][q] = xv + yv; sm.dr[t][q] = xv - yv; }
    }
}

// r[a][b] for rows i = row0 + 4 ty + a, columns j = col0 + 4 tx + b.
__device__ __forceinline__ void residual_tile(const float *__restrict__ x,
                                              const float *__restrict__ y, int64_t n, int d,
                                              int64_t row0, int64_t col0, StressSmem &sm,
                                              float (&r)[4][4]) {
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
    float aself = 0.f;   // a of point threadIdx.x % 64 of the row (< 64) or column (< 128) tile
    for (int c0 = 0; c0 < d; c0 += SC) {
        const int dc = d - c0 < SC ? d - c0 : SC;
        __syncthreads();
        stage_sd(x, y, n, d, row0, col0, c0, dc, sm);
        __syncthreads();
        if (threadIdx.x < 2 * SR) {
            const int p = threadIdx.x & (SR - 1);
            const bool col = threadIdx.x >= SR;
            for (int t = 0; t < dc; ++t) {
                const int q = sw(t, p);
                aself = col ? fmaf(sm.sc[t][q], sm.dc[t][q], aself) : fmaf(sm.sr[t][q], sm.dr[t][q], aself);
            }
        }
        for (int t = 0; t < dc; ++t) {
            const int qi = sw(t, 4 * ty), qj = sw(t, 4 * tx);
            const float4 s_i = *reinterpret_cast<const float4 *>(&sm.sr[t][qi]);
            const float4 d_i = *reinterpret_cast<const float4 *>(&sm.dr[t][qi]);
            const float4 s_j = *reinterpret_cast<const float4 *>(&sm.sc[t][qj]);
            const float4 d_j = *reinterpret_cast<const float4 *>(&sm.dc[t][qj]);
            const float si[4] = {s_i.x, s_i.y, s_i.z, s_i.w}, di[4] = {d_i.x, d_i.y, d_i.z, d_i.w};
            const float sj[4] = {s_j.x, s_j.y, s_j.z, s_j.w}, dj[4] = {d_j.x, d_j.y, d_j.z, d_j.w};
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(si[a], dj[b], fmaf(di[a], sj[b], acc[a][b]));
        }
    }
    if (threadIdx.x < SR) sm.ar[threadIdx.x] = aself;
    else if (threadIdx.x < 2 * SR) sm.ac[threadIdx.x - SR] = aself;
    __syncthreads();
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) r[a][b] = (sm.ar[4 * ty + a] + sm.ac[4 * tx + b]) - acc[a][b];
}

template <int MAP>
__global__ void __launch_bounds__(256) k_stress_fwd(int64_t n, int d, const float *__restrict__ x,
                                                    const float *__restrict__ y,
                                                    float *__restrict__ d_out, int nb,
                                                    double *__restrict__ partials) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    StressSmem &sm = *reinterpret_cast<StressSmem *>(smem_raw);
    __shared__ TileSmem dsm;
    __shared__ float red[16];
    const List2 L = decode2<MAP>(blockIdx.x, blockIdx.y, nb);
    if (L.cnt == 0) {   // a block outside the simplex exits at once
        if (threadIdx.x == 0) partials[blockIdx.x + (int64_t)gridDim.x * blockIdx.y] = 0.0;
        return;
    }
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float hi = 0.f, lo = 0.f;
#pragma unroll 1
    for (int t = 0; t < L.cnt; ++t) {
        const int X = t ? L.x[1] : L.x[0], Y = t ? L.y[1] : L.y[0];
        const int64_t row0 = (int64_t)Y * SR, col0 = (int64_t)X * SR;
        float r[4][4];
        residual_tile(x, y, n, d, row0, col0, sm, r);
        float loc = 0.f;
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int64_t i = row0 + 4 * ty + a, j = col0 + 4 * tx + b;
                if (j < i && i < n) loc = fmaf(r[a][b], r[a][b], loc);
            }
        add_ff(hi, lo, loc, 0.f);
        if (d_out) {
            // the packed D itself: FP32 difference form on 32 x 32 sub-tiles
            for (int sub = 0; sub < 4; ++sub) {
                const int64_t r0 = row0 + 32 * (sub >> 1), c0 = col0 + 32 * (sub & 1);
                if (c0 > r0 + 31) continue;
                float D[4] = {0.f, 0.f, 0.f, 0.f};
                tile_sqdist(x, n, d, r0, c0, dsm, D);
                const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
                const int64_t j = c0 + lane;
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    const int64_t i = r0 + w + 8 * m;
                    if (j <= i && i < n) d_out[i * (i + 1) / 2 + j] = D[m];
                }
            }
        }
        __syncthreads();
    }
    const double s = block_sum_ff<256>(hi, lo, red);
    if (threadIdx.x == 0) partials[blockIdx.x + (int64_t)gridDim.x * blockIdx.y] = s;
}

// out[p][t] += scale * sum_q W[p][q] (xs[p][t] - xo[q][t]) for the 64 points
// p of one side, as a register-blocked product: thread (tx, ty) owns points
// 4 ty + a and coordinates 4 tx + b of the current 64-coordinate chunk.
// W = C for the row side (C stored [j][i]), C^T for the column side.
__device__ __forceinline__ void side_grad(const float *__restrict__ x, int64_t n, int d,
                                          int64_t p0, int64_t q0, bool columns,
                                          const StressSmem &sm, float scale4,
                                          float *__restrict__ grad, float (*xo)[SR],
                                          float (*xs)[SR]) {
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    for (int c0 = 0; c0 < d; c0 += SR) {
        const int dc = d - c0 < SR ? d - c0 : SR;
        __syncthreads();
        // xo[q][t]: x of the other side's point q; xs[p][t]: x of this side's point p
        for (int e = threadIdx.x; e < 2 * SR * SR; e += 256) {
            const int side = e / (SR * SR), rem = e - side * SR * SR;
            const int p = rem / SR, t = rem - p * SR;
            const int64_t g = (side ? p0 : q0) + p;
            const float v = (t < dc && g < n) ? __ldg(x + g * d + c0 + t) : 0.f;
            if (side) xs[p][t] = v; else xo[p][t] = v;
        }
        __syncthreads();
        float acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
        for (int q = 0; q < SR; ++q) {
            float w[4];
            if (!columns) {   // W[p][q] = C_pq, stored at C[q][p]
                const float4 c = *reinterpret_cast<const float4 *>(&sm.C[q][4 * ty]);
                w[0] = c.x; w[1] = c.y; w[2] = c.z; w[3] = c.w;
            } else {          // W[p][q] = C_qp, stored at C[p][q]
#pragma unroll
                for (int a = 0; a < 4; ++a) w[a] = sm.C[4 * ty + a][q];
            }
            const float4 xv = *reinterpret_cast<const float4 *>(&xo[q][4 * tx]);
            const float xq[4] = {xv.x, xv.y, xv.z, xv.w};
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(w[a], xq[b], acc[a][b]);
        }
        const float *wsum = columns ? sm.csum : sm.rsum;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int p = 4 * ty + a;
            const int64_t g = p0 + p;
            if (g >= n) continue;
            float o[4];
#pragma unroll
            for (int b = 0; b < 4; ++b) o[b] = scale4 * fmaf(xs[p][4 * tx + b], wsum[p], -acc[a][b]);
            float *dst = grad + g * d + c0 + 4 * tx;
            if ((d & 3) == 0 && 4 * tx + 3 < dc) {
                atomicAdd(reinterpret_cast<float4 *>(dst), make_float4(o[0], o[1], o[2], o[3]));
            } else {
#pragma unroll
                for (int b = 0; b < 4; ++b)
                    if (4 * tx + b < dc) atomicAdd(dst + b, o[b]);
            }
        }
    }
}

// With `partials`, the loss of the same residual tiles as well (one FP64
// partial per block): loss and gradient in one pass.
template <int MAP>
__global__ void __launch_bounds__(256) k_stress_bwd(int64_t n, int d, const float *__restrict__ x,
                                                    const float *__restrict__ y, float scale4,
                                                    int nb, float *__restrict__ grad,
                                                    double *__restrict__ partials) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    StressSmem &sm = *reinterpret_cast<StressSmem *>(smem_raw);
    __shared__ float red[16];
    float hi = 0.f, lo = 0.f;
    // the x tiles of the gradient products reuse the S / Delta staging area
    float (*xo)[SR] = reinterpret_cast<float (*)[SR]>(&sm.sr[0][0]);
    float (*xs)[SR] = xo + SR;
    static_assert(2 * SR * SR <= 4 * SC * SR, "x staging fits the S/Delta area");
    const List2 L = decode2<MAP>(blockIdx.x, blockIdx.y, nb);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll 1
    for (int t = 0; t < L.cnt; ++t) {
        const int X = t ? L.x[1] : L.x[0], Y = t ? L.y[1] : L.y[0];
        const int64_t row0 = (int64_t)Y * SR, col0 = (int64_t)X * SR;
        float r[4][4];
        residual_tile(x, y, n, d, row0, col0, sm, r);
        float loc = 0.f;
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int64_t i = row0 + 4 * ty + a, j = col0 + 4 * tx + b;
                const float c = (j < i && i < n) ? r[a][b] : 0.f;
                sm.C[4 * tx + b][4 * ty + a] = c;
                loc = fmaf(c, c, loc);
            }
        if (partials) add_ff(hi, lo, loc, 0.f);
        __syncthreads();
        if (threadIdx.x < SR) {
            float s = 0.f;
            for (int q = 0; q < SR; ++q) s += sm.C[q][threadIdx.x];   // row i: sum over j
            sm.rsum[threadIdx.x] = s;
        } else if (threadIdx.x < 2 * SR) {
            const int p = threadIdx.x - SR;
            float s = 0.f;
            for (int q = 0; q < SR; ++q) s += sm.C[p][q];             // column j: sum over i
            sm.csum[p] = s;
        }
        // rows i (points of block Y) against columns j, then columns against rows
        side_grad(x, n, d, row0, col0, false, sm, scale4, grad, xo, xs);
        side_grad(x, n, d, col0, row0, true, sm, scale4, grad, xo, xs);
        __syncthreads();
    }
    if (partials) {
        const double s = block_sum_ff<256>(hi, lo, red);
        if (threadIdx.x == 0) partials[blockIdx.x + (int64_t)gridDim.x * blockIdx.y] = s;
    }
}

static int stress_check(int64_t n, int64_t d, const float *x, const float *y, int map, int prec,
                        Grid &g, int64_t &nb) {
    if (n < 1 || d < 1 || !x || !y || map < MAP_LAMBDA || map > MAP_RB) return SIMPLEX_EINVAL;
    if (prec < SIMPLEX_PREC_FP32 || prec > SIMPLEX_PREC_AUTO) return SIMPLEX_EINVAL;
    if (prec == SIMPLEX_PREC_BF16X3 && !stress_umma_ok(d)) return SIMPLEX_EUNSUPPORTED;
    if (!aligned(x, 4) || !aligned(y, 4)) return SIMPLEX_EALIGN;
    if (d > (1 << 24) || n > ((int64_t)1 << 31) || n * d > ((int64_t)1 << 40)) return SIMPLEX_EOVERFLOW;
    nb = (n + SR - 1) / SR;
    g = grid2(nb, map);
    if (!grid_fits(g)) return SIMPLEX_EOVERFLOW;
    return SIMPLEX_OK;
}

constexpr int kStressSmem = (int)sizeof(StressSmem);

// The tile's shared memory exceeds the 48 KB default of a launch; opt in
// once per device for every instantiation.
static int stress_optin() {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e);
    static bool done[64] = {};
    if (dev < 0 || dev >= 64) return SIMPLEX_EUNSUPPORTED;
    if (!done[dev]) {
        const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
        if ((e = cudaFuncSetAttribute(k_stress_fwd<MAP_LAMBDA>, a, kStressSmem)) != cudaSuccess ||
            (e = cudaFuncSetAttribute(k_stress_fwd<MAP_BBOX>, a, kStressSmem)) != cudaSuccess ||
            (e = cudaFuncSetAttribute(k_stress_fwd<MAP_LINEAR>, a, kStressSmem)) != cudaSuccess ||
            (e = cudaFuncSetAttribute(k_stress_fwd<MAP_RB>, a, kStressSmem)) != cudaSuccess ||
            (e = cudaFuncSetAttribute(k_stress_bwd<MAP_LAMBDA>, a, kStressSmem)) != cudaSuccess ||
            (e = cudaFuncSetAttribute(k_stress_bwd<MAP_BBOX>, a, kStressSmem)) != cudaSuccess ||
            (e = cudaFuncSetAttribute(k_stress_bwd<MAP_LINEAR>, a, kStressSmem)) != cudaSuccess ||
            (e = cudaFuncSetAttribute(k_stress_bwd<MAP_RB>, a, kStressSmem)) != cudaSuccess)
            return cuda_status(e);
        done[dev] = true;
    }
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
    if (stress_use_umma(d, prec))
        return stress_umma_run(false, n, d, x, y, d_out, loss, 0.0, nullptr, map, workspace, ws_bytes,
                               (cudaStream_t)stream);
    const int64_t blocks = g.gx * g.gy;
    if (!workspace || ws_bytes < 8 * (blocks + kReduceSlots) || !aligned(workspace, 256))
        return SIMPLEX_EWORKSPACE;
    if ((st = stress_optin())) return st;
    cudaStream_t s = (cudaStream_t)stream;
    double *partials = (double *)workspace;
    prof_begin(s);
    if (map == MAP_LAMBDA) k_stress_fwd<MAP_LAMBDA><<<dim_of(g), 256, kStressSmem, s>>>(n, (int)d, x, y, d_out, (int)nb, partials);
    else if (map == MAP_BBOX) k_stress_fwd<MAP_BBOX><<<dim_of(g), 256, kStressSmem, s>>>(n, (int)d, x, y, d_out, (int)nb, partials);
    else if (map == MAP_RB) k_stress_fwd<MAP_RB><<<dim_of(g), 256, kStressSmem, s>>>(n, (int)d, x, y, d_out, (int)nb, partials);
    else k_stress_fwd<MAP_LINEAR><<<dim_of(g), 256, kStressSmem, s>>>(n, (int)d, x, y, d_out, (int)nb, partials);
    prof_end(s);
    note_launches(1);
    if ((st = launch_status())) return st;
    return reduce_partials(partials, blocks, partials + blocks, loss, s);
}

// Gradient (times gscale) and, when `loss` is not NULL, the loss from the
// same pass.
static int stress_grad(int64_t n, int64_t d, const float *x, const float *y, double gscale,
                       float *grad, double *loss, int map, int prec, void *workspace,
                       int64_t ws_bytes, cudaStream_t s) {
    if (!grad) return SIMPLEX_EINVAL;
    Grid g;
    int64_t nb;
    int st = stress_check(n, d, x, y, map, prec, g, nb);
    if (st) return st;
    if (!aligned(grad, 16) || (loss && !aligned(loss, 8))) return SIMPLEX_EALIGN;
    if (stress_use_umma(d, prec))
        return stress_umma_run(true, n, d, x, y, nullptr, loss, gscale, grad, map, workspace, ws_bytes, s);
    const int64_t blocks = g.gx * g.gy;
    double *partials = nullptr;
    if (loss) {
        if (!workspace || ws_bytes < 8 * (blocks + kReduceSlots) || !aligned(workspace, 256))
            return SIMPLEX_EWORKSPACE;
        partials = (double *)workspace;
    }
    if ((st = stress_optin())) return st;
    if ((st = cuda_status(cudaMemsetAsync(grad, 0, sizeof(float) * (size_t)(n * d), s)))) return st;
    const float scale4 = (float)(4.0 * gscale);
    prof_begin(s);
    if (map == MAP_LAMBDA) k_stress_bwd<MAP_LAMBDA><<<dim_of(g), 256, kStressSmem, s>>>(n, (int)d, x, y, scale4, (int)nb, grad, partials);
    else if (map == MAP_BBOX) k_stress_bwd<MAP_BBOX><<<dim_of(g), 256, kStressSmem, s>>>(n, (int)d, x, y, scale4, (int)nb, grad, partials);
    else if (map == MAP_RB) k_stress_bwd<MAP_RB><<<dim_of(g), 256, kStressSmem, s>>>(n, (int)d, x, y, scale4, (int)nb, grad, partials);
    else k_stress_bwd<MAP_LINEAR><<<dim_of(g), 256, kStressSmem, s>>>(n, (int)d, x, y, scale4, (int)nb, grad, partials);
    prof_end(s);
    note_launches(1);
    if ((st = launch_status())) return st;
    return loss ? reduce_partials(partials, blocks, partials + blocks, loss, s) : SIMPLEX_OK;
}

extern "C" int simplex_stress_bwd(int64_t n, int64_t d, const float *x, const float *y,
                                  double gscale, float *grad, int map, int prec, void *workspace,
                                  int64_t ws_bytes, void *stream) {
    return stress_grad(n, d, x, y, gscale, grad, nullptr, map, prec, workspace, ws_bytes,
                       (cudaStream_t)stream);
}

extern "C" int simplex_stress_fwd_bwd(int64_t n, int64_t d, const float *x, const float *y,
                                      double gscale, float *grad, double *loss, int map, int prec,
                                      void *workspace, int64_t ws_bytes, void *stream) {
    if (!loss) return SIMPLEX_EINVAL;
    return stress_grad(n, d, x, y, gscale, grad, loss, map, prec, workspace, ws_bytes,
                       (cudaStream_t)stream);
}
