// stress_umma.cu -- stress loss and its gradient with every pair product on
// the 5th-generation tensor cores (tcgen05, TMEM accumulators, TMA-staged
// operands), for d % 32 == 0 and d <= 96.  Tiles of 128 x 128 pairs (rows i
// of block Y, columns j of block X, X <= Y) of the 2-simplex {j < i}, chosen
// by a block-space map (Sec. III-A); the EDM is the paper's 2-simplex example
// (Sec. I).
//
// With S = x + y, Delta = x - y and a_i = S_i . Delta_i, the residual is
//   r_ij = D_ij - delta_ij = a_i + a_j - M_ij,  M_ij = S_i . Delta_j + Delta_i . S_j,
// so M is one product of K = 2d: P = [S | Delta] (rows i) times Q = [Delta | S]
// (rows j).  P and Q are split into BF16 hi + lo and M accumulates
// hi.hi + hi.lo + lo.hi in FP32 in tensor memory (GEMM1).
//
// Forward: L = sum_{j<i} r_ij^2, from the accumulator in the epilogue, in
// steps of 128 x 256 pairs (k_stress_umma_fwd: a two-CTA cluster per
// 256 x 256 super-block of the map, N = 256 MMAs, the column blocks' Q tiles
// shared by TMA multicast).
//
// Backward: dL/dx_i = 4 sum_{j != i} r_ij (x_i - x_j).  The epilogue writes
// the masked residual tile C (C_ij = r_ij for valid j < i, else 0) to shared
// memory as BF16 hi + lo, and GEMM2 forms both sides of the tile:
//   rows    G_Y = C   [X_X | 1],   grad_i += 4 (G_Y[i][d] x_i - G_Y[i][0:d])
//   columns G_X = C^T [X_Y | 1],   grad_j += 4 (G_X[j][d] x_j - G_X[j][0:d])
// with X^T stored transposed (d rows of coordinates, a row of ones giving the
// row / column sums of C in column d of the accumulator, zero rows up to
// d + 16).  The C tile serves as the K-major A operand of the row side and,
// read M-major through its descriptor, as C^T for the column side.  Each
// CTA walks chunks of 32 consecutive grid blocks of the map's grid (dealt
// by tile count, so that the CTAs finish together), along which the row
// block Y stays fixed for runs of tiles (with the
// lambda map for 2^floor(log2 wy) consecutive grid blocks of row wy), so G_Y
// accumulates in TMEM over a run and is flushed once per run; G_X (two
// buffers where TMEM has room) is flushed per tile.  Flushes are FP32 vector
// atomics into grad.
//
// Both kernels are persistent and warp-specialised, one CTA per SM: warp 0
// issues TMA loads into a two-stage ring (backward: 64 KB stages of GEMM1
// chunks, then GEMM2 coordinate tiles; forward: 96 KB stages), warp 1
// issues the MMAs (the accumulation of step t+1 runs while the epilogue
// drains step t), eight epilogue warps (two per TMEM lane quarter) read the
// accumulators.  Every wait is bounded (simplex_device_errors).
#include <cstddef>
#include <mutex>

#include "common.cuh"
#include "kernels.h"
#include "umma.cuh"

namespace sx {
namespace summa {

using namespace umma;

constexpr int TM = 128;                        // tile rows (i)
constexpr int TN = 128;                        // tile columns (j)
constexpr int KC = 64;                         // K chunk: 64 BF16 = one 128-byte swizzle row
constexpr int TILE_BYTES = TM * KC * 2;        // 16 KB: 128 rows x 64 BF16
constexpr int STAGE_BYTES = 4 * TILE_BYTES;    // 64 KB
constexpr int kStages = 2;                     // ring depth of the backward kernel
constexpr int C_BYTES = 4 * TILE_BYTES;        // C hi, lo for column halves 0, 1
constexpr int kEpiWarps = 8;
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr int kTmemCols = 512;
constexpr int kGY = 256;                       // TMEM column of G_Y (after two GEMM1 accumulators)
// G_X buffer b sits at kGY + NG (1 + b): two buffers when they fit (NG <= 80,
// d <= 64), so that GEMM2 of a tile does not wait for the previous tile's flush
__host__ __device__ inline int gx_buffers(int NG) { return kGY + 3 * NG <= kTmemCols ? 2 : 1; }
constexpr int kMaxCtas = 1024;

__device__ int g_error;   // set when a bounded wait runs out

struct Ctl {
    uint64_t full[kStages], empty[kStages];   // ring: TMA -> MMA -> TMA
    uint64_t tfull[2], tempty[2];             // GEMM1 accumulators: MMA -> epilogue -> MMA
    uint64_t cready;                          // C tile written (epilogue -> MMA)
    uint64_t g2done;                          // GEMM2 of a tile complete (MMA -> epilogue)
    uint64_t gxfree[2];                       // a G_X buffer read out (epilogue -> MMA)
    uint64_t gyfree;                          // G_Y read out at the end of a run (epilogue -> MMA)
    uint64_t done;                            // every MMA of the block complete
    uint32_t tmem;
    int fail;
    alignas(16) float acol[kEpiWarps][64];    // a_j of each epilogue warp's 64 columns
    float red[2 * (kThreads / 32)];
};

constexpr int kCtlBytes = 4096;
constexpr int SMEM_BYTES = 1024 + kStages * STAGE_BYTES + C_BYTES + kCtlBytes;
static_assert(sizeof(Ctl) <= kCtlBytes, "control block");
static_assert(offsetof(Ctl, acol) % 16 == 0, "float4 reads of a_j");
static_assert(SMEM_BYTES <= 227 * 1024, "shared memory per block");

// The tiles a CTA handles.  The map's grid (gx x gy, x fastest) lists the
// T = nb(nb+1)/2 tiles of the 2-simplex of blocks in its order (zero, one
// or two per grid block); that sequence is cut into N = q gridDim.x chunks
// of equal size (chunk c holds tiles floor(c T / N) .. floor((c+1) T / N) - 1,
// so sizes differ by one tile at most, about kChunk each), and in round k
// CTA b takes chunk k gridDim.x + (b + k) mod gridDim.x (the rotation mixes
// the chunk sizes each CTA gets): every CTA gets the same number of tiles,
// whatever the map's idle grid blocks or two-tile rows (the lambda map's
// diagonal-pair row, the bounding box's empty upper half).  A prologue scans
// the tiles of the grid blocks and finds each chunk's first grid block.
// Along a grid row the row block Y stays fixed for runs of tiles (with the
// lambda map for 2^floor(log2 wy) consecutive grid blocks of row wy), so
// within a chunk G_Y accumulates over runs of up to kChunk tiles.
constexpr int kChunk = 32;
constexpr int kScanBlock = 1024;   // grid blocks per block of the scan

template <int MAP>
__device__ __forceinline__ List2 decode_grid2(int64_t w, int wx, int wy, int nb) {
    return MAP == MAP_LINEAR ? decode2_linear(w, nb) : decode2<MAP>((uint32_t)wx, (uint32_t)wy, nb);
}

// Tiles of each grid block: their exclusive prefix within each scan block
// (loc) and each scan block's total (bsum).
template <int MAP>
__global__ void __launch_bounds__(kScanBlock) k_tile_scan(int64_t total, int gx, int nb, int *__restrict__ loc,
                                                          int64_t *__restrict__ bsum) {
    __shared__ int wsum[kScanBlock / 32];
    const int64_t w = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
    int c = 0;
    if (w < total) {
        const int wy = (int)(w / gx), wx = (int)(w - (int64_t)wy * gx);
        c = decode_grid2<MAP>(w, wx, wy, nb).cnt;
    }
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    int v = c;   // inclusive scan within the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    if (lane == 31) wsum[wp] = v;
    __syncthreads();
    if (wp == 0) {
        int t = wsum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += u;
        }
        wsum[lane] = t;   // inclusive over warps
    }
    __syncthreads();
    const int before = wp ? wsum[wp - 1] : 0;
    if (w < total) loc[w] = before + v - c;
    if (threadIdx.x == kScanBlock - 1) bsum[blockIdx.x] = wsum[31];
}

// Exclusive prefix of the scan blocks' totals, in place (one block).
__global__ void __launch_bounds__(1024) k_bsum_scan(int64_t nblk, int64_t *__restrict__ bsum) {
    __shared__ int64_t part[32];
    int64_t carry = 0;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    for (int64_t base = 0; base < nblk; base += 1024) {
        const int64_t i = base + threadIdx.x;
        const int64_t c = i < nblk ? bsum[i] : 0;
        int64_t v = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t u = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += u;
        }
        if (lane == 31) part[wp] = v;
        __syncthreads();
        if (wp == 0) {
            int64_t t = part[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t u = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += u;
            }
            part[lane] = t;
        }
        __syncthreads();
        const int64_t before = carry + (wp ? part[wp - 1] : 0);
        if (i < nblk) bsum[i] = before + v - c;
        carry += part[31];
        __syncthreads();
    }
}

// First tile of each chunk: 2 w + s for grid block w and its tile s.  The
// tile r = floor(c T / N) lies in the last grid block whose prefix is <= r
// (a block after it with no tile has the same prefix, so that block holds
// tiles): a binary search over the scan blocks, then within one.
__global__ void __launch_bounds__(256) k_chunk_starts(int64_t total, int64_t nblk, int64_t T, int64_t N,
                                                      const int *__restrict__ loc,
                                                      const int64_t *__restrict__ boff, int64_t *__restrict__ start) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const int64_t r = c * T / N;
    int64_t lo = 0, hi = nblk - 1;   // last scan block with boff <= r
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (boff[mid] <= r) lo = mid; else hi = mid - 1;
    }
    const int64_t b = lo, rr = r - boff[b];
    int64_t a = b * kScanBlock, z = (b + 1) * kScanBlock < total ? (b + 1) * kScanBlock - 1 : total - 1;
    while (a < z) {
        const int64_t mid = (a + z + 1) >> 1;
        if (loc[mid] <= rr) a = mid; else z = mid - 1;
    }
    start[c] = 2 * a + (rr - loc[a]);
}

template <int MAP>
struct ChunkWalk {
    const int64_t *start;
    int64_t k, c, w, T, N;
    int left, sub, wx, wy, gx, nb;
    __device__ ChunkWalk(int gx_, int nb_, int64_t T_, int64_t N_, const int64_t *start_)
        : start(start_), k(0), T(T_), N(N_), left(0), gx(gx_), nb(nb_) {
        open();
    }
    __device__ void open() {
        c = k * gridDim.x + (blockIdx.x + k) % gridDim.x;
        if (c >= N) { left = 0; return; }
        const int64_t s0 = start[c];
        w = s0 >> 1;
        sub = (int)(s0 & 1);
        left = (int)((c + 1) * T / N - c * T / N);
        wy = (int)(w / gx);
        wx = (int)(w - (int64_t)wy * gx);
    }
    __device__ bool next(int &X, int &Y) {
        for (;;) {
            if (left == 0) {
                ++k;
                if (k * gridDim.x >= N) return false;
                open();
                continue;
            }
            const List2 L = decode_grid2<MAP>(w, wx, wy, nb);
            if (sub < L.cnt) {
                X = sub ? L.x[1] : L.x[0];
                Y = sub ? L.y[1] : L.y[0];
                ++sub;
                --left;
                return true;
            }
            ++w;
            sub = 0;
            if (++wx == gx) { wx = 0; ++wy; }
        }
    }
};

// Next ring stage for the producer: waits until it is free and arms it for
// `bytes` of TMA data.
template <int S>
__device__ __forceinline__ bool ring_acquire(Ctl &ctl, uint32_t s_stages, uint32_t &it,
                                             uint32_t bytes, uint32_t &dst, uint32_t &bar,
                                             volatile int *fail) {
    const uint32_t s = it % S, ph = (it / S) & 1;
    if (!mbar_wait(smem_u32(&ctl.empty[s]), ph ^ 1, fail, &g_error)) return false;
    bar = smem_u32(&ctl.full[s]);
    dst = s_stages + s * STAGE_BYTES;
    mbar_expect_tx(bar, bytes);
    ++it;
    return true;
}

// Next ring stage for the MMA issuer: waits until its data has landed.
template <int S>
__device__ __forceinline__ bool ring_take(Ctl &ctl, uint32_t s_stages, uint32_t it, uint32_t &src,
                                          volatile int *fail) {
    const uint32_t s = it % S;
    if (!mbar_wait(smem_u32(&ctl.full[s]), (it / S) & 1, fail, &g_error)) return false;
    tc_fence_after();
    src = s_stages + s * STAGE_BYTES;
    return true;
}

// Coordinates of block B as X^T tiles: rows t = 0 .. NG-1, columns
// B*128 .. B*128 + 127 as two 64-column boxes, hi then lo.
__device__ __forceinline__ void load_xt(const CUtensorMap *mh, const CUtensorMap *ml, int B,
                                        uint32_t dst, uint32_t box, uint32_t bar) {
    tma_load_2d(dst, mh, B * TN, 0, bar);
    tma_load_2d(dst + box, mh, B * TN + 64, 0, bar);
    tma_load_2d(dst + 2 * box, ml, B * TN, 0, bar);
    tma_load_2d(dst + 3 * box, ml, B * TN + 64, 0, bar);
}

// The sides of a finished accumulator (rows of block B, or its columns):
// grad_p = scale4 (S_p x_p - sum_q c_pq x_q) with S_p = sum_q c_pq, so the
// flush adds -scale4 G[row][0:d] to grad (FP32 vector atomics, nothing
// read back) and the row's sum G[row][d] to S[row]; a last pass adds
// scale4 S_p x_p (k_stress_sx), so no coordinate is loaded here.  This
// thread: its lane quarter's row, its half of the d coordinates (the sum
// once, by half 0).  All lanes execute the TMEM loads.
__device__ __forceinline__ void flush_g(uint32_t tmem, uint32_t gcol, int B, int quarter, int half,
                                        int lane, int d, int64_t n, float scale4, float *__restrict__ grad,
                                        float *__restrict__ S) {
    const uint32_t tl = tmem + ((uint32_t)(32 * quarter) << 16) + gcol;
    const float s = tmem_ld1(tl + (uint32_t)d);
    const int64_t row = (int64_t)B * TM + 32 * quarter + lane;
    const int hw = d >> 1;
    for (int c = 0; c < hw; c += 16) {
        float v[16];
        tmem_ld16(tl + (uint32_t)(half * hw + c), v);
        if (row < n) {
            float *gr = grad + row * d + half * hw + c;
#pragma unroll
            for (int q = 0; q < 16; q += 4)
                atomicAdd(reinterpret_cast<float4 *>(gr + q),
                          make_float4(-scale4 * v[q], -scale4 * v[q + 1], -scale4 * v[q + 2], -scale4 * v[q + 3]));
        }
    }
    if (half == 0 && row < n) atomicAdd(S + row, s);
}

// grad_p += scale4 S_p x_p, the row-sum part of every flush (see flush_g).
__global__ void __launch_bounds__(256) k_stress_sx(const float *__restrict__ x, const float *__restrict__ S,
                                                   int64_t n, int d, float scale4, float *__restrict__ grad) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;   // float4 of grad
    if (e >= n * d / 4) return;
    const int64_t p = 4 * e / d;
    const float f = scale4 * S[p];
    const float4 xv = reinterpret_cast<const float4 *>(x)[e];
    float4 g = reinterpret_cast<float4 *>(grad)[e];
    g.x = fmaf(f, xv.x, g.x); g.y = fmaf(f, xv.y, g.y); g.z = fmaf(f, xv.z, g.z); g.w = fmaf(f, xv.w, g.w);
    reinterpret_cast<float4 *>(grad)[e] = g;
}

// a = S . Delta of a tile's columns col0 + 64 half + lane and + 32 (ca, cb)
// and of its row row0 + r (ri), for one epilogue thread; 0 past n.
__device__ __forceinline__ void load_a(const float *__restrict__ a, int64_t n, int X, int Y, int half,
                                       int r, int lane, float &ca, float &cb, float &ri) {
    const int64_t j0 = (int64_t)X * TN + 64 * half + lane, j1 = j0 + 32, i = (int64_t)Y * TM + r;
    ca = j0 < n ? __ldg(a + j0) : 0.0f;
    cb = j1 < n ? __ldg(a + j1) : 0.0f;
    ri = i < n ? __ldg(a + i) : 0.0f;
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&h);
}

// The backward kernel (gradient): 128 x 128 tiles, GEMM1 then GEMM2.  With
// `partials` it also sums the loss from the same residual tiles (one FP64
// partial per CTA): loss and gradient in one pass.
template <int MAP>
__global__ void __launch_bounds__(kThreads, 1)
    k_stress_umma_bwd(const __grid_constant__ CUtensorMap mPh, const __grid_constant__ CUtensorMap mPl,
                      const __grid_constant__ CUtensorMap mQh, const __grid_constant__ CUtensorMap mQl,
                      const __grid_constant__ CUtensorMap mTh, const __grid_constant__ CUtensorMap mTl,
                      float *__restrict__ S, const float *__restrict__ a, int64_t n, int d, int nb,
                      int gx, int64_t T, int64_t nchunks, const int64_t *__restrict__ start,
                      float scale4, float *__restrict__ grad, double *__restrict__ partials, int qshift) {
    using Walk = ChunkWalk<MAP>;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    constexpr int NS = kStages;
    unsigned char *cbuf = base + kStages * STAGE_BYTES;   // the C tile
    Ctl &ctl = *reinterpret_cast<Ctl *>(cbuf + C_BYTES);
    const uint32_t s_stages = smem_u32(base), s_c = smem_u32(cbuf);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    volatile int *fail = &ctl.fail;
    const int NG = d + 16;                       // GEMM2 N: d coordinates, the ones row, zero rows
    const int nc1 = (2 * d) / KC;                // GEMM1 K chunks
    const uint32_t xt_box = (uint32_t)NG * 128;  // bytes of one 64-column X^T box

    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(smem_u32(&ctl.full[s]), 1);
            mbar_init(smem_u32(&ctl.empty[s]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&ctl.tfull[b]), 1);
            mbar_init(smem_u32(&ctl.tempty[b]), kEpiWarps);
        }
        mbar_init(smem_u32(&ctl.cready), kEpiWarps);
        mbar_init(smem_u32(&ctl.g2done), 1);
        mbar_init(smem_u32(&ctl.gxfree[0]), kEpiWarps);
        mbar_init(smem_u32(&ctl.gxfree[1]), kEpiWarps);
        mbar_init(smem_u32(&ctl.gyfree), kEpiWarps);
        mbar_init(smem_u32(&ctl.done), 1);
        ctl.fail = *reinterpret_cast<volatile int *>(&g_error) ? 1 : 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        prefetch_map(&mPh);
        prefetch_map(&mPl);
        prefetch_map(&mQh);
        prefetch_map(&mQl);
        prefetch_map(&mTh);
        prefetch_map(&mTl);
    }
    if (warp == 1) tmem_alloc(smem_u32(&ctl.tmem), kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = ctl.tmem;
    float lhi = 0.f, llo = 0.f;   // loss partial (with `partials`)

    if (warp == 0) {
        // ---------------- TMA producer
        if (lane == 0) {
            Walk walk(gx, nb, T, nchunks, start);
            uint32_t it = 0, dst, bar;
            int X, Y, pX = 0, pY = 0;
            bool ok = true, have = false;
            while (ok && !*fail && walk.next(X, Y)) {
                for (int c = 0; c < nc1; ++c) {
                    if (!(ok = ring_acquire<NS>(ctl, s_stages, it, STAGE_BYTES, dst, bar, fail))) break;
                    tma_load_2d(dst, &mPh, c * KC, Y * TM, bar);
                    tma_load_2d(dst + TILE_BYTES, &mPl, c * KC, Y * TM, bar);
                    const int qx = (c * KC + qshift) % (2 * d);   // Q chunk c (qshift: Q read from P)
                    tma_load_2d(dst + 2 * TILE_BYTES, &mQh, qx, X * TN, bar);
                    tma_load_2d(dst + 3 * TILE_BYTES, &mQl, qx, X * TN, bar);
                }
                if (ok && have) {
                    // GEMM2 operands of the previous tile: X^T of its columns, then of its rows
                    if ((ok = ring_acquire<NS>(ctl, s_stages, it, 4 * xt_box, dst, bar, fail)))
                        load_xt(&mTh, &mTl, pX, dst, xt_box, bar);
                    if (ok && (ok = ring_acquire<NS>(ctl, s_stages, it, 4 * xt_box, dst, bar, fail)))
                        load_xt(&mTh, &mTl, pY, dst, xt_box, bar);
                }
                pX = X; pY = Y; have = true;
            }
            if (ok && !*fail && have) {
                if ((ok = ring_acquire<NS>(ctl, s_stages, it, 4 * xt_box, dst, bar, fail)))
                    load_xt(&mTh, &mTl, pX, dst, xt_box, bar);
                if (ok && (ok = ring_acquire<NS>(ctl, s_stages, it, 4 * xt_box, dst, bar, fail)))
                    load_xt(&mTh, &mTl, pY, dst, xt_box, bar);
            }
            // a failed block waits (bounded) for the loads it may have in flight
            if (*fail)
                for (uint32_t k = it > (uint32_t)NS ? it - NS : 0; k < it; ++k)
                    mbar_drain(smem_u32(&ctl.full[k % NS]), (k / NS) & 1);
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer: the whole warp, converged, so the
        // descriptors stay warp-uniform; one elected lane issues each BF16
        // step's three products at once, from descriptors stepped off a
        // per-stage base.  The warp shares its scheduler with two epilogue
        // warps and a 128 x 80 x 16 MMA of GEMM2 runs about 40 cycles, so the
        // instructions between MMAs decide whether the tensor pipe idles.
        {
            const uint32_t id1 = idesc_bf16(TM, TN, false, false);
            const uint32_t id_row = idesc_bf16(TM, NG, false, false);
            const uint32_t id_col = idesc_bf16(TM, NG, true, false);
            const uint64_t dc = sw128_desc(s_c);                     // C, K-major (rows side)
            const uint64_t dct = sw128_desc(s_c, TILE_BYTES, 1024);  // C read M-major (columns side)
            Walk walk(gx, nb, T, nchunks, start);
            uint32_t it = 0, t = 0, src;
            int X, Y, prevY = -1, prev2Y = -1;
            bool ok = true;
            const int ngx = gx_buffers(NG);
            uint32_t runs = 0;   // run changes after the first tile
            // GEMM2 of tile u (its row block continues the previous tile's run if
            // sameY).  Waits: C tile written; this tile's G_X buffer read out (the
            // flush of tile u - ngx); G_Y read out when a new run starts.
            auto gemm2 = [&](uint32_t u, bool sameY) -> bool {
                if (!mbar_wait(smem_u32(&ctl.cready), u & 1, fail, &g_error)) return false;
                const uint32_t b = u % (uint32_t)ngx;
                if (u >= (uint32_t)ngx &&
                    !mbar_wait(smem_u32(&ctl.gxfree[b]), (u / (uint32_t)ngx - 1) & 1, fail, &g_error))
                    return false;
                if (u >= 1 && !sameY) {
                    ++runs;
                    if (!mbar_wait(smem_u32(&ctl.gyfree), (runs - 1) & 1, fail, &g_error)) return false;
                }
                tc_fence_after();
                const uint32_t tgx = tmem + kGY + (uint32_t)NG * (1 + b);
                // rows: G_Y (+)= C [X_X | 1], K = j over the two column halves of C
                if (!ring_take<NS>(ctl, s_stages, it, src, fail)) return false;
                const uint64_t dx = sw128_desc(src);
#pragma unroll
                for (int h = 0; h < 2; ++h)
#pragma unroll
                    for (int ks = 0; ks < KC / 16; ++ks) {
                        const uint32_t acc = (h == 0 && ks == 0 && !sameY) ? 0u : 1u;
                        mma_bf16x3_w(tmem + kGY, desc_add(dc, h * TILE_BYTES + ks * 32),
                                     desc_add(dc, (2 + h) * TILE_BYTES + ks * 32),
                                     desc_add(dx, h * xt_box + ks * 32), desc_add(dx, (2 + h) * xt_box + ks * 32),
                                     id_row, acc);
                    }
                mma_commit_w(smem_u32(&ctl.empty[it % NS]));
                ++it;
                // columns: G_X = C^T [X_Y | 1], K = i; A is C read M-major (M = j
                // over the two 64-column halves, LBO = one half tile apart)
                if (!ring_take<NS>(ctl, s_stages, it, src, fail)) return false;
                const uint64_t dy = sw128_desc(src);
#pragma unroll
                for (int ks = 0; ks < TM / 16; ++ks) {
                    const uint32_t hb = (uint32_t)(ks >> 2), kb = (uint32_t)(ks & 3) * 32;
                    mma_bf16x3_w(tgx, desc_add(dct, ks * 2048), desc_add(dct, 2 * TILE_BYTES + ks * 2048),
                                 desc_add(dy, hb * xt_box + kb), desc_add(dy, (2 + hb) * xt_box + kb), id_col,
                                 ks ? 1u : 0u);
                }
                mma_commit_w(smem_u32(&ctl.empty[it % NS]));
                ++it;
                mma_commit_w(smem_u32(&ctl.g2done));
                return true;
            };
            while (ok && !*fail && walk.next(X, Y)) {
                const uint32_t acc = t & 1, aph = (t >> 1) & 1;
                if (!(ok = mbar_wait(smem_u32(&ctl.tempty[acc]), aph ^ 1, fail, &g_error))) break;
                tc_fence_after();
                const uint32_t dtm = tmem + acc * TN;
                for (int c = 0; c < nc1; ++c) {
                    if (!(ok = ring_take<NS>(ctl, s_stages, it, src, fail))) break;
                    const uint64_t d0 = sw128_desc(src);   // P hi, P lo, Q hi, Q lo tiles of the stage
#pragma unroll
                    for (int ks = 0; ks < KC / 16; ++ks) {
                        const uint32_t ko = ks * 32;
                        mma_bf16x3_w(dtm, desc_add(d0, ko), desc_add(d0, TILE_BYTES + ko),
                                     desc_add(d0, 2 * TILE_BYTES + ko), desc_add(d0, 3 * TILE_BYTES + ko), id1,
                                     (c > 0 || ks > 0) ? 1u : 0u);
                    }
                    mma_commit_w(smem_u32(&ctl.empty[it % NS]));
                    ++it;
                }
                if (!ok) break;
                mma_commit_w(smem_u32(&ctl.tfull[acc]));
                if (t >= 1 && !(ok = gemm2(t - 1, t >= 2 && prevY == prev2Y))) break;
                prev2Y = prevY;
                prevY = Y;
                ++t;
            }
            if (ok && !*fail && t >= 1) gemm2(t - 1, t >= 2 && prevY == prev2Y);
            // everything issued has completed before the block releases TMEM
            mma_commit_w(smem_u32(&ctl.done));
            mbar_drain(smem_u32(&ctl.done), 0);
        }
    } else {
        // ---------------- epilogue: 8 warps, two per TMEM lane quarter
        const int ew = warp - 2;                 // 0..7
        const int quarter = warp & 3;            // TMEM lanes 32*quarter .. +31
        const int half = ew >> 2;                // columns [64*half, 64*half + 64)
        const int r = 32 * quarter + lane;       // this thread's row in the tile
        float *ac = &ctl.acol[ew][0];
        const int ngx = gx_buffers(NG);
        unsigned char *rowh = cbuf + half * TILE_BYTES + (r >> 3) * 1024 + (r & 7) * 128;
        unsigned char *rowl = rowh + 2 * TILE_BYTES;
        Walk walk(gx, nb, T, nchunks, start);
        uint32_t t = 0;
        int X, Y, pX = 0, pY = 0;
        bool have = walk.next(X, Y);
        // a of the current tile's columns (va, vb) and row (vi), loaded a tile ahead
        float va = 0.f, vb = 0.f, vi = 0.f;
        if (have) load_a(a, n, X, Y, half, r, lane, va, vb, vi);
        while (have && !*fail) {
            int Xn, Yn;
            const bool hn = walk.next(Xn, Yn);
            float na = 0.f, nbv = 0.f, ni = 0.f;
            if (hn) load_a(a, n, Xn, Yn, half, r, lane, na, nbv, ni);
            const uint32_t acc = t & 1, aph = (t >> 1) & 1;
            const int64_t row0 = (int64_t)Y * TM, jb = (int64_t)X * TN + 64 * half;
            __syncwarp();   // the previous tile's reads of ac are done
            ac[lane] = va;
            ac[lane + 32] = vb;
            const int64_t i = row0 + r;
            const float ai = vi;
            // valid columns q < lim: j < n, and j < i on a diagonal tile
            int64_t lim64 = i < n ? n - jb : 0;
            if (X == Y && i - jb < lim64) lim64 = i - jb;
            const int lim = lim64 < 0 ? 0 : (lim64 > 64 ? 64 : (int)lim64);
            __syncwarp();
            if (!mbar_wait(smem_u32(&ctl.tfull[acc]), aph, fail, &g_error)) break;
            tc_fence_after();
            float v[64];
            {
                float v0[32], v1[32];
                const uint32_t taddr = tmem + acc * TN + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(64 * half);
                tmem_ld64(taddr, v0, v1);
#pragma unroll
                for (int q = 0; q < 32; ++q) { v[q] = v0[q]; v[32 + q] = v1[q]; }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&ctl.tempty[acc]));
#pragma unroll
            for (int q = 0; q < 64; q += 4) {
                const float4 aj = *reinterpret_cast<const float4 *>(ac + q);
                const float al4[4] = {aj.x, aj.y, aj.z, aj.w};
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float rq = (ai + al4[k]) - v[q + k];
                    v[q + k] = q + k < lim ? rq : 0.0f;
                }
            }
            if (partials) {   // the loss from the same residuals (loss and gradient in one pass)
                float sq = 0.f;
#pragma unroll
                for (int q = 0; q < 64; ++q) sq = fmaf(v[q], v[q], sq);
                add_ff(lhi, llo, sq, 0.f);
            }
            // the C buffer is free once GEMM2 of the previous tile has completed
            if (t >= 1 && !mbar_wait(smem_u32(&ctl.g2done), (t - 1) & 1, fail, &g_error)) break;
            tc_fence_after();
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                uint32_t ph[4], pl[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float f0 = v[8 * c + 2 * k], f1 = v[8 * c + 2 * k + 1];
                    const __nv_bfloat162 hh = __floats2bfloat162_rn(f0, f1);   // both rounded at once
                    ph[k] = *reinterpret_cast<const uint32_t *>(&hh);
                    pl[k] = pack_bf16(f0 - __low2float(hh), f1 - __high2float(hh));
                }
                const int off = (c ^ (r & 7)) << 4;
                *reinterpret_cast<uint4 *>(rowh + off) = make_uint4(ph[0], ph[1], ph[2], ph[3]);
                *reinterpret_cast<uint4 *>(rowl + off) = make_uint4(pl[0], pl[1], pl[2], pl[3]);
            }
            fence_proxy_async();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&ctl.cready));
            if (t >= 1) {
                // the previous tile's sides: its columns always, its rows at the end of a run
                const uint32_t pb = (t - 1) % (uint32_t)ngx;
                flush_g(tmem, kGY + NG * (1 + pb), pX, quarter, half, lane, d, n, scale4, grad, S);
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&ctl.gxfree[pb]));
                if (Y != pY) {
                    flush_g(tmem, kGY, pY, quarter, half, lane, d, n, scale4, grad, S);
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(smem_u32(&ctl.gyfree));
                }
            }
            pX = X;
            pY = Y;
            X = Xn; Y = Yn; have = hn;
            va = na; vb = nbv; vi = ni;
            ++t;
        }
        if (!*fail && t >= 1 &&
            mbar_wait(smem_u32(&ctl.g2done), (t - 1) & 1, fail, &g_error)) {
            tc_fence_after();
            flush_g(tmem, kGY + NG * (1 + (t - 1) % (uint32_t)ngx), pX, quarter, half, lane, d, n, scale4,
                    grad, S);
            flush_g(tmem, kGY, pY, quarter, half, lane, d, n, scale4, grad, S);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tmem, kTmemCols);
    }
    if (partials) {
        const double s = block_sum_ff<kThreads>(lhi, llo, ctl.red);
        if (tid == 0) partials[blockIdx.x] = s;
    }
}

// ---------------------------------------------------------------- forward in 128 x 256 steps

// The forward kernel in 128 x 256 steps.  A two-CTA cluster walks the map's
// grid of 256 x 256 super-blocks (sX, sY); CTA r computes row block
// Y = 2 sY + r against both column blocks 2 sX and 2 sX + 1 with M = 128,
// N = 256 MMAs (both column blocks in one 256-row B operand).  Each CTA
// loads its own row block's P tiles and multicasts the Q tiles of column
// block 2 sX + r into both CTAs, so per K chunk a CTA reads 64 KB from L2 for
// 128 x 256 pairs (the 128 x 128 steps with a shared row block read 96 KB for
// two 128 x 128 tiles).  A quadrant above the diagonal (r = 0 on a diagonal
// super-block) or past the last block is computed and contributes nothing.
namespace f256 {

constexpr int TN2 = 2 * TN;                    // 256 columns per step
constexpr int A_BYTES = TILE_BYTES;            // 16 KB: 128 rows x 64 BF16
constexpr int B_BYTES = 2 * TILE_BYTES;        // 32 KB: 256 rows x 64 BF16
constexpr int STAGE = 2 * A_BYTES + 2 * B_BYTES;   // 96 KB: P hi, P lo, Q hi, Q lo
constexpr int NS = 2;

struct Ctl2 {
    uint64_t full[NS], empty[NS];   // ring: TMA -> MMA -> TMA (both CTAs release a stage)
    uint64_t tfull[2], tempty[2];   // accumulators: MMA -> epilogue -> MMA
    uint64_t done;                  // every MMA of the block complete
    uint32_t tmem;
    int fail;
    alignas(16) float acol[kEpiWarps][TN];   // a_j of each epilogue warp's 128 columns
    float red[2 * (kThreads / 32)];
};

constexpr int kCtl2Bytes = 8192;
constexpr int SMEM2 = 1024 + NS * STAGE + kCtl2Bytes;
static_assert(sizeof(Ctl2) <= kCtl2Bytes, "control block");
static_assert(SMEM2 <= 227 * 1024, "shared memory per block");
static_assert(2 * TN2 <= kTmemCols, "two accumulators of 256 columns");

template <int MAP>
__global__ void __launch_bounds__(kThreads, 1)
    k_stress_umma_fwd(const __grid_constant__ CUtensorMap mPh, const __grid_constant__ CUtensorMap mPl,
                    const __grid_constant__ CUtensorMap mQh, const __grid_constant__ CUtensorMap mQl,
                    const float *__restrict__ a, int64_t n, int d, int nb, int nb2, int gx,
                    int64_t total, double *__restrict__ partials, int qshift) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    Ctl2 &ctl = *reinterpret_cast<Ctl2 *>(base + NS * STAGE);
    const uint32_t s_stages = smem_u32(base);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    volatile int *fail = &ctl.fail;
    const int nc1 = (2 * d) / KC;   // K chunks
    const uint32_t rank = cluster_rank();

    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(smem_u32(&ctl.full[s]), 1);
            mbar_init(smem_u32(&ctl.empty[s]), 2);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&ctl.tfull[b]), 1);
            mbar_init(smem_u32(&ctl.tempty[b]), kEpiWarps);
        }
        mbar_init(smem_u32(&ctl.done), 1);
        ctl.fail = *reinterpret_cast<volatile int *>(&g_error) ? 1 : 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        prefetch_map(&mPh);
        prefetch_map(&mPl);
        prefetch_map(&mQh);
        prefetch_map(&mQl);
    }
    if (warp == 1) tmem_alloc(smem_u32(&ctl.tmem), kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    cluster_sync();   // the peer's barriers exist before any multicast reaches them
    const uint32_t tmem = ctl.tmem;
    float lhi = 0.f, llo = 0.f;

    if (warp == 0) {
        // ---------------- TMA producer
        if (lane == 0) {
            SuperWalk<MAP> walk(gx, total, nb2);
            uint32_t it = 0;
            int sX, sY;
            bool ok = true;
            while (ok && !*fail && walk.next(sX, sY)) {
                const int Y = 2 * sY + (int)rank, Xr = 2 * sX + (int)rank;
                for (int c = 0; c < nc1; ++c) {
                    const uint32_t s = it % NS, ph = (it / NS) & 1;
                    // free once both CTAs' MMAs have read the stage
                    if (!(ok = mbar_wait(smem_u32(&ctl.empty[s]), ph ^ 1, fail, &g_error))) break;
                    const uint32_t bar = smem_u32(&ctl.full[s]), dst = s_stages + s * STAGE;
                    mbar_expect_tx(bar, STAGE);
                    tma_load_2d(dst, &mPh, c * KC, Y * TM, bar);
                    tma_load_2d(dst + A_BYTES, &mPl, c * KC, Y * TM, bar);
                    // this CTA's column block, rows 128 r .. 128 r + 127 of both CTAs' B
                    const int qx = (c * KC + qshift) % (2 * d);   // Q chunk c (qshift: Q read from P)
                    tma_load_2d_mc(dst + 2 * A_BYTES + rank * TILE_BYTES, &mQh, qx, Xr * TN, bar, 3);
                    tma_load_2d_mc(dst + 2 * A_BYTES + B_BYTES + rank * TILE_BYTES, &mQl, qx, Xr * TN,
                                   bar, 3);
                    ++it;
                }
            }
            // a failed block waits (bounded) for the loads it may have in flight
            if (*fail)
                for (uint32_t k = it > (uint32_t)NS ? it - NS : 0; k < it; ++k)
                    mbar_drain(smem_u32(&ctl.full[k % NS]), (k / NS) & 1);
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer
        {   // the whole warp, converged; one elected lane issues
            const uint32_t id = idesc_bf16(TM, TN2, false, false);
            SuperWalk<MAP> walk(gx, total, nb2);
            uint32_t it = 0, t = 0;
            int sX, sY;
            bool ok = true;
            while (ok && !*fail && walk.next(sX, sY)) {
                const uint32_t acc = t & 1, aph = (t >> 1) & 1;
                if (!(ok = mbar_wait(smem_u32(&ctl.tempty[acc]), aph ^ 1, fail, &g_error))) break;
                tc_fence_after();
                const uint32_t dtm = tmem + acc * TN2;
                for (int c = 0; c < nc1; ++c) {
                    const uint32_t s = it % NS;
                    if (!(ok = mbar_wait(smem_u32(&ctl.full[s]), (it / NS) & 1, fail, &g_error))) break;
                    tc_fence_after();
                    const uint32_t src = s_stages + s * STAGE;
                    const uint64_t d0 = sw128_desc(src);
#pragma unroll
                    for (int ks = 0; ks < KC / 16; ++ks) {
                        const uint32_t ko = ks * 32;
                        mma_bf16x3_w(dtm, desc_add(d0, ko), desc_add(d0, A_BYTES + ko), desc_add(d0, 2 * A_BYTES + ko),
                                     desc_add(d0, 2 * A_BYTES + B_BYTES + ko), id, (c > 0 || ks > 0) ? 1u : 0u);
                    }
                    // the stage is free once this CTA's MMAs and the peer's have read it
                    mma_commit_mc_w(smem_u32(&ctl.empty[s]), 3);
                    ++it;
                }
                if (!ok) break;
                mma_commit_w(smem_u32(&ctl.tfull[acc]));
                ++t;
            }
            // everything issued has completed before the block releases TMEM
            mma_commit_w(smem_u32(&ctl.done));
            mbar_drain(smem_u32(&ctl.done), 0);
        }
    } else {
        // ---------------- epilogue: 8 warps, two per TMEM lane quarter, one
        // column block each
        const int ew = warp - 2;                 // 0..7
        const int quarter = warp & 3;            // TMEM lanes 32*quarter .. +31
        const int h = ew >> 2;                   // column block 2 sX + h: accumulator columns 128 h ..
        const int r = 32 * quarter + lane;       // this thread's row in the tile
        float *ac = &ctl.acol[ew][0];
        SuperWalk<MAP> walk(gx, total, nb2);
        uint32_t t = 0;
        int sX, sY;
        while (!*fail && walk.next(sX, sY)) {
            const int Y = 2 * sY + (int)rank, X = 2 * sX + h;
            const uint32_t acc = t & 1, aph = (t >> 1) & 1;
            const int64_t i = (int64_t)Y * TM + r, jb = (int64_t)X * TN;
            __syncwarp();   // the previous step's reads of ac are done
#pragma unroll
            for (int q = 0; q < TN; q += 32) {
                const int64_t j = jb + q + lane;
                ac[q + lane] = j < n ? __ldg(a + j) : 0.0f;
            }
            const float ai = i < n ? __ldg(a + i) : 0.0f;
            // valid columns q < lim: j < n, j < i on a diagonal tile; none above
            // the diagonal or past the last block
            int64_t lim64 = (i < n && X <= Y && Y < nb) ? n - jb : 0;
            if (X == Y && i - jb < lim64) lim64 = i - jb;
            const int lim = lim64 < 0 ? 0 : (lim64 > TN ? TN : (int)lim64);
            __syncwarp();
            if (!mbar_wait(smem_u32(&ctl.tfull[acc]), aph, fail, &g_error)) break;
            tc_fence_after();
            float sq = 0.f;
#pragma unroll
            for (int part = 0; part < 2; ++part) {
                float v0[32], v1[32];
                const uint32_t taddr = tmem + acc * TN2 + ((uint32_t)(32 * quarter) << 16) +
                                       (uint32_t)(TN * h + 64 * part);
                tmem_ld64(taddr, v0, v1);
#pragma unroll
                for (int q = 0; q < 32; q += 4) {
                    const int c0 = 64 * part + q;
                    const float4 a0 = *reinterpret_cast<const float4 *>(ac + c0);
                    const float4 a1 = *reinterpret_cast<const float4 *>(ac + c0 + 32);
                    const float x0[4] = {a0.x, a0.y, a0.z, a0.w}, x1[4] = {a1.x, a1.y, a1.z, a1.w};
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        float r0 = (ai + x0[k]) - v0[q + k];
                        float r1 = (ai + x1[k]) - v1[q + k];
                        r0 = c0 + k < lim ? r0 : 0.0f;
                        r1 = c0 + 32 + k < lim ? r1 : 0.0f;
                        sq = fmaf(r0, r0, sq);
                        sq = fmaf(r1, r1, sq);
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&ctl.tempty[acc]));
            add_ff(lhi, llo, sq, 0.f);
            ++t;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tmem, kTmemCols);
    }
    const double s = block_sum_ff<kThreads>(lhi, llo, ctl.red);
    if (tid == 0) partials[blockIdx.x] = s;
    // neither CTA of a pair leaves while the other may still multicast into
    // its shared memory or arrive on its barriers
    cluster_sync();
}

}  // namespace f256

// P = [S | Delta], Q = [Delta | S] (BF16 hi, lo; rows of 2d; Q only when
// Qh is given), a = S . Delta in FP32, and for the backward pass X^T hi, lo (rows t < d: coordinates; row d:
// ones; rows d+1 .. NG-1: zeros; row pitch `pitch`).  32 points per block.
__global__ void __launch_bounds__(256) k_stress_prep(const float *__restrict__ x,
                                                     const float *__restrict__ y, int64_t n, int d,
                                                     int NG, int64_t pitch,
                                                     __nv_bfloat16 *__restrict__ Ph,
                                                     __nv_bfloat16 *__restrict__ Pl,
                                                     __nv_bfloat16 *__restrict__ Qh,
                                                     __nv_bfloat16 *__restrict__ Ql,
                                                     __nv_bfloat16 *__restrict__ Th,
                                                     __nv_bfloat16 *__restrict__ Tl,
                                                     float *__restrict__ a) {
    __shared__ float xs[32][97];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i0 = (int64_t)blockIdx.x * 32;
    for (int p = warp; p < 32; p += 8) {
        const int64_t i = i0 + p;
        if (i >= n) break;
        float acc = 0.f;
        for (int t = lane; t < d; t += 32) {
            const float xv = __ldg(x + i * d + t), yv = __ldg(y + i * d + t);
            const float S = xv + yv, D = xv - yv;
            const __nv_bfloat16 sh = __float2bfloat16_rn(S), dh = __float2bfloat16_rn(D);
            const __nv_bfloat16 sl = __float2bfloat16_rn(S - __bfloat162float(sh));
            const __nv_bfloat16 dl = __float2bfloat16_rn(D - __bfloat162float(dh));
            const int64_t o = i * 2 * d + t;
            Ph[o] = sh; Pl[o] = sl; Ph[o + d] = dh; Pl[o + d] = dl;
            if (Qh) { Qh[o] = dh; Ql[o] = dl; Qh[o + d] = sh; Ql[o + d] = sl; }
            acc = fmaf(S, D, acc);
            xs[p][t] = xv;
        }
        acc = warp_sum_f32(acc);
        if (lane == 0) a[i] = acc;
    }
    if (Th) {
        __syncthreads();
        for (int e = threadIdx.x; e < NG * 32; e += 256) {
            const int t = e >> 5, p = e & 31;
            const int64_t i = i0 + p;
            if (i >= n) continue;
            const float v = t < d ? xs[p][t] : (t == d ? 1.0f : 0.0f);
            const __nv_bfloat16 h = __float2bfloat16_rn(v);
            Th[t * pitch + i] = h;
            Tl[t * pitch + i] = __float2bfloat16_rn(v - __bfloat162float(h));
        }
    }
}

struct Layout {
    int64_t Ph, Pl, Qh, Ql, Th, Tl, a, part, edm, deal, sums, total, pitch;
};

// The backward's chunks of the tile sequence: q per CTA, about kChunk
// tiles each and at least four per CTA.
static int64_t chunks_of(int64_t T, int64_t ctas) {
    int64_t q = (T + ctas * kChunk - 1) / (ctas * kChunk);
    return ctas * (q < 4 ? 4 : q);
}

static Layout layout_of(int64_t n, int64_t d, bool bwd) {
    Layout L;
    const int64_t pq = align_up(n * 2 * d * 2, 1024);
    L.pitch = align_up(n, 8);
    const int64_t xt = bwd ? align_up((d + 16) * L.pitch * 2, 1024) : 0;
    L.Ph = 0; L.Pl = pq; L.Qh = 2 * pq; L.Ql = 3 * pq;
    L.Th = 4 * pq; L.Tl = L.Th + xt;
    L.a = L.Tl + xt;
    L.part = L.a + align_up(n * 4, 1024);
    L.edm = L.part + align_up(8 * (kMaxCtas + kReduceSlots), 1024);
    L.deal = L.edm + ((!bwd && d % 64 == 0) ? edm_umma_workspace_bytes(n, d) : 0);
    // backward: the tile scan of the grid blocks (int each), the scan
    // blocks' offsets and the chunk starts (int64 each), for the largest
    // grid of any map and the most CTAs
    int64_t deal_bytes = 0;
    if (bwd) {
        const int64_t nb = (n + TM - 1) / TM;
        int64_t most = 0;
        for (int mp = MAP_LAMBDA; mp <= MAP_RB; ++mp) {
            const Grid g = grid2(nb, mp);
            if (g.gx * g.gy > most) most = g.gx * g.gy;
        }
        const int64_t nblk = (most + kScanBlock - 1) / kScanBlock;
        deal_bytes = align_up(4 * most, 1024) + align_up(8 * nblk, 1024) +
                     align_up(8 * chunks_of(nb * (nb + 1) / 2, kMaxCtas), 1024);
    }
    L.sums = L.deal + deal_bytes;   // backward: the per-point sums S of the flushes
    L.total = L.sums + (bwd ? align_up(4 * n, 1024) : 0);
    return L;
}

static cudaError_t optin_bwd() {
    const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_stress_umma_bwd<MAP_LAMBDA>, a, SMEM_BYTES)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_stress_umma_bwd<MAP_BBOX>, a, SMEM_BYTES)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_stress_umma_bwd<MAP_RB>, a, SMEM_BYTES)) != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_stress_umma_bwd<MAP_LINEAR>, a, SMEM_BYTES);
}

static cudaError_t optin_fwd256() {
    const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(f256::k_stress_umma_fwd<MAP_LAMBDA>, a, f256::SMEM2)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(f256::k_stress_umma_fwd<MAP_BBOX>, a, f256::SMEM2)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(f256::k_stress_umma_fwd<MAP_RB>, a, f256::SMEM2)) != cudaSuccess) return e;
    return cudaFuncSetAttribute(f256::k_stress_umma_fwd<MAP_LINEAR>, a, f256::SMEM2);
}

static int smem_optin() {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e);
    static std::mutex mu;
    static bool done[64] = {};
    if (dev < 0 || dev >= 64) return SIMPLEX_EUNSUPPORTED;
    std::lock_guard<std::mutex> lk(mu);
    if (!done[dev]) {
        if ((e = optin_fwd256()) != cudaSuccess || (e = optin_bwd()) != cudaSuccess)
            return cuda_status(e);
        done[dev] = true;
    }
    return SIMPLEX_OK;
}

static cudaError_t launch_bwd(int map, unsigned ctas, cudaStream_t s, const CUtensorMap *m, float *S,
                              const float *a, int64_t n, int d, int nb, int gx, int64_t T, int64_t nchunks,
                              const int64_t *start, float scale4, float *grad, double *partials, int qshift) {
    if (map == MAP_LAMBDA)
        k_stress_umma_bwd<MAP_LAMBDA><<<ctas, kThreads, SMEM_BYTES, s>>>(
            m[0], m[1], m[2], m[3], m[4], m[5], S, a, n, d, nb, gx, T, nchunks, start, scale4, grad,
            partials, qshift);
    else if (map == MAP_BBOX)
        k_stress_umma_bwd<MAP_BBOX><<<ctas, kThreads, SMEM_BYTES, s>>>(
            m[0], m[1], m[2], m[3], m[4], m[5], S, a, n, d, nb, gx, T, nchunks, start, scale4, grad,
            partials, qshift);
    else if (map == MAP_RB)
        k_stress_umma_bwd<MAP_RB><<<ctas, kThreads, SMEM_BYTES, s>>>(
            m[0], m[1], m[2], m[3], m[4], m[5], S, a, n, d, nb, gx, T, nchunks, start, scale4, grad,
            partials, qshift);
    else
        k_stress_umma_bwd<MAP_LINEAR><<<ctas, kThreads, SMEM_BYTES, s>>>(
            m[0], m[1], m[2], m[3], m[4], m[5], S, a, n, d, nb, gx, T, nchunks, start, scale4, grad,
            partials, qshift);
    return cudaGetLastError();
}

// The backward's prologue: the tile scan of the map's grid and the first
// tile of every chunk, into the workspace.
static cudaError_t chunk_starts(int map, int64_t total, int gx, int nb, int64_t T, int64_t nchunks, int *loc,
                                int64_t *boff, int64_t *start, cudaStream_t s) {
    const int64_t nblk = (total + kScanBlock - 1) / kScanBlock;
    const unsigned b = (unsigned)nblk;
    if (map == MAP_LAMBDA) k_tile_scan<MAP_LAMBDA><<<b, kScanBlock, 0, s>>>(total, gx, nb, loc, boff);
    else if (map == MAP_BBOX) k_tile_scan<MAP_BBOX><<<b, kScanBlock, 0, s>>>(total, gx, nb, loc, boff);
    else if (map == MAP_RB) k_tile_scan<MAP_RB><<<b, kScanBlock, 0, s>>>(total, gx, nb, loc, boff);
    else k_tile_scan<MAP_LINEAR><<<b, kScanBlock, 0, s>>>(total, gx, nb, loc, boff);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_bsum_scan<<<1, 1024, 0, s>>>(nblk, boff);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_chunk_starts<<<(unsigned)((nchunks + 255) / 256), 256, 0, s>>>(total, nblk, T, nchunks, loc, boff, start);
    return cudaGetLastError();
}

// The forward runs as two-CTA clusters in 128 x 256 steps.
static cudaError_t launch_fwd(int map, unsigned ctas, cudaStream_t s, const CUtensorMap *m, const float *a,
                              int64_t n, int d, int nb, int nb2, int gx, int64_t total, double *partials,
                              int qshift) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ctas);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = f256::SMEM2;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (map == MAP_LAMBDA)
        return cudaLaunchKernelEx(&cfg, f256::k_stress_umma_fwd<MAP_LAMBDA>, m[0], m[1], m[2], m[3], a, n, d, nb,
                                  nb2, gx, total, partials, qshift);
    if (map == MAP_BBOX)
        return cudaLaunchKernelEx(&cfg, f256::k_stress_umma_fwd<MAP_BBOX>, m[0], m[1], m[2], m[3], a, n, d, nb,
                                  nb2, gx, total, partials, qshift);
    if (map == MAP_RB)
        return cudaLaunchKernelEx(&cfg, f256::k_stress_umma_fwd<MAP_RB>, m[0], m[1], m[2], m[3], a, n, d, nb,
                                  nb2, gx, total, partials, qshift);
    return cudaLaunchKernelEx(&cfg, f256::k_stress_umma_fwd<MAP_LINEAR>, m[0], m[1], m[2], m[3], a, n, d, nb,
                              nb2, gx, total, partials, qshift);
}

// Two-CTA clusters of the forward kernel that fit on the device at once (one
// CTA per SM), once per device; half the SM count if the query fails.
static int64_t max_pairs(int sms) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return sms / 2;
    static std::mutex mu;
    static int64_t cached[64] = {};
    std::lock_guard<std::mutex> lk(mu);
    if (!cached[dev]) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(sms & ~1));
        cfg.blockDim = dim3(kThreads);
        cfg.dynamicSmemBytes = f256::SMEM2;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 2;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int num = 0;
        if (cudaOccupancyMaxActiveClusters(&num, f256::k_stress_umma_fwd<MAP_LAMBDA>, &cfg) != cudaSuccess ||
            num < 1) {
            cudaGetLastError();
            num = sms / 2;
        }
        cached[dev] = num;
    }
    return cached[dev];
}

}  // namespace summa

bool stress_umma_ok(int64_t d) { return d >= 32 && d <= 96 && d % 32 == 0; }

bool stress_use_umma(int64_t d, int prec) {
    return (prec == SIMPLEX_PREC_BF16X3 || prec == SIMPLEX_PREC_AUTO) && stress_umma_ok(d);
}

int64_t stress_umma_workspace_bytes(int64_t n, int64_t d, bool bwd) {
    return 1024 + summa::layout_of(n, d, bwd).total;
}

int stress_umma_run(bool bwd, int64_t n, int64_t d, const float *x, const float *y, float *d_out,
                    double *loss, double gscale, float *grad, int map, void *ws, int64_t ws_bytes,
                    cudaStream_t s) {
    using namespace summa;
    if (!stress_umma_ok(d)) return SIMPLEX_EUNSUPPORTED;
    if (!aligned(x, 16)) return SIMPLEX_EALIGN;
    if (!ws || ws_bytes < stress_umma_workspace_bytes(n, d, bwd) || !aligned(ws, 256))
        return SIMPLEX_EWORKSPACE;
    const int64_t nb = (n + TM - 1) / TM;
    const Grid g = grid2(nb, map);
    if (!grid_fits(g)) return SIMPLEX_EOVERFLOW;
    const Layout L = layout_of(n, d, bwd);
    unsigned char *w = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(ws) + 1023) & ~uintptr_t(1023));
    auto bf = [&](int64_t off) { return reinterpret_cast<__nv_bfloat16 *>(w + off); };
    float *a = reinterpret_cast<float *>(w + L.a);
    double *partials = reinterpret_cast<double *>(w + L.part);
    const int NG = (int)d + 16;
    // Q = [Delta | S] is P = [S | Delta] with its two halves swapped: where d
    // is a multiple of the K chunk, Q's chunk c is P's chunk at column
    // (64 c + d) mod 2d, so the kernels read Q's tiles from P's memory (one
    // operand copy fewer to write and to keep in L2); otherwise Q is written.
    const bool qview = d % KC == 0;
    const int qshift = qview ? (int)d : 0;
    CUtensorMap m[6];
    if (!make_map_bf16(&m[0], bf(L.Ph), n, 2 * d, 2 * d, TM) ||
        !make_map_bf16(&m[1], bf(L.Pl), n, 2 * d, 2 * d, TM))
        return SIMPLEX_ECUDA;
    if (qview) {
        m[2] = m[0];
        m[3] = m[1];
    } else if (!make_map_bf16(&m[2], bf(L.Qh), n, 2 * d, 2 * d, TM) ||
               !make_map_bf16(&m[3], bf(L.Ql), n, 2 * d, 2 * d, TM)) {
        return SIMPLEX_ECUDA;
    }
    if (bwd) {
        if (!make_map_bf16(&m[4], bf(L.Th), NG, n, L.pitch, NG) ||
            !make_map_bf16(&m[5], bf(L.Tl), NG, n, L.pitch, NG))
            return SIMPLEX_ECUDA;
    } else {
        m[4] = m[0];   // unused by the forward kernel
        m[5] = m[1];
    }
    int st = smem_optin();
    if (st) return st;
    k_stress_prep<<<(unsigned)((n + 31) / 32), 256, 0, s>>>(
        x, y, n, (int)d, NG, L.pitch, bf(L.Ph), bf(L.Pl), qview ? nullptr : bf(L.Qh), qview ? nullptr : bf(L.Ql),
        bwd ? bf(L.Th) : nullptr, bwd ? bf(L.Tl) : nullptr, a);
    note_launches(1);
    if ((st = launch_status())) return st;
    int dev = 0, sms = 0;
    if ((st = cuda_status(cudaGetDevice(&dev)))) return st;
    if ((st = cuda_status(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)))) return st;
    int64_t ctas;
    cudaError_t le;
    if (bwd) {
        const int64_t total = g.gx * g.gy, T = nb * (nb + 1) / 2;
        ctas = T < sms ? T : sms;
        if (ctas > kMaxCtas) ctas = kMaxCtas;
        const int64_t nchunks = chunks_of(T, ctas);
        const int64_t nblk = (total + kScanBlock - 1) / kScanBlock;
        int *loc = reinterpret_cast<int *>(w + L.deal);
        int64_t *boff = reinterpret_cast<int64_t *>(w + L.deal + align_up(4 * total, 1024));
        int64_t *start = reinterpret_cast<int64_t *>(reinterpret_cast<unsigned char *>(boff) + align_up(8 * nblk, 1024));
        if ((st = cuda_status(chunk_starts(map, total, (int)g.gx, (int)nb, T, nchunks, loc, boff, start, s))))
            return st;
        note_launches(3);
        float *S = reinterpret_cast<float *>(w + L.sums);
        if ((st = cuda_status(cudaMemsetAsync(grad, 0, sizeof(float) * (size_t)(n * d), s)))) return st;
        if ((st = cuda_status(cudaMemsetAsync(S, 0, sizeof(float) * (size_t)n, s)))) return st;
        prof_begin(s);
        le = launch_bwd(map, (unsigned)ctas, s, m, S, a, n, (int)d, (int)nb, (int)g.gx, T, nchunks, start,
                        (float)(4.0 * gscale), grad, loss ? partials : nullptr, qshift);
    } else {
        // two-CTA clusters over the map's grid of 256 x 256 super-blocks
        const int64_t nb2 = (nb + 1) / 2;
        const Grid g2 = grid2(nb2, map);
        if (!grid_fits(g2)) return SIMPLEX_EOVERFLOW;
        const int64_t total2 = g2.gx * g2.gy;
        int64_t clusters = max_pairs(sms);
        if (clusters > total2) clusters = total2;
        if (clusters > kMaxCtas / 2) clusters = kMaxCtas / 2;
        ctas = 2 * clusters;
        prof_begin(s);
        le = launch_fwd(map, (unsigned)ctas, s, m, a, n, (int)d, (int)nb, (int)nb2, (int)g2.gx, total2,
                        partials, qshift);
    }
    prof_end(s);
    note_launches(1);
    if (le != cudaSuccess) return cuda_status(le);
    if ((st = launch_status())) return st;
    if (bwd) {
        const int64_t f4 = n * d / 4;
        k_stress_sx<<<(unsigned)((f4 + 255) / 256), 256, 0, s>>>(x, reinterpret_cast<const float *>(w + L.sums), n,
                                                              (int)d, (float)(4.0 * gscale), grad);
        note_launches(1);
        if ((st = launch_status())) return st;
        return loss ? reduce_partials(partials, ctas, partials + kMaxCtas, loss, s) : SIMPLEX_OK;
    }
    if ((st = reduce_partials(partials, ctas, partials + kMaxCtas, loss, s))) return st;
    if (!d_out) return SIMPLEX_OK;
    // the packed D itself: tensor-core EDM where it applies, else FP32
    if (d % 64 == 0)
        return simplex_edm_packed(n, d, x, d_out, map, SIMPLEX_PREC_BF16X3, w + L.edm,
                                  edm_umma_workspace_bytes(n, d), s);
    return simplex_edm_packed(n, d, x, d_out, map, SIMPLEX_PREC_FP32, nullptr, 0, s);
}

int stress_umma_errors(cudaStream_t s) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e);
    int h = 0;
    if ((e = cudaMemcpyFromSymbol(&h, summa::g_error, sizeof(int))) != cudaSuccess) return cuda_status(e);
    if (h) {
        const int zero = 0;
        if ((e = cudaMemcpyToSymbol(summa::g_error, &zero, sizeof(int))) != cudaSuccess)
            return cuda_status(e);
        return SIMPLEX_ETIMEOUT;
    }
    return SIMPLEX_OK;
}

}  // namespace sx
