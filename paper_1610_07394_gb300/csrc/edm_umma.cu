// edm_umma.cu -- packed EDM with the Gram term on the 5th-generation tensor
// cores (tcgen05, TMEM accumulators, TMA-staged operands), for large d.
//
// For a 128 x 128 tile of pairs (rows i of block Y, columns j of block X,
// X <= Y, the block chosen by a block-space map of Sec. III-A):
//   D_ij = |x_i|^2 + |x_j|^2 - 2 g_ij,   g_ij = x_i . x_j,
// with g from BF16 operands split as x = hi + lo (hi = bf16(x),
// lo = bf16(x - hi)):  g ~ hi_i.hi_j + hi_i.lo_j + lo_i.hi_j, accumulated in
// FP32 in tensor memory.  The norms are FP32 sums of the original FP32
// coordinates.  Entries with D < |x_i|^2/64 + |x_j|^2/64 (where the Gram
// form cancels) are recomputed in FP32 from the coordinates; the diagonal is
// exactly 0.
//
// Persistent and warp-specialised, one CTA per SM, over the chosen map's grid
// of 256 x 256 super-blocks (the map over ceil(nb / 2) blocks).  Warp 0
// issues the TMA loads of the BF16 operand tiles of each K chunk, warp 1 the
// tcgen05.mma instructions (M = 128, K = 16, three products per K step) into
// TMEM accumulators, and eight epilogue warps (two per TMEM lane quarter)
// read a finished accumulator with tcgen05.ld, form D, stage rows through
// shared memory and write each packed row segment with one bulk copy, while
// the MMA warp already fills the next accumulator.  Two kernels:
//  * k_edm_umma_wide (d < 128, bound by the stores): N = 128 tiles, K chunks
//    of 64 (128-byte swizzle); a CTA takes a super-block as two steps of two
//    horizontally adjacent tiles, so that a row of a step is one segment of
//    up to 256 outputs (a copy of up to 1 KB);
//  * k_edm_umma (d >= 128, bound by the operand loads and the MMAs): two-CTA
//    clusters walk the super-blocks in the same order, CTA r computing row
//    block 2 sY + r against both column blocks with N = 256 MMAs, its
//    column block's tiles multicast into both CTAs; K chunks of 32
//    (64-byte swizzle) keep three operand stages beside the row staging.
// Every mbarrier wait is bounded in time; a wait that runs out sets a device
// error flag (simplex_device_errors) and the block stops instead of hanging.
#include <cstddef>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "kernels.h"
#include "umma.cuh"

namespace sx {
namespace umma {

constexpr int TM = 128;                        // tile rows (i)
constexpr int TN = 128;                        // tile columns (j)
constexpr int KC = 64;                         // K chunk: 64 BF16 = one 128-byte swizzle row
constexpr int TILE_BYTES = TM * KC * 2;        // 16 KB per operand tile
constexpr int STAGE_BYTES = 4 * TILE_BYTES;    // A_hi, A_lo, B_hi, B_lo
// K-major BF16 operands, M = TM, N = TN.
constexpr uint32_t kIdesc = idesc_bf16(TM, TN, false, false);

__device__ int g_error;   // set when a bounded wait runs out

// x = hi + lo in BF16 and |x|^2 in FP32, one warp per row.
__global__ void __launch_bounds__(256) k_split_bf16(const float *__restrict__ x, int64_t n, int d,
                                                    __nv_bfloat16 *__restrict__ xh,
                                                    __nv_bfloat16 *__restrict__ xl,
                                                    float *__restrict__ nrm) {
    const int64_t row = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    const float *xr = x + row * d;
    float acc = 0.f;
    for (int t = lane; t < d; t += 32) {
        const float v = __ldg(xr + t);
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        xh[row * d + t] = h;
        xl[row * d + t] = __float2bfloat16_rn(v - __bfloat162float(h));
        acc = fmaf(v, v, acc);
    }
    acc = warp_sum_f32(acc);
    if (lane == 0) nrm[row] = acc;
}

// |x_i - x_j|^2 in FP32 from the coordinates (kept out of line: it is rare).
__device__ __noinline__ float exact_sqdist(const float *__restrict__ x, int64_t i, int64_t j, int d) {
    const float *xi = x + i * d, *xj = x + j * d;
    float acc = 0.0f;
    for (int e = 0; e < d; ++e) {
        const float df = __ldg(xi + e) - __ldg(xj + e);
        acc = fmaf(df, df, acc);
    }
    return acc;
}

constexpr int kStages = 3;                     // operand stages of the d >= 128 kernel
constexpr int kEpiWarps = 8;                   // two per TMEM lane quarter
constexpr int kThreads = 64 + 32 * kEpiWarps;  // producer, MMA, epilogue warps

// Epilogue staging of one TMEM lane quarter (the two warps that read it):
// 32 rows of the tile's 128 columns, row pitch 132 floats.  A row is written
// at an offset of (its global address mod 16 bytes) / 4 floats, so that the
// 16-byte-aligned body of the global row segment starts at a 16-byte-aligned
// shared address and one cp.async.bulk of up to 512 bytes copies it.
// Rows sit at stg_row(r): 8 floats of padding after every 8 rows.  The
// offset of row r = i - i0 (i0 a multiple of 32) is T(i) mod 4 = T(r) mod 4
// plus a constant, with period 8 in r (0 1 3 2 2 3 1 0), and the pitch is
// 4 words mod 32, so without the padding rows r, r + 8, r + 16, r + 24 hit
// the same bank when a warp's 32 lanes each write their own row; with it
// the 32 lanes hit 32 banks for any column, and row starts stay 16-byte
// aligned.
constexpr int kRowPitch = 132;
constexpr int kQuarterFloats = 32 * kRowPitch + 24;   // 32 staging rows + padding
__device__ __forceinline__ int stg_row(int r, int pitch) { return r * pitch + 8 * (r >> 3); }

struct PCtl {
    uint64_t full[kStages], empty[kStages];   // operand stages: TMA -> MMA -> TMA
    uint64_t tfull[2], tempty[2];             // accumulators: MMA -> epilogue -> MMA
    uint32_t tmem;
    int fail;
    uint64_t sfull[4], sfree[4];              // per lane quarter: staging written / copied out
    alignas(16) float ncol[kEpiWarps][64];    // each epilogue warp's column norms (float4 reads)
};

constexpr int kCtlBytes = 3072;
constexpr int kStageBytes = 4 * kQuarterFloats * 4;   // four lane quarters
static_assert(sizeof(PCtl) <= kCtlBytes, "control block");
static_assert(offsetof(PCtl, ncol) % 16 == 0, "float4 reads of the column norms");

// Norms of a tile's rows and columns for one epilogue thread: columns
// col0 + 64 half + lane and + 32 (a, b) and its row row0 + r (ni); 0 past n.
__device__ __forceinline__ void load_norms(const float *__restrict__ nrm, int64_t n, int X, int Y,
                                           int half, int r, int lane, float &a, float &b,
                                           float &ni) {
    const int64_t j0 = (int64_t)X * TN + 64 * half + lane, j1 = j0 + 32, i = (int64_t)Y * TM + r;
    a = j0 < n ? __ldg(nrm + j0) : 0.0f;
    b = j1 < n ? __ldg(nrm + j1) : 0.0f;
    ni = i < n ? __ldg(nrm + i) : 0.0f;
}

// The kernel for d >= 128 (bound by the operand loads and the MMAs): two-CTA
// clusters walk the map's grid of 256 x 256 super-blocks in the same order;
// per super-block (sX, sY) CTA r computes row block Y = 2 sY + r against both
// column blocks 2 sX and 2 sX + 1 with M = 128, N = 256 MMAs, loading its own
// row block's tiles and multicasting its column block's tiles into rows
// 128 r .. 128 r + 127 of both CTAs' B operand, so that per K chunk a CTA
// reads 64 KB from L2 for 128 x 256 pairs.  K chunks of 32 in the 64-byte
// swizzle make a stage 48 KB, so three stages fit beside the row staging;
// the epilogue takes the step's two 128-column halves in turn, like a tile
// each (a half above the diagonal or past the last block is not written).
constexpr int KC2 = 32;                        // K chunk: 32 BF16 = one 64-byte swizzle row
constexpr int SUB = TM * KC2 * 2;              // 8 KB: 128 rows x 32 BF16
constexpr int PSTAGE = 6 * SUB;                // A hi, A lo (8 KB each), B hi, B lo (16 KB each)
constexpr int kPAccCols = 4 * TN;              // two 256-column accumulators
constexpr int PSMEM2_BYTES = 1024 + kStages * PSTAGE + kStageBytes + kCtlBytes;
static_assert(PSMEM2_BYTES <= 227 * 1024, "shared memory per block");
constexpr uint32_t kIdesc256 = idesc_bf16(TM, 2 * TN, false, false);

template <int MAP, bool TILES>
__global__ void __launch_bounds__(kThreads, 1) k_edm_umma(const __grid_constant__ CUtensorMap map_hi,
                                                          const __grid_constant__ CUtensorMap map_lo,
                                                          const __grid_constant__ CUtensorMap map_out,
                                                          const float *__restrict__ x,
                                                          const float *__restrict__ nrm,
                                                          float *__restrict__ out, int64_t n, int d,
                                                          int nb, int nb2, int gx, int64_t total) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    float *stg_all = reinterpret_cast<float *>(base + kStages * PSTAGE);
    PCtl &ctl = *reinterpret_cast<PCtl *>(base + kStages * PSTAGE + kStageBytes);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t s_stage = smem_u32(base);
    volatile int *fail = &ctl.fail;

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(smem_u32(&ctl.full[s]), 1);
            mbar_init(smem_u32(&ctl.empty[s]), 2);   // both CTAs release a stage
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(smem_u32(&ctl.tfull[a]), 1);
            mbar_init(smem_u32(&ctl.tempty[a]), kEpiWarps);
        }
        for (int q = 0; q < 4; ++q) {
            mbar_init(smem_u32(&ctl.sfull[q]), 2);
            mbar_init(smem_u32(&ctl.sfree[q]), 2);
        }
        ctl.fail = *reinterpret_cast<volatile int *>(&g_error) ? 1 : 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        prefetch_map(&map_hi);
        prefetch_map(&map_lo);
    }
    if (warp == 1) tmem_alloc(smem_u32(&ctl.tmem), kPAccCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    cluster_sync();   // the peer's barriers exist before any multicast reaches them
    const uint32_t tmem = ctl.tmem;
    const int nchunks = (d + KC2 - 1) / KC2;
    const uint32_t rank = cluster_rank();

    if (warp == 0) {
        // ---------------- TMA producer
        if (lane == 0) {
            SuperWalk<MAP> walk(gx, total, nb2);
            int sX, sY;
            uint32_t it = 0;
            bool ok = true;
            while (ok && !*fail && walk.next(sX, sY)) {
                const int Y = 2 * sY + (int)rank, Xr = 2 * sX + (int)rank;
                for (int c = 0; c < nchunks; ++c, ++it) {
                    const uint32_t s = it % kStages, ph = (it / kStages) & 1;
                    // free once both CTAs' MMAs have read the stage
                    if (!(ok = mbar_wait(smem_u32(&ctl.empty[s]), ph ^ 1, fail, &g_error))) break;
                    const uint32_t bar = smem_u32(&ctl.full[s]), dst = s_stage + s * PSTAGE;
                    mbar_expect_tx(bar, PSTAGE);
                    tma_load_2d(dst, &map_hi, c * KC2, Y * TM, bar);
                    tma_load_2d(dst + SUB, &map_lo, c * KC2, Y * TM, bar);
                    // this CTA's column block, rows 128 r .. 128 r + 127 of both CTAs' B
                    tma_load_2d_mc(dst + (2 + rank) * SUB, &map_hi, c * KC2, Xr * TN, bar, 3);
                    tma_load_2d_mc(dst + (4 + rank) * SUB, &map_lo, c * KC2, Xr * TN, bar, 3);
                }
            }
            // a failed block waits (bounded) for the loads it may have in flight
            if (*fail)
                for (uint32_t k = it > (uint32_t)kStages ? it - kStages : 0; k < it; ++k)
                    mbar_drain(smem_u32(&ctl.full[k % kStages]), (k / kStages) & 1);
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer
        {   // the whole warp, converged; one elected lane issues
            SuperWalk<MAP> walk(gx, total, nb2);
            int sX, sY;
            uint32_t it = 0, tt = 0;
            bool ok = true;
            while (ok && !*fail && walk.next(sX, sY)) {
                const uint32_t acc = tt & 1, aph = (tt >> 1) & 1;
                if (!(ok = mbar_wait(smem_u32(&ctl.tempty[acc]), aph ^ 1, fail, &g_error))) break;
                tc_fence_after();
                const uint32_t dtm = tmem + acc * (2 * TN);
                for (int c = 0; c < nchunks; ++c, ++it) {
                    const uint32_t s = it % kStages;
                    if (!(ok = mbar_wait(smem_u32(&ctl.full[s]), (it / kStages) & 1, fail, &g_error))) break;
                    tc_fence_after();
                    const uint32_t src = s_stage + s * PSTAGE;
                    const uint64_t d0 = sw64_desc(src);
#pragma unroll
                    for (int ks = 0; ks < KC2 / 16; ++ks) {
                        const uint32_t koff = ks * 32;
                        mma_bf16x3_w(dtm, desc_add(d0, koff), desc_add(d0, SUB + koff), desc_add(d0, 2 * SUB + koff),
                                     desc_add(d0, 4 * SUB + koff), kIdesc256, (c > 0 || ks > 0) ? 1u : 0u);
                    }
                    // the stage is free once this CTA's MMAs and the peer's have read it
                    mma_commit_mc_w(smem_u32(&ctl.empty[s]), 3);
                }
                if (ok) mma_commit_w(smem_u32(&ctl.tfull[acc]));
                ++tt;
            }
        }
    } else {
        // ---------------- epilogue: 8 warps, two per TMEM lane quarter
        const int ew = warp - 2;                 // 0..7
        const int quarter = warp & 3;            // TMEM lanes 32*quarter .. +31
        const int half = ew >> 2;                // columns [64*half, 64*half + 64) of a half-step
        const int r = 32 * quarter + lane;       // this thread's row in the step
        float *stg = stg_all + quarter * kQuarterFloats;   // shared with the other half's warp
        float *nc = &ctl.ncol[ew][0];            // this warp's 64 column norms
        // tile-packed output: this warp's two 32 x 32 boxes (its 64 columns of
        // rows 32 quarter .. +31 of a tile), 128-byte swizzle, 1024-byte aligned
        unsigned char *boxes = reinterpret_cast<unsigned char *>(stg_all) + (quarter * 2 + half) * 8192;
        bool inflight = false;
        SuperWalk<MAP> walk(gx, total, nb2);
        int sX, sY;
        uint32_t tt = 0, st = 0;   // steps, and half-steps staged and written
        bool ok = true;
        // norms of a step, loaded a step ahead: this warp's two columns in each
        // half-step (cn[2 u], cn[2 u + 1]) and this thread's row (rn)
        auto load_step = [&](int sXs, int sYs, float (&cn)[4], float &rn) {
#pragma unroll
            for (int u = 0; u < 2; ++u)
                load_norms(nrm, n, 2 * sXs + u, 2 * sYs + (int)rank, half, r, lane, cn[2 * u], cn[2 * u + 1], rn);
        };
        bool have = walk.next(sX, sY);
        float pcn[4] = {0.f, 0.f, 0.f, 0.f}, prn = 0.f;
        if (have) load_step(sX, sY, pcn, prn);
        while (have && ok && !*fail) {
            int sXn, sYn;
            const bool hn = walk.next(sXn, sYn);
            float ncn[4] = {0.f, 0.f, 0.f, 0.f}, nrn = 0.f;
            if (hn) load_step(sXn, sYn, ncn, nrn);
            const int Y = 2 * sY + (int)rank;
            const uint32_t acc = tt & 1, aph = (tt >> 1) & 1;
            if (!(ok = mbar_wait(smem_u32(&ctl.tfull[acc]), aph, fail, &g_error))) break;
            tc_fence_after();
#pragma unroll 1
            for (int u = 0; u < 2 && ok; ++u) {
                // half-step u: column block X = 2 sX + u, accumulator columns 128 u ..
                const int X = 2 * sX + u;
                const bool valid = X <= Y && Y < nb;
                const int64_t row0 = (int64_t)Y * TM, col0 = (int64_t)X * TN;
                const float pa = u ? pcn[2] : pcn[0], pb = u ? pcn[3] : pcn[1], ni = prn;   // constant indices
                __syncwarp();   // the previous half-step's reads of nc are done
                nc[lane] = pa;
                nc[lane + 32] = pb;
                const int64_t i = row0 + r;
                const bool diag = (X == Y);
                // packed index of this row's first column in the half-step and in
                // this warp's half; floats from the row start back to the previous
                // 16-byte boundary of out
                const int64_t grow = i * (i + 1) / 2 + col0, gbase = grow + 64 * half;
                const int shift = (int)((reinterpret_cast<uintptr_t>(out + grow) >> 2) & 3);
                float *myrow = stg + stg_row(lane, kRowPitch) + shift + 64 * half;
                __syncwarp();
                float v0[32], v1[32];
                const uint32_t taddr = tmem + acc * (2 * TN) + ((uint32_t)(32 * quarter) << 16) +
                                       (uint32_t)(TN * u + 64 * half);
                tmem_ld64(taddr, v0, v1);
                if (u == 1) {
                    // the accumulator is read: hand it back to the MMA warp
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(smem_u32(&ctl.tempty[acc]));
                }
                if (!valid) continue;   // above the diagonal or past the last block
                // D = |x_i|^2 + |x_j|^2 - 2 g; flag entries with D < (|x_i|^2 + |x_j|^2)/64
                float lows[4] = {1.0f, 1.0f, 1.0f, 1.0f};
#pragma unroll
                for (int q = 0; q < 32; q += 4) {
                    const float4 a = *reinterpret_cast<const float4 *>(nc + q);
                    const float4 b = *reinterpret_cast<const float4 *>(nc + 32 + q);
                    const float sa[4] = {ni + a.x, ni + a.y, ni + a.z, ni + a.w};
                    const float sb[4] = {ni + b.x, ni + b.y, ni + b.z, ni + b.w};
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        v0[q + k] = fmaf(-2.0f, v0[q + k], sa[k]);
                        v1[q + k] = fmaf(-2.0f, v1[q + k], sb[k]);
                        lows[k] = fminf(lows[k], fminf(fmaf(-0.015625f, sa[k], v0[q + k]),
                                                       fmaf(-0.015625f, sb[k], v1[q + k])));
                    }
                }
                const float low = fminf(fminf(lows[0], lows[1]), fminf(lows[2], lows[3]));
                if (__any_sync(0xffffffffu, low < 0.0f)) {
#pragma unroll
                    for (int q = 0; q < 64; ++q) {
                        float &vq = q < 32 ? v0[q] : v1[q - 32];
                        const int64_t j = col0 + 64 * half + q;
                        const float sj = ni + nc[q];
                        if (vq < 0.015625f * sj && i < n && j < n && i != j) vq = exact_sqdist(x, i, j, d);
                    }
                }
                if constexpr (TILES) {
                    // the whole tile, padding and diagonal masked, as two boxes
                    // of the tile-packed output (TMA tensor stores)
                    if (row0 + TM > n || col0 + TN > n || diag) {
#pragma unroll
                        for (int q = 0; q < 64; ++q) {
                            float &vq = q < 32 ? v0[q] : v1[q - 32];
                            const int64_t j = col0 + 64 * half + q;
                            if (i >= n || j >= n || i == j) vq = 0.0f;
                        }
                    }
                    if (inflight) {
                        if (lane == 0) bulk_wait_read();
                        __syncwarp();
                    }
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        *reinterpret_cast<float4 *>(boxes + box_chunk_off(lane, c)) =
                            make_float4(v0[4 * c], v0[4 * c + 1], v0[4 * c + 2], v0[4 * c + 3]);
                        *reinterpret_cast<float4 *>(boxes + 4096 + box_chunk_off(lane, c)) =
                            make_float4(v1[4 * c], v1[4 * c + 1], v1[4 * c + 2], v1[4 * c + 3]);
                    }
                    fence_proxy_async();
                    __syncwarp();
                    if (lane == 0) {
                        const int slot = (int)((int64_t)Y * (Y + 1) / 2 + X);
                        tma_store_3d(&map_out, smem_u32(boxes), 64 * half, 32 * quarter, slot);
                        tma_store_3d(&map_out, smem_u32(boxes + 4096), 64 * half + 32, 32 * quarter, slot);
                        bulk_commit();
                    }
                    inflight = true;
                    continue;
                }
                // the staging is free once both warps' copies of the previous half-step have read it
                if (st > 0) {
                    bulk_wait_read();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(smem_u32(&ctl.sfree[quarter]));
                    if (!(ok = mbar_wait(smem_u32(&ctl.sfree[quarter]), (st - 1) & 1, fail, &g_error))) break;
                }
#pragma unroll
                for (int q = 0; q < 32; ++q) { myrow[q] = v0[q]; myrow[32 + q] = v1[q]; }
                fence_proxy_async();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&ctl.sfull[quarter]));
                if (!(ok = mbar_wait(smem_u32(&ctl.sfull[quarter]), st & 1, fail, &g_error))) break;
                if (!diag) {
                    // One bulk copy per row segment of the half-step (128 columns,
                    // both halves): lanes 0-15 of this warp take rows 16 half .. +15;
                    // the ragged head and tail (at most 3 floats each) by plain stores.
                    const int rr = 16 * half + lane;
                    const int64_t ir = row0 + 32 * quarter + rr;
                    if (lane < 16 && ir < n) {
                        const int64_t gb = ir * (ir + 1) / 2 + col0;
                        const int sh = (int)((reinterpret_cast<uintptr_t>(out + gb) >> 2) & 3);
                        const float *sr = stg + stg_row(rr, kRowPitch) + sh;   // column c at sr[c]
                        const int h = (4 - sh) & 3;
                        const int body = (128 - h) & ~3;
                        bulk_store(out + gb + h, smem_u32(sr + h), (uint32_t)body * 4);
                        bulk_commit();
                        for (int e = 0; e < h; ++e) out[gb + e] = sr[e];
                        for (int e = h + body; e < 128; ++e) out[gb + e] = sr[e];
                    }
                } else if (i < n && 64 * half <= r) {
                    // diagonal block: columns j <= i only, plain stores
                    const int rc = r - 64 * half;             // diagonal column, local
                    const int last = rc < 63 ? rc : 63;
                    if (rc <= 63) myrow[rc] = 0.0f;           // D_ii = 0 exactly
                    for (int e = 0; e <= last; ++e) out[gbase + e] = myrow[e];
                }
                ++st;
            }
            ++tt;
            sX = sXn; sY = sYn; have = hn;
#pragma unroll
            for (int q = 0; q < 4; ++q) pcn[q] = ncn[q];
            prn = nrn;
        }
    }
    bulk_wait_all();   // staging rows must stay valid until the copies have read them
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tmem, kPAccCols);
    }
    // neither CTA of a pair leaves while the other may still multicast into
    // its shared memory or arrive on its barriers
    cluster_sync();
}

// ---------------------------------------------------------------- rows of 256 columns

// The kernel for d < 128, where the packed stores bound it, in steps of two
// horizontally adjacent tiles: each CTA walks the map's grid of 256 x 256
// super-blocks (sX, sY) and takes a super-block as two steps (row block
// 2 sY + s against column blocks 2 sX and 2 sX + 1), so that each row of a
// step is one packed segment of up to 256 outputs, written by one bulk copy
// of up to 1 KB.  The bulk copies cost a fixed time per copy besides their
// bytes, and copies of 1 KB instead of 512 B take a quarter off the store
// time.  One 64 KB operand stage (A and B of one tile; the stores leave the
// loads time to spare), four 128-column TMEM accumulators (two steps), and
// staging of 32 rows x 256 columns per TMEM lane quarter.
namespace wide {

constexpr int kWStages = 1;
constexpr int kWPitch = 260;                          // 256 columns + the shift to 16 bytes
constexpr int kWQuarterFloats = 32 * kWPitch + 24;    // rows at stg_row(r, kWPitch)
constexpr int kWStageBytes = 4 * kWQuarterFloats * 4; // four lane quarters
constexpr int kWAccCols = 4 * TN;                     // four accumulators

struct WCtl {
    uint64_t full[kWStages], empty[kWStages];   // operand stage: TMA -> MMA -> TMA
    uint64_t tfull[4], tempty[4];               // accumulators: MMA -> epilogue -> MMA
    uint64_t sfull[4], sfree[4];                // per lane quarter: staging written / copied out
    uint32_t tmem;
    int fail;
    alignas(16) float ncol[kEpiWarps][TN];      // each epilogue warp's 128 column norms
};

constexpr int kWCtlBytes = 8192;
constexpr int WSMEM_BYTES = 1024 + kWStages * STAGE_BYTES + kWStageBytes + kWCtlBytes;
static_assert(sizeof(WCtl) <= kWCtlBytes, "control block");
static_assert(offsetof(WCtl, ncol) % 16 == 0, "float4 reads of the column norms");
static_assert(WSMEM_BYTES <= 227 * 1024, "shared memory per block");

// The steps of a CTA: super-blocks w = blockIdx.x + k gridDim.x of the
// map's grid over nb2 = ceil(nb / 2) blocks of 256, two steps each (row
// blocks 2 sY, 2 sY + 1; a row block past the last is skipped).
template <int MAP>
struct StepWalk {
    int64_t w, total;
    int wx, wy, gx, nb2, nb, step, sX, sY, pend, px, py;
    __device__ StepWalk(int gx_, int64_t total_, int nb2_, int nb_)
        : w(blockIdx.x), total(total_), gx(gx_), nb2(nb2_), nb(nb_), step(2), sX(0), sY(0), pend(0),
          px(0), py(0) {
        wy = (int)(blockIdx.x / (unsigned)gx_);
        wx = (int)(blockIdx.x - (unsigned)wy * (unsigned)gx_);
    }
    // the next step: column blocks X0 = 2 sX and X0 + 1, row block Y
    __device__ bool next(int &X0, int &Y) {
        for (;;) {
            if (step >= 2) {
                if (pend) {
                    pend = 0;
                    sX = px; sY = py;
                } else {
                    bool found = false;
                    while (w < total) {
                        const List2 L = MAP == MAP_LINEAR ? decode2_linear(w, nb2)
                                                          : decode2<MAP>((uint32_t)wx, (uint32_t)wy, nb2);
                        w += gridDim.x;
                        wx += (int)gridDim.x;
                        while (wx >= gx) { wx -= gx; ++wy; }
                        if (L.cnt == 0) continue;
                        sX = L.x[0]; sY = L.y[0];
                        if (L.cnt > 1) { pend = 1; px = L.x[1]; py = L.y[1]; }
                        found = true;
                        break;
                    }
                    if (!found) return false;
                }
                step = 0;
            }
            X0 = 2 * sX;
            Y = 2 * sY + step;
            ++step;
            if (Y < nb) return true;
        }
    }
};

template <int MAP, bool TILES>
__global__ void __launch_bounds__(kThreads, 1) k_edm_umma_wide(const __grid_constant__ CUtensorMap map_hi,
                                                               const __grid_constant__ CUtensorMap map_lo,
                                                               const __grid_constant__ CUtensorMap map_out,
                                                               const float *__restrict__ x,
                                                               const float *__restrict__ nrm,
                                                               float *__restrict__ out, int64_t n, int d,
                                                               int nb, int nb2, int gx, int64_t total) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    float *stg_all = reinterpret_cast<float *>(base + kWStages * STAGE_BYTES);
    WCtl &ctl = *reinterpret_cast<WCtl *>(base + kWStages * STAGE_BYTES + kWStageBytes);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t s_stages = smem_u32(base);
    volatile int *fail = &ctl.fail;

    if (tid == 0) {
        for (int s = 0; s < kWStages; ++s) {
            mbar_init(smem_u32(&ctl.full[s]), 1);
            mbar_init(smem_u32(&ctl.empty[s]), 1);
        }
        for (int a = 0; a < 4; ++a) {
            mbar_init(smem_u32(&ctl.tfull[a]), 1);
            mbar_init(smem_u32(&ctl.tempty[a]), kEpiWarps / 2);   // the four warps of that tile
        }
        for (int q = 0; q < 4; ++q) {
            mbar_init(smem_u32(&ctl.sfull[q]), 2);
            mbar_init(smem_u32(&ctl.sfree[q]), 2);
        }
        ctl.fail = *reinterpret_cast<volatile int *>(&g_error) ? 1 : 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        prefetch_map(&map_hi);
        prefetch_map(&map_lo);
    }
    if (warp == 1) tmem_alloc(smem_u32(&ctl.tmem), kWAccCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = ctl.tmem;
    const int nchunks = (d + KC - 1) / KC;

    if (warp == 0) {
        // ---------------- TMA producer: per step the two tiles, per tile its K chunks
        if (lane == 0) {
            StepWalk<MAP> walk(gx, total, nb2, nb);
            int X0, Y;
            uint32_t it = 0;
            bool ok = true;
            while (ok && !*fail && walk.next(X0, Y)) {
                for (int t = 0; t < 2 && ok; ++t)
                    for (int c = 0; c < nchunks; ++c, ++it) {
                        const int s = (int)(it % kWStages);
                        const uint32_t ph = (it / kWStages) & 1;
                        if (!(ok = mbar_wait(smem_u32(&ctl.empty[s]), ph ^ 1, fail, &g_error))) break;
                        const uint32_t bar = smem_u32(&ctl.full[s]);
                        const uint32_t dst = s_stages + s * STAGE_BYTES;
                        mbar_expect_tx(bar, STAGE_BYTES);
                        tma_load_2d(dst + 0 * TILE_BYTES, &map_hi, c * KC, Y * TM, bar);
                        tma_load_2d(dst + 1 * TILE_BYTES, &map_lo, c * KC, Y * TM, bar);
                        tma_load_2d(dst + 2 * TILE_BYTES, &map_hi, c * KC, (X0 + t) * TN, bar);
                        tma_load_2d(dst + 3 * TILE_BYTES, &map_lo, c * KC, (X0 + t) * TN, bar);
                    }
            }
            // a failed block waits (bounded) for its loads in flight
            if (*fail && it > 0) {
                const uint32_t last = it - 1;
                mbar_drain(smem_u32(&ctl.full[last % kWStages]), (last / kWStages) & 1);
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer: tile tt into accumulator tt mod 4
        {   // the whole warp, converged; one elected lane issues
            StepWalk<MAP> walk(gx, total, nb2, nb);
            int X0, Y;
            uint32_t it = 0, tt = 0;
            bool ok = true;
            while (ok && !*fail && walk.next(X0, Y)) {
                for (int t = 0; t < 2 && ok; ++t, ++tt) {
                    const uint32_t acc = tt & 3, use = tt >> 2;
                    if (!(ok = mbar_wait(smem_u32(&ctl.tempty[acc]), (use & 1) ^ 1, fail, &g_error))) break;
                    tc_fence_after();
                    const uint32_t dtm = tmem + acc * TN;
                    for (int c = 0; c < nchunks; ++c, ++it) {
                        const int s = (int)(it % kWStages);
                        if (!(ok = mbar_wait(smem_u32(&ctl.full[s]), (it / kWStages) & 1, fail, &g_error)))
                            break;
                        tc_fence_after();
                        const uint32_t src = s_stages + s * STAGE_BYTES;
                        const uint64_t d0 = sw128_desc(src);   // A hi, A lo, B hi, B lo tiles of the stage
#pragma unroll
                        for (int ks = 0; ks < KC / 16; ++ks) {
                            const uint32_t koff = ks * 32;
                            mma_bf16x3_w(dtm, desc_add(d0, koff), desc_add(d0, TILE_BYTES + koff),
                                         desc_add(d0, 2 * TILE_BYTES + koff), desc_add(d0, 3 * TILE_BYTES + koff),
                                         kIdesc, (c > 0 || ks > 0) ? 1u : 0u);
                        }
                        mma_commit_w(smem_u32(&ctl.empty[s]));
                    }
                    if (ok) mma_commit_w(smem_u32(&ctl.tfull[acc]));
                }
            }
        }
    } else if constexpr (TILES) {
        // ---------------- epilogue, tile-packed output: warp (quarter, h) owns
        // rows 32 quarter .. +31 of the step's tile h, one contiguous 16 KB
        // block of the output; it stages them as four 32 x 32 boxes in the
        // 128-byte swizzle (conflict-free: lane = row) and writes each with a
        // TMA tensor store as soon as it is staged (one bulk group per box),
        // so that a box waits only for its own previous store to have read it
        // and three boxes stay in flight while the fourth is written
        const int ew = warp - 2;
        const int quarter = warp & 3;
        const int h = ew >> 2;
        const int r = 32 * quarter + lane;
        unsigned char *boxes = reinterpret_cast<unsigned char *>(stg_all) + ew * 16384;
        const uint32_t sbox = smem_u32(boxes);
        float *nc = &ctl.ncol[ew][0];
        StepWalk<MAP> walk(gx, total, nb2, nb);
        int X0, Y;
        uint32_t tt = 0;
        auto load_step = [&](int X0s, int Ys, float (&cn)[4], float &rn) {
            const int64_t cb = (int64_t)X0s * TN + TN * h + lane, ii = (int64_t)Ys * TM + r;
#pragma unroll
            for (int q = 0; q < 4; ++q) cn[q] = cb + 32 * q < n ? __ldg(nrm + cb + 32 * q) : 0.0f;
            rn = ii < n ? __ldg(nrm + ii) : 0.0f;
        };
        bool have = walk.next(X0, Y);
        float pcn[4] = {0.f, 0.f, 0.f, 0.f}, prn = 0.f;
        if (have) load_step(X0, Y, pcn, prn);
        while (have && !*fail) {
            int X0n, Yn;
            const bool hn = walk.next(X0n, Yn);
            float ncn[4] = {0.f, 0.f, 0.f, 0.f}, nrn = 0.f;
            if (hn) load_step(X0n, Yn, ncn, nrn);
            const uint32_t acc = (tt + h) & 3, use = (tt + h) >> 2;
            const int X = X0 + h;
            const bool valid = X <= Y;             // X < nb follows from Y < nb
            const int64_t row0 = (int64_t)Y * TM, colh = (int64_t)X * TN;
            __syncwarp();   // the previous step's reads of nc are done
#pragma unroll
            for (int q = 0; q < 4; ++q) nc[32 * q + lane] = pcn[q];
            const int64_t i = row0 + r;
            const float ni = prn;
            __syncwarp();
            if (!mbar_wait(smem_u32(&ctl.tfull[acc]), use & 1, fail, &g_error)) break;
            tc_fence_after();
            if (valid) {
                // padding rows / columns (last tile row) and the diagonal are masked
                const bool mask = row0 + TM > n || colh + TN > n || X == Y;
#pragma unroll 1
                for (int part = 0; part < 2; ++part) {
                    float v0[32], v1[32];
                    tmem_ld64(tmem + acc * TN + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(64 * part), v0, v1);
                    const float *ncp = nc + 64 * part;
                    float lows[4] = {1.0f, 1.0f, 1.0f, 1.0f};
#pragma unroll
                    for (int q = 0; q < 32; q += 4) {
                        const float4 a = *reinterpret_cast<const float4 *>(ncp + q);
                        const float4 b = *reinterpret_cast<const float4 *>(ncp + 32 + q);
                        const float sa[4] = {ni + a.x, ni + a.y, ni + a.z, ni + a.w};
                        const float sb[4] = {ni + b.x, ni + b.y, ni + b.z, ni + b.w};
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            v0[q + k] = fmaf(-2.0f, v0[q + k], sa[k]);
                            v1[q + k] = fmaf(-2.0f, v1[q + k], sb[k]);
                            lows[k] = fminf(lows[k], fminf(fmaf(-0.015625f, sa[k], v0[q + k]),
                                                           fmaf(-0.015625f, sb[k], v1[q + k])));
                        }
                    }
                    const float low = fminf(fminf(lows[0], lows[1]), fminf(lows[2], lows[3]));
                    if (__any_sync(0xffffffffu, low < 0.0f)) {
#pragma unroll
                        for (int q = 0; q < 64; ++q) {
                            float &vq = q < 32 ? v0[q] : v1[q - 32];
                            const int64_t j = colh + 64 * part + q;
                            const float sj = ni + ncp[q];
                            if (vq < 0.015625f * sj && i < n && j < n && i != j) vq = exact_sqdist(x, i, j, d);
                        }
                    }
                    if (mask) {
#pragma unroll
                        for (int q = 0; q < 64; ++q) {
                            float &vq = q < 32 ? v0[q] : v1[q - 32];
                            const int64_t j = colh + 64 * part + q;
                            if (i >= n || j >= n || i == j) vq = 0.0f;
                        }
                    }
                    if (part == 1) {
                        // the accumulator is read: hand it back to the MMA warp
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(smem_u32(&ctl.tempty[acc]));
                    }
                    const int slot = (int)((int64_t)Y * (Y + 1) / 2 + X);
#pragma unroll
                    for (int k = 0; k < 2; ++k) {
                        const int b = 2 * part + k;
                        const float *v = k == 0 ? v0 : v1;
                        // box b's previous store (four bulk groups ago) has read it
                        if (lane == 0) bulk_wait_read_le<3>();
                        __syncwarp();
#pragma unroll
                        for (int c = 0; c < 8; ++c)
                            *reinterpret_cast<float4 *>(boxes + b * 4096 + box_chunk_off(lane, c)) =
                                make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
                        fence_proxy_async();
                        __syncwarp();
                        if (lane == 0) {
                            tma_store_3d(&map_out, sbox + b * 4096, 32 * b, 32 * quarter, slot);
                            bulk_commit();
                        }
                    }
                }
            } else {
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&ctl.tempty[acc]));
            }
            tt += 2;
            X0 = X0n; Y = Yn; have = hn;
#pragma unroll
            for (int q = 0; q < 4; ++q) pcn[q] = ncn[q];
            prn = nrn;
        }
    } else {
        // ---------------- epilogue: 8 warps; warp (quarter, h) reads TMEM lanes
        // 32 quarter .. +31 of the step's tile h (columns 128 h .. of the step)
        const int ew = warp - 2;                 // 0..7
        const int quarter = warp & 3;
        const int h = ew >> 2;
        const int r = 32 * quarter + lane;       // this thread's row in the step
        float *stg = stg_all + quarter * kWQuarterFloats;   // shared with the other tile's warp
        float *nc = &ctl.ncol[ew][0];
        StepWalk<MAP> walk(gx, total, nb2, nb);
        int X0, Y;
        uint32_t tt = 0, st = 0;   // tiles, steps
        // norms of a step's columns (this warp's tile, four per lane) and of
        // this thread's row, loaded a step ahead
        auto load_step = [&](int X0s, int Ys, float (&cn)[4], float &rn) {
            const int64_t cb = (int64_t)X0s * TN + TN * h + lane, ii = (int64_t)Ys * TM + r;
#pragma unroll
            for (int q = 0; q < 4; ++q) cn[q] = cb + 32 * q < n ? __ldg(nrm + cb + 32 * q) : 0.0f;
            rn = ii < n ? __ldg(nrm + ii) : 0.0f;
        };
        bool have = walk.next(X0, Y);
        float pcn[4] = {0.f, 0.f, 0.f, 0.f}, prn = 0.f;
        if (have) load_step(X0, Y, pcn, prn);
        while (have && !*fail) {
            int X0n, Yn;
            const bool hn = walk.next(X0n, Yn);
            float ncn[4] = {0.f, 0.f, 0.f, 0.f}, nrn = 0.f;
            if (hn) load_step(X0n, Yn, ncn, nrn);
            const uint32_t acc = (tt + h) & 3, use = (tt + h) >> 2;
            const int64_t row0 = (int64_t)Y * TM, col0 = (int64_t)X0 * TN, colh = col0 + TN * h;
            __syncwarp();   // the previous step's reads of nc are done
#pragma unroll
            for (int q = 0; q < 4; ++q) nc[32 * q + lane] = pcn[q];
            const int64_t i = row0 + r;
            const float ni = prn;
            // staging row of row i: step column c at myrow[c], offset by the
            // floats from the row start back to the previous 16-byte boundary of out
            const int64_t grow = i * (i + 1) / 2 + col0;
            const int shift = (int)((reinterpret_cast<uintptr_t>(out + grow) >> 2) & 3);
            float *myrow = stg + stg_row(lane, kWPitch) + shift;
            __syncwarp();
            if (!mbar_wait(smem_u32(&ctl.tfull[acc]), use & 1, fail, &g_error)) break;
            tc_fence_after();
            // part p: columns 64 p .. 64 p + 63 of this warp's tile.  Part 0 is
            // read and formed before the wait for the staging, so that it
            // overlaps the previous step's copies.
            bool staged_ok = true;
#pragma unroll 1
            for (int part = 0; part < 2; ++part) {
                float v0[32], v1[32];
                const uint32_t taddr =
                    tmem + acc * TN + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(64 * part);
                tmem_ld64(taddr, v0, v1);
                const float *ncp = nc + 64 * part;
                // D = |x_i|^2 + |x_j|^2 - 2 g; flag entries with D < (|x_i|^2 + |x_j|^2)/64
                float lows[4] = {1.0f, 1.0f, 1.0f, 1.0f};
#pragma unroll
                for (int q = 0; q < 32; q += 4) {
                    const float4 a = *reinterpret_cast<const float4 *>(ncp + q);
                    const float4 b = *reinterpret_cast<const float4 *>(ncp + 32 + q);
                    const float sa[4] = {ni + a.x, ni + a.y, ni + a.z, ni + a.w};
                    const float sb[4] = {ni + b.x, ni + b.y, ni + b.z, ni + b.w};
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        v0[q + k] = fmaf(-2.0f, v0[q + k], sa[k]);
                        v1[q + k] = fmaf(-2.0f, v1[q + k], sb[k]);
                        lows[k] = fminf(lows[k], fminf(fmaf(-0.015625f, sa[k], v0[q + k]),
                                                       fmaf(-0.015625f, sb[k], v1[q + k])));
                    }
                }
                const float low = fminf(fminf(lows[0], lows[1]), fminf(lows[2], lows[3]));
                if (__any_sync(0xffffffffu, low < 0.0f)) {
#pragma unroll
                    for (int q = 0; q < 64; ++q) {
                        float &vq = q < 32 ? v0[q] : v1[q - 32];
                        const int64_t j = colh + 64 * part + q;
                        const float sj = ni + ncp[q];
                        if (vq < 0.015625f * sj && i < n && j < n && i != j) vq = exact_sqdist(x, i, j, d);
                    }
                }
                // the staging is free once both warps' copies of the previous step have read it
                if (part == 0 && st > 0) {
                    bulk_wait_read();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(smem_u32(&ctl.sfree[quarter]));
                    if (!mbar_wait(smem_u32(&ctl.sfree[quarter]), (st - 1) & 1, fail, &g_error)) {
                        staged_ok = false;
                        break;
                    }
                }
                float *dst = myrow + TN * h + 64 * part;
#pragma unroll
                for (int q = 0; q < 32; ++q) { dst[q] = v0[q]; dst[32 + q] = v1[q]; }
            }
            if (!staged_ok) break;
            // the accumulator is read: hand it back to the MMA warp
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&ctl.tempty[acc]));
            // D_ii = 0 exactly (the diagonal column, where it falls in this warp's tile)
            const int64_t cdiag = i - colh;
            if (cdiag >= 0 && cdiag < TN) myrow[TN * h + (int)cdiag] = 0.0f;
            fence_proxy_async();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&ctl.sfull[quarter]));
            if (!mbar_wait(smem_u32(&ctl.sfull[quarter]), st & 1, fail, &g_error)) break;
            // One bulk copy per row of the step (lanes 0-15 of this warp: rows
            // 16 h .. 16 h + 15 of the quarter): the columns j <= i, j < n of
            // the 256, its ragged head and tail (at most 3 floats each) by
            // plain stores.
            const int rr = 16 * h + lane;
            const int64_t ir = row0 + 32 * quarter + rr;
            if (lane < 16 && ir < n) {
                const int64_t lim = (ir + 1 < n ? ir + 1 : n) - col0;
                const int len = lim <= 0 ? 0 : (lim >= 2 * TN ? 2 * TN : (int)lim);
                const int64_t gb = ir * (ir + 1) / 2 + col0;
                const int sh = (int)((reinterpret_cast<uintptr_t>(out + gb) >> 2) & 3);
                const float *sr = stg + stg_row(rr, kWPitch) + sh;   // column c at sr[c]
                const int hd = ((4 - sh) & 3) < len ? ((4 - sh) & 3) : len;
                const int body = (len - hd) & ~3;
                if (body > 0) {
                    bulk_store(out + gb + hd, smem_u32(sr + hd), (uint32_t)body * 4);
                    bulk_commit();
                }
                for (int e = 0; e < hd; ++e) out[gb + e] = sr[e];
                for (int e = hd + body; e < len; ++e) out[gb + e] = sr[e];
            }
            tt += 2;
            ++st;
            X0 = X0n; Y = Yn; have = hn;
#pragma unroll
            for (int q = 0; q < 4; ++q) pcn[q] = ncn[q];
            prn = nrn;
        }
    }
    bulk_wait_all();   // staging rows must stay valid until the copies have read them
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tmem, kWAccCols);
    }
}

}  // namespace wide

template <bool TILES>
static cudaError_t optin_layout() {
    const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_edm_umma<MAP_LAMBDA, TILES>, a, PSMEM2_BYTES)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(k_edm_umma<MAP_BBOX, TILES>, a, PSMEM2_BYTES)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(k_edm_umma<MAP_LINEAR, TILES>, a, PSMEM2_BYTES)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(k_edm_umma<MAP_RB, TILES>, a, PSMEM2_BYTES)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(wide::k_edm_umma_wide<MAP_LAMBDA, TILES>, a, wide::WSMEM_BYTES)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(wide::k_edm_umma_wide<MAP_BBOX, TILES>, a, wide::WSMEM_BYTES)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(wide::k_edm_umma_wide<MAP_LINEAR, TILES>, a, wide::WSMEM_BYTES)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(wide::k_edm_umma_wide<MAP_RB, TILES>, a, wide::WSMEM_BYTES)) != cudaSuccess)
        return e;
    return cudaSuccess;
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
        if ((e = optin_layout<false>()) != cudaSuccess || (e = optin_layout<true>()) != cudaSuccess)
            return cuda_status(e);
        done[dev] = true;
    }
    return SIMPLEX_OK;
}

// Operand tiles are shared by a CTA pair where the kernel is bound by loading
// them (d >= 128: four or more K chunks per tile); at d = 64 the packed output
// writes bound it.
static bool use_multicast(int64_t d) { return d >= 128; }

// Two-CTA clusters that fit on the device at once (one CTA per SM), once per
// device; half the SM count if the query fails.
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
        cfg.dynamicSmemBytes = PSMEM2_BYTES;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 2;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int num = 0;
        if (cudaOccupancyMaxActiveClusters(&num, k_edm_umma<MAP_LAMBDA, false>, &cfg) != cudaSuccess || num < 1) {
            cudaGetLastError();
            num = sms / 2;
        }
        cached[dev] = num;
    }
    return cached[dev];
}

}  // namespace umma

// BF16 hi and lo copies (1024-byte aligned for the tensor maps) and the FP32
// norms, plus slack to align the caller's (256-byte aligned) workspace.
int64_t edm_umma_workspace_bytes(int64_t n, int64_t d) {
    return 1024 + 2 * umma::align_up(n * d * 2, 1024) + umma::align_up(n * 4, 1024);
}

namespace umma {

// One launch of the d < 128 kernel (one CTA per SM) for a map and layout.
template <bool TILES>
static void launch_wide(int map, unsigned ctas, cudaStream_t s, const CUtensorMap &mh, const CUtensorMap &ml,
                        const CUtensorMap &mo, const float *x, const float *nrm, float *out, int64_t n, int d,
                        int nb, int nb2, int gx, int64_t total) {
    const int sm = wide::WSMEM_BYTES;
    if (map == MAP_LAMBDA)
        wide::k_edm_umma_wide<MAP_LAMBDA, TILES><<<ctas, kThreads, sm, s>>>(mh, ml, mo, x, nrm, out, n, d, nb, nb2, gx, total);
    else if (map == MAP_BBOX)
        wide::k_edm_umma_wide<MAP_BBOX, TILES><<<ctas, kThreads, sm, s>>>(mh, ml, mo, x, nrm, out, n, d, nb, nb2, gx, total);
    else if (map == MAP_RB)
        wide::k_edm_umma_wide<MAP_RB, TILES><<<ctas, kThreads, sm, s>>>(mh, ml, mo, x, nrm, out, n, d, nb, nb2, gx, total);
    else
        wide::k_edm_umma_wide<MAP_LINEAR, TILES><<<ctas, kThreads, sm, s>>>(mh, ml, mo, x, nrm, out, n, d, nb, nb2, gx, total);
}

// One launch of the d >= 128 kernel (two-CTA clusters) for a map and layout.
template <bool TILES>
static cudaError_t launch_pairs(int map, const cudaLaunchConfig_t &cfg, const CUtensorMap &mh,
                                const CUtensorMap &ml, const CUtensorMap &mo, const float *x,
                                const float *nrm, float *out, int64_t n, int d, int nb, int nb2, int gx,
                                int64_t total) {
    if (map == MAP_LAMBDA)
        return cudaLaunchKernelEx(&cfg, k_edm_umma<MAP_LAMBDA, TILES>, mh, ml, mo, x, nrm, out, n, d, nb, nb2, gx, total);
    if (map == MAP_BBOX)
        return cudaLaunchKernelEx(&cfg, k_edm_umma<MAP_BBOX, TILES>, mh, ml, mo, x, nrm, out, n, d, nb, nb2, gx, total);
    if (map == MAP_RB)
        return cudaLaunchKernelEx(&cfg, k_edm_umma<MAP_RB, TILES>, mh, ml, mo, x, nrm, out, n, d, nb, nb2, gx, total);
    return cudaLaunchKernelEx(&cfg, k_edm_umma<MAP_LINEAR, TILES>, mh, ml, mo, x, nrm, out, n, d, nb, nb2, gx, total);
}

}  // namespace umma

int edm_umma_run(int64_t n, int64_t d, const float *x, float *out, int map, bool tiles, void *ws,
                 int64_t ws_bytes, cudaStream_t s) {
    using namespace umma;
    if (d % KC != 0) return SIMPLEX_EUNSUPPORTED;
    if (!ws || ws_bytes < edm_umma_workspace_bytes(n, d) || !aligned(ws, 256))
        return SIMPLEX_EWORKSPACE;
    if (tiles && !aligned(out, 16)) return SIMPLEX_EALIGN;   // TMA tensor stores
    const int64_t nb = (n + TM - 1) / TM;
    const Grid g = grid2(nb, map);
    if (!grid_fits(g)) return SIMPLEX_EOVERFLOW;
    if (tiles && nb * (nb + 1) / 2 > INT32_MAX) return SIMPLEX_EOVERFLOW;   // tile coordinate of a store
    unsigned char *w = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(ws) + 1023) & ~uintptr_t(1023));
    __nv_bfloat16 *xh = reinterpret_cast<__nv_bfloat16 *>(w);
    __nv_bfloat16 *xl = reinterpret_cast<__nv_bfloat16 *>(w + align_up(n * d * 2, 1024));
    float *nrm = reinterpret_cast<float *>(w + 2 * align_up(n * d * 2, 1024));
    // 128-byte swizzle, K boxes of 64 for the d < 128 kernel; 64-byte swizzle,
    // K boxes of 32 for the d >= 128 kernel
    CUtensorMap mh, ml, mo;
    std::memset(&mo, 0, sizeof(mo));
    const bool wide_rows = !use_multicast(d);
    if (wide_rows ? (!make_map_bf16(&mh, xh, n, d, d, TM) || !make_map_bf16(&ml, xl, n, d, d, TM))
                  : (!make_map_bf16_sw64(&mh, xh, n, d, d, TM) || !make_map_bf16_sw64(&ml, xl, n, d, d, TM)))
        return SIMPLEX_ECUDA;
    if (tiles && !make_map_tiles_f32(&mo, out, nb * (nb + 1) / 2)) return SIMPLEX_ECUDA;
    int st = smem_optin();
    if (st) return st;
    k_split_bf16<<<(unsigned)((n + 7) / 8), 256, 0, s>>>(x, n, (int)d, xh, xl, nrm);
    note_launches(1);
    if ((st = launch_status())) return st;
    // persistent grid: one CTA per SM walks the map's grid with stride gridDim.x
    int dev = 0, sms = 0;
    if ((st = cuda_status(cudaGetDevice(&dev)))) return st;
    if ((st = cuda_status(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)))) return st;
    // the map's grid of 256 x 256 super-blocks
    const int64_t nb2 = (nb + 1) / 2;
    const Grid g2 = grid2(nb2, map);
    if (!grid_fits(g2)) return SIMPLEX_EOVERFLOW;
    const int64_t total2 = g2.gx * g2.gy;
    if (wide_rows) {
        // one CTA per SM, steps of two horizontally adjacent tiles
        const unsigned ctas = (unsigned)(total2 < sms ? total2 : sms);
        prof_begin(s);
        if (tiles) launch_wide<true>(map, ctas, s, mh, ml, mo, x, nrm, out, n, (int)d, (int)nb, (int)nb2, (int)g2.gx, total2);
        else launch_wide<false>(map, ctas, s, mh, ml, mo, x, nrm, out, n, (int)d, (int)nb, (int)nb2, (int)g2.gx, total2);
    } else {
        // two-CTA clusters
        int64_t clusters = max_pairs(sms);
        if (clusters > total2) clusters = total2;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(2 * clusters));
        cfg.blockDim = dim3(kThreads);
        cfg.dynamicSmemBytes = PSMEM2_BYTES;
        cfg.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 2;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        prof_begin(s);
        const cudaError_t e = tiles ? launch_pairs<true>(map, cfg, mh, ml, mo, x, nrm, out, n, (int)d, (int)nb, (int)nb2, (int)g2.gx, total2)
                                    : launch_pairs<false>(map, cfg, mh, ml, mo, x, nrm, out, n, (int)d, (int)nb, (int)nb2, (int)g2.gx, total2);
        if (e != cudaSuccess) { prof_end(s); return cuda_status(e); }
    }
    prof_end(s);
    note_launches(1);
    return launch_status();
}

int umma_device_errors(cudaStream_t s) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e);
    int h = 0;
    if ((e = cudaMemcpyFromSymbol(&h, umma::g_error, sizeof(int))) != cudaSuccess) return cuda_status(e);
    if (h) {
        const int zero = 0;
        if ((e = cudaMemcpyToSymbol(umma::g_error, &zero, sizeof(int))) != cudaSuccess)
            return cuda_status(e);
        return SIMPLEX_ETIMEOUT;
    }
    return SIMPLEX_OK;
}

}  // namespace sx


