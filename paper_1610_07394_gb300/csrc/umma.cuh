// umma.cuh -- 5th-generation tensor core (tcgen05), TMA and mbarrier helpers
// shared by the tensor-core kernels of libsimplex (inline PTX, sm_103a).
//
// Every wait is bounded: a wait that runs out sets the block's fail flag and
// the translation unit's device error flag, and the caller stops instead of
// hanging.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>

#include <cstdint>
#include <mutex>

#include "maps.cuh"

namespace sx {
namespace umma {

constexpr long long kWaitCycles = 4000000000LL;   // ~2 s at 2 GHz
constexpr uint32_t kSuspendNs = 200000;           // suspend hint of one try_wait

// Instruction descriptor of tcgen05.mma kind::f16 with D = F32 (bits 4-5),
// A = B = BF16 (bits 7-9, 10-12), A / B major-ness (bits 15 / 16: 0 = K-major,
// 1 = MN-major), N >> 3 (bits 17-22), M >> 4 (bits 24-28).
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n, bool a_mn_major, bool b_mn_major) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((a_mn_major ? 1u : 0u) << 15) |
           ((b_mn_major ? 1u : 0u) << 16) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// One potentially blocking test of the phase: the thread may be suspended
// up to kSuspendNs while the phase is incomplete (instead of spinning).
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(phase), "r"(kSuspendNs)
        : "memory");
    return ok != 0;
}

// Waits for the phase of parity `phase` to complete, at most kWaitCycles, or
// until another thread of the block has flagged a failure.  A wait that runs
// out sets *fail and the device flag *gerr.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase, volatile int *fail,
                                          int *gerr) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, phase)) {
        if (*fail) return false;
        if (clock64() - t0 > kWaitCycles) {
            *fail = 1;
            atomicExch(gerr, 1);
            return false;
        }
    }
    return true;
}

// Bounded wait without failure bookkeeping (draining copies on the way out).
__device__ __forceinline__ void mbar_drain(uint32_t bar, uint32_t phase) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, phase) && clock64() - t0 < kWaitCycles) {
    }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// global -> shared bulk copy completing on `bar` (addresses 16-byte aligned,
// size a multiple of 16)
__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes,
                                          uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

// The same 2-D tile load, written at the same shared offset of every CTA of
// the cluster in `mask` and completing on each one's mbarrier at `bar`.
__device__ __forceinline__ void tma_load_2d_mc(uint32_t dst, const CUtensorMap *map, int x, int y,
                                               uint32_t bar, uint16_t mask) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.multicast::cluster"
        " [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar), "h"(mask)
        : "memory");
}

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// Every thread of every CTA of the cluster (release / acquire of shared memory).
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                     : "memory");
}

__device__ __forceinline__ void prefetch_map(const CUtensorMap *map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// shared -> global bulk copy (addresses 16-byte aligned, size a multiple of 16)
__device__ __forceinline__ void bulk_store(float *gdst, uint32_t ssrc, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gdst),
                 "r"(ssrc), "r"(bytes)
                 : "memory");
}

// shared -> global TMA tensor store of one box of a 3-D map (bulk group);
// the box is read from shared memory in the map's swizzle
__device__ __forceinline__ void tma_store_3d(const CUtensorMap *map, uint32_t ssrc, int x, int y, int z) {
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y), "r"(z), "r"(ssrc)
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() {
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

// waits until this thread's committed bulk copies have read their sources
__device__ __forceinline__ void bulk_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

// waits until at most N of this thread's most recent bulk groups are still
// reading their shared-memory sources
template <int N>
__device__ __forceinline__ void bulk_wait_read_le() {
    asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void bulk_wait_all() {
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// generic-proxy shared-memory writes -> visible to the async proxy (TMA, MMA)
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// tcgen05.mma kind::f16 (BF16 in, FP32 accumulate in TMEM): the three
// products of a BF16 hi + lo step, D (+)= Ah Bh + Ah Bl + Al Bh, issued from a
// converged warp.  The whole warp executes the call and one elected lane (the
// lowest active, the same one every time) issues all three, so the
// descriptors stay warp-uniform and the step costs one election; A hi is
// kept in the tensor core's collector buffer for the second product (fill,
// then lastuse), so it is read from shared memory once.  The first product
// accumulates into D when `accumulate` is non-zero, the other two always.
__device__ __forceinline__ void mma_bf16x3_w(uint32_t tmem_d, uint64_t ah, uint64_t al, uint64_t bh,
                                             uint64_t bl, uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p, e, t;\n\t"
        "elect.sync _|e, 0xffffffff;\n\t"
        "setp.ne.b32 p, %6, 0;\n\t"
        "setp.eq.b32 t, %6, %6;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16.collector::a::fill [%0], %1, %3, %5, p;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16.collector::a::lastuse [%0], %1, %4, %5, t;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %2, %3, %5, t;\n\t}" ::"r"(tmem_d),
        "l"(ah), "l"(al), "l"(bh), "l"(bl), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Shared-memory matrix descriptor of an operand tile in the 128-byte swizzle
// layout (8 rows of 128 bytes per 1024-byte atom, 16-byte chunks of row r
// XOR-permuted by r mod 8; tile base 1024-byte aligned, so base offset 0):
// start address >> 4 (bits 0-13), leading byte offset >> 4 (bits 16-29),
// stride byte offset >> 4 (bits 32-45), version 1 (bit 46), swizzle mode
// 2 = 128 B (bits 61-63).
//  K-major (rows are M or N, 64 K-elements per row): the stride offset is
//    the distance between 8-row groups (1024); the leading offset is unused.
//  MN-major (rows are K, 64 M- or N-elements per row): the stride offset is
//    the distance between 8-row groups along K (1024), the leading offset
//    the distance between the 64-element atoms along M or N.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr, uint32_t lbo = 16,
                                               uint32_t sbo = 1024) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// The descriptor of the tile `bytes` further on: the start address field
// (bits 0-13, address >> 4) advanced, valid while the address stays inside
// the 256 KB shared window (no carry out of the field) and `bytes` is a
// multiple of 16.
__device__ __forceinline__ uint64_t desc_add(uint64_t desc, uint32_t bytes) { return desc + (bytes >> 4); }

// The same for an operand tile in the 64-byte swizzle layout (8 rows of 64
// bytes per 512-byte atom, 16-byte chunks of row r XOR-permuted by
// (r / 2) mod 4; tile base 512-byte aligned): K-major, stride offset 512
// between 8-row groups, swizzle mode 4 = 64 B.
__device__ __forceinline__ uint64_t sw64_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(512 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)4 << 61;
    return d;
}

// Arrives on `bar` once every tcgen05 operation issued so far by the elected
// lane has completed (from the same converged warp).
__device__ __forceinline__ void mma_commit_w(uint32_t bar) {
    asm volatile(
        "{\n\t.reg .pred e;\n\t"
        "elect.sync _|e, 0xffffffff;\n\t"
        "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n\t}" ::"r"(bar)
        : "memory");
}

// The same on the mbarrier at `bar` of every CTA of the cluster in `mask`.
__device__ __forceinline__ void mma_commit_mc_w(uint32_t bar, uint16_t mask) {
    asm volatile(
        "{\n\t.reg .pred e;\n\t"
        "elect.sync _|e, 0xffffffff;\n\t"
        "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
        " [%0], %1;\n\t}" ::"r"(bar), "h"(mask)
        : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t cols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem),
                 "r"(cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t cols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(cols)
                 : "memory");
}

// 64 consecutive FP32 columns of this thread's TMEM lane: two loads, one wait.
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, float (&v0)[32], float (&v1)[32]) {
    uint32_t r[64];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]),
          "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]),
          "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]), "=r"(r[49]),
          "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]),
          "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]),
          "=r"(r[62]), "=r"(r[63])
        : "r"(taddr + 32));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int t = 0; t < 32; ++t) {
        v0[t] = __uint_as_float(r[t]);
        v1[t] = __uint_as_float(r[32 + t]);
    }
}

// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int t = 0; t < 16; ++t) v[t] = __uint_as_float(r[t]);
}

// One FP32 column of this thread's TMEM lane.
__device__ __forceinline__ float tmem_ld1(uint32_t taddr) {
    uint32_t r;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r) : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    return __uint_as_float(r);
}

// The super-blocks of a cluster: the map's grid over nb2 = ceil(nb / 2)
// blocks of 256, every cluster-th grid block, both CTAs of a cluster in the
// same order (the multicast of a stage needs both on the same super-block).
template <int MAP>
struct SuperWalk {
    int64_t w, total;
    int wx, wy, gx, nb2, stride, pend, px, py;
    __device__ SuperWalk(int gx_, int64_t total_, int nb2_)
        : total(total_), gx(gx_), nb2(nb2_), pend(0), px(0), py(0) {
        stride = (int)(gridDim.x >> 1);
        w = blockIdx.x >> 1;
        wy = (int)(w / gx_);
        wx = (int)(w - (int64_t)wy * gx_);
    }
    __device__ bool next(int &sX, int &sY) {
        if (pend) { pend = 0; sX = px; sY = py; return true; }
        while (w < total) {
            const List2 L = MAP == MAP_LINEAR ? decode2_linear(w, nb2)
                                              : decode2<MAP>((uint32_t)wx, (uint32_t)wy, nb2);
            w += stride;
            wx += stride;
            while (wx >= gx) { wx -= gx; ++wy; }
            if (L.cnt == 0) continue;
            sX = L.x[0]; sY = L.y[0];
            if (L.cnt > 1) { pend = 1; px = L.x[1]; py = L.y[1]; }
            return true;
        }
        return false;
    }
};

// ---------------------------------------------------------------- host side

// cuTensorMapEncodeTiled through the runtime's driver entry point (the
// library links only the CUDA runtime).
using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                 const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                 const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

inline EncodeTiled encode_fn() {
    static std::once_flag once;
    static EncodeTiled fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
    });
    return fn;
}

// A rows x cols BF16 matrix with row pitch `pitch` elements (pitch * 2 a
// multiple of 16 bytes, base 16-byte aligned), boxes of box_rows rows x 64
// columns (128 bytes: one swizzle row), 128-byte swizzle, zero fill outside.
inline bool make_map_bf16(CUtensorMap *m, void *ptr, int64_t rows, int64_t cols, int64_t pitch,
                          int box_rows) {
    EncodeTiled f = encode_fn();
    if (!f) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)pitch * 2};
    const cuuint32_t box[2] = {64u, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return f(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, ptr, dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The same map with boxes of 32 BF16 (64 bytes) per row in the 64-byte swizzle.
inline bool make_map_bf16_sw64(CUtensorMap *m, void *ptr, int64_t rows, int64_t cols, int64_t pitch,
                               int box_rows) {
    EncodeTiled f = encode_fn();
    if (!f) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)pitch * 2};
    const cuuint32_t box[2] = {32u, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return f(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, ptr, dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The tile-packed EDM output as a 3-D FP32 tensor [tiles][128 rows][128
// columns] (base 16-byte aligned), boxes of 32 columns x 32 rows of one tile
// (4 KB, one 128-byte swizzle row per tile row), 128-byte swizzle.
inline bool make_map_tiles_f32(CUtensorMap *m, float *out, int64_t tiles) {
    EncodeTiled f = encode_fn();
    if (!f) return false;
    const cuuint64_t dims[3] = {128u, 128u, (cuuint64_t)tiles};
    const cuuint64_t strides[2] = {128u * 4u, 128u * 128u * 4u};
    const cuuint32_t box[3] = {32u, 32u, 1u};
    const cuuint32_t estr[3] = {1, 1, 1};
    return f(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, out, dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Shared-memory byte offset of float4 chunk c (0..7) of row r (0..31) inside a
// 32 x 32 FP32 box in the 128-byte swizzle (box base 1024-byte aligned): the
// chunk index is XORed with the row index mod 8, so the 32 lanes of a warp,
// each writing chunk c of its own row, spread over all 32 banks.
__host__ __device__ constexpr uint32_t box_chunk_off(int r, int c) {
    return (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4));
}

inline int64_t align_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

}  // namespace umma
}  // namespace sx
