// atm.cu -- Axilrod-Teller-Muto triple-dipole energy and forces over the
// 3-simplex {i < j < k} (Sec. I: the triple-interaction n-body problem is a
// 3-simplex problem), one 32^3 tile of triples per data block, the block
// chosen by a block-space map (Sec. III-C two-branch map, bounding box, or
// linear enumeration with cube roots).
//
// Per triple (i, j, k) with edge vectors e_ij = x_j - x_i, e_ik = x_k - x_i,
// e_jk = x_k - x_j, softened squares s = |e|^2 + eps, r = s^{-1/2} and unit
// vectors u = e r:
//   cos g_i = u_ij . u_ik,  cos g_j = -u_ij . u_jk,  cos g_k = u_ik . u_jk,
//   e = nu r_ij^3 r_ik^3 r_jk^3 (1 + 3 cos g_i cos g_j cos g_k).
// The cosines are dot products of edge vectors, never the law of cosines on
// squared lengths: for a triangle with one short side the latter cancels
// catastrophically in FP32, and such close triples dominate E.  r^3 is
// formed once per pair as 1/(s sqrt(s)) (two correctly rounded operations),
// so R^3 = r_ij^3 r_ik^3 r_jk^3 carries few roundings.
//
// Tile layout (256 threads): thread (ti, tj), ti, tj in [0, 16), owns the
// four pairs (i, j) = (ti + 16p, tj + 16q), p, q in {0, 1}, and walks the 32
// points k of the third tile.  Pair terms are computed once per tile and
// kept in shared memory: for each (j, k) and (i, k) the unit vector and r^3
// (energy) or r (forces).  The order constraint and the padding past n are
// folded into the pair terms: a pair outside i < j < k < n gets u = 0 and
// r = 0, which zeroes its triples without a branch.  Per-thread sums are
// FP32 within a tile and FP64 across tiles; the block sum is FP64 and one
// FP64 partial per block goes to the workspace, reduced deterministically by
// a second pass.
#include <mutex>

#include "common.cuh"
#include "kernels.h"
#include "umma.cuh"

namespace sx {

constexpr int R_ = kAtmRho;  // 32

// Loads the three point tiles (zero past n).
__device__ __forceinline__ void load_tiles(const float *__restrict__ x, int64_t n, int I, int J,
                                           int K, float4 (*xs)[R_]) {
    const int tid = threadIdx.x;
    if (tid < 3 * R_) {
        const int which = tid / R_, o = tid % R_;
        const int blk = which == 0 ? I : which == 1 ? J : K;
        const int64_t g = (int64_t)blk * R_ + o;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (g < n) v = make_float4(__ldg(x + 3 * g), __ldg(x + 3 * g + 1), __ldg(x + 3 * g + 2), 0.f);
        xs[which][o] = v;
    }
}

// Pair terms: (u, r^3) of the edge from -> to, zero outside the simplex.
__device__ __forceinline__ float4 edge(float4 from, float4 to) {
    return make_float4(to.x - from.x, to.y - from.y, to.z - from.z, 0.0f);
}

__device__ __forceinline__ float4 pair_term(float4 from, float4 to, bool valid, float eps) {
    const float4 e = edge(from, to);
    if (!valid) return make_float4(0.f, 0.f, 0.f, 0.f);
    const float s = fmaf(e.x, e.x, fmaf(e.y, e.y, fmaf(e.z, e.z, eps)));
    const float q = sqrtf(s);
    const float r = 1.0f / q;
    return make_float4(e.x * r, e.y * r, e.z * r, 1.0f / (s * q));
}

__device__ __forceinline__ float dot3(float4 a, float4 b) {
    return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z));
}

// Energy tables, laid out for packed FP32x2 arithmetic over the thread's two
// i-slots p = 0, 1 (i = ti and ti + 16):
//   ec[k][0][ti] = (u_ik0.x, u_ik1.x, u_ik0.y, u_ik1.y), ec[k][1][ti] = (u_ik0.z, u_ik1.z, r_ik0^3, r_ik1^3)
//   eb[k][q][0][tj] = (u.x, u.x, u.y, u.y), eb[k][q][1][tj] = (u.z, u.z, r^3, r^3) of pair (j = tj + 16q, k),
// each (j, k) value duplicated so one broadcast load feeds both lanes.  A
// warp's 16 distinct ti read 256 contiguous bytes (two wavefronts, no bank
// conflict); its two tj read two addresses (one broadcast wavefront).
struct AtmEnergySmem {
    float4 xs[3][R_];
    float4 ec[R_][2][16];
    float4 eb[R_][2][2][16];
};

__device__ __forceinline__ void put_pair(float4 &lo, float4 &hi, int lane, float4 v) {
    float *a = reinterpret_cast<float *>(&lo), *b = reinterpret_cast<float *>(&hi);
    a[lane] = v.x; a[2 + lane] = v.y; b[lane] = v.z; b[2 + lane] = v.w;
}

__device__ __forceinline__ void build_energy_tables(int64_t n, int I, int J, int K, float eps,
                                                    AtmEnergySmem &S) {
    for (int e = threadIdx.x; e < R_ * R_; e += 256) {
        const int k = e >> 5, o = e & 31, half = o >> 4, t = o & 15;
        const int64_t gi = (int64_t)I * R_ + o, gj = (int64_t)J * R_ + o, gk = (int64_t)K * R_ + k;
        const float4 c = pair_term(S.xs[0][o], S.xs[2][k], gi < gk && gk < n, eps);
        put_pair(S.ec[k][0][t], S.ec[k][1][t], half, c);
        const float4 b = pair_term(S.xs[1][o], S.xs[2][k], gj < gk && gk < n, eps);
        S.eb[k][half][0][t] = make_float4(b.x, b.x, b.y, b.y);
        S.eb[k][half][1][t] = make_float4(b.z, b.z, b.w, b.w);
    }
}

__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }

// Two triples (i0, j, k) and (i1, j, k) in the two lanes: with the unit
// vectors of the pairs and the product w = r_ik^3 r_jk^3,
//   acc += w (1 - 3 (u_ij.u_ik)(u_ij.u_jk)(u_ik.u_jk)),
// i.e. the term e / (nu r_ij^3) (cos g_j = -u_ij.u_jk); r_ij^3 multiplies the
// sum over k afterwards.  14 packed FP32x2 operations.
__device__ __forceinline__ void triple_energy2(const float2 (&uij)[3], float4 C0, float4 C1,
                                               float4 B0, float4 B1, float2 &acc) {
    const float2 cx = lo2(C0), cy = hi2(C0), cz = lo2(C1), cw = hi2(C1);
    const float2 bx = lo2(B0), by = hi2(B0), bz = lo2(B1), bw = hi2(B1);
    const float2 ci = __ffma2_rn(uij[0], cx, __ffma2_rn(uij[1], cy, __fmul2_rn(uij[2], cz)));
    const float2 cj = __ffma2_rn(uij[0], bx, __ffma2_rn(uij[1], by, __fmul2_rn(uij[2], bz)));
    const float2 ck = __ffma2_rn(cx, bx, __ffma2_rn(cy, by, __fmul2_rn(cz, bz)));
    const float2 c3 = __fmul2_rn(__fmul2_rn(ci, cj), ck);
    const float2 t = __ffma2_rn(make_float2(-3.0f, -3.0f), c3, make_float2(1.0f, 1.0f));
    acc = __ffma2_rn(__fmul2_rn(cw, bw), t, acc);
}

// Two triples (i0, j, k), (i1, j, k) in the two lanes, from the scaled
// vectors v = r^(3/2) u of the pair tables:
//   s0 += r_ik^3 r_jk^3,
//   s1 += (v_ij.v_ik)(v_ij.v_jk)(v_ik.v_jk) = r_ij^3 r_ik^3 r_jk^3 (u_ij.u_ik)(u_ij.u_jk)(u_ik.u_jk),
// so that the energy of the pair (i, j) over its k is r_ij^3 s0 - 3 s1
// (cos g_j = -u_ij.u_jk).  12 packed FP32x2 operations.
__device__ __forceinline__ void triple_energy2s(const float2 (&vij)[3], float4 C0, float4 C1,
                                                float4 B0, float4 B1, float2 &s0, float2 &s1) {
    const float2 cx = lo2(C0), cy = hi2(C0), cz = lo2(C1), cw = hi2(C1);
    const float2 bx = lo2(B0), by = hi2(B0), bz = lo2(B1), bw = hi2(B1);
    const float2 ci = __ffma2_rn(vij[0], cx, __ffma2_rn(vij[1], cy, __fmul2_rn(vij[2], cz)));
    const float2 cj = __ffma2_rn(vij[0], bx, __ffma2_rn(vij[1], by, __fmul2_rn(vij[2], bz)));
    const float2 ck = __ffma2_rn(cx, bx, __ffma2_rn(cy, by, __fmul2_rn(cz, bz)));
    s1 = __ffma2_rn(__fmul2_rn(ci, cj), ck, s1);
    s0 = __ffma2_rn(cw, bw, s0);
}

// The grid's z-layers run in reverse launch order (block z decodes grid layer
// gz - 1 - z): the lambda map's last layers hold the J = K plane, whose
// diagonal-pair row gives blocks two tiles each; launched first, they finish
// inside the grid instead of trailing its last wave.  The map is unchanged.

// The (up to two) data blocks of a grid block, read without dynamic indexing.
__device__ __forceinline__ void block_of(const List3 &L, int t, int &I, int &J, int &K) {
    I = t ? L.i[1] : L.i[0];
    J = t ? L.j[1] : L.j[0];
    K = t ? L.k[1] : L.k[0];
}

template <int MAP>
__global__ void __launch_bounds__(256, 4) k_atm_energy(int64_t n, const float *__restrict__ x,
                                                       float nu, float eps, int nb, int p,
                                                       double *__restrict__ partials) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    AtmEnergySmem &S = *reinterpret_cast<AtmEnergySmem *>(smem_raw);
    __shared__ float red[16];
    const List3 L = decode3<MAP>(blockIdx.x, blockIdx.y, gridDim.z - 1 - blockIdx.z, p, nb);
    if (L.cnt == 0) {   // a block outside the simplex exits at once
        if (threadIdx.x == 0)
            partials[blockIdx.x + (int64_t)gridDim.x * (blockIdx.y + (int64_t)gridDim.y * blockIdx.z)] = 0.0;
        return;
    }
    const int ti = threadIdx.x & 15, tj = threadIdx.x >> 4;
    float hi = 0.f, lo = 0.f;
#pragma unroll 1
    for (int t = 0; t < L.cnt; ++t) {
        int I, J, K;
        block_of(L, t, I, J, K);
        if (t) __syncthreads();
        load_tiles(x, n, I, J, K, S.xs);
        __syncthreads();
        build_energy_tables(n, I, J, K, eps, S);
        // pair constants: u_ij of slots (p, q) packed over p, and r_ij^3
        float2 uij[2][3];
        float ra3[2][2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int64_t gj = (int64_t)J * R_ + tj + 16 * q;
            const float4 u0 = pair_term(S.xs[0][ti], S.xs[1][tj + 16 * q],
                                              (int64_t)I * R_ + ti < gj && gj < n, eps);
            const float4 u1 = pair_term(S.xs[0][ti + 16], S.xs[1][tj + 16 * q],
                                              (int64_t)I * R_ + ti + 16 < gj && gj < n, eps);
            uij[q][0] = make_float2(u0.x, u1.x);
            uij[q][1] = make_float2(u0.y, u1.y);
            uij[q][2] = make_float2(u0.z, u1.z);
            ra3[0][q] = u0.w;
            ra3[1][q] = u1.w;
        }
        __syncthreads();
        float2 acc0 = make_float2(0.f, 0.f), acc1 = make_float2(0.f, 0.f);
#pragma unroll 4
        for (int k = 0; k < R_; ++k) {
            const float4 C0 = S.ec[k][0][ti], C1 = S.ec[k][1][ti];
            const float4 B00 = S.eb[k][0][0][tj], B01 = S.eb[k][0][1][tj];
            const float4 B10 = S.eb[k][1][0][tj], B11 = S.eb[k][1][1][tj];
            triple_energy2(uij[0], C0, C1, B00, B01, acc0);
            triple_energy2(uij[1], C0, C1, B10, B11, acc1);
        }
        add_ff(hi, lo, acc0.x * ra3[0][0], 0.f);
        add_ff(hi, lo, acc0.y * ra3[1][0], 0.f);
        add_ff(hi, lo, acc1.x * ra3[0][1], 0.f);
        add_ff(hi, lo, acc1.y * ra3[1][1], 0.f);
    }
    const double s = block_sum_ff<256>(hi, lo, red);
    if (threadIdx.x == 0) {
        const int64_t bid = blockIdx.x + (int64_t)gridDim.x * (blockIdx.y + (int64_t)gridDim.y * blockIdx.z);
        partials[bid] = (double)nu * s;
    }
}

// ---------------------------------------------------------------- pair tables

// The pair table of every block pair (B1 <= B2) of the 2-simplex of blocks,
// computed once per call instead of once per tile.  For the pairs (a in B1,
// b in B2) it holds the scaled edge vector v = r^(3/2) u (u = r (x_b - x_a))
// and r^3 = (|x_b - x_a|^2 + eps)^-3/2, all zero unless a < b < n, packed
// over pairs of consecutive b for FP32x2 arithmetic:
//   tab[h][0][a] = (v_b0.x, v_b1.x, v_b0.y, v_b1.y),
//   tab[h][1][a] = (v_b0.z, v_b1.z, r_b0^3, r_b1^3),   b0 = 2h, b1 = 2h + 1.
// One form serves every role: a tile (I, J, K) copies the tables of (I, K)
// and (J, K) into shared memory as they are (one bulk copy each) and reads
// its pair constants (i, j) from the table of (I, J).  With the scaled
// vectors the product of the three dot products of a triple is
// r_ij^3 r_ik^3 r_jk^3 (u_ij.u_ik)(u_ij.u_jk)(u_ik.u_jk) directly
// (triple_energy2s).
constexpr int kTabPair = (R_ / 2) * 2 * R_;        // float4 per block pair (16 KB)
constexpr int64_t kTabMaxBytes = int64_t(8) << 30; // larger tables: per-tile tables instead

// (r^(3/2) u, r^3) of the edge from -> to, zero outside the simplex.
__device__ __forceinline__ float4 scaled_pair_term(float4 from, float4 to, bool valid, float eps) {
    const float4 c = pair_term(from, to, valid, eps);
    const float h = sqrtf(c.w);
    return make_float4(c.x * h, c.y * h, c.z * h, c.w);
}

__host__ __device__ inline int64_t pair_slot(int B1, int B2) {
    return (int64_t)B2 * (B2 + 1) / 2 + B1;
}

inline int64_t atm_table_bytes(int64_t nb) { return nb * (nb + 1) / 2 * kTabPair * 16; }

template <int MAP>
__global__ void __launch_bounds__(256) k_atm_pairtab(int64_t n, const float *__restrict__ x,
                                                     float eps, int nb, float4 *__restrict__ tab) {
    __shared__ float4 xs[2][R_];
    const List2 L = decode2<MAP>(blockIdx.x, blockIdx.y, nb);
    const int tid = threadIdx.x;
#pragma unroll 1
    for (int t = 0; t < L.cnt; ++t) {
        const int B1 = t ? L.x[1] : L.x[0], B2 = t ? L.y[1] : L.y[0];
        if (t) __syncthreads();
        if (tid < 2 * R_) {
            const int which = tid / R_, o = tid % R_;
            const int64_t g = (int64_t)(which ? B2 : B1) * R_ + o;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (g < n) v = make_float4(__ldg(x + 3 * g), __ldg(x + 3 * g + 1), __ldg(x + 3 * g + 2), 0.f);
            xs[which][o] = v;
        }
        __syncthreads();
        float4 *out = tab + pair_slot(B1, B2) * kTabPair;
        for (int e = tid; e < (R_ / 2) * R_; e += 256) {
            const int h = e / R_, a = e % R_, b0 = 2 * h, b1 = 2 * h + 1;
            const int64_t ga = (int64_t)B1 * R_ + a;
            const int64_t g0 = (int64_t)B2 * R_ + b0, g1 = (int64_t)B2 * R_ + b1;
            const float4 u0 = scaled_pair_term(xs[0][a], xs[1][b0], ga < g0 && g0 < n, eps);
            const float4 u1 = scaled_pair_term(xs[0][a], xs[1][b1], ga < g1 && g1 < n, eps);
            out[(2 * h) * R_ + a] = make_float4(u0.x, u1.x, u0.y, u1.y);
            out[(2 * h + 1) * R_ + a] = make_float4(u0.z, u1.z, u0.w, u1.w);
        }
    }
}

__device__ int g_atm_error;   // set when a bounded wait of the energy kernel runs out

// A tile's two tables: ik = table of (I, K) (a = i, b = k), jk = table of
// (J, K) (a = j, b = k).  A warp of k_atm_energy_tab reads 8 distinct i of ik
// (128 contiguous bytes) and 4 distinct j of jk per load: no bank conflict.
struct AtmEnergyTabSmem {
    float4 ik[R_ / 2][2][R_];
    float4 jk[R_ / 2][2][R_];
    uint64_t bar;
};

// v_ij of the pair (i, j) of a tile in both lanes, from the (I, J) table
// (entry a = i, lane j & 1 of the step holding b = j).
__device__ __forceinline__ void pair_const(const float4 *__restrict__ tij, int i, int j, float2 (&v)[3]) {
    const float4 *e = tij + (j >> 1) * 2 * R_ + i;
    const float4 a = __ldg(e), b = __ldg(e + R_);
    const bool odd = j & 1;
    const float vx = odd ? a.y : a.x, vy = odd ? a.w : a.z, vz = odd ? b.y : b.x;
    v[0] = make_float2(vx, vx);
    v[1] = make_float2(vy, vy);
    v[2] = make_float2(vz, vz);
}

// r_ij^3 of the pair (i, j) from the (I, J) table.
__device__ __forceinline__ float pair_r3(const float4 *__restrict__ tij, int i, int j) {
    const float4 b = __ldg(tij + (j >> 1) * 2 * R_ + R_ + i);
    return (j & 1) ? b.w : b.z;
}

// Bounded wait for a tile's tables; a timeout flags the error and drains
// (bounded), and the block then finishes with a NaN result.
__device__ __forceinline__ void wait_tables(uint32_t bar, uint32_t parity, bool &bad) {
    if (bad) return;
    const long long t0 = clock64();
    while (!umma::mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > umma::kWaitCycles) {
            atomicExch(&g_atm_error, 1);
            umma::mbar_drain(bar, parity);
            bad = true;
            return;
        }
    }
}

// The energy kernel fed by the pair tables, register-blocked.  Per tile, one
// thread starts two bulk copies (2 x 16 KB) of the (I, K) and (J, K) tables
// into shared memory and every thread reads its pair constants (v_ij, r_ij^3)
// from the (I, J) table meanwhile; then a packed triple loop over the scaled
// vectors (triple_energy2s) whose two lanes are two consecutive k.  128
// threads per tile, thread (ti, tj) = (t mod 8, t / 8) owns the 4 x 2 pairs
// (i, j) = (ti + 8 p, tj + 16 q), and per step (two consecutive k) loads
// the four (i, k) and the two (j, k) table entries: 12 shared loads of
// 128 bits for 16 triples, where 2 x 2 pairs per thread take 8 for 8.  A
// 128-bit shared load takes two wavefronts when a warp's lanes read at most
// a few distinct 16-byte words and four when they read eight or more, so
// per step a warp of this layout spends 8 x 4 on its (i, k) loads (eight
// distinct i) and 4 x 2 on its (j, k) loads (four distinct j): 40
// wavefronts for 512 triples, against 24 for 256 in the 2 x 2 layout (16
// distinct i, two distinct j), four schedulers sharing the one
// shared-memory pipe.  Tiles on a diagonal plane run the same loop (their
// tables are zero outside i < j < k; skipping their empty steps, as the 2 x 2
// layout did, changed nothing here).  Four blocks per SM (120 registers): at
// n = 1024 the kernel takes 0.0944 ms against 0.0979 ms with 2 x 2 pairs per
// thread and 256 threads, at n = 4096 2.22e12 triples/s against 2.12e12.
template <int MAP>
__global__ void __launch_bounds__(128, 4) k_atm_energy_tab(const float4 *__restrict__ tab, float nu, int nb,
                                                           int p, double *__restrict__ partials) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    AtmEnergyTabSmem &S = *reinterpret_cast<AtmEnergyTabSmem *>(smem_raw);
    __shared__ float red[8];
    const List3 L = decode3<MAP>(blockIdx.x, blockIdx.y, gridDim.z - 1 - blockIdx.z, p, nb);
    const int64_t bid = blockIdx.x + (int64_t)gridDim.x * (blockIdx.y + (int64_t)gridDim.y * blockIdx.z);
    if (L.cnt == 0) {   // a block outside the simplex exits at once
        if (threadIdx.x == 0) partials[bid] = 0.0;
        return;
    }
    const int ti = threadIdx.x & 7, tj = threadIdx.x >> 3;
    const uint32_t bar = umma::smem_u32(&S.bar);
    if (threadIdx.x == 0) {
        umma::mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    float hi = 0.f, lo = 0.f;
    bool bad = false;
#pragma unroll 1
    for (int t = 0; t < L.cnt; ++t) {
        int I, J, K;
        block_of(L, t, I, J, K);
        if (t) __syncthreads();   // every thread is done with the previous tile's tables
        if (threadIdx.x == 0 && !bad) {
            umma::mbar_expect_tx(bar, (uint32_t)(2 * kTabPair * 16));
            umma::bulk_load(umma::smem_u32(&S.ik[0][0][0]), tab + pair_slot(I, K) * kTabPair,
                            kTabPair * 16, bar);
            umma::bulk_load(umma::smem_u32(&S.jk[0][0][0]), tab + pair_slot(J, K) * kTabPair,
                            kTabPair * 16, bar);
        }
        const float4 *tij = tab + pair_slot(I, J) * kTabPair;
        float2 vij[4][2][3];
#pragma unroll
        for (int pp = 0; pp < 4; ++pp)
#pragma unroll
            for (int q = 0; q < 2; ++q) pair_const(tij, ti + 8 * pp, tj + 16 * q, vij[pp][q]);
        wait_tables(bar, (uint32_t)t & 1, bad);
        float2 s0[4][2], s1[4][2];
#pragma unroll
        for (int pp = 0; pp < 4; ++pp)
#pragma unroll
            for (int q = 0; q < 2; ++q) s0[pp][q] = s1[pp][q] = make_float2(0.f, 0.f);
#pragma unroll 1
        for (int h = 0; h < R_ / 2; ++h) {
            const float4 B00 = S.jk[h][0][tj], B01 = S.jk[h][1][tj];
            const float4 B10 = S.jk[h][0][tj + 16], B11 = S.jk[h][1][tj + 16];
#pragma unroll
            for (int pp = 0; pp < 4; ++pp) {
                const float4 C0 = S.ik[h][0][ti + 8 * pp], C1 = S.ik[h][1][ti + 8 * pp];
                triple_energy2s(vij[pp][0], C0, C1, B00, B01, s0[pp][0], s1[pp][0]);
                triple_energy2s(vij[pp][1], C0, C1, B10, B11, s0[pp][1], s1[pp][1]);
            }
        }
#pragma unroll
        for (int pp = 0; pp < 4; ++pp)
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const float ra3 = pair_r3(tij, ti + 8 * pp, tj + 16 * q);
                add_ff(hi, lo, fmaf(ra3, s0[pp][q].x + s0[pp][q].y, -3.0f * (s1[pp][q].x + s1[pp][q].y)), 0.f);
            }
    }
    const bool any_bad = __syncthreads_or(bad) != 0;
    const double s = block_sum_ff<128>(hi, lo, red);
    if (threadIdx.x == 0) partials[bid] = any_bad ? __longlong_as_double(0x7ff8000000000000LL) : (double)nu * s;
}

// ---------------------------------------------------------------- forces

// Pair terms of the forces, from the edge vector e = x_b - x_a of a pair and
// its softened square s = |e|^2 + eps: the scaled edge w = e / s (= r u with
// r = s^-1/2, u the unit vector), s, r^3 = s^-3/2 and q = 1/s = r^2; all zero
// outside the simplex.  With scaled edges the vertex dot products of a
// triangle (sides a = ij, b = jk, c = ik) carry the r factors the
// derivatives need:
//   P_i = w_ij . w_ik = cos_i r_a r_c,   P_j = w_ij . w_jk = -cos_j r_a r_b,
//   P_k = w_ik . w_jk = cos_k r_b r_c,
// so X = cos_j cos_k r_a r_c = -P_j P_k s_b, Y = cos_i cos_k r_a r_b =
// P_i P_k s_c, Z = cos_i cos_j r_b r_c = -P_i P_j s_a and the cosine product
// Cp = -P_i P_j P_k s_a s_b s_c.
struct PairTerms {
    float wx, wy, wz, s, r3, q;
};

__device__ __forceinline__ PairTerms pair_terms(float4 from, float4 to, bool valid, float eps) {
    PairTerms t;
    if (!valid) { t.wx = t.wy = t.wz = t.s = t.r3 = t.q = 0.0f; return t; }
    const float4 e = edge(from, to);
    const float s = fmaf(e.x, e.x, fmaf(e.y, e.y, fmaf(e.z, e.z, eps)));
    const float sq = sqrtf(s);
    t.s = s;
    t.q = 1.0f / s;
    t.r3 = 1.0f / (s * sq);
    t.wx = e.x * t.q; t.wy = e.y * t.q; t.wz = e.z * t.q;
    return t;
}

// Force tables, laid out for packed FP32x2 arithmetic over the thread's two
// i-slots p (lanes x, y: i = ti and ti + 16):
//   fc[k][0][ti] = (w_ik0.x, w_ik1.x, w_ik0.y, w_ik1.y)
//   fc[k][1][ti] = (w_ik0.z, w_ik1.z, s_ik0,   s_ik1)
//   fc[k][2][ti] = (r_ik0^3, r_ik1^3, q_ik0,   q_ik1)
//   fb[k][h][0..2][tj] = the same three vectors of pair (j = tj + 16 h, k),
//   each value duplicated into both lanes (one broadcast load feeds both).
// A persistent block walks many tiles: the side-coefficient matrices and the
// point tiles are double-buffered (tile t uses buffer t & 1) so that the next
// tile's tables, points and pair constants load while this tile's forces
// are assembled; the (i, k) sums, which the triple loop adds atomically into
// a zeroed matrix, are triple-buffered (buffer t mod 3), so that the matrix
// of tile t + 2 is zeroed during tile t and one block barrier per tile
// orders everything.
struct AtmForceSmem {
    float4 fc[R_][3][16];
    float4 fb[R_][2][3][16];
    float4 xs[2][3][R_];
    float wjk[2][R_][R_ + 1];   // [k][j]: sum over i of de/db
    float wik[3][R_][R_ + 1];   // [k][i]: sum over j of de/dc
    float wij[2][R_][R_ + 1];   // [i][j]: sum over k of de/da
    uint64_t bar;               // the tile's force tables landed (table-fed kernel)
    int tq[2][4];               // tiles t and t + 1: (I, J, K, valid), slot t & 1
    long long walk_w;           // the grid block being split into tiles
    long long walk_end;         // end of the run of grid blocks the block has claimed
    int walk_sub;               // the next tile of walk_w
    int walk_pos[4];            // walk_w's place in the hand-out order (HandoutPos)
};

__device__ __forceinline__ void build_force_tables(int64_t n, int I, int J, int K, float eps,
                                                   const float4 (*xs)[R_], AtmForceSmem &S) {
    for (int e = threadIdx.x; e < R_ * R_; e += 256) {
        const int k = e >> 5, o = e & 31, half = o >> 4, t = o & 15;
        const int64_t gi = (int64_t)I * R_ + o, gj = (int64_t)J * R_ + o, gk = (int64_t)K * R_ + k;
        const PairTerms c = pair_terms(xs[0][o], xs[2][k], gi < gk && gk < n, eps);
        put_pair(S.fc[k][0][t], S.fc[k][1][t], half, make_float4(c.wx, c.wy, c.wz, c.s));
        float *f2 = reinterpret_cast<float *>(&S.fc[k][2][t]);
        f2[half] = c.r3; f2[2 + half] = c.q;
        const PairTerms b = pair_terms(xs[1][o], xs[2][k], gj < gk && gk < n, eps);
        S.fb[k][half][0][t] = make_float4(b.wx, b.wx, b.wy, b.wy);
        S.fb[k][half][1][t] = make_float4(b.wz, b.wz, b.s, b.s);
        S.fb[k][half][2][t] = make_float4(b.r3, b.r3, b.q, b.q);
    }
}

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// The pair (i, j) of a thread's i-slots (both lanes) as the triple loop uses
// it: the scaled edge w_ij, s_a, q_a = 1/s_a and g_a = 1.5 r_a^3.
struct PairPack {
    float2 wx, wy, wz;
    float2 sa, qa, ga;
};

// Two triples (i0, j, k), (i1, j, k) in the two lanes.  With e = R^3 (1 + 3 Cp)
// (R^3 = r_a^3 r_b^3 r_c^3) and its derivatives by the squared sides
//   de/da = 1.5 R^3 (X + Y - Z - H q_a),  de/db = 1.5 R^3 (Y + Z - X - H q_b),
//   de/dc = 1.5 R^3 (X + Z - Y - H q_c),  H = 1 + 5 Cp
// (from e = P^-3/2 + 3 D P^-5/2, P = s_a s_b s_c, D the product of the three
// vertex dot products), written with g = 1.5 R^3 and S = X + Y + Z as
//   e = g (2/3 + 2 Cp),  de/da = g (S - 2 Z - H q_a), ...
// The energy goes to acc, de/da to wa (summed over k in registers), de/dc to
// ecs (summed over the thread's two j) and de/db, summed over the two
// i-lanes, is returned.  32 packed operations and one scalar add.
__device__ __forceinline__ float triple_grad2(const PairPack &c, float4 C0, float4 C1, float4 C2,
                                              float4 B0, float4 B1, float4 B2, float2 &acc,
                                              float2 &wa, float2 &ecs) {
    const float2 cx = f2(C0.x, C0.y), cy = f2(C0.z, C0.w), cz = f2(C1.x, C1.y), sc = f2(C1.z, C1.w);
    const float2 rc3 = f2(C2.x, C2.y), qc = f2(C2.z, C2.w);
    const float2 bx = f2(B0.x, B0.y), by = f2(B0.z, B0.w), bz = f2(B1.x, B1.y), sb = f2(B1.z, B1.w);
    const float2 rb3 = f2(B2.x, B2.y), qb = f2(B2.z, B2.w);
    const float2 pi = fma2(c.wx, cx, fma2(c.wy, cy, mul2(c.wz, cz)));
    const float2 pj = fma2(c.wx, bx, fma2(c.wy, by, mul2(c.wz, bz)));
    const float2 pk = fma2(cx, bx, fma2(cy, by, mul2(cz, bz)));
    const float2 t1 = mul2(pk, sb), t2 = mul2(pk, sc);     // shared by X, Y and Cp
    const float2 xn = mul2(pj, t1);                         // -X
    const float2 y = mul2(pi, t2);                          //  Y
    const float2 zn = mul2(mul2(pi, pj), c.sa);             // -Z
    const float2 cpn = mul2(mul2(zn, t1), sc);              // -Cp = -Z pk sb sc
    const float2 g = mul2(c.ga, mul2(rb3, rc3));            // 1.5 R^3
    acc = fma2(g, fma2(f2(-2.0f, -2.0f), cpn, f2(2.0f / 3.0f, 2.0f / 3.0f)), acc);
    const float2 nh = fma2(f2(5.0f, 5.0f), cpn, f2(-1.0f, -1.0f));   // -H
    // S - 2Z, S - 2Y, S - 2X with S = X + Y + Z, from w = S - 2X = y + xn - zn:
    // S - 2Z = 2y - w, S - 2Y = -2zn - w (the negated addend folds into the FMA)
    const float2 w = add2(fma2(zn, f2(-1.0f, -1.0f), y), xn);
    const float2 nw = f2(-w.x, -w.y);
    wa = fma2(g, fma2(nh, c.qa, fma2(f2(2.0f, 2.0f), y, nw)), wa);
    ecs = fma2(g, fma2(nh, qc, fma2(f2(-2.0f, -2.0f), zn, nw)), ecs);
    const float2 eb = mul2(g, fma2(nh, qb, w));
    return eb.x + eb.y;
}

// Sum over the 16 lanes of a half-warp (xor 8, 4, 2, 1) of 16 values per
// lane, scattered: lane l ends with the total of value l & 15.  30 shuffles
// and adds instead of 16 full reductions.
__device__ __forceinline__ float reduce_scatter16(float (&v)[16], int lane) {
#pragma unroll
    for (int w = 8; w >= 1; w >>= 1) {
        const bool up = (lane & w) != 0;
#pragma unroll
        for (int m = 0; m < w; ++m) {
            const float send = up ? v[m] : v[m + w];
            const float keep = up ? v[m + w] : v[m];
            v[m] = keep + __shfl_xor_sync(0xffffffffu, send, w);
        }
    }
    return v[0];
}

// ---------------------------------------------------------------- force tables

// The force tables of every block pair (B1 <= B2) of the 2-simplex of
// blocks, computed once per call instead of once per tile, in the layout of
// AtmForceSmem's fc and fb so that a tile (I, J, K) copies the tables of
// (I, K) and (J, K) into shared memory as they are:
//   fc form [b][3][16]: pairs (a = t, b) and (a = t + 16, b) in the two
//       lanes of (w.x, w.y), (w.z, s), (r^3, q);
//   fb form [b][2][3][16]: pair (a = t + 16 h, b), each value in both lanes;
// from pair_terms, zero unless a < b < n.  72 KB per block pair.
constexpr int kFTabFc = R_ * 3 * 16;               // float4 of the fc form (24 KB)
constexpr int kFTabFb = R_ * 2 * 3 * 16;           // float4 of the fb form (48 KB)
constexpr int kFTabPair = kFTabFc + kFTabFb;       // float4 per block pair (72 KB)
constexpr int64_t kFTabMaxBytes = int64_t(16) << 30;   // larger: per-tile tables instead

template <int MAP>
__global__ void __launch_bounds__(256) k_atm_forcetab(int64_t n, const float *__restrict__ x,
                                                      float eps, int nb, float4 *__restrict__ tab) {
    __shared__ float4 xs[2][R_];
    const List2 L = decode2<MAP>(blockIdx.x, blockIdx.y, nb);
    const int tid = threadIdx.x;
#pragma unroll 1
    for (int t = 0; t < L.cnt; ++t) {
        const int B1 = t ? L.x[1] : L.x[0], B2 = t ? L.y[1] : L.y[0];
        if (t) __syncthreads();
        if (tid < 2 * R_) {
            const int which = tid / R_, o = tid % R_;
            const int64_t g = (int64_t)(which ? B2 : B1) * R_ + o;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (g < n) v = make_float4(__ldg(x + 3 * g), __ldg(x + 3 * g + 1), __ldg(x + 3 * g + 2), 0.f);
            xs[which][o] = v;
        }
        __syncthreads();
        float4 *fc = tab + pair_slot(B1, B2) * kFTabPair;
        float4 *fb = fc + kFTabFc;
        for (int e = tid; e < R_ * 16; e += 256) {
            const int b = e >> 4, a = e & 15;
            const int64_t gb = (int64_t)B2 * R_ + b, ga = (int64_t)B1 * R_ + a;
            const PairTerms c0 = pair_terms(xs[0][a], xs[1][b], ga < gb && gb < n, eps);
            const PairTerms c1 = pair_terms(xs[0][a + 16], xs[1][b], ga + 16 < gb && gb < n, eps);
            fc[(3 * b + 0) * 16 + a] = make_float4(c0.wx, c1.wx, c0.wy, c1.wy);
            fc[(3 * b + 1) * 16 + a] = make_float4(c0.wz, c1.wz, c0.s, c1.s);
            fc[(3 * b + 2) * 16 + a] = make_float4(c0.r3, c1.r3, c0.q, c1.q);
            fb[((2 * b + 0) * 3 + 0) * 16 + a] = make_float4(c0.wx, c0.wx, c0.wy, c0.wy);
            fb[((2 * b + 0) * 3 + 1) * 16 + a] = make_float4(c0.wz, c0.wz, c0.s, c0.s);
            fb[((2 * b + 0) * 3 + 2) * 16 + a] = make_float4(c0.r3, c0.r3, c0.q, c0.q);
            fb[((2 * b + 1) * 3 + 0) * 16 + a] = make_float4(c1.wx, c1.wx, c1.wy, c1.wy);
            fb[((2 * b + 1) * 3 + 1) * 16 + a] = make_float4(c1.wz, c1.wz, c1.s, c1.s);
            fb[((2 * b + 1) * 3 + 2) * 16 + a] = make_float4(c1.r3, c1.r3, c1.q, c1.q);
        }
    }
}

// The tiles of a persistent block, handed out dynamically: one thread claims
// the next run of `claim` grid blocks from a counter shared by all blocks of
// the launch (atomicAdd) and splits them into their tiles (up to two per
// grid block; blocks outside the simplex give none), so the work is balanced
// whatever each block's share of idle grid blocks.  A run of up to 8 grid
// blocks per atomic keeps the claims off the loader's path where the map's
// grid is mostly idle (lambda at a non-power of two pads nb up to p; at
// n = 12000 25.3 M grid blocks hold 8.9 M tiles), and the host keeps at
// least 64 claims per persistent block.  The walk state lives in shared
// memory.
//
// Order of the hand-out.  A tile (I, J, K) reads the tables of (I, K) and
// (J, K).  In the map's grid order (x fastest, then y, then z) one of the two
// changes with every block, and half of the lambda cube (its reflected case,
// (J, K) = (h + x, h + y)) meets a table again only one whole z-layer later,
// far beyond the L2.  So where the grid's x and y extents are multiples of 8
// the counter walks 8 x 8 patches of the (x, y) plane, and within a patch all
// z-layers (from the top: the J = K plane's layers of two tiles per block go
// first) before the next patch; within a layer the 64 blocks of the patch.
// Every (I, K) and (J, K) table is then used about eight times within a
// patch's span of tiles.  Which grid blocks exist, and the data blocks they
// map to, are the map's; only the order in which the persistent blocks take
// them changes.
// A hand-out position c as counters that step to c + 1 without division:
// patch order (gx, gy multiples of 8): a = offset in the 8 x 8 patch, b =
// z-layer counted from the top, e, f = the patch's column and row; grid
// order otherwise: a = x, b = y, e = z-layer counted from the top.  Set
// from c (two divisions) once per claim.
struct HandoutPos {
    int a, b, e, f;
};

__device__ __forceinline__ bool patch_order(int gx, int gy) { return (gx & 7) == 0 && (gy & 7) == 0; }

__device__ __forceinline__ HandoutPos handout_pos(int64_t c, int gx, int gy, int gz) {
    HandoutPos h;
    if (patch_order(gx, gy)) {
        const int64_t per_patch = 64 * (int64_t)gz;
        const int64_t patch = c / per_patch, r = c - patch * per_patch;
        const int pgx = gx >> 3;
        h.a = (int)(r & 63);
        h.b = (int)(r >> 6);
        h.f = (int)(patch / pgx);
        h.e = (int)(patch - (int64_t)h.f * pgx);
    } else {
        const int64_t gxy = (int64_t)gx * gy;
        const int64_t zz = c / gxy, rem = c - zz * gxy;
        h.b = (int)(rem / gx);
        h.a = (int)(rem - (int64_t)h.b * gx);
        h.e = (int)zz;
        h.f = 0;
    }
    return h;
}

// Steps a patch-order position to the next one.
__device__ __forceinline__ void handout_step(HandoutPos &h, int gx, int gz) {
    if (++h.a == 64) {
        h.a = 0;
        if (++h.b == gz) {
            h.b = 0;
            if (++h.e == (gx >> 3)) { h.e = 0; ++h.f; }
        }
    }
}

// The grid block of a hand-out position (see grab_tile for the order).
__device__ __forceinline__ void handout_block(const HandoutPos &h, int gx, int gy, int gz, uint32_t &x,
                                              uint32_t &y, uint32_t &z) {
    if (patch_order(gx, gy)) {
        x = (uint32_t)(8 * h.e + (h.a & 7));
        y = (uint32_t)(8 * h.f + (h.a >> 3));
        z = (uint32_t)(gz - 1 - h.b);
    } else {
        x = (uint32_t)h.a;
        y = (uint32_t)h.b;
        z = (uint32_t)(gz - 1 - h.e);
    }
}

template <int MAP>
__device__ void grab_tile(unsigned long long *ctr, int gx, int gy, int gz, int p, int nb, int claim,
                          AtmForceSmem &S, int slot) {
    const int64_t total = (int64_t)gx * gy * gz;
    long long w = S.walk_w, end = S.walk_end;
    int sub = S.walk_sub;
    HandoutPos h{S.walk_pos[0], S.walk_pos[1], S.walk_pos[2], S.walk_pos[3]};
    int *out = S.tq[slot];
    const bool patches = patch_order(gx, gy);
    for (;;) {
        if (w < end) {
            uint32_t bx, by, bz;
            handout_block(h, gx, gy, gz, bx, by, bz);
            const List3 L = decode3<MAP>(bx, by, bz, p, nb);
            if (sub < L.cnt) {
                int I, J, K;
                block_of(L, sub, I, J, K);
                out[0] = I; out[1] = J; out[2] = K; out[3] = 1;
                S.walk_w = w;
                S.walk_end = end;
                S.walk_sub = sub + 1;
                S.walk_pos[0] = h.a; S.walk_pos[1] = h.b; S.walk_pos[2] = h.e; S.walk_pos[3] = h.f;
                return;
            }
            ++w;
            sub = 0;
            if (patches) {
                handout_step(h, gx, gz);
            } else if (++h.a == gx) {
                h.a = 0;
                if (++h.b == gy) { h.b = 0; ++h.e; }
            }
            continue;
        }
        // the next run of `claim` hand-out positions
        w = (long long)atomicAdd(ctr, 1ull) * claim;
        end = w + claim < total ? w + claim : total;
        sub = 0;
        if (w >= total) {
            out[3] = 0;
            S.walk_w = w;
            S.walk_end = w;
            S.walk_sub = 0;
            return;
        }
        h = handout_pos(w, gx, gy, gz);
    }
}

// The pair constants of the thread's pairs (i = ti, ti + 16; j = tj + 16 q)
// from the fc form of the (I, J) force table (both i-slots in the two lanes).
__device__ __forceinline__ void load_pair_consts(const float4 *__restrict__ tab, int I, int J, int ti,
                                                 int tj, PairPack (&pc)[2]) {
    const float4 *tij = tab + pair_slot(I, J) * kFTabPair + ti;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const float4 *e = tij + 3 * (tj + 16 * q) * 16;
        const float4 C0 = __ldg(e), C1 = __ldg(e + 16), C2 = __ldg(e + 32);
        pc[q].wx = f2(C0.x, C0.y); pc[q].wy = f2(C0.z, C0.w); pc[q].wz = f2(C1.x, C1.y);
        pc[q].sa = f2(C1.z, C1.w); pc[q].ga = f2(1.5f * C2.x, 1.5f * C2.y); pc[q].qa = f2(C2.z, C2.w);
    }
}

// Persistent energy-and-forces kernel: each block walks tiles (32^3 triples)
// of the map's grid with stride gridDim.x.  Per tile: wait for its (i, k) and
// (j, k) tables (TAB: two bulk copies of the force tables of
// k_atm_forcetab issued during the previous tile; else built here from the
// points), the packed triple loop (per thread 2 x 2 pairs (i, j), 32 k)
// forming the energy and the side coefficients, the (j, k) sides reduced by
// a half-warp reduce-scatter and the (i, k) sides by one xor-16 exchange and
// shared atomics; then, while the next tile's tables, points and pair
// constants load, the forces of the tile's 96 atoms, grad_p = 2 sum_q w_pq
// (x_p - x_q), added once per tile and atom by FP64 atomics.  The
// coefficient matrices and point tiles are double-buffered, so a tile costs
// two block barriers.  One FP64 energy partial per block.
template <int MAP, bool TAB>
__global__ void __launch_bounds__(256, 2) k_atm_forces(int64_t n, const float *__restrict__ x,
                                                       float nu, float eps, int nb, int gx, int gy,
                                                       int gz, int p, int claim, const float4 *__restrict__ tab,
                                                       unsigned long long *__restrict__ ctr,
                                                       double *__restrict__ partials,
                                                       double *__restrict__ forces) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    AtmForceSmem &S = *reinterpret_cast<AtmForceSmem *>(smem_raw);
    __shared__ float red[16];
    const int tid = threadIdx.x, ti = tid & 15, tj = tid >> 4, lane = tid & 31;
    const uint32_t bar = umma::smem_u32(&S.bar);
    if (TAB && tid == 0) {
        umma::mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (tid == 0) {
        S.walk_w = 0;
        S.walk_end = 0;
        S.walk_sub = 0;
        S.walk_pos[0] = S.walk_pos[1] = S.walk_pos[2] = S.walk_pos[3] = 0;
        grab_tile<MAP>(ctr, gx, gy, gz, p, nb, claim, S, 0);
        grab_tile<MAP>(ctr, gx, gy, gz, p, nb, claim, S, 1);
    }
    bool bad = false;   // a bounded wait ran out (block-uniform after each tile)
    float hi = 0.f, lo = 0.f;
    PairPack pc[2];
    __syncthreads();
    int I = S.tq[0][0], J = S.tq[0][1], K = S.tq[0][2];
    bool have = S.tq[0][3] != 0;
    // the first tile's tables, points and pair constants
    auto issue_tables = [&](int Ii, int Ji, int Ki) {
        umma::mbar_expect_tx(bar, (uint32_t)(kFTabPair * 16));
        umma::bulk_load(umma::smem_u32(&S.fc[0][0][0]), tab + pair_slot(Ii, Ki) * kFTabPair, kFTabFc * 16, bar);
        umma::bulk_load(umma::smem_u32(&S.fb[0][0][0][0]), tab + pair_slot(Ji, Ki) * kFTabPair + kFTabFc,
                        kFTabFb * 16, bar);
    };
    if (have) {
        if (TAB && tid == 0) issue_tables(I, J, K);
        load_tiles(x, n, I, J, K, S.xs[0]);
        for (int e = tid; e < 2 * R_ * (R_ + 1); e += 256) (&S.wik[0][0][0])[e] = 0.0f;
        if (TAB) load_pair_consts(tab, I, J, ti, tj, pc);
    }
    __syncthreads();   // the first tile's points and the first two zeroed (i, k) matrices
    uint32_t t = 0;
    int b3 = 0;        // t mod 3
#pragma unroll 1
    while (have) {
        const int b = (int)(t & 1);
        if (!TAB) {
            // the points of this tile (loaded during the last tile) are
            // visible and the last tile's loop is done with the tables
            __syncthreads();
            build_force_tables(n, I, J, K, eps, S.xs[b], S);
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int64_t gj = (int64_t)J * R_ + tj + 16 * q;
                const PairTerms a0 = pair_terms(S.xs[b][0][ti], S.xs[b][1][tj + 16 * q],
                                                (int64_t)I * R_ + ti < gj && gj < n, eps);
                const PairTerms a1 = pair_terms(S.xs[b][0][ti + 16], S.xs[b][1][tj + 16 * q],
                                                (int64_t)I * R_ + ti + 16 < gj && gj < n, eps);
                pc[q].wx = f2(a0.wx, a1.wx); pc[q].wy = f2(a0.wy, a1.wy); pc[q].wz = f2(a0.wz, a1.wz);
                pc[q].sa = f2(a0.s, a1.s); pc[q].qa = f2(a0.q, a1.q); pc[q].ga = f2(1.5f * a0.r3, 1.5f * a1.r3);
            }
            __syncthreads();
        } else if (!bad) {
            // bounded wait for the tables; a timeout flags the error and drains (bounded)
            const long long t0 = clock64();
            while (!umma::mbar_try_wait(bar, t & 1)) {
                if (clock64() - t0 > umma::kWaitCycles) {
                    atomicExch(&g_atm_error, 1);
                    umma::mbar_drain(bar, t & 1);
                    bad = true;
                    break;
                }
            }
        }
        float2 acc[2] = {f2(0.f, 0.f), f2(0.f, 0.f)};
        float2 wa[2] = {f2(0.f, 0.f), f2(0.f, 0.f)};
#pragma unroll 1
        for (int k0 = 0; k0 < R_; k0 += 8) {
            float vb[16], vc[16];   // vb[8q + kk]: side (j_q, k); vc[8p + kk]: side (i_p, k)
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) {
                const int k = k0 + kk;
                const float4 C0 = S.fc[k][0][ti], C1 = S.fc[k][1][ti], C2 = S.fc[k][2][ti];
                float2 ecs = f2(0.f, 0.f);
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const float4 B0 = S.fb[k][q][0][tj], B1 = S.fb[k][q][1][tj], B2 = S.fb[k][q][2][tj];
                    vb[8 * q + kk] = triple_grad2(pc[q], C0, C1, C2, B0, B1, B2, acc[q], wa[q], ecs);
                }
                vc[kk] = ecs.x;
                vc[8 + kk] = ecs.y;
            }
            // (j, k) sides: sum over the 16 i of this half-warp; lane ti ends
            // with j = tj + 16 (ti >> 3), k = k0 + (ti & 7)
            const float sb = reduce_scatter16(vb, lane);
            S.wjk[b][k0 + (ti & 7)][tj + 16 * (ti >> 3)] = sb;
            // (i, k) sides: sum over the two tj of this warp (lanes l, l ^ 16),
            // then over the warps by shared atomics
            const bool up = (lane & 16) != 0;
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                const float send = up ? vc[m] : vc[m + 8];
                const float keep = up ? vc[m + 8] : vc[m];
                vc[m] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
            }
            const int ip = ti + 16 * (up ? 1 : 0);
#pragma unroll
            for (int m = 0; m < 8; ++m) atomicAdd(&S.wik[b3][k0 + m][ip], vc[m]);
        }
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            S.wij[b][ti][tj + 16 * q] = wa[q].x;
            S.wij[b][ti + 16][tj + 16 * q] = wa[q].y;
        }
        add_ff(hi, lo, acc[0].x + acc[1].x, 0.f);
        add_ff(hi, lo, acc[0].y + acc[1].y, 0.f);
        // the tile's sums are complete and its tables no longer read
        bad = __syncthreads_or(bad) != 0;
        if (bad) break;
        // the next tile (taken during the previous tile); a loader thread
        // takes the one after it into the slot this tile's entry held
        const int *nx = S.tq[(t + 1) & 1];
        const int In = nx[0], Jn = nx[1], Kn = nx[2];
        const bool hn = nx[3] != 0;
        if (hn && tid == 6 * R_) grab_tile<MAP>(ctr, gx, gy, gz, p, nb, claim, S, (int)(t & 1));
        if (hn) {
            // the next tile's tables (into the free table buffer), points
            // (into the other buffer) and pair constants
            if (TAB && tid == 0) issue_tables(In, Jn, Kn);
            if (TAB) load_pair_consts(tab, In, Jn, ti, tj, pc);
            if (tid >= 6 * R_) {
                const int e0 = tid - 6 * R_;
                for (int e = e0; e < 3 * R_; e += 256 - 6 * R_) {
                    const int which = e / R_, o = e % R_;
                    const int blk = which == 0 ? In : which == 1 ? Jn : Kn;
                    const int64_t g = (int64_t)blk * R_ + o;
                    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (g < n) v = make_float4(__ldg(x + 3 * g), __ldg(x + 3 * g + 1), __ldg(x + 3 * g + 2), 0.f);
                    S.xs[b ^ 1][which][o] = v;
                }
            }
        }
        // the (i, k) matrix of tile t + 2 (last read by the assembly of tile
        // t - 1, which every warp finished before this tile's barrier)
        if (tid >= 6 * R_) {
            const int z3 = b3 == 0 ? 2 : b3 - 1;
            for (int e = tid - 6 * R_; e < R_ * (R_ + 1); e += 256 - 6 * R_) (&S.wik[z3][0][0])[e] = 0.0f;
        }
        // Pair coefficients -> forces of the tile's 96 atoms: atom p (thread
        // pair 2p, 2p + 1, one per partner block) sums w_pq (x_p - x_q).
        if (tid < 6 * R_) {
            const int atom = tid >> 1, half = tid & 1;
            const int which = atom / R_, o = atom % R_;
            const float *wrow;
            int stride;
            const float4 *xq;
            if (which == 0) {
                if (half == 0) { wrow = &S.wij[b][o][0]; stride = 1; xq = S.xs[b][1]; }
                else { wrow = &S.wik[b3][0][o]; stride = R_ + 1; xq = S.xs[b][2]; }
            } else if (which == 1) {
                if (half == 0) { wrow = &S.wij[b][0][o]; stride = R_ + 1; xq = S.xs[b][0]; }
                else { wrow = &S.wjk[b][0][o]; stride = R_ + 1; xq = S.xs[b][2]; }
            } else {
                if (half == 0) { wrow = &S.wjk[b][o][0]; stride = 1; xq = S.xs[b][1]; }
                else { wrow = &S.wik[b3][o][0]; stride = 1; xq = S.xs[b][0]; }
            }
            const float4 xp = S.xs[b][which][o];
            float gx_ = 0.f, gy_ = 0.f, gz_ = 0.f;
#pragma unroll 8
            for (int q = 0; q < R_; ++q) {
                const float w = wrow[q * stride];
                const float4 v = xq[q];
                gx_ = fmaf(w, xp.x - v.x, gx_);
                gy_ = fmaf(w, xp.y - v.y, gy_);
                gz_ = fmaf(w, xp.z - v.z, gz_);
            }
            gx_ += __shfl_xor_sync(0xffffffffu, gx_, 1);
            gy_ += __shfl_xor_sync(0xffffffffu, gy_, 1);
            gz_ += __shfl_xor_sync(0xffffffffu, gz_, 1);
            const int blk = which == 0 ? I : which == 1 ? J : K;
            const int64_t g = (int64_t)blk * R_ + o;
            if (half == 0 && g < n) {
                const float f = -2.0f * nu;   // F = -dE/dx, the tile's part in FP32, summed in FP64
                atomicAdd(forces + 3 * g, (double)(f * gx_));
                atomicAdd(forces + 3 * g + 1, (double)(f * gy_));
                atomicAdd(forces + 3 * g + 2, (double)(f * gz_));
            }
        }
        I = In; J = Jn; K = Kn;
        have = hn;
        ++t;
        b3 = b3 == 2 ? 0 : b3 + 1;
    }
    if (partials) {
        const bool any_bad = __syncthreads_or(bad) != 0;
        const double s = block_sum_ff<256>(hi, lo, red);
        if (tid == 0)
            partials[blockIdx.x] = any_bad ? __longlong_as_double(0x7ff8000000000000LL) : (double)nu * s;
    }
}

constexpr int kEnergySmem = (int)sizeof(AtmEnergySmem);
constexpr int kEnergyTabSmem = (int)sizeof(AtmEnergyTabSmem);

// Both kernels' shared memory exceeds the 48 KB default of a launch; opt in
// once per device for every instantiation.
static int smem_optin() {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e);
    static std::mutex mu;
    static bool done[64] = {};
    if (dev < 0 || dev >= 64) return SIMPLEX_EUNSUPPORTED;
    std::lock_guard<std::mutex> lk(mu);
    if (!done[dev]) {
        const int fb = (int)sizeof(AtmForceSmem);
        const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
        if ((e = cudaFuncSetAttribute(k_atm_forces<MAP_LAMBDA, false>, a, fb)) != cudaSuccess ||
            (e = cudaFuncSetAttribute(k_atm_forces<MAP_BBOX, false>, a, fb)) != cudaSuccess ||
            (e = cudaFuncSetAttribute(k_atm_forces<MAP_LINEAR, false>, a, fb)) != cudaSuccess ||
            (e = cudaFuncSetAttribute(k_atm_forces<MAP_LAMBDA, true>, a, fb)) != cudaSuccess ||
            (e = cudaFuncSetAttribute(k_atm_forces<MAP_BBOX, true>, a, fb)) != cudaSuccess ||
            (e = cudaFuncSetAttribute(k_atm_forces<MAP_LINEAR, true>, a, fb)) != cudaSuccess ||
            (e = cudaFuncSetAttribute(k_atm_energy<MAP_LAMBDA>, a, kEnergySmem)) != cudaSuccess ||
            (e = cudaFuncSetAttribute(k_atm_energy<MAP_BBOX>, a, kEnergySmem)) != cudaSuccess ||
            (e = cudaFuncSetAttribute(k_atm_energy<MAP_LINEAR>, a, kEnergySmem)) != cudaSuccess ||
            (e = cudaFuncSetAttribute(k_atm_energy_tab<MAP_LAMBDA>, a, kEnergyTabSmem)) != cudaSuccess ||
            (e = cudaFuncSetAttribute(k_atm_energy_tab<MAP_BBOX>, a, kEnergyTabSmem)) != cudaSuccess ||
            (e = cudaFuncSetAttribute(k_atm_energy_tab<MAP_LINEAR>, a, kEnergyTabSmem)) != cudaSuccess)
            return cuda_status(e);
        done[dev] = true;
    }
    return SIMPLEX_OK;
}

// Blocks of a persistent kernel: as many as are resident on the device at
// once (occupancy of `kern` with 256 threads and `smem` bytes), at most
// `work` (the grid blocks to walk).
template <typename Kern>
static int persistent_blocks(Kern kern, int smem, int64_t work, int &ctas) {
    int dev = 0, sms = 0, occ = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 256, smem);
    if (e != cudaSuccess) return cuda_status(e);
    if (occ < 1) return SIMPLEX_EUNSUPPORTED;
    const int64_t c = (int64_t)occ * sms;
    ctas = (int)(c < work ? c : work);
    return SIMPLEX_OK;
}

static int atm_check(int64_t n, int64_t d, const float *x, int map, void *ws, int64_t ws_bytes,
                     Grid &g, int64_t &nb, int64_t extra = 0) {
    if (n < 1 || d != 3 || !x || map < MAP_LAMBDA || map > MAP_LINEAR) return d != 3 && d > 0 ? SIMPLEX_EUNSUPPORTED : SIMPLEX_EINVAL;
    if (!aligned(x, 4)) return SIMPLEX_EALIGN;
    if (n > (1 << 22)) return SIMPLEX_EOVERFLOW;
    nb = (n + R_ - 1) / R_;
    g = grid3(nb, map);
    if (!grid_fits(g)) return SIMPLEX_EOVERFLOW;
    const int64_t need = extra + 8 * (g.gx * g.gy * g.gz + kReduceSlots);
    if (!ws || ws_bytes < need || !aligned(ws, 256)) return SIMPLEX_EWORKSPACE;
    return SIMPLEX_OK;
}

// Bytes of the pair tables of simplex_atm_energy (0 where they would exceed
// kTabMaxBytes and the per-tile tables are used instead).
static int64_t energy_table_bytes(int64_t nb) {
    const int64_t t = atm_table_bytes(nb);
    return t <= kTabMaxBytes ? t : 0;
}

// Bytes of the force tables of simplex_atm_forces (0 where they would exceed
// kFTabMaxBytes and the tables are built per tile instead).
static int64_t force_table_bytes(int64_t nb) {
    const int64_t t = nb * (nb + 1) / 2 * kFTabPair * 16;
    return t <= kFTabMaxBytes ? t : 0;
}

// The forces' workspace: [force tables][the tile counter, 16 bytes][FP64
// partials (one per block of the persistent grid; room for one per grid
// block)][reduction slots].
constexpr int64_t kCounterBytes = 16;

int64_t atm_forces_workspace_bytes(int64_t n, int map) {
    const int64_t nb = (n + R_ - 1) / R_;
    const Grid g = grid3(nb, map);
    return force_table_bytes(nb) + kCounterBytes + 8 * (g.gx * g.gy * g.gz + kReduceSlots);
}

int64_t atm_energy_workspace_bytes(int64_t n, int map) {
    const int64_t nb = (n + R_ - 1) / R_;
    const Grid g = grid3(nb, map);
    return energy_table_bytes(nb) + 8 * (g.gx * g.gy * g.gz + kReduceSlots);
}

int atm_device_errors(cudaStream_t s) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e);
    int h = 0;
    if ((e = cudaMemcpyFromSymbol(&h, g_atm_error, sizeof(int))) != cudaSuccess) return cuda_status(e);
    if (h) {
        const int zero = 0;
        if ((e = cudaMemcpyToSymbol(g_atm_error, &zero, sizeof(int))) != cudaSuccess) return cuda_status(e);
        return SIMPLEX_ETIMEOUT;
    }
    return SIMPLEX_OK;
}

}  // namespace sx

using namespace sx;

extern "C" int simplex_atm_energy(int64_t n, int64_t d, const float *x, float nu, float eps,
                                  double *energy, int map, void *workspace, int64_t ws_bytes,
                                  void *stream) {
    if (!energy) return SIMPLEX_EINVAL;
    if (n < 1 || n > (1 << 22)) return n < 1 ? SIMPLEX_EINVAL : SIMPLEX_EOVERFLOW;
    const int64_t tab_bytes = energy_table_bytes((n + R_ - 1) / R_);
    Grid g;
    int64_t nb;
    int st = atm_check(n, d, x, map, workspace, ws_bytes, g, nb, tab_bytes);
    if (st) return st;
    if (!aligned(energy, 8)) return SIMPLEX_EALIGN;
    cudaStream_t s = (cudaStream_t)stream;
    // workspace: [pair tables][one FP64 partial per grid block][reduction slots]
    float4 *tab = (float4 *)workspace;
    double *partials = (double *)((char *)workspace + tab_bytes);
    const int64_t blocks = g.gx * g.gy * g.gz;
    double *tmp = partials + blocks;
    if ((st = smem_optin())) return st;
    if (tab_bytes) {
        const Grid g2 = grid2(nb, map);
        if (!grid_fits(g2)) return SIMPLEX_EOVERFLOW;
        if (map == MAP_LAMBDA) k_atm_pairtab<MAP_LAMBDA><<<dim_of(g2), 256, 0, s>>>(n, x, eps, (int)nb, tab);
        else if (map == MAP_BBOX) k_atm_pairtab<MAP_BBOX><<<dim_of(g2), 256, 0, s>>>(n, x, eps, (int)nb, tab);
        else k_atm_pairtab<MAP_LINEAR><<<dim_of(g2), 256, 0, s>>>(n, x, eps, (int)nb, tab);
        note_launches(1);
        if ((st = launch_status())) return st;
    }
    prof_begin(s);
    if (tab_bytes) {
        if (map == MAP_LAMBDA) k_atm_energy_tab<MAP_LAMBDA><<<dim_of(g), 128, kEnergyTabSmem, s>>>(tab, nu, (int)nb, g.p, partials);
        else if (map == MAP_BBOX) k_atm_energy_tab<MAP_BBOX><<<dim_of(g), 128, kEnergyTabSmem, s>>>(tab, nu, (int)nb, g.p, partials);
        else k_atm_energy_tab<MAP_LINEAR><<<dim_of(g), 128, kEnergyTabSmem, s>>>(tab, nu, (int)nb, g.p, partials);
    } else {
        if (map == MAP_LAMBDA) k_atm_energy<MAP_LAMBDA><<<dim_of(g), 256, kEnergySmem, s>>>(n, x, nu, eps, (int)nb, g.p, partials);
        else if (map == MAP_BBOX) k_atm_energy<MAP_BBOX><<<dim_of(g), 256, kEnergySmem, s>>>(n, x, nu, eps, (int)nb, g.p, partials);
        else k_atm_energy<MAP_LINEAR><<<dim_of(g), 256, kEnergySmem, s>>>(n, x, nu, eps, (int)nb, g.p, partials);
    }
    prof_end(s);
    note_launches(1);
    if ((st = launch_status())) return st;
    return reduce_partials(partials, blocks, tmp, energy, s);
}

extern "C" int simplex_atm_forces(int64_t n, int64_t d, const float *x, float nu, float eps,
                                  double *energy, double *forces, int map, void *workspace,
                                  int64_t ws_bytes, void *stream) {
    if (!forces) return SIMPLEX_EINVAL;
    Grid g;
    int64_t nb = (n + R_ - 1) / R_;
    const int64_t ftab = n >= 1 ? force_table_bytes(nb) : 0;
    int st = atm_check(n, d, x, map, workspace, ws_bytes, g, nb, ftab + kCounterBytes);
    if (st) return st;
    if (!aligned(forces, 8) || (energy && !aligned(energy, 8))) return SIMPLEX_EALIGN;
    cudaStream_t s = (cudaStream_t)stream;
    const float4 *tab = (const float4 *)workspace;
    unsigned long long *ctr = (unsigned long long *)((char *)workspace + ftab);
    double *partials = energy ? (double *)((char *)workspace + ftab + kCounterBytes) : nullptr;
    const int64_t blocks = g.gx * g.gy * g.gz;
    if ((st = cuda_status(cudaMemsetAsync(forces, 0, sizeof(double) * 3 * (size_t)n, s)))) return st;
    if ((st = cuda_status(cudaMemsetAsync(ctr, 0, sizeof(unsigned long long), s)))) return st;
    const int smem = (int)sizeof(AtmForceSmem);
    if ((st = smem_optin())) return st;
    if (ftab) {
        const Grid g2 = grid2(nb, map);
        if (!grid_fits(g2)) return SIMPLEX_EOVERFLOW;
        float4 *wt = (float4 *)workspace;
        if (map == MAP_LAMBDA) k_atm_forcetab<MAP_LAMBDA><<<dim_of(g2), 256, 0, s>>>(n, x, eps, (int)nb, wt);
        else if (map == MAP_BBOX) k_atm_forcetab<MAP_BBOX><<<dim_of(g2), 256, 0, s>>>(n, x, eps, (int)nb, wt);
        else k_atm_forcetab<MAP_LINEAR><<<dim_of(g2), 256, 0, s>>>(n, x, eps, (int)nb, wt);
        note_launches(1);
        if ((st = launch_status())) return st;
    }
    // persistent: as many blocks as are resident at once, each walking the grid
    int ctas = 0;
    if (ftab) {
        if (map == MAP_LAMBDA) st = persistent_blocks(k_atm_forces<MAP_LAMBDA, true>, smem, blocks, ctas);
        else if (map == MAP_BBOX) st = persistent_blocks(k_atm_forces<MAP_BBOX, true>, smem, blocks, ctas);
        else st = persistent_blocks(k_atm_forces<MAP_LINEAR, true>, smem, blocks, ctas);
    } else {
        if (map == MAP_LAMBDA) st = persistent_blocks(k_atm_forces<MAP_LAMBDA, false>, smem, blocks, ctas);
        else if (map == MAP_BBOX) st = persistent_blocks(k_atm_forces<MAP_BBOX, false>, smem, blocks, ctas);
        else st = persistent_blocks(k_atm_forces<MAP_LINEAR, false>, smem, blocks, ctas);
    }
    if (st) return st;
    const int gx = (int)g.gx, gy = (int)g.gy, gz = (int)g.gz;
    // grid blocks per claim: up to 8, at least 64 claims per persistent block
    int64_t claim64 = blocks / ((int64_t)ctas * 64);
    const int claim = (int)(claim64 < 1 ? 1 : (claim64 > 8 ? 8 : claim64));
    prof_begin(s);
    if (ftab) {
        if (map == MAP_LAMBDA) k_atm_forces<MAP_LAMBDA, true><<<ctas, 256, smem, s>>>(n, x, nu, eps, (int)nb, gx, gy, gz, g.p, claim, tab, ctr, partials, forces);
        else if (map == MAP_BBOX) k_atm_forces<MAP_BBOX, true><<<ctas, 256, smem, s>>>(n, x, nu, eps, (int)nb, gx, gy, gz, g.p, claim, tab, ctr, partials, forces);
        else k_atm_forces<MAP_LINEAR, true><<<ctas, 256, smem, s>>>(n, x, nu, eps, (int)nb, gx, gy, gz, g.p, claim, tab, ctr, partials, forces);
    } else {
        if (map == MAP_LAMBDA) k_atm_forces<MAP_LAMBDA, false><<<ctas, 256, smem, s>>>(n, x, nu, eps, (int)nb, gx, gy, gz, g.p, claim, nullptr, ctr, partials, forces);
        else if (map == MAP_BBOX) k_atm_forces<MAP_BBOX, false><<<ctas, 256, smem, s>>>(n, x, nu, eps, (int)nb, gx, gy, gz, g.p, claim, nullptr, ctr, partials, forces);
        else k_atm_forces<MAP_LINEAR, false><<<ctas, 256, smem, s>>>(n, x, nu, eps, (int)nb, gx, gy, gz, g.p, claim, nullptr, ctr, partials, forces);
    }
    prof_end(s);
    note_launches(1);
    if ((st = launch_status())) return st;
    if (energy) return reduce_partials(partials, ctas, partials + blocks, energy, s);
    return SIMPLEX_OK;
}

// ---------------------------------------------------------------- no-alloc entry

namespace sx {

// Scratch of simplex_atm_energy_noalloc: one FP64 partial per grid block plus
// the reduction's slots, in a fixed array of this library's device image.
// Every GPU that loads the library holds these 4 MiB until the process exits.
constexpr int64_t kNoAllocScratchDoubles = int64_t(1) << 19;
static __device__ __align__(256) double g_atm_noalloc_scratch[kNoAllocScratchDoubles];

// Device address of that array on the current device.  In host code the
// array's name is a host-side stand-in, not a device address, so the address
// is looked up with cudaGetSymbolAddress once per device (with that device
// current, on the first call made there) and cached.
static int noalloc_scratch(double **out) {
    constexpr int kMaxDevices = 64;
    static std::mutex mu;
    static double *addr[kMaxDevices] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e);
    if (dev < 0 || dev >= kMaxDevices) return SIMPLEX_EUNSUPPORTED;
    std::lock_guard<std::mutex> lk(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_atm_noalloc_scratch);
        if (e != cudaSuccess) return cuda_status(e);
        addr[dev] = static_cast<double *>(p);
    }
    *out = addr[dev];
    return SIMPLEX_OK;
}

}  // namespace sx

extern "C" int simplex_atm_energy_noalloc(int64_t n, int64_t d, const float *x, float nu,
                                          float eps, double *energy, int map, void *stream) {
    if (!energy) return SIMPLEX_EINVAL;
    if (n < 1 || d != 3 || !x || map < MAP_LAMBDA || map > MAP_LINEAR)
        return d != 3 && d > 0 ? SIMPLEX_EUNSUPPORTED : SIMPLEX_EINVAL;
    if (!aligned(x, 4) || !aligned(energy, 8)) return SIMPLEX_EALIGN;
    if (n > (1 << 22)) return SIMPLEX_EOVERFLOW;
    const int64_t nb = (n + R_ - 1) / R_;
    const Grid g = grid3(nb, map);
    if (!grid_fits(g)) return SIMPLEX_EOVERFLOW;
    const int64_t blocks = g.gx * g.gy * g.gz;
    if (blocks + kReduceSlots > kNoAllocScratchDoubles) return SIMPLEX_ESCRATCH;
    double *scratch = nullptr;
    int st = noalloc_scratch(&scratch);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    double *partials = scratch, *tmp = scratch + blocks;
    if ((st = smem_optin())) return st;
    prof_begin(s);
    if (map == MAP_LAMBDA) k_atm_energy<MAP_LAMBDA><<<dim_of(g), 256, kEnergySmem, s>>>(n, x, nu, eps, (int)nb, g.p, partials);
    else if (map == MAP_BBOX) k_atm_energy<MAP_BBOX><<<dim_of(g), 256, kEnergySmem, s>>>(n, x, nu, eps, (int)nb, g.p, partials);
    else k_atm_energy<MAP_LINEAR><<<dim_of(g), 256, kEnergySmem, s>>>(n, x, nu, eps, (int)nb, g.p, partials);
    prof_end(s);
    note_launches(1);
    if ((st = launch_status())) return st;
    return reduce_partials(partials, blocks, tmp, energy, s);
}
