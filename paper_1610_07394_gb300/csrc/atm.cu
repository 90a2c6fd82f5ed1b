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

namespace sx {

constexpr int R_ = kAtmRho;  // 32

struct AtmTables {
    float4 xs[3][R_];        // tiles I, J, K: (x, y, z, 0)
    float4 tb[R_][2][16];    // [k][q][t]: (u_jk, r_jk^3 or r_jk) of pair (j = t + 16q, k)
    float4 tc[R_][2][16];    // [k][p][t]: (u_ik, r_ik^3 or r_ik) of pair (i = t + 16p, k)
};

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

// Pair terms.  CUBE selects r^3 (energy) or r (forces) in the w slot.
__device__ __forceinline__ float4 edge(float4 from, float4 to) {
    return make_float4(to.x - from.x, to.y - from.y, to.z - from.z, 0.0f);
}

template <bool CUBE>
__device__ __forceinline__ float4 pair_term(float4 from, float4 to, bool valid, float eps) {
    const float4 e = edge(from, to);
    if (!valid) return make_float4(0.f, 0.f, 0.f, 0.f);
    const float s = fmaf(e.x, e.x, fmaf(e.y, e.y, fmaf(e.z, e.z, eps)));
    const float q = sqrtf(s);
    const float r = 1.0f / q;
    return make_float4(e.x * r, e.y * r, e.z * r, CUBE ? 1.0f / (s * q) : r);
}

template <bool CUBE>
__device__ __forceinline__ void build_tables(int64_t n, int I, int J, int K, float eps,
                                             AtmTables &T) {
    for (int e = threadIdx.x; e < R_ * R_; e += 256) {
        const int k = e >> 5, o = e & 31, half = o >> 4, t = o & 15;
        const int64_t gi = (int64_t)I * R_ + o, gj = (int64_t)J * R_ + o, gk = (int64_t)K * R_ + k;
        T.tb[k][half][t] = pair_term<CUBE>(T.xs[1][o], T.xs[2][k], gj < gk && gk < n, eps);
        T.tc[k][half][t] = pair_term<CUBE>(T.xs[0][o], T.xs[2][k], gi < gk && gk < n, eps);
    }
}

struct PairConst {
    float4 u;    // u_ij, w = r_ij^3 (energy) or r_ij (forces); 0 outside i < j < n
    float3 f;    // -3 u_ij
};

template <bool CUBE>
__device__ __forceinline__ PairConst pair_const(int64_t n, int I, int J, int i, int j, float eps,
                                                const AtmTables &T) {
    PairConst c;
    const int64_t gi = (int64_t)I * R_ + i, gj = (int64_t)J * R_ + j;
    c.u = pair_term<CUBE>(T.xs[0][i], T.xs[1][j], gi < gj && gj < n, eps);
    c.f = make_float3(-3.0f * c.u.x, -3.0f * c.u.y, -3.0f * c.u.z);
    return c;
}

__device__ __forceinline__ float dot3(float4 a, float4 b) {
    return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z));
}

__device__ __forceinline__ float dot3(float3 a, float4 b) {
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
        const float4 c = pair_term<true>(S.xs[0][o], S.xs[2][k], gi < gk && gk < n, eps);
        put_pair(S.ec[k][0][t], S.ec[k][1][t], half, c);
        const float4 b = pair_term<true>(S.xs[1][o], S.xs[2][k], gj < gk && gk < n, eps);
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
    const List3 L = decode3<MAP>(blockIdx.x, blockIdx.y, blockIdx.z, p, nb);
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
            const float4 u0 = pair_term<true>(S.xs[0][ti], S.xs[1][tj + 16 * q],
                                              (int64_t)I * R_ + ti < gj && gj < n, eps);
            const float4 u1 = pair_term<true>(S.xs[0][ti + 16], S.xs[1][tj + 16 * q],
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

// ---------------------------------------------------------------- forces

struct AtmForceSmem {
    AtmTables T;
    float tb3[R_][2][16];    // r_jk^3 of the pairs of T.tb
    float tc3[R_][2][16];    // r_ik^3 of the pairs of T.tc
    float wjk[R_][R_ + 1];   // [k][j]: sum over i of de/db
    float wik[R_][R_ + 1];   // [k][i]: sum over j of de/dc
    float wij[R_][R_ + 1];   // [i][j]: sum over k of de/da
};

// One triple: energy into acc and the derivatives of e (without nu) with
// respect to the squared sides a = |e_ij|^2, b = |e_jk|^2, c = |e_ik|^2.
// From e = R^3 (1 + 3 D R^2) with D = d_i d_j d_k (vertex dot products,
// 2 d_i = a + c - b, 2 d_j = a + b - c, 2 d_k = b + c - a) and R^2 = 1/P:
//   de/da = R^3 (3 R^2 dD/da - 1.5 (1 + 5 D R^2) r_a^2),
//   dD/da = (d_j d_k + d_i d_k - d_i d_j)/2, and likewise for b, c.
// In cosines (Cp = cos_i cos_j cos_k = D R^2, d_j d_k R^2 = cos_j cos_k r_a r_c,
// d_i d_k R^2 = cos_i cos_k r_a r_b, d_i d_j R^2 = cos_i cos_j r_b r_c):
//   de/da = 1.5 R^3 (X + Y - Z - H r_a^2),  de/db = 1.5 R^3 (Y + Z - X - H r_b^2),
//   de/dc = 1.5 R^3 (X + Z - Y - H r_c^2),
// with X = cos_j cos_k r_a r_c, Y = cos_i cos_k r_a r_b, Z = cos_i cos_j r_b r_c,
// H = 1 + 5 Cp.  B = (u_jk, r_jk), C = (u_ik, r_ik); R^3 is the product of the
// three pairs' r^3 = 1/(s sqrt(s)), as in the energy kernel.
__device__ __forceinline__ void triple_grad(float4 B, float4 C, float rb3, float rc3,
                                            const PairConst &c, float ra3, float &acc, float &ea,
                                            float &eb, float &ec) {
    const float ra = c.u.w, rb = B.w, rc = C.w;
    const float ci = dot3(c.u, C);
    const float cj = -dot3(c.u, B);
    const float ck = dot3(C, B);
    const float cjk = cj * ck, cik = ci * ck, cij = ci * cj;
    const float Cp = ci * cjk;
    const float rab = ra * rb;
    const float X = cjk * (ra * rc), Y = cik * rab, Z = cij * (rb * rc);
    const float R3 = (ra3 * rc3) * rb3;
    acc = fmaf(R3, fmaf(3.0f, Cp, 1.0f), acc);
    const float H = fmaf(5.0f, Cp, 1.0f);
    const float h = 1.5f * R3;
    const float S = X + Y + Z;
    ea = h * fmaf(-H, ra * ra, fmaf(-2.0f, Z, S));
    eb = h * fmaf(-H, rb * rb, fmaf(-2.0f, X, S));
    ec = h * fmaf(-H, rc * rc, fmaf(-2.0f, Y, S));
}

// r^3 of every table pair, 1/(s sqrt(s)) from the stored unit vector's s.
__device__ __forceinline__ float cube_r(float4 from, float4 to, bool valid, float eps) {
    if (!valid) return 0.0f;
    const float4 e = edge(from, to);
    const float s = fmaf(e.x, e.x, fmaf(e.y, e.y, fmaf(e.z, e.z, eps)));
    return 1.0f / (s * sqrtf(s));
}

template <int MAP>
__global__ void __launch_bounds__(256) k_atm_forces(int64_t n, const float *__restrict__ x,
                                                    float nu, float eps, int nb, int p,
                                                    double *__restrict__ partials,
                                                    double *__restrict__ forces) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    AtmForceSmem &S = *reinterpret_cast<AtmForceSmem *>(smem_raw);
    __shared__ float red[16];
    AtmTables &T = S.T;
    const List3 L = decode3<MAP>(blockIdx.x, blockIdx.y, blockIdx.z, p, nb);
    const int tid = threadIdx.x, ti = tid & 15, tj = tid >> 4, lane = tid & 31;
    float hi = 0.f, lo = 0.f;
#pragma unroll 1
    for (int t = 0; t < L.cnt; ++t) {
        int I, J, K;
        block_of(L, t, I, J, K);
        if (t) __syncthreads();
        load_tiles(x, n, I, J, K, T.xs);
        for (int e = tid; e < R_ * (R_ + 1); e += 256) (&S.wik[0][0])[e] = 0.0f;
        __syncthreads();
        build_tables<false>(n, I, J, K, eps, T);
        for (int e = tid; e < R_ * R_; e += 256) {
            const int k = e >> 5, o = e & 31, half = o >> 4, tt = o & 15;
            const int64_t gi = (int64_t)I * R_ + o, gj = (int64_t)J * R_ + o, gk = (int64_t)K * R_ + k;
            S.tb3[k][half][tt] = cube_r(T.xs[1][o], T.xs[2][k], gj < gk && gk < n, eps);
            S.tc3[k][half][tt] = cube_r(T.xs[0][o], T.xs[2][k], gi < gk && gk < n, eps);
        }
        PairConst pc[2][2];
        float ra3[2][2];
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                pc[a][b] = pair_const<false>(n, I, J, ti + 16 * a, tj + 16 * b, eps, T);
                const int64_t gi = (int64_t)I * R_ + ti + 16 * a, gj = (int64_t)J * R_ + tj + 16 * b;
                ra3[a][b] = cube_r(T.xs[0][ti + 16 * a], T.xs[1][tj + 16 * b], gi < gj && gj < n, eps);
            }
        __syncthreads();
        float acc = 0.0f;
        float wa[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
        for (int k = 0; k < R_; ++k) {
            const float4 B0 = T.tb[k][0][tj], B1 = T.tb[k][1][tj];
            const float4 C0 = T.tc[k][0][ti], C1 = T.tc[k][1][ti];
            const float b30 = S.tb3[k][0][tj], b31 = S.tb3[k][1][tj];
            const float c30 = S.tc3[k][0][ti], c31 = S.tc3[k][1][ti];
            float ea, eb[2][2], ec[2][2];
            triple_grad(B0, C0, b30, c30, pc[0][0], ra3[0][0], acc, ea, eb[0][0], ec[0][0]); wa[0][0] += ea;
            triple_grad(B1, C0, b31, c30, pc[0][1], ra3[0][1], acc, ea, eb[0][1], ec[0][1]); wa[0][1] += ea;
            triple_grad(B0, C1, b30, c31, pc[1][0], ra3[1][0], acc, ea, eb[1][0], ec[1][0]); wa[1][0] += ea;
            triple_grad(B1, C1, b31, c31, pc[1][1], ra3[1][1], acc, ea, eb[1][1], ec[1][1]); wa[1][1] += ea;
            // side (j, k): sum over the 16 i of this half-warp (lanes with the same tj)
            float sb0 = eb[0][0] + eb[1][0], sb1 = eb[0][1] + eb[1][1];
#pragma unroll
            for (int o = 1; o < 16; o <<= 1) {
                sb0 += __shfl_xor_sync(0xffffffffu, sb0, o);
                sb1 += __shfl_xor_sync(0xffffffffu, sb1, o);
            }
            if (ti == 0) { S.wjk[k][tj] = sb0; S.wjk[k][tj + 16] = sb1; }
            // side (i, k): sum over the two tj of this warp, then across warps
            float sc0 = ec[0][0] + ec[0][1], sc1 = ec[1][0] + ec[1][1];
            sc0 += __shfl_xor_sync(0xffffffffu, sc0, 16);
            sc1 += __shfl_xor_sync(0xffffffffu, sc1, 16);
            if (lane < 16) { atomicAdd(&S.wik[k][ti], sc0); atomicAdd(&S.wik[k][ti + 16], sc1); }
        }
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b) S.wij[ti + 16 * a][tj + 16 * b] = wa[a][b];
        add_ff(hi, lo, acc, 0.f);
        __syncthreads();
        // Pair coefficients -> gradient: grad_p += 2 sum_q w_pq (x_p - x_q).
        if (tid < 6 * R_) {
            const int atom = tid >> 1, half = tid & 1;
            float gx = 0.f, gy = 0.f, gz = 0.f;
            const int which = atom / R_, o = atom % R_;
            const float4 xp = T.xs[which][o];
            for (int q = 0; q < R_; ++q) {
                float w;
                float4 xq;
                if (which == 0) {
                    if (half == 0) { w = S.wij[o][q]; xq = T.xs[1][q]; }
                    else { w = S.wik[q][o]; xq = T.xs[2][q]; }
                } else if (which == 1) {
                    if (half == 0) { w = S.wij[q][o]; xq = T.xs[0][q]; }
                    else { w = S.wjk[q][o]; xq = T.xs[2][q]; }
                } else {
                    if (half == 0) { w = S.wjk[o][q]; xq = T.xs[1][q]; }
                    else { w = S.wik[o][q]; xq = T.xs[0][q]; }
                }
                gx = fmaf(w, xp.x - xq.x, gx);
                gy = fmaf(w, xp.y - xq.y, gy);
                gz = fmaf(w, xp.z - xq.z, gz);
            }
            gx += __shfl_xor_sync(0xffffffffu, gx, 1);
            gy += __shfl_xor_sync(0xffffffffu, gy, 1);
            gz += __shfl_xor_sync(0xffffffffu, gz, 1);
            const int blk = which == 0 ? I : which == 1 ? J : K;
            const int64_t g = (int64_t)blk * R_ + o;
            if (half == 0 && g < n) {
                const double f = -2.0 * (double)nu;
                atomicAdd(forces + 3 * g, f * gx);
                atomicAdd(forces + 3 * g + 1, f * gy);
                atomicAdd(forces + 3 * g + 2, f * gz);
            }
        }
    }
    if (partials) {
        const double s = block_sum_ff<256>(hi, lo, red);
        if (tid == 0) {
            const int64_t bid = blockIdx.x + (int64_t)gridDim.x * (blockIdx.y + (int64_t)gridDim.y * blockIdx.z);
            partials[bid] = (double)nu * s;
        }
    }
}

constexpr int kEnergySmem = (int)sizeof(AtmEnergySmem);

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
        if ((e = cudaFuncSetAttribute(k_atm_forces<MAP_LAMBDA>, a, fb)) != cudaSuccess ||
            (e = cudaFuncSetAttribute(k_atm_forces<MAP_BBOX>, a, fb)) != cudaSuccess ||
            (e = cudaFuncSetAttribute(k_atm_forces<MAP_LINEAR>, a, fb)) != cudaSuccess ||
            (e = cudaFuncSetAttribute(k_atm_energy<MAP_LAMBDA>, a, kEnergySmem)) != cudaSuccess ||
            (e = cudaFuncSetAttribute(k_atm_energy<MAP_BBOX>, a, kEnergySmem)) != cudaSuccess ||
            (e = cudaFuncSetAttribute(k_atm_energy<MAP_LINEAR>, a, kEnergySmem)) != cudaSuccess)
            return cuda_status(e);
        done[dev] = true;
    }
    return SIMPLEX_OK;
}

static int atm_check(int64_t n, int64_t d, const float *x, int map, void *ws, int64_t ws_bytes,
                     Grid &g, int64_t &nb) {
    if (n < 1 || d != 3 || !x || map < MAP_LAMBDA || map > MAP_LINEAR) return d != 3 && d > 0 ? SIMPLEX_EUNSUPPORTED : SIMPLEX_EINVAL;
    if (!aligned(x, 4)) return SIMPLEX_EALIGN;
    if (n > (1 << 22)) return SIMPLEX_EOVERFLOW;
    nb = (n + R_ - 1) / R_;
    g = grid3(nb, map);
    if (!grid_fits(g)) return SIMPLEX_EOVERFLOW;
    const int64_t need = 8 * (g.gx * g.gy * g.gz + kReduceSlots);
    if (!ws || ws_bytes < need || !aligned(ws, 256)) return SIMPLEX_EWORKSPACE;
    return SIMPLEX_OK;
}

}  // namespace sx

using namespace sx;

extern "C" int simplex_atm_energy(int64_t n, int64_t d, const float *x, float nu, float eps,
                                  double *energy, int map, void *workspace, int64_t ws_bytes,
                                  void *stream) {
    if (!energy) return SIMPLEX_EINVAL;
    Grid g;
    int64_t nb;
    int st = atm_check(n, d, x, map, workspace, ws_bytes, g, nb);
    if (st) return st;
    if (!aligned(energy, 8)) return SIMPLEX_EALIGN;
    cudaStream_t s = (cudaStream_t)stream;
    double *partials = (double *)workspace;
    const int64_t blocks = g.gx * g.gy * g.gz;
    double *tmp = partials + blocks;
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

extern "C" int simplex_atm_forces(int64_t n, int64_t d, const float *x, float nu, float eps,
                                  double *energy, double *forces, int map, void *workspace,
                                  int64_t ws_bytes, void *stream) {
    if (!forces) return SIMPLEX_EINVAL;
    Grid g;
    int64_t nb;
    int st = atm_check(n, d, x, map, workspace, ws_bytes, g, nb);
    if (st) return st;
    if (!aligned(forces, 8) || (energy && !aligned(energy, 8))) return SIMPLEX_EALIGN;
    cudaStream_t s = (cudaStream_t)stream;
    double *partials = energy ? (double *)workspace : nullptr;
    const int64_t blocks = g.gx * g.gy * g.gz;
    if ((st = cuda_status(cudaMemsetAsync(forces, 0, sizeof(double) * 3 * (size_t)n, s)))) return st;
    const int smem = (int)sizeof(AtmForceSmem);
    if ((st = smem_optin())) return st;
    prof_begin(s);
    if (map == MAP_LAMBDA) k_atm_forces<MAP_LAMBDA><<<dim_of(g), 256, smem, s>>>(n, x, nu, eps, (int)nb, g.p, partials, forces);
    else if (map == MAP_BBOX) k_atm_forces<MAP_BBOX><<<dim_of(g), 256, smem, s>>>(n, x, nu, eps, (int)nb, g.p, partials, forces);
    else k_atm_forces<MAP_LINEAR><<<dim_of(g), 256, smem, s>>>(n, x, nu, eps, (int)nb, g.p, partials, forces);
    prof_end(s);
    note_launches(1);
    if ((st = launch_status())) return st;
    if (energy) return reduce_partials(partials, blocks, partials + blocks, energy, s);
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
