// common.cuh -- shared helpers of libsimplex's kernels and C entry points.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#include "../../include/simplex.h"
#include "maps.cuh"

namespace sx {

// Records a failed CUDA call for simplex_last_cuda_error().
void set_cuda_error(cudaError_t e);

// Tracing: event pair around an entry point's main kernel (when profiling is
// on) and a count of every kernel launched.
void prof_begin(cudaStream_t s);
void prof_end(cudaStream_t s);
void note_launches(int k);

// Returns SIMPLEX_ECUDA (recording the error) if the last launch failed.
inline int launch_status() {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { set_cuda_error(e); return SIMPLEX_ECUDA; }
    return SIMPLEX_OK;
}

inline int cuda_status(cudaError_t e) {
    if (e != cudaSuccess) { set_cuda_error(e); return SIMPLEX_ECUDA; }
    return SIMPLEX_OK;
}

inline bool aligned(const void *p, uintptr_t a) { return ((uintptr_t)p % a) == 0; }

// Grid limits of a launch: x < 2^31, y and z < 2^16.
inline bool grid_fits(const Grid &g) {
    return g.gx >= 1 && g.gy >= 1 && g.gz >= 1 && g.gx <= 2147483647LL && g.gy <= 65535 &&
           g.gz <= 65535;
}

inline dim3 dim_of(const Grid &g) { return dim3((unsigned)g.gx, (unsigned)g.gy, (unsigned)g.gz); }

__device__ __forceinline__ double warp_sum_f64(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_sum_f32(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over a block of NT threads (NT a multiple of 32) in FP64; the result
// is valid in thread 0.  `red` holds NT/32 doubles of shared memory.
template <int NT>
__device__ __forceinline__ double block_sum_f64(double v, double *red) {
    v = warp_sum_f64(v);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x < 32) {
        s = (lane < NT / 32) ? red[lane] : 0.0;
        s = warp_sum_f64(s);
    }
    return s;
}

// Compensated FP32 sums: (hi, lo) carries a value and the rounding error of
// its additions (Knuth's TwoSum), so block sums keep ~2x FP32 precision
// without FP64 arithmetic, which is slow on this part.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// (hi, lo) += (h2, l2), renormalised.
__device__ __forceinline__ void add_ff(float &hi, float &lo, float h2, float l2) {
    float s, e;
    two_sum(hi, h2, s, e);
    e += lo + l2;
    hi = s + e;
    lo = e - (hi - s);
}

// Block sum of (hi, lo) pairs over NT threads; the FP64 result is valid in
// thread 0.  `red` holds 2 * NT/32 floats of shared memory.
template <int NT>
__device__ __forceinline__ double block_sum_ff(float hi, float lo, float *red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
        const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
        add_ff(hi, lo, h2, l2);
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { red[2 * w] = hi; red[2 * w + 1] = lo; }
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0) {
        // the warps' pairs combined in FP32 (FP64 is slow on this part), one conversion
        float h = red[0], l = red[1];
        for (int t = 1; t < NT / 32; ++t) add_ff(h, l, red[2 * t], red[2 * t + 1]);
        s = (double)h + (double)l;
    }
    return s;
}

// Deterministic FP64 sum of `count` per-block partials into *out (written,
// not accumulated): pass 1 reduces fixed chunks into tmp[], pass 2 sums tmp.
// tmp needs kReduceSlots doubles.
constexpr int kReduceSlots = 1024;
int reduce_partials(const double *partials, int64_t count, double *tmp, double *out,
                    cudaStream_t s);

}  // namespace sx
