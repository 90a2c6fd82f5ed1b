// cover.cu -- decode tables and coverage counts of the block-space maps.
//
// simplex_map_blocks / simplex_map_blocks_host evaluate the maps of maps.cuh
// for every grid block (Sec. III-A eq. (map2d), Sec. III-C); simplex_map2 and
// simplex_map3 launch each map's grid and count, per element of the simplex,
// how many threads reach it (it must be exactly one: the map is a bijection
// onto Delta_n^m, volumes of Sec. III-A/III-B) and how many threads reach
// none.
#include "common.cuh"

namespace sx {

// Writes one table entry (2m int32) for grid block w of shape g.
template <int M>
SX_HD void table_entry(int map, const Grid &g, int nb, int64_t w, int32_t *e) {
    const uint32_t wx = (uint32_t)(w % g.gx);
    const uint32_t wy = (uint32_t)((w / g.gx) % g.gy);
    const uint32_t wz = (uint32_t)(w / (g.gx * g.gy));
    for (int t = 0; t < 2 * M; ++t) e[t] = -1;
    if (M == 2) {
        List2 L = map == MAP_LAMBDA ? decode2_lambda(wx, wy, nb)
                : map == MAP_BBOX   ? decode2_bbox(wx, wy, nb)
                : map == MAP_RB     ? decode2_rb(wx, wy, nb)
                                    : decode2_linear(w, nb);
        for (int t = 0; t < L.cnt; ++t) { e[2 * t] = L.x[t]; e[2 * t + 1] = L.y[t]; }
    } else {
        List3 L = map == MAP_LAMBDA ? decode3_lambda(wx, wy, wz, g.p, nb)
                : map == MAP_BBOX   ? decode3_bbox(wx, wy, wz, nb)
                                    : decode3_linear(w, nb);
        for (int t = 0; t < L.cnt; ++t) {
            e[3 * t] = L.i[t]; e[3 * t + 1] = L.j[t]; e[3 * t + 2] = L.k[t];
        }
    }
}

template <int M>
__global__ void k_map_blocks(int map, Grid g, int nb, int64_t total, int32_t *out) {
    for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < total;
         w += (int64_t)gridDim.x * blockDim.x)
        table_entry<M>(map, g, nb, w, out + 2 * M * w);
}

// The idle threads of a block are counted in the barrier that ends it
// (__syncthreads_count: one bar.red.popc over the block's predicates; every
// thread of the block reaches it) and added by one global atomic per block.

// One thread per (r, c) of a rho x rho block; see simplex_map2 in simplex.h.
template <int MAP>
__global__ void k_cover2(int64_t n, int rho, int nb, int32_t *count,
                         unsigned long long *idle) {
    const int r = threadIdx.y, c = threadIdx.x;
    const List2 L = decode2<MAP>(blockIdx.x, blockIdx.y, nb);
    bool took = false;
    if (L.pair) {
        for (int extra = 0; extra < 2; ++extra) {
            if (extra && c != 0) break;
            const int cc = extra ? rho : c;
            int64_t i, j;
            if (cc <= r) { i = (int64_t)L.d0 * rho + r; j = (int64_t)L.d0 * rho + cc; }
            else { i = (int64_t)L.d1 * rho + (rho - 1 - r); j = (int64_t)L.d1 * rho + (cc - r - 1); }
            if (i < n) { atomicAdd(count + (i * (i + 1) / 2 + j), 1); took = true; }
        }
    } else if (L.cnt > 0) {
        const int64_t i = (int64_t)L.y[0] * rho + r, j = (int64_t)L.x[0] * rho + c;
        if (j <= i && i < n) { atomicAdd(count + (i * (i + 1) / 2 + j), 1); took = true; }
    }
    const int idle_threads = __syncthreads_count(!took);
    if (r == 0 && c == 0 && idle_threads) atomicAdd(idle, (unsigned long long)idle_threads);
}

// One thread per (a, b, c) of a rho^3 block; see simplex_map3 in simplex.h.
template <int MAP>
__global__ void k_cover3(int64_t n, int rho, int nb, int p, int32_t *count,
                         unsigned long long *idle) {
    const int a = threadIdx.x, b = threadIdx.y, c = threadIdx.z;
    const List3 L = decode3<MAP>(blockIdx.x, blockIdx.y, blockIdx.z, p, nb);
    bool took = false;
    for (int t = 0; t < L.cnt; ++t) {
        // n <= 3,000,000 (checked by simplex_map3): the coordinates fit in
        // 32 bits; the tetrahedral number k(k+1)/2 * (k+2) / 3 stays below
        // 2^64 in unsigned 64-bit arithmetic
        const int i = L.i[t] * rho + a, j = L.j[t] * rho + b, k = L.k[t] * rho + c;
        if (i <= j && j <= k && k < n) {
            const uint64_t kk = (uint32_t)k, jj = (uint32_t)j;
            const uint64_t tet_k = kk * (kk + 1) / 2 * (kk + 2) / 3;
            atomicAdd(count + (tet_k + jj * (jj + 1) / 2 + (uint32_t)i), 1);
            took = true;
        }
    }
    const int idle_threads = __syncthreads_count(!took);
    if ((a | b | c) == 0 && idle_threads) atomicAdd(idle, (unsigned long long)idle_threads);
}

// Every map has an m = 2 form; the rectangular box has no m = 3 form.
static bool valid_map(int m, int map) {
    return map >= MAP_LAMBDA && (map <= MAP_LINEAR || (m == 2 && map == MAP_RB));
}

}  // namespace sx

using namespace sx;

extern "C" int64_t simplex_grid_blocks(int m, int64_t nb, int map) {
    if ((m != 2 && m != 3) || nb < 1 || nb > (1 << 20) || !valid_map(m, map)) return -1;
    Grid g = m == 2 ? grid2(nb, map) : grid3(nb, map);
    return g.gx * g.gy * g.gz;
}

extern "C" int simplex_map_blocks_host(int m, int64_t nb, int map, int32_t *out) {
    int64_t total = simplex_grid_blocks(m, nb, map);
    if (total < 0 || !out) return SIMPLEX_EINVAL;
    if (nb > 65535) return SIMPLEX_EOVERFLOW;
    Grid g = m == 2 ? grid2(nb, map) : grid3(nb, map);
    for (int64_t w = 0; w < total; ++w) {
        if (m == 2) table_entry<2>(map, g, (int)nb, w, out + 4 * w);
        else table_entry<3>(map, g, (int)nb, w, out + 6 * w);
    }
    return SIMPLEX_OK;
}

extern "C" int simplex_map_blocks(int m, int64_t nb, int map, int32_t *out, void *stream) {
    int64_t total = simplex_grid_blocks(m, nb, map);
    if (total < 0 || !out) return SIMPLEX_EINVAL;
    if (nb > 65535) return SIMPLEX_EOVERFLOW;
    if (!aligned(out, 4)) return SIMPLEX_EALIGN;
    Grid g = m == 2 ? grid2(nb, map) : grid3(nb, map);
    cudaStream_t s = (cudaStream_t)stream;
    const int threads = 256;
    int64_t blocks = (total + threads - 1) / threads;
    if (blocks > 152 * 64) blocks = 152 * 64;
    prof_begin(s);
    if (m == 2) k_map_blocks<2><<<(unsigned)blocks, threads, 0, s>>>(map, g, (int)nb, total, out);
    else k_map_blocks<3><<<(unsigned)blocks, threads, 0, s>>>(map, g, (int)nb, total, out);
    prof_end(s);
    note_launches(1);
    return launch_status();
}

extern "C" int simplex_map2(int64_t n, int rho, int map, int32_t *count, int64_t *idle,
                            void *stream) {
    if (rho == 0) rho = 16;
    if (n < 1 || rho < 1 || rho > 32 || !valid_map(2, map) || !count || !idle) return SIMPLEX_EINVAL;
    if (!aligned(count, 4) || !aligned(idle, 8)) return SIMPLEX_EALIGN;
    const int64_t nb = (n + rho - 1) / rho;
    if (n > (int64_t)1 << 31) return SIMPLEX_EOVERFLOW;
    Grid g = grid2(nb, map);
    if (!grid_fits(g)) return SIMPLEX_EOVERFLOW;
    cudaStream_t s = (cudaStream_t)stream;
    int st = cuda_status(cudaMemsetAsync(count, 0, sizeof(int32_t) * (size_t)(n * (n + 1) / 2), s));
    if (st) return st;
    if ((st = cuda_status(cudaMemsetAsync(idle, 0, sizeof(int64_t), s)))) return st;
    dim3 blk(rho, rho);
    unsigned long long *id = (unsigned long long *)idle;
    prof_begin(s);
    if (map == MAP_LAMBDA) k_cover2<MAP_LAMBDA><<<dim_of(g), blk, 0, s>>>(n, rho, (int)nb, count, id);
    else if (map == MAP_BBOX) k_cover2<MAP_BBOX><<<dim_of(g), blk, 0, s>>>(n, rho, (int)nb, count, id);
    else if (map == MAP_RB) k_cover2<MAP_RB><<<dim_of(g), blk, 0, s>>>(n, rho, (int)nb, count, id);
    else k_cover2<MAP_LINEAR><<<dim_of(g), blk, 0, s>>>(n, rho, (int)nb, count, id);
    prof_end(s);
    note_launches(1);
    return launch_status();
}

extern "C" int simplex_map3(int64_t n, int rho, int map, int32_t *count, int64_t *idle,
                            void *stream) {
    if (rho == 0) rho = 8;
    if (n < 1 || rho < 1 || rho > 10 || !valid_map(3, map) || !count || !idle) return SIMPLEX_EINVAL;
    if (!aligned(count, 4) || !aligned(idle, 8)) return SIMPLEX_EALIGN;
    if (n > 3000000) return SIMPLEX_EOVERFLOW;   // keeps k(k+1)(k+2) < 2^63
    const int64_t nb = (n + rho - 1) / rho;
    Grid g = grid3(nb, map);
    if (!grid_fits(g)) return SIMPLEX_EOVERFLOW;
    cudaStream_t s = (cudaStream_t)stream;
    int st = cuda_status(cudaMemsetAsync(count, 0, sizeof(int32_t) * (size_t)(n * (n + 1) * (n + 2) / 6), s));
    if (st) return st;
    if ((st = cuda_status(cudaMemsetAsync(idle, 0, sizeof(int64_t), s)))) return st;
    dim3 blk(rho, rho, rho);
    unsigned long long *id = (unsigned long long *)idle;
    prof_begin(s);
    if (map == MAP_LAMBDA) k_cover3<MAP_LAMBDA><<<dim_of(g), blk, 0, s>>>(n, rho, (int)nb, g.p, count, id);
    else if (map == MAP_BBOX) k_cover3<MAP_BBOX><<<dim_of(g), blk, 0, s>>>(n, rho, (int)nb, g.p, count, id);
    else k_cover3<MAP_LINEAR><<<dim_of(g), blk, 0, s>>>(n, rho, (int)nb, g.p, count, id);
    prof_end(s);
    note_launches(1);
    return launch_status();
}
