// cover.cu -- decode tables and coverage counts of the block-space maps.
//
// simplex_map_blocks / simplex_map_blocks_host evaluate the maps of maps.cuh
// for every grid block (Sec. III-A eq. (map2d), Sec. III-C, Sec. III-D);
// simplex_map2, simplex_map3 and simplex_map4 launch each map's grid and
// count, per element of the simplex, how many threads reach it (it must be
// exactly one: the map covers Delta_n^m once, volumes of Sec. III-A/III-B)
// and how many threads reach none.
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
        for (int t = 0; t < L.cnt; ++t) { e[2 * t] = t ? L.x[1] : L.x[0]; e[2 * t + 1] = t ? L.y[1] : L.y[0]; }
    } else {
        List3 L = map == MAP_LAMBDA ? decode3_lambda(wx, wy, wz, g.p, nb)
                : map == MAP_BBOX   ? decode3_bbox(wx, wy, wz, nb)
                                    : decode3_linear(w, nb);
        for (int t = 0; t < L.cnt; ++t) {
            e[3 * t] = t ? L.i[1] : L.i[0];
            e[3 * t + 1] = t ? L.j[1] : L.j[0];
            e[3 * t + 2] = t ? L.k[1] : L.k[0];
        }
    }
}

// One m = 4 table entry (8 int32: (I, J, K, L) and an unused slot of -1).
SX_HD void table_entry4(int map, const Grid4 &g, int nb, int64_t w, int32_t *e) {
    const uint32_t x = (uint32_t)(w % g.gx);
    const uint32_t y = (uint32_t)((w / g.gx) % g.gy);
    const uint32_t z = (uint32_t)((w / (g.gx * g.gy)) % g.gz);
    const uint32_t ww = (uint32_t)(w / (g.gx * g.gy * g.gz));
    for (int t = 0; t < 8; ++t) e[t] = -1;
    const Blk4 B = map == MAP_LAMBDA ? decode4_lambda(x, y, z, ww, g.p, nb) : decode4_bbox(x, y, z, ww, nb);
    if (B.ok) { e[0] = B.i; e[1] = B.j; e[2] = B.k; e[3] = B.l; }
}

__global__ void k_map_blocks4(int map, Grid4 g, int nb, int64_t total, int32_t *out) {
    for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < total;
         w += (int64_t)gridDim.x * blockDim.x)
        table_entry4(map, g, nb, w, out + 8 * w);
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
        const int i = (t ? L.i[1] : L.i[0]) * rho + a, j = (t ? L.j[1] : L.j[0]) * rho + b,
                  k = (t ? L.k[1] : L.k[0]) * rho + c;
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

// Packed index of (i <= j <= k <= l): C(l+3, 4) + C(k+2, 3) + C(j+1, 2) + i,
// the first term as T(l) T(l+2) / 6 (T the triangular numbers) so that no
// product exceeds 2^63 for l < 2^16.
__device__ __forceinline__ int64_t index4(int i, int j, int k, int l) {
    const int64_t tl = (int64_t)l * (l + 1) / 2, tl2 = (int64_t)(l + 2) * (l + 3) / 2;
    return tl * tl2 / 6 + (int64_t)k * (k + 1) * (k + 2) / 6 + (int64_t)j * (j + 1) / 2 + i;
}

// Division by a divisor fixed at launch: floor(x / d) = (umulhi(x, m) + x) >> s
// with s = ceil(log2 d) and m = floor(2^32 (2^s - d) / d) + 1, exact for
// x < 2^31 (the round-up multiplier of Granlund and Montgomery, "Division by
// invariant integers using multiplication", PLDI 1994).
struct FastDiv {
    uint32_t d, m, s;
};

static FastDiv make_fastdiv(uint32_t d) {
    FastDiv f;
    f.d = d;
    f.s = 0;
    while ((1ull << f.s) < d) ++f.s;
    f.m = (uint32_t)((((1ull << 32) * ((1ull << f.s) - d)) / d) + 1);
    return f;
}

__device__ __forceinline__ uint32_t fast_div(uint32_t x, const FastDiv &f) {
    return (__umulhi(x, f.m) + x) >> f.s;
}

// One thread per (a, b, c, d) of a RHO^4 block (blockDim (RHO, RHO, RHO^2),
// threadIdx.z = c + RHO d) on the 4-D grid of grid4 (blockIdx.x = x + gx z,
// blockIdx.y = y, blockIdx.z = w); see simplex_map4 in simplex.h.
template <int MAP, int RHO>
__global__ void k_cover4(int64_t n, int nb, int p, FastDiv gx, int32_t *count,
                         unsigned long long *idle) {
    const int a = threadIdx.x, b = threadIdx.y, c = threadIdx.z % RHO, d = threadIdx.z / RHO;
    const uint32_t z = fast_div(blockIdx.x, gx), x = blockIdx.x - z * gx.d;
    const Blk4 B = MAP == MAP_LAMBDA ? decode4_lambda(x, blockIdx.y, z, blockIdx.z, p, nb)
                                     : decode4_bbox(x, blockIdx.y, z, blockIdx.z, nb);
    bool took = false;
    if (B.ok) {
        const int i = B.i * RHO + a, j = B.j * RHO + b, k = B.k * RHO + c, l = B.l * RHO + d;
        if (i <= j && j <= k && k <= l && l < n) {
            atomicAdd(count + index4(i, j, k, l), 1);
            took = true;
        }
    }
    const int idle_threads = __syncthreads_count(!took);
    if ((a | b | threadIdx.z) == 0 && idle_threads) atomicAdd(idle, (unsigned long long)idle_threads);
}

// The plane K = L of the lambda map: the 3-simplex of blocks {I <= J <= K},
// launched on the m = 3 lambda grid, block (I, J, K) taken as (I, J, K, K).
template <int RHO>
__global__ void k_cover4_plane(int64_t n, int nb, int p3, int32_t *count, unsigned long long *idle) {
    const int a = threadIdx.x, b = threadIdx.y, c = threadIdx.z % RHO, d = threadIdx.z / RHO;
    const List3 L = decode3<MAP_LAMBDA>(blockIdx.x, blockIdx.y, blockIdx.z, p3, nb);
    bool took = false;
    for (int t = 0; t < L.cnt; ++t) {
        const int Kb = t ? L.k[1] : L.k[0];
        const int i = (t ? L.i[1] : L.i[0]) * RHO + a, j = (t ? L.j[1] : L.j[0]) * RHO + b, k = Kb * RHO + c,
                  l = Kb * RHO + d;
        if (i <= j && j <= k && k <= l && l < n) {
            atomicAdd(count + index4(i, j, k, l), 1);
            took = true;
        }
    }
    const int idle_threads = __syncthreads_count(!took);
    if ((a | b | threadIdx.z) == 0 && idle_threads) atomicAdd(idle, (unsigned long long)idle_threads);
}

template <int RHO>
static void launch_cover4(int map, int64_t n, int nb, const Grid4 &g, int32_t *count,
                          unsigned long long *idle, cudaStream_t s) {
    const dim3 blk(RHO, RHO, RHO * RHO);
    const dim3 grd((unsigned)(g.gx * g.gz), (unsigned)g.gy, (unsigned)g.gw);
    const FastDiv gx = make_fastdiv((uint32_t)g.gx);
    if (map == MAP_LAMBDA) {
        k_cover4<MAP_LAMBDA, RHO><<<grd, blk, 0, s>>>(n, nb, g.p, gx, count, idle);
        const Grid g3 = grid3(nb, MAP_LAMBDA);
        k_cover4_plane<RHO><<<dim_of(g3), blk, 0, s>>>(n, nb, g3.p, count, idle);
    } else {
        k_cover4<MAP_BBOX, RHO><<<grd, blk, 0, s>>>(n, nb, 0, gx, count, idle);
    }
}

// Every map has an m = 2 form; the rectangular box has no m = 3 form.
// m = 4: the lambda map and the bounding box.
static bool valid_map(int m, int map) {
    if (m == 4) return map == MAP_LAMBDA || map == MAP_BBOX;
    return map >= MAP_LAMBDA && (map <= MAP_LINEAR || (m == 2 && map == MAP_RB));
}

}  // namespace sx

using namespace sx;

extern "C" int64_t simplex_grid_blocks(int m, int64_t nb, int map) {
    if (m < 2 || m > 4 || nb < 1 || nb > (1 << 20) || !valid_map(m, map)) return -1;
    if (m == 4) {
        if (nb > 4096) return -1;
        const Grid4 g = grid4(nb, map);
        return g.gx * g.gy * g.gz * g.gw;
    }
    Grid g = m == 2 ? grid2(nb, map) : grid3(nb, map);
    return g.gx * g.gy * g.gz;
}

extern "C" int simplex_map_blocks_host(int m, int64_t nb, int map, int32_t *out) {
    int64_t total = simplex_grid_blocks(m, nb, map);
    if (total < 0 || !out) return SIMPLEX_EINVAL;
    if (nb > 65535) return SIMPLEX_EOVERFLOW;
    if (m == 4) {
        const Grid4 g4 = grid4(nb, map);
        for (int64_t w = 0; w < total; ++w) table_entry4(map, g4, (int)nb, w, out + 8 * w);
        return SIMPLEX_OK;
    }
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
    cudaStream_t s = (cudaStream_t)stream;
    const int threads = 256;
    int64_t blocks = (total + threads - 1) / threads;
    if (blocks > 152 * 64) blocks = 152 * 64;
    prof_begin(s);
    if (m == 4) {
        k_map_blocks4<<<(unsigned)blocks, threads, 0, s>>>(map, grid4(nb, map), (int)nb, total, out);
    } else {
        Grid g = m == 2 ? grid2(nb, map) : grid3(nb, map);
        if (m == 2) k_map_blocks<2><<<(unsigned)blocks, threads, 0, s>>>(map, g, (int)nb, total, out);
        else k_map_blocks<3><<<(unsigned)blocks, threads, 0, s>>>(map, g, (int)nb, total, out);
    }
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
    if (n > 3000000) return SIMPLEX_EOVERFLOW;   // keeps the packed index and its products in 64 bits
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

extern "C" int simplex_map4(int64_t n, int rho, int map, int32_t *count, int64_t *idle,
                            void *stream) {
    if (rho == 0) rho = 4;
    if (n < 1 || rho < 1 || rho > 5 || !valid_map(4, map) || !count || !idle) return SIMPLEX_EINVAL;
    if (!aligned(count, 4) || !aligned(idle, 8)) return SIMPLEX_EALIGN;
    if (n > 65536) return SIMPLEX_EOVERFLOW;   // keeps the packed index below 2^63
    const int64_t nb = (n + rho - 1) / rho;
    const Grid4 g = grid4(nb, map);
    if (g.gx * g.gz > 0x7fffffffLL || g.gy > 65535 || g.gw > 65535) return SIMPLEX_EOVERFLOW;
    const int64_t vol = (n * (n + 1) / 2) * ((n + 2) * (n + 3) / 2) / 6;
    cudaStream_t s = (cudaStream_t)stream;
    int st = cuda_status(cudaMemsetAsync(count, 0, sizeof(int32_t) * (size_t)vol, s));
    if (st) return st;
    if ((st = cuda_status(cudaMemsetAsync(idle, 0, sizeof(int64_t), s)))) return st;
    unsigned long long *id = (unsigned long long *)idle;
    prof_begin(s);
    switch (rho) {
        case 1: launch_cover4<1>(map, n, (int)nb, g, count, id, s); break;
        case 2: launch_cover4<2>(map, n, (int)nb, g, count, id, s); break;
        case 3: launch_cover4<3>(map, n, (int)nb, g, count, id, s); break;
        case 4: launch_cover4<4>(map, n, (int)nb, g, count, id, s); break;
        default: launch_cover4<5>(map, n, (int)nb, g, count, id, s); break;
    }
    prof_end(s);
    note_launches(map == MAP_LAMBDA ? 2 : 1);
    return launch_status();
}
