/*
 * simplex.h -- C ABI of libsimplex: block-space maps over discrete orthogonal
 * simplices and the simplex-domain kernels they drive, for one GB300 (sm_103a).
 *
 * Paper: C. A. Navarro, B. Bustos, N. Hitschfeld, "Possibilities of Recursive
 * GPU Mapping for Discrete Orthogonal Simplices", arXiv 1610.07394.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Pointers marked "device" are CUDA device pointers owned by the caller;
 *    the library never frees or retains them.  `stream` is a cudaStream_t
 *    (NULL = legacy default stream).  Work is enqueued on `stream` and the
 *    call returns without synchronising; outputs are valid once the stream
 *    reaches that point.
 *  - Points are FP32, row-major n x d (row stride d floats).
 *  - 2-simplex elements are pairs (i, j) with 0 <= j <= i < n, stored packed
 *    row-major lower: index i(i+1)/2 + j (64-bit).  3-simplex elements are
 *    triples 0 <= i <= j <= k < n, index k(k+1)(k+2)/6 + j(j+1)/2 + i.
 *  - A block is a tile of rho consecutive points; nb = ceil(n / rho).  The
 *    maps send grid blocks to data blocks:
 *      SIMPLEX_MAP_LAMBDA  the recursive O(1) map (Sec. III-A eq. (map2d) for
 *                          m=2; Sec. III-C two-branch map for m=3), nb padded
 *                          up to a power of two and filtered ("approach n
 *                          from above", Sec. III-A);
 *      SIMPLEX_MAP_BBOX    bounding box f(x) = x with out-of-domain blocks
 *                          exiting at once (Sec. I);
 *      SIMPLEX_MAP_LINEAR  linear enumeration inverted with square / cube
 *                          roots plus an exact integer fix-up (Sec. I and
 *                          Sec. II on the earlier block-space maps);
 *      SIMPLEX_MAP_RB      rectangular box, 2-simplex only (Sec. II: the RB
 *                          strategy for packed triangular matrices applied
 *                          to the parallel space): the block triangle cut
 *                          at half height, grid row k holding triangle rows
 *                          floor(nb/2) + k and floor(nb/2) - 1 - k, no idle
 *                          block for any nb.  The 3-simplex entry points
 *                          (simplex_map3, ATM) return SIMPLEX_EINVAL for it.
 *  - Return value: a simplex_status.  Argument errors are detected before
 *    anything is enqueued and leave outputs untouched.  A failed launch
 *    returns SIMPLEX_ECUDA; simplex_last_cuda_error() gives the cudaError_t.
 *    Asynchronous faults surface at the caller's next synchronisation.
 *  - Scratch: entry points that need scratch take (workspace, ws_bytes),
 *    device memory owned by the caller, at least simplex_workspace_bytes()
 *    bytes and 256-byte aligned.  The library allocates no device memory.
 */
#ifndef SIMPLEX_H
#define SIMPLEX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SIMPLEX_OK = 0,
    SIMPLEX_EINVAL = 1,       /* bad size, map, precision, or NULL pointer   */
    SIMPLEX_EALIGN = 2,       /* pointer not aligned as documented           */
    SIMPLEX_EOVERFLOW = 3,    /* size exceeds 64-bit indices or grid limits  */
    SIMPLEX_EUNSUPPORTED = 4, /* valid request the library does not serve    */
    SIMPLEX_ECUDA = 5,        /* a CUDA call failed                          */
    SIMPLEX_EWORKSPACE = 6,   /* workspace missing, too small or misaligned  */
    SIMPLEX_ESCRATCH = 7,     /* problem too large for the library's static
                                 scratch (simplex_atm_energy_noalloc)        */
    SIMPLEX_ETIMEOUT = 8      /* a bounded device-side wait ran out          */
} simplex_status;

typedef enum {
    SIMPLEX_MAP_LAMBDA = 0,
    SIMPLEX_MAP_BBOX = 1,
    SIMPLEX_MAP_LINEAR = 2,
    SIMPLEX_MAP_RB = 3
} simplex_map;

typedef enum {
    SIMPLEX_PREC_FP32 = 0,    /* every step in FP32 (difference form)        */
    SIMPLEX_PREC_BF16X3 = 1,  /* Gram term on tensor cores, split BF16 hi+lo */
    SIMPLEX_PREC_AUTO = 2     /* library choice by d                          */
} simplex_prec;

typedef enum {
    SIMPLEX_OP_MAP2 = 0, SIMPLEX_OP_MAP3 = 1, SIMPLEX_OP_EDM = 2,
    SIMPLEX_OP_ATM_ENERGY = 3, SIMPLEX_OP_ATM_FORCES = 4,
    SIMPLEX_OP_STRESS_FWD = 5, SIMPLEX_OP_STRESS_BWD = 6, SIMPLEX_OP_STRESS_FWD_BWD = 7
} simplex_op;

/* ABI version of this header (bumped on any signature change or added entry
 * point or map; 2 added simplex_stress_fwd_bwd, 3 SIMPLEX_MAP_RB, 4
 * simplex_map4 and the m = 4 tables, 5 simplex_edm_tiles and
 * simplex_edm_tiles_len). */
int simplex_abi_version(void);

/* Human-readable text of a status code (static storage). */
const char *simplex_strerror(int status);

/* cudaError_t of the last failed CUDA call made by this library on the
 * calling thread (0 if none). */
int simplex_last_cuda_error(void);

/* Block edge rho used by an operation (the library's tile size), for callers
 * that want nb = ceil(n / rho). */
int simplex_block_rho(int op, int64_t d, int prec);

/*
 * Number of grid blocks a map launches over nb data blocks per side for an
 * m-simplex (m = 2, 3 or 4), or -1 on bad arguments.  Grid shapes: LAMBDA
 * m=2 (p/2) x p, m=3 (p/2) x (p/2) x (p/2 + p/4 + 2) with p the power of two
 * >= max(nb, 2) (the last two z-layers are the plane J = K, mapped by the
 * 2-simplex map), m=4 (p/2)^3 x (p/2 + p/8) (p >= 8; + 1 layer at p = 4,
 * none at p = 2) for the blocks I <= J <= K < L only (the plane K = L takes
 * the m = 3 grid, see simplex_map4); BBOX nb^m; LINEAR nb(nb+1)/2 or
 * nb(nb+1)(nb+2)/6; RB (m=2) (nb + 1 - nb mod 2) x ceil(nb/2) = nb(nb+1)/2.
 * m = 4 takes LAMBDA and BBOX only, nb <= 4096.
 */
int64_t simplex_grid_blocks(int m, int64_t nb, int map);

/*
 * Decode table of a map (Sec. III-A eq. (map2d) / Sec. III-C / Sec. III-D):
 * for every grid block w (x fastest, then y, then z, then w for m = 4) the
 * data blocks it is sent to, (X0, Y0, X1, Y1) for m=2 (X = column block <=
 * Y = row block), (I0, J0, K0, I1, J1, K1) for m=3 or (I0, J0, K0, L0, -1,
 * -1, -1, -1) for m=4, with -1 in unused slots.  The second
 * slot is used only by grid row 0 of the 2-simplex map, which takes the
 * diagonal blocks 2w and 2w+1 (the paper leaves the diagonal out; this is
 * the library's reading).
 * out: device, simplex_grid_blocks(m, nb, map) * (2m) int32.
 */
int simplex_map_blocks(int m, int64_t nb, int map, int32_t *out, void *stream);

/* The same table computed on the host by the same decode functions
 * (no GPU needed).  out: host memory of the same size. */
int simplex_map_blocks_host(int m, int64_t nb, int map, int32_t *out);

/*
 * Coverage of Delta_n^2 (Sec. III-A): launch the map's grid with rho x rho
 * threads per block, every thread adds 1 to count[] for each element it is
 * sent to, and threads sent to no element add 1 to *idle.
 * Thread (r, c) of a block sent to (X, Y) takes element (Y rho + r, X rho + c)
 * when column <= row < n.  A grid-row-0 block of the 2-simplex map reads its
 * two diagonal triangles as one rho x (rho+1) rectangle: cell (r, c) is
 * element (r, c) of block 2w when c <= r, else element (rho-1-r, c-r-1) of
 * block 2w+1; thread (r, c) takes cell (r, c) and, if c == 0, cell (r, rho).
 * n >= 1; rho in [1, 32] (0 = 16).
 * count: device, n(n+1)/2 int32 (zeroed by the call); idle: device, 1 int64.
 */
int simplex_map2(int64_t n, int rho, int map, int32_t *count, int64_t *idle,
                 void *stream);

/*
 * Coverage of Delta_n^3 (Sec. III-B/III-C): rho^3 threads per block; a block
 * walks its list of data blocks in order and thread (a, b, c) takes element
 * (I rho + a, J rho + b, K rho + c) of each when i <= j <= k < n.
 * n >= 1; rho in [1, 10] (0 = 8).
 * count: device, n(n+1)(n+2)/6 int32 (zeroed by the call); idle: device, 1 int64.
 */
int simplex_map3(int64_t n, int rho, int map, int32_t *count, int64_t *idle,
                 void *stream);

/*
 * Coverage of Delta_n^4 = {i <= j <= k <= l < n} (Sec. III-D: the recursive
 * set with r = 1/2 and beta = 2, V(S_n^4) = (n^4 - n)/14; the paper gives
 * the set and its volume but no map, so the map is this library's reading:
 * the blocks I <= J <= K < L of one level, split at half size h, are the
 * copies L L L L and H H H H (recursion) and the cross terms, which one h^4
 * orthotope covers with idle points: local (a, b, c, d) goes to
 *   (a, b, h+d, h+c)   if a <= b, d < c;
 *   (a, b, c, h+d)     if a <= b, b <= c <= d;
 *   (a, h+c, h+d, h+b) if a <= b, c <= d, a <= c, d < b;
 *   (c, d, a, h+b)     if b < a, c <= d <= a;
 *   (a, h+b, h+d, h+c) if b < a, b <= d < c;
 * and nowhere otherwise).  rho^4 threads per block, blockDim (rho, rho,
 * rho^2); thread (a, b, c + rho d) takes element (I rho + a, J rho + b,
 * K rho + c, L rho + d) when i <= j <= k <= l < n.  LAMBDA launches two
 * grids: the m = 4 grid of simplex_grid_blocks(4, ...) and, for the plane
 * K = L, the m = 3 lambda grid with block (I, J, K) taken as (I, J, K, K).
 * BBOX launches nb^4 blocks.  Packed index of (i, j, k, l):
 * l(l+1)(l+2)(l+3)/24 + k(k+1)(k+2)/6 + j(j+1)/2 + i.
 * n in [1, 65536]; rho in [1, 5] (0 = 4); map LAMBDA or BBOX (else EINVAL).
 * count: device, n(n+1)(n+2)(n+3)/24 int32 (zeroed by the call); idle:
 * device, 1 int64.
 */
int simplex_map4(int64_t n, int rho, int map, int32_t *count, int64_t *idle,
                 void *stream);

/*
 * Packed lower-triangular Euclidean distance matrix (Sec. I: the EDM is a
 * 2-simplex problem): out[i(i+1)/2 + j] = |x_i - x_j|^2 (squared distance)
 * for 0 <= j <= i < n; the diagonal is exactly 0.
 * x: device, n*d FP32, 4-byte aligned.  out: device, n(n+1)/2 FP32.
 * prec: SIMPLEX_PREC_FP32 (difference form, any d, 32 x 32 tiles) or
 * SIMPLEX_PREC_BF16X3: |x_i|^2 + |x_j|^2 - 2 x_i.x_j with the Gram term on
 * tensor cores (tcgen05, FP32 accumulation in tensor memory) from a BF16
 * split x = hi + lo (three products hi.hi + hi.lo + lo.hi), FP32 norms, and
 * an FP32 recompute of entries below (|x_i|^2 + |x_j|^2)/64; 128 x 128 tiles;
 * needs d % 64 == 0.  AUTO picks BF16X3 when d >= 64 and d % 64 == 0.
 * BF16X3 needs workspace (simplex_workspace_bytes; 1024-byte aligned) for
 * the BF16 copies and the norms.  Its device waits are bounded: check
 * simplex_device_errors() when a result must be trusted.
 */
int simplex_edm_packed(int64_t n, int64_t d, const float *x, float *out, int map,
                       int prec, void *workspace, int64_t ws_bytes, void *stream);

/*
 * The same squared distances in a tile-packed layout, where every 128 x 128
 * tile of the matrix is one contiguous block of 64 KB.  Sec. II cites the
 * rectangular-box (RB) packing of a triangular matrix into whole rectangles;
 * this is that idea on the data side, at tile granularity: the triangle of
 * tiles is stored without gaps, each tile a dense rectangle, so a kernel
 * writes a tile (or a 32-row quarter of it, 16 KB) with a few large copies
 * instead of one copy per row segment of the row-major packing.
 * Layout: nt = ceil(n / 128) tile rows; tile (I, J), 0 <= J <= I < nt, holds
 * rows 128 I .. 128 I + 127 and columns 128 J .. 128 J + 127, stored row-major
 * at floats [s * 16384, (s + 1) * 16384) with s = I(I+1)/2 + J (the tiles in
 * packed lower order, the same for every map).  So pair (i, j), j <= i, is at
 *   ((i/128)(i/128 + 1)/2 + j/128) * 16384 + (i mod 128) * 128 + (j mod 128).
 * A diagonal tile (I = J) holds the whole square: its entry (a, b) with b > a
 * is |x_i - x_j|^2 for (i, j) = (128 I + a, 128 I + b), formed the same way as
 * the lower entries (so equal to its mirror within the stated tolerance);
 * the diagonal is exactly 0.  Entries whose row or column is >= n (the
 * padding of the last tile row when n is not a multiple of 128) are 0.
 * out: device, simplex_edm_tiles_len(n) FP32 (nt(nt+1)/2 * 16384 floats,
 * 0.2% more than n(n+1)/2 at n = 65536), every float written by the call;
 * 16-byte aligned on the tensor-core path (its tiles leave by TMA tensor
 * stores; SIMPLEX_EALIGN otherwise), 4-byte aligned on the FP32 path.  The
 * other arguments, precisions, workspace and errors are those of
 * simplex_edm_packed; SIMPLEX_EOVERFLOW also when nt(nt+1)/2 >= 2^31.
 */
int simplex_edm_tiles(int64_t n, int64_t d, const float *x, float *out, int map,
                      int prec, void *workspace, int64_t ws_bytes, void *stream);

/* Floats of the tile-packed EDM of n points, nt(nt+1)/2 * 16384 with
 * nt = ceil(n / 128); -1 when n < 1 or n > 2^31. */
int64_t simplex_edm_tiles_len(int64_t n);

/*
 * Axilrod-Teller-Muto triple-dipole energy over the 3-simplex (Sec. I:
 * triple-interaction n-body is a 3-simplex problem):
 *   E = sum_{i<j<k} nu (1 + 3 cos g_i cos g_j cos g_k) / (r_ij r_jk r_ki)^3,
 * every squared side softened r^2 -> r^2 + eps in the cosines' norms and in
 * the denominator (cosines from the law of cosines on unsoftened squares).
 * d must be 3.  x: device, n*3 FP32.  energy: device, 1 double (written).
 * Per-triple arithmetic is FP32; the reduction across blocks is FP64.
 */
int simplex_atm_energy(int64_t n, int64_t d, const float *x, float nu, float eps,
                       double *energy, int map, void *workspace, int64_t ws_bytes,
                       void *stream);

/*
 * ATM forces F = -dE/dx (n x 3 FP64, written) and, if `energy` is not NULL,
 * the energy, over the tiles of the same block grid: every triple adds
 * dE/d(r^2) of its three sides to per-pair coefficients, which are turned
 * into forces once per tile; forces accumulate in FP64.  A persistent kernel
 * (as many blocks as are resident at once) takes the map's grid blocks in
 * launch order from a counter in the workspace.  Workspace:
 * simplex_workspace_bytes(SIMPLEX_OP_ATM_FORCES, ...) bytes, 256-byte
 * aligned: the pair terms of every block pair (72 KB each, computed once per
 * call, up to 16 GB; beyond that the tiles build their own), the 16-byte
 * tile counter (zeroed by the call) and FP64 partials, one per grid block at
 * most.  Calls that share a workspace must not overlap.
 */
int simplex_atm_forces(int64_t n, int64_t d, const float *x, float nu, float eps,
                       double *energy, double *forces, int map, void *workspace,
                       int64_t ws_bytes, void *stream);

/*
 * Stress loss over the packed EDM: L = sum_{i<j} (D_ij - delta_ij)^2 with
 * D_ij = |x_i - x_j|^2 and delta_ij = |y_i - y_j|^2 recomputed from y.
 * x, y: device, n*d FP32.  d_out: device, n(n+1)/2 FP32, or NULL to skip
 * storing D.  loss: device, 1 double (written).
 */
int simplex_stress_fwd(int64_t n, int64_t d, const float *x, const float *y,
                       float *d_out, double *loss, int map, int prec,
                       void *workspace, int64_t ws_bytes, void *stream);

/*
 * Gradient of the stress loss times `gscale`:
 *   grad_i = gscale * 4 sum_{j != i} (D_ij - delta_ij)(x_i - x_j),
 * with D and delta recomputed (never stored).  grad: device, n*d FP32,
 * 16-byte aligned, written (zeroed by the call).
 */
int simplex_stress_bwd(int64_t n, int64_t d, const float *x, const float *y,
                       double gscale, float *grad, int map, int prec,
                       void *workspace, int64_t ws_bytes, void *stream);

/*
 * Loss and gradient in one pass (Sec. I: one sweep of the 2-simplex of
 * pairs serves both): grad as simplex_stress_bwd (times gscale, written) and
 * loss as simplex_stress_fwd (device, 1 double, written, not scaled), both
 * from the same residual tiles.  Workspace: simplex_workspace_bytes(
 * SIMPLEX_OP_STRESS_FWD_BWD, ...) bytes, 256-byte aligned (per-block loss
 * partials, and the tensor-core operands where prec selects them, with the
 * tensor-core backward's chunk starts and per-point row sums).
 * SIMPLEX_EINVAL if loss or grad is NULL.
 */
int simplex_stress_fwd_bwd(int64_t n, int64_t d, const float *x, const float *y,
                           double gscale, float *grad, double *loss, int map, int prec,
                           void *workspace, int64_t ws_bytes, void *stream);

/* Synchronises `stream` and reports whether any bounded device-side wait of
 * the tensor-core kernels ran out since the last check (SIMPLEX_ETIMEOUT,
 * flag cleared), else SIMPLEX_OK. */
int simplex_device_errors(void *stream);

/* Bytes of workspace an operation needs (0 if none, -1 on bad arguments). */
int64_t simplex_workspace_bytes(int op, int64_t n, int64_t d, int map, int prec);

/*
 * simplex_atm_energy without any device allocation, for callers that cannot
 * allocate: a plug-in handed only a stream and its tensors by a host
 * framework whose caching allocator owns the device memory (a side
 * cudaMalloc can fail or fragment that pool), or a latency-critical loop
 * that must not call cudaMalloc/cudaFree because they can synchronise the
 * device.  The paper has no counterpart.  It runs the energy kernel that
 * builds its pair tables per tile (simplex_atm_energy precomputes them into
 * its workspace), so the two agree to FP32 rounding (well within 1e-6
 * relative), not bit for bit.
 *
 * Scratch is a fixed 4 MiB array inside the library (one FP64 per grid block
 * plus 1024 reduction slots), held by every GPU that loads the library until
 * the process exits.  Problems whose grid needs more return SIMPLEX_ESCRATCH
 * before any work.  The rule is simplex_grid_blocks(3, ceil(n/32), map) +
 * 1024 <= 524288; in points that accepts n <= 4096 with the lambda map,
 * n <= 2560 with BBOX and n <= 4640 with LINEAR.  The first call on each
 * device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture.  The array needs no
 * clearing: every slot a call reads is written earlier in that call.  All
 * calls share the one array, so calls that can overlap on the GPU (different
 * streams, or different host threads) race and corrupt each other's result:
 * order them on one stream.  Arguments as simplex_atm_energy.
 */
int simplex_atm_energy_noalloc(int64_t n, int64_t d, const float *x, float nu, float eps,
                               double *energy, int map, void *stream);

/*
 * Tracing.  simplex_profile(1) clears the counters and starts recording;
 * simplex_profile(0) stops.  While on, every entry point records a CUDA
 * event pair around its main kernel on the call's stream (host bookkeeping
 * only; at most 65536 pairs are kept).  The library counts every kernel it
 * launches whether recording or not.
 */
int simplex_profile(int on);

/* Waits for the recorded events and returns the summed duration of the
 * timed main-kernel launches (ms), how many were timed, and how many kernels
 * the library launched since the last simplex_profile(1).  Any pointer may
 * be NULL. */
int simplex_profile_read(double *main_ms, int64_t *main_launches, int64_t *all_launches);

#ifdef __cplusplus
}
#endif

#endif /* SIMPLEX_H */
