// kernels.h -- tile sizes and sizing helpers shared between the kernels'
// translation units and the C entry points of libsimplex (private header).
#pragma once
#include <cstdint>

#include <cuda_runtime.h>

namespace sx {

constexpr int kEdmRho = 32;      // SIMT EDM tile: 32 x 32 pairs, 256 threads
constexpr int kAtmRho = 32;      // ATM tile: 32 x 32 x 32 triples, 256 threads
constexpr int kStressRho = 64;   // stress tile: 64 x 64 pairs, 256 threads

int edm_rho(int64_t d, int prec);
int64_t atm_energy_workspace_bytes(int64_t n, int map);
int64_t atm_forces_workspace_bytes(int64_t n, int map);
int atm_device_errors(cudaStream_t s);
int64_t edm_workspace_bytes(int64_t n, int64_t d, int map, int prec);

// Tensor-core EDM (edm_umma.cu): tiles of 128 x 128 pairs, d % 64 == 0.
constexpr int kEdmUmmaRho = 128;
int64_t edm_umma_workspace_bytes(int64_t n, int64_t d);
// tiles: the tile-packed output layout (simplex_edm_tiles) instead of the
// packed rows (simplex_edm_packed)
int edm_umma_run(int64_t n, int64_t d, const float *x, float *out, int map, bool tiles, void *ws,
                 int64_t ws_bytes, cudaStream_t s);
int umma_device_errors(cudaStream_t s);

// Tensor-core stress loss and gradient (stress_umma.cu): tiles of 128 x 128
// pairs, d % 32 == 0 and d <= 96.
constexpr int kStressUmmaRho = 128;
bool stress_umma_ok(int64_t d);
bool stress_use_umma(int64_t d, int prec);
int64_t stress_umma_workspace_bytes(int64_t n, int64_t d, bool bwd);
int stress_umma_run(bool bwd, int64_t n, int64_t d, const float *x, const float *y, float *d_out,
                    double *loss, double gscale, float *grad, int map, void *ws, int64_t ws_bytes,
                    cudaStream_t s);
int stress_umma_errors(cudaStream_t s);

}  // namespace sx
