// kernels.h -- tile sizes and sizing helpers shared between the kernels'
// translation units and the C entry points of libsimplex (private header).
#pragma once
#include <cstdint>

namespace sx {

constexpr int kEdmRho = 32;      // SIMT EDM tile: 32 x 32 pairs, 256 threads
constexpr int kAtmRho = 32;      // ATM tile: 32 x 32 x 32 triples, 256 threads
constexpr int kStressRho = 32;   // stress tile: 32 x 32 pairs, 256 threads

int edm_rho(int64_t d, int prec);
int64_t edm_workspace_bytes(int64_t n, int64_t d, int map, int prec);

}  // namespace sx
