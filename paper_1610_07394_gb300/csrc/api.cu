// api.cu -- status handling, workspace sizing and the FP64 cross-block
// reduction shared by the entry points of libsimplex.
#include <atomic>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace sx {

static thread_local int g_last_cuda_error = 0;

void set_cuda_error(cudaError_t e) { g_last_cuda_error = (int)e; }

// ---------------------------------------------------------------- tracing

namespace {
struct Profiler {
    std::mutex mu;
    bool on = false;
    std::vector<cudaEvent_t> ev;     // start/stop pairs, reused across sessions
    size_t used = 0;                 // events recorded this session (even count)
    bool open = false;
};
Profiler g_prof;
std::atomic<int64_t> g_launches{0};
constexpr size_t kMaxPairs = 65536;
}  // namespace

void note_launches(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

static void prof_record(cudaStream_t s, bool begin) {
    std::lock_guard<std::mutex> lk(g_prof.mu);
    if (!g_prof.on) return;
    if (begin) {
        if (g_prof.used + 2 > 2 * kMaxPairs) return;
        while (g_prof.ev.size() < g_prof.used + 2) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return;
            g_prof.ev.push_back(e);
        }
        if (cudaEventRecord(g_prof.ev[g_prof.used], s) == cudaSuccess) g_prof.open = true;
    } else if (g_prof.open) {
        if (cudaEventRecord(g_prof.ev[g_prof.used + 1], s) == cudaSuccess) g_prof.used += 2;
        g_prof.open = false;
    }
}

void prof_begin(cudaStream_t s) { prof_record(s, true); }
void prof_end(cudaStream_t s) { prof_record(s, false); }

// Pass 1: block b sums partials [b*chunk, (b+1)*chunk) into tmp[b].
__global__ void __launch_bounds__(256) k_reduce_chunks(const double *__restrict__ partials,
                                                       int64_t count, int64_t chunk,
                                                       double *__restrict__ tmp) {
    __shared__ double red[8];
    const int64_t lo = blockIdx.x * chunk;
    const int64_t hi = lo + chunk < count ? lo + chunk : count;
    double v = 0.0;
    for (int64_t t = lo + threadIdx.x; t < hi; t += 256) v += partials[t];
    v = block_sum_f64<256>(v, red);
    if (threadIdx.x == 0) tmp[blockIdx.x] = v;
}

// Pass 2: one block sums tmp[0 .. slots) into *out.
__global__ void __launch_bounds__(256) k_reduce_final(const double *__restrict__ tmp, int slots,
                                                      double *__restrict__ out) {
    __shared__ double red[8];
    double v = 0.0;
    for (int t = threadIdx.x; t < slots; t += 256) v += tmp[t];
    v = block_sum_f64<256>(v, red);
    if (threadIdx.x == 0) *out = v;
}

// Small counts: one block of 1024 threads sums the partials directly.
__global__ void __launch_bounds__(1024) k_reduce_small(const double *__restrict__ partials,
                                                       int count, double *__restrict__ out) {
    __shared__ double red[32];
    double v = 0.0;
    for (int t = threadIdx.x; t < count; t += 1024) v += partials[t];
    v = block_sum_f64<1024>(v, red);
    if (threadIdx.x == 0) *out = v;
}

int reduce_partials(const double *partials, int64_t count, double *tmp, double *out,
                    cudaStream_t s) {
    if (count <= 65536) {
        k_reduce_small<<<1, 1024, 0, s>>>(partials, (int)count, out);
        note_launches(1);
        return launch_status();
    }
    int64_t chunk = (count + kReduceSlots - 1) / kReduceSlots;
    if (chunk < 1) chunk = 1;
    const int slots = (int)((count + chunk - 1) / chunk);
    k_reduce_chunks<<<slots, 256, 0, s>>>(partials, count, chunk, tmp);
    int st = launch_status();
    if (st) return st;
    k_reduce_final<<<1, 256, 0, s>>>(tmp, slots, out);
    note_launches(2);
    return launch_status();
}

}  // namespace sx

using namespace sx;

extern "C" int simplex_abi_version(void) { return 5; }

extern "C" int simplex_profile(int on) {
    std::lock_guard<std::mutex> lk(g_prof.mu);
    if (on) {
        g_prof.used = 0;
        g_prof.open = false;
        g_launches.store(0);
    }
    g_prof.on = on != 0;
    return SIMPLEX_OK;
}

extern "C" int simplex_profile_read(double *main_ms, int64_t *main_launches,
                                    int64_t *all_launches) {
    std::lock_guard<std::mutex> lk(g_prof.mu);
    double total = 0.0;
    for (size_t t = 0; t + 1 < g_prof.used; t += 2) {
        cudaError_t e = cudaEventSynchronize(g_prof.ev[t + 1]);
        if (e != cudaSuccess) return cuda_status(e);
        float ms = 0.f;
        if ((e = cudaEventElapsedTime(&ms, g_prof.ev[t], g_prof.ev[t + 1])) != cudaSuccess)
            return cuda_status(e);
        total += ms;
    }
    if (main_ms) *main_ms = total;
    if (main_launches) *main_launches = (int64_t)(g_prof.used / 2);
    if (all_launches) *all_launches = g_launches.load();
    return SIMPLEX_OK;
}

extern "C" const char *simplex_strerror(int status) {
    switch (status) {
        case SIMPLEX_OK: return "ok";
        case SIMPLEX_EINVAL: return "invalid argument (size, map, precision or NULL pointer)";
        case SIMPLEX_EALIGN: return "pointer not aligned as required";
        case SIMPLEX_EOVERFLOW: return "size exceeds index or grid limits";
        case SIMPLEX_EUNSUPPORTED: return "request not supported by this library";
        case SIMPLEX_ECUDA: return "CUDA call failed (see simplex_last_cuda_error)";
        case SIMPLEX_EWORKSPACE: return "workspace missing, too small or misaligned";
        case SIMPLEX_ESCRATCH: return "problem too large for the library's static scratch";
        case SIMPLEX_ETIMEOUT: return "a bounded device-side wait ran out";
        default: return "unknown status";
    }
}

extern "C" int simplex_last_cuda_error(void) { return g_last_cuda_error; }

extern "C" int simplex_device_errors(void *stream) {
    cudaStream_t s = (cudaStream_t)stream;
    const int a = umma_device_errors(s);
    const int b = stress_umma_errors(s);
    const int c = atm_device_errors(s);
    return a != SIMPLEX_OK ? a : (b != SIMPLEX_OK ? b : c);
}

extern "C" int simplex_block_rho(int op, int64_t d, int prec) {
    switch (op) {
        case SIMPLEX_OP_MAP2: return 16;
        case SIMPLEX_OP_MAP3: return 8;
        case SIMPLEX_OP_EDM: return edm_rho(d, prec);
        case SIMPLEX_OP_ATM_ENERGY:
        case SIMPLEX_OP_ATM_FORCES: return kAtmRho;
        case SIMPLEX_OP_STRESS_FWD:
        case SIMPLEX_OP_STRESS_BWD:
        case SIMPLEX_OP_STRESS_FWD_BWD: return stress_use_umma(d, prec) ? kStressUmmaRho : kStressRho;
        default: return -1;
    }
}

extern "C" int64_t simplex_workspace_bytes(int op, int64_t n, int64_t d, int map, int prec) {
    if (n < 1 || d < 1 || map < MAP_LAMBDA || map > MAP_RB) return -1;
    // the rectangular box has no 3-simplex form
    const bool m3 = op == SIMPLEX_OP_MAP3 || op == SIMPLEX_OP_ATM_ENERGY || op == SIMPLEX_OP_ATM_FORCES;
    if (m3 && map == MAP_RB) return -1;
    switch (op) {
        case SIMPLEX_OP_MAP2:
        case SIMPLEX_OP_MAP3: return 0;
        case SIMPLEX_OP_EDM: return edm_workspace_bytes(n, d, map, prec);
        case SIMPLEX_OP_ATM_ENERGY: return atm_energy_workspace_bytes(n, map);
        case SIMPLEX_OP_ATM_FORCES: return atm_forces_workspace_bytes(n, map);
        case SIMPLEX_OP_STRESS_FWD: {
            if (stress_use_umma(d, prec)) return stress_umma_workspace_bytes(n, d, false);
            const int64_t nb = (n + kStressRho - 1) / kStressRho;
            const Grid g = grid2(nb, map);
            return 8 * (g.gx * g.gy * g.gz + kReduceSlots);
        }
        case SIMPLEX_OP_STRESS_BWD:
            return stress_use_umma(d, prec) ? stress_umma_workspace_bytes(n, d, true) : 0;
        case SIMPLEX_OP_STRESS_FWD_BWD: {
            if (stress_use_umma(d, prec)) return stress_umma_workspace_bytes(n, d, true);
            const int64_t nb = (n + kStressRho - 1) / kStressRho;
            const Grid g = grid2(nb, map);
            return 8 * (g.gx * g.gy + kReduceSlots);
        }
        default: return -1;
    }
}
