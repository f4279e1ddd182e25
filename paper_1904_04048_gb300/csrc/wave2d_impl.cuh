// Internal host-side definitions shared by the library's translation units.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <string>
#include <type_traits>

#include "../../include/wave2d.h"
#include "kernels.cuh"

namespace w2d {

// -------------------------------------------------------------- errors
int set_error(int code, const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);

// -------------------------------------------------------------- allocation
struct Allocator {
    wave2d_alloc_fn alloc = nullptr;
    wave2d_free_fn release = nullptr;
    void* ctx = nullptr;
};
Allocator current_allocator();
void* dev_alloc(const Allocator& a, size_t bytes, cudaStream_t s);
void dev_free(const Allocator& a, void* p, size_t bytes, cudaStream_t s);

extern std::atomic<int64_t> g_launches;

constexpr int kGhost = 16;  // ghost ring width (elements) on every side

inline size_t round_up(size_t v, size_t m) { return (v + m - 1) / m * m; }

}  // namespace w2d

struct wave2d {
    // problem
    int nx = 0, ny = 0, bc = 0, dtype = 0, flags = 0, scheme = 0, R = 1;
    double h = 0, tau = 0, c = 0, lam = 0, lam_max = 0;
    double a[3] = {0, 0, 0}, b[3] = {0, 0, 0};
    // device
    int device = 0, num_sms = 0, l2_bytes = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    w2d::Allocator alloc;
    int G = w2d::kGhost, pitch = 0, rows = 0;
    size_t elem = 0, plane_bytes = 0;
    void* base = nullptr;
    size_t base_bytes = 0;
    void* hi[2] = {nullptr, nullptr};
    void* lo[2] = {nullptr, nullptr};
    // scratch
    double* partials = nullptr;
    size_t partial_blocks = 0;
    unsigned* counter = nullptr;
    double* acc_eval = nullptr;   // 4 doubles, error_vs_exact
    double* acc_track = nullptr;  // 4 doubles, space-time accumulation
    int* status = nullptr;
    double* tab_eval = nullptr;   // 2 nx + 2 ny doubles
    double* tab_track = nullptr;  // 2 nx + 2 ny doubles
    // state
    int cur = 0;  // plane holding u^k
    int64_t k = 0;
    bool initialized = false;
    bool tracking = false;
    wave2d_exact track_ex{};
    // tuning
    wave2d_tune tune{};
    int kernel = WAVE2D_KERNEL_SIMPLE;
    int tile_h = 32;
    // TMA descriptors: [plane] for u^k (halo box) and u^{k-1} (tile box)
    CUtensorMap tm_cur[2], tm_prev[2];
    bool tma_ready = false;
    // graph of an even number of steps per starting parity
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int graph_steps = 0;

    w2d::Level level(int p) const { return w2d::Level{hi[p], lo[p]}; }
    w2d::Geo geo() const { return w2d::Geo{nx, ny, pitch, G}; }
};
