// Internal host-side definitions shared by the library's translation units.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <string>
#include <type_traits>

#include <nvtx3/nvToolsExt.h>

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

// NVTX range around a library call (visible to profilers that record NVTX,
// e.g. ncu --nvtx --nvtx-include "wave2d_step_n/"); costs nothing without one.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

inline size_t round_up(size_t v, size_t m) { return (v + m - 1) / m * m; }

#define W2D_CUDA(call, what)                                   \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return w2d::cuda_fail(e_, what); \
    } while (0)

#define W2D_LAUNCHED(what)                                         \
    do {                                                           \
        cudaError_t e_ = cudaGetLastError();                       \
        if (e_ != cudaSuccess) return w2d::cuda_fail(e_, what);     \
        w2d::g_launches.fetch_add(1, std::memory_order_relaxed);   \
    } while (0)

}  // namespace w2d

struct wave2d {
    // problem
    int nx = 0, ny = 0, bc = 0, dtype = 0, flags = 0, scheme = 0, R = 1;
    double h = 0, tau = 0, c = 0, lam = 0, lam_max = 0;
    double a[3] = {0, 0, 0}, b[3] = {0, 0, 0};
    // derived schemes: number of classes of the chain in use (0 for the
    // Section 6 schemes), stencil nodes, and the class coefficients at lambda
    int nclass = 0, npoints = 0;
    double ca[8] = {}, cb[8] = {};
    bool diff_sums = false;  // WAVE2D_DIFF_SUMS: class sums from differences to the centre
    bool diff_form = false;  // WAVE2D_DIFF_FORM: planes u^k (cur), scratch (prv), d^k (dpl)
    int dpl = 2;             // difference form: plane of d^k (2 or 3; the streaming kernel alternates them)
    // device
    int device = 0, num_sms = 0, l2_bytes = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    w2d::Allocator alloc;
    int G = w2d::kGhost, pitch = 0, rows = 0;
    size_t elem = 0, plane_bytes = 0;
    void* base = nullptr;
    size_t base_bytes = 0;
    void* hi[4] = {nullptr, nullptr, nullptr, nullptr};  // level planes (hi parts)
    void* lo[4] = {nullptr, nullptr, nullptr, nullptr};  // lo parts (FP32x2 only)
    int nlevels = 2;  // 4 for FP32: a second pair for the out-of-place temporal kernel
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
    int cur = 0, prv = 1;  // planes holding u^k and u^{k-1}
    int gw = 1;            // periodic image rings kept valid by every writer
    bool rings_stale = false;  // streaming launches left the current rings unwritten (see stream.cu)
    int64_t k = 0;
    bool initialized = false;
    bool tracking = false;
    wave2d_exact track_ex{};
    // tuning
    wave2d_tune tune{};
    int kernel = WAVE2D_KERNEL_SIMPLE;
    int tile_h = 32;
    int temporal_t = 4, temporal_oh = 64;  // levels per launch and output rows per tile
    // TMA descriptors per plane: u^k halo box and u^{k-1} tile box of the
    // one-step kernel; region box of the temporal kernel (for reg_key)
    CUtensorMap tm_cur[4], tm_prev[4], tm_reg[4];
    bool tma_ready = false;
    int reg_key = -1;
    // captured runs of steps, keyed by the starting (cur, prv) planes
    cudaGraphExec_t graph[32] = {};
    int graph_end[32] = {};  // plane state after a replay, as plane_key()
    // (cur, prv, dpl) as one index: the key of a captured graph
    int plane_key() const { return (dpl & 1) * 16 + cur * 4 + prv; }
    void set_plane_key(int key) {
        dpl = 2 + key / 16;
        cur = key % 16 / 4;
        prv = key % 4;
    }
    int graph_steps = 0;

    w2d::Level level(int p) const { return w2d::Level{hi[p], lo[p]}; }
    w2d::Geo geo() const { return w2d::Geo{nx, ny, pitch, G}; }
};

namespace w2d {
// Derived schemes and difference sums (chain.cu, chain_tma.cu): launches of
// the class-chain kernels for a handle with nclass > 0.
int chain_first_step(wave2d* h, const double* du0, const double* dv0, const ExactTab& ex, const Reduce& rd);
int chain_simple_step(wave2d* h, bool track, const ExactTab& ex, const Reduce& rd);
int chain_tma_step(wave2d* h);
void chain_tma_box(const wave2d* h, int& box_w, int& box_h, int& tile_w, int& tile_h);
// Register-streaming temporal kernel (stream.cu): T levels of a handle whose
// kernel is WAVE2D_KERNEL_STREAM, out of place into the other pair of planes.
// On periodic grids it may leave the current levels' ghost rings stale
// (rings_stale); stream_fresh_rings rebuilds them and must run before any
// other kernel reads the planes' rings and before a library call returns.
int stream_launch(wave2d* h);
// One two-step of a double-float (FP32x2) Section 6 handle, two nodes per
// thread in packed arithmetic (df2.cu); equal to k2_simple's result.
int df2_simple_step(wave2d* h, const Coef3<df>& a);
int stream_fresh_rings(wave2d* h);
// Guard-band canaries (canary.cu): fill the untouched cells of every plane
// when the handle has WAVE2D_CANARY.
int canary_fill(wave2d* h);
// Server support (batch.cu, wave2d.cu): replace a batch's members keeping its
// streams and tuning; batched norms copied to pinned host memory without a
// wait; release a handle in stream order without a wait.
int batch_set_handles(wave2d_batch* b, wave2d_t* handles, int n, int rows = 0);
int batch_norms_async(wave2d* const* hs, int n, cudaStream_t st, const Allocator& al, double* host_out);
void release_handle_nosync(wave2d* h);
// Derivation and stability limit (scheme.cu).
int derive_scheme(int m, wave2d_scheme* out);
int check_scheme(const wave2d_scheme* s);
double poly_at(const double* c, double lam);
double scheme_lambda_max(const wave2d_scheme* s);
}  // namespace w2d
