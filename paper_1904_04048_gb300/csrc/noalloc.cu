// Allocation-free FP64 error norms of a caller-owned field.
//
// Same reduction as wave2d_error_vs_exact (kernels.cuh: exact_at,
// error_terms, reduce_finalize), but every piece of scratch it needs -- the
// per-block partial sums, the finishing counter, the result slots, the
// status word and the separable exact-solution tables -- lives in one
// file-scope __device__ array instead of memory allocated by a handle.  Every
// GPU that loads the library holds this array (kNoAllocScratchBytes) until
// the process exits.
#include <cmath>
#include <cstring>
#include <mutex>

#include "wave2d_impl.cuh"

namespace w2d {
namespace {

constexpr int kNoAllocMaxN = 8192;  // largest nx and ny accepted
constexpr int kBlocksX = 16, kBlocksY = 128;
constexpr size_t kPartials = 4 * (size_t)kBlocksX * kBlocksY;  // doubles
constexpr size_t kMisc = 32;                                   // acc[4], counter, status
constexpr size_t kTables = 4 * (size_t)kNoAllocMaxN;           // P, R (nx) and Q, S (ny)
constexpr size_t kScratchDoubles = kPartials + kMisc + kTables;
constexpr size_t kNoAllocScratchBytes = kScratchDoubles * sizeof(double);

// Shared by every call on a device; the contents persist between calls.
__device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (cudaGetSymbolAddress) and cached.
int scratch_address(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return set_error(WAVE2D_ERR_ARG, "device index %d not supported", dev);
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-allocation scratch)");
        g_addr[dev] = static_cast<double*>(p);
    }
    *out = g_addr[dev];
    return WAVE2D_OK;
}

// Separable exact-solution tables (the layout of ExactTab in kernels.cuh),
// evaluated on the device so the call needs no host staging buffer.
__global__ void k_noalloc_tables(double* tab, int nx, int ny, double h, double x_off, int kind, double m,
                                 double k1, double k2) {
    const double pi = 3.14159265358979323846;
    double* P = tab;
    double* R = P + nx;
    double* Q = R + nx;
    double* S = Q + ny;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nx + ny; q += gridDim.x * blockDim.x) {
        const bool isx = q < nx;
        const int i = isx ? q : q - nx;
        const double x = (i + x_off) * h;
        double a = 0.0, b = 0.0;
        if (kind == WAVE2D_EXACT_STANDING) {
            a = sin(2.0 * pi * m * x);
        } else if (kind == WAVE2D_EXACT_PLANE) {
            const double k = isx ? k1 : k2;
            a = cos(k * x);
            b = sin(k * x);
        }
        if (isx) {
            P[i] = a;
            R[i] = b;
        } else {
            Q[i] = a;
            S[i] = b;
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k4_norms_plain(const T* __restrict__ u, int nx, int ny, long long ld,
                                                      ExactTab ex, Reduce rd) {
    double s0 = 0, s1 = 0, m0 = 0, m1 = 0;
    for (int j = blockIdx.y; j < ny; j += gridDim.y)
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nx; i += gridDim.x * blockDim.x)
            error_terms((double)u[(size_t)j * ld + i], exact_at(ex, i, j), s0, s1, m0, m1, rd.status);
    reduce_finalize<256>(s0, s1, m0, m1, rd);
}

}  // namespace
}  // namespace w2d

using namespace w2d;

extern "C" int wave2d_error_norms_noalloc(const void* field, int dtype, int nx, int ny, int64_t ld, double h,
                                          double c, double t, const wave2d_exact* ex, double* rel_l2,
                                          double* rel_linf, void* stream) {
    if (!field) return set_error(WAVE2D_ERR_ARG, "null field");
    if (dtype != WAVE2D_F32 && dtype != WAVE2D_F64)
        return set_error(WAVE2D_ERR_ARG, "no-allocation norms take an F32 or F64 field (got dtype %d)", dtype);
    if (nx < 1 || ny < 1 || nx > kNoAllocMaxN || ny > kNoAllocMaxN)
        return set_error(WAVE2D_ERR_ARG,
                         "no-allocation norms: grid %d x %d outside 1..%d per side (fixed scratch of %zu bytes)",
                         nx, ny, kNoAllocMaxN, kNoAllocScratchBytes);
    if (ld < nx) return set_error(WAVE2D_ERR_ARG, "row stride %lld is smaller than nx %d", (long long)ld, nx);
    if (!(h > 0) || !(c > 0) || !std::isfinite(h) || !std::isfinite(c) || !std::isfinite(t))
        return set_error(WAVE2D_ERR_ARG, "h and c must be positive and finite, t finite");
    wave2d_exact none{};
    if (!ex) ex = &none;
    if ((ex->kind != WAVE2D_EXACT_NONE && ex->kind != WAVE2D_EXACT_STANDING && ex->kind != WAVE2D_EXACT_PLANE) ||
        !std::isfinite(ex->amp) || !std::isfinite(ex->m) || !std::isfinite(ex->k1) || !std::isfinite(ex->k2) ||
        !std::isfinite(ex->x_off))
        return set_error(WAVE2D_ERR_ARG, "invalid exact-solution description");

    double* base = nullptr;
    int rc = scratch_address(&base);
    if (rc != WAVE2D_OK) return rc;
    double* partials = base;
    double* acc = base + kPartials;
    unsigned* counter = reinterpret_cast<unsigned*>(acc + 4);
    int* status = reinterpret_cast<int*>(acc + 5);
    double* tab = base + kPartials + kMisc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    // The counter and status word must start at zero; earlier calls leave
    // the counter at zero, but a call cut short would not.
    cudaError_t e = cudaMemsetAsync(acc, 0, kMisc * sizeof(double), s);
    if (e != cudaSuccess) return cuda_fail(e, "scratch reset");

    ExactTab et{};
    et.kind = ex->kind;
    et.P = tab;
    et.R = tab + nx;
    et.Q = tab + 2 * (size_t)nx;
    et.S = tab + 2 * (size_t)nx + ny;
    const double pi = 3.14159265358979323846;
    if (ex->kind == WAVE2D_EXACT_STANDING) {
        et.w0 = ex->amp * std::sin(2.0 * std::sqrt(2.0) * pi * ex->m * c * t);
    } else if (ex->kind == WAVE2D_EXACT_PLANE) {
        const double w = c * std::sqrt(ex->k1 * ex->k1 + ex->k2 * ex->k2);
        et.w0 = ex->amp * std::cos(w * t);
        et.w1 = ex->amp * std::sin(w * t);
    }
    if (ex->kind != WAVE2D_EXACT_NONE) {
        k_noalloc_tables<<<(nx + ny + 255) / 256, 256, 0, s>>>(tab, nx, ny, h, ex->x_off, ex->kind, ex->m, ex->k1,
                                                                ex->k2);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "no-allocation table kernel launch");
        g_launches.fetch_add(1);
    }
    const Reduce rd{partials, counter, acc, status, 0};
    const dim3 grd(std::min((nx + 255) / 256, kBlocksX), std::min(ny, kBlocksY));
    if (dtype == WAVE2D_F32)
        k4_norms_plain<float><<<grd, 256, 0, s>>>(static_cast<const float*>(field), nx, ny, (long long)ld, et, rd);
    else
        k4_norms_plain<double><<<grd, 256, 0, s>>>(static_cast<const double*>(field), nx, ny, (long long)ld, et, rd);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "no-allocation norm kernel launch");
    g_launches.fetch_add(1);

    double res[6];
    e = cudaMemcpyAsync(res, acc, sizeof res, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "no-allocation norm result copy");
    int st = 0;
    std::memcpy(&st, &res[5], sizeof st);
    if (ex->kind == WAVE2D_EXACT_NONE) {
        if (rel_l2) *rel_l2 = std::sqrt(res[0]);
        if (rel_linf) *rel_linf = res[2];
    } else {
        if (rel_l2) *rel_l2 = std::sqrt(res[0] / res[1]);
        if (rel_linf) *rel_linf = res[2] / res[3];
    }
    if (st & STATUS_NONFINITE) return set_error(WAVE2D_ERR_NONFINITE, "the field contains NaN or Inf");
    return WAVE2D_OK;
}
