// Arithmetic throughput of the GPU the library runs on: the denominators of
// the ALU rooflines (FP32 lane operations for the temporally blocked FP32
// kernels, FP64 for the FP64 path).
//
// Each probe keeps K independent dependency chains per thread, so the pipe,
// not the latency of one chain, sets the rate; the grid holds 4 blocks of 512
// threads per SM.  A lane operation is one add or one fused multiply-add of
// one lane (a packed f32x2 instruction counts two).  Best of five timed
// launches after three warm-up launches, CUDA events on the caller's stream.
#include <algorithm>
#include <cstring>

#include "wave2d_impl.cuh"

namespace w2d {
namespace {

constexpr int kChains = 8;
constexpr int kThreads = 512;
constexpr int kBlocksPerSm = 4;
constexpr int kIters = 1 << 14;

__global__ void __launch_bounds__(kThreads) k_peak_ffma(float* out, int iters, float a, float b) {
    float x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = threadIdx.x * 1e-3f + k;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int k = 0; k < kChains; ++k) x[k] = __fmaf_rn(x[k], a, b);
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) k_peak_ffma2(float* out, int iters, float a, float b) {
    f2x x[kChains];
    const f2x aa = pk2(a, a), bb = pk2(b, b);
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = pk2(threadIdx.x * 1e-3f + k, threadIdx.x * 1e-3f + k + 0.5f);
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int k = 0; k < kChains; ++k) x[k] = fma2(x[k], aa, bb);
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
        float lo, hi;
        upk2(x[k], lo, hi);
        s += lo + hi;
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) k_peak_fadd(float* out, int iters, float a, float b) {
    float x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = threadIdx.x * 1e-3f + k;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int k = 0; k < kChains; ++k) x[k] = __fadd_rn(x[k], (k & 1) ? a : b);
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) k_peak_dfma(double* out, int iters, double a, double b) {
    double x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = threadIdx.x * 1e-3 + k;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int k = 0; k < kChains; ++k) x[k] = __fma_rn(x[k], a, b);
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace w2d

using namespace w2d;

extern "C" int wave2d_alu_peaks(wave2d_alu_peaks_t* out, void* stream_ptr) {
    NvtxRange nvtx_range("wave2d_alu_peaks");
    if (!out) return set_error(WAVE2D_ERR_ARG, "null argument");
    std::memset(out, 0, sizeof *out);
    cudaStream_t st = static_cast<cudaStream_t>(stream_ptr);
    int dev = 0, sms = 0, clk = 0;
    W2D_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    W2D_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "device attribute");
    W2D_CUDA(cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev), "device attribute");
    const int blocks = sms * kBlocksPerSm;
    const size_t bytes = (size_t)blocks * kThreads * sizeof(double);
    const Allocator al = current_allocator();
    void* buf = dev_alloc(al, bytes, st);
    if (!buf) return set_error(WAVE2D_ERR_OOM, "peak probe buffer allocation failed");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = WAVE2D_OK;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        rc = set_error(WAVE2D_ERR_CUDA, "event create failed");
    // time one probe: best of 5 launches after 3 warm-ups; lane operations per second
    auto probe = [&](auto launch, double lane_ops_per_thread) -> double {
        if (rc != WAVE2D_OK) return 0.0;
        for (int w = 0; w < 3; ++w) launch();
        float best = 0.0f;
        for (int r = 0; r < 5; ++r) {
            cudaEventRecord(e0, st);
            launch();
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                rc = cuda_fail(cudaGetLastError(), "peak probe");
                return 0.0;
            }
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (r == 0 || ms < best) best = ms;
        }
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "peak probe launch");
            return 0.0;
        }
        return (double)blocks * kThreads * lane_ops_per_thread / (best * 1e-3);
    };
    float* f = static_cast<float*>(buf);
    double* d = static_cast<double*>(buf);
    out->fp32_fma = probe([&] { k_peak_ffma<<<blocks, kThreads, 0, st>>>(f, kIters, 0.999f, 1e-3f); },
                          (double)kIters * kChains);
    out->fp32_fma2 = probe([&] { k_peak_ffma2<<<blocks, kThreads, 0, st>>>(f, kIters, 0.999f, 1e-3f); },
                           2.0 * kIters * kChains);
    out->fp32_add = probe([&] { k_peak_fadd<<<blocks, kThreads, 0, st>>>(f, kIters, 0.999f, 1e-3f); },
                          (double)kIters * kChains);
    // FP64 runs at a small fraction of the FP32 rate on GB300: 1/16 of the iterations
    out->fp64_fma = probe([&] { k_peak_dfma<<<blocks, kThreads, 0, st>>>(d, kIters / 16, 0.999, 1e-3); },
                          (double)(kIters / 16) * kChains);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    dev_free(al, buf, bytes, st);
    out->sms = sms;
    out->clock_khz = clk;
    return rc;
}
