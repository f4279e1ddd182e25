// Guard-band canaries (WAVE2D_CANARY): beyond the ghost cells the one-level
// kernels write (R rings of images; in x up to three more columns, where a
// periodic image is stored as a whole 16-byte vector), every level plane
// holds cells that no kernel of such a handle may write and whose values no
// result depends on: the rest of the ghost ring and the row padding.  (The
// temporal kernels of a zero-boundary handle read them, for nodes outside the
// grid that they force to zero, and write none.)  They are filled with a NaN
// bit pattern; wave2d_canary_check counts cells whose bits changed, a check
// against stray writes into the planes.
#include "wave2d_impl.cuh"

namespace w2d {
namespace {

constexpr uint32_t kCanary32 = 0x7fc0cafeu;
constexpr uint64_t kCanary64 = 0x7ff8cafecafecafeull;

// Plane cell (column c, row r) in storage coordinates; its grid position is
// (c - G, r - G).  A canary cell lies more than R rows or R + 4 columns
// outside the grid.
__device__ __forceinline__ bool is_canary(int c, int r, const Geo& g, int R) {
    const int i = c - g.G, j = r - g.G;
    return i < -R - 4 || i >= g.nx + R + 4 || j < -R || j >= g.ny + R;
}

template <typename W>
__global__ void k_canary(W* plane, Geo g, int R, int rows, W pattern, unsigned long long* changed) {
    const long long n = (long long)g.pitch * rows;
    unsigned long long bad = 0;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(q % g.pitch), r = (int)(q / g.pitch);
        if (!is_canary(c, r, g, R)) continue;
        if (changed) bad += plane[q] != pattern;
        else plane[q] = pattern;
    }
    if (changed && bad) atomicAdd(changed, bad);
}

int for_planes(wave2d* h, unsigned long long* changed) {
    const int grid = 4 * h->num_sms;
    for (int p = 0; p < 4; ++p) {
        for (void* plane : {h->hi[p], h->lo[p]}) {
            if (!plane) continue;
            if (h->elem == 8)
                k_canary<uint64_t><<<grid, 256, 0, h->stream>>>((uint64_t*)plane, h->geo(), h->R, h->rows,
                                                                kCanary64, changed);
            else
                k_canary<uint32_t><<<grid, 256, 0, h->stream>>>((uint32_t*)plane, h->geo(), h->R, h->rows,
                                                                kCanary32, changed);
            W2D_LAUNCHED("canary kernel launch");
        }
    }
    return WAVE2D_OK;
}

}  // namespace

int canary_fill(wave2d* h) {
    if (!(h->flags & WAVE2D_CANARY)) return WAVE2D_OK;
    return for_planes(h, nullptr);
}

}  // namespace w2d

using namespace w2d;

extern "C" int wave2d_canary_check(wave2d_t h, int64_t* changed) {
    if (!h || !changed) return set_error(WAVE2D_ERR_ARG, "null argument");
    if (!(h->flags & WAVE2D_CANARY)) return set_error(WAVE2D_ERR_STATE, "handle was created without WAVE2D_CANARY");
    unsigned long long* d = (unsigned long long*)dev_alloc(h->alloc, 256, h->stream);
    if (!d) return set_error(WAVE2D_ERR_OOM, "canary counter allocation failed");
    unsigned long long host = 0;
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof host, h->stream);
    int rc = e == cudaSuccess ? for_planes(h, d) : cuda_fail(e, "canary counter reset");
    if (rc == WAVE2D_OK) {
        e = cudaMemcpyAsync(&host, d, sizeof host, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) rc = cuda_fail(e, "canary check");
    }
    dev_free(h->alloc, d, 256, h->stream);
    if (rc == WAVE2D_OK) *changed = (int64_t)host;
    return rc;
}
