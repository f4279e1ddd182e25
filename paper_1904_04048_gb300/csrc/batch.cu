// Batched time stepping of many independent simulations of different sizes,
// schemes, Courant numbers and step counts (FP32 storage).
//
// A run advances instance i by steps[i] levels in quanta of Tq levels.  The
// instances are ordered by decreasing step count, so the instances still
// running at quantum q are a prefix of that order, and one launch per quantum
// covers the tiles of all of them: block b finds its instance by binary
// search over the tiles' prefix sums.  Every block stages its tile's region
// with TMA and advances it min(Tq, levels left) levels in shared memory with
// the same per-node arithmetic as the single-grid kernels (region_advance,
// region_store), so every instance ends bit for bit where it would alone.
// The sequence of quanta is captured once in a CUDA graph and replayed.
// Levels alternate between the two pairs of planes of each handle (plane
// p -> p ^ 2 per quantum), exactly as the single-grid temporal kernel does.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <type_traits>
#include <vector>

#include "kernels_stream.cuh"
#include "kernels_temporal.cuh"
#include "wave2d_impl.cuh"

namespace w2d {

constexpr int kBatchRVW = 64;  // region width in 16-byte vectors
constexpr int kBatchNW = 8;    // warps per CTA

struct BatchInst {
    const CUtensorMap* tm;  // region maps of the four planes (global memory)
    float* planes[4];
    Geo g;
    Coef3<float> a;
    int scheme;
    int cur0, prv0;  // planes of u^k and u^{k-1} when the run starts
    int tiles_x;
    int rh;          // rows of this instance's region box
    long long steps; // levels to advance in this run
};

template <int S, bool PER>
__device__ __forceinline__ void batch_advance(float* Q, float* P, int Ti, int rh, int gx0, int gy0, const Geo& g,
                                              const Coef3<float>& a) {
    // the lane widths of the single-grid temporal kernel: two columns per lane
    // for radius-1 schemes, four for the 13-point scheme
    auto adv = [&](auto Tc) {
        constexpr int TT = decltype(Tc)::value;
        if constexpr (S == 13) region_advance<S, PER, kBatchRVW, TT, kBatchNW>(Q, P, rh, gx0, gy0, g, a);
        else region_advance2<S, PER, kBatchRVW, TT, kBatchNW>(Q, P, rh, gx0, gy0, g, a);
    };
    switch (Ti) {
        case 1: adv(std::integral_constant<int, 1>{}); break;
        case 2: adv(std::integral_constant<int, 2>{}); break;
        case 3: adv(std::integral_constant<int, 3>{}); break;
        default: adv(std::integral_constant<int, 4>{}); break;
    }
}

template <bool PER>
__global__ void __launch_bounds__(kBatchNW * 32, 1)
    k6_batch_step(const BatchInst* __restrict__ insts, const int* __restrict__ tile_prefix, int n_active, int q,
                  int Tq, int OH, int gw, int* status) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
    float* Q = reinterpret_cast<float*>(smem_raw + 1024);
    const int tid = threadIdx.x;
    const int b = blockIdx.x;
    int lo = 0, hi = n_active;  // tile_prefix[lo] <= b < tile_prefix[lo + 1]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(tile_prefix + mid) <= b) lo = mid;
        else hi = mid;
    }
    const BatchInst& I = insts[lo];
    const Geo g = I.g;
    const int rh = I.rh;
    float* P = Q + 4 * kBatchRVW * rh;
    const int local = b - __ldg(tile_prefix + lo);
    const int tx = local % I.tiles_x, ty = local / I.tiles_x;
    const int Ti = (int)min((long long)Tq, I.steps - (long long)Tq * q);
    const int par = (q & 1) * 2;
    const int in_cur = I.cur0 ^ par, in_prv = I.prv0 ^ par;
    const int R = (I.scheme == 13) ? 2 : 1;
    const int OWV = kBatchRVW - 2 * Tq, OW = 4 * OWV, HY = R * Tq;
    const int gx0 = tx * OW - 4 * Tq, gy0 = ty * OH - HY;

    if (tid == 0) {
        mbar_init(bar, 1);
        fence_barrier_init();
        fence_proxy_async_smem();
    }
    __syncthreads();
    if (tid == 0) {
        mbar_arrive_expect_tx(bar, 2u * (unsigned)(4 * kBatchRVW * rh * 4));
        tma_load_2d(Q, I.tm + in_cur, bar, g.G + gx0, g.G + gy0);
        tma_load_2d(P, I.tm + in_prv, bar, g.G + gx0, g.G + gy0);
    }
    const bool ok = mbar_wait_bounded(bar, 0, status);
    if (!__syncthreads_and(ok)) {
        if (tid == 0) mbar_wait_bounded(bar, 0, status);
        return;
    }
    const Coef3<float> a = I.a;
    switch (I.scheme) {
        case 5: batch_advance<5, PER>(Q, P, Ti, rh, gx0, gy0, g, a); break;
        case 9: batch_advance<9, PER>(Q, P, Ti, rh, gx0, gy0, g, a); break;
        default: batch_advance<13, PER>(Q, P, Ti, rh, gx0, gy0, g, a); break;
    }
    const bool edge = PER && (tx * OW < gw || tx * OW + OW > g.nx - gw || ty * OH < gw || ty * OH + OH > g.ny - gw);
    region_store<PER, kBatchRVW, kBatchNW>((Ti & 1) ? P : Q, (Ti & 1) ? Q : P, HY, OH, Tq, OWV, gx0, gy0, g,
                                           I.planes[in_cur ^ 2], I.planes[in_prv ^ 2], gw, edge);
}

// Register-streaming batch (zero boundary): one warp per strip, over the
// strips of all instances of one scheme in a launch.  Warp w finds its
// instance by binary search over the strips' prefix sums and walks that
// instance's strip exactly as the single-grid streaming kernel does
// (stream_strip), T levels out of place into the other pair of planes; the
// pairs alternate with the launch's parity q.
struct StreamInst {
    float* planes[4];
    Geo g;
    Coef3<float> a;
    int cur0, prv0;  // planes of u^k and u^{k-1} at the instance's launch of parity 0
    int strips_x;
};

template <int S, int T>
__global__ void __launch_bounds__(kBatchStreamWarps * 32)
    k7_batch_stream(const StreamInst* __restrict__ insts, const int* __restrict__ strip_prefix, int n_active, int q,
                    int L) {
    constexpr int NB = StreamCfg<S, T>::NB;
    extern __shared__ float4 stream_smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int strip = blockIdx.x * kBatchStreamWarps + warp;
    if (strip >= __ldg(strip_prefix + n_active)) return;  // whole warps only
    int lo = 0, hi = n_active;  // strip_prefix[lo] <= strip < strip_prefix[lo + 1]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(strip_prefix + mid) <= strip) lo = mid;
        else hi = mid;
    }
    const StreamInst& I = insts[lo];
    const int par = (q & 1) * 2;
    const int ic = I.cur0 ^ par, ip = I.prv0 ^ par;
    stream_strip<S, false, T, false>(I.planes[ic], I.planes[ip], I.planes[ic ^ 2], I.planes[ip ^ 2], I.g, I.a,
                                     I.strips_x, strip - __ldg(strip_prefix + lo), L,
                                     stream_smem + warp * NB * 2 * 32, lane);
}

// Batched first step (Eq. A1): one node per thread, blocks of 32 x 8 nodes
// mapped to instances through prefix sums.
struct BatchFirst {
    const double* u0;
    const double* v0;
    float* plane0;  // receives u^1 (plane 0)
    float* plane1;  // receives u^0 (plane 1)
    Geo g;
    Coef3<double> ahalf, b;
    double tau;
    int scheme;
    int blocks_x;
};

template <int S, bool PER>
__device__ __forceinline__ void batch_first_node(const BatchFirst& F, int i, int j, int gw) {
    const Nbr<double> u = gather_bc(F.u0, F.g.nx, F.g.ny, PER, i, j);
    const Nbr<double> v = gather_bc(F.v0, F.g.nx, F.g.ny, PER, i, j);
    const double u1 = first_step_update<S>(u, v, F.ahalf, F.b, F.tau);
    const size_t o = off(F.g, i, j);
    const float q0 = __double2float_rn(u.c), q1 = __double2float_rn(u1);
    F.plane1[o] = q0;
    F.plane0[o] = q1;
    if (PER) {
        write_images<DT_F32>(Level{F.plane1, nullptr}, F.g, i, j, q0, gw);
        write_images<DT_F32>(Level{F.plane0, nullptr}, F.g, i, j, q1, gw);
    }
}

template <bool PER>
__global__ void __launch_bounds__(256) k6_batch_first(const BatchFirst* __restrict__ fs, const int* __restrict__ prefix,
                                                      int n, int gw) {
    const int b = blockIdx.x;
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(prefix + mid) <= b) lo = mid;
        else hi = mid;
    }
    const BatchFirst& F = fs[lo];
    const int local = b - __ldg(prefix + lo);
    const int i = (local % F.blocks_x) * 32 + threadIdx.x, j = (local / F.blocks_x) * 8 + threadIdx.y;
    if (i >= F.g.nx || j >= F.g.ny) return;
    switch (F.scheme) {
        case 5: batch_first_node<5, PER>(F, i, j, gw); break;
        case 9: batch_first_node<9, PER>(F, i, j, gw); break;
        default: batch_first_node<13, PER>(F, i, j, gw); break;
    }
}

// Batched FP64 norms of the current level: per block partial sums of u^2 and
// max |u| over 8 rows, then one block per instance reduces them in order.
struct BatchNorm {
    const float* plane;
    Geo g;
    int blocks;  // row chunks of 8
    int first;   // index of its first partial
};

__global__ void __launch_bounds__(256) k6_batch_norm_partial(const BatchNorm* __restrict__ ns, const int* __restrict__ prefix,
                                                             int n, double* partials) {
    const int b = blockIdx.x;
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(prefix + mid) <= b) lo = mid;
        else hi = mid;
    }
    const BatchNorm& B = ns[lo];
    const int chunk = b - __ldg(prefix + lo);
    double s = 0, m = 0;
    for (int j = chunk * 8; j < min(chunk * 8 + 8, B.g.ny); ++j)
        for (int i = threadIdx.x; i < B.g.nx; i += blockDim.x) {
            const double v = (double)B.plane[off(B.g, i, j)];
            s = __fma_rn(v, v, s);
            m = fmax(m, fabs(v));
        }
    __shared__ double sh[2][8];
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    }
    if ((threadIdx.x & 31) == 0) {
        sh[0][threadIdx.x >> 5] = s;
        sh[1][threadIdx.x >> 5] = m;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, c = 0;
        for (int w = 0; w < 8; ++w) {
            a += sh[0][w];
            c = fmax(c, sh[1][w]);
        }
        partials[2 * (size_t)(B.first + chunk)] = a;
        partials[2 * (size_t)(B.first + chunk) + 1] = c;
    }
}

__global__ void k6_batch_norm_final(const BatchNorm* __restrict__ ns, const double* __restrict__ partials, double* out) {
    const BatchNorm& B = ns[blockIdx.x];
    if (threadIdx.x != 0) return;
    double s = 0, m = 0;
    for (int c = 0; c < B.blocks; ++c) {
        s += partials[2 * (size_t)(B.first + c)];
        m = fmax(m, partials[2 * (size_t)(B.first + c) + 1]);
    }
    out[2 * blockIdx.x] = std::sqrt(s);
    out[2 * blockIdx.x + 1] = m;
}

}  // namespace w2d

using namespace w2d;

struct wave2d_batch {
    std::vector<wave2d*> hs;
    cudaStream_t stream = nullptr;
    Allocator alloc;
    int bc = 0;
    int Tq = 4, OH = 32;
    int num_sms = 0;
    // device tables (one allocation, rebuilt per plan)
    void* dev = nullptr;
    size_t dev_bytes = 0;
    // plan of the last run
    std::vector<int64_t> plan_steps;
    std::vector<int> plan_start;  // cur * 4 + prv of every handle when the plan was built
    std::vector<int> order;
    cudaGraphExec_t graph = nullptr;
    int graph_launches = 0;
    int plan_Tq = 0, plan_OH = 0;
    cudaEvent_t ev = nullptr;  // stream ordering with the members
    bool direct = false;       // launch the quanta directly instead of capturing a graph
    std::vector<int> plan_grids, plan_active;
    const void* plan_insts = nullptr;
    const int* plan_prefix = nullptr;
    int plan_smem = 0;
    // register-streaming runs (WAVE2D_KERNEL_STREAM, zero boundary): one
    // branch of launches per scheme on its own stream, forked from and joined
    // to the batch stream
    int kernel = WAVE2D_KERNEL_TEMPORAL;
    int plan_kernel = 0;
    struct SLaunch {
        int scheme, T, grid, n_active, q, branch;
        const void* insts;
        const int* prefix;
    };
    std::vector<SLaunch> plan_slaunches;
    cudaStream_t side[3] = {};
    cudaEvent_t ev_fork = nullptr, ev_join[3] = {};
};

namespace {

// Order the batch stream after every member's stream (join) and every
// member's stream after the batch stream (release), so batch calls and
// single-handle calls on other streams never overlap.
int order_streams(wave2d_batch* b, bool join) {
    for (wave2d* h : b->hs) {
        if (h->stream == b->stream) continue;
        cudaStream_t from = join ? h->stream : b->stream, to = join ? b->stream : h->stream;
        cudaError_t e = cudaEventRecord(b->ev, from);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(to, b->ev, 0);
        if (e != cudaSuccess) return cuda_fail(e, "stream ordering");
    }
    return WAVE2D_OK;
}

void free_plan(wave2d_batch* b) {
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    if (b->dev) {
        dev_free(b->alloc, b->dev, b->dev_bytes, b->stream);
        b->dev = nullptr;
        b->dev_bytes = 0;
    }
    b->plan_steps.clear();
    b->plan_slaunches.clear();
}

int encode_region(CUtensorMap* tm, void* plane, const wave2d* h, int rh) {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return set_error(WAVE2D_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
        fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    const cuuint64_t dims[2] = {(cuuint64_t)h->pitch, (cuuint64_t)h->rows};
    const cuuint64_t strides[1] = {(cuuint64_t)h->pitch * 4};
    const cuuint32_t box[2] = {(cuuint32_t)(4 * kBatchRVW), (cuuint32_t)rh};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, plane, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(WAVE2D_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return WAVE2D_OK;
}

int region_rows(int scheme, int OH, int Tq) { return OH + 2 * ((scheme == 13) ? 2 : 1) * Tq; }

// Build the tables of a run and capture its quanta in a graph.
int build_plan(wave2d_batch* b, const int64_t* steps) {
    free_plan(b);
    const int n = (int)b->hs.size();
    b->order.resize(n);
    std::iota(b->order.begin(), b->order.end(), 0);
    std::stable_sort(b->order.begin(), b->order.end(), [&](int x, int y) { return steps[x] > steps[y]; });
    const int Tq = b->Tq, OH = b->OH;
    const int OW = 4 * (kBatchRVW - 2 * Tq);
    std::vector<BatchInst> insts(n);
    std::vector<int> prefix(n + 1, 0);
    std::vector<CUtensorMap> maps(4 * (size_t)n);
    for (int r = 0; r < n; ++r) {
        wave2d* h = b->hs[b->order[r]];
        BatchInst& I = insts[r];
        I.g = h->geo();
        I.a = Coef3<float>{(float)h->a[0], (float)h->a[1], (float)h->a[2]};
        I.scheme = h->scheme;
        I.cur0 = h->cur;
        I.prv0 = h->prv;
        I.tiles_x = (h->nx + OW - 1) / OW;
        I.rh = region_rows(h->scheme, OH, Tq);
        I.steps = steps[b->order[r]];
        for (int p = 0; p < 4; ++p) {
            I.planes[p] = reinterpret_cast<float*>(h->hi[p]);
            int rc = encode_region(&maps[4 * (size_t)r + p], h->hi[p], h, I.rh);
            if (rc != WAVE2D_OK) return rc;
        }
        prefix[r + 1] = prefix[r] + I.tiles_x * ((h->ny + OH - 1) / OH);
    }
    // device layout: maps (64-byte aligned), insts, prefix
    const size_t maps_bytes = round_up(maps.size() * sizeof(CUtensorMap), 256);
    const size_t insts_bytes = round_up(insts.size() * sizeof(BatchInst), 256);
    const size_t prefix_bytes = round_up(prefix.size() * sizeof(int), 256);
    b->dev_bytes = maps_bytes + insts_bytes + prefix_bytes;
    b->dev = dev_alloc(b->alloc, b->dev_bytes, b->stream);
    if (!b->dev) return set_error(WAVE2D_ERR_OOM, "batch table allocation failed");
    char* base = (char*)b->dev;
    CUtensorMap* dmaps = (CUtensorMap*)base;
    BatchInst* dinsts = (BatchInst*)(base + maps_bytes);
    int* dprefix = (int*)(base + maps_bytes + insts_bytes);
    for (int r = 0; r < n; ++r) insts[r].tm = dmaps + 4 * (size_t)r;
    cudaError_t e = cudaMemcpyAsync(dmaps, maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dinsts, insts.data(), insts.size() * sizeof(BatchInst), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dprefix, prefix.data(), prefix.size() * sizeof(int), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "batch table upload");

    // Capture the quanta.
    const int64_t max_steps = n ? steps[b->order[0]] : 0;
    const int64_t nq = (max_steps + Tq - 1) / Tq;
    const int rh_max = region_rows(13, OH, Tq);
    const int smem = 1024 + 2 * 4 * kBatchRVW * rh_max * 4;
    const bool per = b->bc == WAVE2D_BC_PERIODIC;
    auto kern = per ? k6_batch_step<true> : k6_batch_step<false>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(batch kernel)");
    const int gw = per ? kGhost : 0;
    int* status = b->hs[0]->status;
    b->plan_grids.clear();
    b->plan_active.clear();
    int active = n;
    for (int64_t q = 0; q < nq; ++q) {
        while (active > 0 && insts[active - 1].steps <= (int64_t)Tq * q) --active;
        if (active == 0) break;
        b->plan_grids.push_back(prefix[active]);
        b->plan_active.push_back(active);
    }
    b->plan_insts = dinsts;
    b->plan_prefix = dprefix;
    b->plan_smem = smem;
    b->plan_steps.assign(steps, steps + n);
    b->plan_Tq = Tq;
    b->plan_OH = OH;
    if (b->direct) return WAVE2D_OK;
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "begin capture");
    int launches = 0;
    for (size_t q = 0; q < b->plan_grids.size(); ++q) {
        kern<<<b->plan_grids[q], kBatchNW * 32, smem, b->stream>>>(dinsts, dprefix, b->plan_active[q], (int)q, Tq, OH,
                                                                 gw, status);
        ++launches;
    }
    cudaError_t le = cudaGetLastError();
    e = cudaStreamEndCapture(b->stream, &graph);
    if (le != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return cuda_fail(le, "batch kernel launch");
    }
    if (e != cudaSuccess) return cuda_fail(e, "end capture");
    e = cudaGraphInstantiate(&b->graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
    b->graph_launches = launches;
    return WAVE2D_OK;
}

// Plan of a register-streaming run: per scheme, the instances sorted by their
// number of full launches (steps / T), one launch of T levels per quantum over
// those still running, then one launch per remainder r = steps mod T (r levels)
// over the instances that have it, each instance at the parity its full
// launches left it in.
// Levels per launch of a streaming batch for scheme S: the batch quantum for
// the 13-point scheme, half as much again (6 for a quantum of 4) for the
// radius-1 schemes, whose halo columns round up to 8 for depths 5..8 (the
// single-grid kernel's measurement: 9-point level 13.4 us at T = 4, 11.7 at 6).
int stream_depth(int S, int Tq) { return S == 13 ? Tq : std::min(6, Tq + Tq / 2); }

int build_stream_plan(wave2d_batch* b, const int64_t* steps) {
    free_plan(b);
    const int n = (int)b->hs.size();
    const int L = b->OH;
    struct Table {
        std::vector<StreamInst> insts;
        std::vector<int> prefix;
        int scheme, T, branch;
        int64_t nq_max;  // full-launch tables: launches; remainder tables: 1
        std::vector<int64_t> nq;  // full launches per instance (full-launch tables)
    };
    std::vector<Table> tables;
    const int schemes[3] = {13, 9, 5};
    for (int br = 0; br < 3; ++br) {
        const int S = schemes[br];
        const int T = stream_depth(S, b->Tq);
        std::vector<int> idx;
        for (int i = 0; i < n; ++i)
            if (b->hs[i]->scheme == S && steps[i] > 0) idx.push_back(i);
        if (idx.empty()) continue;
        std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return steps[x] / T > steps[y] / T; });
        auto inst_of = [&](int i, int t, int flip) {
            wave2d* h = b->hs[i];
            StreamInst I{};
            for (int p = 0; p < 4; ++p) I.planes[p] = reinterpret_cast<float*>(h->hi[p]);
            I.g = h->geo();
            I.a = Coef3<float>{(float)h->a[0], (float)h->a[1], (float)h->a[2]};
            I.cur0 = h->cur ^ flip;
            I.prv0 = h->prv ^ flip;
            const int R = (S == 13) ? 2 : 1, HX = (R * t + 3) / 4 * 4, OW = 128 - 2 * HX;
            I.strips_x = (h->nx + OW - 1) / OW;
            return std::make_pair(I, I.strips_x * ((h->ny + L - 1) / L));
        };
        Table full;
        full.scheme = S;
        full.T = T;
        full.branch = br;
        full.prefix.push_back(0);
        for (int i : idx) {
            if (steps[i] / T == 0) break;
            auto pr = inst_of(i, T, 0);
            full.insts.push_back(pr.first);
            full.prefix.push_back(full.prefix.back() + pr.second);
            full.nq.push_back(steps[i] / T);
        }
        full.nq_max = full.nq.empty() ? 0 : full.nq[0];
        if (!full.insts.empty()) tables.push_back(std::move(full));
        for (int r = 1; r < T; ++r) {
            Table rem;
            rem.scheme = S;
            rem.T = r;
            rem.branch = br;
            rem.nq_max = 1;
            rem.prefix.push_back(0);
            for (int i : idx) {
                if (steps[i] % T != r) continue;
                auto pr = inst_of(i, r, (int)((steps[i] / T) & 1) * 2);
                rem.insts.push_back(pr.first);
                rem.prefix.push_back(rem.prefix.back() + pr.second);
            }
            if (!rem.insts.empty()) tables.push_back(std::move(rem));
        }
    }
    size_t bytes = 0;
    std::vector<size_t> at(tables.size());
    for (size_t t = 0; t < tables.size(); ++t) {
        at[t] = bytes;
        bytes += round_up(tables[t].insts.size() * sizeof(StreamInst), 256) +
                 round_up(tables[t].prefix.size() * sizeof(int), 256);
    }
    b->dev_bytes = std::max<size_t>(bytes, 256);
    b->dev = dev_alloc(b->alloc, b->dev_bytes, b->stream);
    if (!b->dev) return set_error(WAVE2D_ERR_OOM, "batch table allocation failed");
    b->plan_slaunches.clear();
    for (size_t t = 0; t < tables.size(); ++t) {
        Table& tb = tables[t];
        char* base = (char*)b->dev + at[t];
        StreamInst* di = (StreamInst*)base;
        int* dp = (int*)(base + round_up(tb.insts.size() * sizeof(StreamInst), 256));
        cudaError_t e = cudaMemcpyAsync(di, tb.insts.data(), tb.insts.size() * sizeof(StreamInst),
                                        cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dp, tb.prefix.data(), tb.prefix.size() * sizeof(int), cudaMemcpyHostToDevice, b->stream);
        if (e != cudaSuccess) return cuda_fail(e, "batch table upload");
        int active = (int)tb.insts.size();
        for (int64_t q = 0; q < tb.nq_max; ++q) {
            if (!tb.nq.empty())
                while (active > 0 && tb.nq[active - 1] <= q) --active;
            if (active == 0) break;
            const int grid = (tb.prefix[active] + kBatchStreamWarps - 1) / kBatchStreamWarps;
            b->plan_slaunches.push_back({tb.scheme, tb.T, grid, active, (int)q, tb.branch, di, dp});
        }
    }
    return WAVE2D_OK;  // pageable uploads return once the host tables may be released
}

template <int S>
cudaError_t launch_k7(const wave2d_batch::SLaunch& l, int L, cudaStream_t st) {
    if constexpr (S != 13) {
        if (l.T == 5) {
            k7_batch_stream<S, 5><<<l.grid, kBatchStreamWarps * 32, stream_smem_bytes<S, 5, kBatchStreamWarps>(), st>>>(
                (const StreamInst*)l.insts, l.prefix, l.n_active, l.q, L);
            return cudaGetLastError();
        }
        if (l.T == 6) {
            k7_batch_stream<S, 6><<<l.grid, kBatchStreamWarps * 32, stream_smem_bytes<S, 6, kBatchStreamWarps>(), st>>>(
                (const StreamInst*)l.insts, l.prefix, l.n_active, l.q, L);
            return cudaGetLastError();
        }
    }
    switch (l.T) {
        case 1: k7_batch_stream<S, 1><<<l.grid, kBatchStreamWarps * 32, stream_smem_bytes<S, 1, kBatchStreamWarps>(), st>>>(
                    (const StreamInst*)l.insts, l.prefix, l.n_active, l.q, L); break;
        case 2: k7_batch_stream<S, 2><<<l.grid, kBatchStreamWarps * 32, stream_smem_bytes<S, 2, kBatchStreamWarps>(), st>>>(
                    (const StreamInst*)l.insts, l.prefix, l.n_active, l.q, L); break;
        case 3: k7_batch_stream<S, 3><<<l.grid, kBatchStreamWarps * 32, stream_smem_bytes<S, 3, kBatchStreamWarps>(), st>>>(
                    (const StreamInst*)l.insts, l.prefix, l.n_active, l.q, L); break;
        default: k7_batch_stream<S, 4><<<l.grid, kBatchStreamWarps * 32, stream_smem_bytes<S, 4, kBatchStreamWarps>(), st>>>(
                    (const StreamInst*)l.insts, l.prefix, l.n_active, l.q, L); break;
    }
    return cudaGetLastError();
}

// Issue the launches of a streaming plan: each scheme's launches in order on
// its own stream, forked from the batch stream and joined back to it.
int issue_stream_plan(wave2d_batch* b, int& launches) {
    launches = 0;
    bool used[3] = {false, false, false};
    for (const auto& l : b->plan_slaunches) used[l.branch] = true;
    cudaError_t e = cudaSuccess;
    if (!b->ev_fork) e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
    for (int br = 0; br < 3 && e == cudaSuccess; ++br) {  // created on first use, kept for the batch's life
        if (!b->ev_join[br]) e = cudaEventCreateWithFlags(&b->ev_join[br], cudaEventDisableTiming);
        if (e == cudaSuccess && !b->side[br]) e = cudaStreamCreateWithFlags(&b->side[br], cudaStreamNonBlocking);
    }
    if (e != cudaSuccess) return cuda_fail(e, "batch stream create");
    e = cudaEventRecord(b->ev_fork, b->stream);
    for (int br = 0; br < 3 && e == cudaSuccess; ++br)
        if (used[br]) e = cudaStreamWaitEvent(b->side[br], b->ev_fork, 0);
    for (const auto& l : b->plan_slaunches) {
        if (e != cudaSuccess) break;
        cudaStream_t st = b->side[l.branch];
        e = l.scheme == 13 ? launch_k7<13>(l, b->OH, st) : l.scheme == 9 ? launch_k7<9>(l, b->OH, st)
                                                                         : launch_k7<5>(l, b->OH, st);
        ++launches;
    }
    for (int br = 0; br < 3 && e == cudaSuccess; ++br)
        if (used[br]) {
            e = cudaEventRecord(b->ev_join[br], b->side[br]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->ev_join[br], 0);
        }
    if (e != cudaSuccess) return cuda_fail(e, "batched streaming launch");
    return WAVE2D_OK;
}

int capture_stream_plan(wave2d_batch* b) {
    if (b->direct) return WAVE2D_OK;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "begin capture");
    int launches = 0;
    const int rc = issue_stream_plan(b, launches);
    e = cudaStreamEndCapture(b->stream, &graph);
    if (rc != WAVE2D_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "end capture");
    e = cudaGraphInstantiate(&b->graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
    b->graph_launches = launches;
    return WAVE2D_OK;
}

// Launch the quanta of the current plan one by one (direct mode).
int launch_direct(wave2d_batch* b) {
    const bool per = b->bc == WAVE2D_BC_PERIODIC;
    auto kern = per ? k6_batch_step<true> : k6_batch_step<false>;
    const int gw = per ? kGhost : 0;
    for (size_t q = 0; q < b->plan_grids.size(); ++q) {
        kern<<<b->plan_grids[q], kBatchNW * 32, b->plan_smem, b->stream>>>(
            (const BatchInst*)b->plan_insts, b->plan_prefix, b->plan_active[q], (int)q, b->Tq, b->OH, gw,
            b->hs[0]->status);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "batch kernel launch");
        g_launches.fetch_add(1);
    }
    return WAVE2D_OK;
}

bool stream_mode(const wave2d_batch* b) { return b->kernel == WAVE2D_KERNEL_STREAM && b->bc == WAVE2D_BC_ZERO; }

bool same_plan(const wave2d_batch* b, const int64_t* steps) {
    if ((!b->graph && !b->direct) || !b->dev || b->plan_Tq != b->Tq || b->plan_OH != b->OH ||
        b->plan_kernel != (stream_mode(b) ? 1 : 0) || b->plan_steps.size() != b->hs.size())
        return false;
    for (size_t i = 0; i < b->hs.size(); ++i)
        if (b->plan_steps[i] != steps[i] || b->plan_start[i] != b->hs[i]->cur * 4 + b->hs[i]->prv) return false;
    return true;
}

int run_once(wave2d_batch* b, const int64_t* steps) {
    const int n = (int)b->hs.size();
    // A plan records each handle's starting planes (the pairs alternate per
    // quantum); it is replayed only when they and the step counts match.
    const bool sm = stream_mode(b);
    if (!same_plan(b, steps)) {
        int rc = sm ? build_stream_plan(b, steps) : build_plan(b, steps);
        if (rc == WAVE2D_OK && sm) rc = capture_stream_plan(b);
        if (rc != WAVE2D_OK) return rc;
        b->plan_steps.assign(steps, steps + n);
        b->plan_Tq = b->Tq;
        b->plan_OH = b->OH;
        b->plan_kernel = sm ? 1 : 0;
        b->plan_start.resize(n);
        for (int i = 0; i < n; ++i) b->plan_start[i] = b->hs[i]->cur * 4 + b->hs[i]->prv;
    }
    if (b->direct && sm) {
        int launches = 0;
        int rc = issue_stream_plan(b, launches);
        if (rc != WAVE2D_OK) return rc;
        g_launches.fetch_add(launches);
    } else if (b->direct) {
        int rc = launch_direct(b);
        if (rc != WAVE2D_OK) return rc;
    } else {
        cudaError_t e = cudaGraphLaunch(b->graph, b->stream);
        if (e != cudaSuccess) return cuda_fail(e, "batch graph launch");
        g_launches.fetch_add(b->graph_launches);
    }
    for (int i = 0; i < n; ++i) {
        wave2d* h = b->hs[i];
        const int64_t Ti = sm ? stream_depth(h->scheme, b->Tq) : b->Tq;
        const int64_t nq = (steps[i] + Ti - 1) / Ti;
        if (nq & 1) {
            h->cur ^= 2;
            h->prv ^= 2;
        }
        h->k += steps[i];
        for (auto& gx : h->graph)
            if (gx) {
                cudaGraphExecDestroy(gx);
                gx = nullptr;
            }
    }
    return WAVE2D_OK;
}

}  // namespace

namespace w2d {

// Replace the members of a batch (validated as at create: F32, one boundary
// and device, no repeats) and drop its plan; its streams, events and tuning
// stay.  For callers that advance a changing set of handles (the server).
int batch_set_handles(wave2d_batch* b, wave2d_t* handles, int n, int rows) {
    if (!b || !handles || n < 1) return set_error(WAVE2D_ERR_ARG, "batch needs at least one handle");
    for (int i = 0; i < n; ++i)
        if (!handles[i] || handles[i]->dtype != WAVE2D_F32 || handles[i]->bc != b->bc)
            return set_error(WAVE2D_ERR_ARG, "batch member %d does not match the batch", i);
    free_plan(b);
    b->hs.assign(handles, handles + n);
    if (rows > 0) b->OH = rows;
    return WAVE2D_OK;
}

// FP64 sqrt(sum u^2) and max |u| of the current level of each handle (all on
// stream st), written to host_out[2 i], host_out[2 i + 1] by an asynchronous
// copy: host_out must be pinned and stay valid until st passes an event
// recorded after this call.  Scratch is allocated and freed in stream order.
int batch_norms_async(wave2d* const* hs, int n, cudaStream_t st, const Allocator& al, double* host_out) {
    std::vector<BatchNorm> ns(n);
    std::vector<int> prefix(n + 1, 0);
    int chunks = 0;
    for (int i = 0; i < n; ++i) {
        const wave2d* h = hs[i];
        ns[i].plane = reinterpret_cast<const float*>(h->hi[h->cur]);
        ns[i].g = h->geo();
        ns[i].blocks = (h->ny + 7) / 8;
        ns[i].first = chunks;
        chunks += ns[i].blocks;
        prefix[i + 1] = chunks;
    }
    const size_t ns_bytes = round_up(n * sizeof(BatchNorm), 256), pre_bytes = round_up((n + 1) * sizeof(int), 256);
    const size_t part_bytes = round_up(2 * (size_t)chunks * sizeof(double), 256);
    const size_t total = ns_bytes + pre_bytes + part_bytes + 2 * n * sizeof(double);
    char* dev = (char*)dev_alloc(al, total, st);
    if (!dev) return set_error(WAVE2D_ERR_OOM, "batch norm allocation failed");
    double* part = (double*)(dev + ns_bytes + pre_bytes);
    double* res = (double*)(dev + ns_bytes + pre_bytes + part_bytes);
    cudaError_t e = cudaMemcpyAsync(dev, ns.data(), n * sizeof(BatchNorm), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dev + ns_bytes, prefix.data(), (n + 1) * sizeof(int), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        k6_batch_norm_partial<<<chunks, 256, 0, st>>>((const BatchNorm*)dev, (const int*)(dev + ns_bytes), n, part);
        k6_batch_norm_final<<<n, 32, 0, st>>>((const BatchNorm*)dev, part, res);
        e = cudaGetLastError();
        if (e == cudaSuccess) g_launches.fetch_add(2);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_out, res, 2 * n * sizeof(double), cudaMemcpyDeviceToHost, st);
    dev_free(al, dev, total, st);
    if (e != cudaSuccess) return cuda_fail(e, "batch norms");
    return WAVE2D_OK;
}

}  // namespace w2d

extern "C" {

int wave2d_batch_create(wave2d_t* handles, int n, const wave2d_tune* opt, wave2d_batch_t* out) {
    if (!handles || !out || n < 1) return set_error(WAVE2D_ERR_ARG, "batch needs at least one handle");
    *out = nullptr;
    for (int i = 0; i < n; ++i) {
        if (!handles[i]) return set_error(WAVE2D_ERR_ARG, "null handle %d", i);
        if (handles[i]->dtype != WAVE2D_F32) return set_error(WAVE2D_ERR_ARG, "batched stepping needs F32 storage");
        if (handles[i]->flags & WAVE2D_CANARY)
            return set_error(WAVE2D_ERR_ARG, "handles with guard-band canaries are not batched");
        if (handles[i]->bc == WAVE2D_BC_ODD)
            return set_error(WAVE2D_ERR_ARG, "batched stepping covers the zero and periodic boundaries");
        if (handles[i]->nclass > 0)
            return set_error(WAVE2D_ERR_ARG,
                             "batched stepping covers the 5-, 9- and 13-point schemes with plain sums only");
        if (handles[i]->bc != handles[0]->bc) return set_error(WAVE2D_ERR_ARG, "all handles of a batch share one boundary");
        if (handles[i]->device != handles[0]->device) return set_error(WAVE2D_ERR_ARG, "all handles of a batch share one device");
        for (int j = 0; j < i; ++j)
            if (handles[j] == handles[i]) return set_error(WAVE2D_ERR_ARG, "handle %d appears twice", i);
    }
    const bool stream_kernel = opt && opt->kernel == WAVE2D_KERNEL_STREAM;
    if (opt && opt->kernel != 0 && opt->kernel != WAVE2D_KERNEL_TEMPORAL && !stream_kernel)
        return set_error(WAVE2D_ERR_ARG, "batch kernel must be 0, WAVE2D_KERNEL_TEMPORAL or WAVE2D_KERNEL_STREAM");
    if (stream_kernel && handles[0]->bc != WAVE2D_BC_ZERO)
        return set_error(WAVE2D_ERR_ARG, "batched register streaming covers the zero boundary");
    if (opt && opt->temporal_t != 0 && (opt->temporal_t < 1 || opt->temporal_t > 4))
        return set_error(WAVE2D_ERR_ARG, "batch quantum must be 1..4 levels");
    if (opt && opt->tile_h != 0 && !stream_kernel && opt->tile_h != 32 && opt->tile_h != 64)
        return set_error(WAVE2D_ERR_ARG, "batch tile height must be 32 or 64");
    if (opt && opt->tile_h != 0 && stream_kernel && (opt->tile_h < 8 || opt->tile_h > 1024))
        return set_error(WAVE2D_ERR_ARG, "batch strip rows must be 8..1024");
    wave2d_batch* b = new (std::nothrow) wave2d_batch();
    if (!b) return set_error(WAVE2D_ERR_OOM, "host allocation failed");
    b->hs.assign(handles, handles + n);
    b->stream = handles[0]->stream;
    b->alloc = handles[0]->alloc;
    b->bc = handles[0]->bc;
    b->num_sms = handles[0]->num_sms;
    if (stream_kernel) {
        b->kernel = WAVE2D_KERNEL_STREAM;
        b->OH = 64;
    }
    if (opt && opt->temporal_t) b->Tq = opt->temporal_t;
    if (opt && opt->tile_h) b->OH = opt->tile_h;
    b->direct = opt && opt->use_graph == 0;
    cudaError_t e = cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        delete b;
        return cuda_fail(e, "event create");
    }
    *out = b;
    return WAVE2D_OK;
}

void wave2d_batch_destroy(wave2d_batch_t b) {
    if (!b) return;
    const bool graph = b->graph != nullptr;
    free_plan(b);  // tables freed in stream order
    // a captured run may still be executing; direct launches need no wait
    if (graph || b->side[0] || b->side[1] || b->side[2]) cudaStreamSynchronize(b->stream);
    for (int br = 0; br < 3; ++br) {
        if (b->side[br]) cudaStreamDestroy(b->side[br]);
        if (b->ev_join[br]) cudaEventDestroy(b->ev_join[br]);
    }
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->ev) cudaEventDestroy(b->ev);
    delete b;
}

static int batch_first_step_impl(wave2d_batch_t b, const double* const* u0, const double* const* v0, int on_device);

int wave2d_batch_first_step(wave2d_batch_t b, const double* const* u0, const double* const* v0, int on_device) {
    NvtxRange nvtx_range("wave2d_batch_first_step");
    if (!b || !u0 || !v0) return set_error(WAVE2D_ERR_ARG, "null argument");
    int rc = order_streams(b, true);
    if (rc == WAVE2D_OK) rc = batch_first_step_impl(b, u0, v0, on_device);
    const int rc2 = order_streams(b, false);
    return rc != WAVE2D_OK ? rc : rc2;
}

static int batch_first_step_impl(wave2d_batch_t b, const double* const* u0, const double* const* v0, int on_device) {
    const int n = (int)b->hs.size();
    const bool per = b->bc == WAVE2D_BC_PERIODIC;
    size_t stage_doubles = 0;
    for (int i = 0; i < n; ++i) {
        if (!u0[i] || !v0[i]) return set_error(WAVE2D_ERR_ARG, "null initial data for instance %d", i);
        if (!on_device) stage_doubles += 2 * (size_t)b->hs[i]->nx * b->hs[i]->ny;
    }
    std::vector<BatchFirst> fs(n);
    std::vector<int> prefix(n + 1, 0);
    const size_t fs_bytes = round_up(n * sizeof(BatchFirst), 256), pre_bytes = round_up((n + 1) * sizeof(int), 256);
    const size_t total = fs_bytes + pre_bytes + stage_doubles * sizeof(double);
    char* dev = (char*)dev_alloc(b->alloc, total, b->stream);
    if (!dev) return set_error(WAVE2D_ERR_OOM, "batch staging allocation failed");
    double* stage = (double*)(dev + fs_bytes + pre_bytes);
    int rc = WAVE2D_OK;
    for (int i = 0; i < n && rc == WAVE2D_OK; ++i) {
        wave2d* h = b->hs[i];
        const size_t nn = (size_t)h->nx * h->ny;
        BatchFirst& F = fs[i];
        if (on_device) {
            F.u0 = u0[i];
            F.v0 = v0[i];
        } else {
            cudaError_t e = cudaMemcpyAsync(stage, u0[i], nn * sizeof(double), cudaMemcpyHostToDevice, b->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(stage + nn, v0[i], nn * sizeof(double), cudaMemcpyHostToDevice, b->stream);
            if (e != cudaSuccess) rc = cuda_fail(e, "batch upload");
            F.u0 = stage;
            F.v0 = stage + nn;
            stage += 2 * nn;
        }
        F.plane0 = reinterpret_cast<float*>(h->hi[0]);
        F.plane1 = reinterpret_cast<float*>(h->hi[1]);
        F.g = h->geo();
        F.ahalf = Coef3<double>{h->a[0] / 2, h->a[1] / 2, h->a[2] / 2};
        F.b = Coef3<double>{h->b[0], h->b[1], h->b[2]};
        F.tau = h->tau;
        F.scheme = h->scheme;
        F.blocks_x = (h->nx + 31) / 32;
        prefix[i + 1] = prefix[i] + F.blocks_x * ((h->ny + 7) / 8);
    }
    // Batched runs keep the full ghost ring valid for the periodic boundary.
    const int gw = per ? kGhost : 0;
    if (rc == WAVE2D_OK) {
        cudaError_t e = cudaMemcpyAsync(dev, fs.data(), n * sizeof(BatchFirst), cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dev + fs_bytes, prefix.data(), (n + 1) * sizeof(int), cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) {
            auto kern = per ? k6_batch_first<true> : k6_batch_first<false>;
            kern<<<prefix[n], dim3(32, 8), 0, b->stream>>>((const BatchFirst*)dev, (const int*)(dev + fs_bytes), n, gw);
            e = cudaGetLastError();
            if (e == cudaSuccess) g_launches.fetch_add(1);
        }
        // pageable host arrays are staged by the copy calls themselves; only
        // the device tables' uploads above need nothing more
        if (e != cudaSuccess) rc = cuda_fail(e, "batch first step");
    }
    dev_free(b->alloc, dev, total, b->stream);
    if (rc != WAVE2D_OK) return rc;
    for (wave2d* h : b->hs) {
        h->cur = 0;
        h->prv = 1;
        h->k = 1;
        h->initialized = true;
        if (per) h->gw = std::max(h->gw, (int)kGhost);
        for (auto& gx : h->graph)
            if (gx) {
                cudaGraphExecDestroy(gx);
                gx = nullptr;
            }
    }
    return WAVE2D_OK;
}

static int batch_run_impl(wave2d_batch_t b, const int64_t* steps);

int wave2d_batch_run(wave2d_batch_t b, const int64_t* steps) {
    NvtxRange nvtx_range("wave2d_batch_run");
    if (!b || !steps) return set_error(WAVE2D_ERR_ARG, "null argument");
    int rc = order_streams(b, true);
    if (rc == WAVE2D_OK) rc = batch_run_impl(b, steps);
    const int rc2 = order_streams(b, false);
    return rc != WAVE2D_OK ? rc : rc2;
}

static int batch_run_impl(wave2d_batch_t b, const int64_t* steps) {
    const int n = (int)b->hs.size();
    for (int i = 0; i < n; ++i) {
        if (steps[i] < 0) return set_error(WAVE2D_ERR_ARG, "negative step count for instance %d", i);
        if (!b->hs[i]->initialized) return set_error(WAVE2D_ERR_STATE, "instance %d has no state yet", i);
        if ((b->hs[i]->cur ^ b->hs[i]->prv) != 1 || (b->hs[i]->cur >> 1) != (b->hs[i]->prv >> 1))
            return set_error(WAVE2D_ERR_STATE, "instance %d levels are not in one plane pair", i);
    }
    if (b->bc == WAVE2D_BC_PERIODIC) {
        // the batched kernel reads the full ghost ring
        for (wave2d* h : b->hs) {
            if (h->gw < kGhost) {
                h->gw = kGhost;
                const long long total = (long long)(h->nx + 2 * h->gw) * (h->ny + 2 * h->gw);
                const int grid = (int)std::min<long long>((total + 255) / 256, 8LL * h->num_sms);
                for (int p : {h->cur, h->prv}) {
                    k_refresh_ghosts<DT_F32, BCM_PERIODIC><<<grid, 256, 0, b->stream>>>(h->level(p), h->geo(), h->gw);
                    cudaError_t e = cudaGetLastError();
                    if (e != cudaSuccess) return cuda_fail(e, "ghost refresh");
                    g_launches.fetch_add(1);
                }
            }
        }
    }
    return run_once(b, steps);
}

static int batch_autotune_impl(wave2d_batch_t b, const int64_t* steps, int64_t probe_steps, wave2d_tune* best);

int wave2d_batch_autotune(wave2d_batch_t b, const int64_t* steps, int64_t probe_steps, wave2d_tune* best) {
    NvtxRange nvtx_range("wave2d_batch_autotune");
    if (!b || !steps) return set_error(WAVE2D_ERR_ARG, "null argument");
    int rc = order_streams(b, true);
    if (rc == WAVE2D_OK) rc = batch_autotune_impl(b, steps, probe_steps, best);
    const int rc2 = order_streams(b, false);
    return rc != WAVE2D_OK ? rc : rc2;
}

static int batch_autotune_impl(wave2d_batch_t b, const int64_t* steps, int64_t probe_steps, wave2d_tune* best) {
    if (probe_steps < 1) return set_error(WAVE2D_ERR_ARG, "probe_steps must be >= 1");
    const int n = (int)b->hs.size();
    for (int i = 0; i < n; ++i)
        if (!b->hs[i]->initialized) return set_error(WAVE2D_ERR_STATE, "instance %d has no state yet", i);
    // Snapshot the two current levels of every instance.
    size_t snap_bytes = 0;
    for (wave2d* h : b->hs) snap_bytes += 2 * h->plane_bytes;
    char* snap = (char*)dev_alloc(b->alloc, snap_bytes, b->stream);
    if (!snap) return set_error(WAVE2D_ERR_OOM, "batch autotune snapshot allocation failed");
    struct Saved { int cur, prv, gw; int64_t k; };
    std::vector<Saved> saved(n);
    auto copy_all = [&](bool save) -> int {
        char* sp = snap;
        for (int i = 0; i < n; ++i) {
            wave2d* h = b->hs[i];
            if (save) saved[i] = Saved{h->cur, h->prv, h->gw, h->k};
            const int planes[2] = {saved[i].cur, saved[i].prv};
            for (int q = 0; q < 2; ++q, sp += h->plane_bytes) {
                cudaError_t e = save ? cudaMemcpyAsync(sp, h->hi[planes[q]], h->plane_bytes, cudaMemcpyDeviceToDevice, b->stream)
                                     : cudaMemcpyAsync(h->hi[planes[q]], sp, h->plane_bytes, cudaMemcpyDeviceToDevice, b->stream);
                if (e != cudaSuccess) return cuda_fail(e, "batch autotune snapshot copy");
            }
            h->cur = saved[i].cur;
            h->prv = saved[i].prv;
            h->k = saved[i].k;
        }
        return WAVE2D_OK;
    };
    std::vector<int64_t> probe(n);
    for (int i = 0; i < n; ++i) probe[i] = std::min<int64_t>(steps[i], probe_steps);
    int rc = copy_all(true);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (rc == WAVE2D_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
        rc = set_error(WAVE2D_ERR_CUDA, "event create failed");
    // candidates: (kernel, levels per launch, rows per tile or strip); the
    // register-streaming batch for the zero boundary
    struct Cand { int kernel, T, rows; };
    std::vector<Cand> cands = {{WAVE2D_KERNEL_TEMPORAL, 2, 32}, {WAVE2D_KERNEL_TEMPORAL, 2, 64},
                               {WAVE2D_KERNEL_TEMPORAL, 4, 32}, {WAVE2D_KERNEL_TEMPORAL, 4, 64}};
    if (b->bc == WAVE2D_BC_ZERO)
        for (int T : {2, 3, 4})
            for (int rows : {16, 32, 64}) cands.push_back({WAVE2D_KERNEL_STREAM, T, rows});
    const int kernel0 = b->kernel, T0 = b->Tq, OH0 = b->OH;
    float best_ms = -1;
    int best_c = -1;
    for (int c = 0; c < (int)cands.size() && rc == WAVE2D_OK; ++c) {
        b->kernel = cands[c].kernel;
        b->Tq = cands[c].T;
        b->OH = cands[c].rows;
        rc = copy_all(false);
        if (rc == WAVE2D_OK) rc = run_once(b, probe.data());  // builds the plan and warms up
        if (rc == WAVE2D_OK) rc = copy_all(false);
        if (rc != WAVE2D_OK) break;
        cudaEventRecord(e0, b->stream);
        rc = run_once(b, probe.data());
        cudaEventRecord(e1, b->stream);
        if (rc != WAVE2D_OK) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            rc = set_error(WAVE2D_ERR_CUDA, "batch autotune timing failed");
            break;
        }
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (best_ms < 0 || ms < best_ms) {
            best_ms = ms;
            best_c = c;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    const int rc2 = copy_all(false);
    cudaStreamSynchronize(b->stream);
    dev_free(b->alloc, snap, snap_bytes, b->stream);
    free_plan(b);
    if (rc == WAVE2D_OK) rc = rc2;
    if (best_c >= 0) {
        b->kernel = cands[best_c].kernel;
        b->Tq = cands[best_c].T;
        b->OH = cands[best_c].rows;
    } else {
        b->kernel = kernel0;
        b->Tq = T0;
        b->OH = OH0;
    }
    if (best) {
        std::memset(best, 0, sizeof *best);
        best->kernel = b->kernel;
        best->temporal_t = b->Tq;
        best->tile_h = b->OH;
    }
    return rc;
}

static int batch_norms_impl(wave2d_batch_t b, double* out);

int wave2d_batch_norms(wave2d_batch_t b, double* out) {
    NvtxRange nvtx_range("wave2d_batch_norms");
    if (!b || !out) return set_error(WAVE2D_ERR_ARG, "null argument");
    int rc = order_streams(b, true);
    if (rc == WAVE2D_OK) rc = batch_norms_impl(b, out);
    const int rc2 = order_streams(b, false);
    return rc != WAVE2D_OK ? rc : rc2;
}

static int batch_norms_impl(wave2d_batch_t b, double* out) {
    const int n = (int)b->hs.size();
    std::vector<BatchNorm> ns(n);
    std::vector<int> prefix(n + 1, 0);
    int chunks = 0;
    for (int i = 0; i < n; ++i) {
        wave2d* h = b->hs[i];
        if (!h->initialized) return set_error(WAVE2D_ERR_STATE, "instance %d has no state yet", i);
        ns[i].plane = reinterpret_cast<const float*>(h->hi[h->cur]);
        ns[i].g = h->geo();
        ns[i].blocks = (h->ny + 7) / 8;
        ns[i].first = chunks;
        chunks += ns[i].blocks;
        prefix[i + 1] = chunks;
    }
    const size_t ns_bytes = round_up(n * sizeof(BatchNorm), 256), pre_bytes = round_up((n + 1) * sizeof(int), 256);
    const size_t part_bytes = round_up(2 * (size_t)chunks * sizeof(double), 256);
    const size_t total = ns_bytes + pre_bytes + part_bytes + 2 * n * sizeof(double);
    char* dev = (char*)dev_alloc(b->alloc, total, b->stream);
    if (!dev) return set_error(WAVE2D_ERR_OOM, "batch norm allocation failed");
    double* part = (double*)(dev + ns_bytes + pre_bytes);
    double* res = (double*)(dev + ns_bytes + pre_bytes + part_bytes);
    cudaError_t e = cudaMemcpyAsync(dev, ns.data(), n * sizeof(BatchNorm), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dev + ns_bytes, prefix.data(), (n + 1) * sizeof(int), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) {
        k6_batch_norm_partial<<<chunks, 256, 0, b->stream>>>((const BatchNorm*)dev, (const int*)(dev + ns_bytes), n, part);
        k6_batch_norm_final<<<n, 32, 0, b->stream>>>((const BatchNorm*)dev, part, res);
        e = cudaGetLastError();
        if (e == cudaSuccess) g_launches.fetch_add(2);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, res, 2 * n * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    dev_free(b->alloc, dev, total, b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "batch norms");
    return WAVE2D_OK;
}

}  // extern "C"
