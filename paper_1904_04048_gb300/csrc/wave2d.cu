// C-ABI implementation of include/wave2d.h: handles, memory, dispatch.
//
// The paper's method (arXiv:1904.04048, Sections 3 and 6) runs entirely in the
// kernels of kernels.cuh; this file validates arguments, lays out device
// memory, builds the coefficient tables of Section 6 and the TMA descriptors,
// and launches the kernels on the handle's stream.
#include <cudaTypedefs.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "kernels_temporal.cuh"
#include "stencil_chain.cuh"
#include "wave2d_impl.cuh"

namespace w2d {

// ------------------------------------------------------------------ errors
static thread_local std::string t_err;

int set_error(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_err = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    return set_error(e == cudaErrorMemoryAllocation ? WAVE2D_ERR_OOM : WAVE2D_ERR_CUDA, "%s: %s (%s)",
                     what, cudaGetErrorString(e), cudaGetErrorName(e));
}

std::atomic<int64_t> g_launches{0};

// -------------------------------------------------------------- allocation
static std::mutex g_alloc_mu;
static Allocator g_alloc;

Allocator current_allocator() {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    return g_alloc;
}

void* dev_alloc(const Allocator& a, size_t bytes, cudaStream_t s) {
    if (bytes == 0) bytes = 256;
    if (a.alloc) return a.alloc(bytes, (void*)s, a.ctx);
    void* p = nullptr;
    if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void dev_free(const Allocator& a, void* p, size_t bytes, cudaStream_t s) {
    if (!p) return;
    if (a.release) {
        a.release(p, bytes, (void*)s, a.ctx);
        return;
    }
    cudaFreeAsync(p, s);
}

// ------------------------------------------------------------ coefficients
// Section 6: Eq. comp5.1/5.2, comp9.1/9.2, comp13.1/13.2 written as
// Lambda_a / Lambda_b coefficients; conventional comparison schemes: b = 0
// and, for nine points, the isotropic Laplacian of Eq. comp9.2b.
static void scheme_coefficients(int scheme, bool conventional, double lam, double a[3], double b[3]) {
    const double l2 = lam * lam, l4 = l2 * l2;
    a[0] = a[1] = a[2] = b[0] = b[1] = b[2] = 0.0;
    switch (scheme) {
        case 5:
            a[0] = l2;
            b[0] = l2 / 6.0;
            break;
        case 9:
            if (conventional) {
                a[0] = 2.0 * l2 / 3.0;
                a[1] = l2 / 6.0;
            } else {
                a[0] = l2 * (1.0 - l2 / 3.0);
                a[1] = l4 / 6.0;
                b[0] = l2 / 6.0 * (1.0 - l2 / 5.0);
                b[1] = l4 / 60.0;
            }
            break;
        case 13:
            a[0] = l2 * (4.0 - 2.0 * l2) / 3.0;
            a[1] = l4 / 6.0;
            a[2] = l2 * (l2 - 1.0) / 12.0;
            b[0] = l2 / 6.0 * (4.0 / 3.0 - 2.0 * l2 / 5.0);
            b[1] = l4 / 60.0;
            b[2] = l2 / 6.0 * (l2 / 20.0 - 1.0 / 12.0);
            break;
    }
    if (conventional) b[0] = b[1] = b[2] = 0.0;
}

static double lambda_max_of(int scheme, bool conventional) {
    switch (scheme) {
        case 5:
        case 13:
            return 1.0 / std::sqrt(2.0);
        case 9:
            return conventional ? std::sqrt(3.0) / 2.0 : std::sqrt((3.0 - std::sqrt(3.0)) / 2.0);
    }
    return 0.0;
}

template <typename V>
static Coef3<V> coef_as(const double a[3]);
template <>
Coef3<double> coef_as<double>(const double a[3]) { return {a[0], a[1], a[2]}; }
template <>
Coef3<float> coef_as<float>(const double a[3]) {
    return {(float)a[0], (float)a[1], (float)a[2]};
}
static df split_df(double v) {
    const float h = (float)v;
    return {h, (float)(v - (double)h)};
}
template <>
Coef3<df> coef_as<df>(const double a[3]) { return {split_df(a[0]), split_df(a[1]), split_df(a[2])}; }

// --------------------------------------------------------------- dispatch
template <int V>
using IC = std::integral_constant<int, V>;
template <bool V>
using BC_ = std::integral_constant<bool, V>;

template <typename Fn>
static void dispatch_s(int scheme, Fn&& fn) {
    switch (scheme) {
        case 5: fn(IC<5>{}); break;
        case 9: fn(IC<9>{}); break;
        default: fn(IC<13>{}); break;
    }
}
template <typename Fn>
static void dispatch_dt(int dt, Fn&& fn) {
    switch (dt) {
        case DT_F64: fn(IC<DT_F64>{}); break;
        case DT_F32: fn(IC<DT_F32>{}); break;
        default: fn(IC<DT_F32X2>{}); break;
    }
}
template <typename Fn>
static void dispatch_bc(int bc, Fn&& fn) {
    switch (bc) {
        case WAVE2D_BC_PERIODIC: fn(IC<BCM_PERIODIC>{}); break;
        case WAVE2D_BC_ODD: fn(IC<BCM_ODD>{}); break;
        default: fn(IC<BCM_ZERO>{}); break;
    }
}
template <typename Fn>
static void dispatch_bool(bool v, Fn&& fn) {
    if (v) fn(BC_<true>{});
    else fn(BC_<false>{});
}

// Kernels that advance T levels per launch (out of place, full ghost ring).
static bool is_multilevel(int kernel) { return kernel == WAVE2D_KERNEL_TEMPORAL || kernel == WAVE2D_KERNEL_STREAM; }
// Handles those kernels take (FP32 is checked separately): the Section 6
// schemes with plain sums, zero or periodic boundary; with guard-band
// canaries the zero boundary only, where they write inside the grid alone
// (the ghost cells they read beyond R feed only nodes forced to zero).
static bool multilevel_ok(const wave2d* h) {
    return h->nclass == 0 && h->bc != WAVE2D_BC_ODD && !((h->flags & WAVE2D_CANARY) && h->bc != WAVE2D_BC_ZERO);
}
// Handles the register-streaming kernel takes: FP32 storage; a Section 6
// scheme, or a class chain of one to three classes (the 5-, 9- and 13-point
// stencils: difference sums, difference form, or a derived scheme's plain
// sums); boundary as multilevel_ok.  The difference form on a periodic grid
// needs rows of whole vectors (the kernel reads d^k at wrapped coordinates;
// no ring images of d^k are kept).
static bool stream_ok(const wave2d* h) {
    return h->dtype == DT_F32 && h->nclass <= 3 && h->bc != WAVE2D_BC_ODD &&
           !((h->flags & WAVE2D_CANARY) && h->bc != WAVE2D_BC_ZERO) &&
           (!h->diff_form || h->bc == WAVE2D_BC_ZERO || (h->nx % 4 == 0 && h->ny >= 16));
}

// ----------------------------------------------------------- TMA encoding
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

static int encode_plane(CUtensorMap* tm, void* plane, const wave2d* h, int box_w, int box_h) {
    auto enc = tensor_map_encoder();
    if (!enc) return set_error(WAVE2D_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
    const cuuint64_t dims[2] = {(cuuint64_t)h->pitch, (cuuint64_t)h->rows};
    const cuuint64_t strides[1] = {(cuuint64_t)h->pitch * h->elem};
    const cuuint32_t box[2] = {(cuuint32_t)box_w, (cuuint32_t)box_h};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(tm, h->elem == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                     plane, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(WAVE2D_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return WAVE2D_OK;
}

// Tile configurations of the TMA kernel (rows per tile, warps, stages).
constexpr int kTmaNW = 8;
constexpr int kTmaStages = 3;

template <typename T, int S, int TH>
static int tma_box(int& bw, int& bh, int& tw) {
    using C = TmaCfg<T, S, TH, kTmaNW>;
    bw = C::BOX_W;
    bh = C::BOX_H;
    tw = C::TW;
    return C::STAGE_BYTES;
}

static int prepare_tma(wave2d* h) {
    if (h->dtype == DT_F32X2) return set_error(WAVE2D_ERR_ARG, "TMA kernel supports F32 and F64 storage");
    int bw = 0, bh = 0, tw = 0, th = 32;
    int rc = WAVE2D_OK;
    if (h->nclass > 0) {
        chain_tma_box(h, bw, bh, tw, th);
    } else {
        dispatch_s(h->scheme, [&](auto Sc) {
            constexpr int S = decltype(Sc)::value;
            if (h->dtype == DT_F32) tma_box<float, S, 32>(bw, bh, tw);
            else tma_box<double, S, 32>(bw, bh, tw);
        });
    }
    for (int p = 0; p < h->nlevels && rc == WAVE2D_OK; ++p) {
        rc = encode_plane(&h->tm_cur[p], h->hi[p], h, bw, bh);
        if (rc == WAVE2D_OK) rc = encode_plane(&h->tm_prev[p], h->hi[p], h, tw, th);
    }
    h->tma_ready = (rc == WAVE2D_OK);
    return rc;
}

// Temporal kernel: region width in vectors and warps per CTA.
constexpr int kTempRVW = 64;
// Warps per CTA: 8 for tiles of 16, 24 or 32 rows (two or three CTAs share
// an SM), 16 for 64-row tiles (one CTA of 160 KB per SM, 16 warps).
template <int OH>
constexpr int temp_nw() { return OH == 64 ? 16 : 8; }

static int prepare_temporal(wave2d* h) {
    const int key = h->scheme * 10000 + h->temporal_oh * 10 + h->temporal_t;
    if (h->reg_key == key) return WAVE2D_OK;
    int rh = 0;
    dispatch_s(h->scheme, [&](auto Sc) {
        constexpr int S = decltype(Sc)::value;
        constexpr int R = (S == 13) ? 2 : 1;
        rh = h->temporal_oh + 2 * R * h->temporal_t;
    });
    for (int p = 0; p < h->nlevels; ++p) {
        int rc = encode_plane(&h->tm_reg[p], h->hi[p], h, 4 * kTempRVW, rh);
        if (rc != WAVE2D_OK) return rc;
    }
    h->reg_key = key;
    return WAVE2D_OK;
}

// ------------------------------------------------------------ exact tables
// u_e(i, j) = w0 (P_i Q_j - R_i S_j) + w1 (R_i Q_j + P_i S_j); see kernels.cuh.
static void exact_tables(const wave2d* h, const wave2d_exact& ex, std::vector<double>& tab) {
    tab.assign(2 * (size_t)h->nx + 2 * (size_t)h->ny, 0.0);
    double* P = tab.data();
    double* R = P + h->nx;
    double* Q = R + h->nx;
    double* S = Q + h->ny;
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < h->nx; ++i) {
        const double x = (i + ex.x_off) * h->h;
        if (ex.kind == WAVE2D_EXACT_STANDING) P[i] = std::sin(2.0 * pi * ex.m * x);
        else if (ex.kind == WAVE2D_EXACT_PLANE) {
            P[i] = std::cos(ex.k1 * x);
            R[i] = std::sin(ex.k1 * x);
        }
    }
    for (int j = 0; j < h->ny; ++j) {
        const double y = (j + ex.x_off) * h->h;
        if (ex.kind == WAVE2D_EXACT_STANDING) Q[j] = std::sin(2.0 * pi * ex.m * y);
        else if (ex.kind == WAVE2D_EXACT_PLANE) {
            Q[j] = std::cos(ex.k2 * y);
            S[j] = std::sin(ex.k2 * y);
        }
    }
}

static void exact_weights(const wave2d* h, const wave2d_exact& ex, double t, double& w0, double& w1) {
    const double pi = 3.14159265358979323846;
    w0 = w1 = 0.0;
    if (ex.kind == WAVE2D_EXACT_STANDING) {
        w0 = ex.amp * std::sin(2.0 * std::sqrt(2.0) * pi * ex.m * h->c * t);
    } else if (ex.kind == WAVE2D_EXACT_PLANE) {
        const double w = h->c * std::sqrt(ex.k1 * ex.k1 + ex.k2 * ex.k2);
        w0 = ex.amp * std::cos(w * t);
        w1 = ex.amp * std::sin(w * t);
    }
}

static ExactTab make_tab(const wave2d* h, const double* dev_tab, const wave2d_exact& ex, double t) {
    ExactTab et{};
    et.kind = ex.kind;
    et.P = dev_tab;
    et.R = dev_tab + h->nx;
    et.Q = dev_tab + 2 * (size_t)h->nx;
    et.S = dev_tab + 2 * (size_t)h->nx + h->ny;
    exact_weights(h, ex, t, et.w0, et.w1);
    return et;
}

static Reduce make_reduce(const wave2d* h, double* acc, int accumulate) {
    return Reduce{h->partials, h->counter, acc, h->status, accumulate};
}

// ------------------------------------------------------------ launches
static dim3 grid2d(const wave2d* h) { return dim3((h->nx + 31) / 32, (h->ny + 7) / 8); }

static int launch_first_step(wave2d* h, const double* du0, const double* dv0) {
    double ahalf[3] = {h->a[0] / 2, h->a[1] / 2, h->a[2] / 2};
    const Coef3<double> ca = coef_as<double>(ahalf), cb = coef_as<double>(h->b);
    const ExactTab ex = make_tab(h, h->tab_track, h->track_ex, h->tau);
    const Reduce rd = make_reduce(h, h->acc_track, 1);
    if (h->nclass > 0) return chain_first_step(h, du0, dv0, ex, rd);
    const Level L0 = h->level(1), L1 = h->level(0);  // u^0 -> plane 1 (u^{k-1}), u^1 -> plane 0
    dispatch_dt(h->dtype, [&](auto DTc) {
        dispatch_s(h->scheme, [&](auto Sc) {
            dispatch_bc(h->bc, [&](auto Pc) {
                dispatch_bool(h->tracking, [&](auto Tc) {
                    k1_first_step<decltype(DTc)::value, decltype(Sc)::value, decltype(Pc)::value,
                                  decltype(Tc)::value><<<grid2d(h), dim3(32, 8), 0, h->stream>>>(
                        du0, dv0, L0, L1, h->geo(), ca, cb, h->tau, ex, rd, h->gw);
                });
            });
        });
    });
    W2D_LAUNCHED("first-step kernel launch");
    return WAVE2D_OK;
}

static int launch_simple_step(wave2d* h, bool track) {
    const Level cur = h->level(h->cur), nxt = h->level(h->prv);
    const ExactTab ex = track ? make_tab(h, h->tab_track, h->track_ex, (double)(h->k + 1) * h->tau) : ExactTab{};
    const Reduce rd = make_reduce(h, h->acc_track, 1);
    if (h->nclass > 0) return chain_simple_step(h, track, ex, rd);
    // FP32x2 without per-step norms above 2^20 nodes: the packed two-node
    // kernel (the same result; measured on GB300, 13-point: 36.9 against 41.0
    // us per level at 2048^2, 129 against 167 at 4096^2, 480 against 646 at
    // 8192^2, but 8-12 % slower at 512^2 and 1024^2, where the one-node
    // kernel's occupancy wins)
    if (h->dtype == DT_F32X2 && !track && (int64_t)h->nx * h->ny > (int64_t(1) << 20))
        return df2_simple_step(h, coef_as<df>(h->a));
    dispatch_dt(h->dtype, [&](auto DTc) {
        constexpr int DT = decltype(DTc)::value;
        using V = typename St<DT>::V;
        const Coef3<V> a = coef_as<V>(h->a);
        dispatch_s(h->scheme, [&](auto Sc) {
            dispatch_bc(h->bc, [&](auto Pc) {
                dispatch_bool(track, [&](auto Tc) {
                    k2_simple<DT, decltype(Sc)::value, decltype(Pc)::value, decltype(Tc)::value>
                        <<<grid2d(h), dim3(32, 8), 0, h->stream>>>(cur, nxt, h->geo(), a, ex, rd, h->gw);
                });
            });
        });
    });
    W2D_LAUNCHED("two-step kernel launch");
    return WAVE2D_OK;
}

template <typename T, int S, int BCM>
static int launch_tma_t(wave2d* h) {
    constexpr int TH = 32;
    using C = TmaCfg<T, S, TH, kTmaNW>;
    auto kern = k2_tma<T, S, BCM, TH, kTmaNW, kTmaStages>;
    const int smem = 2048 + kTmaStages * C::STAGE_BYTES;
    static thread_local int configured_smem = -1;  // per instantiation
    if (configured_smem != smem) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(TMA kernel)");
        configured_smem = smem;
    }
    static thread_local int occ = 0;
    if (occ == 0) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kTmaNW * 32, smem);
        if (e != cudaSuccess || occ < 1) occ = 1;
    }
    const int tiles_x = (h->nx + C::TW - 1) / C::TW;
    const int tiles_y = (h->ny + TH - 1) / TH;
    const int n_tiles = tiles_x * tiles_y;
    int per_sm = h->tune.ctas_per_sm;
    if (per_sm <= 0) per_sm = (2.0 * (double)h->plane_bytes <= 1.25 * (double)h->l2_bytes) ? occ : 1;
    per_sm = std::max(1, std::min(per_sm, occ));
    const int grid = std::min(n_tiles, per_sm * h->num_sms);
    kern<<<grid, kTmaNW * 32, smem, h->stream>>>(h->tm_cur[h->cur], h->tm_prev[h->prv],
                                                 reinterpret_cast<T*>(h->hi[h->prv]), h->geo(),
                                                 coef_as<T>(h->a), tiles_x, n_tiles, h->gw, h->status);
    W2D_LAUNCHED("TMA two-step kernel launch");
    return WAVE2D_OK;
}

static int launch_tma_step(wave2d* h) {
    if (h->nclass > 0) return chain_tma_step(h);
    int rc = WAVE2D_OK;
    dispatch_s(h->scheme, [&](auto Sc) {
        constexpr int S = decltype(Sc)::value;
        dispatch_bc(h->bc, [&](auto Pc) {
            constexpr int P = decltype(Pc)::value;
            rc = (h->dtype == DT_F32) ? launch_tma_t<float, S, P>(h) : launch_tma_t<double, S, P>(h);
        });
    });
    return rc;
}

// T two-steps in one launch, out of place into the other pair of planes.
template <int S, bool PER, int OH, int T>
static int launch_temporal_t(wave2d* h) {
    using C = TemporalCfg<S, kTempRVW, OH, T>;
    constexpr int kTempNW = temp_nw<OH>();
    auto kern = k3_temporal<S, PER, kTempRVW, OH, T, kTempNW>;
    const int smem = 1024 + 2 * C::BUF_BYTES;
    static thread_local bool configured = false;  // per instantiation
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(temporal kernel)");
        configured = true;
    }
    // The levels move to the other pair with their roles kept (plane p -> p ^ 2),
    // so two launches bring every level back to its plane.
    const int oc = h->cur ^ 2, op = h->prv ^ 2;
    const int tiles_x = (h->nx + C::OW - 1) / C::OW;
    const int tiles_y = (h->ny + OH - 1) / OH;
    kern<<<tiles_x * tiles_y, kTempNW * 32, smem, h->stream>>>(
        h->tm_reg[h->cur], h->tm_reg[h->prv], reinterpret_cast<float*>(h->hi[oc]),
        reinterpret_cast<float*>(h->hi[op]), h->geo(), coef_as<float>(h->a), tiles_x, h->gw, h->status);
    W2D_LAUNCHED("temporal two-step kernel launch");
    h->cur = oc;
    h->prv = op;
    return WAVE2D_OK;
}

static int launch_temporal(wave2d* h) {
    int rc = WAVE2D_OK;
    dispatch_s(h->scheme, [&](auto Sc) {
        constexpr int S = decltype(Sc)::value;
        dispatch_bool(h->bc == WAVE2D_BC_PERIODIC, [&](auto Pc) {
            constexpr bool P = decltype(Pc)::value;
            const int T = h->temporal_t, OH = h->temporal_oh;
            auto by_oh = [&](auto Tc) {
                constexpr int TT = decltype(Tc)::value;
                switch (OH) {
                    case 16: rc = launch_temporal_t<S, P, 16, TT>(h); break;
                    case 24: rc = launch_temporal_t<S, P, 24, TT>(h); break;
                    case 64: rc = launch_temporal_t<S, P, 64, TT>(h); break;
                    default: rc = launch_temporal_t<S, P, 32, TT>(h); break;
                }
            };
            if (T == 2) by_oh(IC<2>{});
            else if (T == 3) by_oh(IC<3>{});
            else by_oh(IC<4>{});
        });
    });
    return rc;
}

// Advance by one launch: T levels for the temporal kernel when at least T
// remain, else one level.  Returns the number of levels advanced (< 0: error).
// All n levels in one cooperative launch of k2_persist (grid barrier between
// levels), blocks capped at the number that can be resident at once.
template <int DT, int S, int BCM>
static int launch_persist_t(wave2d* h, int n) {
    auto kern = k2_persist<DT, S, BCM>;
    static int per_sm = -1;  // resident blocks of 512 threads per SM for this instantiation
    if (per_sm < 0) {
        int v = 0;
        W2D_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kern, 512, 0), "occupancy query");
        per_sm = std::max(1, v);
    }
    // One block per SM with the nodes spread evenly (blocks of 64 .. 512
    // threads), more blocks of 512 only where a block per SM cannot hold a
    // node per thread: every SM then carries the same share of a level (at
    // 256^2 FP64 the level's arithmetic, not memory, sets its length, and
    // 256 blocks on 152 SMs gave two thirds of the SMs twice the work).
    const long long nn = (long long)h->nx * h->ny;
    const long long per_block = (nn + h->num_sms - 1) / h->num_sms;
    const int threads = (int)std::min<long long>(512, std::max<long long>(64, (per_block + 31) / 32 * 32));
    const int blocks = (int)std::max<long long>(
        1, std::min<long long>((nn + threads - 1) / threads, (long long)per_sm * h->num_sms));
    unsigned long long* arrived = reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(h->counter) + 128);
    W2D_CUDA(cudaMemsetAsync(arrived, 0, sizeof(unsigned long long), h->stream), "barrier reset");
    Level A = h->level(h->cur), B = h->level(h->prv);
    Geo g = h->geo();
    Coef3<typename St<DT>::V> a = coef_as<typename St<DT>::V>(h->a);
    int* status = h->status;
    int gw = h->gw;
    long long limit = kWaitLimitCycles;
    void* args[] = {&A, &B, &g, &a, &n, &arrived, &status, &gw, &limit};
    W2D_CUDA(cudaLaunchCooperativeKernel((const void*)kern, dim3(blocks), dim3(threads), args, 0, h->stream),
             "persistent kernel launch");
    W2D_LAUNCHED("persistent kernel launch");
    return WAVE2D_OK;
}

static int launch_persist(wave2d* h, int n) {
    int rc = WAVE2D_OK;
    dispatch_dt(h->dtype, [&](auto DTc) {
        dispatch_s(h->scheme, [&](auto Sc) {
            constexpr int DT = decltype(DTc)::value, S = decltype(Sc)::value;
            if (h->bc == WAVE2D_BC_PERIODIC) rc = launch_persist_t<DT, S, BCM_PERIODIC>(h, n);
            else if (h->bc == WAVE2D_BC_ODD) rc = launch_persist_t<DT, S, BCM_ODD>(h, n);
            else rc = launch_persist_t<DT, S, BCM_ZERO>(h, n);
        });
    });
    if (rc != WAVE2D_OK) return rc;
    if (n & 1) std::swap(h->cur, h->prv);
    h->k += n;
    return WAVE2D_OK;
}

static int launch_block(wave2d* h, int64_t remaining) {
    int rc;
    if (h->kernel == WAVE2D_KERNEL_STREAM && remaining >= h->temporal_t) {
        rc = stream_launch(h);
        if (rc != WAVE2D_OK) return rc;
        h->k += h->temporal_t;
        return h->temporal_t;
    }
    rc = stream_fresh_rings(h);  // the kernels below read the ghost rings
    if (rc != WAVE2D_OK) return rc;
    if (h->kernel == WAVE2D_KERNEL_TEMPORAL && remaining >= h->temporal_t) {
        rc = launch_temporal(h);
        if (rc != WAVE2D_OK) return rc;
        h->k += h->temporal_t;
        return h->temporal_t;
    }
    if (h->kernel == WAVE2D_KERNEL_TMA || is_multilevel(h->kernel)) rc = launch_tma_step(h);
    else rc = launch_simple_step(h, false);
    if (rc != WAVE2D_OK) return rc;
    std::swap(h->cur, h->prv);
    h->k += 1;
    return 1;
}

// Rewrite the periodic images of the current two levels in the first gw rings.
static int refresh_ghosts(wave2d* h) {
    if (h->bc == WAVE2D_BC_ZERO || !h->initialized) return WAVE2D_OK;
    const long long total = (long long)(h->nx + 2 * h->gw) * (h->ny + 2 * h->gw);
    const int grid = (int)std::min<long long>((total + 255) / 256, 8LL * h->num_sms);
    for (int p : {h->cur, h->prv}) {
        dispatch_dt(h->dtype, [&](auto DTc) {
            if (h->bc == WAVE2D_BC_ODD)
                k_refresh_ghosts<decltype(DTc)::value, BCM_ODD><<<grid, 256, 0, h->stream>>>(h->level(p), h->geo(), h->gw);
            else
                k_refresh_ghosts<decltype(DTc)::value, BCM_PERIODIC><<<grid, 256, 0, h->stream>>>(h->level(p), h->geo(),
                                                                                                  h->gw);
        });
        W2D_LAUNCHED("ghost refresh kernel launch");
    }
    return WAVE2D_OK;
}

static void drop_graphs(wave2d* h) {
    for (auto& g : h->graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    h->graph_steps = 0;
}

static int select_kernel(wave2d* h) {
    int want = h->tune.kernel;
    if (want == WAVE2D_KERNEL_AUTO) {
        // FP32: the streaming kernel wherever it applies, the TMA kernel for
        // other handles, from 65536 nodes.  Measured on GB300 (periodic,
        // streaming with its default depth and strip rows): the Section 6
        // schemes 1.4-2.0x faster than the TMA kernel and 1.1-1.5x faster than
        // the tiled temporal kernel at 256^2 - 768^2, 1.1-1.7x (temporal) at
        // 1024^2, 1.4-2.2x at 2048^2, 1.3-2.3x at 4096^2; the class chains of
        // up to three classes (which have no tiled temporal kernel) 1.1-1.9x
        // faster than their one-level TMA kernel at 512^2 and 1024^2, 1.5-2.1x
        // at 2048^2, 1.6-3.1x at 4096^2.  The tiled temporal kernel stays
        // available by name and to the autotuner.  FP64 and FP32x2 are bound
        // by arithmetic on GB300 (measured: the one-node kernel is as fast at
        // 4096^2 and 2.4x faster at 256^2), so they keep it.
        const int64_t nodes = (int64_t)h->nx * h->ny;
        want = (h->dtype != DT_F32 || nodes < 65536) ? WAVE2D_KERNEL_SIMPLE
               : stream_ok(h)                        ? WAVE2D_KERNEL_STREAM
                                                     : WAVE2D_KERNEL_TMA;
    }
    if (want == WAVE2D_KERNEL_TEMPORAL && (h->dtype != DT_F32 || !multilevel_ok(h))) want = WAVE2D_KERNEL_TMA;
    if (want == WAVE2D_KERNEL_STREAM && !stream_ok(h)) want = WAVE2D_KERNEL_TMA;
    if (want == WAVE2D_KERNEL_PERSISTENT && (h->nclass > 0 || h->diff_sums || h->diff_form))
        want = WAVE2D_KERNEL_SIMPLE;
    if (want == WAVE2D_KERNEL_TMA && h->dtype == DT_F32X2) want = WAVE2D_KERNEL_SIMPLE;
    if ((want == WAVE2D_KERNEL_TMA || is_multilevel(want)) && !h->tma_ready) {
        int rc = prepare_tma(h);  // the multi-level kernels finish runs with single TMA steps
        if (rc != WAVE2D_OK) return rc;
    }
    if (want == WAVE2D_KERNEL_STREAM) {
        // default depth: 6 levels per launch for the radius-1 schemes (their
        // halo columns round up to 8 for any T in 5..8, so deeper blocking
        // costs no extra columns; measured on GB300 at 4096^2: 9-point level
        // 13.4 us at T = 4, 11.7 at T = 6), 4 for the 13-point scheme (its
        // registers allow no deeper ring at 4 CTAs per SM)
        // (difference form: 4 levels, 3 for the 13-point stencil, whose d
        // rows take the registers of a deeper ring)
        const int tt = h->tune.temporal_t;
        const bool r2 = h->nclass == 0 ? h->scheme == 13 : h->nclass == 3;  // the 13-point stencil
        if (h->diff_form)
            h->temporal_t = (tt >= 2 && tt <= 4) ? tt : (r2 ? 3 : 4);
        else
            h->temporal_t = ((tt >= 2 && tt <= 4) || tt == 6) ? tt : (r2 ? 4 : 6);
        // rows per strip by default: the most of 64, 32 and 16 that still
        // makes at least 6 strips per SM (measured on GB300: the 2RT rows a
        // strip recomputes at its start cost less than a second wave of
        // strips, but a grid of too few strips leaves SMs idle; 4096^2 takes
        // 64 rows, 2368 strips; 2048^2 32 rows; 1024^2 and below 16)
        if (h->tune.tile_h > 0) {
            h->temporal_oh = h->tune.tile_h;
        } else {
            const int hx = (h->R * h->temporal_t + 3) / 4 * 4, ow = 128 - 2 * hx;
            const int64_t sx = (h->nx + ow - 1) / ow, want_strips = 6 * (int64_t)h->num_sms;
            h->temporal_oh = sx * ((h->ny + 63) / 64) >= want_strips   ? 64
                             : sx * ((h->ny + 31) / 32) >= want_strips ? 32
                                                                       : 16;
        }
    }
    if (want == WAVE2D_KERNEL_TEMPORAL) {
        const int tt = h->tune.temporal_t;
        h->temporal_t = (tt >= 2 && tt <= 4) ? tt : 4;
        // default tile rows: the autotuner's choice on GB300 (3 CTAs per SM for
        // the 9-point scheme, 2 for the others)
        h->temporal_oh = h->tune.tile_h > 0 ? h->tune.tile_h : (h->scheme == 9 ? 24 : 32);
        int rc = prepare_temporal(h);
        if (rc != WAVE2D_OK) return rc;
    }
    // Periodic images: one-level kernels read R nodes beyond an edge, the
    // temporal kernel up to the full ghost ring.
    const int gw = is_multilevel(want) ? h->G : h->R;
    const bool deeper = gw > h->gw;
    h->gw = gw;
    h->kernel = want;
    drop_graphs(h);
    if (deeper) return refresh_ghosts(h);
    return WAVE2D_OK;
}

static bool want_graph(const wave2d* h, int64_t n) {
    if (h->tune.use_graph == 0) return false;
    if (h->tune.use_graph > 0) return n >= 2;
    return n >= 64 && (int64_t)h->nx * h->ny <= (1 << 22);
}

constexpr int kGraphSteps = 48;

// A graph of kGraphSteps levels (a multiple of 2 T for every depth the
// multi-level kernels take) returns the levels to the planes they started
// in, so one graph per starting (cur, prv, dpl) is replayed.
static int run_graph(wave2d* h, int64_t& n) {
    const int key = h->plane_key();
    static_assert(kGraphSteps % 4 == 0 && kGraphSteps % 6 == 0 && kGraphSteps % 8 == 0 && kGraphSteps % 12 == 0,
                  "graph length must be a multiple of 2T");
    if (!h->graph[key]) {
        const int64_t k0 = h->k;
        cudaGraph_t g = nullptr;
        W2D_CUDA(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
        const int64_t before = g_launches.load();
        int64_t done = 0;
        int rc = WAVE2D_OK;
        while (done < kGraphSteps) {
            const int adv = launch_block(h, kGraphSteps - done);
            if (adv < 0) {
                rc = adv;
                break;
            }
            done += adv;
        }
        if (rc == WAVE2D_OK) rc = stream_fresh_rings(h);  // a replay ends with valid rings
        const int64_t launched = g_launches.load() - before;
        cudaError_t e = cudaStreamEndCapture(h->stream, &g);
        g_launches.store(before);  // captured launches run only when the graph does
        h->graph_end[key] = h->plane_key();
        h->set_plane_key(key);
        h->k = k0;
        if (rc != WAVE2D_OK) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) return cuda_fail(e, "end capture");
        e = cudaGraphInstantiate(&h->graph[key], g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
        h->graph_steps = (int)launched;
    }
    if (h->graph_end[key] != key) {
        // The captured run does not end where it started: replay it once.
        if (n >= kGraphSteps) {
            W2D_CUDA(cudaGraphLaunch(h->graph[key], h->stream), "graph launch");
            g_launches.fetch_add(h->graph_steps);
            h->set_plane_key(h->graph_end[key]);
            h->k += kGraphSteps;
            n -= kGraphSteps;
        }
        return WAVE2D_OK;
    }
    while (n >= kGraphSteps) {
        W2D_CUDA(cudaGraphLaunch(h->graph[key], h->stream), "graph launch");
        g_launches.fetch_add(h->graph_steps);
        h->k += kGraphSteps;
        n -= kGraphSteps;
    }
    return WAVE2D_OK;
}

static bool valid_exact(const wave2d_exact* ex) {
    return ex && (ex->kind == WAVE2D_EXACT_NONE || ex->kind == WAVE2D_EXACT_STANDING ||
                  ex->kind == WAVE2D_EXACT_PLANE) &&
           std::isfinite(ex->amp) && std::isfinite(ex->m) && std::isfinite(ex->k1) &&
           std::isfinite(ex->k2) && std::isfinite(ex->x_off);
}

static int check_status(wave2d* h) {
    int st = 0;
    W2D_CUDA(cudaMemcpyAsync(&st, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream), "status copy");
    W2D_CUDA(cudaStreamSynchronize(h->stream), "stream synchronize");
    if (st & STATUS_TIMEOUT) {
        cudaMemsetAsync(h->status, 0, sizeof(int), h->stream);
        return set_error(WAVE2D_ERR_TIMEOUT, "a device-side wait exceeded its limit");
    }
    return WAVE2D_OK;
}

// out = a - b (FP64), for the conversions between (u^{k-1}, u^k) and the
// difference form's (d^k, u^k).
__global__ void k_combine(const double* a, const double* b, double* out, size_t n) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = __dsub_rn(a[i], b[i]);
}

// Self-test of the bounded wait: an mbarrier that nothing ever completes is
// waited on with a short limit; the wait gives up, raises STATUS_TIMEOUT and
// the kernel returns.  No copy is in flight, so nothing needs draining.
__global__ void k_selftest_wait(int* status, long long limit) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_barrier_init();
    }
    __syncthreads();
    mbar_wait_bounded(&bar, 0, status, limit);
}

}  // namespace w2d

using namespace w2d;

// ======================================================================
// C ABI
// ======================================================================
extern "C" {

const char* wave2d_last_error(void) { return t_err.c_str(); }

int64_t wave2d_launch_count(void) { return g_launches.load(); }

double wave2d_lambda_max(int scheme, int conventional) { return lambda_max_of(scheme, conventional != 0); }

int wave2d_set_allocator(wave2d_alloc_fn alloc, wave2d_free_fn release, void* ctx) {
    if ((alloc == nullptr) != (release == nullptr))
        return set_error(WAVE2D_ERR_ARG, "allocator hook needs both alloc and free (or neither)");
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_alloc.alloc = alloc;
    g_alloc.release = release;
    g_alloc.ctx = alloc ? ctx : nullptr;
    return WAVE2D_OK;
}

static void release_handle(wave2d* h) {
    if (!h) return;
    drop_graphs(h);
    if (h->base) {
        dev_free(h->alloc, h->base, h->base_bytes, h->stream);
        cudaStreamSynchronize(h->stream);
    }
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

// Validation shared by both constructors.
static int check_grid(const wave2d_grid* grid, double hh, double tau, double c, int allowed_flags) {
    if (grid->nx < 1 || grid->ny < 1 || grid->nx > 65536 || grid->ny > 65536)
        return set_error(WAVE2D_ERR_ARG, "grid size %d x %d outside 1..65536", grid->nx, grid->ny);
    if (grid->bc != WAVE2D_BC_ZERO && grid->bc != WAVE2D_BC_PERIODIC && grid->bc != WAVE2D_BC_ODD)
        return set_error(WAVE2D_ERR_ARG, "unknown boundary condition %d", grid->bc);
    if (grid->dtype != WAVE2D_F64 && grid->dtype != WAVE2D_F32 && grid->dtype != WAVE2D_F32X2)
        return set_error(WAVE2D_ERR_ARG, "unknown dtype %d", grid->dtype);
    if (grid->flags & ~allowed_flags) return set_error(WAVE2D_ERR_ARG, "unsupported flags 0x%x", grid->flags);
    if ((grid->flags & WAVE2D_DIFF_SUMS) && grid->dtype == WAVE2D_F32X2)
        return set_error(WAVE2D_ERR_ARG, "difference sums are available for F32 and F64 storage");
    if ((grid->flags & WAVE2D_DIFF_FORM) && grid->dtype != WAVE2D_F32)
        return set_error(WAVE2D_ERR_ARG, "the difference form is available for F32 storage");
    if (!(hh > 0) || !(tau > 0) || !(c > 0) || !std::isfinite(hh) || !std::isfinite(tau) || !std::isfinite(c))
        return set_error(WAVE2D_ERR_ARG, "h, tau and c must be positive and finite");
    return WAVE2D_OK;
}

// Device side of a new handle whose problem fields (sizes, scheme,
// coefficients, radius) are set: stream, level planes, scratch, kernel.
static int create_device_state(wave2d* h, const wave2d_grid* grid) {
    h->alloc = current_allocator();
    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->l2_bytes, cudaDevAttrL2CacheSize, h->device);
    if (e != cudaSuccess) return cuda_fail(e, "no usable CUDA device");
    h->stream = (cudaStream_t)grid->stream;
    if (!h->stream) {
        e = cudaStreamCreate(&h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "stream create");
        h->own_stream = true;
    }

    // Layout: level planes, then scratch.  FP32 keeps two pairs of levels
    // (the temporal kernel writes out of place); FP32x2 keeps hi and lo
    // planes of two levels; FP64 two levels.
    h->elem = (h->dtype == WAVE2D_F64) ? 8 : 4;
    // FP32: a second pair of planes for the out-of-place multi-level kernels
    // (the Section 6 schemes and class chains of up to three classes); the
    // difference form keeps u^k and d^k, each with a second plane
    h->nlevels = (h->dtype == WAVE2D_F32 && (h->nclass <= 3 || h->diff_form)) ? 4 : 2;
    h->gw = h->R;
    h->G = kGhost;
    h->pitch = (int)round_up((size_t)h->nx + 2 * kGhost, 32);
    h->rows = h->ny + 2 * kGhost;
    h->plane_bytes = round_up((size_t)h->pitch * h->rows * h->elem, 1024);
    const int nplanes = (h->dtype == WAVE2D_F32X2) ? 4 : h->nlevels;
    const size_t k2_blocks = (size_t)((h->nx + 31) / 32) * ((h->ny + 7) / 8);
    h->partial_blocks = std::max<size_t>(k2_blocks, 64 * 1024);
    const size_t tab_doubles = 2 * (size_t)h->nx + 2 * (size_t)h->ny;
    const size_t scratch = round_up(h->partial_blocks * 4 * sizeof(double), 256) + 256 /*counter*/ +
                           256 /*acc_eval*/ + 256 /*acc_track*/ + 256 /*status*/ +
                           2 * round_up(tab_doubles * sizeof(double), 256);
    h->base_bytes = nplanes * h->plane_bytes + scratch;
    h->base = dev_alloc(h->alloc, h->base_bytes, h->stream);
    if (!h->base) return set_error(WAVE2D_ERR_OOM, "device allocation of %zu bytes failed", h->base_bytes);
    char* p = (char*)h->base;
    for (int q = 0; q < h->nlevels; ++q) h->hi[q] = p + q * h->plane_bytes;
    if (h->dtype == WAVE2D_F32X2)
        for (int q = 0; q < 2; ++q) h->lo[q] = p + (2 + q) * h->plane_bytes;
    p += nplanes * h->plane_bytes;
    h->partials = (double*)p;
    p += round_up(h->partial_blocks * 4 * sizeof(double), 256);
    h->counter = (unsigned*)p;
    p += 256;
    h->acc_eval = (double*)p;
    p += 256;
    h->acc_track = (double*)p;
    p += 256;
    h->status = (int*)p;
    p += 256;
    h->tab_eval = (double*)p;
    p += round_up(tab_doubles * sizeof(double), 256);
    h->tab_track = (double*)p;
    e = cudaMemsetAsync(h->base, 0, h->base_bytes, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "memset");
    int rc = canary_fill(h);
    if (rc != WAVE2D_OK) return rc;
    return select_kernel(h);
}

static void set_problem(wave2d* h, const wave2d_grid* grid, double hh, double tau, double c) {
    h->nx = grid->nx;
    h->ny = grid->ny;
    h->bc = grid->bc;
    h->dtype = grid->dtype;
    h->flags = grid->flags;
    h->h = hh;
    h->tau = tau;
    h->c = c;
    h->lam = c * tau / hh;
}

int wave2d_create(const wave2d_grid* grid, double hh, double tau, double c, int scheme, wave2d_t* out) {
    NvtxRange nvtx_range("wave2d_create");
    if (!grid || !out) return set_error(WAVE2D_ERR_ARG, "null argument");
    *out = nullptr;
    if (scheme != 5 && scheme != 9 && scheme != 13)
        return set_error(WAVE2D_ERR_ARG, "scheme must be 5, 9 or 13 (got %d)", scheme);
    int rc = check_grid(grid, hh, tau, c,
                        WAVE2D_ALLOW_UNSTABLE | WAVE2D_CONVENTIONAL | WAVE2D_DIFF_SUMS | WAVE2D_DIFF_FORM |
                            WAVE2D_CANARY);
    if (rc != WAVE2D_OK) return rc;
    const bool conventional = (grid->flags & WAVE2D_CONVENTIONAL) != 0;
    const double lam = c * tau / hh;
    const double lmax = lambda_max_of(scheme, conventional);
    if (lam > lmax * (1.0 + 1e-12) && !(grid->flags & WAVE2D_ALLOW_UNSTABLE))
        return set_error(WAVE2D_ERR_UNSTABLE, "Courant number %.17g exceeds the stability limit %.17g of the %d-point scheme",
                         lam, lmax, scheme);

    wave2d* h = new (std::nothrow) wave2d();
    if (!h) return set_error(WAVE2D_ERR_OOM, "host allocation failed");
    set_problem(h, grid, hh, tau, c);
    h->scheme = scheme;
    h->R = scheme == 13 ? 2 : 1;
    h->npoints = scheme;
    h->lam_max = lmax;
    scheme_coefficients(scheme, conventional, lam, h->a, h->b);
    if (grid->flags & (WAVE2D_DIFF_SUMS | WAVE2D_DIFF_FORM)) {
        // The class-chain kernels carry the difference sums and form: the
        // Section 6 scheme is its first one, two or three classes.
        h->diff_sums = true;
        h->diff_form = (grid->flags & WAVE2D_DIFF_FORM) != 0;
        h->nclass = scheme == 5 ? 1 : scheme == 9 ? 2 : 3;
        for (int q = 0; q < 3; ++q) {
            h->ca[q] = h->a[q];
            h->cb[q] = h->b[q];
        }
    }
    rc = create_device_state(h, grid);
    if (rc != WAVE2D_OK) {
        release_handle(h);
        return rc;
    }
    *out = h;
    return WAVE2D_OK;
}

int wave2d_create_scheme(const wave2d_grid* grid, double hh, double tau, double c, const wave2d_scheme* s,
                         wave2d_t* out) {
    NvtxRange nvtx_range("wave2d_create_scheme");
    if (!grid || !out) return set_error(WAVE2D_ERR_ARG, "null argument");
    *out = nullptr;
    int rc = check_scheme(s);
    if (rc != WAVE2D_OK) return rc;
    rc = check_grid(grid, hh, tau, c, WAVE2D_ALLOW_UNSTABLE | WAVE2D_DIFF_SUMS | WAVE2D_DIFF_FORM | WAVE2D_CANARY);
    if (rc != WAVE2D_OK) return rc;
    const double lam = c * tau / hh;
    const double lmax = scheme_lambda_max(s);
    if (lam > lmax * (1.0 + 1e-12) && !(grid->flags & WAVE2D_ALLOW_UNSTABLE))
        return set_error(WAVE2D_ERR_UNSTABLE, "Courant number %.17g exceeds the stability limit %.17g of the derived scheme",
                         lam, lmax);
    wave2d* h = new (std::nothrow) wave2d();
    if (!h) return set_error(WAVE2D_ERR_OOM, "host allocation failed");
    set_problem(h, grid, hh, tau, c);
    h->scheme = 0;
    h->diff_form = (grid->flags & WAVE2D_DIFF_FORM) != 0;
    h->diff_sums = (grid->flags & (WAVE2D_DIFF_SUMS | WAVE2D_DIFF_FORM)) != 0;
    h->nclass = s->n_classes;
    h->R = chain_radius(s->n_classes);
    h->npoints = chain_points(s->n_classes);
    if (s->n_points > 0) h->npoints = s->n_points;
    h->lam_max = lmax;
    for (int q = 0; q < s->n_classes; ++q) {
        h->ca[q] = poly_at(s->a[q], lam);
        h->cb[q] = poly_at(s->b[q], lam);
    }
    for (int q = 0; q < 3 && q < s->n_classes; ++q) {
        h->a[q] = h->ca[q];
        h->b[q] = h->cb[q];
    }
    rc = create_device_state(h, grid);
    if (rc != WAVE2D_OK) {
        release_handle(h);
        return rc;
    }
    *out = h;
    return WAVE2D_OK;
}

void wave2d_destroy(wave2d_t h) { release_handle(h); }

int wave2d_set_tuning(wave2d_t h, const wave2d_tune* tune) {
    if (!h || !tune) return set_error(WAVE2D_ERR_ARG, "null argument");
    if (tune->kernel < 0 || tune->kernel > WAVE2D_KERNEL_PERSISTENT)
        return set_error(WAVE2D_ERR_ARG, "unknown kernel %d", tune->kernel);
    if (tune->kernel == WAVE2D_KERNEL_PERSISTENT && (h->nclass > 0 || h->diff_sums || h->diff_form))
        return set_error(WAVE2D_ERR_ARG, "the persistent kernel covers the 5-, 9- and 13-point schemes with plain sums");
    if (tune->kernel == WAVE2D_KERNEL_TMA && h->dtype == WAVE2D_F32X2)
        return set_error(WAVE2D_ERR_ARG, "the TMA kernel supports F32 and F64 storage only");
    const bool multi = is_multilevel(tune->kernel);
    if (multi && (h->flags & WAVE2D_CANARY) && h->bc != WAVE2D_BC_ZERO)
        return set_error(WAVE2D_ERR_ARG,
                         "with guard-band canaries the temporal kernels take the zero boundary only (periodic "
                         "images fill the whole ghost ring)");
    if (multi && h->bc == WAVE2D_BC_ODD)
        return set_error(WAVE2D_ERR_ARG, "the temporal kernels cover the zero and periodic boundaries");
    if (tune->kernel == WAVE2D_KERNEL_TEMPORAL && h->nclass > 0)
        return set_error(WAVE2D_ERR_ARG,
                         "the tiled temporal kernel covers the 5-, 9- and 13-point schemes with plain sums only");
    if (tune->kernel == WAVE2D_KERNEL_STREAM && h->nclass > 3)
        return set_error(WAVE2D_ERR_ARG, "the streaming kernel covers stencils of at most three classes (13 points)");
    if (tune->kernel == WAVE2D_KERNEL_STREAM && h->diff_form && !stream_ok(h))
        return set_error(WAVE2D_ERR_ARG,
                         "difference-form streaming takes the zero boundary or a periodic grid with nx %% 4 == 0, "
                         "ny >= 16");
    if (tune->kernel == WAVE2D_KERNEL_STREAM && h->diff_form && tune->temporal_t > 4)
        return set_error(WAVE2D_ERR_ARG, "temporal_t of difference-form streaming must be 0 (auto), 2, 3 or 4 (got %d)",
                         tune->temporal_t);
    if (tune->kernel == WAVE2D_KERNEL_TEMPORAL &&
        !(tune->temporal_t == 0 || (tune->temporal_t >= 2 && tune->temporal_t <= 4)))
        return set_error(WAVE2D_ERR_ARG, "temporal_t of the tiled kernel must be 0 (auto), 2, 3 or 4 (got %d)",
                         tune->temporal_t);
    if (tune->kernel == WAVE2D_KERNEL_STREAM &&
        !(tune->temporal_t == 0 || (tune->temporal_t >= 2 && tune->temporal_t <= 4) || tune->temporal_t == 6))
        return set_error(WAVE2D_ERR_ARG, "temporal_t of the streaming kernel must be 0 (auto), 2, 3, 4 or 6 (got %d)",
                         tune->temporal_t);
    if (tune->kernel == WAVE2D_KERNEL_TEMPORAL && !(tune->tile_h == 0 || tune->tile_h == 16 ||
                                                    tune->tile_h == 24 || tune->tile_h == 32 || tune->tile_h == 64))
        return set_error(WAVE2D_ERR_ARG, "temporal tile_h must be 0 (auto), 16, 24, 32 or 64 (got %d)", tune->tile_h);
    if (tune->kernel == WAVE2D_KERNEL_STREAM && !(tune->tile_h == 0 || (tune->tile_h >= 8 && tune->tile_h <= 4096)))
        return set_error(WAVE2D_ERR_ARG, "streaming strip rows must be 0 (auto) or 8 .. 4096 (got %d)", tune->tile_h);
    if (tune->ctas_per_sm < 0 || tune->ctas_per_sm > 32)
        return set_error(WAVE2D_ERR_ARG, "ctas_per_sm must be 0 (auto) or 1..32");
    h->tune = *tune;
    return select_kernel(h);
}

int wave2d_get_info(wave2d_t h, wave2d_info_t* info) {
    if (!h || !info) return set_error(WAVE2D_ERR_ARG, "null argument");
    std::memset(info, 0, sizeof *info);
    info->lambda = h->lam;
    info->h = h->h;
    info->tau = h->tau;
    info->c = h->c;
    for (int q = 0; q < 3; ++q) {
        info->a[q] = h->a[q];
        info->b[q] = h->b[q];
    }
    info->lambda_max = h->lam_max;
    info->k = h->k;
    info->scheme = h->scheme;
    info->radius = h->R;
    info->dtype = h->dtype;
    info->bc = h->bc;
    info->nx = h->nx;
    info->ny = h->ny;
    info->pitch = h->pitch;
    info->ghost = h->G;
    info->device_bytes = (int64_t)h->base_bytes;
    info->kernel = h->kernel;
    info->temporal_t = is_multilevel(h->kernel) ? h->temporal_t : 1;
    info->n_classes = h->nclass;
    info->n_points = h->npoints;
    for (int q = 0; q < 8; ++q) {
        info->class_a[q] = h->ca[q];
        info->class_b[q] = h->cb[q];
    }
    return WAVE2D_OK;
}

int wave2d_track_error(wave2d_t h, const wave2d_exact* ex) {
    if (!h) return set_error(WAVE2D_ERR_ARG, "null handle");
    if (!ex) {
        h->tracking = false;
        return WAVE2D_OK;
    }
    if (!valid_exact(ex)) return set_error(WAVE2D_ERR_ARG, "invalid exact-solution description");
    h->track_ex = *ex;
    std::vector<double> tab;
    exact_tables(h, *ex, tab);
    W2D_CUDA(cudaMemcpyAsync(h->tab_track, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice,
                             h->stream),
             "exact table upload");
    W2D_CUDA(cudaStreamSynchronize(h->stream), "stream synchronize");
    h->tracking = true;
    return WAVE2D_OK;
}

int wave2d_first_step(wave2d_t h, const double* u0, const double* v0, int on_device) {
    NvtxRange nvtx_range("wave2d_first_step");
    if (!h || !u0 || !v0) return set_error(WAVE2D_ERR_ARG, "null argument");
    const size_t n = (size_t)h->nx * h->ny;
    const double* du0 = u0;
    const double* dv0 = v0;
    void* stage = nullptr;
    if (!on_device) {
        stage = dev_alloc(h->alloc, 2 * n * sizeof(double), h->stream);
        if (!stage) return set_error(WAVE2D_ERR_OOM, "staging allocation failed");
        W2D_CUDA(cudaMemcpyAsync(stage, u0, n * sizeof(double), cudaMemcpyHostToDevice, h->stream), "u0 upload");
        W2D_CUDA(cudaMemcpyAsync((double*)stage + n, v0, n * sizeof(double), cudaMemcpyHostToDevice, h->stream),
                 "v0 upload");
        du0 = (const double*)stage;
        dv0 = (const double*)stage + n;
    }
    W2D_CUDA(cudaMemsetAsync(h->acc_track, 0, 4 * sizeof(double), h->stream), "reset accumulators");
    h->dpl = 2;  // difference form: d^1 goes to plane 2
    int rc = launch_first_step(h, du0, dv0);
    if (stage) dev_free(h->alloc, stage, 2 * n * sizeof(double), h->stream);
    if (rc != WAVE2D_OK) return rc;
    h->cur = 0;  // plane 0 holds u^1, plane 1 holds u^0
    h->prv = 1;
    h->k = 1;
    h->initialized = true;
    drop_graphs(h);
    return WAVE2D_OK;
}

int wave2d_step_n(wave2d_t h, int64_t n) {
    NvtxRange nvtx_range("wave2d_step_n");
    if (!h) return set_error(WAVE2D_ERR_ARG, "null handle");
    if (n < 0) return set_error(WAVE2D_ERR_ARG, "negative step count");
    if (!h->initialized) return set_error(WAVE2D_ERR_STATE, "step_n before first_step or set_state");
    if (h->tracking) {
        for (int64_t s = 0; s < n; ++s) {
            int rc = launch_simple_step(h, true);
            if (rc != WAVE2D_OK) return rc;
            std::swap(h->cur, h->prv);
            h->k += 1;
        }
        return WAVE2D_OK;
    }
    if (h->kernel == WAVE2D_KERNEL_PERSISTENT) {
        int rc = stream_fresh_rings(h);
        while (rc == WAVE2D_OK && n > 0) {
            const int m = (int)std::min<int64_t>(n, 1 << 30);
            rc = launch_persist(h, m);
            n -= m;
        }
        return rc;
    }
    if (want_graph(h, n)) {
        int rc = run_graph(h, n);
        if (rc != WAVE2D_OK) return rc;
    }
    while (n > 0) {
        const int adv = launch_block(h, n);
        if (adv < 0) return adv;
        n -= adv;
    }
    return stream_fresh_rings(h);
}

int wave2d_error_vs_exact(wave2d_t h, const wave2d_exact* ex, double* rel_l2, double* rel_linf,
                          double* spacetime_E) {
    NvtxRange nvtx_range("wave2d_error_vs_exact");
    if (!h) return set_error(WAVE2D_ERR_ARG, "null handle");
    if (!h->initialized) return set_error(WAVE2D_ERR_STATE, "no time level computed yet");
    wave2d_exact none{};
    if (!ex) ex = &none;
    if (!valid_exact(ex)) return set_error(WAVE2D_ERR_ARG, "invalid exact-solution description");
    std::vector<double> tab;
    if (ex->kind != WAVE2D_EXACT_NONE) {
        exact_tables(h, *ex, tab);
        W2D_CUDA(cudaMemcpyAsync(h->tab_eval, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice,
                                 h->stream),
                 "exact table upload");
    }
    const ExactTab et = make_tab(h, h->tab_eval, *ex, (double)h->k * h->tau);
    const Reduce rd = make_reduce(h, h->acc_eval, 0);
    // about 8 blocks per SM, each thread looping over many nodes: every block
    // ends in a block reduction and one atomic on the shared counter, which
    // dominated the time at 4096^2 with a block per row
    const int gx = std::min((h->nx + 255) / 256, 16);
    const dim3 grd(gx, std::max(1, std::min(h->ny, 8 * h->num_sms / gx)));
    dispatch_dt(h->dtype, [&](auto DTc) {
        k4_norms<decltype(DTc)::value><<<grd, 256, 0, h->stream>>>(h->level(h->cur), h->geo(), et, rd);
    });
    W2D_LAUNCHED("norm kernel launch");
    double acc[4], accT[4];
    int st = 0;
    W2D_CUDA(cudaMemcpyAsync(acc, h->acc_eval, sizeof acc, cudaMemcpyDeviceToHost, h->stream), "norm copy");
    W2D_CUDA(cudaMemcpyAsync(accT, h->acc_track, sizeof accT, cudaMemcpyDeviceToHost, h->stream), "norm copy");
    W2D_CUDA(cudaMemcpyAsync(&st, h->status, sizeof st, cudaMemcpyDeviceToHost, h->stream), "status copy");
    W2D_CUDA(cudaStreamSynchronize(h->stream), "stream synchronize");
    if (ex->kind == WAVE2D_EXACT_NONE) {
        if (rel_l2) *rel_l2 = std::sqrt(acc[0]);
        if (rel_linf) *rel_linf = acc[2];
    } else {
        if (rel_l2) *rel_l2 = std::sqrt(acc[0] / acc[1]);
        if (rel_linf) *rel_linf = acc[2] / acc[3];
    }
    if (spacetime_E) *spacetime_E = h->tracking ? std::sqrt(accT[0] / accT[1]) : NAN;
    if (st) cudaMemsetAsync(h->status, 0, sizeof(int), h->stream);
    if (st & STATUS_TIMEOUT) return set_error(WAVE2D_ERR_TIMEOUT, "a device-side wait exceeded its limit");
    if (st & STATUS_NONFINITE) return set_error(WAVE2D_ERR_NONFINITE, "the field contains NaN or Inf");
    return WAVE2D_OK;
}

int wave2d_get_state(wave2d_t h, double* u_prev, double* u_cur, int64_t* k) {
    NvtxRange nvtx_range("wave2d_get_state");
    if (!h) return set_error(WAVE2D_ERR_ARG, "null handle");
    if (!h->initialized) return set_error(WAVE2D_ERR_STATE, "no state yet");
    const size_t n = (size_t)h->nx * h->ny;
    double* stage = (double*)dev_alloc(h->alloc, 2 * n * sizeof(double), h->stream);
    if (!stage) return set_error(WAVE2D_ERR_OOM, "staging allocation failed");
    dispatch_dt(h->dtype, [&](auto DTc) {
        constexpr int DT = decltype(DTc)::value;
        k_pack<DT><<<grid2d(h), dim3(32, 8), 0, h->stream>>>(h->level(h->diff_form ? h->dpl : h->prv), h->geo(), stage);
        k_pack<DT><<<grid2d(h), dim3(32, 8), 0, h->stream>>>(h->level(h->cur), h->geo(), stage + n);
        if (h->diff_form)  // u^{k-1} = u^k - d^k, in FP64
            k_combine<<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(stage + n, stage, stage, n);
    });
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && u_prev)
        e = cudaMemcpyAsync(u_prev, stage, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess && u_cur)
        e = cudaMemcpyAsync(u_cur, stage + n, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    dev_free(h->alloc, stage, 2 * n * sizeof(double), h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "get_state");
    g_launches.fetch_add(h->diff_form ? 3 : 2);
    if (k) *k = h->k;
    return check_status(h);
}

int wave2d_set_state(wave2d_t h, const double* u_prev, const double* u_cur, int64_t k, int on_device) {
    NvtxRange nvtx_range("wave2d_set_state");
    if (!h || !u_prev || !u_cur) return set_error(WAVE2D_ERR_ARG, "null argument");
    if (k < 1) return set_error(WAVE2D_ERR_ARG, "level index k must be >= 1");
    const size_t n = (size_t)h->nx * h->ny;
    const double* dp = u_prev;
    const double* dc = u_cur;
    double* stage = nullptr;
    if (!on_device) {
        stage = (double*)dev_alloc(h->alloc, 2 * n * sizeof(double), h->stream);
        if (!stage) return set_error(WAVE2D_ERR_OOM, "staging allocation failed");
        W2D_CUDA(cudaMemcpyAsync(stage, u_prev, n * sizeof(double), cudaMemcpyHostToDevice, h->stream), "upload");
        W2D_CUDA(cudaMemcpyAsync(stage + n, u_cur, n * sizeof(double), cudaMemcpyHostToDevice, h->stream), "upload");
        dp = stage;
        dc = stage + n;
    }
    h->cur = 0;
    h->prv = 1;
    h->dpl = 2;
    double* dstage = nullptr;
    if (h->diff_form) {  // d^k = u^k - u^{k-1}, formed in FP64
        dstage = (double*)dev_alloc(h->alloc, n * sizeof(double), h->stream);
        if (!dstage) {
            if (stage) dev_free(h->alloc, stage, 2 * n * sizeof(double), h->stream);
            return set_error(WAVE2D_ERR_OOM, "staging allocation failed");
        }
        k_combine<<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(dc, dp, dstage, n);
        dp = dstage;
    }
    dispatch_dt(h->dtype, [&](auto DTc) {
        constexpr int DT = decltype(DTc)::value;
        dispatch_bc(h->bc, [&](auto Pc) {
            k_unpack<DT, decltype(Pc)::value><<<grid2d(h), dim3(32, 8), 0, h->stream>>>(
                dp, h->level(h->diff_form ? h->dpl : 1), h->geo(), h->gw);
            k_unpack<DT, decltype(Pc)::value><<<grid2d(h), dim3(32, 8), 0, h->stream>>>(dc, h->level(0), h->geo(), h->gw);
        });
    });
    cudaError_t e = cudaGetLastError();
    if (stage) dev_free(h->alloc, stage, 2 * n * sizeof(double), h->stream);
    if (dstage) dev_free(h->alloc, dstage, n * sizeof(double), h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "set_state");
    g_launches.fetch_add(h->diff_form ? 3 : 2);
    h->k = k;
    h->initialized = true;
    drop_graphs(h);
    return WAVE2D_OK;
}

int64_t wave2d_raw_bytes(wave2d_t h) {
    if (!h) return set_error(WAVE2D_ERR_ARG, "null handle");
    return (int64_t)((h->dtype == WAVE2D_F32X2 ? 4 : 2) * h->plane_bytes);
}

// Raw layout: [u^{k-1} hi][u^k hi] (+ [u^{k-1} lo][u^k lo] for F32X2), each
// plane_bytes long, ghost ring included; difference form: [d^k][u^k].
int wave2d_get_raw(wave2d_t h, void* dst, int64_t bytes, int64_t* k) {
    if (!h || !dst) return set_error(WAVE2D_ERR_ARG, "null argument");
    if (!h->initialized) return set_error(WAVE2D_ERR_STATE, "no state yet");
    if (bytes < wave2d_raw_bytes(h)) return set_error(WAVE2D_ERR_ARG, "buffer too small");
    char* d = (char*)dst;
    const int order[2] = {h->diff_form ? h->dpl : h->prv, h->cur};
    for (int q = 0; q < 2; ++q) {
        W2D_CUDA(cudaMemcpyAsync(d + q * h->plane_bytes, h->hi[order[q]], h->plane_bytes, cudaMemcpyDeviceToHost,
                                 h->stream),
                 "raw copy");
        if (h->lo[0])
            W2D_CUDA(cudaMemcpyAsync(d + (2 + q) * h->plane_bytes, h->lo[order[q]], h->plane_bytes,
                                     cudaMemcpyDeviceToHost, h->stream),
                     "raw copy");
    }
    W2D_CUDA(cudaStreamSynchronize(h->stream), "stream synchronize");
    if (k) *k = h->k;
    return WAVE2D_OK;
}

int wave2d_set_raw(wave2d_t h, const void* src, int64_t bytes, int64_t k) {
    if (!h || !src) return set_error(WAVE2D_ERR_ARG, "null argument");
    if (k < 1) return set_error(WAVE2D_ERR_ARG, "level index k must be >= 1");
    if (bytes < wave2d_raw_bytes(h)) return set_error(WAVE2D_ERR_ARG, "buffer too small");
    const char* s = (const char*)src;
    h->cur = 1;  // plane 0 <- u^{k-1}, plane 1 <- u^k (difference form: plane 2 <- d^k)
    h->prv = 0;
    h->dpl = 2;
    for (int q = 0; q < 2; ++q) {
        const int plane = (q == 0 && h->diff_form) ? h->dpl : q;
        W2D_CUDA(cudaMemcpyAsync(h->hi[plane], s + q * h->plane_bytes, h->plane_bytes, cudaMemcpyHostToDevice,
                                 h->stream),
                 "raw copy");
        if (h->lo[0])
            W2D_CUDA(cudaMemcpyAsync(h->lo[q], s + (2 + q) * h->plane_bytes, h->plane_bytes, cudaMemcpyHostToDevice,
                                     h->stream),
                     "raw copy");
    }
    W2D_CUDA(cudaStreamSynchronize(h->stream), "stream synchronize");
    h->k = k;
    h->initialized = true;
    drop_graphs(h);
    int rc = canary_fill(h);  // the copied planes carry the source's guard band
    if (rc != WAVE2D_OK) return rc;
    return refresh_ghosts(h);  // the copied rings may come from a shallower mode
}

// Rows [j0, j0 + nrows) of the two state planes, in the storage type, to or
// from a packed buffer of nrows * nx values per plane (two such blocks, hi
// then lo, for F32X2).  Plane order as in the raw layout: u^{k-1} (d^k for the
// difference form), then u^k.
static int copy_rows(wave2d* h, int j0, int nrows, void* prev, void* cur, const void* cprev, const void* ccur,
                     int on_device, bool to_handle) {
    if (!h) return set_error(WAVE2D_ERR_ARG, "null handle");
    if (!h->initialized) return set_error(WAVE2D_ERR_STATE, "no state yet");
    if (j0 < 0 || nrows < 0 || j0 + (int64_t)nrows > h->ny)
        return set_error(WAVE2D_ERR_ARG, "rows [%d, %d) outside 0 .. %d", j0, j0 + nrows, h->ny);
    if (nrows == 0) return WAVE2D_OK;
    const size_t el = h->elem, rowb = (size_t)h->nx * el, block = rowb * nrows;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice
                                          : (to_handle ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost);
    const int planes[2] = {h->diff_form ? h->dpl : h->prv, h->cur};
    for (int q = 0; q < 2; ++q) {
        char* ext = static_cast<char*>(to_handle ? const_cast<void*>(q ? ccur : cprev) : (q ? cur : prev));
        if (!ext) return set_error(WAVE2D_ERR_ARG, "null row buffer");
        for (int part = 0; part < (h->lo[0] ? 2 : 1); ++part) {
            char* base = static_cast<char*>(part ? h->lo[planes[q]] : h->hi[planes[q]]);
            char* pl = base + ((size_t)(j0 + h->G) * h->pitch + h->G) * el;
            char* buf = ext + part * block;
            const cudaError_t e = to_handle
                ? cudaMemcpy2DAsync(pl, (size_t)h->pitch * el, buf, rowb, rowb, nrows, kind, h->stream)
                : cudaMemcpy2DAsync(buf, rowb, pl, (size_t)h->pitch * el, rowb, nrows, kind, h->stream);
            if (e != cudaSuccess) return cuda_fail(e, "row copy");
        }
    }
    if (to_handle) {
        // periodic / odd images in the ghost ring follow the new rows
        h->rings_stale = false;
        int rc = refresh_ghosts(h);
        if (rc != WAVE2D_OK) return rc;
    }
    if (!on_device) W2D_CUDA(cudaStreamSynchronize(h->stream), "stream synchronize");
    return WAVE2D_OK;
}

int wave2d_get_rows(wave2d_t h, int j0, int nrows, void* prev, void* cur, int on_device) {
    NvtxRange nvtx_range("wave2d_get_rows");
    return copy_rows(h, j0, nrows, prev, cur, nullptr, nullptr, on_device, false);
}

int wave2d_set_rows(wave2d_t h, int j0, int nrows, const void* prev, const void* cur, int on_device) {
    NvtxRange nvtx_range("wave2d_set_rows");
    return copy_rows(h, j0, nrows, nullptr, nullptr, prev, cur, on_device, true);
}

int wave2d_error_sums(wave2d_t h, const wave2d_exact* ex, int j0, int nrows, int64_t row_shift, double* sums) {
    NvtxRange nvtx_range("wave2d_error_sums");
    if (!h || !sums) return set_error(WAVE2D_ERR_ARG, "null argument");
    if (!h->initialized) return set_error(WAVE2D_ERR_STATE, "no time level computed yet");
    if (j0 < 0 || nrows < 1 || j0 + (int64_t)nrows > h->ny)
        return set_error(WAVE2D_ERR_ARG, "rows [%d, %d) outside 0 .. %d", j0, j0 + nrows, h->ny);
    wave2d_exact none{};
    if (!ex) ex = &none;
    if (!valid_exact(ex)) return set_error(WAVE2D_ERR_ARG, "invalid exact-solution description");
    // tables of the exact solution: P, R over the nx columns, Q, S over the
    // rows j0 .. j0 + nrows - 1 placed at global rows j + row_shift
    std::vector<double> tab(2 * (size_t)h->nx + 2 * (size_t)nrows, 0.0);
    double* P = tab.data();
    double* R = P + h->nx;
    double* Q = R + h->nx;
    double* S = Q + nrows;
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < h->nx; ++i) {
        const double x = (i + ex->x_off) * h->h;
        if (ex->kind == WAVE2D_EXACT_STANDING) P[i] = std::sin(2.0 * pi * ex->m * x);
        else if (ex->kind == WAVE2D_EXACT_PLANE) {
            P[i] = std::cos(ex->k1 * x);
            R[i] = std::sin(ex->k1 * x);
        }
    }
    for (int j = 0; j < nrows; ++j) {
        const double y = ((double)(j0 + j + row_shift) + ex->x_off) * h->h;
        if (ex->kind == WAVE2D_EXACT_STANDING) Q[j] = std::sin(2.0 * pi * ex->m * y);
        else if (ex->kind == WAVE2D_EXACT_PLANE) {
            Q[j] = std::cos(ex->k2 * y);
            S[j] = std::sin(ex->k2 * y);
        }
    }
    if (ex->kind != WAVE2D_EXACT_NONE)
        W2D_CUDA(cudaMemcpyAsync(h->tab_eval, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice,
                                 h->stream),
                 "exact table upload");
    ExactTab et{};
    et.kind = ex->kind;
    et.P = h->tab_eval;
    et.R = h->tab_eval + h->nx;
    et.Q = h->tab_eval + 2 * (size_t)h->nx;
    et.S = h->tab_eval + 2 * (size_t)h->nx + nrows;
    exact_weights(h, *ex, (double)h->k * h->tau, et.w0, et.w1);
    const Reduce rd = make_reduce(h, h->acc_eval, 0);
    // the rows as a grid of their own: the level planes shifted by j0 rows
    Level L = h->level(h->cur);
    const size_t shift = (size_t)j0 * h->pitch * h->elem;
    L.hi = static_cast<char*>(L.hi) + shift;
    if (L.lo) L.lo = static_cast<char*>(L.lo) + shift;
    const Geo g{h->nx, nrows, h->pitch, h->G};
    const int gx = std::min((h->nx + 255) / 256, 16);
    const dim3 grd(gx, std::max(1, std::min(nrows, 8 * h->num_sms / gx)));
    dispatch_dt(h->dtype, [&](auto DTc) {
        k4_norms<decltype(DTc)::value><<<grd, 256, 0, h->stream>>>(L, g, et, rd);
    });
    W2D_LAUNCHED("norm kernel launch");
    int st = 0;
    W2D_CUDA(cudaMemcpyAsync(sums, h->acc_eval, 4 * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "norm copy");
    W2D_CUDA(cudaMemcpyAsync(&st, h->status, sizeof st, cudaMemcpyDeviceToHost, h->stream), "status copy");
    W2D_CUDA(cudaStreamSynchronize(h->stream), "stream synchronize");
    if (st) cudaMemsetAsync(h->status, 0, sizeof(int), h->stream);
    if (st & STATUS_TIMEOUT) return set_error(WAVE2D_ERR_TIMEOUT, "a device-side wait exceeded its limit");
    if (st & STATUS_NONFINITE) return set_error(WAVE2D_ERR_NONFINITE, "the field contains NaN or Inf");
    return WAVE2D_OK;
}

int wave2d_diff_norms(wave2d_t a, wave2d_t b, double* rel_l2, double* rel_linf) {
    NvtxRange nvtx_range("wave2d_diff_norms");
    if (!a || !b) return set_error(WAVE2D_ERR_ARG, "null handle");
    if (!a->initialized || !b->initialized) return set_error(WAVE2D_ERR_STATE, "no time level computed yet");
    if (a->nx != b->nx || a->ny != b->ny) return set_error(WAVE2D_ERR_ARG, "the two grids differ in size");
    if (a->device != b->device) return set_error(WAVE2D_ERR_ARG, "the two handles live on different devices");
    if (a->k != b->k) return set_error(WAVE2D_ERR_STATE, "the two handles are at different levels");
    // b's writes are ordered before a's stream reads them
    cudaEvent_t ev = nullptr;
    W2D_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "event create");
    cudaEventRecord(ev, b->stream);
    cudaStreamWaitEvent(a->stream, ev, 0);
    cudaEventDestroy(ev);
    const Reduce rd = make_reduce(a, a->acc_eval, 0);
    const int gx = std::min((a->nx + 255) / 256, 16);
    const dim3 grd(gx, std::max(1, std::min(a->ny, 8 * a->num_sms / gx)));
    dispatch_dt(a->dtype, [&](auto DA) {
        dispatch_dt(b->dtype, [&](auto DB) {
            k_diff_norms<decltype(DA)::value, decltype(DB)::value><<<grd, 256, 0, a->stream>>>(
                a->level(a->cur), a->geo(), b->level(b->cur), b->geo(), rd);
        });
    });
    W2D_LAUNCHED("difference norm kernel launch");
    double acc[4];
    int st = 0;
    W2D_CUDA(cudaMemcpyAsync(acc, a->acc_eval, sizeof acc, cudaMemcpyDeviceToHost, a->stream), "norm copy");
    W2D_CUDA(cudaMemcpyAsync(&st, a->status, sizeof st, cudaMemcpyDeviceToHost, a->stream), "status copy");
    W2D_CUDA(cudaStreamSynchronize(a->stream), "stream synchronize");
    if (rel_l2) *rel_l2 = std::sqrt(acc[0] / acc[1]);
    if (rel_linf) *rel_linf = acc[2] / acc[3];
    if (st) cudaMemsetAsync(a->status, 0, sizeof(int), a->stream);
    if (st & STATUS_TIMEOUT) return set_error(WAVE2D_ERR_TIMEOUT, "a device-side wait exceeded its limit");
    if (st & STATUS_NONFINITE) return set_error(WAVE2D_ERR_NONFINITE, "the field contains NaN or Inf");
    return WAVE2D_OK;
}

int wave2d_autotune(wave2d_t h, int64_t steps, wave2d_tune* best) {
    NvtxRange nvtx_range("wave2d_autotune");
    if (!h) return set_error(WAVE2D_ERR_ARG, "null handle");
    if (steps < 1) return set_error(WAVE2D_ERR_ARG, "autotune needs steps >= 1");
    if (!h->initialized) return set_error(WAVE2D_ERR_STATE, "autotune needs an initialised state");
    std::vector<wave2d_tune> cands;
    auto add = [&](int kernel, int tile_h, int T, int per_sm) {
        wave2d_tune t{};
        t.kernel = kernel;
        t.tile_h = tile_h;
        t.temporal_t = T;
        t.use_graph = -1;
        t.ctas_per_sm = per_sm;
        cands.push_back(t);
    };
    const bool persist_ok = h->nclass == 0 && !h->diff_sums && !h->diff_form &&
                            (int64_t)h->nx * h->ny <= (int64_t(1) << 20);
    if (h->dtype == WAVE2D_F32 && !multilevel_ok(h)) {
        add(WAVE2D_KERNEL_TMA, 0, 0, 1);
        add(WAVE2D_KERNEL_TMA, 0, 0, 2);
        add(WAVE2D_KERNEL_SIMPLE, 0, 0, 0);
        if (stream_ok(h))
            for (int T : {2, 3, 4, 6})
                for (int rows : {16, 32, 64})
                    if (T <= 4 || !h->diff_form) add(WAVE2D_KERNEL_STREAM, rows, T, 0);
    } else if (h->dtype == WAVE2D_F32) {
        add(WAVE2D_KERNEL_TMA, 0, 0, 1);
        add(WAVE2D_KERNEL_TMA, 0, 0, 2);
        for (int T : {2, 3, 4})
            for (int oh : {16, 24, 32, 64}) add(WAVE2D_KERNEL_TEMPORAL, oh, T, 0);
        for (int T : {2, 3, 4, 6})
            for (int rows : {16, 24, 32, 48, 64}) add(WAVE2D_KERNEL_STREAM, rows, T, 0);
    } else if (h->dtype == WAVE2D_F64) {
        add(WAVE2D_KERNEL_TMA, 0, 0, 1);
        add(WAVE2D_KERNEL_TMA, 0, 0, 2);
        add(WAVE2D_KERNEL_SIMPLE, 0, 0, 0);
    } else {
        add(WAVE2D_KERNEL_SIMPLE, 0, 0, 0);
    }
    if (persist_ok) add(WAVE2D_KERNEL_PERSISTENT, 0, 0, 0);
    if (h->tracking || cands.size() == 1) {
        h->tune = cands[0];
        int rc = select_kernel(h);
        if (best) *best = h->tune;
        return rc;
    }
    // Snapshot the two current levels (hi and lo planes).
    const int np = h->lo[0] ? 2 : 1;
    const size_t snap_bytes = 2 * (size_t)np * h->plane_bytes;
    char* snap = (char*)dev_alloc(h->alloc, snap_bytes, h->stream);
    if (!snap) return set_error(WAVE2D_ERR_OOM, "autotune snapshot allocation failed");
    const int cur0 = h->cur, prv0 = h->prv, dpl0 = h->dpl;
    const int64_t k0 = h->k;
    auto copy_levels = [&](bool save) -> int {
        const int planes[2] = {cur0, h->diff_form ? dpl0 : prv0};
        for (int q = 0; q < 2; ++q)
            for (int part = 0; part < np; ++part) {
                void* dev = part == 0 ? h->hi[planes[q]] : h->lo[planes[q]];
                char* sp = snap + ((size_t)q * np + part) * h->plane_bytes;
                cudaError_t e = save ? cudaMemcpyAsync(sp, dev, h->plane_bytes, cudaMemcpyDeviceToDevice, h->stream)
                                     : cudaMemcpyAsync(dev, sp, h->plane_bytes, cudaMemcpyDeviceToDevice, h->stream);
                if (e != cudaSuccess) return cuda_fail(e, "autotune snapshot copy");
            }
        h->cur = cur0;
        h->prv = prv0;
        h->dpl = dpl0;
        h->k = k0;
        return WAVE2D_OK;
    };
    int rc = copy_levels(true);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (rc == WAVE2D_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
        rc = set_error(WAVE2D_ERR_CUDA, "event create failed");
    float best_ms = 0;
    wave2d_tune chosen = cands[0];
    for (size_t c = 0; c < cands.size() && rc == WAVE2D_OK; ++c) {
        rc = copy_levels(false);
        if (rc != WAVE2D_OK) break;
        h->tune = cands[c];
        rc = select_kernel(h);
        if (rc == WAVE2D_OK) rc = refresh_ghosts(h);
        if (rc == WAVE2D_OK) rc = wave2d_step_n(h, std::min<int64_t>(steps, 8));  // warm-up
        if (rc != WAVE2D_OK) break;
        // a multi-level candidate is timed on whole launches (a multiple of
        // its depth), so the one-level steps that finish an uneven run do not
        // count against it; candidates are compared per level
        const int64_t depth = is_multilevel(h->kernel) ? h->temporal_t : 1;
        const int64_t levels = std::max<int64_t>(depth, steps / depth * depth);
        cudaEventRecord(e0, h->stream);
        rc = wave2d_step_n(h, levels);
        cudaEventRecord(e1, h->stream);
        if (rc != WAVE2D_OK) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            rc = set_error(WAVE2D_ERR_CUDA, "autotune timing failed");
            break;
        }
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= (float)levels;
        if (c == 0 || ms < best_ms) {
            best_ms = ms;
            chosen = cands[c];
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    const int rc_restore = copy_levels(false);
    dev_free(h->alloc, snap, snap_bytes, h->stream);
    if (rc == WAVE2D_OK) rc = rc_restore;
    if (rc != WAVE2D_OK) return rc;
    h->tune = chosen;
    rc = select_kernel(h);
    if (rc == WAVE2D_OK) rc = refresh_ghosts(h);
    if (rc == WAVE2D_OK) rc = check_status(h);
    if (best) *best = chosen;
    return rc;
}

int wave2d_selftest_timeout(wave2d_t h, int64_t limit_cycles) {
    if (!h) return set_error(WAVE2D_ERR_ARG, "null handle");
    if (limit_cycles < 1 || limit_cycles > (1LL << 31))
        return set_error(WAVE2D_ERR_ARG, "limit must be 1 .. 2^31 cycles");
    k_selftest_wait<<<1, 32, 0, h->stream>>>(h->status, (long long)limit_cycles);
    W2D_LAUNCHED("self-test kernel launch");
    // the persistent kernel's grid barrier: one block waiting for an arrival
    // that never comes
    unsigned long long* arrived = reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(h->counter) + 128);
    W2D_CUDA(cudaMemsetAsync(arrived, 0, sizeof(unsigned long long), h->stream), "barrier reset");
    k_selftest_grid_wait<<<1, 32, 0, h->stream>>>(arrived, h->status, (long long)limit_cycles);
    W2D_LAUNCHED("self-test kernel launch");
    return WAVE2D_OK;
}

int wave2d_sync(wave2d_t h) {
    if (!h) return set_error(WAVE2D_ERR_ARG, "null handle");
    return check_status(h);
}

}  // extern "C"

namespace w2d {
// Release a handle that shares its stream with its owner without waiting:
// the memory is freed in stream order, after the work already queued.
void release_handle_nosync(wave2d* h) {
    if (!h) return;
    if (h->own_stream) {
        release_handle(h);
        return;
    }
    drop_graphs(h);
    if (h->base) dev_free(h->alloc, h->base, h->base_bytes, h->stream);
    delete h;
}
}  // namespace w2d
