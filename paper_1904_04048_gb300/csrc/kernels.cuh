// CUDA kernels of the wave2d library (sm_103a).
//
//   k1_first_step   first time step, Eq. A1 (comp5.1, comp9.1, comp13.1), FP64 math
//   k2_simple       two-step, Eq. A2 (comp5.2, comp9.2, comp13.2), one node per
//                   thread, optional fused space-time error reduction (Eq. error)
//   k2_tma          two-step through TMA-staged shared-memory tiles with a
//                   multi-stage mbarrier pipeline, register-rotated rows
//   k4_norms        FP64 error norms against a separable exact solution
//   k_pack/k_unpack conversion between level planes and plain FP64 arrays
//
// Level planes: a field of nx*ny nodes is stored with a ghost ring of G nodes
// on every side in a row-major plane of `pitch` elements per row and ny + 2G
// rows; node (i, j) lives at (j + G) * pitch + (i + G).  Zero boundary: the
// ring holds zeros and is never written.  Periodic boundary: every kernel that
// writes a node within gw of an edge also writes its periodic images into the
// first gw rings (gw = R, the stencil radius, for one-level kernels; deeper
// when temporal blocking reads a wider halo), so readers never wrap indices.
// Odd boundary (the zero boundary continued as an odd function beyond the
// boundary nodes -1 and nx): writers store the negated mirror images
// u(-2 - i) = -u(i), u(2 nx - i) = -u(i) (and their products at the corners)
// in the first gw rings; the boundary nodes themselves stay zero.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "stencil_ops.cuh"

namespace w2d {

enum { DT_F64 = 0, DT_F32 = 1, DT_F32X2 = 2 };
enum { BCM_ZERO = 0, BCM_PERIODIC = 1, BCM_ODD = 2 };  // boundary modes (WAVE2D_BC_*)
enum { STATUS_NONFINITE = 1, STATUS_TIMEOUT = 2 };

struct Level {
    void* hi;  // value plane (the high part for double-float)
    void* lo;  // low part for double-float, else null
};

struct Geo {
    int nx, ny, pitch, G;
};

__device__ __forceinline__ size_t off(const Geo& g, int i, int j) {
    return (size_t)(j + g.G) * (size_t)g.pitch + (size_t)(i + g.G);
}

template <int DT>
struct St;
template <>
struct St<DT_F32> {
    using V = float;
    __device__ static V ldg(const Level& L, size_t o) { return __ldg((const float*)L.hi + o); }
    __device__ static V ldcg(const Level& L, size_t o) { return __ldcg((const float*)L.hi + o); }
    __device__ static V ld(const Level& L, size_t o) { return ((const float*)L.hi)[o]; }
    __device__ static void st(const Level& L, size_t o, V v) { ((float*)L.hi)[o] = v; }
    __device__ static double to_d(V v) { return (double)v; }
    __device__ static V from_d(double d) { return __double2float_rn(d); }
};
template <>
struct St<DT_F64> {
    using V = double;
    __device__ static V ldg(const Level& L, size_t o) { return __ldg((const double*)L.hi + o); }
    __device__ static V ldcg(const Level& L, size_t o) { return __ldcg((const double*)L.hi + o); }
    __device__ static V ld(const Level& L, size_t o) { return ((const double*)L.hi)[o]; }
    __device__ static void st(const Level& L, size_t o, V v) { ((double*)L.hi)[o] = v; }
    __device__ static double to_d(V v) { return v; }
    __device__ static V from_d(double d) { return d; }
};
template <>
struct St<DT_F32X2> {
    using V = df;
    __device__ static V ldg(const Level& L, size_t o) {
        return {__ldg((const float*)L.hi + o), __ldg((const float*)L.lo + o)};
    }
    __device__ static V ldcg(const Level& L, size_t o) {
        return {__ldcg((const float*)L.hi + o), __ldcg((const float*)L.lo + o)};
    }
    __device__ static V ld(const Level& L, size_t o) {
        return {((const float*)L.hi)[o], ((const float*)L.lo)[o]};
    }
    __device__ static void st(const Level& L, size_t o, V v) {
        ((float*)L.hi)[o] = v.hi;
        ((float*)L.lo)[o] = v.lo;
    }
    __device__ static double to_d(V v) { return (double)v.hi + (double)v.lo; }
    __device__ static V from_d(double d) {
        float h = __double2float_rn(d);
        return {h, __double2float_rn(d - (double)h)};
    }
};

// Periodic images of node (i, j) in the first gw rings of ghosts.  A kernel
// that advances one level reads at most R nodes away, so writers pass
// gw = R (gw <= G): only nodes within R of an edge have images to write.
template <int DT>
__device__ __forceinline__ void write_images(const Level& L, const Geo& g, int i, int j,
                                             typename St<DT>::V v, int gw) {
    if (i >= gw && i < g.nx - gw && j >= gw && j < g.ny - gw) return;
    const int mxr = (gw + g.nx - 1) / g.nx, myr = (gw + g.ny - 1) / g.ny;
    for (int my = -myr; my <= myr; ++my) {
        const int jj = j + my * g.ny;
        if (jj < -gw || jj >= g.ny + gw) continue;
        for (int mx = -mxr; mx <= mxr; ++mx) {
            if (mx == 0 && my == 0) continue;
            const int ii = i + mx * g.nx;
            if (ii < -gw || ii >= g.nx + gw) continue;
            St<DT>::st(L, off(g, ii, jj), v);
        }
    }
}

// Periodic images of a whole aligned vector of `vec` nodes (x a multiple of
// vec) in the first gw ghost rings.  Valid when nx is a multiple of vec and
// nx, ny >= 2 gw: a node within gw of an edge then has exactly one image per
// wrapped direction, and the images of an aligned vector are aligned vectors
// inside the ring (gw <= G).  Images of the vector's other nodes are written
// too; they are equally correct.
template <typename VT>
__device__ __forceinline__ void store_vec_images(VT* base, const Geo& g, int x, int y, VT v, int gw,
                                                 int vec) {
    const bool ylo = y < gw, yhi = y >= g.ny - gw;
    const bool xlo = x < gw, xhi = x + vec > g.nx - gw;
    if (!(ylo || yhi || xlo || xhi)) return;
    const long long P = g.pitch;
    auto at = [&](int xx, int yy) { return base + ((long long)(yy + g.G) * P + (xx + g.G)) / vec; };
    if (ylo) *at(x, y + g.ny) = v;
    if (yhi) *at(x, y - g.ny) = v;
    if (xlo) {
        *at(x + g.nx, y) = v;
        if (ylo) *at(x + g.nx, y + g.ny) = v;
        if (yhi) *at(x + g.nx, y - g.ny) = v;
    }
    if (xhi) {
        *at(x - g.nx, y) = v;
        if (ylo) *at(x - g.nx, y + g.ny) = v;
        if (yhi) *at(x - g.nx, y - g.ny) = v;
    }
}

__device__ __forceinline__ float vneg(float a) { return -a; }
__device__ __forceinline__ double vneg(double a) { return -a; }
__device__ __forceinline__ df vneg(df a) { return df_neg(a); }

// Odd continuation: the positions p of the ghost band [-gw, n + gw) that hold
// node i (sign +1: p = i + m P) or its negation (sign -1: p = -2 - i + m P),
// P = 2 (n + 1) the period of the odd extension; the boundary nodes -1 and n
// are never among them.
template <int DT>
__device__ __forceinline__ void write_images_odd(const Level& L, const Geo& g, int i, int j,
                                                 typename St<DT>::V v, int gw) {
    if (i >= gw && i < g.nx - gw && j >= gw && j < g.ny - gw) return;
    const int Px = 2 * (g.nx + 1), Py = 2 * (g.ny + 1);
    const int mx = (gw + Px - 1) / Px + 1, my = (gw + Py - 1) / Py + 1;
    const typename St<DT>::V nv = vneg(v);
    for (int ky = -my; ky <= my; ++ky)
        for (int ty = 0; ty < 2; ++ty) {
            const int jj = ty ? (-2 - j + ky * Py) : (j + ky * Py);
            if (jj < -gw || jj >= g.ny + gw || jj == -1 || jj == g.ny) continue;
            for (int kx = -mx; kx <= mx; ++kx)
                for (int tx = 0; tx < 2; ++tx) {
                    const int ii = tx ? (-2 - i + kx * Px) : (i + kx * Px);
                    if (ii < -gw || ii >= g.nx + gw || ii == -1 || ii == g.nx) continue;
                    if (ii >= 0 && ii < g.nx && jj >= 0 && jj < g.ny) continue;  // the node itself
                    St<DT>::st(L, off(g, ii, jj), (tx ^ ty) ? nv : v);
                }
        }
}

template <int DT, int BCM>
__device__ __forceinline__ void write_images_bc(const Level& L, const Geo& g, int i, int j,
                                                typename St<DT>::V v, int gw) {
    if constexpr (BCM == BCM_PERIODIC) write_images<DT>(L, g, i, j, v, gw);
    else if constexpr (BCM == BCM_ODD) write_images_odd<DT>(L, g, i, j, v, gw);
}

// ---------------------------------------------------------------------------
// Exact solution as a separable sum (FP64 tables built on the host):
//   u_e(i, j) = w0 (P_i Q_j - R_i S_j) + w1 (R_i Q_j + P_i S_j)
// STANDING: P = sin(2 pi m x1), Q = sin(2 pi m x2), R = S = 0, w0 = amp sin(w t)
// PLANE:    P = cos(k1 x1), R = sin(k1 x1), Q = cos(k2 x2), S = sin(k2 x2),
//           w0 = amp cos(w t), w1 = amp sin(w t)   (cos(a + b - wt) expanded)
// ---------------------------------------------------------------------------
struct ExactTab {
    const double* P;
    const double* R;
    const double* Q;
    const double* S;
    double w0, w1;
    int kind;  // 0 = none
};

__device__ __forceinline__ double exact_at(const ExactTab& ex, int i, int j) {
    if (ex.kind == 0) return 0.0;
    const double p = ex.P[i], r = ex.R[i], q = ex.Q[j], s = ex.S[j];
    return __dadd_rn(__dmul_rn(ex.w0, __dsub_rn(__dmul_rn(p, q), __dmul_rn(r, s))),
                     __dmul_rn(ex.w1, __dadd_rn(__dmul_rn(r, q), __dmul_rn(p, s))));
}

// Deterministic grid reduction: per-block partials, the last block to finish
// sums them in a fixed order.  acc[0] = sum (u-u_e)^2, acc[1] = sum u_e^2,
// acc[2] = max |u-u_e|, acc[3] = max |u_e|.  accumulate = 1 adds into acc
// (space-time sums), 0 overwrites it.
struct Reduce {
    double* partials;
    unsigned* counter;
    double* acc;
    int* status;
    int accumulate;
};

template <int NT>
__device__ __forceinline__ void reduce_finalize(double s0, double s1, double m0, double m1,
                                                const Reduce& rd) {
    constexpr int NW = NT / 32;
    __shared__ double sh[4][NW];
    __shared__ int is_last;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int lane = tid & 31, wid = tid >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        m0 = fmax(m0, __shfl_xor_sync(0xffffffffu, m0, o));
        m1 = fmax(m1, __shfl_xor_sync(0xffffffffu, m1, o));
    }
    if (lane == 0) {
        sh[0][wid] = s0;
        sh[1][wid] = s1;
        sh[2][wid] = m0;
        sh[3][wid] = m1;
    }
    __syncthreads();
    const unsigned nb = gridDim.x * gridDim.y;
    if (tid == 0) {
        double a = 0, b = 0, c = 0, d = 0;
        for (int w = 0; w < NW; ++w) {
            a += sh[0][w];
            b += sh[1][w];
            c = fmax(c, sh[2][w]);
            d = fmax(d, sh[3][w]);
        }
        const unsigned bid = blockIdx.y * gridDim.x + blockIdx.x;
        rd.partials[4 * (size_t)bid + 0] = a;
        rd.partials[4 * (size_t)bid + 1] = b;
        rd.partials[4 * (size_t)bid + 2] = c;
        rd.partials[4 * (size_t)bid + 3] = d;
        __threadfence();
        const unsigned prev = atomicAdd(rd.counter, 1u);
        is_last = (prev == nb - 1);
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    double a = 0, b = 0, c = 0, d = 0;
    for (unsigned q = tid; q < nb; q += NT) {
        a += __ldcg(rd.partials + 4 * (size_t)q + 0);
        b += __ldcg(rd.partials + 4 * (size_t)q + 1);
        c = fmax(c, __ldcg(rd.partials + 4 * (size_t)q + 2));
        d = fmax(d, __ldcg(rd.partials + 4 * (size_t)q + 3));
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
        c = fmax(c, __shfl_xor_sync(0xffffffffu, c, o));
        d = fmax(d, __shfl_xor_sync(0xffffffffu, d, o));
    }
    __syncthreads();
    if (lane == 0) {
        sh[0][wid] = a;
        sh[1][wid] = b;
        sh[2][wid] = c;
        sh[3][wid] = d;
    }
    __syncthreads();
    if (tid == 0) {
        a = 0, b = 0, c = 0, d = 0;
        for (int w = 0; w < NW; ++w) {
            a += sh[0][w];
            b += sh[1][w];
            c = fmax(c, sh[2][w]);
            d = fmax(d, sh[3][w]);
        }
        if (rd.accumulate) {
            rd.acc[0] += a;
            rd.acc[1] += b;
            rd.acc[2] = fmax(rd.acc[2], c);
            rd.acc[3] = fmax(rd.acc[3], d);
        } else {
            rd.acc[0] = a;
            rd.acc[1] = b;
            rd.acc[2] = c;
            rd.acc[3] = d;
        }
        *rd.counter = 0u;  // ready for the next launch (stream-ordered)
        __threadfence();
    }
}

__device__ __forceinline__ void error_terms(double v, double ue, double& s0, double& s1, double& m0,
                                            double& m1, int* status) {
    if (!isfinite(v)) atomicOr(status, STATUS_NONFINITE);
    const double d = v - ue;
    s0 = __fma_rn(d, d, s0);
    s1 = __fma_rn(ue, ue, s1);
    m0 = fmax(m0, fabs(d));
    m1 = fmax(m1, fabs(ue));
}

// ---------------------------------------------------------------------------
// K1: first time step (Eq. A1), FP64, one node per thread.
// ---------------------------------------------------------------------------
// Interior index of position i under the odd continuation about the
// boundary nodes -1 and n (sign flipped per reflection); -1 for a boundary
// node.
__device__ __forceinline__ int odd_index(int i, int n, double& sign) {
    for (;;) {
        if (i == -1 || i == n) return -1;
        if (i < -1) { i = -2 - i; sign = -sign; continue; }
        if (i > n) { i = 2 * n - i; sign = -sign; continue; }
        return i;
    }
}

__device__ __forceinline__ double fetch_bc(const double* __restrict__ a, int nx, int ny, int bcm, int i, int j) {
    if (bcm == BCM_PERIODIC) {
        i = ((i % nx) + nx) % nx;
        j = ((j % ny) + ny) % ny;
    } else if (bcm == BCM_ODD) {
        double sign = 1.0;
        i = odd_index(i, nx, sign);
        j = odd_index(j, ny, sign);
        if (i < 0 || j < 0) return 0.0;
        return sign * __ldg(a + (size_t)j * nx + i);
    } else if (i < 0 || i >= nx || j < 0 || j >= ny) {
        return 0.0;
    }
    return __ldg(a + (size_t)j * nx + i);
}

__device__ __forceinline__ Nbr<double> gather_bc(const double* __restrict__ a, int nx, int ny,
                                                 int per, int i, int j) {
    Nbr<double> u;
    u.c = fetch_bc(a, nx, ny, per, i, j);
    u.e = fetch_bc(a, nx, ny, per, i + 1, j);
    u.w = fetch_bc(a, nx, ny, per, i - 1, j);
    u.n = fetch_bc(a, nx, ny, per, i, j + 1);
    u.s = fetch_bc(a, nx, ny, per, i, j - 1);
    u.ne = fetch_bc(a, nx, ny, per, i + 1, j + 1);
    u.nw = fetch_bc(a, nx, ny, per, i - 1, j + 1);
    u.se = fetch_bc(a, nx, ny, per, i + 1, j - 1);
    u.sw = fetch_bc(a, nx, ny, per, i - 1, j - 1);
    u.ee = fetch_bc(a, nx, ny, per, i + 2, j);
    u.ww = fetch_bc(a, nx, ny, per, i - 2, j);
    u.nn = fetch_bc(a, nx, ny, per, i, j + 2);
    u.ss = fetch_bc(a, nx, ny, per, i, j - 2);
    return u;
}

template <int DT, int S, int BCM, bool TRACK>
__global__ void __launch_bounds__(256) k1_first_step(const double* __restrict__ u0,
                                                     const double* __restrict__ v0, Level L0,
                                                     Level L1, Geo g, Coef3<double> ahalf,
                                                     Coef3<double> b, double tau, ExactTab ex,
                                                     Reduce rd, int gw) {
    using T = St<DT>;
    const int i = blockIdx.x * 32 + threadIdx.x;
    const int j = blockIdx.y * 8 + threadIdx.y;
    double s0 = 0, s1 = 0, m0 = 0, m1 = 0;
    if (i < g.nx && j < g.ny) {
        const Nbr<double> u = gather_bc(u0, g.nx, g.ny, BCM, i, j);
        const Nbr<double> v = gather_bc(v0, g.nx, g.ny, BCM, i, j);
        const double u1 = first_step_update<S>(u, v, ahalf, b, tau);
        const size_t o = off(g, i, j);
        const typename T::V q0 = T::from_d(u.c), q1 = T::from_d(u1);
        T::st(L0, o, q0);
        T::st(L1, o, q1);
        if (BCM != BCM_ZERO) {
            write_images_bc<DT, BCM>(L0, g, i, j, q0, gw);
            write_images_bc<DT, BCM>(L1, g, i, j, q1, gw);
        }
        if (TRACK) error_terms(T::to_d(q1), exact_at(ex, i, j), s0, s1, m0, m1, rd.status);
    }
    if (TRACK) reduce_finalize<256>(s0, s1, m0, m1, rd);
}

// ---------------------------------------------------------------------------
// K2 simple: one node per thread, neighbours through the read-only cache.
// ---------------------------------------------------------------------------
template <int DT, int S, int BCM, bool TRACK>
__global__ void __launch_bounds__(256) k2_simple(Level cur, Level nxt, Geo g,
                                                 Coef3<typename St<DT>::V> a, ExactTab ex,
                                                 Reduce rd, int gw) {
    using T = St<DT>;
    using V = typename T::V;
    const int i = blockIdx.x * 32 + threadIdx.x;
    const int j = blockIdx.y * 8 + threadIdx.y;
    double s0 = 0, s1 = 0, m0 = 0, m1 = 0;
    if (i < g.nx && j < g.ny) {
        const size_t o = off(g, i, j);
        const size_t P = (size_t)g.pitch;
        Nbr<V> u;
        u.c = T::ldg(cur, o);
        u.e = T::ldg(cur, o + 1);
        u.w = T::ldg(cur, o - 1);
        u.n = T::ldg(cur, o + P);
        u.s = T::ldg(cur, o - P);
        if constexpr (S >= 9) {
            u.ne = T::ldg(cur, o + P + 1);
            u.nw = T::ldg(cur, o + P - 1);
            u.se = T::ldg(cur, o - P + 1);
            u.sw = T::ldg(cur, o - P - 1);
        }
        if constexpr (S == 13) {
            u.ee = T::ldg(cur, o + 2);
            u.ww = T::ldg(cur, o - 2);
            u.nn = T::ldg(cur, o + 2 * P);
            u.ss = T::ldg(cur, o - 2 * P);
        }
        const V p = T::ld(nxt, o);
        const V r = two_step_update<S>(u, p, a);
        T::st(nxt, o, r);
        if (BCM != BCM_ZERO) write_images_bc<DT, BCM>(nxt, g, i, j, r, gw);
        if (TRACK) error_terms(T::to_d(r), exact_at(ex, i, j), s0, s1, m0, m1, rd.status);
    }
    if (TRACK) reduce_finalize<256>(s0, s1, m0, m1, rd);
}

// ---------------------------------------------------------------------------
// K4: FP64 norms of one level against the exact solution.
// ---------------------------------------------------------------------------
template <int DT>
__global__ void __launch_bounds__(256) k4_norms(Level L, Geo g, ExactTab ex, Reduce rd) {
    using T = St<DT>;
    double s0 = 0, s1 = 0, m0 = 0, m1 = 0;
    for (int j = blockIdx.y; j < g.ny; j += gridDim.y)
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.nx; i += gridDim.x * blockDim.x)
            error_terms(T::to_d(T::ld(L, off(g, i, j))), exact_at(ex, i, j), s0, s1, m0, m1,
                        rd.status);
    reduce_finalize<256>(s0, s1, m0, m1, rd);
}

// ---------------------------------------------------------------------------
// K2 persistent: every level of a run in one cooperative launch, for grids
// too small to fill the GPU, where a launch per level costs more than the
// level itself.  Blocks stride over the nodes of a level (one node per thread
// per pass, as in k2_simple: the same per-node arithmetic, in place over
// u^{k-1}), then meet at a grid barrier before the next level.  Neighbours are
// read through L2 (ld.global.cg): another SM wrote them a level ago, and L1 is
// not coherent between SMs.
// ---------------------------------------------------------------------------

// Grid barrier: a 64-bit arrival count that only grows; barrier e of a launch
// completes when every block has arrived e + 1 times.  The wait is bounded
// (limit SM clocks): on expiry the block raises STATUS_TIMEOUT and returns
// false, and the kernel ends (the other blocks then expire at their next
// barrier).  Needs every block resident: a cooperative launch.
__device__ __forceinline__ bool grid_barrier(unsigned long long* arrived, unsigned long long target, int* status,
                                            long long limit) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        ok = 1;
        __threadfence();  // this block's stores of the level before the arrival
        atomicAdd(arrived, 1ull);
        const long long t0 = clock64();
        while (*(volatile unsigned long long*)arrived < target) {
            if (clock64() - t0 > limit) {
                atomicOr(status, STATUS_TIMEOUT);
                ok = 0;
                break;
            }
        }
        __threadfence();  // the other blocks' stores before this block's next reads
    }
    __syncthreads();
    return ok != 0;
}

template <int DT, int S, int BCM>
__global__ void __launch_bounds__(512) k2_persist(Level A, Level B, Geo g, Coef3<typename St<DT>::V> a,
                                                  int n_levels, unsigned long long* arrived, int* status, int gw,
                                                  long long limit) {
    using T = St<DT>;
    using V = typename T::V;
    const long long nn = (long long)g.nx * g.ny;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const size_t P = (size_t)g.pitch;
    for (int l = 0; l < n_levels; ++l) {
        const Level cur = (l & 1) ? B : A;  // u^k
        const Level nxt = (l & 1) ? A : B;  // u^{k-1}, overwritten with u^{k+1}
        for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < nn; q += stride) {
            const int i = (int)(q % g.nx), j = (int)(q / g.nx);
            const size_t o = off(g, i, j);
            Nbr<V> u;
            u.c = T::ldcg(cur, o);
            u.e = T::ldcg(cur, o + 1);
            u.w = T::ldcg(cur, o - 1);
            u.n = T::ldcg(cur, o + P);
            u.s = T::ldcg(cur, o - P);
            if constexpr (S >= 9) {
                u.ne = T::ldcg(cur, o + P + 1);
                u.nw = T::ldcg(cur, o + P - 1);
                u.se = T::ldcg(cur, o - P + 1);
                u.sw = T::ldcg(cur, o - P - 1);
            }
            if constexpr (S == 13) {
                u.ee = T::ldcg(cur, o + 2);
                u.ww = T::ldcg(cur, o - 2);
                u.nn = T::ldcg(cur, o + 2 * P);
                u.ss = T::ldcg(cur, o - 2 * P);
            }
            const V r = two_step_update<S>(u, T::ldcg(nxt, o), a);
            T::st(nxt, o, r);
            if (BCM != BCM_ZERO) write_images_bc<DT, BCM>(nxt, g, i, j, r, gw);
        }
        if (l + 1 < n_levels && !grid_barrier(arrived, (unsigned long long)(l + 1) * gridDim.x, status, limit))
            return;
    }
}

// Self-test of the grid barrier's bounded wait: one block waits for arrivals
// that never come (target 2, one arrival), gives up after `limit` clocks and
// raises STATUS_TIMEOUT.
static __global__ void k_selftest_grid_wait(unsigned long long* arrived, int* status, long long limit) {
    grid_barrier(arrived, 2ull, status, limit);
}

// Norms of the difference of two fields of the same grid (any storage types),
// relative to the second: the sums of k4_norms with b's value in place of the
// exact solution.
template <int DTA, int DTB>
__global__ void __launch_bounds__(256) k_diff_norms(Level A, Geo ga, Level B, Geo gb, Reduce rd) {
    double s0 = 0, s1 = 0, m0 = 0, m1 = 0;
    for (int j = blockIdx.y; j < ga.ny; j += gridDim.y)
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ga.nx; i += gridDim.x * blockDim.x)
            error_terms(St<DTA>::to_d(St<DTA>::ld(A, off(ga, i, j))), St<DTB>::to_d(St<DTB>::ld(B, off(gb, i, j))),
                        s0, s1, m0, m1, rd.status);
    reduce_finalize<256>(s0, s1, m0, m1, rd);
}

// ---------------------------------------------------------------------------
// Plane <-> plain FP64 array.
// ---------------------------------------------------------------------------
template <int DT>
__global__ void __launch_bounds__(256) k_pack(Level L, Geo g, double* __restrict__ out) {
    const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y;
    if (i < g.nx && j < g.ny) out[(size_t)j * g.nx + i] = St<DT>::to_d(St<DT>::ld(L, off(g, i, j)));
}

template <int DT, int BCM>
__global__ void __launch_bounds__(256) k_unpack(const double* __restrict__ in, Level L, Geo g, int gw) {
    const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y;
    if (i < g.nx && j < g.ny) {
        const typename St<DT>::V v = St<DT>::from_d(in[(size_t)j * g.nx + i]);
        St<DT>::st(L, off(g, i, j), v);
        if (BCM != BCM_ZERO) write_images_bc<DT, BCM>(L, g, i, j, v, gw);
    }
}

// ---------------------------------------------------------------------------
// TMA / mbarrier primitives (inline PTX).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* tm, uint64_t* bar, int x,
                                            int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Spin on an mbarrier phase with a deadline: ~2^31 SM clocks (about a second
// at the GB300 clocks).  Returns false and raises STATUS_TIMEOUT on expiry.
constexpr long long kWaitLimitCycles = 1LL << 31;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, int* status,
                                                  long long limit = kWaitLimitCycles) {
    if (mbar_test_wait(bar, parity)) return true;
    const long long t0 = clock64();
    unsigned ns = 16;
    while (!mbar_test_wait(bar, parity)) {
        if (clock64() - t0 > limit) {
            atomicOr(status, STATUS_TIMEOUT);
            return false;
        }
        __nanosleep(ns);
        if (ns < 256) ns <<= 1;
    }
    return true;
}

// ---------------------------------------------------------------------------
// K2 TMA: persistent CTAs walk the tiles of the grid.  Per tile one thread
// issues two TMA box loads into a pipeline stage (u^k with a halo of R rows
// and one 16-byte vector of columns on each side, u^{k-1} without halo);
// NSTAGES tiles are in flight per CTA.  Each warp owns TH/NW output rows of
// the tile; lane l owns one 16-byte column vector and walks down its rows
// keeping the 2R+1 rows it needs in registers, so every shared-memory row is
// read once per warp.  Stores go straight to global memory (in place over
// u^{k-1}, which this tile has already staged).
// ---------------------------------------------------------------------------
template <typename T>
struct TmaVec;
template <>
struct TmaVec<float> {
    static constexpr int N = 4;
};
template <>
struct TmaVec<double> {
    static constexpr int N = 2;
};

template <typename T, int S, int TH, int NW>
struct TmaCfg {
    static constexpr int VEC = TmaVec<T>::N;
    static constexpr int R = (S == 13) ? 2 : 1;
    static constexpr int TW = 32 * VEC;
    static constexpr int BOX_W = TW + 2 * VEC;
    static constexpr int BOX_H = TH + 2 * R;
    static constexpr int CUR_BYTES = ((BOX_W * BOX_H * (int)sizeof(T)) + 127) / 128 * 128;
    static constexpr int PREV_BYTES = ((TW * TH * (int)sizeof(T)) + 127) / 128 * 128;
    static constexpr int STAGE_BYTES = CUR_BYTES + PREV_BYTES;
    static constexpr int RPW = TH / NW;
    static_assert(TH % NW == 0, "rows per warp");
    static_assert(BOX_W <= 256 && BOX_H <= 256, "TMA box limit");
};

template <typename T, int NV>
struct RowBuf {
    T a[NV + 4];  // x-2, x-1, x .. x+NV-1, x+NV, x+NV+1
};

template <typename T, int NV>
__device__ __forceinline__ RowBuf<T, NV> load_row(const T* row, int lane) {
    RowBuf<T, NV> r;
    if constexpr (NV == 4) {
        const float2 lp = *reinterpret_cast<const float2*>(row + (lane + 1) * 4 - 2);
        const float4 v = *reinterpret_cast<const float4*>(row + (lane + 1) * 4);
        const float2 rp = *reinterpret_cast<const float2*>(row + (lane + 2) * 4);
        r.a[0] = lp.x; r.a[1] = lp.y;
        r.a[2] = v.x; r.a[3] = v.y; r.a[4] = v.z; r.a[5] = v.w;
        r.a[6] = rp.x; r.a[7] = rp.y;
    } else {
        const double2 lp = *reinterpret_cast<const double2*>(row + (lane + 1) * 2 - 2);
        const double2 v = *reinterpret_cast<const double2*>(row + (lane + 1) * 2);
        const double2 rp = *reinterpret_cast<const double2*>(row + (lane + 2) * 2);
        r.a[0] = lp.x; r.a[1] = lp.y;
        r.a[2] = v.x; r.a[3] = v.y;
        r.a[4] = rp.x; r.a[5] = rp.y;
    }
    return r;
}

template <typename T, int S, int BCM, int TH, int NW, int NSTAGES>
__global__ void __launch_bounds__(NW * 32, 1)
    k2_tma(const __grid_constant__ CUtensorMap tm_cur, const __grid_constant__ CUtensorMap tm_prev,
           T* __restrict__ nxt, Geo g, Coef3<T> a, int tiles_x, int n_tiles, int gw, int* status) {
    using C = TmaCfg<T, S, TH, NW>;
    constexpr int VEC = C::VEC, R = C::R, TW = C::TW, BOX_W = C::BOX_W, RPW = C::RPW;
    constexpr int DT = sizeof(T) == 4 ? DT_F32 : DT_F64;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);
    unsigned char* stages = smem_raw + 1024;
    __shared__ int abort_flag;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        for (int s = 0; s < NSTAGES; ++s) mbar_init(&bars[s], 1);
        fence_barrier_init();
        fence_proxy_async_smem();
        abort_flag = 0;
    }
    __syncthreads();

    auto issue = [&](int t, int s) {
        const int tx = t % tiles_x, ty = t / tiles_x;
        unsigned char* st = stages + (size_t)s * C::STAGE_BYTES;
        mbar_arrive_expect_tx(&bars[s], (unsigned)(BOX_W * C::BOX_H * sizeof(T) + TW * TH * sizeof(T)));
        tma_load_2d(st, &tm_cur, &bars[s], g.G + tx * TW - VEC, g.G + ty * TH - R);
        tma_load_2d(st + C::CUR_BYTES, &tm_prev, &bars[s], g.G + tx * TW, g.G + ty * TH);
    };

    const int stride = gridDim.x;
    if (tid == 0) {
        for (int s = 0; s < NSTAGES; ++s) {
            const int t = blockIdx.x + s * stride;
            if (t < n_tiles) issue(t, s);
        }
    }

    int it = 0;
    for (int t = blockIdx.x; t < n_tiles; t += stride, ++it) {
        const int s = it % NSTAGES;
        const unsigned parity = (unsigned)(it / NSTAGES) & 1u;
        const bool ok = mbar_wait_bounded(&bars[s], parity, status);
        if (!__syncthreads_and(ok)) {
            if (tid == 0) abort_flag = 1;
            break;
        }
        const T* cur_s = reinterpret_cast<const T*>(stages + (size_t)s * C::STAGE_BYTES);
        const T* prev_s = reinterpret_cast<const T*>(stages + (size_t)s * C::STAGE_BYTES + C::CUR_BYTES);
        const int tx = t % tiles_x, ty = t / tiles_x;
        const int x = tx * TW + lane * VEC;  // first column of this lane's vector
        const int r0 = warp * RPW;            // first output row of this warp (tile coords)
        const bool edge = BCM != BCM_ZERO && (tx * TW < gw || tx * TW + TW > g.nx - gw || ty * TH < gw ||
                                              ty * TH + TH > g.ny - gw);
        // whole-vector images: periodic mode only (odd images are mirrored)
        const bool vec_images = BCM == BCM_PERIODIC && (g.nx % VEC == 0) && g.nx >= 2 * gw && g.ny >= 2 * gw;

        // register window: win[q] holds tile row (r - R + q) of u^k
        RowBuf<T, VEC> win[2 * R + 1];
#pragma unroll
        for (int q = 1; q < 2 * R + 1; ++q) win[q] = load_row<T, VEC>(cur_s + (r0 + q - 1) * BOX_W, lane);
#pragma unroll
        for (int r = 0; r < RPW; ++r) {
#pragma unroll
            for (int q = 0; q < 2 * R; ++q) win[q] = win[q + 1];
            win[2 * R] = load_row<T, VEC>(cur_s + (r0 + r + 2 * R) * BOX_W, lane);
            T pv[VEC];
            if constexpr (VEC == 4) {
                const float4 p = *reinterpret_cast<const float4*>(prev_s + (r0 + r) * TW + lane * 4);
                pv[0] = p.x; pv[1] = p.y; pv[2] = p.z; pv[3] = p.w;
            } else {
                const double2 p = *reinterpret_cast<const double2*>(prev_s + (r0 + r) * TW + lane * 2);
                pv[0] = p.x; pv[1] = p.y;
            }
            T out[VEC];
#pragma unroll
            for (int e = 0; e < VEC; ++e) {
                Nbr<T> u;
                const RowBuf<T, VEC>& c = win[R];
                const RowBuf<T, VEC>& up = win[R + 1];
                const RowBuf<T, VEC>& dn = win[R - 1];
                u.c = c.a[e + 2];
                u.e = c.a[e + 3];
                u.w = c.a[e + 1];
                u.n = up.a[e + 2];
                u.s = dn.a[e + 2];
                if constexpr (S >= 9) {
                    u.ne = up.a[e + 3];
                    u.nw = up.a[e + 1];
                    u.se = dn.a[e + 3];
                    u.sw = dn.a[e + 1];
                }
                if constexpr (S == 13) {
                    u.ee = c.a[e + 4];
                    u.ww = c.a[e];
                    u.nn = win[R + 2].a[e + 2];
                    u.ss = win[R - 2].a[e + 2];
                }
                out[e] = two_step_update<S>(u, pv[e], a);
            }
            const int y = ty * TH + r0 + r;
            if (y < g.ny) {
                T* gp = nxt + off(g, x, y);
                if (x + VEC <= g.nx) {
                    if constexpr (VEC == 4) {
                        const float4 v = make_float4(out[0], out[1], out[2], out[3]);
                        *reinterpret_cast<float4*>(gp) = v;
                        if (edge && vec_images) store_vec_images(reinterpret_cast<float4*>(nxt), g, x, y, v, gw, 4);
                    } else {
                        const double2 v = make_double2(out[0], out[1]);
                        *reinterpret_cast<double2*>(gp) = v;
                        if (edge && vec_images) store_vec_images(reinterpret_cast<double2*>(nxt), g, x, y, v, gw, 2);
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < VEC; ++e)
                        if (x + e < g.nx) gp[e] = out[e];
                }
            }
        }
        if (edge && !vec_images) {
            // Odd images, or grids too small or not a multiple of the vector
            // width: images node by node, in a rolled loop that re-reads the
            // stored values.
            const Level L{nxt, nullptr};
#pragma unroll 1
            for (int r = 0; r < RPW; ++r) {
                const int y = ty * TH + r0 + r;
                if (y >= g.ny) break;
#pragma unroll 1
                for (int e = 0; e < VEC; ++e)
                    if (x + e < g.nx) write_images_bc<DT, BCM>(L, g, x + e, y, nxt[off(g, x + e, y)], gw);
            }
        }
        __syncthreads();  // every warp is done with stage s
        if (tid == 0) {
            const int tn = t + NSTAGES * stride;
            if (tn < n_tiles) issue(tn, s);
        }
    }

    if (abort_flag && tid == 0) {
        // Drain: wait (bounded) for the copies still in flight before exit.
        int it2 = it;
        for (int t = blockIdx.x + it * stride; t < n_tiles && it2 < it + NSTAGES; t += stride, ++it2)
            mbar_wait_bounded(&bars[it2 % NSTAGES], (unsigned)(it2 / NSTAGES) & 1u, status);
    }
}

}  // namespace w2d
