// Host side of the derived schemes: the derivation of Sections 4-5 of
// arXiv:1904.04048 for any initial segment M*_{<=m} (FP64), and the von
// Neumann stability limit of a scheme in class form.  No device code.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <utility>
#include <vector>

#include "stencil_chain.cuh"
#include "wave2d_impl.cuh"

namespace w2d {
namespace {

constexpr int kMaxSegment = 49;
constexpr int kPow = 9;  // powers of lambda 0..8

// Ordinal number of x1^a1 x2^a2 in the ordered set M* (Eq. g).
int ordinal_g(int a1, int a2) {
    const int s = (a1 + a2) * (a1 + a2 + 1) / 2;
    return a2 < a1 ? s + (a1 - a2) : s + (a2 - a1 + 1);
}

// Stencil index of a McKinney exponent (Eq. invMcKinney): 0, -1, 1, -2, 2, ...
int q_of_alpha(int a) { return (a % 2 ? -1 : 1) * ((a + 1) / 2); }

// q^e for small integers: exact in FP64 (|q| <= 4, e <= 9); 0^0 = 1.
double ipow(int q, int e) {
    double r = 1.0;
    for (int i = 0; i < e; ++i) r *= q;
    return r;
}

double double_factorial(int k) {
    double r = 1.0;
    for (; k > 1; k -= 2) r *= k;
    return r;
}

// A applied to the scaled monomial (y1/h)^a1 (y2/h)^a2 is c lambda^(a1+a2)
// with c = (a1-1)!! (a2-1)!! / (a1+a2-1)!! for even a1, a2 and 0 otherwise
// (Eq. exact1); B / tau gives c / (a1 + a2 + 1) (Eq. exact2).
double a_integral(int a1, int a2) {
    if (a1 % 2 || a2 % 2) return 0.0;
    return double_factorial(a1 - 1) * double_factorial(a2 - 1) / double_factorial(a1 + a2 - 1);
}

// Error-free transforms for the compensated residual.
inline void two_sum(double a, double b, double& s, double& e) {
    s = a + b;
    const double bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
inline void two_prod(double a, double b, double& p, double& e) {
    p = a * b;
    e = std::fma(a, b, -p);
}

// Dense LU with partial pivoting of an n x n row-major matrix.
struct Lu {
    int n = 0;
    std::vector<double> m;
    std::vector<int> piv;
    bool factor(const std::vector<double>& a, int nn) {
        n = nn;
        m = a;
        piv.resize(n);
        for (int k = 0; k < n; ++k) {
            int p = k;
            for (int r = k + 1; r < n; ++r)
                if (std::fabs(m[(size_t)r * n + k]) > std::fabs(m[(size_t)p * n + k])) p = r;
            if (m[(size_t)p * n + k] == 0.0) return false;
            piv[k] = p;
            if (p != k)
                for (int c = 0; c < n; ++c) std::swap(m[(size_t)k * n + c], m[(size_t)p * n + c]);
            for (int r = k + 1; r < n; ++r) {
                const double f = m[(size_t)r * n + k] / m[(size_t)k * n + k];
                m[(size_t)r * n + k] = f;
                for (int c = k + 1; c < n; ++c) m[(size_t)r * n + c] -= f * m[(size_t)k * n + c];
            }
        }
        return true;
    }
    void solve(std::vector<double>& b) const {
        for (int k = 0; k < n; ++k) std::swap(b[k], b[piv[k]]);
        for (int r = 0; r < n; ++r)
            for (int c = 0; c < r; ++c) b[r] -= m[(size_t)r * n + c] * b[c];
        for (int r = n - 1; r >= 0; --r) {
            for (int c = r + 1; c < n; ++c) b[r] -= m[(size_t)r * n + c] * b[c];
            b[r] /= m[(size_t)r * n + r];
        }
    }
};

// x with M x = rhs: LU solve, then two refinement rounds whose residual
// rhs - M x is summed with compensated products and sums.
std::vector<double> solve_refined(const Lu& lu, const std::vector<double>& M, const std::vector<double>& rhs) {
    const int n = lu.n;
    std::vector<double> x = rhs;
    lu.solve(x);
    for (int round = 0; round < 2; ++round) {
        std::vector<double> r(n);
        for (int i = 0; i < n; ++i) {
            double s = rhs[i], c = 0.0;
            for (int j = 0; j < n; ++j) {
                double p, pe, t, te;
                two_prod(M[(size_t)i * n + j], -x[j], p, pe);
                two_sum(s, p, t, te);
                s = t;
                c += te + pe;
            }
            r[i] = s + c;
        }
        lu.solve(r);
        for (int i = 0; i < n; ++i) x[i] += r[i];
    }
    return x;
}

int chain_index(int q1, int q2) {
    for (int c = 0; c < kMaxClasses; ++c)
        if (chain_q1(c) == q1 && chain_q2(c) == q2) return c;
    return -1;
}

}  // namespace

int derive_scheme(int m, wave2d_scheme* out) {
    if (m < 1 || m > kMaxSegment) return set_error(WAVE2D_ERR_ARG, "segment m = %d outside 1..%d", m, kMaxSegment);
    // 1. The segment M*_{<=m}: the m monomials of smallest ordinal g.
    std::vector<std::pair<int, int>> monos;
    for (int d = 0; d <= 12; ++d)
        for (int a1 = 0; a1 <= d; ++a1) monos.push_back({a1, d - a1});
    std::sort(monos.begin(), monos.end(), [](const std::pair<int, int>& x, const std::pair<int, int>& y) {
        return ordinal_g(x.first, x.second) < ordinal_g(y.first, y.second);
    });
    monos.resize(m);
    // 2. Nodes: McKinney images of the exponents.
    std::vector<std::pair<int, int>> nodes;
    for (auto& mu : monos) nodes.push_back({q_of_alpha(mu.first), q_of_alpha(mu.second)});
    {
        auto sorted = nodes;
        std::sort(sorted.begin(), sorted.end());
        if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end())
            return set_error(WAVE2D_ERR_ARG, "segment m = %d: nodes are not distinct", m);
    }
    // 3. The weights w_q of A (and B / tau) satisfy the moment conditions
    //    sum_q w_q mu_s(q) = A(mu_s) for every monomial of the segment, i.e.
    //    D^T w = A(mu) with D[r][s] = mu_s(node r) (Eq. matrix1; w = D^{-T} A(mu)
    //    is the Lagrange-basis form of Eq. Lagrange).  One right-hand side per
    //    power of lambda.
    std::vector<double> Mt((size_t)m * m);
    for (int r = 0; r < m; ++r)
        for (int s = 0; s < m; ++s)
            Mt[(size_t)s * m + r] = ipow(nodes[r].first, monos[s].first) * ipow(nodes[r].second, monos[s].second);
    Lu lu;
    if (!lu.factor(Mt, m)) return set_error(WAVE2D_ERR_ARG, "segment m = %d: D is singular", m);
    std::vector<std::vector<double>> wa(kPow, std::vector<double>(m, 0.0)), wb = wa;
    double scale = 0.0;
    for (int p = 0; p < kPow; p += 2) {
        std::vector<double> ra(m, 0.0), rb(m, 0.0);
        bool any = false;
        for (int s = 0; s < m; ++s)
            if (monos[s].first + monos[s].second == p) {
                ra[s] = a_integral(monos[s].first, monos[s].second);
                rb[s] = ra[s] / (p + 1);
                any = any || ra[s] != 0.0;
            }
        if (!any) continue;
        wa[p] = solve_refined(lu, Mt, ra);
        wb[p] = solve_refined(lu, Mt, rb);
        for (int r = 0; r < m; ++r) scale = std::max(scale, std::max(std::fabs(wa[p][r]), std::fabs(wb[p][r])));
    }
    const double tiny = 1e-13 * scale;
    for (int p = 0; p < kPow; ++p)
        for (int r = 0; r < m; ++r) {
            if (std::fabs(wa[p][r]) < tiny) wa[p][r] = 0.0;
            if (std::fabs(wb[p][r]) < tiny) wb[p][r] = 0.0;
        }
    // 4. Group the non-zero nodes into classes and check the symmetry.
    wave2d_scheme s{};
    s.segment = m;
    bool seen[kMaxClasses] = {};
    int points = 1;
    std::map<std::pair<int, int>, int> index;
    for (int r = 0; r < m; ++r) index[nodes[r]] = r;
    for (int r = 0; r < m; ++r) {
        if (nodes[r] == std::make_pair(0, 0)) continue;
        bool nonzero = false;
        for (int p = 0; p < kPow; ++p) nonzero = nonzero || wa[p][r] != 0.0 || wb[p][r] != 0.0;
        if (!nonzero) continue;
        ++points;
        const int a = std::abs(nodes[r].first), b = std::abs(nodes[r].second);
        const int c = chain_index(std::max(a, b), std::min(a, b));
        if (c < 0)
            return set_error(WAVE2D_ERR_ARG, "segment m = %d: node (%d, %d) lies outside the class chain", m,
                             nodes[r].first, nodes[r].second);
        if (seen[c]) continue;
        seen[c] = true;
        // every node of the class must carry the same weights
        const int q1 = chain_q1(c), q2 = chain_q2(c);
        const int orbit[8][2] = {{q1, q2}, {-q1, -q2}, {-q2, q1}, {q2, -q1},
                                 {q2, q1}, {-q2, -q1}, {-q1, q2}, {q1, -q2}};
        for (int o = 0; o < chain_nodes(c); ++o) {
            auto it = index.find({orbit[o][0], orbit[o][1]});
            for (int p = 0; p < kPow; ++p) {
                const double va = it == index.end() ? 0.0 : wa[p][it->second];
                const double vb = it == index.end() ? 0.0 : wb[p][it->second];
                if (std::fabs(va - wa[p][r]) > 1e-12 * scale || std::fabs(vb - wb[p][r]) > 1e-12 * scale)
                    return set_error(WAVE2D_ERR_ARG,
                                     "segment m = %d: the weights are not symmetric on class (%d, %d)", m, q1, q2);
            }
        }
        for (int p = 0; p < kPow; ++p) {
            s.a[c][p] = 2.0 * wa[p][r];
            s.b[c][p] = wb[p][r];
        }
        s.n_classes = std::max(s.n_classes, c + 1);
    }
    if (s.n_classes == 0) return set_error(WAVE2D_ERR_ARG, "segment m = %d gives no stencil beyond the centre", m);
    s.radius = chain_radius(s.n_classes);
    s.n_points = points;
    *out = s;
    return WAVE2D_OK;
}

double poly_at(const double* c, double lam) {
    double v = 0.0;
    for (int p = kPow - 1; p >= 0; --p) v = v * lam + c[p];
    return v;
}

int check_scheme(const wave2d_scheme* s) {
    if (!s) return set_error(WAVE2D_ERR_ARG, "null scheme");
    if (s->n_classes < 1 || s->n_classes > kMaxClasses)
        return set_error(WAVE2D_ERR_ARG, "n_classes must be 1..%d (got %d)", kMaxClasses, s->n_classes);
    for (int c = 0; c < kMaxClasses; ++c)
        for (int p = 0; p < kPow; ++p) {
            if (!std::isfinite(s->a[c][p]) || !std::isfinite(s->b[c][p]))
                return set_error(WAVE2D_ERR_ARG, "scheme coefficients must be finite");
            if (c >= s->n_classes && (s->a[c][p] != 0.0 || s->b[c][p] != 0.0))
                return set_error(WAVE2D_ERR_ARG, "coefficient of class %d beyond n_classes = %d", c, s->n_classes);
        }
    return WAVE2D_OK;
}

double scheme_lambda_max(const wave2d_scheme* s) {
    // sigma_c(theta) = sum over the class of (cos(q . theta) - 1)
    //               = -2 sum sin^2(q . theta / 2)  (no cancellation near 0)
    constexpr int N = 129;
    const double pi = 3.14159265358979323846;
    const int nc = s->n_classes;
    std::vector<double> sig((size_t)nc * N * N);
    for (int c = 0; c < nc; ++c) {
        const int q1 = chain_q1(c), q2 = chain_q2(c);
        const int orbit[8][2] = {{q1, q2}, {-q1, -q2}, {-q2, q1}, {q2, -q1},
                                 {q2, q1}, {-q2, -q1}, {-q1, q2}, {q1, -q2}};
        for (int i = 0; i < N; ++i)
            for (int j = 0; j < N; ++j) {
                const double t1 = pi * i / (N - 1), t2 = pi * j / (N - 1);
                double v = 0.0;
                for (int o = 0; o < chain_nodes(c); ++o) {
                    const double sn = std::sin(0.5 * (orbit[o][0] * t1 + orbit[o][1] * t2));
                    v -= 2.0 * sn * sn;
                }
                sig[((size_t)c * N + i) * N + j] = v;
            }
    }
    auto stable = [&](double lam) {
        double a[kMaxClasses];
        for (int c = 0; c < nc; ++c) a[c] = poly_at(s->a[c], lam);
        for (size_t q = 0; q < (size_t)N * N; ++q) {
            double S = 0.0;
            for (int c = 0; c < nc; ++c) S += a[c] * sig[(size_t)c * N * N + q];
            if (S < -4.0 - 1e-13 || S > 1e-13) return false;
        }
        return true;
    };
    const double step = 1.0 / 512;
    double lam = 0.0;
    while (lam + step <= 2.0 && stable(lam + step)) lam += step;
    double lo = lam, hi = lam + step;
    for (int it = 0; it < 60; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (stable(mid)) lo = mid;
        else hi = mid;
    }
    return lo;
}

}  // namespace w2d

extern "C" {

int wave2d_derive_scheme(int32_t m, wave2d_scheme* out) {
    if (!out) return w2d::set_error(WAVE2D_ERR_ARG, "null argument");
    return w2d::derive_scheme(m, out);
}

int wave2d_scheme_lambda_max(const wave2d_scheme* s, double* out) {
    if (!out) return w2d::set_error(WAVE2D_ERR_ARG, "null argument");
    const int rc = w2d::check_scheme(s);
    if (rc != WAVE2D_OK) return rc;
    *out = w2d::scheme_lambda_max(s);
    return WAVE2D_OK;
}

}  // extern "C"
