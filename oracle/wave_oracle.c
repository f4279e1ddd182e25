/*
 * Plain FP64 CPU oracle for the explicit stencil schemes of Khutoryansky,
 * "Explicit stencil computation schemes generated by Poisson's formula for
 * the 2D wave equation" (arXiv:1904.04048).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code with the CUDA library.
 *
 * Every update below is written the way the paper prints it in Section 6:
 * the first-time-step expressions (Eq. comp5.1, comp5.1a, comp9.1, comp9.1b,
 * comp13.1 and the conventional 13-point first step named in Section 6.3) and
 * the two-step expressions (Eq. comp5.2, comp9.2, comp9.2b, comp13.2), with
 * the stencil sums delta / epsilon of Eq. notations2.  Compiled with
 * -ffp-contract=off so that no FMA contraction changes the rounding.
 *
 * Array convention: a field on an nx-by-ny node set is stored row-major,
 * element (i, j) at index j*nx + i, where i counts along x1 and j along x2.
 * Boundary handling (Section 6.1.2 and Section 6.3):
 *   ORC_BC_ZERO      nodes outside 0..nx-1 / 0..ny-1 hold zero at every level
 *                    (the grid boundary condition of Section 6.1.2, extended
 *                    to a zero ring of width 2 for the 13-point scheme);
 *   ORC_BC_PERIODIC  indices wrap modulo nx / ny (Section 6.3).
 *   ORC_BC_ODD       the Dirichlet condition of Section 6.1.2 (u = 0 on the
 *                    boundary nodes i = -1 and i = nx, likewise in j) with the
 *                    field continued beyond them as an odd function:
 *                    u(-1 - k) = -u(-1 + k), u(nx + k) = -u(nx - k).  For
 *                    radius-1 stencils this reads only the boundary nodes and
 *                    equals ORC_BC_ZERO; for wider ones it is the reflection
 *                    the paper leaves open for the 13-point scheme.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

enum { ORC_BC_ZERO = 0, ORC_BC_PERIODIC = 1, ORC_BC_ODD = 2 };

/* Odd continuation of an index about the boundary nodes -1 and n: returns the
 * interior index and multiplies *sign by -1 per reflection; -1 for a
 * boundary node (value 0). */
static int odd_index(int i, int n, double *sign)
{
    for (;;) {
        if (i == -1 || i == n) return -1;
        if (i < -1) { i = -2 - i; *sign = -*sign; continue; }
        if (i > n) { i = 2 * n - i; *sign = -*sign; continue; }
        return i;
    }
}
enum { ORC_EXACT_NONE = 0, ORC_EXACT_STANDING = 1, ORC_EXACT_PLANE = 2 };

/* Value of a grid function at node (i, j) under the boundary rule. */
static double at(const double *u, int nx, int ny, int bc, int i, int j)
{
    if (bc == ORC_BC_PERIODIC) {
        i = ((i % nx) + nx) % nx;
        j = ((j % ny) + ny) % ny;
        return u[(size_t)j * nx + i];
    }
    if (bc == ORC_BC_ODD) {
        double sign = 1.0;
        i = odd_index(i, nx, &sign);
        j = odd_index(j, ny, &sign);
        if (i < 0 || j < 0) return 0.0;
        return sign * u[(size_t)j * nx + i];
    }
    if (i < 0 || i >= nx || j < 0 || j >= ny)
        return 0.0;
    return u[(size_t)j * nx + i];
}

/* delta_ij(q1,q2) of Eq. notations2: the four 90-degree rotations of the
 * offset (q1,q2) about node (i,j), summed in the printed order, minus four
 * times the centre value.  (The printed "i1-q1" in the third term is read as
 * i-q1.)  The same sum over v0 is epsilon_ij(q1,q2). */
static double delta(const double *u, int nx, int ny, int bc, int i, int j, int q1, int q2)
{
    double s = at(u, nx, ny, bc, i + q1, j + q2);
    s = s + at(u, nx, ny, bc, i - q2, j + q1);
    s = s + at(u, nx, ny, bc, i - q1, j - q2);
    s = s + at(u, nx, ny, bc, i + q2, j - q1);
    return s - 4.0 * at(u, nx, ny, bc, i, j);
}

/* ---------------------------------------------------------------------- */
/* Coefficients as printed in Section 6.  For reporting and for the tests  */
/* that re-derive them from Sections 4-5: the updates below use the printed */
/* expressions directly, not this table.                                   */
/*   a[0..2]  multiply delta(1,0), delta(1,1), delta(2,0) in the two-step   */
/*   b[0..2]  multiply epsilon(1,0), epsilon(1,1), epsilon(2,0) in the first */
/*            step, divided by tau (the first step adds tau * b . epsilon)  */
/* The first step adds a/2 . delta(u0); conventional = 1 selects the        */
/* comparison schemes (Eq. comp5.1a, comp9.1b/9.2b, conventional 13-point),  */
/* whose b are zero.  Returns 0, or -1 for an unknown scheme.               */
/* ---------------------------------------------------------------------- */
int oracle_coeffs(int scheme, int conventional, double lam, double *a, double *b)
{
    double l2 = lam * lam;
    a[0] = a[1] = a[2] = 0.0;
    b[0] = b[1] = b[2] = 0.0;
    if (scheme == 5) {
        a[0] = l2;                                   /* Eq. comp5.2 */
        if (!conventional) b[0] = l2 / 6.0;          /* Eq. comp5.1 */
        return 0;
    }
    if (scheme == 9) {
        if (conventional) {                          /* Eq. comp9.2b */
            a[0] = l2 * (2.0 / 3.0);
            a[1] = l2 * (1.0 / 6.0);
        } else {                                     /* Eq. comp9.2 */
            a[0] = l2 * (1.0 - l2 / 3.0);
            a[1] = l2 * (l2 / 6.0);
            b[0] = (l2 / 6.0) * (1.0 - l2 / 5.0);    /* Eq. comp9.1 */
            b[1] = (l2 / 6.0) * (l2 / 10.0);
        }
        return 0;
    }
    if (scheme == 13) {                              /* Eq. comp13.2 */
        a[0] = l2 * ((4.0 - 2.0 * l2) / 3.0);
        a[1] = l2 * (l2 / 6.0);
        a[2] = l2 * ((l2 - 1.0) / 12.0);
        if (!conventional) {                         /* Eq. comp13.1 */
            b[0] = (l2 / 6.0) * (4.0 / 3.0 - 2.0 * l2 / 5.0);
            b[1] = (l2 / 6.0) * (l2 / 10.0);
            b[2] = (l2 / 6.0) * (l2 / 20.0 - 1.0 / 12.0);
        }
        return 0;
    }
    return -1;
}

/* ---------------------------------------------------------------------- */
/* First time step, Eq. A1 in the discrete forms of Section 6.            */
/* ---------------------------------------------------------------------- */
static double first_step_point(int scheme, int conventional, int bc, int nx, int ny,
                               double lam, double tau, const double *u0, const double *v0,
                               int i, int j)
{
    double l2 = lam * lam;
    double c = u0[(size_t)j * nx + i] + tau * v0[(size_t)j * nx + i];
    if (scheme == 5) {
        /* Eq. comp5.1 (new) and Eq. comp5.1a (conventional) */
        double r = c + (l2 / 2.0) * delta(u0, nx, ny, bc, i, j, 1, 0);
        if (!conventional)
            r = r + (tau * l2 / 6.0) * delta(v0, nx, ny, bc, i, j, 1, 0);
        return r;
    }
    if (scheme == 9) {
        if (conventional) {
            /* Eq. comp9.1b */
            return c + (l2 / 2.0) * ((2.0 / 3.0) * delta(u0, nx, ny, bc, i, j, 1, 0) +
                                     (1.0 / 6.0) * delta(u0, nx, ny, bc, i, j, 1, 1));
        }
        /* Eq. comp9.1 */
        double r = c + (l2 / 2.0) * ((1.0 - l2 / 3.0) * delta(u0, nx, ny, bc, i, j, 1, 0) +
                                     (l2 / 6.0) * delta(u0, nx, ny, bc, i, j, 1, 1));
        r = r + (tau * l2 / 6.0) * ((1.0 - l2 / 5.0) * delta(v0, nx, ny, bc, i, j, 1, 0) +
                                    (l2 / 10.0) * delta(v0, nx, ny, bc, i, j, 1, 1));
        return r;
    }
    /* scheme 13: Eq. comp13.1; the conventional first step drops the epsilon
     * bracket (central difference in time for v, Section 6.3). */
    double r = c + (l2 / 2.0) * (((4.0 - 2.0 * l2) / 3.0) * delta(u0, nx, ny, bc, i, j, 1, 0) +
                                 (l2 / 6.0) * delta(u0, nx, ny, bc, i, j, 1, 1) +
                                 ((l2 - 1.0) / 12.0) * delta(u0, nx, ny, bc, i, j, 2, 0));
    if (!conventional)
        r = r + (tau * l2 / 6.0) * ((4.0 / 3.0 - 2.0 * l2 / 5.0) * delta(v0, nx, ny, bc, i, j, 1, 0) +
                                    (l2 / 10.0) * delta(v0, nx, ny, bc, i, j, 1, 1) +
                                    (l2 / 20.0 - 1.0 / 12.0) * delta(v0, nx, ny, bc, i, j, 2, 0));
    return r;
}

/* ---------------------------------------------------------------------- */
/* Second and next time steps, Eq. A2 in the discrete forms of Section 6. */
/* ---------------------------------------------------------------------- */
static double two_step_point(int scheme, int conventional, int bc, int nx, int ny, double lam,
                             const double *uk, const double *ukm1, int i, int j)
{
    double l2 = lam * lam;
    double base = 2.0 * uk[(size_t)j * nx + i] - ukm1[(size_t)j * nx + i];
    if (scheme == 5) {
        /* Eq. comp5.2 */
        return base + l2 * delta(uk, nx, ny, bc, i, j, 1, 0);
    }
    if (scheme == 9) {
        if (conventional) /* Eq. comp9.2b */
            return base + l2 * ((2.0 / 3.0) * delta(uk, nx, ny, bc, i, j, 1, 0) +
                                 (1.0 / 6.0) * delta(uk, nx, ny, bc, i, j, 1, 1));
        /* Eq. comp9.2 */
        return base + l2 * ((1.0 - l2 / 3.0) * delta(uk, nx, ny, bc, i, j, 1, 0) +
                            (l2 / 6.0) * delta(uk, nx, ny, bc, i, j, 1, 1));
    }
    /* Eq. comp13.2, with the printed delta^0 read as delta^k */
    return base + l2 * (((4.0 - 2.0 * l2) / 3.0) * delta(uk, nx, ny, bc, i, j, 1, 0) +
                        (l2 / 6.0) * delta(uk, nx, ny, bc, i, j, 1, 1) +
                        ((l2 - 1.0) / 12.0) * delta(uk, nx, ny, bc, i, j, 2, 0));
}

static int valid_scheme(int scheme) { return scheme == 5 || scheme == 9 || scheme == 13; }

int oracle_first_step(int scheme, int conventional, int bc, int nx, int ny, double lam, double tau,
                      const double *u0, const double *v0, double *u1)
{
    if (!valid_scheme(scheme) || nx <= 0 || ny <= 0) return -1;
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i)
            u1[(size_t)j * nx + i] =
                first_step_point(scheme, conventional, bc, nx, ny, lam, tau, u0, v0, i, j);
    return 0;
}

int oracle_two_step(int scheme, int conventional, int bc, int nx, int ny, double lam,
                    const double *uk, const double *ukm1, double *ukp1)
{
    if (!valid_scheme(scheme) || nx <= 0 || ny <= 0) return -1;
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i)
            ukp1[(size_t)j * nx + i] = two_step_point(scheme, conventional, bc, nx, ny, lam, uk, ukm1, i, j);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Exact benchmark solutions.                                              */
/*   STANDING: p[0]*sin(2 pi p[1] x1) sin(2 pi p[1] x2) sin(2 sqrt2 pi p[1] c t) */
/*             (Eq. "exact sol" of Section 6.1.2 for p = {1, 1})           */
/*   PLANE:    p[0]*cos(p[1] x1 + p[2] x2 - c |k| t), k = (p[1], p[2])      */
/* Node (i, j) sits at x1 = (i + x_off) h, x2 = (j + x_off) h.             */
/* ---------------------------------------------------------------------- */
static double exact_value(int kind, const double *p, double c, double x1, double x2, double t)
{
    const double pi = 3.14159265358979323846;
    if (kind == ORC_EXACT_STANDING) {
        double m = p[1];
        return p[0] * sin(2.0 * pi * m * x1) * sin(2.0 * pi * m * x2) *
               sin(2.0 * sqrt(2.0) * pi * m * c * t);
    }
    if (kind == ORC_EXACT_PLANE) {
        double kk = sqrt(p[1] * p[1] + p[2] * p[2]);
        return p[0] * cos(p[1] * x1 + p[2] * x2 - c * kk * t);
    }
    return 0.0;
}

/* Sums over all nodes at time t: out[0] += sum (u - u_e)^2, out[1] += sum u_e^2,
 * out[2] = max(out[2], max |u - u_e|).  These are the per-level parts of the
 * relative error E(n, n_t) of Eq. error. */
void oracle_error_sums(const double *u, int nx, int ny, double h, double x_off, int kind,
                       const double *p, double c, double t, double *out)
{
    double se = 0.0, sx = 0.0, mx = out[2];
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            double ue = exact_value(kind, p, c, (i + x_off) * h, (j + x_off) * h, t);
            double d = u[(size_t)j * nx + i] - ue;
            se = se + d * d;
            sx = sx + ue * ue;
            if (fabs(d) > mx) mx = fabs(d);
        }
    out[0] += se;
    out[1] += sx;
    out[2] = mx;
}

/* Whole time-stepping algorithm of Section 3: the first step (Eq. A1), then
 * n_t - 1 two-steps (Eq. A2).  On return u_prev = u^{n_t-1}, u_cur = u^{n_t}
 * (for n_t == 0: u_prev = u_cur = u^0).  If kind != ORC_EXACT_NONE, err[0..2]
 * receive the sums of oracle_error_sums accumulated over k = 1..n_t (the
 * numerator and denominator of E(n, n_t), Eq. error) and the space-time
 * maximum error.  Returns 0, or -1 on bad arguments / allocation failure. */
int oracle_run(int scheme, int conventional, int bc, int nx, int ny, double lam, double tau,
               const double *u0, const double *v0, int64_t n_t, double h, double x_off,
               int kind, const double *p, double c, double *u_prev, double *u_cur, double *err)
{
    if (!valid_scheme(scheme) || nx <= 0 || ny <= 0 || n_t < 0) return -1;
    size_t n = (size_t)nx * ny;
    if (err) { err[0] = err[1] = err[2] = 0.0; }
    if (n_t == 0) {
        memcpy(u_prev, u0, n * sizeof(double));
        memcpy(u_cur, u0, n * sizeof(double));
        return 0;
    }
    double *a = (double *)malloc(n * sizeof(double));
    double *b = (double *)malloc(n * sizeof(double));
    double *w = (double *)malloc(n * sizeof(double));
    if (!a || !b || !w) { free(a); free(b); free(w); return -1; }
    memcpy(a, u0, n * sizeof(double));
    oracle_first_step(scheme, conventional, bc, nx, ny, lam, tau, u0, v0, b);
    if (err && kind != ORC_EXACT_NONE) oracle_error_sums(b, nx, ny, h, x_off, kind, p, c, tau, err);
    /* a = u^{k-1}, b = u^k */
    for (int64_t k = 1; k < n_t; ++k) {
        oracle_two_step(scheme, conventional, bc, nx, ny, lam, b, a, w);
        double *t = a; a = b; b = w; w = t;
        if (err && kind != ORC_EXACT_NONE)
            oracle_error_sums(b, nx, ny, h, x_off, kind, p, c, (double)(k + 1) * tau, err);
    }
    memcpy(u_prev, a, n * sizeof(double));
    memcpy(u_cur, b, n * sizeof(double));
    free(a); free(b); free(w);
    return 0;
}

/* Continue the two-step recursion from a given pair (u^{k-1}, u^k) for
 * n_more steps, in place: on return u_prev/u_cur hold the last two levels. */
int oracle_continue(int scheme, int conventional, int bc, int nx, int ny, double lam,
                    double *u_prev, double *u_cur, int64_t n_more)
{
    if (!valid_scheme(scheme) || nx <= 0 || ny <= 0 || n_more < 0) return -1;
    size_t n = (size_t)nx * ny;
    double *w = (double *)malloc(n * sizeof(double));
    double *a = (double *)malloc(n * sizeof(double));
    double *b = (double *)malloc(n * sizeof(double));
    if (!w || !a || !b) { free(w); free(a); free(b); return -1; }
    memcpy(a, u_prev, n * sizeof(double));
    memcpy(b, u_cur, n * sizeof(double));
    for (int64_t k = 0; k < n_more; ++k) {
        oracle_two_step(scheme, conventional, bc, nx, ny, lam, b, a, w);
        double *t = a; a = b; b = w; w = t;
    }
    memcpy(u_prev, a, n * sizeof(double));
    memcpy(u_cur, b, n * sizeof(double));
    free(w); free(a); free(b);
    return 0;
}

/* ------------------------------------------------------------------------
 * Node-weight form of the algorithm, for any stencil produced by the
 * derivation of Sections 4-5 (Eq. Lagrange with the weights A phi_q and
 * B phi_q of Eq. exact1 / exact2):
 *   u^1_ij     = sum_q wa[q] u^0_{i+q1, j+q2} + tau sum_q wb[q] v^0_{i+q1, j+q2}   (Eq. A1)
 *   u^{k+1}_ij = 2 sum_q wa[q] u^k_{i+q1, j+q2} - u^{k-1}_ij                       (Eq. A2)
 * with wa[q] = A phi_q and wb[q] = B phi_q / tau evaluated at the Courant
 * number, the sums taken in the order the nodes are given, and the boundary
 * read through at().  For the segments of the 5-, 9- and 13-point schemes
 * this is the same operator as the printed Section 6 forms above.
 * ------------------------------------------------------------------------ */
static double node_sum(const double *u, int nx, int ny, int bc, int i, int j, int n_nodes,
                       const int *q1, const int *q2, const double *w)
{
    double s = 0.0;
    for (int q = 0; q < n_nodes; ++q)
        s = s + w[q] * at(u, nx, ny, bc, i + q1[q], j + q2[q]);
    return s;
}

/* First step then n_t - 1 two-steps in the node-weight form.  On return
 * u_prev = u^{n_t-1}, u_cur = u^{n_t} (n_t == 0: both u^0).  Returns 0, or -1
 * on bad arguments / allocation failure. */
int oracle_run_nodes(int bc, int nx, int ny, int n_nodes, const int *q1, const int *q2,
                     const double *wa, const double *wb, double tau, const double *u0,
                     const double *v0, int64_t n_t, double *u_prev, double *u_cur)
{
    if (nx <= 0 || ny <= 0 || n_t < 0 || n_nodes <= 0) return -1;
    size_t n = (size_t)nx * ny;
    if (n_t == 0) {
        memcpy(u_prev, u0, n * sizeof(double));
        memcpy(u_cur, u0, n * sizeof(double));
        return 0;
    }
    double *a = (double *)malloc(n * sizeof(double));
    double *b = (double *)malloc(n * sizeof(double));
    double *w = (double *)malloc(n * sizeof(double));
    if (!a || !b || !w) { free(a); free(b); free(w); return -1; }
    memcpy(a, u0, n * sizeof(double));
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i)
            b[(size_t)j * nx + i] = node_sum(u0, nx, ny, bc, i, j, n_nodes, q1, q2, wa) +
                                    tau * node_sum(v0, nx, ny, bc, i, j, n_nodes, q1, q2, wb);
    for (int64_t k = 1; k < n_t; ++k) {
#pragma omp parallel for schedule(static)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i)
                w[(size_t)j * nx + i] = 2.0 * node_sum(b, nx, ny, bc, i, j, n_nodes, q1, q2, wa) -
                                        a[(size_t)j * nx + i];
        double *t = a; a = b; b = w; w = t;
    }
    memcpy(u_prev, a, n * sizeof(double));
    memcpy(u_cur, b, n * sizeof(double));
    free(a); free(b); free(w);
    return 0;
}

int oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}
