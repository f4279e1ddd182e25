"""The boundary driven from plain C on the GPU: a C99 program linked against
libwave2d.so, with no Python in between, runs the standing wave of Section
6.1.2 (u0 = 0, v0 = 2 sqrt2 pi c sin 2 pi x1 sin 2 pi x2, unit square,
Dirichlet zero boundary, lambda = 0.707) through wave2d_create ->
wave2d_track_error -> wave2d_first_step -> wave2d_step_n ->
wave2d_error_vs_exact on the device, in FP64, and prints the paper's
space-time error E(n, n_t) (Eq. error).  The values must match Table 1 to
the five digits it prints: E_P5(20, 20) = 5.6800e-5 (new first step, Eq.
comp5.1) and E_C5(40, 40) = 4.1234e-3 (conventional first step, Eq.
comp5.1a)."""
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INC = os.path.join(ROOT, "include")
PKG = os.path.join(ROOT, "paper_1904_04048_gb300")

PROGRAM = r"""
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include "wave2d.h"

/* E(n, n_t) of the 5-point scheme for the standing wave; conventional = 1
 * selects the central-difference first step.  Returns 0 on success. */
static int run(int n, int n_t, int conventional, double *E) {
    const double pi = 3.14159265358979323846, lam = 0.707, c = 1.0;
    const int nn = n - 1;                /* interior nodes of the unit square */
    const double h = 1.0 / n, tau = lam * h / c;
    wave2d_grid g = {nn, nn, WAVE2D_BC_ZERO, WAVE2D_F64, conventional ? WAVE2D_CONVENTIONAL : 0, 0, NULL};
    wave2d_exact ex = {WAVE2D_EXACT_STANDING, 0, 1.0, 1.0, 0.0, 0.0, 1.0};
    wave2d_t sim = NULL;
    double l2 = 0.0, linf = 0.0;
    double *u0 = calloc((size_t)nn * nn, sizeof(double));
    double *v0 = calloc((size_t)nn * nn, sizeof(double));
    int i, j, rc;
    if (!u0 || !v0) return -100;
    for (j = 0; j < nn; ++j)
        for (i = 0; i < nn; ++i)
            v0[j * nn + i] = 2.0 * sqrt(2.0) * pi * c * sin(2 * pi * (i + 1) * h) * sin(2 * pi * (j + 1) * h);
    rc = wave2d_create(&g, h, tau, c, 5, &sim);
    if (rc == WAVE2D_OK) rc = wave2d_track_error(sim, &ex);
    if (rc == WAVE2D_OK) rc = wave2d_first_step(sim, u0, v0, 0);
    if (rc == WAVE2D_OK) rc = wave2d_step_n(sim, n_t - 1);
    if (rc == WAVE2D_OK) rc = wave2d_error_vs_exact(sim, &ex, &l2, &linf, E);
    if (rc != WAVE2D_OK) fprintf(stderr, "wave2d error %d: %s\n", rc, wave2d_last_error());
    wave2d_destroy(sim);
    free(u0);
    free(v0);
    return rc;
}

int main(void) {
    double ep = 0.0, ec = 0.0;
    if (run(20, 20, 0, &ep) != 0) return 1;
    if (run(40, 40, 1, &ec) != 0) return 1;
    printf("E_P5_20_20 %.9e\n", ep);
    printf("E_C5_40_40 %.9e\n", ec);
    return 0;
}
"""


def test_c_program_reproduces_table_1_on_the_gpu(tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    if not shutil.which("gcc"):
        pytest.skip("gcc not found")
    from paper_1904_04048_gb300 import build
    build.build()
    src = tmp_path / "table1.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "table1"
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", f"-I{INC}", str(src), "-o", str(exe), f"-L{PKG}",
                    "-l:libwave2d.so", f"-Wl,-rpath,{PKG}", "-lm"], check=True)
    res = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stderr
    got = dict(ln.split() for ln in res.stdout.strip().splitlines())
    # Table 1 prints five significant digits: within half a unit of the last one
    for key, printed, last_unit in (("E_P5_20_20", 5.6800e-5, 1e-9), ("E_C5_40_40", 4.1234e-3, 1e-7)):
        E = float(got[key])
        assert abs(E - printed) <= 0.5 * last_unit, (key, E, printed)
