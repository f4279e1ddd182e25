"""The boundary from plain C (no Python in between, no GPU needed): the
header compiles as strict C99 and C++11, and a C program linked against
libwave2d.so calls the host-side entry points — the stability limits, the
derivation of a scheme from its monomial segment and its limit, the memory
estimate — and the error path of wave2d_create."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INC = os.path.join(ROOT, "include")
PKG = os.path.join(ROOT, "paper_1904_04048_gb300")

PROGRAM = r"""
#include <math.h>
#include <stdio.h>
#include "wave2d.h"

int main(void) {
    wave2d_scheme s;
    double lmax = 0.0;
    wave2d_grid g = {64, 64, WAVE2D_BC_PERIODIC, WAVE2D_F32, 0, 0, NULL};
    wave2d_t h = NULL;
    int rc;
    printf("lambda_max_13 %.15f\n", wave2d_lambda_max(13, 0));
    printf("lambda_max_9c %.15f\n", wave2d_lambda_max(9, 1));
    rc = wave2d_derive_scheme(28, &s);
    printf("derive_28 %d classes %d points %d radius %d\n", rc, s.n_classes, s.n_points, s.radius);
    rc = wave2d_scheme_lambda_max(&s, &lmax);
    printf("lambda_max_28 %d %.12f\n", rc, lmax);
    rc = wave2d_derive_scheme(23, &s);
    printf("derive_23 %d %s\n", rc, rc ? "rejected" : "accepted");
    printf("required_bytes %lld\n", (long long)wave2d_required_bytes(1024, 1024, WAVE2D_F32));
    rc = wave2d_create(&g, 1.0 / 64, 2.0 / 64, 1.0, 13, &h);  /* lambda = 2: unstable */
    printf("create_unstable %d %s\n", rc, wave2d_last_error());
    return 0;
}
"""


@pytest.mark.parametrize("std,lang", [("c99", "c"), ("c++11", "c++")])
def test_header_compiles_strictly(std, lang):
    cc = "gcc" if lang == "c" else "g++"
    if not shutil.which(cc):
        pytest.skip(f"{cc} not found")
    subprocess.run([cc, f"-std={std}", "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only", "-x", lang,
                    os.path.join(INC, "wave2d.h")], check=True)


def test_c_program_calls_the_host_entry_points(tmp_path):
    if not shutil.which("gcc"):
        pytest.skip("gcc not found")
    from paper_1904_04048_gb300 import build
    build.build()
    src = tmp_path / "prog.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "prog"
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", f"-I{INC}", str(src), "-o", str(exe), f"-L{PKG}",
                    "-l:libwave2d.so", f"-Wl,-rpath,{PKG}", "-lm"], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    lines = dict(ln.split(" ", 1) for ln in out.strip().splitlines())
    assert abs(float(lines["lambda_max_13"]) - 2 ** -0.5) < 1e-15
    assert abs(float(lines["lambda_max_9c"]) - 3 ** 0.5 / 2) < 1e-15
    assert lines["derive_28"] == "0 classes 5 points 25 radius 3"
    rc, lmax = lines["lambda_max_28"].split()
    assert rc == "0" and abs(float(lmax) - 2 ** -0.5) < 1e-9
    assert lines["derive_23"].startswith("-1 ")
    assert int(lines["required_bytes"]) > 4 * 1024 * 1024 * 4
    assert lines["create_unstable"].startswith("-2 ")  # WAVE2D_ERR_UNSTABLE
