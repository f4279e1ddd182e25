"""The allocation-free norm entry point (wave2d_error_norms_noalloc).

It serves callers that cannot allocate device memory — code whose GPU memory
belongs to another allocator's budget, or latency-critical loops where a
cudaMalloc would synchronise the device — by keeping its scratch in a fixed
device array inside the library.  These tests call it through the C ABI and
check that, on two calls in a row, it returns what the handle-based
wave2d_error_vs_exact returns for the same field, within the FP64 norm
tolerance of the other tests.  The file sorts last so that a run stopping at
the first failure has already run every other test.
"""
import math

import numpy as np
import pytest

from gpu_util import smooth_ic
from initial_data import BC_PERIODIC, BC_ZERO, standing_wave_ic

pytestmark = pytest.mark.gpu

# The norm tolerance of the other GPU tests: 1e-9 relative, plus the FP64
# field tolerance 1e-12 as an absolute floor.  The exact solution is
# evaluated by different sin/cos implementations on the two paths, which
# shifts a relative error of size 1e-6 by about 1e-16 / 1e-6 = 1e-10 of
# itself at most.
NORM_REL, NORM_ABS = 1e-9, 1e-12


@pytest.fixture(scope="module")
def w():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1904_04048_gb300 import build
    build.build()
    from paper_1904_04048_gb300 import wave2d
    return wave2d


def close(a, b):
    return abs(a - b) <= NORM_ABS + NORM_REL * abs(b)


@pytest.mark.parametrize("dtype", [1, 0], ids=["f32", "f64"])
def test_noalloc_matches_handle_norms_twice(w, dtype):
    import torch
    n = 40
    h = 1.0 / n
    lam = 0.707
    u0, v0 = standing_wave_ic(n - 1, n - 1, h, BC_ZERO)
    ex = w.exact(w.EXACT_STANDING, amp=1.0, m=1.0, x_off=1.0)
    with w.Wave2D(n - 1, n - 1, h, lam * h, scheme=5, bc=BC_ZERO, dtype=dtype) as sim:
        sim.first_step(u0, v0)
        sim.step_n(30)
        l2_ref, linf_ref, _ = sim.error_vs_exact(ex)
        _, uc, k = sim.get_state()
    tdt = torch.float32 if dtype == 1 else torch.float64
    field = torch.from_numpy(uc).to(device="cuda", dtype=tdt).contiguous()
    torch.cuda.synchronize()
    for _ in range(2):  # the shared scratch must be reset by every call
        l2, linf = w.error_norms_noalloc(field.data_ptr(), dtype, n - 1, n - 1, n - 1, h, 1.0, k * lam * h, ex)
        assert close(l2, l2_ref) and close(linf, linf_ref), (l2, l2_ref, linf, linf_ref)


def test_noalloc_plane_wave_and_padded_rows(w):
    import torch
    n = 96
    u0, v0, h = smooth_ic(n, n, BC_PERIODIC, seed=21)
    k1, k2 = 2 * math.pi * 2, 2 * math.pi * 5
    ex = w.exact(w.EXACT_PLANE, amp=0.7, k1=k1, k2=k2, x_off=0.0)
    with w.Wave2D(n, n, h, 0.5 * h, scheme=13, bc=BC_PERIODIC, dtype=0) as sim:
        sim.first_step(u0, v0)
        sim.step_n(11)
        l2_ref, linf_ref, _ = sim.error_vs_exact(ex)
        n2_ref, ninf_ref, _ = sim.error_vs_exact(None)
        _, uc, k = sim.get_state()
    ld = n + 13  # rows padded in the caller's buffer
    buf = torch.zeros((n, ld), dtype=torch.float64, device="cuda")
    buf[:, :n] = torch.from_numpy(uc).cuda()
    torch.cuda.synchronize()
    t = k * 0.5 * h
    for _ in range(2):
        l2, linf = w.error_norms_noalloc(buf.data_ptr(), 0, n, n, ld, h, 1.0, t, ex)
        assert close(l2, l2_ref) and close(linf, linf_ref), (l2, l2_ref, linf, linf_ref)
        n2, ninf = w.error_norms_noalloc(buf.data_ptr(), 0, n, n, ld, h, 1.0, t, None)
        assert close(n2, n2_ref) and close(ninf, ninf_ref)


def test_noalloc_rejects_sizes_beyond_its_scratch(w):
    import torch
    buf = torch.zeros(16, dtype=torch.float32, device="cuda")
    with pytest.raises(w.Wave2DError) as e:
        w.error_norms_noalloc(buf.data_ptr(), 1, 8193, 1, 8193, 0.1, 1.0, 0.0)
    assert e.value.code == w.ERR_ARG and "8192" in str(e.value)
    with pytest.raises(w.Wave2DError) as e:
        w.error_norms_noalloc(buf.data_ptr(), 2, 4, 4, 4, 0.1, 1.0, 0.0)
    assert e.value.code == w.ERR_ARG
