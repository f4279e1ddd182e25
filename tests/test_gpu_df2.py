"""Double-float (FP32x2) two-step in packed arithmetic, two nodes per thread
(csrc/df2.cu), the kernel of FP32x2 handles above 2^20 nodes: it must
reproduce the one-node kernel bit for bit.

The one-node kernel runs when per-step norms are tracked (its reduction
path), and the persistent kernel evaluates the same per-node arithmetic one
node per thread; both serve as references.  Covered: the 5-, 9- and 13-point
schemes, zero, periodic and odd boundaries, odd and even row widths (a last
pair of one node), a grid 65 nodes wide; and parity with the FP64 oracle at
the FP32x2 tolerance."""
import numpy as np
import pytest

from gpu_util import TOL, rel_errors, smooth_ic
from initial_data import BC_ODD, BC_PERIODIC, BC_ZERO, LAMBDA_MAX

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def w():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1904_04048_gb300 import build
    build.build()
    from paper_1904_04048_gb300 import wave2d
    return wave2d


def _run(w, scheme, u0, v0, h, lam, steps, bc, mode):
    ny, nx = u0.shape
    with w.Wave2D(nx, ny, h, lam * h, scheme=scheme, bc=bc, dtype=w.F32X2) as sim:
        if mode == "packed":
            sim.set_tuning(kernel=w.KERNEL_SIMPLE, use_graph=0)
        elif mode == "tracked":          # one-node kernel with per-step norms
            sim.set_tuning(kernel=w.KERNEL_SIMPLE, use_graph=0)
            sim.track_error(w.exact(w.EXACT_PLANE, k1=1.0))
        else:
            sim.set_tuning(kernel=w.KERNEL_PERSISTENT)
        sim.first_step(u0, v0)
        sim.step_n(steps - 1)
        return sim.get_state()


# every shape above 2^20 nodes, where FP32x2 handles take the packed kernel
SHAPES = [(2049, 2049), (4100, 1100), (65, 65536)]


@pytest.mark.parametrize("scheme", [5, 9, 13])
@pytest.mark.parametrize("bc", [BC_ZERO, BC_PERIODIC, BC_ODD], ids=["zero", "periodic", "odd"])
def test_packed_equals_one_node_bitwise(w, scheme, bc):
    lam = 0.9 * LAMBDA_MAX[scheme]
    for nx, ny in SHAPES:
        assert nx * ny > 1 << 20
        u0, v0, h = smooth_ic(nx, ny, bc, seed=nx * 7 + ny + scheme)
        a = _run(w, scheme, u0, v0, h, lam, 13, bc, "packed")
        b = _run(w, scheme, u0, v0, h, lam, 13, bc, "tracked")
        c = _run(w, scheme, u0, v0, h, lam, 13, bc, "persistent")
        assert a[2] == b[2] == c[2] == 13
        for x, y, z in zip(a[:2], b[:2], c[:2]):
            assert np.array_equal(x, y) and np.array_equal(x, z), (nx, ny)


@pytest.mark.parametrize("scheme", [5, 9, 13])
def test_packed_parity_with_oracle(orc, w, scheme):
    """A 2100 x 2000 grid (above 2^20 nodes), 8 levels: the FP64 oracle on
    the full grid takes a few seconds."""
    nx, ny = 2100, 2000
    u0, v0, h = smooth_ic(nx, ny, BC_PERIODIC, seed=scheme)
    lam = 0.9 * LAMBDA_MAX[scheme]
    steps = 8
    up, uc, _ = _run(w, scheme, u0, v0, h, lam, steps, BC_PERIODIC, "packed")
    rp, rc, _ = orc.run(scheme, u0, v0, lam, lam * h, steps, bc=BC_PERIODIC)
    for got, ref in ((uc, rc), (up, rp)):
        l2, linf = rel_errors(got, ref)
        assert l2 < TOL[2] and linf < TOL[2], (l2, linf)
