"""Shared helpers of the GPU tests (inputs and tolerance checks)."""
import numpy as np

from initial_data import BC_PERIODIC, BC_ZERO, gaussian_pulse, x_offset

# Parity tolerances on relative L2 and relative L-infinity against the FP64
# oracle, per storage type, for runs of up to 1000 steps (FP32x2: 10^4).
# FP64: rounding differences only (FMA contraction, summation order).
# FP32: storage rounding of u^k each step dominates (about 3e-6 measured at
#       512^2 after 1000 steps for the 13-point scheme).
# FP32x2: double-float storage and arithmetic (about 2^-47 per operation).
TOL = {0: 1e-12, 1: 1e-5, 2: 1e-10}


def smooth_ic(nx, ny, bc, seed=0):
    """Sum of three Gaussians for u0 and two for v0 with seeded centres."""
    rng = np.random.default_rng(seed)
    h = 1.0 / max(nx, ny)
    off = x_offset(bc)
    lo = np.array([off * h, off * h])
    span = np.array([nx * h, ny * h])
    u0 = np.zeros((ny, nx))
    v0 = np.zeros((ny, nx))
    for k in range(3):
        c = lo + rng.uniform(0.2, 0.8, 2) * span
        u0 += rng.uniform(-1, 1) * gaussian_pulse(nx, ny, h, bc, center=tuple(c), sigma=0.08 * span.max())
    for k in range(2):
        c = lo + rng.uniform(0.2, 0.8, 2) * span
        v0 += rng.uniform(-3, 3) * gaussian_pulse(nx, ny, h, bc, center=tuple(c), sigma=0.1 * span.max())
    return u0, v0, h


def rel_errors(got, ref):
    d = got - ref
    return float(np.linalg.norm(d) / np.linalg.norm(ref)), float(np.max(np.abs(d)) / np.max(np.abs(ref)))
