"""Seeded synthetic inputs shared by the oracle tests and the CUDA path.

This module produces initial data (u0, v0) on grid nodes and the workload
recipes (instance lists, request streams).  It holds none of the method's
arithmetic: no stencil, no coefficient, no time stepping.  Both sides of every
parity test take their inputs from here and from nowhere else.

Grid geometry (Section 6.1.2 and Section 6.3 of the paper):
* ``BC_ZERO``: nx updated nodes per row at x = (i + 1) h, i = 0..nx-1; the
  boundary nodes x = 0 and x = (nx + 1) h hold u = 0.  With h = 1/n and
  nx = n - 1 this is the paper's node set {0 < i < n} on the unit square.
* ``BC_PERIODIC``: nx nodes at x = i h with h = 1/nx, wrapping.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

BC_ZERO = 0
BC_PERIODIC = 1
BC_ODD = 2  # the zero-boundary node set with odd continuation beyond the boundary nodes


def x_offset(bc: int) -> float:
    """Offset (in units of h) of node 0 from the origin."""
    return 0.0 if bc == BC_PERIODIC else 1.0


def coords(n: int, h: float, bc: int) -> np.ndarray:
    return (np.arange(n, dtype=np.float64) + x_offset(bc)) * h


def mesh(nx: int, ny: int, h: float, bc: int):
    """(X1, X2) arrays of shape (ny, nx): X1[j, i] = x1 of node (i, j)."""
    x1 = coords(nx, h, bc)
    x2 = coords(ny, h, bc)
    return np.meshgrid(x1, x2, indexing="xy")


# --------------------------------------------------------------------------
# Exact-solution initial data
# --------------------------------------------------------------------------

def standing_wave_ic(nx, ny, h, bc=BC_ZERO, c=1.0, m=1.0, amp=1.0):
    """Initial data of the standing wave amp*sin(2 pi m x1) sin(2 pi m x2) sin(2 sqrt2 pi m c t)
    (Eq. "exact sol" and Eq. "Exact IC" for m = amp = 1): u0 = 0,
    v0 = amp * 2 sqrt2 pi m c sin(2 pi m x1) sin(2 pi m x2)."""
    X1, X2 = mesh(nx, ny, h, bc)
    u0 = np.zeros((ny, nx))
    v0 = amp * 2.0 * math.sqrt(2.0) * math.pi * m * c * np.sin(2 * math.pi * m * X1) * np.sin(2 * math.pi * m * X2)
    return u0, v0


def plane_wave_ic(nx, ny, h, k1, k2, bc=BC_PERIODIC, c=1.0, amp=1.0):
    """Initial data of the plane wave amp*cos(k.x - c|k| t): u0 = amp cos(k.x),
    v0 = amp c|k| sin(k.x)."""
    X1, X2 = mesh(nx, ny, h, bc)
    ph = k1 * X1 + k2 * X2
    w = c * math.hypot(k1, k2)
    return amp * np.cos(ph), amp * w * np.sin(ph)


def plane_wave_k(n: int, m1: int, m2: int):
    """Wave vector 2 pi (m1, m2) of a mode periodic on the unit square."""
    return 2 * math.pi * m1, 2 * math.pi * m2


# --------------------------------------------------------------------------
# Gaussian pulses and band-limited noise
# --------------------------------------------------------------------------

def gaussian_pulse(nx, ny, h, bc=BC_ZERO, center=None, sigma=0.05, amp=1.0):
    """amp * exp(-|x - x0|^2 / (2 sigma^2)); x0 defaults to the centre of the
    node set so that the pulse is exactly D4-symmetric on the grid."""
    X1, X2 = mesh(nx, ny, h, bc)
    if center is None:
        off = x_offset(bc)
        center = ((nx - 1) / 2.0 + off) * h, ((ny - 1) / 2.0 + off) * h
    d2 = (X1 - center[0]) ** 2 + (X2 - center[1]) ** 2
    return amp * np.exp(-d2 / (2.0 * sigma * sigma))


def pulses_and_noise(n: int, seed: int = 2019, n_pulses: int = 16, bc: int = BC_PERIODIC,
                     nyquist_fraction: float = 1.0 / 8.0):
    """Multi-pulse displacement and band-limited random velocity on an n x n
    grid with h = 1/n.

    u0 = sum_p a_p exp(-|x - x_p|^2 / (2 sigma_p^2)) with x_p ~ U[0,1)^2,
    sigma_p ~ U(0.01, 0.05), a_p ~ U(-1, 1); distances are taken to the nearest
    periodic image so that u0 is smooth across the wrap.
    v0 = Re IFFT of complex normal noise kept only for integer wave numbers
    |k| < nyquist_fraction * (n/2), scaled so that max |v0| = 1.
    """
    rng = np.random.default_rng(seed)
    h = 1.0 / n
    centers = rng.uniform(0.0, 1.0, size=(n_pulses, 2))
    sigmas = rng.uniform(0.01, 0.05, size=n_pulses)
    amps = rng.uniform(-1.0, 1.0, size=n_pulses)
    x = coords(n, h, bc)
    u0 = np.zeros((n, n))
    for (cx, cy), s, a in zip(centers, sigmas, amps):
        dx = x - cx
        dy = x - cy
        if bc == BC_PERIODIC:
            dx = dx - np.round(dx)
            dy = dy - np.round(dy)
        gx = np.exp(-dx * dx / (2 * s * s))
        gy = np.exp(-dy * dy / (2 * s * s))
        u0 += a * np.outer(gy, gx)
    kidx = np.fft.fftfreq(n, d=1.0 / n)
    K1, K2 = np.meshgrid(kidx, kidx, indexing="xy")
    mask = np.hypot(K1, K2) < nyquist_fraction * (n / 2.0)
    noise = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    v0 = np.ascontiguousarray(np.real(np.fft.ifft2(noise * mask)))
    v0 /= np.max(np.abs(v0))
    return u0, v0


# --------------------------------------------------------------------------
# Workload recipes
# --------------------------------------------------------------------------

# Stability limits of the three schemes (Eq. stability5, stability9 read as
# sqrt((3 - sqrt3)/2), and Section 6.3): needed to draw Courant numbers.
LAMBDA_MAX = {5: 1.0 / math.sqrt(2.0), 9: math.sqrt((3.0 - math.sqrt(3.0)) / 2.0),
              13: 1.0 / math.sqrt(2.0)}


@dataclass
class Instance:
    n: int
    scheme: int
    lam: float
    steps: int
    sigma: float = 0.05


def batch_instances(count: int = 512, seed: int = 4, n_min: int = 64, n_max: int = 1024,
                    steps_min: int = 100, steps_max: int = 2000):
    """Independent simulations for a batched run: n log-uniform in
    [n_min, n_max], scheme uniform in {5, 9, 13}, Courant number uniform in
    (0.3, 0.9 lambda_max), step count uniform in {steps_min..steps_max}."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        scheme = int(rng.choice([5, 9, 13]))
        lam = float(rng.uniform(0.3, 0.9 * LAMBDA_MAX[scheme]))
        steps = int(rng.integers(steps_min, steps_max + 1))
        out.append(Instance(n=n, scheme=scheme, lam=lam, steps=steps))
    return out


@dataclass
class Request:
    arrival_s: float
    inst: Instance


def request_stream(count: int = 2000, rate_hz: float = 200.0, seed: int = 5, n_min: int = 128,
                   n_max: int = 2048, steps_min: int = 100, steps_max: int = 5000):
    """Poisson arrivals (exponential gaps of mean 1/rate) of simulations with
    n log-uniform in [n_min, n_max], mixed schemes, Courant number uniform in
    (0.3, 0.9 lambda_max) and uniform step counts."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for _ in range(count):
        t += float(rng.exponential(1.0 / rate_hz))
        n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        scheme = int(rng.choice([5, 9, 13]))
        lam = float(rng.uniform(0.3, 0.9 * LAMBDA_MAX[scheme]))
        steps = int(rng.integers(steps_min, steps_max + 1))
        out.append(Request(arrival_s=t, inst=Instance(n=n, scheme=scheme, lam=lam, steps=steps)))
    return out


def instance_ic(inst: Instance):
    """Centred Gaussian pulse (v0 = 0) for a batched / served instance with
    zero boundary, h = 1/(n + 1)."""
    h = 1.0 / (inst.n + 1)
    u0 = gaussian_pulse(inst.n, inst.n, h, BC_ZERO, sigma=inst.sigma)
    return u0, np.zeros_like(u0), h
