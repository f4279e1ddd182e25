"""A slab's local solver made of the FP64 oracle (test infrastructure): the
CPU stand-in for a wave2d handle in the decomposition tests, so the slab
plan, the halo bookkeeping, the exchange protocol and the combined norms run
on CPU ranks without a GPU.  Boundary as the GPU handle of a slab: the
grid's condition, applied by the oracle to the slab's local rows."""
import math

import numpy as np


class OracleSolver:
    def __init__(self, oracle, scheme, nx, ny_local, lam, tau, bc, h, c=1.0):
        self.o = oracle
        self.scheme, self.nx, self.ny = scheme, nx, ny_local
        self.lam, self.tau, self.bc, self.h, self.c = lam, tau, bc, h, c
        self.prev = self.cur = None
        self.k = 0

    def first_step(self, u0, v0):
        self.prev = np.array(u0, dtype=np.float64)
        self.cur = self.o.first_step(self.scheme, u0, v0, self.lam, self.tau, bc=self.bc)
        self.k = 1

    def step_n(self, n):
        self.prev, self.cur = self.o.continue_run(self.scheme, self.prev, self.cur, self.lam, n, bc=self.bc)
        self.k += n

    def row_block_shape(self, n):
        return (n, self.nx), np.float64

    def get_rows(self, j0, n, prev, cur):
        prev.numpy()[...] = self.prev[j0:j0 + n]
        cur.numpy()[...] = self.cur[j0:j0 + n]

    def set_rows(self, j0, n, prev, cur):
        self.prev[j0:j0 + n] = prev.numpy()
        self.cur[j0:j0 + n] = cur.numpy()

    def error_sums(self, ex, j0, nrows, row_shift):
        """Plane wave ex = (k1, k2): u_e = cos(k1 x + k2 y - c |k| t) at the
        global rows j + row_shift, x = i h, y = j h."""
        k1, k2 = ex
        t = self.k * self.tau
        x = np.arange(self.nx) * self.h
        y = (np.arange(j0, j0 + nrows) + row_shift) * self.h
        ue = np.cos(k1 * x[None, :] + k2 * y[:, None] - self.c * math.hypot(k1, k2) * t)
        d = self.cur[j0:j0 + nrows] - ue
        return [float(np.sum(d * d)), float(np.sum(ue * ue)), float(np.max(np.abs(d))), float(np.max(np.abs(ue)))]

    def sync(self):
        pass
