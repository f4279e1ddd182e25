"""The level schedule of the register-streaming kernel (k5_stream), replayed
on the CPU with row labels instead of values.

The kernel keeps, for every level t < T, the last 2D + 1 rows in a register
ring whose slot for row y is (y - rho0) mod (2D + 1), and addresses the slots
statically inside groups of 2D + 1 unrolled steps (D = R, the stencil
radius).  At step `step` (input row rho = rho0 + step) it computes level t on
row rho - t D from the rows rho - t D - R .. rho - t D + R of level t - 1 and
row rho - t D of level t - 2 (level -1: the u^{k-1} row loaded for the step),
skips level t while step < t (D + R), and from step T (D + R) on stores
level T and level T - 1 of row rho - T D.  This test checks, for every scheme
radius, depth and strip height the tuning accepts, that

* each slot the kernel reads holds exactly the row the stencil needs at that
  moment (no slot overwritten too early, none read before it is written);
* every level-t row it computes depends only on rows computed from valid
  inputs (level 0: rows >= rho0 that were loaded), so the stored rows are
  the true levels k + T and k + T - 1;
* the stored rows are exactly the strip's output rows y0 .. y0 + L - 1.
"""
import pytest


def replay_strip(R, T, L, y0=0):
    D = R
    WIN = 2 * D + 1
    rho0 = y0 - R * T
    nsteps = L + T * (D + R)
    ring = [[None] * WIN for _ in range(T)]      # row label held by each slot of levels 0 .. T-1
    valid = [set() for _ in range(T + 1)]        # rows of each level computed from valid inputs
    stored = []
    for base in range(0, nsteps, WIN):
        for s in range(WIN):                      # the unrolled group: s is a compile-time slot
            step = base + s
            if step >= nsteps:
                break
            rho = rho0 + step
            assert (rho - rho0) % WIN == s
            ring[0][s] = rho
            valid[0].add(rho)                     # loaded input row
            pm = rho - D                          # u^{k-1} row loaded with this step
            top = None
            for t in range(1, T + 1):
                if step < t * (D + R):
                    continue
                r = rho - t * D
                cs = (s - t * D) % WIN
                window = [ring[t - 1][(cs + d) % WIN] for d in range(-R, R + 1)]
                assert window == [r + d for d in range(-R, R + 1)], (t, step, window)
                prev = pm if t == 1 else ring[t - 2][cs]
                assert prev == r
                ok = all(y in valid[t - 1] for y in window) and (t == 1 or r in valid[t - 2])
                if ok:
                    valid[t].add(r)
                if t < T:
                    ring[t][cs] = r
                else:
                    top = r
            if step < T * (D + R):
                continue
            ro = rho - T * D
            ps = (s - T * D) % WIN
            assert top == ro and ring[T - 1][ps] == ro
            assert ro in valid[T] and ro in valid[T - 1]
            stored.append(ro)
    assert stored == list(range(y0, y0 + L))


@pytest.mark.parametrize("R", [1, 2])
@pytest.mark.parametrize("T", [2, 3, 4, 6])
@pytest.mark.parametrize("L", [8, 9, 16, 17, 37, 48, 64])
def test_ring_schedule(R, T, L):
    replay_strip(R, T, L)
    replay_strip(R, T, L, y0=5 * L)


def test_first_valid_rows_are_the_halo_bound():
    """Level t is valid from row rho0 + t R: the R T rows of input above the
    strip (and below it, by symmetry of the window) are exactly enough."""
    for R in (1, 2):
        for T in (2, 3, 4, 6):
            D, rho0 = R, -R * T
            for t in range(1, T + 1):
                first_step = t * (D + R)
                assert rho0 + first_step - t * D == rho0 + t * R


def replay_strip_difference_form(R, T, L, y0=0):
    """The difference form's schedule: level t on row r = rho - t D takes
    d^{t-1} of row r from the d row level t - 1 computed D steps earlier
    (a second ring per level, slot (r - rho0) mod (2D + 1)), or for t = 1
    the d^k row loaded with the step (the prev plane's row rho - D); the
    stored rows are u^{k+T} and d^{k+T} of the strip's output rows."""
    D = R
    WIN = 2 * D + 1
    rho0 = y0 - R * T
    nsteps = L + T * (D + R)
    ring = [[None] * WIN for _ in range(T)]      # u rows of levels 0 .. T-1
    ringd = [[None] * WIN for _ in range(T)]     # d rows of levels 1 .. T-1 (index 0 unused)
    valid = [set() for _ in range(T + 1)]
    valid_d = [set() for _ in range(T + 1)]
    stored = []
    for base in range(0, nsteps, WIN):
        for s in range(WIN):
            step = base + s
            if step >= nsteps:
                break
            rho = rho0 + step
            ring[0][s] = rho
            valid[0].add(rho)
            pm = rho - D                          # d^k row loaded with this step
            valid_d[0].add(pm)
            top = dtop = None
            for t in range(1, T + 1):
                if step < t * (D + R):
                    continue
                r = rho - t * D
                cs = (s - t * D) % WIN
                window = [ring[t - 1][(cs + d) % WIN] for d in range(-R, R + 1)]
                assert window == [r + d for d in range(-R, R + 1)], (t, step, window)
                dprev = pm if t == 1 else ringd[t - 1][cs]
                assert dprev == r, (t, step, dprev, r)
                if all(y in valid[t - 1] for y in window) and r in valid_d[t - 1]:
                    valid[t].add(r)
                    valid_d[t].add(r)
                if t < T:
                    ring[t][cs] = r
                    ringd[t][cs] = r
                else:
                    top = dtop = r
            if step < T * (D + R):
                continue
            ro = rho - T * D
            assert top == ro and dtop == ro
            assert ro in valid[T] and ro in valid_d[T]
            stored.append(ro)
    assert stored == list(range(y0, y0 + L))


@pytest.mark.parametrize("R", [1, 2])
@pytest.mark.parametrize("T", [2, 3, 4])
@pytest.mark.parametrize("L", [8, 9, 16, 17, 37, 64])
def test_ring_schedule_difference_form(R, T, L):
    replay_strip_difference_form(R, T, L)
    replay_strip_difference_form(R, T, L, y0=3 * L)
