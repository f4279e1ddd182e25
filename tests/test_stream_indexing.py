"""Index arithmetic of the register-streaming kernel (k5_stream), replayed on
the CPU: for ragged and degenerate grids, every strip height the tuning
accepts near the edges and every scheme and depth, each global load stays in
the level plane (ghost ring and row padding included) at a 16-byte aligned
address (on periodic grids read at wrapped coordinates: inside the grid, at
the node the periodic image holds), the cp.async ring slots stay in the CTA's
shared memory, and the stored vectors cover every grid node exactly once.

The model restates the kernel's constants and formulas (kernels_stream.cuh):
strips of 32 C columns (C = 4 nodes per lane) with HX = R T rounded up to a
vector of halo columns on each side, L output rows, input rows
rho0 = y0 - R T .. rho0 + L + 2 R T - 1 plus the PF rows copied ahead,
u^{k-1} rows one stencil radius behind, rows clamped to the last stored row,
columns to the last 4-node vector of the stored row."""
import itertools

import pytest

G = 16            # ghost ring width (kGhost)
C = 4             # nodes per lane
WARPS = 4         # warps per CTA
DEPTHS = [2, 3, 4, 6]   # levels per launch the tuning accepts


def ring_slots(scheme):
    """Ring slots per warp and rows copied ahead (StreamCfg::NB, ::PF)."""
    nb = 8 if scheme == 13 else 4
    return nb, nb - 2


def plane_geometry(nx, ny):
    pitch = -(-(nx + 2 * G) // 32) * 32
    return pitch, ny + 2 * G


def stream_row(y, ny, ymax, wrap):
    if not wrap:
        return min(y, ymax)
    r = y + ny if y < 0 else y
    return min(r - ny, ny - 1) if r >= ny else r


def replay(nx, ny, scheme, T, L, periodic=False):
    R = 2 if scheme == 13 else 1
    NB, PF = ring_slots(scheme)
    HX = (R * T + 3) // 4 * 4
    W = 32 * C
    OW = W - 2 * HX
    pitch, rows = plane_geometry(nx, ny)
    n_el = pitch * rows
    strips_x, strips_y = -(-nx // OW), -(-ny // L)
    ymax = ny + G - 1

    def off(i, j):
        return (j + G) * pitch + (i + G)

    wrap = periodic and nx % 4 == 0 and ny >= 16   # the launcher's condition
    covered = {}
    for strip in range(strips_x * strips_y):
        warp = strip % WARPS
        x0, y0 = (strip % strips_x) * OW, (strip // strips_x) * L
        rho0, nsteps = y0 - R * T, L + 2 * R * T
        for lane in range(32):
            xl = x0 - HX + C * lane
            xload = min(xl, pitch - G - C)
            if wrap:
                xload = xl % nx
                assert xload + C <= nx                  # the wrapped vector stays whole
            assert xl >= -G
            for step in range(nsteps + PF):            # copies issued up to PF steps ahead
                rho = rho0 + step
                for y in (rho, rho - R):                # u^k row and u^{k-1} row
                    yr = stream_row(y, ny, ymax, wrap)
                    o = off(xload, yr)
                    assert 0 <= o and o + C <= n_el and o % 4 == 0
                    if wrap:                            # the node the periodic image holds
                        assert 0 <= yr < ny and (xload - xl) % nx == 0
                        assert (yr - y) % ny == 0 or y >= 2 * ny   # rows past 2 ny feed no stored node
                slot = step % NB
                smem = ((warp * NB + slot) * 2 + 1) * 32 + lane   # plane 1 is the larger index
                assert smem < WARPS * NB * 2 * 32
            if not (HX <= C * lane < HX + OW and xl < nx):
                continue
            for step in range(2 * R * T, nsteps):
                ro = rho0 + step - T * R
                assert y0 <= ro < y0 + L
                if ro >= ny:
                    continue
                for e in range(4):
                    if xl + e < nx:
                        o = off(xl + e, ro)
                        assert 0 <= o < n_el
                        covered[(xl + e, ro)] = covered.get((xl + e, ro), 0) + 1
    assert len(covered) == nx * ny and set(covered.values()) == {1}


SHAPES = [(1, 1), (5, 3), (13, 31), (64, 64), (121, 1), (1, 200), (120, 17), (300, 97), (1000, 333)]


@pytest.mark.parametrize("scheme", [5, 9, 13])
@pytest.mark.parametrize("T", DEPTHS)
@pytest.mark.parametrize("L", [8, 16, 37, 64])
@pytest.mark.parametrize("periodic", [False, True], ids=["clamped", "periodic"])
def test_loads_in_bounds_and_stores_cover_each_node_once(scheme, T, L, periodic):
    for nx, ny in SHAPES + [(4, 16), (16, 17), (64, 20)]:
        replay(nx, ny, scheme, T, L, periodic)


def test_halo_reaches_every_dependency():
    """A node stored at level T depends on level-0 nodes up to R T rows and
    columns away; the strip's halo columns and warm-up rows must hold all of
    them (else a stored node would read a halo lane's unfinished value)."""
    for scheme, T in itertools.product((5, 9, 13), DEPTHS):
        R = 2 if scheme == 13 else 1
        HX = (R * T + 3) // 4 * 4
        assert HX >= R * T and HX <= G and R * (T + 1) < G
        NB, PF = ring_slots(scheme)
        assert PF + 2 <= NB   # a slot is refilled two steps after its last read


def wrap(i, n):
    return i % n


def ring_cells(nx, ny, gw):
    """The (cell, source) pairs k5_ring_images writes for one plane, with the
    launch's grid (x blocks over a band row, y = 2 gw band rows plus the
    side-band blocks) and its loops replayed thread by thread."""
    gx = min((nx + 2 * gw + 255) // 256, 16)
    side = max(1, min((ny * 2 * gw + 255) // 256 // gx, 64))
    out = []
    for by in range(2 * gw + side):
        for bx in range(gx):
            for t in range(256):
                if by < 2 * gw:
                    j = by - gw if by < gw else ny + (by - gw)
                    i = bx * 256 + t - gw
                    while i < nx + gw:
                        out.append(((i, j), (wrap(i, nx), wrap(j, ny))))
                        i += gx * 256
                else:
                    rpb = max(1, 256 // (2 * gw))
                    base = (by - 2 * gw) * gx + bx
                    while base * rpb < ny:
                        j, c = base * rpb + t // (2 * gw), t % (2 * gw)
                        if j < ny and t < rpb * 2 * gw:
                            i = c - gw if c < gw else nx + (c - gw)
                            out.append(((i, j), (wrap(i, nx), j)))
                        base += side * gx
    return out


@pytest.mark.parametrize("nx,ny", [(1, 1), (5, 3), (13, 31), (120, 17), (300, 97), (700, 2)])
def test_ring_images_cover_the_ring_once(nx, ny):
    gw = G
    cells = ring_cells(nx, ny, gw)
    targets = [c for c, _ in cells]
    ring = {(i, j) for i in range(-gw, nx + gw) for j in range(-gw, ny + gw)
            if not (0 <= i < nx and 0 <= j < ny)}
    assert len(targets) == len(set(targets)) and set(targets) == ring
    for (i, j), (si, sj) in cells:
        assert 0 <= si < nx and 0 <= sj < ny and (si - i) % nx == 0 and (sj - j) % ny == 0
