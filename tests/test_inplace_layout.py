"""Host-side check of the in-place streaming scheme's index arithmetic (the
address rules of step_inplace.cu restated in Python): in both phases every
address lies inside the buffer, each cell writes exactly the slots it read,
and no slot belongs to two cells, so the update is race-free in place.  The
GPU tests (test_gpu_inplace.py) then show the kernels compute what the
two-buffer scheme computes."""

import itertools

import pytest

E19 = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1), (1, 1, 0),
       (-1, 1, 0), (1, -1, 0), (-1, -1, 0), (1, 0, 1), (-1, 0, 1), (1, 0, -1), (-1, 0, -1), (0, 1, 1),
       (0, -1, 1), (0, 1, -1), (0, -1, -1)]
E7 = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]
E = E19 + E7


def opp(q):
    lst, base = (E19, 0) if q < 19 else (E7, 19)
    return base + lst.index(tuple(-v for v in E[q]))


def slots(nx, ny, nz, periodic, phase):
    """Per cell: (slots read, slots written) as flat element indices."""
    cells = nx * ny * nz
    P = (cells + 63) // 64 * 64
    M = 2 ** 32

    def wrap(x, y, z):
        return ((z % nz) * ny + (y % ny)) * nx + (x % nx)

    out = {}
    for z, y, x in itertools.product(range(nz), range(ny), range(nx)):
        me = (z * ny + y) * nx + x
        reads, writes = [], []
        for q in range(26):
            ex, ey, ez = E[q]
            o = opp(q)
            off = ex + ey * nx + ez * nx * ny
            if phase == 1:
                reads.append(q * P + me)
                writes.append(o * P + me)
                continue
            if periodic:
                reads.append(o * P + wrap(x - ex, y - ey, z - ez))
                writes.append(q * P + wrap(x + ex, y + ey, z + ez))
                continue
            # the kernel's 32-bit offset tables: nb = opp P - off, bb = q P,
            # sn = q P + off, sb = opp P (all modulo 2^32)
            arrives_from_wall = not (0 <= x - ex < nx and 0 <= y - ey < ny and 0 <= z - ez < nz)
            leaves_box = not (0 <= x + ex < nx and 0 <= y + ey < ny and 0 <= z + ez < nz)
            reads.append((me + ((q * P) if arrives_from_wall else (o * P - off))) % M)
            writes.append((me + ((o * P) if leaves_box else (q * P + off))) % M)
        out[(x, y, z)] = (reads, writes, P, cells)
    return out


@pytest.mark.parametrize("grid", [(2, 3, 2), (2, 2, 2), (13, 10, 7), (16, 12, 10), (5, 9, 4)])
@pytest.mark.parametrize("periodic", [False, True])
@pytest.mark.parametrize("phase", [0, 1])
def test_in_place_slots_are_private_and_in_range(grid, periodic, phase):
    seen = set()
    for cell, (reads, writes, P, cells) in slots(*grid, periodic, phase).items():
        for a in reads + writes:
            assert 0 <= a < 26 * P and a % P < cells, (cell, a)
        assert sorted(reads) == sorted(writes), cell
        assert len(set(reads)) == 26, cell
        assert not (seen & set(reads)), cell
        seen |= set(reads)
    assert len(seen) == 26 * grid[0] * grid[1] * grid[2]


@pytest.mark.parametrize("grid", [(1, 1, 1), (1, 3, 2), (3, 1, 1)])
def test_degenerate_periodic_boxes(grid):
    for phase in (0, 1):
        seen = set()
        for cell, (reads, writes, P, cells) in slots(*grid, True, phase).items():
            assert sorted(reads) == sorted(writes)
            assert not (seen & set(reads))
            seen |= set(reads)
