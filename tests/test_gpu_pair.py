"""The step kernel with two cells per thread (packed FP32x2 collision,
2-element loads and stores) against the one-cell kernel, bit for bit, and
against the FP64 oracle.

Both kernels compute every value with the same sequence of individually
rounded operations, and the paired kernel hands each cell the same
stochastic-rounding bits, so the stored state must be identical after any
number of steps, for every storage format and wall type.
"""

import numpy as np
import pytest

import oracle
from paper_1511_04633_gb300 import inputs

pytestmark = pytest.mark.gpu

STEP_TOL = 1e-6
LATTICE = (0.03, 0.05, 2e-3)


@pytest.fixture(scope="module")
def dm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1511_04633_gb300 import dmrt
    dmrt.load()
    return dmrt


def _pair_and_single(dm, grid, wall, pair_loads=0, **kw):
    two = dm.Cavity(grid, wall_type=wall, cells_per_thread=2, pair_loads=pair_loads, **kw)
    one = dm.Cavity(grid, wall_type=wall, cells_per_thread=1, **kw)
    assert two.params["cells_per_thread"] == 2
    assert one.params["cells_per_thread"] == 1
    if pair_loads:
        assert two.params["pair_loads"] == pair_loads
    return two, one


def _assert_same(a, b):
    fa, ga = a.populations()
    fb, gb = b.populations()
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)
    for x, y in zip(a.fields(), b.fields()):
        assert np.array_equal(x, y)
    for w in (0, 1):
        assert a.nusselt(w) == b.nusselt(w)


# grids: the smallest box, one pair per row with ragged y, rows of 65 pairs
# (five tiles of 16, the last with one pair), a 16-pair row with 8 rows a
# block, 19 pairs in one tile of 32, 48 pairs in three tiles of 16; rows of a
# multiple of 8 cells (32, 8, 136, 96) also run with the TMA-staged loads for
# 16-bit storage
GRIDS = [(2, 3, 2), (2, 9, 5), (130, 6, 4), (32, 17, 6), (38, 20, 13), (8, 3, 4), (136, 5, 7),
         (96, 7, 5)]


@pytest.mark.parametrize("loads", [1, 2], ids=["direct", "staged"])
@pytest.mark.parametrize("rounding", [0, 1], ids=["auto", "nearest"])
@pytest.mark.parametrize("storage", [0, 1, 2], ids=["f32", "bf16", "f16"])
@pytest.mark.parametrize("wall", [1, 2, 3])
@pytest.mark.parametrize("grid", GRIDS, ids=lambda g: "x".join(map(str, g)))
def test_bitwise_equal_to_one_cell_kernel(dm, grid, wall, storage, rounding, loads):
    if storage == 0 and rounding == 1:
        pytest.skip("FP32 storage has one rounding mode")
    if loads == 2 and (storage == 0 or grid[0] % 8):
        pytest.skip("staged loads need 16-bit storage and rows of a multiple of 8 cells")
    rnd = dm.ROUND_NEAREST if rounding == 1 else dm.ROUND_AUTO
    two, one = _pair_and_single(dm, grid, wall, pair_loads=loads, lattice=LATTICE, storage=storage,
                                rounding=rnd)
    f = inputs.random_populations(grid, 19, seed=500 + wall)
    g = inputs.random_thermal_populations(grid, seed=600 + wall)
    for h in (two, one):
        h.set_populations(f, g)
    for n in (1, 1, 5):
        two.step(n)
        one.step(n)
        _assert_same(two, one)


@pytest.mark.parametrize("storage", [0, 1, 2], ids=["f32", "bf16", "f16"])
@pytest.mark.parametrize("wall", [1, 2, 3])
@pytest.mark.parametrize("grid", [(2, 3, 2), (130, 6, 4), (32, 17, 6)],
                         ids=lambda g: "x".join(map(str, g)))
def test_inplace_bitwise_equal_to_one_cell_kernels(dm, grid, wall, storage):
    """In-place streaming, both phases (odd and even step counts): the paired
    kernels read and write the same slots with the same values."""
    two, one = _pair_and_single(dm, grid, wall, lattice=LATTICE, storage=storage,
                                streaming=dm.STREAM_INPLACE)
    f = inputs.random_populations(grid, 19, seed=700 + wall)
    g = inputs.random_thermal_populations(grid, seed=800 + wall)
    for h in (two, one):
        h.set_populations(f, g)
    for n in (1, 1, 3):
        two.step(n)
        one.step(n)
        _assert_same(two, one)


@pytest.mark.parametrize("loads", [1, 2], ids=["direct", "staged"])
@pytest.mark.parametrize("storage", [0, 1, 2], ids=["f32", "bf16", "f16"])
def test_graph_replayed_intervals_from_rest(dm, storage, loads):
    """Whole residual intervals replay captured graphs of the paired kernel;
    a developing Type 2 flow from rest stays bitwise with the one-cell run."""
    if loads == 2 and storage == 0:
        pytest.skip("staged loads need 16-bit storage")
    grid = (48, 40, 36)
    two, one = _pair_and_single(dm, grid, 2, pair_loads=loads, Ra=1e5, storage=storage,
                                residual_interval=50)
    for h in (two, one):
        h.step(7)
        h.step(400)
    _assert_same(two, one)
    # the same fields, summed over different block shapes: the residuals'
    # double-float sums may differ in their last bits only
    assert two.residual() == pytest.approx(one.residual(), rel=1e-11)
    assert dm.dmrt_get_stats(two.h)["step_launches"] == 407


@pytest.mark.parametrize("wall", [1, 2, 3])
@pytest.mark.parametrize("grid", [(16, 12, 10), (2, 5, 3), (66, 7, 4)],
                         ids=lambda g: "x".join(map(str, g)))
def test_one_step_parity_with_the_oracle(dm, grid, wall):
    """One paired FP32 step from random populations against the FP64 oracle."""
    cav = dm.Cavity(grid, wall_type=wall, lattice=LATTICE, cells_per_thread=2)
    orc = oracle.Oracle(grid, wall, *LATTICE)
    f = inputs.random_populations(grid, 19, seed=21 + wall)
    g = inputs.random_thermal_populations(grid, seed=31 + wall)
    cav.set_populations(f, g)
    orc.set_populations(f.astype(np.float64), g.astype(np.float64))
    cav.step(1)
    orc.step(1)
    fc, gc = cav.populations()
    fo, go = orc.populations()
    assert np.abs(fc - fo).max() <= STEP_TOL
    assert np.abs(gc - go).max() <= STEP_TOL


def test_auto_choice_and_rejected_requests(dm):
    """Auto takes two cells on even rows of walled boxes, one otherwise; two
    cells on an odd row or a periodic box are refused."""
    assert dm.Cavity((16, 8, 8), 1e4, storage=dm.STORE_BF16).params["cells_per_thread"] == 2
    assert dm.Cavity((15, 8, 8), 1e4, storage=dm.STORE_BF16).params["cells_per_thread"] == 1
    assert dm.Cavity((16, 8, 8), 1e4).params["cells_per_thread"] == 2
    assert dm.Cavity((16, 8, 8), 1e4, wall_type=0).params["cells_per_thread"] == 1
    assert dm.Cavity((16, 8, 8), 1e4, storage=dm.STORE_F16,
                     streaming=dm.STREAM_INPLACE).params["cells_per_thread"] == 2
    assert dm.Cavity((16, 8, 8), 1e4, storage=dm.STORE_F16, wall_type=0,
                     streaming=dm.STREAM_INPLACE).params["cells_per_thread"] == 1
    bad = [dict(grid=(15, 8, 8)), dict(grid=(16, 8, 8), wall_type=0),
           dict(grid=(15, 8, 8), streaming=dm.STREAM_INPLACE)]
    for kw in bad:
        grid = kw.pop("grid")
        with pytest.raises(dm.DmrtError) as ei:
            dm.Cavity(grid, lattice=LATTICE, cells_per_thread=2, **kw)
        assert ei.value.status == dm.ERR_ARG
    with pytest.raises(dm.DmrtError):
        dm.Cavity((16, 8, 8), lattice=LATTICE, cells_per_thread=3)
    # staged loads: on request, for 16-bit two-buffer storage with rows of a
    # multiple of 8 cells; auto takes the direct loads
    assert dm.Cavity((16, 8, 8), 1e4, storage=dm.STORE_BF16).params["pair_loads"] == 1
    assert dm.Cavity((16, 8, 8), 1e4, storage=dm.STORE_BF16, pair_loads=2).params["pair_loads"] == 2
    assert dm.Cavity((18, 8, 8), 1e4, storage=dm.STORE_BF16).params["pair_loads"] == 1
    assert dm.Cavity((16, 8, 8), 1e4, storage=dm.STORE_BF16,
                     streaming=dm.STREAM_INPLACE).params["pair_loads"] == 0
    assert dm.Cavity((16, 8, 8), 1e4).params["pair_loads"] == 1
    for kw in (dict(grid=(18, 8, 8), storage=dm.STORE_BF16), dict(grid=(16, 8, 8)),
               dict(grid=(16, 8, 8), storage=dm.STORE_BF16, streaming=dm.STREAM_INPLACE)):
        grid = kw.pop("grid")
        with pytest.raises(dm.DmrtError) as ei:
            dm.Cavity(grid, lattice=LATTICE, cells_per_thread=2, pair_loads=2, **kw)
        assert ei.value.status == dm.ERR_ARG
    with pytest.raises(dm.DmrtError):
        dm.dmrt_create((16, 8, 8), 1e4, cells_per_thread=-1)


@pytest.mark.parametrize("storage", [1, 2], ids=["bf16", "f16"])
def test_inplace_graph_intervals_match_two_buffers(dm, storage):
    """Paired in-place and paired two-buffer runs of 7 + 4 x 75 steps from
    rest (odd intervals alternate the layout) hold the same state."""
    grid = (40, 24, 20)
    ab = dm.Cavity(grid, 3e4, wall_type=3, storage=storage, residual_interval=75)
    ip = dm.Cavity(grid, 3e4, wall_type=3, storage=storage, residual_interval=75,
                   streaming=dm.STREAM_INPLACE)
    assert ab.params["cells_per_thread"] == ip.params["cells_per_thread"] == 2
    for h in (ab, ip):
        h.step(7)
        h.step(300)
    _assert_same(ab, ip)
    assert ab.residual() == ip.residual()


@pytest.mark.parametrize("storage", [1, 2], ids=["bf16", "f16"])
@pytest.mark.parametrize("wall", [1, 2, 3])
def test_staged_loads_over_several_slabs(dm, storage, wall):
    """A 256 x 192 x 24 box gives every staged block four slabs in a row (the
    three-stage ring wraps); direct and staged loads and one cell per thread
    agree bitwise after 1, 2 and 5 steps from random populations."""
    grid = (256, 192, 24)
    kw = dict(wall_type=wall, lattice=LATTICE, storage=storage)
    staged = dm.Cavity(grid, cells_per_thread=2, pair_loads=2, **kw)
    direct = dm.Cavity(grid, cells_per_thread=2, pair_loads=1, **kw)
    one = dm.Cavity(grid, cells_per_thread=1, **kw)
    assert staged.params["pair_loads"] == 2 and direct.params["pair_loads"] == 1
    f = inputs.random_populations(grid, 19, seed=900 + wall)
    g = inputs.random_thermal_populations(grid, seed=910 + wall)
    for h in (staged, direct, one):
        h.set_populations(f, g)
    for n in (1, 1, 3):
        for h in (staged, direct, one):
            h.step(n)
        _assert_same(staged, direct)
        _assert_same(staged, one)
    staged.sync()


@pytest.mark.parametrize("loads", [1, 2], ids=["direct", "staged"])
def test_full_size_step_of_the_256_cube_bf16(dm, loads):
    """The 256^3 Type 3 Ra = 1e6 BF16 cavity of the benchmark: 30 steps from
    rest, paired and one-cell kernels bitwise equal on every plane."""
    grid = (256, 256, 256)
    two, one = _pair_and_single(dm, grid, 3, pair_loads=loads, Ra=1e6, storage=dm.STORE_BF16)
    for h in (two, one):
        h.step(30)
    fa, ga = two.populations()
    fb, gb = one.populations()
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)
