"""In-place streaming (one population buffer, two alternating kernels)
against the two-buffer scheme, bit for bit, and against the FP64 oracle.

The in-place scheme changes only where each stored value sits, never how it
is computed (the wall rules are applied on reading, the stochastic-rounding
bits are keyed by the producing cell and direction), so every call of the API
must return exactly what the two-buffer handle returns after the same steps.
"""

import numpy as np
import pytest

import oracle
from paper_1511_04633_gb300 import inputs

pytestmark = pytest.mark.gpu

STEP_TOL = 1e-6
FIELD_TOL = 1e-5
NU_RTOL = 1e-4


@pytest.fixture(scope="module")
def dm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1511_04633_gb300 import dmrt
    dmrt.load()
    return dmrt


def _twins(dm, grid, wall, **kw):
    ab = dm.Cavity(grid, wall_type=wall, streaming=dm.STREAM_AB, **kw)
    ip = dm.Cavity(grid, wall_type=wall, streaming=dm.STREAM_INPLACE, **kw)
    return ab, ip


def _assert_same(ab, ip, walls=True):
    fa, ga = ab.populations()
    fi, gi = ip.populations()
    assert np.array_equal(fa, fi) and np.array_equal(ga, gi)
    for x, y in zip(ab.fields(), ip.fields()):
        assert np.array_equal(x, y)
    if walls:
        for w in (0, 1):
            assert ab.nusselt(w) == ip.nusselt(w)
            assert ab.nusselt_flux(w) == ip.nusselt_flux(w)
            assert np.array_equal(ab.nusselt_local(w), ip.nusselt_local(w))


@pytest.mark.parametrize("storage", [0, 1, 2], ids=["f32", "bf16", "f16"])
@pytest.mark.parametrize("wall", [0, 1, 2, 3])
@pytest.mark.parametrize("grid", [(13, 10, 7), (2, 3, 2)])
def test_bitwise_equal_to_two_buffers_from_random_state(dm, storage, wall, grid):
    """Random populations, then 1, 2 and 5 more steps: the state (read back
    from either layout) and every derived quantity match bitwise."""
    ab, ip = _twins(dm, grid, wall, lattice=(0.03, 0.05, 2e-3), storage=storage)
    f = inputs.random_populations(grid, 19, seed=300 + wall)
    g = inputs.random_thermal_populations(grid, seed=400 + wall)
    for h in (ab, ip):
        h.set_populations(f, g)
    _assert_same(ab, ip, walls=wall != 0)
    for n in (1, 1, 3):
        ab.step(n)
        ip.step(n)
        _assert_same(ab, ip, walls=wall != 0)


@pytest.mark.parametrize("storage", [0, 1], ids=["f32", "bf16"])
@pytest.mark.parametrize("K", [6, 7])
def test_graph_replayed_intervals_and_residuals(dm, storage, K):
    """Whole residual intervals replay captured graphs; an odd K starts every
    other interval from the streamed layout."""
    grid = (20, 18, 16)
    ab, ip = _twins(dm, grid, 3, Ra=5e4, storage=storage, residual_interval=K)
    for h in (ab, ip):
        h.step(3)
        h.step(10 * K)
    _assert_same(ab, ip)
    assert ab.residual() == ip.residual()
    st = dm.dmrt_get_stats(ip.h)
    assert st["step_launches"] == 3 + 10 * K


def test_matches_the_oracle_from_rest(dm):
    """32^3, Type 1, Ra = 1e3 from rest for 501 steps (an odd count ends in
    the streamed layout)."""
    grid = (32, 32, 32)
    ip = dm.Cavity(grid, 1e3, wall_type=1, streaming=dm.STREAM_INPLACE)
    orc = oracle.Oracle.physical(grid, 1, 1e3)
    ip.step(501)
    orc.step(501)
    for a, b in zip(ip.fields(), orc.fields()):
        assert np.abs(a - b).max() <= FIELD_TOL
    for w in (0, 1):
        for a, b in zip(ip.nusselt(w), orc.nusselt(w)[0]):
            assert abs(a - b) <= NU_RTOL * abs(b)


@pytest.mark.parametrize("wall", [0, 2])
def test_one_step_parity_in_both_phases(dm, wall):
    grid = (16, 12, 10)
    ip = dm.Cavity(grid, wall_type=wall, lattice=(0.03, 0.05, 2e-3), streaming=dm.STREAM_INPLACE)
    orc = oracle.Oracle(grid, wall, 0.03, 0.05, 2e-3)
    f = inputs.random_populations(grid, 19, seed=11)
    g = inputs.random_thermal_populations(grid, seed=12)
    ip.set_populations(f, g)
    orc.set_populations(f.astype(np.float64), g.astype(np.float64))
    for _ in range(2):  # phase 0, then phase 1
        ip.step(1)
        orc.step(1)
        fi, gi = ip.populations()
        fo, go = orc.populations()
        assert np.abs(fi - fo).max() <= STEP_TOL
        assert np.abs(gi - go).max() <= STEP_TOL


def test_set_and_init_in_the_streamed_layout(dm):
    """Writing a new state after an odd step count returns the buffer to the
    swapped layout and carries the stochastic-rounding counter over."""
    grid = (12, 11, 10)
    ab, ip = _twins(dm, grid, 2, Ra=1e5, storage=1)
    for h in (ab, ip):
        h.step(5)
    rho, u, th = inputs.random_fields(grid, seed=5)
    for h in (ab, ip):
        h.init_fields(rho, u, th)
        h.step(3)
    _assert_same(ab, ip)
    f = inputs.random_populations(grid, 19, seed=6)
    g = inputs.random_thermal_populations(grid, seed=7)
    for h in (ab, ip):
        h.set_populations(f, g)
        h.step(4)
    _assert_same(ab, ip)


def test_anisotropic_diffusion_in_place(dm):
    grid = (14, 12, 10)
    ab, ip = _twins(dm, grid, 1, Ra=2e4)
    D = [[0.05, 0.01, 0.0], [0.01, 0.04, 0.005], [0.0, 0.005, 0.06]]
    for h in (ab, ip):
        h.set_diffusion(D)
        h.step(37)
    _assert_same(ab, ip)


def test_half_the_population_memory(dm):
    grid = (64, 64, 64)
    ab, ip = _twins(dm, grid, 2, Ra=1e5)
    pa, pi = ab.params, ip.params
    assert pa["streaming"] == dm.STREAM_AB and pi["streaming"] == dm.STREAM_INPLACE
    one_buffer = 64 ** 3 * 26 * 4 + 256
    assert pa["device_bytes"] - pi["device_bytes"] == one_buffer


def test_checkpoint_resume_in_place(dm):
    grid, K = (16, 14, 12), 20
    a = dm.Cavity(grid, 1e5, wall_type=2, storage=2, residual_interval=K, streaming=dm.STREAM_INPLACE)
    a.step(2 * K + 3)   # saved in the streamed layout
    blob = a.save()
    a.step(3 * K)
    b = dm.Cavity(grid, 1e5, wall_type=2, storage=2, residual_interval=K, streaming=dm.STREAM_INPLACE)
    b.load(blob)
    b.step(3 * K)
    _assert_same(a, b)
    assert a.residual() == b.residual()
    # a two-buffer handle refuses an in-place checkpoint
    c = dm.Cavity(grid, 1e5, wall_type=2, storage=2, residual_interval=K)
    with pytest.raises(dm.DmrtError) as ei:
        c.load(blob)
    assert ei.value.status == dm.ERR_ARG


def test_full_size_128cube_in_place_matches_two_buffers(dm):
    grid = (128, 128, 128)
    ab, ip = _twins(dm, grid, 2, Ra=1e5)
    for h in (ab, ip):
        h.step(101)
    fa, ga = ab.populations()
    fi, gi = ip.populations()
    assert np.array_equal(fa, fi) and np.array_equal(ga, gi)
    assert ab.nusselt(0) == ip.nusselt(0)


def test_full_size_256cube_in_place_matches_two_buffers(dm):
    """The 256^3 Type 3 Ra = 1e6 workload: in place and with two buffers,
    bitwise the same after an odd number of steps."""
    grid = (256, 256, 256)
    ab, ip = _twins(dm, grid, 3, Ra=1e6)
    for h in (ab, ip):
        h.step(21)
    for x, y in zip(ab.fields(), ip.fields()):
        assert np.array_equal(x, y)
    assert ab.nusselt(0) == ip.nusselt(0)
