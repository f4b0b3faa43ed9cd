"""Ensembles: many cavities advanced by a few launches per time step.  Each member
must evolve exactly like a single cavity handle (same per-cell arithmetic)
and so match the FP64 oracle like one."""

import numpy as np
import pytest

import oracle
from paper_1511_04633_gb300 import inputs

pytestmark = pytest.mark.gpu

FIELD_TOL = 1e-5
NU_RTOL = 1e-4

MEMBERS = [
    {"grid": (16, 16, 16), "Ra": 1e4, "wall": 1},
    {"grid": (20, 18, 16), "Ra": 5e4, "wall": 3},
    {"grid": (24, 24, 24), "Ra": 1e5, "wall": 2},
    {"grid": (37, 20, 13), "Ra": 3e4, "wall": 2},
    {"grid": (12, 12, 12), "Ra": 1e3, "wall": 1},
]


@pytest.fixture(scope="module")
def dm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1511_04633_gb300 import dmrt
    dmrt.load()
    return dmrt


@pytest.mark.parametrize("storage", [0, 1], ids=["f32", "bf16"])
def test_members_evolve_bitwise_like_single_cavities(dm, storage):
    ens = dm.Ensemble(MEMBERS, storage=storage)
    ens.step(250)
    for k, m in enumerate(MEMBERS):
        single = dm.Cavity(m["grid"], m["Ra"], wall_type=m["wall"], storage=storage)
        single.step(250)
        fe, ge = ens.populations(k)
        fs, gs = single.populations()
        assert np.array_equal(fe, fs) and np.array_equal(ge, gs), k


def test_members_match_the_oracle(dm):
    ens = dm.Ensemble(MEMBERS[:3])
    ens.step(300)
    nus = ens.nusselt(0)
    for k, m in enumerate(MEMBERS[:3]):
        o = oracle.Oracle.physical(m["grid"], m["wall"], m["Ra"])
        o.step(300)
        rg, ug, tg = ens.fields(k)
        ro, uo, to = o.fields()
        err = max(np.abs(rg - ro).max(), np.abs(ug - uo).max(), np.abs(tg - to).max())
        assert err <= FIELD_TOL, (k, err)
        no, _ = o.nusselt(0)
        for a, b in zip(nus[k], no):
            assert abs(a - b) <= NU_RTOL * abs(b), (k, nus[k], no)


def test_member_residuals_equal_single_residuals(dm):
    """The same per-cell terms (members evolve bitwise like single handles),
    summed over other blocks: equal up to the last bits of the double-float
    sums."""
    K = 50
    ens = dm.Ensemble(MEMBERS, residual_interval=K)
    ens.step(3 * K)
    r = ens.residual()
    for k, m in enumerate(MEMBERS):
        single = dm.Cavity(m["grid"], m["Ra"], wall_type=m["wall"], residual_interval=K)
        single.step(3 * K)
        assert r[k] == pytest.approx(single.residual(), rel=1e-11)


def test_autotune_keeps_the_state_and_reports(dm):
    ens = dm.Ensemble(MEMBERS)
    ens.step(40)
    before = [ens.populations(k) for k in range(len(MEMBERS))]
    report = ens.autotune(trials=2)
    assert "chosen threads=" in report
    for k in range(len(MEMBERS)):
        f, g = ens.populations(k)
        assert np.array_equal(f, before[k][0]) and np.array_equal(g, before[k][1])
    # still steps correctly with the tuned layout
    ens.step(60)
    single = dm.Cavity(MEMBERS[3]["grid"], MEMBERS[3]["Ra"], wall_type=MEMBERS[3]["wall"])
    single.step(100)
    assert np.array_equal(ens.populations(3)[0], single.populations()[0])


def test_small_ensemble_runs_to_steady(dm):
    members = [{"grid": (10, 10, 10), "Ra": ra, "wall": w}
               for ra, w in ((1e3, 1), (2e3, 2), (5e3, 3), (1e3, 2))]
    ens = dm.Ensemble(members)
    ok, steps, conv = ens.run_to_steady(1e-7, 200_000)
    assert ok and conv == len(members)
    nus = ens.nusselt(0)
    nuc = ens.nusselt(1)
    np.testing.assert_allclose(nus[:, 0], nuc[:, 0], rtol=1e-5)


def test_config4_ensemble_draws_build_and_step(dm):
    draws = inputs.ensemble_draws(64, seed=1234)
    cav = [{"grid": (d["n"],) * 3, "Ra": d["Ra"], "wall": d["wall"]} for d in draws]
    ens = dm.Ensemble(cav)
    ens.step(20)
    r = ens.residual()
    assert np.all(np.isinf(r))  # fewer than two residual points yet
    taus = [ens.params(k)["tau_nu"] for k in range(len(cav))]
    assert min(taus) > 0.5


@pytest.mark.parametrize("streaming", [0, 1], ids=["ab", "inplace"])
def test_config4_full_ensemble_step_matches_the_oracle(dm, streaming):
    """The 64-member ensemble in the benchmark's launch configuration
    (autotuned): after 150 steps from rest, one more step of sampled members
    (the largest, a Type 3 and the highest Ra) must match the oracle's step
    from the same state."""
    draws = inputs.ensemble_draws(64, seed=1234)
    cav = [{"grid": (d["n"],) * 3, "Ra": d["Ra"], "wall": d["wall"]} for d in draws]
    ens = dm.Ensemble(cav, streaming=streaming)
    ens.autotune(trials=2)
    ens.step(150)
    picks = {max(range(64), key=lambda k: cav[k]["grid"][0]),
             next(k for k in range(64) if cav[k]["wall"] == 3),
             max(range(64), key=lambda k: cav[k]["Ra"])}
    orcs = {}
    for k in picks:
        f, g = ens.populations(k)
        o = oracle.Oracle.physical(cav[k]["grid"], cav[k]["wall"], cav[k]["Ra"])
        o.set_populations(f.astype(np.float64), g.astype(np.float64))
        o.step(1)
        orcs[k] = o
    ens.step(1)
    for k, o in orcs.items():
        fe, ge = ens.populations(k)
        fo, go = o.populations()
        assert np.abs(fe - fo).max() <= 1e-6, k
        assert np.abs(ge - go).max() <= 1e-6, k


def test_ensemble_rejects_periodic_members_and_bad_indices(dm):
    with pytest.raises(dm.DmrtError) as ei:
        dm.Ensemble([{"grid": (8, 8, 8), "Ra": 1e4, "wall": 0}])
    assert ei.value.status == dm.ERR_ARG
    ens = dm.Ensemble(MEMBERS[:1])
    rho = np.empty((16, 16, 16), np.float32)
    with pytest.raises(dm.DmrtError) as ei:
        dm.dmrt_ensemble_fields(ens.e, 1, rho=rho)
    assert ei.value.status == dm.ERR_ARG


# ------------------------------------------------------------------ in-place ensembles

def _same_members(a, b, count, walls=True):
    for k in range(count):
        fa, ga = a.populations(k)
        fb, gb = b.populations(k)
        assert np.array_equal(fa, fb) and np.array_equal(ga, gb), k
        for x, y in zip(a.fields(k), b.fields(k)):
            assert np.array_equal(x, y), k
    if walls:
        assert np.array_equal(np.asarray(a.nusselt(0)), np.asarray(b.nusselt(0)))
        assert np.array_equal(np.asarray(a.nusselt(1)), np.asarray(b.nusselt(1)))


@pytest.mark.parametrize("storage", [0, 1, 2], ids=["f32", "bf16", "f16"])
@pytest.mark.parametrize("K", [6, 7])
def test_in_place_ensemble_is_bitwise_the_two_buffer_ensemble(dm, storage, K):
    """Odd and even step counts, graph-replayed intervals of odd and even K,
    residuals: the in-place ensemble returns exactly what the two-buffer one
    does."""
    ab = dm.Ensemble(MEMBERS, storage=storage, residual_interval=K)
    ip = dm.Ensemble(MEMBERS, storage=storage, residual_interval=K, streaming=dm.STREAM_INPLACE)
    for n in (1, 2, 3 * K, 5 * K + 1):
        ab.step(n)
        ip.step(n)
        _same_members(ab, ip, len(MEMBERS))
    assert np.array_equal(np.asarray(ab.residual()), np.asarray(ip.residual()))


def test_in_place_ensemble_members_match_single_in_place_cavities(dm):
    ip = dm.Ensemble(MEMBERS[:3], storage=1, streaming=dm.STREAM_INPLACE)
    ip.step(77)
    for k, m in enumerate(MEMBERS[:3]):
        single = dm.Cavity(m["grid"], m["Ra"], wall_type=m["wall"], storage=1,
                           streaming=dm.STREAM_INPLACE)
        single.step(77)
        fe, ge = ip.populations(k)
        fs, gs = single.populations()
        assert np.array_equal(fe, fs) and np.array_equal(ge, gs), k


def test_in_place_ensemble_init_fields_in_both_layouts(dm):
    """A member's new state is written in whatever layout the ensemble is in
    (here after an odd and an even step count)."""
    ab = dm.Ensemble(MEMBERS, storage=1)
    ip = dm.Ensemble(MEMBERS, storage=1, streaming=dm.STREAM_INPLACE)
    for steps, member in ((5, 1), (4, 3)):
        m = MEMBERS[member]
        rho, u, th = inputs.random_fields(m["grid"], seed=steps)
        for e in (ab, ip):
            e.step(steps)
            e.init_fields(member, rho, u, th)
            e.step(3)
        _same_members(ab, ip, len(MEMBERS))


def test_in_place_ensemble_autotune_keeps_the_state(dm):
    ip = dm.Ensemble(MEMBERS, streaming=dm.STREAM_INPLACE)
    ip.step(41)  # the streamed layout
    before = [ip.populations(k) for k in range(len(MEMBERS))]
    report = ip.autotune(trials=2)
    assert "chosen threads=" in report
    for k in range(len(MEMBERS)):
        f, g = ip.populations(k)
        assert np.array_equal(f, before[k][0]) and np.array_equal(g, before[k][1])
    ab = dm.Ensemble(MEMBERS)
    ab.step(41)
    ip.step(20)
    ab.step(20)
    _same_members(ab, ip, len(MEMBERS))


def test_in_place_ensemble_holds_half_the_populations(dm):
    ab = dm.Ensemble(MEMBERS)
    ip = dm.Ensemble(MEMBERS, streaming=dm.STREAM_INPLACE)
    pa, pi = ab.params(0), ip.params(0)
    assert pi["streaming"] == dm.STREAM_INPLACE
    elems = sum((m["grid"][0] * m["grid"][1] * m["grid"][2] + 63) // 64 * 64 * 26 for m in MEMBERS)
    assert pa["device_bytes"] - pi["device_bytes"] == elems * 4 + 256


# every row length even: the ensemble takes two cells per thread (a 16-wide
# row gives 8-thread rows of pairs, tiles of 16 threads)
EVEN = [
    {"grid": (16, 16, 16), "Ra": 1e4, "wall": 1},
    {"grid": (20, 18, 16), "Ra": 5e4, "wall": 3},
    {"grid": (24, 24, 24), "Ra": 1e5, "wall": 2},
    {"grid": (38, 20, 13), "Ra": 3e4, "wall": 2},
    {"grid": (12, 12, 12), "Ra": 1e3, "wall": 1},
    {"grid": (130, 9, 5), "Ra": 2e5, "wall": 3},
]


@pytest.mark.parametrize("streaming", [0, 1], ids=["ab", "inplace"])
@pytest.mark.parametrize("storage", [0, 1, 2], ids=["f32", "bf16", "f16"])
def test_paired_members_evolve_bitwise_like_single_cavities(dm, storage, streaming):
    """Two cells per thread in the ensemble: every member bitwise equal to a
    single handle and to the same ensemble with one cell per thread, over 73
    steps (an odd count ends the in-place state in the streamed layout)."""
    two = dm.Ensemble(EVEN, storage=storage, streaming=streaming)
    one = dm.Ensemble(EVEN, storage=storage, streaming=streaming, cells_per_thread=1)
    assert two.params(0)["cells_per_thread"] == 2 and one.params(0)["cells_per_thread"] == 1
    two.step(73)
    one.step(73)
    for k, m in enumerate(EVEN):
        single = dm.Cavity(m["grid"], m["Ra"], wall_type=m["wall"], storage=storage, streaming=streaming)
        single.step(73)
        fe, ge = two.populations(k)
        fo, go = one.populations(k)
        fs, gs = single.populations()
        assert np.array_equal(fe, fo) and np.array_equal(ge, go), k
        assert np.array_equal(fe, fs) and np.array_equal(ge, gs), k


def test_paired_ensemble_autotune_and_requests(dm):
    """Autotuning the paired ensemble keeps its state; a member with an odd
    row length means one cell per thread, and asking for two is refused."""
    ens = dm.Ensemble(EVEN, storage=dm.STORE_BF16)
    ref = dm.Ensemble(EVEN, storage=dm.STORE_BF16)
    ens.step(20)
    ref.step(20)
    report = ens.autotune(trials=2)
    assert "threads=128" in report
    ens.step(30)
    ref.step(30)
    for k in range(len(EVEN)):
        fa, ga = ens.populations(k)
        fb, gb = ref.populations(k)
        assert np.array_equal(fa, fb) and np.array_equal(ga, gb), k
    assert dm.Ensemble(MEMBERS).params(0)["cells_per_thread"] == 1
    with pytest.raises(dm.DmrtError):
        dm.Ensemble(MEMBERS, cells_per_thread=2)


# ------------------------------------------------------------------ more members than one launch holds

def _many(count, even):
    """`count` small seeded cavities (edges 6..13, all wall types)."""
    rng = np.random.default_rng(99 if even else 98)
    out = []
    for k in range(count):
        nx, ny, nz = (int(v) for v in rng.integers(6, 14, size=3))
        if even:
            nx += nx & 1
        out.append({"grid": (nx, ny, nz), "Ra": float(10 ** rng.uniform(3, 5)), "wall": 1 + k % 3})
    return out


@pytest.mark.parametrize("even", [False, True], ids=["one_cell", "pairs"])
@pytest.mark.parametrize("streaming", [0, 1], ids=["ab", "inplace"])
def test_ensemble_of_more_members_than_one_launch_holds(dm, streaming, even):
    """A step launch carries at most 64 members' descriptors in its
    parameters; 150 members take three launches per step.  Members in every
    launch (first, last and boundary members) stay bitwise equal to single
    handles, through graph-replayed intervals, and the step count is three
    launches per step."""
    cav = _many(150, even)
    ens = dm.Ensemble(cav, storage=1, streaming=streaming, residual_interval=5)
    assert ens.params(0)["cells_per_thread"] == (2 if even else 1)
    dm.dmrt_ensemble_get_stats(ens.e, reset=True)
    ens.step(23)
    assert dm.dmrt_ensemble_get_stats(ens.e)["step_launches"] == 3 * 23
    for k in (0, 1, 63, 64, 65, 127, 128, 149):
        m = cav[k]
        single = dm.Cavity(m["grid"], m["Ra"], wall_type=m["wall"], storage=1, streaming=streaming)
        single.step(23)
        fe, ge = ens.populations(k)
        fs, gs = single.populations()
        assert np.array_equal(fe, fs) and np.array_equal(ge, gs), k
    r = np.asarray(ens.residual())
    assert np.all(np.isfinite(r))


@pytest.mark.parametrize("storage", [0, 1, 2], ids=["f32", "bf16", "f16"])
@pytest.mark.parametrize("streaming", [0, 1], ids=["ab", "inplace"])
def test_shape_groups_of_more_members_than_one_launch_holds(dm, streaming, storage):
    """With few distinct shapes and even rows, members are stepped by shape
    groups (the shape's offset tables in the launch parameters, the z extent
    repeated per member).  130 members of two interleaved shapes take two
    launches per shape and step; members of every launch stay bitwise equal
    to single handles."""
    shapes = [(10, 8, 6), (12, 10, 9)]
    cav = [{"grid": shapes[k % 2], "Ra": 10 ** (3 + 2 * k / 130), "wall": 1 + k % 3} for k in range(130)]
    ens = dm.Ensemble(cav, storage=storage, streaming=streaming, residual_interval=5)
    dm.dmrt_ensemble_get_stats(ens.e, reset=True)
    ens.step(23)
    assert dm.dmrt_ensemble_get_stats(ens.e)["step_launches"] == 4 * 23
    for k in (0, 1, 126, 127, 128, 129):
        m = cav[k]
        single = dm.Cavity(m["grid"], m["Ra"], wall_type=m["wall"], storage=storage, streaming=streaming)
        single.step(23)
        fe, ge = ens.populations(k)
        fs, gs = single.populations()
        assert np.array_equal(fe, fs) and np.array_equal(ge, gs), k
