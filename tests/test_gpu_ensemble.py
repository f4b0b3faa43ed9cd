"""Ensembles: many cavities advanced by one launch per time step.  Each member
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
    K = 50
    ens = dm.Ensemble(MEMBERS, residual_interval=K)
    ens.step(3 * K)
    r = ens.residual()
    for k, m in enumerate(MEMBERS):
        single = dm.Cavity(m["grid"], m["Ra"], wall_type=m["wall"], residual_interval=K)
        single.step(3 * K)
        assert r[k] == pytest.approx(single.residual(), rel=1e-12)


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


def test_ensemble_rejects_periodic_members_and_bad_indices(dm):
    with pytest.raises(dm.DmrtError) as ei:
        dm.Ensemble([{"grid": (8, 8, 8), "Ra": 1e4, "wall": 0}])
    assert ei.value.status == dm.ERR_ARG
    ens = dm.Ensemble(MEMBERS[:1])
    rho = np.empty((16, 16, 16), np.float32)
    with pytest.raises(dm.DmrtError) as ei:
        dm.dmrt_ensemble_fields(ens.e, 1, rho=rho)
    assert ei.value.status == dm.ERR_ARG
