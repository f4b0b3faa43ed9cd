"""Reduced-precision population storage (BF16 / FP16 deviations from the rest
equilibrium, FP32 collision) against the FP64 oracle and the FP32 path.

Tolerances are stated in units of the 16-bit unit roundoff u (FP16: 2^-11,
BF16: 2^-8), which bounds the relative error of one stored population:
  max |d theta| <= 2 u,  max |d u| <= 2 u u_c (u_c = Ma c_s, the velocity
  scale of Eq. (38)),  |d Nu_3D| / Nu_3D <= 2 u.
Round-to-nearest storage stagnates (per-step changes below half an ulp are
lost), so the library rounds 16-bit stores stochastically by default; the
last test shows the difference.
"""

import math

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

U16 = {1: 2.0 ** -8, 2: 2.0 ** -11}  # BF16, FP16
NAMES = {1: "bf16", 2: "f16"}
UC = 0.1 / math.sqrt(3.0)


@pytest.fixture(scope="module")
def dm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1511_04633_gb300 import dmrt
    dmrt.load()
    return dmrt


@pytest.fixture(scope="module")
def config1_oracle():
    o = oracle.Oracle.physical((32, 32, 32), 1, 1e3)
    o.step(2000)
    rho, u, th = o.fields()
    nu, _ = o.nusselt(0)
    return rho, u, th, nu


@pytest.mark.parametrize("storage", [1, 2], ids=["bf16", "f16"])
def test_config1_trajectory_against_the_oracle(dm, config1_oracle, storage):
    ro, uo, to, no = config1_oracle
    u16 = U16[storage]
    c = dm.Cavity((32, 32, 32), 1e3, wall_type=1, storage=storage)
    c.step(2000)
    r, u, t = c.fields()
    nu = c.nusselt(0)
    assert np.abs(t - to).max() <= 2 * u16
    assert np.abs(u - uo).max() <= 2 * u16 * UC
    assert np.abs(r - ro).max() <= 2 * u16 * 0.1
    assert abs(nu[0] - no[0]) <= 2 * u16 * no[0]


@pytest.mark.parametrize("storage", [1, 2], ids=["bf16", "f16"])
def test_ra1e6_type3_trajectory_against_the_oracle(dm, storage):
    grid = (24, 24, 24)
    o = oracle.Oracle.physical(grid, 3, 1e6)
    o.step(1000)
    _, uo, to = o.fields()
    no, _ = o.nusselt(0)
    u16 = U16[storage]
    c = dm.Cavity(grid, 1e6, wall_type=3, storage=storage)
    c.step(1000)
    _, u, t = c.fields()
    nu = c.nusselt(0)
    assert np.abs(t - to).max() <= 2 * u16
    assert np.abs(u - uo).max() <= 2 * u16 * UC
    assert abs(nu[0] - no[0]) <= 2 * u16 * no[0]


@pytest.fixture(scope="module")
def config3_reduced_oracle():
    """The Type 3, Ra = 1e6 cavity of the 256^3 reduced-precision workload at
    64^3, 600 steps from rest (the FP64 oracle cannot run 256^3)."""
    o = oracle.Oracle.physical((64, 64, 64), 3, 1e6)
    o.step(600)
    _, uo, to = o.fields()
    no, _ = o.nusselt(0)
    return uo, to, no


@pytest.mark.parametrize("storage", [0, 1, 2], ids=["f32", "bf16", "f16"])
def test_config3_at_64cube_against_the_oracle(dm, config3_reduced_oracle, storage):
    uo, to, no = config3_reduced_oracle
    c = dm.Cavity((64, 64, 64), 1e6, wall_type=3, storage=storage)
    c.step(600)
    _, u, t = c.fields()
    nu = c.nusselt(0)
    if storage == 0:
        assert np.abs(t - to).max() <= 1e-5 and np.abs(u - uo).max() <= 1e-5
        assert abs(nu[0] - no[0]) <= 1e-4 * no[0]
    else:
        u16 = U16[storage]
        assert np.abs(t - to).max() <= 2 * u16
        assert np.abs(u - uo).max() <= 2 * u16 * UC
        assert abs(nu[0] - no[0]) <= 2 * u16 * no[0]


@pytest.mark.parametrize("storage", [1, 2], ids=["bf16", "f16"])
def test_steady_nusselt_matches_fp32(dm, storage):
    """Type 1, 50^3, Ra = 1e4: the FP32 steady state against the time mean
    of the 16-bit run (stochastic rounding leaves a noise floor instead of a
    converged state)."""
    grid = (50, 50, 50)
    ref = dm.Cavity(grid, 1e4, wall_type=1)
    ok, _, _ = ref.run_to_steady(1e-7, 100_000)
    assert ok
    nu_ref = ref.nusselt(0)
    c = dm.Cavity(grid, 1e4, wall_type=1, storage=storage)
    c.step(30_000)
    acc = np.zeros(3)
    for _ in range(10):
        c.step(200)
        acc += np.array(c.nusselt(0))
    mean = acc / 10
    assert abs(mean[0] - nu_ref[0]) <= 2 * U16[storage] * nu_ref[0]
    assert abs(mean[1] - nu_ref[1]) <= 2 * U16[storage] * nu_ref[1]


@pytest.mark.parametrize("storage", [1, 2], ids=["bf16", "f16"])
def test_stochastic_rounding_is_bitwise_repeatable(dm, storage):
    a = dm.Cavity((20, 20, 20), 1e5, wall_type=2, storage=storage)
    b = dm.Cavity((20, 20, 20), 1e5, wall_type=2, storage=storage)
    a.step(300)
    b.step(300)
    fa, ga = a.populations()
    fb, gb = b.populations()
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)
    assert a.params["rounding"] == 2


def test_round_to_nearest_stagnates_and_stochastic_rounding_does_not(dm, config1_oracle):
    _, _, to, no = config1_oracle
    err = {}
    for rounding in (1, 2):
        c = dm.Cavity((32, 32, 32), 1e3, wall_type=1, storage=1, rounding=rounding)
        c.step(2000)
        _, _, t = c.fields()
        err[rounding] = float(np.abs(t - to).max())
    assert err[1] > 10 * err[2], err


def test_storage_reports_its_bytes(dm):
    for storage, bpc in ((0, 208), (1, 104), (2, 104)):
        c = dm.Cavity((8, 8, 8), 1e4, wall_type=1, storage=storage)
        assert dm.dmrt_get_stats(c.h)["bytes_per_cell"] == bpc


def _neighbours(v, storage):
    """The two storage values around v (as float64, lo < hi), F16 with its
    2^10 scale."""
    if storage == 1:
        bits = np.array([v], np.float32).view(np.uint32)[0]
        a = np.array([bits & 0xFFFF0000], np.uint32).view(np.float32)[0]
        b = np.array([(bits & 0xFFFF0000) + 0x10000], np.uint32).view(np.float32)[0]
        return tuple(sorted((float(a), float(b))))
    s = np.float32(v) * np.float32(1024.0)
    h = np.float16(s)
    other = np.nextafter(h, np.float16(np.inf) if float(h) < float(s) else np.float16(-np.inf))
    return tuple(sorted((float(h) / 1024.0, float(other) / 1024.0)))


@pytest.mark.parametrize("storage", [1, 2], ids=["bf16", "f16"])
@pytest.mark.parametrize("v", [0.3, -0.123456, 1.0e-3 + 1.7e-7, 0.0123, -4.321e-5, 3.1e-9])
def test_stochastic_rounding_is_unbiased(dm, storage, v):
    """Each rounded copy is one of the two neighbours of v, taken with
    probability (v - lo)/(hi - lo): the store keeps the expected value."""
    import torch
    n = 1 << 20
    v32 = float(np.float32(v))
    x = torch.full((n,), v32, device="cuda", dtype=torch.float32)
    y = dm.dmrt_round_to_storage(x, storage, dm.ROUND_STOCHASTIC, seed=12345).cpu().numpy().astype(np.float64)
    lo, hi = _neighbours(v32, storage)
    assert lo <= v32 <= hi
    up = y == hi
    assert np.all(up | (y == lo))
    p = (v32 - lo) / (hi - lo)
    # 6 sigma of the binomial count plus the 2^-12 resolution of the random bits
    tol = 6.0 * math.sqrt(max(p * (1 - p), 1e-6) / n) + 2.0 ** -12
    assert abs(up.mean() - p) <= tol, (up.mean(), p)
    # a second seed draws different bits; the same seed the same ones
    y2 = dm.dmrt_round_to_storage(x, storage, dm.ROUND_STOCHASTIC, seed=12345).cpu().numpy()
    assert np.array_equal(y2.astype(np.float64), y)


@pytest.mark.parametrize("storage", [1, 2], ids=["bf16", "f16"])
def test_round_to_nearest_storage(dm, storage):
    import torch
    rng = np.random.default_rng(3)
    v = (rng.standard_normal(4096) * 0.05).astype(np.float32)
    y = dm.dmrt_round_to_storage(torch.from_numpy(v).cuda(), storage, dm.ROUND_NEAREST).cpu().numpy()
    if storage == 1:
        ref = torch.from_numpy(v).to(torch.bfloat16).float().numpy()
    else:
        ref = ((v * np.float32(1024.0)).astype(np.float16).astype(np.float32) / np.float32(1024.0))
    assert np.array_equal(y, ref)


@pytest.mark.parametrize("storage", [1, 2], ids=["bf16", "f16"])
def test_config3_full_size_one_step_matches_the_oracle(dm, storage):
    """The reduced-precision workload at full size (256^3, Type 3, Ra = 1e6)
    in the launch shape the benchmark times: after 100 GPU steps from rest,
    one more GPU step must equal the oracle's step from the same stored state
    up to the rounding of one 16-bit store (below one unit in the last place
    of the stored value) plus FP32 round-off."""
    grid = (256, 256, 256)
    gpu = dm.Cavity(grid, 1e6, wall_type=3, storage=storage)
    gpu.step(100)
    f, g = gpu.populations()
    orc = oracle.Oracle.physical(grid, 3, 1e6)
    orc.set_populations(f.astype(np.float64), g.astype(np.float64))
    del f, g
    gpu.step(1)
    orc.step(1)
    rel = 2.0 ** -7 if storage == 1 else 2.0 ** -10
    w = oracle.weights19()[:, None, None, None]
    fg, gg = gpu.populations()
    fo, go = orc.populations()
    # deviations from the rest equilibrium are what the 16-bit store holds
    dg, do = fg.astype(np.float64) - w, fo - w
    assert np.all(np.abs(dg - do) <= rel * np.abs(do) + 1e-6)
    assert np.all(np.abs(gg.astype(np.float64) - go) <= rel * np.abs(go) + 1e-6)
