"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: each checks it against an
independent definition (moment polynomials named in Eq. (22), lattice
isotropy, textbook LBGK, conservation laws, closed-form solutions of the
diffusion and shear-wave problems, symmetry of the cavity).
"""

import math

import numpy as np
import pytest

from paper_1511_04633_gb300 import inputs


# ------------------------------------------------------------------ matrices

def _moment_polynomials(e):
    """The moments of Eq. (22), written from their physical definitions
    (d'Humieres D3Q19 basis) as polynomials of one velocity e = (ex, ey, ez)."""
    ex, ey, ez = e
    e2 = ex * ex + ey * ey + ez * ez
    return [
        1,                                   # rho
        19 * e2 - 30,                        # e (energy)
        (21 * e2 * e2 - 53 * e2 + 24) / 2,   # epsilon (energy square)
        ex, (5 * e2 - 9) * ex,               # j_x, q_x
        ey, (5 * e2 - 9) * ey,               # j_y, q_y
        ez, (5 * e2 - 9) * ez,               # j_z, q_z
        3 * ex * ex - e2,                    # 3 p_xx
        (3 * e2 - 5) * (3 * ex * ex - e2),   # 3 pi_xx
        ey * ey - ez * ez,                   # p_ww
        (3 * e2 - 5) * (ey * ey - ez * ez),  # pi_ww
        ex * ey, ey * ez, ex * ez,           # p_xy, p_yz, p_xz
        (ey * ey - ez * ez) * ex,            # m_x
        (ez * ez - ex * ex) * ey,            # m_y
        (ex * ex - ey * ey) * ez,            # m_z
    ]


def test_printed_M_is_singular_and_row14_fix_restores_rank(orc):
    Mp = orc.matrix_M(printed=True)
    M = orc.matrix_M()
    assert np.linalg.matrix_rank(Mp) == 18
    assert np.linalg.matrix_rank(M) == 19
    diff = np.argwhere(Mp != M)
    assert {tuple(d) for d in diff} == {(13, 9), (13, 10)}


def test_M_rows_are_the_moment_polynomials_of_eq22(orc):
    E = orc.velocities19()
    M = orc.matrix_M()
    P = np.array([_moment_polynomials(e) for e in E]).T
    np.testing.assert_array_equal(M, P)


def test_M_is_orthogonal_with_dhumieres_norms(orc):
    M = orc.matrix_M()
    G = M @ M.T
    norms = [19, 2394, 252, 10, 40, 10, 40, 10, 40, 36, 72, 12, 24, 4, 4, 4, 8, 8, 8]
    np.testing.assert_array_equal(G, np.diag(norms))


def test_inverses_by_oracle_elimination(orc):
    M = orc.matrix_M()
    N = orc.matrix_N()
    Mi = orc.invert(M)
    Ni = orc.invert(N)
    np.testing.assert_allclose(M @ Mi, np.eye(19), atol=1e-14)
    np.testing.assert_allclose(Mi @ M, np.eye(19), atol=1e-14)
    np.testing.assert_allclose(N @ Ni, np.eye(7), atol=1e-14)
    # orthogonality gives the inverse in closed form: M^T diag(1/|M_k|^2)
    np.testing.assert_allclose(Mi, M.T / np.sum(M * M, axis=1), atol=1e-15)
    with pytest.raises(np.linalg.LinAlgError):
        orc.invert(orc.matrix_M(printed=True))


def test_N_rows_are_the_d3q7_moment_polynomials(orc):
    E = orc.velocities7()
    N = orc.matrix_N()
    rows = []
    for ex, ey, ez in E:
        e2 = ex * ex + ey * ey + ez * ez
        rows.append([1, ex, ey, ez, 6 - 7 * e2, 3 * ex * ex - e2, ey * ey - ez * ez])
    np.testing.assert_array_equal(N, np.array(rows).T)
    G = N @ N.T
    np.testing.assert_array_equal(G, np.diag([7, 2, 2, 2, 42, 12, 4]))


# ------------------------------------------------------------------ lattices

def test_d3q19_velocity_set_and_weight_isotropy(orc):
    E = orc.velocities19().astype(float)
    w = orc.weights19()
    assert sorted(map(tuple, E.astype(int))) == sorted(
        [(0, 0, 0)] + [tuple(v) for v in np.vstack([np.eye(3), -np.eye(3)]).astype(int)]
        + [(a, b, 0) for a in (1, -1) for b in (1, -1)]
        + [(a, 0, b) for a in (1, -1) for b in (1, -1)]
        + [(0, a, b) for a in (1, -1) for b in (1, -1)])
    assert abs(w.sum() - 1) < 1e-15
    np.testing.assert_allclose(np.einsum("i,ia->a", w, E), 0, atol=1e-16)
    # second moment c_s^2 delta with c_s^2 = 1/3 (Eq. (13), c = 1)
    np.testing.assert_allclose(np.einsum("i,ia,ib->ab", w, E, E), np.eye(3) / 3, atol=1e-16)
    np.testing.assert_allclose(np.einsum("i,ia,ib,ic->abc", w, E, E, E), 0, atol=1e-16)
    d = np.eye(3)
    iso4 = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
            + np.einsum("ad,bc->abcd", d, d)) / 9
    np.testing.assert_allclose(np.einsum("i,ia,ib,ic,id->abcd", w, E, E, E, E), iso4, atol=1e-16)


def test_d3q7_weights(orc):
    E = orc.velocities7().astype(float)
    w = orc.weights7()
    assert abs(w.sum() - 1) < 1e-15
    # thermal sound speed^2 = eps of Eq. (36) = 1/4
    np.testing.assert_allclose(np.einsum("i,ia,ib->ab", w, E, E), np.eye(3) / 4, atol=1e-16)


# ------------------------------------------------------------------ equilibria, force

def test_feq_moments_are_the_textbook_ones(orc):
    E = orc.velocities19().astype(float)
    rng = np.random.default_rng(1)
    for _ in range(20):
        rho = 1 + 0.1 * rng.uniform(-1, 1)
        V = 0.1 * rng.uniform(-1, 1, 3)
        f = orc.feq(rho, V)
        assert abs(f.sum() - rho) < 1e-14
        np.testing.assert_allclose(E.T @ f, rho * V, atol=1e-15)
        Pi = np.einsum("i,ia,ib->ab", f, E, E)
        np.testing.assert_allclose(Pi, rho / 3 * np.eye(3) + rho * np.outer(V, V), atol=1e-15)


def test_meq_is_M_times_feq_when_rho0_is_local_rho(orc):
    M = orc.matrix_M()
    rng = np.random.default_rng(2)
    for _ in range(20):
        rho = 1 + 0.1 * rng.uniform(-1, 1)
        V = 0.1 * rng.uniform(-1, 1, 3)
        np.testing.assert_allclose(M @ orc.feq(rho, V), orc.meq(rho, rho * V, rho0=rho), atol=5e-15)


def test_thermal_equilibrium_in_velocity_space(orc):
    E = orc.velocities7().astype(float)
    w = orc.weights7()
    Ni = orc.invert(orc.matrix_N())
    rng = np.random.default_rng(3)
    for _ in range(20):
        T = rng.uniform(-0.5, 0.5)
        V = 0.1 * rng.uniform(-1, 1, 3)
        g = Ni @ orc.neq(T, V)
        np.testing.assert_allclose(g, w * T * (1 + 4 * E @ V), atol=1e-16)


def test_force_sums_are_zero_mass_and_rho_G_momentum(orc):
    E = orc.velocities19().astype(float)
    rng = np.random.default_rng(4)
    for _ in range(20):
        rho = 1 + 0.1 * rng.uniform(-1, 1)
        V = 0.1 * rng.uniform(-1, 1, 3)
        G = 1e-3 * rng.uniform(-1, 1, 3)
        F = orc.force(rho, V, G)
        assert abs(F.sum()) < 1e-17
        np.testing.assert_allclose(E.T @ F, rho * G, atol=1e-17)


# ------------------------------------------------------------------ collision

def _cell(orc, gbeta=0.0, nu=0.05, alpha=0.07):
    return orc.Oracle((1, 1, 1), 0, nu, alpha, gbeta)


def test_rates_follow_eq26_and_eq36(orc):
    nu, alpha = 0.05, 0.07
    o = _cell(orc, nu=nu, alpha=alpha)
    s, q = o.rates()
    sn = 1 / (3 * nu + 0.5)
    expect = [1, 1.19, 1.4, 1, 1.2, 1, 1.2, 1, 1.2, sn, 1.4, sn, 1.4, sn, sn, sn, 1.98, 1.98, 1.98]
    np.testing.assert_allclose(s, expect, rtol=0, atol=1e-15)
    np.testing.assert_allclose(q, [1, 1 / (0.5 + 4 * alpha)] * 1 + [1 / (0.5 + 4 * alpha)] * 2 + [1, 1, 1],
                               atol=1e-15)


def test_collision_conserves_mass_momentum_energy_without_force(orc):
    E = orc.velocities19().astype(float)
    o = _cell(orc)
    f = inputs.random_populations((1, 1, 1), 19, seed=5).reshape(19).astype(float)
    g = inputs.random_thermal_populations((1, 1, 1), seed=6).reshape(7).astype(float)
    fo, go = o.collide(f, g)
    assert abs(fo.sum() - f.sum()) < 1e-15
    np.testing.assert_allclose(E.T @ fo, E.T @ f, atol=1e-15)
    assert abs(go.sum() - g.sum()) < 1e-15
    assert np.abs(fo - f).max() > 1e-3  # it did relax something


def test_collision_adds_rho_G_with_force(orc):
    E = orc.velocities19().astype(float)
    gbeta = 2e-3
    o = _cell(orc, gbeta=gbeta)
    f = inputs.random_populations((1, 1, 1), 19, seed=7).reshape(19).astype(float)
    g = inputs.random_thermal_populations((1, 1, 1), seed=8).reshape(7).astype(float)
    fo, go = o.collide(f, g)
    rho, T = f.sum(), g.sum()
    np.testing.assert_allclose(E.T @ fo - E.T @ f, [0, 0, rho * gbeta * T], rtol=1e-12, atol=1e-15)
    # reading A6: the buoyancy vanishes at theta_ref
    o.set_options(theta_ref=T)
    fo2, _ = o.collide(f, g)
    np.testing.assert_allclose(E.T @ fo2, E.T @ f, atol=1e-16)


def test_equilibrium_is_a_fixed_point(orc):
    o = _cell(orc)
    o.set_options(rho0_local=True)
    Ni = orc.invert(orc.matrix_N())
    rho, V, T = 1.03, np.array([0.02, -0.01, 0.03]), 0.2
    f = orc.feq(rho, V)
    g = Ni @ orc.neq(T, V)
    fo, go = o.collide(f, g)
    np.testing.assert_allclose(fo, f, atol=1e-15)
    np.testing.assert_allclose(go, g, atol=1e-16)
    # with rho0 = 1 (Eq. (24) as used) the rest state rho = 1 is still fixed
    o.set_options(rho0_local=False)
    f1 = orc.feq(1.0, V)
    fo1, _ = o.collide(f1, g)
    np.testing.assert_allclose(fo1, f1, atol=1e-15)


def test_single_rate_limit_is_textbook_lbgk(orc):
    """All s_k = 1/tau (and all q_k = 1/tau_g) turns the MRT collision into
    the BGK collision f* = f - (f - f_eq)/tau."""
    E7 = orc.velocities7().astype(float)
    w7 = orc.weights7()
    o = _cell(orc)
    o.set_options(rho0_local=True)
    tau, tau_g = 0.83, 0.71
    o.set_rates(np.full(19, 1 / tau), np.full(7, 1 / tau_g))
    E = orc.velocities19().astype(float)
    for seed in range(5):
        f = inputs.random_populations((1, 1, 1), 19, seed=10 + seed).reshape(19).astype(float)
        g = inputs.random_thermal_populations((1, 1, 1), seed=20 + seed).reshape(7).astype(float)
        rho = f.sum()
        V = E.T @ f / rho
        T = g.sum()
        fo, go = o.collide(f, g)
        np.testing.assert_allclose(fo, f - (f - orc.feq(rho, V)) / tau, atol=1e-15)
        geq = w7 * T * (1 + 4 * E7 @ V)
        np.testing.assert_allclose(go, g - (g - geq) / tau_g, atol=1e-16)


# ------------------------------------------------------------------ lattice units

@pytest.mark.parametrize("H,Ra", [(32, 1e3), (128, 1e5), (256, 1e6), (50, 1e4)])
def test_lattice_units_satisfy_eq38(orc, H, Ra):
    Pr, Ma = 0.71, 0.1
    nu, alpha, gbeta = orc.lattice_from_physics(H, Ra, Pr, Ma)
    uc = math.sqrt(gbeta * 1.0 * H)
    assert abs(uc / math.sqrt(1 / 3) - Ma) < 1e-14
    assert abs(gbeta * H ** 3 * Pr / nu ** 2 - Ra) < 1e-9 * Ra
    assert abs(nu / alpha - Pr) < 1e-14


def test_config1_lattice_values(orc):
    nu, alpha, gbeta = orc.lattice_from_physics(32, 1e3, 0.71, 0.1)
    assert abs(nu - 0.04923) < 5e-6
    assert abs(alpha - 0.06934) < 5e-6
    assert abs(gbeta - 1.0417e-4) < 1e-8


# ------------------------------------------------------------------ whole solver

def test_uniform_periodic_box_gains_rho_G_per_step(orc):
    gbeta, th = 1e-3, 0.3
    o = orc.Oracle((4, 4, 4), 0, 0.05, 0.07, gbeta)
    shape = o.shape
    o.init_fields(np.ones(shape), np.zeros((3,) + shape), np.full(shape, th))
    for n in range(1, 6):
        o.step(1)
        rho, u, T = o.fields()
        np.testing.assert_allclose(T, th, atol=1e-15)
        np.testing.assert_allclose(rho * u[2], n * gbeta * th, rtol=1e-12)
        np.testing.assert_allclose(u[:2], 0, atol=1e-15)


def test_periodic_conservation(orc):
    grid = (8, 6, 5)
    o = orc.Oracle(grid, 0, 0.04, 0.05, 0.0)
    rho0, u0, th0 = inputs.random_fields(grid, seed=30)
    o.init_fields(rho0, u0, th0)
    r0, u_, T0 = o.fields()
    m0 = (r0[None] * u_).sum(axis=(1, 2, 3))
    o.step(200)
    r1, u1, T1 = o.fields()
    assert abs(r1.sum() - r0.sum()) < 1e-12 * r0.sum()
    assert abs(T1.sum() - T0.sum()) < 1e-11
    np.testing.assert_allclose((r1[None] * u1).sum(axis=(1, 2, 3)), m0, atol=1e-12)


@pytest.mark.parametrize("wall", [1, 2, 3])
def test_rest_state_without_gravity(orc, wall):
    grid = (6, 7, 5)
    o = orc.Oracle(grid, wall, 0.05, 0.08, 0.0)
    _, _, th = inputs.random_fields(grid, seed=40 + wall)
    o.init_fields(np.ones(o.shape), np.zeros((3,) + o.shape), th)
    o.step(60)
    rho, u, T = o.fields()
    assert np.abs(u).max() < 1e-14  # round-off of the dense transforms only
    assert np.abs(rho - 1).max() < 1e-14
    assert np.abs(T - th).max() > 1e-3  # the temperature did evolve


@pytest.mark.parametrize("wall", [1, 2, 3])
def test_conduction_limit_is_linear_with_unit_nusselt(orc, wall):
    """g beta = 0: the steady temperature between theta = +1/2 at y = 0 and
    -1/2 at y = H is linear, and it also meets the linear side walls of
    Types 2 and 3; Nu = 1 on both walls (Eqs. (39)-(41))."""
    grid = (6, 12, 5)
    alpha = 0.125  # tau_alpha = 1
    o = orc.Oracle(grid, wall, 0.05, alpha, 0.0)
    o.step(3000)
    _, u, T = o.fields()
    ny = grid[1]
    y = (np.arange(ny) + 0.5) / ny
    exact = np.broadcast_to((0.5 - y)[None, :, None], o.shape)
    assert np.abs(T - exact).max() < 1e-9
    for w in (0, 1):
        (n3, n2, nmax), local = o.nusselt(w)
        assert abs(n3 - 1) < 1e-8 and abs(n2 - 1) < 1e-8 and abs(nmax - 1) < 1e-8
        assert np.abs(local - 1).max() < 1e-8
        # the heat carried across the wall links is the conductive flux alpha / H
        (f3, f2, fmax), flocal = o.nusselt_flux(w)
        assert np.abs(flocal - 1).max() < 1e-8


def _decay_rate(series, n_steps):
    return -math.log(series[-1] / series[0]) / n_steps


def test_shear_wave_decays_at_the_eq26_viscosity(orc):
    """u_x = U sin(k y) in a periodic box decays as exp(-nu k^2 t) with
    nu = (1/s_nu - 1/2)/3 (the textbook viscosity of the shear rate)."""
    ny, nu = 64, 0.04
    grid = (2, ny, 2)
    o = orc.Oracle(grid, 0, nu, 0.05, 0.0)
    k = 2 * math.pi / ny
    y = np.arange(ny)
    u = np.zeros((3,) + o.shape)
    u[0] = 1e-3 * np.sin(k * y)[None, :, None]
    o.init_fields(np.ones(o.shape), u, np.zeros(o.shape))
    o.step(100)  # let the non-equilibrium part settle
    amps = []
    for _ in range(2):
        _, uu, _ = o.fields()
        amps.append(2 * np.mean(uu[0, 0, :, 0] * np.sin(k * y)))
        o.step(800)
    rate = _decay_rate(amps, 800)
    assert abs(rate / (nu * k * k) - 1) < 5e-3


def test_thermal_wave_decays_at_the_eq36_diffusivity(orc):
    nx, alpha = 64, 0.03
    grid = (nx, 2, 2)
    o = orc.Oracle(grid, 0, 0.05, alpha, 0.0)
    k = 2 * math.pi / nx
    x = np.arange(nx)
    th = np.broadcast_to((0.1 * np.cos(k * x))[None, None, :], o.shape)
    o.init_fields(np.ones(o.shape), np.zeros((3,) + o.shape), th)
    o.step(50)
    amps = []
    for _ in range(2):
        _, _, T = o.fields()
        amps.append(2 * np.mean(T[0, 0] * np.cos(k * x)))
        o.step(1000)
    rate = _decay_rate(amps, 1000)
    assert abs(rate / (alpha * k * k) - 1) < 5e-3


def _rotated_tensor(d, angles):
    a, b = angles
    Rz = np.array([[np.cos(a), -np.sin(a), 0], [np.sin(a), np.cos(a), 0], [0, 0, 1]])
    Rx = np.array([[1, 0, 0], [0, np.cos(b), -np.sin(b)], [0, np.sin(b), np.cos(b)]])
    R = Rz @ Rx
    return R @ np.diag(d) @ R.T


@pytest.mark.parametrize("kvec", [(1, 1, 0), (1, 0, 1), (0, 1, -1), (1, 1, 1)])
def test_anisotropic_diffusion_decays_at_k_D_k(orc, kvec):
    """Eqs. (35)-(37) with off-diagonal tau_bar: a theta mode exp(i k.x) in a
    periodic box decays at the textbook rate k.D.k of the full tensor."""
    n = 32
    grid = (n, n, n)
    D = _rotated_tensor([0.02, 0.05, 0.08], (0.6, 0.9))
    o = orc.Oracle(grid, 0, 0.05, 0.05, 0.0)
    o.set_diffusion(D)
    k = 2 * math.pi / n * np.array(kvec, dtype=float)
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    phase = k[0] * x + k[1] * y + k[2] * z
    o.init_fields(np.ones(o.shape), np.zeros((3,) + o.shape), 0.1 * np.cos(phase))
    o.step(20)
    amps = []
    for _ in range(2):
        _, _, T = o.fields()
        amps.append(2 * np.mean(T * np.cos(phase)))
        o.step(300)
    rate = _decay_rate(amps, 300)
    assert abs(rate / (k @ D @ k) - 1) < 1e-2


def test_isotropic_tensor_reproduces_the_default_rates(orc):
    grid = (6, 7, 5)
    a = orc.Oracle.physical(grid, 2, 3e4)
    b = orc.Oracle.physical(grid, 2, 3e4)
    _, alpha, _ = orc.lattice_from_physics(7, 3e4, 0.71, 0.1)
    b.set_diffusion(alpha * np.eye(3))
    a.step(50)
    b.step(50)
    np.testing.assert_allclose(a.populations()[1], b.populations()[1], atol=1e-15)


def test_temperature_is_advected_by_the_flow_velocity(orc):
    """A theta wave in a uniform flow U along x travels at U (n_eq = V T)."""
    nx, U, steps = 64, 0.05, 400
    grid = (nx, 2, 2)
    o = orc.Oracle(grid, 0, 0.05, 0.02, 0.0)
    k = 2 * math.pi / nx
    x = np.arange(nx)
    u = np.zeros((3,) + o.shape)
    u[0] = U
    th = np.broadcast_to((0.1 * np.cos(k * x))[None, None, :], o.shape)
    o.init_fields(np.ones(o.shape), u, th)

    def phase():
        _, _, T = o.fields()
        c = np.sum(T[0, 0] * np.exp(-1j * k * x))
        return np.angle(c)

    p0 = phase()
    o.step(steps)
    p1 = phase()
    shift = ((p0 - p1) % (2 * math.pi)) / k
    assert abs(shift - U * steps) < 0.01 * U * steps


@pytest.mark.parametrize("wall", [1, 2, 3])
def test_mirror_symmetry_in_x(orc, wall):
    """Walls, gravity and the start state are symmetric under x -> H - x, so
    u_x is odd and rho, u_y, u_z, theta are even at every step."""
    grid = (8, 8, 8)
    o = orc.Oracle.physical(grid, wall, 1e5)
    o.step(150)
    rho, u, T = o.fields()
    flip = lambda a: a[..., ::-1]
    assert np.abs(u[0]).max() > 1e-6
    np.testing.assert_allclose(u[0], -flip(u[0]), atol=1e-14)
    for a in (rho, u[1], u[2], T):
        np.testing.assert_allclose(a, flip(a), atol=1e-13)


def test_hot_fluid_rises_along_the_hot_wall(orc):
    """Buoyancy along +z for theta > theta_ref (Eqs. (15), (16)) and the hot
    wall at y = 0 (Eq. (6)): the flow climbs along the hot wall and sinks
    along the cold one, and convection raises Nu above the conduction value
    of 1 (Sec. 4: Nu > 1 for every Ra of Tables 1-8)."""
    o = orc.Oracle.physical((12, 12, 12), 1, 2e4)
    o.step(2500)
    _, u, T = o.fields()
    w_hot = u[2][:, 0, :].mean()      # first fluid layer at the hot wall
    w_cold = u[2][:, -1, :].mean()    # ... at the cold wall
    assert w_hot > 0 > w_cold
    assert T[:, 0, :].mean() > 0 > T[:, -1, :].mean()
    (nu3, _, _), _ = o.nusselt(0)
    assert nu3 > 1.05


# ------------------------------------------------------------------ Nusselt, residual

def test_nusselt_is_exact_for_quadratic_profiles(orc):
    nx, ny, nz = 6, 10, 4
    rng = np.random.default_rng(50)
    a = rng.uniform(0.5, 2.0, size=(nz, nx))
    b = rng.uniform(-0.3, 0.3, size=(nz, nx))
    Y = (np.arange(ny) + 0.5) / ny
    theta = 0.5 - a[:, None, :] * Y[None, :, None] - b[:, None, :] * Y[None, :, None] ** 2
    (n3, n2, nmax), local = orc.nusselt_from_theta(theta, wall=0)
    np.testing.assert_allclose(local, a, atol=1e-12)
    assert abs(n3 - a.mean()) < 1e-12
    assert abs(n2 - a[:, 2:4].mean()) < 1e-12
    assert abs(nmax - a.max()) < 1e-12
    # cold wall: theta(Y=1) must be -1/2 for a consistent profile
    a_c = 1.0 - b
    theta_c = 0.5 - a_c[:, None, :] * Y[None, :, None] - b[:, None, :] * Y[None, :, None] ** 2
    (c3, _, _), local_c = orc.nusselt_from_theta(theta_c, wall=1)
    np.testing.assert_allclose(local_c, a_c + 2 * b, atol=1e-12)
    # odd nx: the single centre column
    (o3, o2, _), loc = orc.nusselt_from_theta(theta[..., :5], wall=0)
    assert abs(o2 - a[:, 2].mean()) < 1e-12


def test_flux_nusselt_balances_at_steady_convection(orc):
    """At a convecting steady state every heat unit entering through the hot
    wall leaves through the cold wall: the link fluxes of the two walls are
    equal (conservation), and the gradient formula agrees with them to its
    discretisation error."""
    o = orc.Oracle.physical((10, 10, 10), 2, 1e4)
    o.step(6000)
    (h3, _, _), _ = o.nusselt_flux(0)
    (c3, _, _), _ = o.nusselt_flux(1)
    assert abs(h3 - c3) < 1e-6 * h3
    (g3, _, _), _ = o.nusselt(0)
    assert abs(g3 - h3) < 0.05 * h3


def test_residual_definition(orc):
    rng = np.random.default_rng(60)
    th0 = rng.normal(size=100)
    u0 = rng.normal(size=(3, 100))
    th1 = th0 + 1e-3 * rng.normal(size=100)
    u1 = u0 + 1e-2 * rng.normal(size=(3, 100))
    r = orc.residual(th1, u1, th0, u0, 100)
    e_t = np.linalg.norm(th1 - th0) / np.linalg.norm(th1)
    e_u = np.linalg.norm(u1 - u0) / np.linalg.norm(u1)
    assert abs(r - max(e_t, e_u) / 100) < 1e-15
    z = np.zeros((3, 100))
    assert orc.residual(th1, z, th1, z, 10) == 0.0


@pytest.mark.parametrize("nu,alpha", [(0.04, 0.02), (0.02, 0.05)])
def test_residual_of_decaying_modes_matches_their_decay_rates(orc, nu, alpha):
    """Reading A11 against what the mathematics fixes.  In a periodic box
    without gravity, a shear mode u_x = U sin(k y) decays as exp(-nu k^2 t)
    and a temperature mode theta = Th cos(k y) as exp(-alpha k^2 t), each on
    its own.  Over K steps the change of a mode decaying at rate lam has norm
    (exp(lam K) - 1) times its current norm, so the residual must be
    max(exp(nu k^2 K) - 1, exp(alpha k^2 K) - 1) / K.  The two cases let
    the velocity and then the temperature term decide the maximum; with
    lam K near 0.4 a norm taken at the older state (1 - exp(-lam K)), a sum
    in place of the maximum, or a second division by K all miss by far more
    than the lattice's O(k^2) departure from the continuum rates (< 1e-3
    here)."""
    ny = 64
    grid = (2, ny, 2)
    k = 2 * math.pi / ny
    lam_u, lam_t = nu * k * k, alpha * k * k
    K = int(0.4 / max(lam_u, lam_t))
    o = orc.Oracle(grid, 0, nu, alpha, 0.0)
    y = np.arange(ny)
    u = np.zeros((3,) + o.shape)
    u[0] = 1e-3 * np.sin(k * y)[None, :, None]
    th = np.broadcast_to((0.1 * np.cos(k * y))[None, :, None], o.shape).copy()
    o.init_fields(np.ones(o.shape), u, th)
    o.step(200)  # let the non-equilibrium part settle
    _, u_prev, t_prev = o.fields()
    o.step(K)
    _, u_now, t_now = o.fields()
    r = orc.residual(t_now, u_now, t_prev, u_prev, K)
    exact = max(math.expm1(lam_u * K), math.expm1(lam_t * K)) / K
    assert abs(r / exact - 1) < 2e-3
    # the plausible mistakes named above, evaluated on the same modes
    older = max(-math.expm1(-lam_u * K), -math.expm1(-lam_t * K)) / K
    summed = (math.expm1(lam_u * K) + math.expm1(lam_t * K)) / K
    assert abs(older / exact - 1) > 0.2 and abs(summed / exact - 1) > 0.2
