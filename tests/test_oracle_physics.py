"""Pins of the oracle's density, EOS, momentum/energy and viscosity (Sec. 3).

Checks are invariants and closed forms that a dropped term, a wrong sign or a
swapped index would break: lattice sums enumerated directly, exact pair
antisymmetry (momentum and L_z), the semi-discrete energy identity that ties
the momentum and energy forms together (readings R4-R6), the pressure
gradient of the rotating patch, and the dissipative sign of the viscosity.
"""
import math

import numpy as np
import pytest

from paper_1905_03344_gb300 import inputs


def _all(orc, f, lz=1.0, gamma=5 / 3, alpha=1.0, beta=2.0, eps=0.01):
    nb = orc.neighbors(f["x"], f["y"], f["z"], f["h"], lz=lz)
    rho = orc.density(f["x"], f["y"], f["z"], f["m"], f["h"], nb, lz=lz)
    P, c = orc.eos(rho, f["u"], gamma)
    ax, ay, az, du, sa, sdu = orc.momentum_energy(f["x"], f["y"], f["z"], f["vx"], f["vy"], f["vz"],
                                                  f["m"], f["h"], rho, P, c, nb, lz=lz,
                                                  alpha=alpha, beta=beta, eps=eps)
    return dict(nb=nb, rho=rho, P=P, c=c, ax=ax, ay=ay, az=az, du=du, sa=sa, sdu=sdu)


def test_interior_density_equals_direct_lattice_sum(orc):
    n = 16
    f = inputs.square_patch(n)
    r = _all(orc, f)
    dx = 1.0 / n
    h = f["h"][0]
    m = f["m"][0]
    R = 3
    s = 0.0
    for a in range(-R, R + 1):
        for b in range(-R, R + 1):
            for d in range(-R, R + 1):
                s += m * orc.w(dx * math.sqrt(a * a + b * b + d * d), h)
    interior = (np.abs(f["x"]) < 0.5 - 3.5 / n) & (np.abs(f["y"]) < 0.5 - 3.5 / n)
    assert np.allclose(r["rho"][interior], s, rtol=1e-13, atol=0)
    # the SPH estimate of rho0 = 1 on a lattice; the self term alone is ~14 %
    assert abs(s - 1.0) < 0.02
    assert m * orc.w(0.0, h) > 0.1


def test_eos_sound_speed_closed_form(orc):
    rng = np.random.default_rng(1)
    rho = rng.uniform(0.1, 3.0, 100)
    u = rng.uniform(0.5, 900.0, 100)
    P, c = orc.eos(rho, u, 5.0 / 3.0)
    # ideal gas: c^2 = gamma (gamma - 1) u, independent of rho; P/rho = (gamma-1) u
    assert np.allclose(c, np.sqrt(10.0 / 9.0 * u), rtol=1e-14)
    assert np.allclose(P / rho, 2.0 / 3.0 * u, rtol=1e-14)


@pytest.mark.parametrize("seed,kernel", [(0, "wendland"), (1, "wendland"), (5, "sinc")])
def test_momentum_and_lz_conserved_exactly(orc, seed, kernel):
    f = inputs.random_cloud(1200, seed=seed, vscale=3.0)
    with orc.kernel(kernel, 6):
        r = _all(orc, f)
    m = f["m"]
    scale = np.sum(m * r["sa"])
    assert scale > 0
    for comp in ("ax", "ay", "az"):
        assert abs(np.sum(m * r[comp])) < 1e-13 * scale
    lz = np.sum(m * (f["x"] * r["ay"] - f["y"] * r["ax"]))
    assert abs(lz) < 1e-13 * scale


@pytest.mark.parametrize("seed,kernel", [(2, "wendland"), (3, "wendland"), (4, "sinc")])
def test_semi_discrete_energy_identity(orc, seed, kernel):
    # sum_i m_i (v_i . a_i + du_i) = 0 pairs the momentum form (R4) with the
    # energy form (R6), viscosity included (R5), for either kernel of Sec. 3
    f = inputs.random_cloud(1200, seed=seed, vscale=3.0)
    with orc.kernel(kernel, 6):
        r = _all(orc, f)
    m = f["m"]
    vdota = f["vx"] * r["ax"] + f["vy"] * r["ay"] + f["vz"] * r["az"]
    total = np.sum(m * (vdota + r["du"]))
    vmag = np.sqrt(f["vx"] ** 2 + f["vy"] ** 2 + f["vz"] ** 2)
    scale = np.sum(m * (vmag * r["sa"] + r["sdu"]))
    assert np.sum(m * r["du"]) != 0.0
    assert abs(total) < 1e-13 * scale
    # the identity is not vacuous: each half alone is far from zero
    assert abs(np.sum(m * vdota)) > 1e-3 * scale


def test_rotating_patch_pressure_gradient(orc):
    # Sec. 4: away from the free surface the SPH momentum sum must reproduce
    # a = -grad P0 / rho0 of the series pressure (the constant offset cancels
    # by lattice symmetry); grad P0 comes from finite differences of the
    # series, not from any SPH formula.  Rigid rotation has v_ij . x_ij = 0,
    # so du vanishes to rounding.
    n = 30
    f = inputs.square_patch(n)
    r = _all(orc, f)
    d = 1e-5
    gx = (inputs.pressure_series(f["x"] + d, f["y"]) - inputs.pressure_series(f["x"] - d, f["y"])) / (2 * d)
    gy = (inputs.pressure_series(f["x"], f["y"] + d) - inputs.pressure_series(f["x"], f["y"] - d)) / (2 * d)
    deep = (np.abs(f["x"]) < 0.5 - 4.0 / n) & (np.abs(f["y"]) < 0.5 - 4.0 / n)
    err = np.hypot(r["ax"][deep] + gx[deep], r["ay"][deep] + gy[deep])
    ref = np.hypot(gx[deep], gy[deep]).max()
    assert err.max() < 0.02 * ref
    assert np.abs(r["az"]).max() < 1e-9 * np.abs(r["sa"]).max()
    assert np.all(np.abs(r["du"]) <= 1e-12 * r["sdu"] + 1e-300)
    # the constant pressure offset pushes the free surface outward
    edge = f["x"] > 0.5 - 0.6 / n
    assert np.all(r["ax"][edge] > 0)


def test_viscosity_dissipates(orc):
    # zero pressure, converging flow v = -x: only the viscosity acts.  It must
    # heat every particle that has neighbours and remove kinetic energy.
    f = inputs.random_cloud(900, seed=7)
    f["u"] = np.zeros_like(f["u"])
    f["vx"], f["vy"], f["vz"] = -f["x"], -f["y"], np.zeros_like(f["z"])
    r = _all(orc, f)
    has = np.diff(r["nb"].off) > 0
    assert np.all(r["du"][has] > 0)
    assert np.sum(f["m"] * (f["vx"] * r["ax"] + f["vy"] * r["ay"])) < 0
    # diverging flow: v_ij . x_ij > 0 for all pairs -> no viscosity, no force
    f["vx"], f["vy"] = f["x"].copy(), f["y"].copy()
    f["vz"] = np.zeros_like(f["z"])
    f["z"] = np.zeros_like(f["z"])
    r = _all(orc, f)
    assert np.all(r["ax"] == 0) and np.all(r["du"] == 0)


def test_viscosity_scales_with_alpha_beta(orc):
    # Pi = (-alpha cbar mu + beta mu^2)/rhobar is linear in (alpha, beta):
    # the viscous parts of du for (1,0) and (0,1) add up to that of (1,1)
    f = inputs.random_cloud(600, seed=8, vscale=2.0)
    base = _all(orc, f, alpha=0.0, beta=0.0)["du"]
    a = _all(orc, f, alpha=1.0, beta=0.0)["du"] - base
    b = _all(orc, f, alpha=0.0, beta=1.0)["du"] - base
    ab = _all(orc, f, alpha=1.0, beta=1.0)["du"] - base
    scale = np.abs(a).max() + np.abs(b).max()
    assert np.abs(a + b - ab).max() < 1e-11 * scale
    assert np.all(a >= -1e-12 * scale) and np.all(b >= -1e-12 * scale)


def test_courant(orc):
    h = np.array([0.1, 0.2, 0.05])
    c = np.array([1.0, 1.0, 2.0])
    assert orc.courant(h, c, 0.2) == pytest.approx(0.2 * 0.025, rel=1e-15)


# ---- the grad-h form (reading R20): Omega and the per-side pressure terms ----

@pytest.mark.parametrize("kernel", ["wendland", "sinc"])
def test_dwdh_is_derivative(orc, kernel):
    with orc.kernel(kernel, 6):
        for h in (1.0, 0.07):
            for v in np.linspace(0.0, 1.95, 21):
                r = v * h
                d = 1e-6 * h
                fd = (orc.w(r, h + d) - orc.w(r, h - d)) / (2 * d)
                assert orc.dwdh(r, h) == pytest.approx(fd, rel=1e-6, abs=1e-8 / h ** 4)


@pytest.mark.parametrize("kernel", ["wendland", "sinc"])
def test_omega_is_the_density_derivative(orc, kernel):
    # Omega_i = 1 + h_i/(3 rho_i) d rho_i / d h_i: a central difference of the
    # density itself (lists of the larger h, a superset) must agree
    f = inputs.random_cloud(800, seed=7, h_lo=0.08, h_hi=0.12)
    with orc.kernel(kernel, 6):
        d = 1e-5
        big = orc.neighbors(f["x"], f["y"], f["z"], f["h"] * (1 + 2 * d))
        rho = orc.density(f["x"], f["y"], f["z"], f["m"], f["h"], big)
        rp = orc.density(f["x"], f["y"], f["z"], f["m"], f["h"] * (1 + d), big)
        rm = orc.density(f["x"], f["y"], f["z"], f["m"], f["h"] * (1 - d), big)
        om = orc.omega(f["x"], f["y"], f["z"], f["m"], f["h"], rho, big)
    # rho_i depends on h_i only (W(r, h_i)): d rho / d h_i by the scaled-h difference
    fd = 1.0 + f["h"] / (3 * rho) * (rp - rm) / (2 * d * f["h"])
    assert np.allclose(om, fd, rtol=0, atol=1e-6)
    assert np.all(np.abs(om - 1.0) > 1e-3)     # not trivially one in a random cloud


@pytest.mark.parametrize("kernel", ["wendland", "sinc"])
def test_omega_near_one_on_a_lattice(orc, kernel):
    n = 16
    f = inputs.square_patch(n)
    with orc.kernel(kernel, 6):
        nb = orc.neighbors(f["x"], f["y"], f["z"], f["h"])
        rho = orc.density(f["x"], f["y"], f["z"], f["m"], f["h"], nb)
        om = orc.omega(f["x"], f["y"], f["z"], f["m"], f["h"], rho, nb)
    interior = (np.abs(f["x"]) < 0.5 - 3.5 / n) & (np.abs(f["y"]) < 0.5 - 3.5 / n)
    assert np.all(np.abs(om[interior] - 1.0) < 0.05)


def test_gradh_with_unit_omega_and_equal_h_is_the_standard_form(orc):
    # with Omega = 1 and one h for all, A_i grad W_i + A_j grad W_j = (A_i + A_j) grad Wbar
    f = inputs.random_cloud(600, seed=9, h_lo=0.1, h_hi=0.1, vscale=2.0)
    std = _all(orc, f)
    gh = orc.momentum_energy(f["x"], f["y"], f["z"], f["vx"], f["vy"], f["vz"], f["m"], f["h"],
                             std["rho"], std["P"], std["c"], std["nb"], omega=np.ones(len(f["x"])))
    scale = np.maximum(std["sa"], 1e-300)
    for k, comp in enumerate(("ax", "ay", "az")):
        assert np.max(np.abs(gh[k] - std[comp]) / scale) < 1e-13
    assert np.max(np.abs(gh[3] - std["du"]) / np.maximum(std["sdu"], 1e-300)) < 1e-13


@pytest.mark.parametrize("kernel", ["wendland", "sinc"])
def test_gradh_conserves_momentum_and_energy(orc, kernel):
    f = inputs.random_cloud(1000, seed=11, vscale=3.0, h_lo=0.06, h_hi=0.12)
    with orc.kernel(kernel, 6):
        nb = orc.neighbors(f["x"], f["y"], f["z"], f["h"])
        rho = orc.density(f["x"], f["y"], f["z"], f["m"], f["h"], nb)
        P, c = orc.eos(rho, f["u"])
        om = orc.omega(f["x"], f["y"], f["z"], f["m"], f["h"], rho, nb)
        ax, ay, az, du, sa, sdu = orc.momentum_energy(f["x"], f["y"], f["z"], f["vx"], f["vy"], f["vz"],
                                                      f["m"], f["h"], rho, P, c, nb, omega=om)
    m = f["m"]
    scale = np.sum(m * sa)
    for a in (ax, ay, az):
        assert abs(np.sum(m * a)) < 1e-13 * scale
    assert abs(np.sum(m * (f["x"] * ay - f["y"] * ax))) < 1e-13 * scale
    vdota = f["vx"] * ax + f["vy"] * ay + f["vz"] * az
    vmag = np.sqrt(f["vx"] ** 2 + f["vy"] ** 2 + f["vz"] ** 2)
    total = np.sum(m * (vdota + du))
    assert abs(total) < 1e-13 * np.sum(m * (vmag * sa + sdu))


@pytest.mark.parametrize("kernel", ["wendland", "sinc"])
def test_omega_of_an_isolated_particle_is_zero(orc, kernel):
    # the self term alone: rho = m W(0, h), dW(0, h)/dh = -3 W(0, h)/h, so
    # Omega = 1 + h/(3 m W(0)) m (-3 W(0)/h) = 0
    f = {k: np.zeros(2) for k in ("x", "y", "z", "vx", "vy", "vz")}
    f.update(x=np.array([0.1, 0.7]), m=np.array([0.5, 0.25]), h=np.array([0.1, 0.05]), u=np.ones(2))
    with orc.kernel(kernel, 6):
        nb = orc.neighbors(f["x"], f["y"], f["z"], f["h"])
        assert nb.off[-1] == 0
        rho = orc.density(f["x"], f["y"], f["z"], f["m"], f["h"], nb)
        om = orc.omega(f["x"], f["y"], f["z"], f["m"], f["h"], rho, nb)
    assert np.all(np.abs(om) < 4e-16)


@pytest.mark.parametrize("v", [0.3, 0.9, 1.4, 1.9])
def test_omega_of_a_wendland_pair(orc, v):
    # two equal particles at r = v h: with S(v) = q^4 (5 - 4q), q = 1 - v/2,
    # d(h^-3 S(r/h))/dh = -h^-4 (3 S + v S'(v)) and v S'(v) = -20 (1-q)^2 q^3:
    #   Omega = 1 - (3 + 3 S - 20 (1-q)^2 q^3) / (3 (1 + S)) = 20 (1-q)^2 q^3 / (3 (1 + S))
    h = 0.1
    f = {k: np.zeros(2) for k in ("x", "y", "z", "vx", "vy", "vz")}
    f.update(x=np.array([0.2, 0.2 + v * h]), m=np.full(2, 0.3), h=np.full(2, h), u=np.ones(2))
    nb = orc.neighbors(f["x"], f["y"], f["z"], f["h"])
    rho = orc.density(f["x"], f["y"], f["z"], f["m"], f["h"], nb)
    om = orc.omega(f["x"], f["y"], f["z"], f["m"], f["h"], rho, nb)
    q = 1.0 - v / 2.0
    S = q ** 4 * (5.0 - 4.0 * q)
    want = 20.0 * (1.0 - q) ** 2 * q ** 3 / (3.0 * (1.0 + S))
    assert om == pytest.approx([want, want], rel=1e-12, abs=1e-15)


@pytest.mark.parametrize("kernel", ["wendland", "sinc"])
@pytest.mark.parametrize("seed", [1, 2])
def test_omega_never_negative(orc, kernel, seed):
    # both kernel shapes decrease on their support, so each neighbour adds a
    # non-negative -v S'(v) to Omega and the self term adds nothing: Omega >= 0
    # up to the rounding of 1 + (a sum near -1)
    f = inputs.random_cloud(1500, seed=seed, h_lo=0.03, h_hi=0.2)
    with orc.kernel(kernel, 6):
        nb = orc.neighbors(f["x"], f["y"], f["z"], f["h"])
        rho = orc.density(f["x"], f["y"], f["z"], f["m"], f["h"], nb)
        om = orc.omega(f["x"], f["y"], f["z"], f["m"], f["h"], rho, nb)
    assert om.min() > -1e-14
    assert om.max() > 0.5
