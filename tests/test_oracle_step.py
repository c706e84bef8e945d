"""Pins of the oracle's timestep: integrators (reading R8), Courant dt with
growth cap (R7), h adaptation (R10), conservation over steps, and the initial
pressure series of the square patch (Sec. 4, reading R12)."""
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spl

from paper_1905_03344_gb300 import inputs


def test_ballistic_motion_is_exact(orc):
    # no pressure, diverging flow (no viscosity): a = 0, du = 0, x moves on a line
    f = inputs.random_cloud(400, seed=1)
    f["u"] = np.zeros_like(f["u"])
    f["z"] = np.zeros_like(f["z"])
    f["vx"], f["vy"], f["vz"] = 0.3 * f["x"], 0.3 * f["y"], np.zeros_like(f["x"])
    x0, y0 = f["x"].copy(), f["y"].copy()
    s = orc.Sim(f, dt_fixed=1e-3, adapt_h=False)
    s.step(7)
    assert np.allclose(s["x"], x0 * (1 + 0.3 * 7e-3), rtol=1e-13)
    assert np.allclose(s["y"], y0 * (1 + 0.3 * 7e-3), rtol=1e-13)
    assert np.all(s["u"] == 0)


def _run_to(orc, f, dt, T):
    s = orc.Sim(f, dt_fixed=dt, adapt_h=False, av_alpha=0.0, av_beta=0.0, use_grid=0)
    s.step(int(round(T / dt)))
    return s


def test_second_order_in_time(orc):
    # Press/leapfrog positions and Adams-Bashforth energy are both second order:
    # errors against a fine run shrink ~4x per halving of dt (Euler would give 2x)
    f = inputs.random_cloud(300, seed=4, vscale=0.5, h_lo=0.15, h_hi=0.2)
    T = 0.04
    ref = _run_to(orc, f, T / 256, T)
    ex, eu = [], []
    for k in (16, 32, 64):
        s = _run_to(orc, f, T / k, T)
        ex.append(np.abs(s["x"] - ref["x"]).max())
        eu.append(np.abs(s["u"] - ref["u"]).max())
    for e in (ex, eu):
        r1, r2 = e[0] / e[1], e[1] / e[2]
        assert 3.0 < r1 < 5.5 and 3.0 < r2 < 5.5, e


def test_first_step_half_kick(orc):
    # step 0: v_1/2 = v_0 + a_0 dt_0 / 2 and u_1 = u_0 + dt_0 du_0 (reading R8)
    f = inputs.random_cloud(300, seed=6, vscale=1.0)
    s = orc.Sim(f, adapt_h=False)
    s.step(1)
    dt = s.dt
    assert np.allclose(s["vx"], f["vx"] + 0.5 * dt * s["ax"], rtol=1e-14, atol=1e-300)
    assert np.allclose(s["u"], f["u"] + dt * s["du"], rtol=1e-14, atol=1e-300)
    assert np.allclose(s["x"], f["x"] + dt * s["vx"], rtol=1e-14, atol=1e-300)
    # second step: full kick with (dt_1 + dt_0)/2 and the AB2 weights
    v1, u1, du0, dt0 = s["vx"].copy(), s["u"].copy(), s["du"].copy(), dt
    s.step(1)
    dt1 = s.dt
    assert np.allclose(s["vx"], v1 + 0.5 * (dt1 + dt0) * s["ax"], rtol=1e-13, atol=1e-300)
    r = dt1 / dt0
    assert np.allclose(s["u"], u1 + dt1 * ((1 + r / 2) * s["du"] - (r / 2) * du0), rtol=1e-13)


def test_courant_and_growth_cap(orc):
    f = inputs.square_patch(10)
    s = orc.Sim(f)
    s.step(1)
    assert s.dt == pytest.approx(0.2 * np.min(f["h"] / s["c"]), rel=1e-15)
    dts = [s.dt]
    for _ in range(6):
        hh = s["h"].copy()
        s.step(1)
        cand = 0.2 * np.min(hh / s["c"])
        assert s.dt == pytest.approx(min(cand, 1.1 * dts[-1]), rel=1e-15)
        dts.append(s.dt)


def test_h_adaptation_fixed_point(orc):
    f = inputs.square_patch(12)
    s = orc.Sim(f)
    s.step(1)
    n = s["nown"].astype(float)
    # h_new = h (1 + (100/n)^(1/3)) / 2: a particle with n = 100 keeps its h
    ratio = s["h"] / f["h"]
    assert np.allclose(ratio, 0.5 * (1 + np.cbrt(100.0 / n)), rtol=1e-14)
    s.step(12)
    deep = (np.abs(s["x"]) < 0.2) & (np.abs(s["y"]) < 0.2)
    assert np.all(np.abs(s["nown"][deep] - 100) <= 12)


def test_conservation_over_steps(orc):
    f = inputs.square_patch(12)
    s = orc.Sim(f)
    c0 = s.conserved()
    s.step(8)
    c1 = s.conserved()
    m = s["m"]
    vscale = np.sum(m * np.sqrt(s["vx"] ** 2 + s["vy"] ** 2 + s["vz"] ** 2))
    lscale = np.sum(m * np.hypot(s["x"], s["y"]) * np.hypot(s["vx"], s["vy"]))
    assert c1[0] == c0[0]
    for q in (1, 2, 3):                         # linear momentum
        assert abs(c1[q] - c0[q]) < 1e-12 * vscale
    assert abs(c1[4] - c0[4]) < 1e-12 * lscale  # L_z about the patch axis
    assert c0[1] == pytest.approx(0.0, abs=1e-14) and c0[2] == pytest.approx(0.0, abs=1e-14)


# --------------------------- the initial pressure --------------------------------

def test_series_zero_on_edges():
    t = np.linspace(-0.5, 0.5, 41)
    for xs, ys in ((np.full_like(t, -0.5), t), (np.full_like(t, 0.5), t),
                   (t, np.full_like(t, -0.5)), (t, np.full_like(t, 0.5))):
        assert np.abs(inputs.pressure_series(xs, ys)).max() < 1e-10


def test_series_satisfies_poisson():
    # grad^2 P0 = 2 rho omega^2 for the rigid rotation (incompressible Euler)
    w = 5.0
    d = 1e-3
    for (x, y) in [(0.0, 0.0), (0.1, -0.2), (-0.3, 0.25)]:
        lap = (inputs.pressure_series(x + d, y) + inputs.pressure_series(x - d, y) +
               inputs.pressure_series(x, y + d) + inputs.pressure_series(x, y - d) -
               4 * inputs.pressure_series(x, y)) / d ** 2
        assert lap == pytest.approx(2 * w * w, rel=0.02)


def test_series_matches_finite_difference_solution():
    # independent solution of grad^2 P = 2 omega^2, P = 0 on the square edges
    w = 5.0

    def solve(M):
        hgrid = 1.0 / M
        k = M - 1
        T = sp.diags([np.ones(k - 1), -2 * np.ones(k), np.ones(k - 1)], [-1, 0, 1])
        I = sp.identity(k)
        A = (sp.kron(I, T) + sp.kron(T, I)) / hgrid ** 2
        sol = spl.spsolve(A.tocsc(), np.full(k * k, 2 * w * w))
        return sol.reshape(k, k)

    vals = []
    for M in (64, 128):
        s = solve(M)
        vals.append(s[M // 2 - 1, M // 2 - 1])           # centre of the square
    centre = (4 * vals[1] - vals[0]) / 3                # Richardson, O(h^4)
    assert inputs.pressure_series(0.0, 0.0) == pytest.approx(centre, rel=2e-5)
    s = solve(128)
    q = s[128 // 4 * 3 - 1, 128 // 2 - 1]               # (x, y) = (0.25, 0)
    assert inputs.pressure_series(0.25, 0.0) == pytest.approx(q, rel=1e-3)


def test_series_symmetry_and_offset():
    g = np.linspace(-0.45, 0.45, 7)
    X, Y = np.meshgrid(g, g)
    P = inputs.pressure_series(X, Y)
    assert np.allclose(P, P.T, rtol=1e-12)              # P(x, y) = P(y, x)
    assert np.allclose(P, P[:, ::-1], rtol=1e-12)        # P(-x, y) = P(x, y)
    assert np.all(P < 0)
    # c0 = 10 omega L / sqrt 2, P_off = rho0 c0^2 / gamma = 750 for omega = 5
    assert inputs.pressure_offset() == pytest.approx(750.0, rel=1e-14)


def test_patch_initial_state():
    f = inputs.square_patch(10)
    assert np.allclose(f["vx"], 5.0 * f["y"]) and np.allclose(f["vy"], -5.0 * f["x"])
    assert f["m"].sum() == pytest.approx(1.0, rel=1e-14)
    assert np.all(f["u"] > 0)
    # 100 neighbours within 2h on average: (4/3) pi (2 h)^3 / dx^3 = 100
    dx = 0.1
    assert 4.0 / 3.0 * math.pi * (2 * f["h"][0]) ** 3 / dx ** 3 == pytest.approx(100.0, rel=1e-12)
