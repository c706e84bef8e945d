"""Pins of the oracle's artificial viscosity (reading R5 of the Monaghan form
cited in Sec. 3) and of its energy sums (the conserved quantities Sec. 4
stresses), against values worked out by hand.

Viscosity.  Two or three particles on the x axis with binary-exact inputs;
rho, P and c are handed to the momentum/energy sum directly, so Pi_ij is the
only unknown.  For each case Pi_ij was worked out with pencil and paper from
R5 (Pi = (-alpha cbar mu + beta mu^2)/rhobar for approaching pairs,
mu = hbar v_ij.x_ij / (r^2 + eps hbar^2), bars = arithmetic means,
alpha = 1, beta = 2, eps = 0.01) and is stored below as an exact fraction.
The second case gives every mean two different ends, so a slip in any of
them (h_i for hbar, rho_i for rhobar, max c for cbar, eps hbar for
eps hbar^2) changes the value.  The kernel gradient is taken from the
oracle's own gradw_fac, pinned by finite differences elsewhere.

Energy sums.  Lattice sums in closed form: on the n^3 square patch,
sum over one axis of x_k^2 = (n^2 - 1)/(12 n), so with m = 1/n^3 and the rigid
rotation v = omega (y, -x): E_kin = omega^2 (n^2 - 1)/(12 n^2) and
L_z = -omega (n^2 - 1)/(6 n^2).  Unequal masses with uniform u and v check
that each sum carries m (and E_kin its 1/2).  Finally the time-discrete
total energy E_kin + E_int, at synchronised times, drifts as dt^2 when the
step is halved (Press positions and Adams-Bashforth energy are both second
order; the semi-discrete energy is conserved exactly, R4-R6)."""
from fractions import Fraction as Fr

import numpy as np
import pytest

from paper_1905_03344_gb300 import inputs


def _line(xs, vxs, h, m, rho, P, c):
    n = len(xs)
    z = np.zeros(n)
    return dict(x=np.array(xs, float), y=z.copy(), z=z.copy(), vx=np.array(vxs, float), vy=z.copy(),
                vz=z.copy(), m=np.array(m, float), h=np.array(h, float), rho=np.array(rho, float),
                P=np.array(P, float), c=np.array(c, float))


def _sums(orc, f, alpha=1.0, beta=2.0, eps=0.01):
    nb = orc.neighbors(f["x"], f["y"], f["z"], f["h"])
    out = orc.momentum_energy(f["x"], f["y"], f["z"], f["vx"], f["vy"], f["vz"], f["m"], f["h"],
                              f["rho"], f["P"], f["c"], nb, alpha=alpha, beta=beta, eps=eps)
    return nb, out


# Case A: i at 0 moving at +1/2 towards j at 1/4 at rest; h = 1/4 on both;
# c = 1 on both; rho = 1 and 2.  x_ij = -1/4, v_ij.x_ij = -1/8, r^2 = 1/16.
#   hbar = 1/4, eps hbar^2 = 1/1600, mu = (1/4)(-1/8) / (101/1600) = -50/101
#   Pi = (50/101 + 2 (50/101)^2) / (3/2) = 6700/10201
PI_A = Fr(6700, 10201)
# Case B: as A but h = (1/4, 1/8), c = (1, 3), rho = (1, 3).
#   hbar = 3/16, eps hbar^2 = 9/25600, r^2 + eps hbar^2 = 1609/25600,
#   hbar v.x = -3/128 = -600/25600, mu = -600/1609, cbar = 2, rhobar = 2
#   Pi = (2 * 600/1609 + 2 (600/1609)^2) / 2 = 1325400/2588881
PI_B = Fr(1325400, 2588881)


def test_viscosity_hand_value_equal_h(orc):
    f = _line([0.0, 0.25], [0.5, 0.0], h=[0.25, 0.25], m=[0.5, 0.25], rho=[1.0, 2.0], P=[0.0, 0.0],
              c=[1.0, 1.0])
    nb, (ax, ay, az, du, _, _) = _sums(orc, f)
    assert list(np.diff(nb.off)) == [1, 1]
    fbar = 0.5 * (orc.gradw_fac(0.25, 0.25) + orc.gradw_fac(0.25, 0.25))
    g = fbar * 0.25                  # grad_i Wbar_ij = -fbar x_ij = +fbar/4 along x
    Pi = float(PI_A)
    # P = 0: a_i = -m_j Pi grad_i Wbar, du_i = m_j (Pi/2) v_ij . grad_i Wbar (v_ij = 1/2)
    assert ax[0] == pytest.approx(-0.25 * Pi * g, rel=1e-14)
    assert ax[1] == pytest.approx(+0.5 * Pi * g, rel=1e-14)
    assert du[0] == pytest.approx(0.25 * 0.5 * Pi * 0.5 * g, rel=1e-14)
    assert du[1] == pytest.approx(0.5 * 0.5 * Pi * 0.5 * g, rel=1e-14)
    assert np.all(ay == 0) and np.all(az == 0)


def test_viscosity_hand_value_unequal_means(orc):
    f = _line([0.0, 0.25], [0.5, 0.0], h=[0.25, 0.125], m=[0.5, 0.25], rho=[1.0, 3.0], P=[0.0, 0.0],
              c=[1.0, 3.0])
    nb, (ax, _, _, du, _, _) = _sums(orc, f)
    assert list(np.diff(nb.off)) == [1, 1]          # r = 2 h_j: only i's support holds the pair
    fbar = 0.5 * (orc.gradw_fac(0.25, 0.25) + orc.gradw_fac(0.25, 0.125))
    assert orc.gradw_fac(0.25, 0.125) == 0.0
    g = fbar * 0.25
    Pi = float(PI_B)
    assert ax[0] == pytest.approx(-0.25 * Pi * g, rel=1e-14)
    assert ax[1] == pytest.approx(+0.5 * Pi * g, rel=1e-14)
    assert du[0] == pytest.approx(0.25 * 0.5 * Pi * 0.5 * g, rel=1e-14)
    assert du[1] == pytest.approx(0.5 * 0.5 * Pi * 0.5 * g, rel=1e-14)
    # the plausible slips give other numbers (all differ from PI_B by > 1 %)
    hb, vr, r2, eps = Fr(3, 16), Fr(-1, 8), Fr(1, 16), Fr(1, 100)

    def pi_of(h, c, rho, epsterm):
        mu = h * vr / (r2 + epsterm)
        return (-1 * c * mu + 2 * mu * mu) / rho

    slips = {"eps hbar": pi_of(hb, 2, 2, eps * hb), "h_i": pi_of(Fr(1, 4), 2, 2, eps * Fr(1, 16)),
             "rho_i": pi_of(hb, 2, 1, eps * hb * hb), "max c": pi_of(hb, 3, 2, eps * hb * hb)}
    assert pi_of(hb, 2, 2, eps * hb * hb) == PI_B
    for k, v in slips.items():
        assert abs(float(v) / float(PI_B) - 1) > 0.01, k


def test_viscosity_with_pressure_terms(orc):
    # case B with pressure: A = P/rho^2 = (1/2, 1); a_i = -m_j (A_i + A_j + Pi) grad,
    # du_i = m_j (A_i + Pi/2) v_ij . grad; j sees A_j in its du
    f = _line([0.0, 0.25], [0.5, 0.0], h=[0.25, 0.125], m=[0.5, 0.25], rho=[1.0, 3.0], P=[0.5, 9.0],
              c=[1.0, 3.0])
    _, (ax, _, _, du, _, _) = _sums(orc, f)
    g = 0.5 * orc.gradw_fac(0.25, 0.25) * 0.25
    Pi = float(PI_B)
    assert ax[0] == pytest.approx(-0.25 * (1.5 + Pi) * g, rel=1e-14)
    assert ax[1] == pytest.approx(+0.5 * (1.5 + Pi) * g, rel=1e-14)
    assert du[0] == pytest.approx(0.25 * (0.5 + Pi / 2) * 0.5 * g, rel=1e-14)
    assert du[1] == pytest.approx(0.5 * (1.0 + Pi / 2) * 0.5 * g, rel=1e-14)


def test_viscosity_off_for_receding_and_grazing_pairs(orc):
    # v_ij . x_ij > 0 (receding) and == 0 (tie, R5: no viscosity): with P = 0 nothing acts
    for vx in ([-0.5, 0.0], [0.0, 0.0]):
        f = _line([0.0, 0.25], vx, h=[0.25, 0.125], m=[0.5, 0.25], rho=[1.0, 3.0], P=[0.0, 0.0],
                  c=[1.0, 3.0])
        _, (ax, _, _, du, _, _) = _sums(orc, f)
        assert np.all(ax == 0) and np.all(du == 0)
    # transverse relative velocity: v_ij . x_ij = 0 exactly
    f = _line([0.0, 0.25], [0.0, 0.0], h=[0.25, 0.125], m=[0.5, 0.25], rho=[1.0, 3.0], P=[0.0, 0.0],
              c=[1.0, 3.0])
    f["vy"] = np.array([0.5, 0.0])
    _, (ax, _, _, du, _, _) = _sums(orc, f)
    assert np.all(ax == 0) and np.all(du == 0)


def test_viscosity_three_particles_sum_over_neighbours(orc):
    # x = 0, 1/4, 1/2 with v = 1/2, 0, -1/2, h = 1/4: pairs (0,1) and (1,2) approach
    # with the case-A geometry; (0,2) sits at r = 2h exactly and is no pair (strict <).
    # Equal rho = 3/2 and c = 1 give mu = -50/101 and Pi = 10050/10201 / (3/2) = PI_A
    # for both pairs.  The middle particle is pushed from both sides, by
    # m_0 Pi g towards +x and m_2 Pi g towards -x, and is heated by both.
    f = _line([0.0, 0.25, 0.5], [0.5, 0.0, -0.5], h=[0.25] * 3, m=[0.5, 0.25, 0.125], rho=[1.5] * 3,
              P=[0.0] * 3, c=[1.0] * 3)
    nb, (ax, _, _, du, _, _) = _sums(orc, f)
    assert list(np.diff(nb.off)) == [1, 2, 1]
    g = orc.gradw_fac(0.25, 0.25) * 0.25
    Pi = float(PI_A)
    assert ax[0] == pytest.approx(-0.25 * Pi * g, rel=1e-14)
    assert ax[2] == pytest.approx(+0.25 * Pi * g, rel=1e-14)
    assert ax[1] == pytest.approx((0.5 - 0.125) * Pi * g, rel=1e-14)
    # du_1 = m_0 (Pi/2)(v_10 . grad_1 Wbar_10) + m_2 (Pi/2)(v_12 . grad_1 Wbar_12), each v.grad = g/2
    assert du[1] == pytest.approx((0.5 + 0.125) * 0.5 * Pi * 0.5 * g, rel=1e-14)
    assert du[0] == pytest.approx(0.25 * 0.5 * Pi * 0.5 * g, rel=1e-14)
    assert du[2] == pytest.approx(0.25 * 0.5 * Pi * 0.5 * g, rel=1e-14)


# ------------------------------ energy sums ------------------------------------

@pytest.mark.parametrize("n,omega", [(10, 5.0), (17, 3.0), (24, 7.5)])
def test_patch_energy_and_lz_closed_forms(orc, n, omega):
    f = inputs.square_patch(n, omega)
    M, Px, Py, Pz, Lz, Ek, Ei = orc.conserved(f["x"], f["y"], f["vx"], f["vy"], f["vz"], f["m"], f["u"])
    assert M == pytest.approx(1.0, rel=1e-15)
    assert Ek == pytest.approx(omega ** 2 * (n * n - 1) / (12.0 * n * n), rel=1e-13)
    assert Lz == pytest.approx(-omega * (n * n - 1) / (6.0 * n * n), rel=1e-13)
    for p in (Px, Py, Pz):
        assert abs(p) < 1e-14 * omega


def test_energy_sums_carry_the_mass(orc):
    # masses k / S (k = 1..N, S = N(N+1)/2, so M = 1), uniform u = 3 and v = (3/4, -1/2, 1/4):
    # E_int = 3 M = 3, P = M v, E_kin = M |v|^2 / 2 = 7/16 (a dropped m gives N x these)
    N = 1000
    k = np.arange(1, N + 1, dtype=float)
    m = k / (N * (N + 1) / 2)
    rng = np.random.default_rng(5)
    x, y = rng.uniform(-1, 1, N), rng.uniform(-1, 1, N)
    out = orc.conserved(x, y, np.full(N, 0.75), np.full(N, -0.5), np.full(N, 0.25), m, np.full(N, 3.0))
    assert out[0] == pytest.approx(1.0, rel=1e-14)
    assert out[1:4] == pytest.approx([0.75, -0.5, 0.25], rel=1e-14)
    assert out[5] == pytest.approx(7.0 / 16.0, rel=1e-14)
    assert out[6] == pytest.approx(3.0, rel=1e-14)
    # u_i = 1 / m_i: E_int = N exactly; v_i = 1/sqrt(m_i) along x: E_kin = N/2
    out = orc.conserved(x, y, 1.0 / np.sqrt(m), np.zeros(N), np.zeros(N), m, 1.0 / m)
    assert out[6] == pytest.approx(float(N), rel=1e-13)
    assert out[5] == pytest.approx(N / 2.0, rel=1e-13)


def _synchronised_energy(orc, f, dt, nsteps):
    """E_kin + E_int at t = nsteps dt: x, u after nsteps steps; v_n from the
    next step as v_{n+1/2} - a_n dt/2 (constant dt)."""
    s = orc.Sim(f, dt_fixed=dt, adapt_h=False, av_alpha=0.0, av_beta=0.0, use_grid=0)
    s.step(nsteps)
    u = s["u"].copy()
    s.step(1)
    vx = s["vx"] - 0.5 * dt * s["ax"]
    vy = s["vy"] - 0.5 * dt * s["ay"]
    vz = s["vz"] - 0.5 * dt * s["az"]
    m = s["m"]
    return float(np.sum(0.5 * m * (vx * vx + vy * vy + vz * vz)) + np.sum(m * u))


def test_total_energy_drift_is_second_order(orc):
    f = inputs.random_cloud(300, seed=4, vscale=0.5, h_lo=0.15, h_hi=0.2)
    T = 0.04
    E0 = float(np.sum(0.5 * f["m"] * (f["vx"] ** 2 + f["vy"] ** 2 + f["vz"] ** 2)) + np.sum(f["m"] * f["u"]))
    drift = []
    for k in (8, 16, 32, 64):
        drift.append(abs(_synchronised_energy(orc, f, T / k, k) - E0))
    ratios = [drift[i] / drift[i + 1] for i in range(3)]
    # each halving of dt divides the drift by about 4 (first order would give 2;
    # measured 4.25, 4.13, 4.07).  Viscosity off: its on/off switch at
    # v_ij . x_ij = 0 makes the drift converge irregularly at these step sizes.
    for r in ratios:
        assert 3.6 < r < 4.6, (drift, ratios)
    assert drift[-1] > 1e3 * np.finfo(float).eps * E0     # above rounding: the test can see the order
