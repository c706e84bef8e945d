"""Pins of the oracle's Wendland kernel (Sec. 3, Eq. 2) against closed forms.

Nothing here re-types the kernel formula: the checks are its normalisation
(a volume integral done by quadrature), the paper's printed sigma_W, the
vanishing at the support edge, and a finite difference of W for the gradient.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


def test_sigma_matches_paper(orc):
    assert orc.sigma_w() == pytest.approx(GOLD["sigma_w"]["value"], rel=1e-15)


@pytest.mark.parametrize("h", [1.0, 0.5, 0.071985, 0.0036])
def test_normalised_to_one(orc, h):
    # int W d^3r = 1: the 1/h^3 factor restored (reading R2) must make this hold for every h
    val, err = integrate.quad(lambda r: 4.0 * math.pi * r * r * orc.w(r, h), 0.0, 2.0 * h,
                              epsabs=0, epsrel=1e-13, limit=200)
    assert val == pytest.approx(1.0, abs=1e-11)


@pytest.mark.parametrize("h", [1.0, 0.3])
def test_center_value_and_support(orc, h):
    assert orc.w(0.0, h) == pytest.approx(GOLD["sigma_w"]["value"] / h ** 3, rel=1e-14)
    sup = GOLD["kernel_support_v"]["value"]
    assert orc.w(sup * h, h) == 0.0
    assert orc.w(1.5 * sup * h, h) == 0.0
    assert orc.gradw_fac(sup * h, h) == 0.0
    # smooth at the edge: W ~ (2 - v)^4 so W(2h - d) / d^4 stays bounded
    d = 1e-3 * h
    assert 0.0 < orc.w(sup * h - d, h) < 1e-9 / h ** 3


@pytest.mark.parametrize("h", [1.0, 0.07])
def test_gradient_is_derivative(orc, h):
    # grad_i W = -f (x_i - x_j) means dW/dr = -f r; compare with a central difference
    for v in np.linspace(0.05, 1.95, 25):
        r = v * h
        d = 1e-6 * h
        fd = (orc.w(r + d, h) - orc.w(r - d, h)) / (2 * d)
        an = -orc.gradw_fac(r, h) * r
        assert an == pytest.approx(fd, rel=1e-6, abs=1e-9 / h ** 4)


def test_monotone_positive(orc):
    vals = [orc.w(v, 1.0) for v in np.linspace(0, 1.999, 200)]
    assert all(a > b for a, b in zip(vals, vals[1:]))
    assert all(v > 0 for v in vals)


# ---- the Sinc family (Sec. 3): W_n = B_n / h^3 sinc^n(pi v / 2), 0 <= v <= 2 ----

def _sinc_n(x, n):
    # numpy's sinc is sin(pi t)/(pi t): sinc(x) = np.sinc(x / pi)
    return np.sinc(x / math.pi) ** n


@pytest.mark.parametrize("n", [3, 4, 5, 6, 7, 8])
def test_sinc_bn_normalises(orc, n):
    # the oracle's B_n comes from composite Simpson; an adaptive Gauss-Kronrod
    # quadrature of the same normalisation integral checks it
    val, _ = integrate.quad(lambda v: 4.0 * math.pi * v * v * _sinc_n(0.5 * math.pi * v, n), 0.0, 2.0,
                            epsabs=0, epsrel=1e-13, limit=200)
    assert orc.sinc_bn(n) * val == pytest.approx(1.0, abs=1e-12)


@pytest.mark.parametrize("h", [1.0, 0.05])
def test_sinc_kernel_integrates_to_one(orc, h):
    with orc.kernel("sinc", 6):
        val, _ = integrate.quad(lambda r: 4.0 * math.pi * r * r * orc.w(r, h), 0.0, 2.0 * h,
                                epsabs=0, epsrel=1e-13, limit=200)
        assert val == pytest.approx(1.0, abs=1e-11)
        # centre value: sinc(0) = 1
        assert orc.w(0.0, h) == pytest.approx(orc.sinc_bn(6) / h ** 3, rel=1e-14)
        assert orc.w(2.0 * h, h) == 0.0 and orc.gradw_fac(2.0 * h, h) == 0.0


@pytest.mark.parametrize("h", [1.0, 0.07])
def test_sinc_gradient_is_derivative(orc, h):
    with orc.kernel("sinc", 6):
        for v in np.linspace(0.02, 1.95, 30):
            r = v * h
            d = 1e-6 * h
            fd = (orc.w(r + d, h) - orc.w(r - d, h)) / (2 * d)
            an = -orc.gradw_fac(r, h) * r
            assert an == pytest.approx(fd, rel=1e-6, abs=1e-9 / h ** 4)


def test_sinc_gradient_at_the_origin(orc):
    # f = B_n n pi^2 / (4 h^5) sinc^(n-1)(x) (sin x - x cos x)/x^3 -> B_n n pi^2 / (12 h^5)
    # as x -> 0 (the series branch), and it joins the direct form continuously at x = 1
    h = 0.4
    with orc.kernel("sinc", 6):
        assert orc.gradw_fac(0.0, h) == pytest.approx(orc.sinc_bn(6) * 6 * math.pi ** 2 / (12 * h ** 5),
                                                      rel=1e-14)
        r1 = 2.0 * h / math.pi  # x = 1
        below, above = orc.gradw_fac(r1 * (1 - 1e-12), h), orc.gradw_fac(r1 * (1 + 1e-12), h)
        assert below == pytest.approx(above, rel=1e-10)


def test_sinc_lattice_density_near_rho0(orc):
    # on a unit-density lattice with the patch's h (~100 neighbours) the SPH
    # density of the normalised Sinc kernel is close to 1
    from paper_1905_03344_gb300 import inputs
    n = 16
    f = inputs.square_patch(n)
    with orc.kernel("sinc", 6):
        nb = orc.neighbors(f["x"], f["y"], f["z"], f["h"])
        rho = orc.density(f["x"], f["y"], f["z"], f["m"], f["h"], nb)
    interior = (np.abs(f["x"]) < 0.5 - 3.5 / n) & (np.abs(f["y"]) < 0.5 - 3.5 / n)
    assert abs(np.mean(rho[interior]) - 1.0) < 0.03
