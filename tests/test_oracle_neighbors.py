"""Pins of the oracle's neighbour sets (symmetric union, reading R11).

The grid search is checked against the O(N^2) definition; the definition is
checked against exact integer lattice counts, symmetry, periodic images and
exact ties.
"""
import math

import numpy as np
import pytest

from paper_1905_03344_gb300 import inputs


def _sets(nb):
    return [set(r.tolist()) for r in nb.rows()]


def _lattice_count(radius_over_dx):
    """#{k in Z^3 \\ 0 : |k|^2 < R^2}, exact in integers (R^2 compared as a float once)."""
    R = int(math.ceil(radius_over_dx)) + 1
    r2 = radius_over_dx ** 2
    c = 0
    for a in range(-R, R + 1):
        for b in range(-R, R + 1):
            for d in range(-R, R + 1):
                if (a, b, d) != (0, 0, 0) and a * a + b * b + d * d < r2:
                    c += 1
    return c


@pytest.mark.parametrize("kind", ["cloud", "lattice", "jitter", "hspread"])
def test_grid_equals_brute_force(orc, kind):
    if kind == "cloud":
        f = inputs.random_cloud(1500, seed=3)
    elif kind == "lattice":
        f = inputs.square_patch(11)
    elif kind == "jitter":
        f = inputs.irregular_patch(12, seed_pos=4, seed_mass=5)
    else:
        f = inputs.random_cloud(1200, seed=9, h_lo=0.01, h_hi=0.12)
    a = orc.neighbors(f["x"], f["y"], f["z"], f["h"], method="brute")
    b = orc.neighbors(f["x"], f["y"], f["z"], f["h"], method="grid")
    assert np.array_equal(a.off, b.off)
    assert np.array_equal(a.col, b.col)
    assert np.array_equal(a.nown, b.nown)


def test_symmetric_no_self(orc):
    f = inputs.random_cloud(800, seed=11, h_lo=0.02, h_hi=0.1)
    nb = orc.neighbors(f["x"], f["y"], f["z"], f["h"], method="brute")
    S = _sets(nb)
    for i, s in enumerate(S):
        assert i not in s
        for j in s:
            assert i in S[j]
    assert np.all(nb.nown <= np.diff(nb.off))


def test_interior_lattice_count_is_integer_point_count(orc):
    n = 16
    f = inputs.square_patch(n)
    nb = orc.neighbors(f["x"], f["y"], f["z"], f["h"], method="brute")
    expect = _lattice_count(2.0 * inputs.ETA)
    assert expect == 92
    interior = (np.abs(f["x"]) < 0.5 - 3.5 / n) & (np.abs(f["y"]) < 0.5 - 3.5 / n)
    assert interior.sum() > 0
    counts = np.diff(nb.off)
    assert np.all(counts[interior] == expect)
    assert np.all(nb.nown[interior] == expect)
    # z is periodic: counts do not depend on the layer, only on (x, y)
    c = counts.reshape(n, n * n)
    assert np.all(c == c[0])


def test_periodic_z_image(orc):
    h = 0.05
    pi = (0.0, 0.0, 0.49)
    pj = (0.0, 0.0, -0.49)        # 0.02 apart through the periodic boundary
    assert orc.pair_in(pi, pj, h, h, lz=1.0) == (True, True)
    assert orc.pair_in(pi, pj, h, h, lz=2.0) == (False, False)


def test_strict_inequality_and_union(orc):
    # r = 2 h_i exactly (all values exact in binary): not a neighbour by h_i
    assert orc.pair_in((0.0, 0, 0), (0.5, 0, 0), 0.25, 0.25) == (False, False)
    nxt = np.nextafter(0.5, 0.0)
    assert orc.pair_in((0.0, 0, 0), (nxt, 0, 0), 0.25, 0.25) == (True, True)
    # union: j reaches i through h_j only; then i is in N(j) by j's own radius
    assert orc.pair_in((0.0, 0, 0), (0.3, 0, 0), 0.1, 0.2) == (True, False)
    assert orc.pair_in((0.3, 0, 0), (0.0, 0, 0), 0.2, 0.1) == (True, True)


def test_near_ties(orc):
    # pairs placed at r = 2h (1 + k ulp) for small k: brute and grid must agree
    rng = np.random.default_rng(5)
    n = 400
    base = rng.uniform(-0.4, 0.4, (n, 3))
    h = np.full(2 * n, 0.03)
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    k = rng.integers(-3, 4, n)
    r = 0.06 * (1.0 + k * 2.0 ** -52)
    other = base + d * r[:, None]
    P = np.vstack([base, other])
    a = orc.neighbors(P[:, 0], P[:, 1], P[:, 2], h, method="brute")
    b = orc.neighbors(P[:, 0], P[:, 1], P[:, 2], h, method="grid")
    assert np.array_equal(a.off, b.off) and np.array_equal(a.col, b.col)
