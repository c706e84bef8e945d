"""CUDA path against the FP64 oracle on small seeded inputs (every call goes
through the C ABI).  Neighbour lists and counts must be bit-exact; the FP64
path must match within 1e-12 and the mixed path within 1e-5 (relative,
normwise; du and viscous terms relative to the sum of term magnitudes)."""
import numpy as np
import pytest

from paper_1905_03344_gb300 import inputs
from gpu_common import conserved_errors, conserved_scales, lists_to_original, normwise, normwise_vec, scaled

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1905_03344_gb300 import binding, build
    build.build()
    binding.lib()
    return binding


def near_ties(n=600, seed=5, k=3):
    rng = np.random.default_rng(seed)
    base = rng.uniform(-0.4, 0.4, (n, 3))
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    r = 0.06 * (1.0 + rng.integers(-k, k + 1, n) * 2.0 ** -52)
    P = np.vstack([base, base + d * r[:, None]])
    N = 2 * n
    return {"x": P[:, 0].copy(), "y": P[:, 1].copy(), "z": P[:, 2].copy(),
            "vx": np.zeros(N), "vy": np.zeros(N), "vz": np.zeros(N),
            "m": np.full(N, 1.0 / N), "h": np.full(N, 0.03), "u": np.ones(N)}


def h_tail(n, seed, h0, tails, lz=1.0):
    """Random cloud with most h = h0 and a few larger: tails is a list of
    (fraction, h_lo, h_hi).  The largest h set apart as big particles, with
    search reaches across many fine cells and, for long reaches, across the
    whole z period.  h0 gives about 30 neighbours: with only a handful, rows
    made of pairs near the edge of a kernel support (q = 1 - r/2h close to
    0, where FP32 loses relative accuracy) would dominate the mixed-path
    error of isolated particles."""
    f = inputs.random_cloud(n, seed=seed, h_lo=h0, h_hi=h0 * 1.1, lz=lz)
    rng = np.random.default_rng(seed + 100)
    idx = rng.permutation(n)
    k0 = 0
    for frac, lo, hi in tails:
        k = int(round(frac * n))
        f["h"][idx[k0:k0 + k]] = rng.uniform(lo, hi, k)
        k0 += k
    f["lz"] = lz
    return f


CASES = {
    "patch20": lambda: inputs.square_patch(20),
    "htail_far": lambda: h_tail(3000, 41, 0.09, [(0.01, 0.3, 0.45), (0.04, 0.12, 0.16)]),
    "htail_near": lambda: h_tail(12000, 42, 0.08, [(0.01, 0.17, 0.2), (0.03, 0.1, 0.12)], lz=3.0),
    "cloud": lambda: inputs.random_cloud(3000, seed=1),
    "hspread": lambda: inputs.random_cloud(2500, seed=2, h_lo=0.01, h_hi=0.15),
    "irregular": lambda: inputs.irregular_patch(16, seed_pos=3, seed_mass=4),
    "zwrap": lambda: inputs.random_cloud(900, seed=3, h_lo=0.12, h_hi=0.3),
    "ties": near_ties,
}


def cap_pairs(n):
    return int(min(n * n, 400 * n) + 16)


def run_lists(B, f, **kw):
    n = len(f["x"])
    kw.setdefault("lz", f.pop("lz", 1.0))
    sim = B.SPH(max(n, 1), max_pairs=cap_pairs(n), **kw)
    sim.set_particles(f)
    sim.find_neighbors()
    off, col, perm = sim.neighbors()
    nown = sim.field("nown")
    nnb = sim.field("nnb")
    sim.close()
    o, c = lists_to_original(off, col, perm, n)
    return o, c, nown, nnb


@pytest.mark.parametrize("case", sorted(CASES))
def test_neighbor_lists_bit_exact(B, orc, case):
    f = CASES[case]()
    lz = f.pop("lz", 1.0)
    ref = orc.neighbors(f["x"], f["y"], f["z"], f["h"], lz)
    o, c, nown, nnb = run_lists(B, f, lz=lz)
    assert np.array_equal(o, ref.off)
    assert np.array_equal(c, ref.col)
    assert np.array_equal(nown.astype(np.int64), ref.nown.astype(np.int64))
    assert np.array_equal(nnb.astype(np.int64), np.diff(ref.off))


@pytest.mark.parametrize("tpp", [1, 2, 4, 8, 16, 32])
@pytest.mark.parametrize("cf", [1.0 / 3.0, 0.4, 0.5, 0.75, 1.0, 2.5])
def test_neighbor_lists_any_launch_shape(B, orc, tpp, cf):
    f = inputs.random_cloud(1500, seed=11, h_lo=0.02, h_hi=0.1)
    ref = orc.neighbors(f["x"], f["y"], f["z"], f["h"])
    o, c, nown, _ = run_lists(B, f, threads_per_particle=tpp, cell_factor=cf)
    assert np.array_equal(o, ref.off) and np.array_equal(c, ref.col)
    assert np.array_equal(nown.astype(np.int64), ref.nown.astype(np.int64))


def _oracle_forces(orc, f, lz=1.0):
    nb = orc.neighbors(f["x"], f["y"], f["z"], f["h"], lz)
    rho = orc.density(f["x"], f["y"], f["z"], f["m"], f["h"], nb, lz)
    P, c = orc.eos(rho, f["u"])
    ax, ay, az, du, sa, sdu = orc.momentum_energy(f["x"], f["y"], f["z"], f["vx"], f["vy"], f["vz"],
                                                  f["m"], f["h"], rho, P, c, nb, lz)
    return dict(rho=rho, P=P, c=c, ax=ax, ay=ay, az=az, du=du, sa=sa, sdu=sdu)


def _gpu_forces(B, f, precision, **kw):
    kw.setdefault("lz", 1.0)
    sim = B.SPH(len(f["x"]), precision=precision, max_pairs=cap_pairs(len(f["x"])), **kw)
    sim.set_particles(f)
    sim.find_neighbors()
    sim.density()
    sim.momentum_energy()
    out = {k: sim.field(k) for k in ("rho", "P", "c", "ax", "ay", "az", "du")}
    sim.close()
    return out


FORCE_CASES = {
    "patch20": lambda: inputs.square_patch(20),
    "htail_far": lambda: h_tail(3000, 43, 0.09, [(0.01, 0.3, 0.45), (0.04, 0.12, 0.16)]),
    "htail_near": lambda: h_tail(12000, 44, 0.08, [(0.01, 0.17, 0.2), (0.03, 0.1, 0.12)], lz=3.0),
    "cloud_av": lambda: inputs.random_cloud(3000, seed=21, vscale=3.0),
    "irregular": lambda: inputs.irregular_patch(16, seed_pos=6, seed_mass=7),
    "zwrap": lambda: inputs.random_cloud(900, seed=8, h_lo=0.12, h_hi=0.3, vscale=2.0),
}


def _check_forces(g, o, tol, report, tag):
    errs = {k: normwise(g[k], o[k]) for k in ("rho", "P", "c")}
    errs["a"] = normwise_vec([g["ax"], g["ay"], g["az"]], [o["ax"], o["ay"], o["az"]])
    for k in ("ax", "ay", "az"):
        errs[k + "/sa"] = scaled(g[k], o[k], o["sa"])
    errs["du/sdu"] = scaled(g["du"], o["du"], o["sdu"])
    errs["rho_median_rel"] = float(np.median(np.abs(g["rho"] - o["rho"]) / np.abs(o["rho"])))
    report[tag] = errs
    for k, v in errs.items():
        if k != "rho_median_rel":
            assert v < tol, (k, v)


@pytest.mark.parametrize("case", sorted(FORCE_CASES))
def test_fp64_pair_sums(B, orc, case, report):
    f = FORCE_CASES[case]()
    lz = f.pop("lz", 1.0)
    _check_forces(_gpu_forces(B, f, "fp64", lz=lz), _oracle_forces(orc, f, lz), 1e-12, report, "fp64/" + case)


@pytest.mark.parametrize("case", sorted(FORCE_CASES))
@pytest.mark.parametrize("tpp", [1, 2, 4, 8, 32])
def test_mixed_pair_sums(B, orc, case, tpp, report):
    f = FORCE_CASES[case]()
    lz = f.pop("lz", 1.0)
    _check_forces(_gpu_forces(B, f, "mixed", threads_per_particle=tpp, lz=lz), _oracle_forces(orc, f, lz), 1e-5,
                  report, "mixed/%s/tpp%d" % (case, tpp))


@pytest.mark.parametrize("case", sorted(FORCE_CASES))
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
@pytest.mark.parametrize("words", [8, 64])
def test_binned_pair_sums(B, orc, case, precision, tol, words, report):
    """Row-length bins: each octave of row lengths summed with its own lanes
    per particle, against the oracle."""
    f = FORCE_CASES[case]()
    lz = f.pop("lz", 1.0)
    _check_forces(_gpu_forces(B, f, precision, pair_bins=words, lz=lz), _oracle_forces(orc, f, lz), tol,
                  report, "bins%d/%s/%s" % (words, precision, case))


def _octave_tpp(c, words):
    """Lanes per particle of a row of c words with a target of `words` per lane."""
    return min(32, max(1, 1 << int(np.ceil(np.log2(max(c, 1) / words))))) if c > words else 1


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_binned_sums_are_the_uniform_sums_of_each_octave(B, orc, precision):
    """A particle's binned density sum is, bit for bit, that of a uniform
    launch with its octave's lanes per particle: the bins change which lanes
    sum a row, never the row.  (The momentum sum reads its neighbours'
    densities, which differ between such runs; it is checked against the
    oracle above.)  In this cloud h grows by e^2 from one side to the other,
    so rows run from 0 to ~190 words and, with 8 words per lane, every
    lanes-per-particle value 1..32 occurs."""
    f = inputs.random_cloud(3000, seed=2)
    f["h"] = 0.02 * np.exp(2.0 * (f["x"] + 0.5))
    rows = np.diff(orc.neighbors(f["x"], f["y"], f["z"], f["h"]).off)
    want = np.array([_octave_tpp(int(c), 8) for c in rows])
    assert set(want) == {1, 2, 4, 8, 16, 32}
    keys = ("rho", "P", "c")
    binned = _gpu_forces(B, dict(f), precision, pair_bins=8)
    uni = {t: _gpu_forces(B, dict(f), precision, threads_per_particle=t, pair_bins=-1) for t in (1, 2, 4, 8, 16, 32)}
    for k in keys:
        pick = np.choose(np.log2(want).astype(int), [uni[t][k] for t in (1, 2, 4, 8, 16, 32)])
        assert np.array_equal(binned[k].view(np.uint64), pick.view(np.uint64)), k


@pytest.mark.parametrize("case", sorted(FORCE_CASES))
def test_mixed_pair_sums_small_cells(B, orc, case, report):
    """Cells of a third of 2 h_s: neighbours three cells away carry the far
    column code and take their offsets from the cell coordinates."""
    f = FORCE_CASES[case]()
    lz = f.pop("lz", 1.0)
    _check_forces(_gpu_forces(B, f, "mixed", threads_per_particle=4, cell_factor=1.0 / 3.0, lz=lz),
                  _oracle_forces(orc, f, lz), 1e-5, report, "mixed/%s/cf1_3" % case)


@pytest.mark.parametrize("case", sorted(FORCE_CASES))
def test_step_density_matches(B, orc, case, report):
    """The timestep's density and EOS against the oracle's first step, at the
    pair-sum tolerance: the inputs of the first step are the same on both
    sides."""
    f = FORCE_CASES[case]()
    lz = f.pop("lz", 1.0)
    n = len(f["x"])
    sim = B.SPH(n, precision="mixed", max_pairs=cap_pairs(n), lz=lz)
    sim.set_particles(f)
    sim.step(1)
    g = {k: sim.field(k) for k in ("rho", "P", "c", "nown")}
    sim.close()
    ref = orc.Sim(f, lz=lz)
    ref.step(1)
    errs = {k: normwise(g[k], ref[k]) for k in ("rho", "P", "c")}
    report["stepdensity/%s" % case] = errs
    assert np.array_equal(g["nown"], ref["nown"])
    for k, v in errs.items():
        assert v < 1e-5, (k, v)


@pytest.mark.parametrize("case", ["patch20", "cloud_av", "irregular", "htail_near"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
def test_sinc_kernel_pair_sums(B, orc, case, precision, tol, report):
    """The Sinc kernel of Sec. 3 (n = 6) in the density and momentum sums."""
    f = FORCE_CASES[case]()
    lz = f.pop("lz", 1.0)
    g = _gpu_forces(B, f, precision, lz=lz, kernel="sinc", kernel_n=6)
    with orc.kernel("sinc", 6):
        o = _oracle_forces(orc, f, lz)
    _check_forces(g, o, tol, report, "sinc/%s/%s" % (precision, case))


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
def test_sinc_kernel_ten_steps(B, orc, precision, tol, report):
    f = inputs.square_patch(20)
    sim = B.SPH(len(f["x"]), precision=precision, kernel="sinc", kernel_n=6)
    sim.set_particles(f)
    ref = orc.Sim(f, kernel="sinc", kernel_n=6)
    hist = []
    for step in range(10):
        dt = sim.step(1)
        ref.step(1)
        assert abs(dt - ref.dt) <= tol * ref.dt, (step, dt, ref.dt)
        g = {k: sim.field(k) for k in ("x", "y", "z", "vx", "vy", "vz", "u", "h", "nown", "rho",
                                       "ax", "ay", "az")}
        hist.append(_compare_state(g, ref, tol, "sinc step %d" % step))
    report["sinc_steps10/%s" % precision] = hist
    sim.close()


def _oracle_forces_gradh(orc, f, lz=1.0):
    nb = orc.neighbors(f["x"], f["y"], f["z"], f["h"], lz)
    rho = orc.density(f["x"], f["y"], f["z"], f["m"], f["h"], nb, lz)
    P, c = orc.eos(rho, f["u"])
    om = orc.omega(f["x"], f["y"], f["z"], f["m"], f["h"], rho, nb, lz)
    ax, ay, az, du, sa, sdu = orc.momentum_energy(f["x"], f["y"], f["z"], f["vx"], f["vy"], f["vz"],
                                                  f["m"], f["h"], rho, P, c, nb, lz, omega=om)
    return dict(rho=rho, P=P, c=c, ax=ax, ay=ay, az=az, du=du, sa=sa, sdu=sdu), om


# The oracle takes Omega = 1 + h/(3 rho) sum m dW/dh as written: a sum near
# -1 added to 1, so its own rounding error in Omega is a few ulp of 1, i.e.
# relative few eps / Omega.  The GPU path sums the non-negative terms of the
# same quantity (no cancellation).  Where the inputs make Omega small (the
# random cloud with h drawn apart from the density: Omega down to 1.5e-6 for
# the Sinc kernel) the comparison allows for the oracle's error.
ORACLE_OMEGA_ULPS = 64


@pytest.mark.parametrize("kernel", ["wendland", "sinc"])
@pytest.mark.parametrize("case", ["patch20", "cloud_av", "irregular", "htail_near", "zwrap"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
def test_grad_h_pair_sums(B, orc, kernel, case, precision, tol, report):
    """The grad-h momentum and energy form (Omega from the dW/dh sum over the
    same neighbours as the density) against the oracle's."""
    f = FORCE_CASES[case]()
    lz = f.pop("lz", 1.0)
    g = _gpu_forces(B, f, precision, lz=lz, kernel=kernel, kernel_n=6, grad_h=1)
    with orc.kernel(kernel, 6):
        o, om = _oracle_forces_gradh(orc, f, lz)
    assert om.min() > 0.0
    tol_eff = tol + ORACLE_OMEGA_ULPS * np.finfo(np.float64).eps / om.min()
    _check_forces(g, o, tol_eff, report, "gradh/%s/%s/%s" % (kernel, precision, case))
    report["gradh/%s/%s/%s" % (kernel, precision, case)]["omega_min"] = float(om.min())


@pytest.mark.parametrize("kernel", ["wendland", "sinc"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
def test_grad_h_ten_steps(B, orc, kernel, precision, tol, report):
    f = inputs.square_patch(20)
    sim = B.SPH(len(f["x"]), precision=precision, kernel=kernel, kernel_n=6, grad_h=1)
    sim.set_particles(f)
    ref = orc.Sim(f, kernel=kernel, kernel_n=6, grad_h=True)
    hist = []
    for step in range(10):
        dt = sim.step(1)
        ref.step(1)
        assert abs(dt - ref.dt) <= tol * ref.dt, (step, dt, ref.dt)
        g = {k: sim.field(k) for k in ("x", "y", "z", "vx", "vy", "vz", "u", "h", "nown", "rho",
                                       "ax", "ay", "az")}
        hist.append(_compare_state(g, ref, tol, "grad-h step %d" % step))
    report["gradh_steps10/%s/%s" % (kernel, precision)] = hist
    sim.close()


def _compare_state(g, o, tol, what):
    errs = {k: normwise(g[k], o[k]) for k in ("x", "y", "u", "h", "rho")}
    errs["v"] = normwise_vec([g["vx"], g["vy"], g["vz"]], [o["vx"], o["vy"], o["vz"]])
    errs["a"] = normwise_vec([g["ax"], g["ay"], g["az"]], [o["ax"], o["ay"], o["az"]])
    dz = g["z"] - o["z"]
    dz -= np.round(dz)
    errs["z"] = float(np.abs(dz).max() / np.abs(o["z"]).max())
    for k, v in errs.items():
        assert v < tol, (what, k, v)
    return errs


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
def test_square_patch_ten_steps(B, orc, precision, tol, report):
    f = inputs.square_patch(20)
    sim = B.SPH(len(f["x"]), precision=precision)
    sim.set_particles(f)
    ref = orc.Sim(f)
    hist = []
    for step in range(10):
        dt = sim.step(1)
        ref.step(1)
        assert abs(dt - ref.dt) <= tol * ref.dt, (step, dt, ref.dt)
        g = {k: sim.field(k) for k in ("x", "y", "z", "vx", "vy", "vz", "u", "h", "nown", "rho",
                                       "ax", "ay", "az")}
        e = _compare_state(g, ref, tol, "step %d" % step)
        e["dt"] = abs(dt - ref.dt) / ref.dt
        # all 7 conserved sums of the step's state against the oracle's
        ce = conserved_errors(sim.conserved(), ref.conserved(),
                              conserved_scales(*[ref[k] for k in ("x", "y", "vx", "vy", "vz", "m", "u")]))
        for k, v in ce.items():
            assert v < tol, (step, k, v)
        e.update({"cons_" + k: v for k, v in ce.items()})
        hist.append(e)
    report["steps10/%s" % precision] = hist
    sim.close()


def test_rows_outgrowing_their_reservation(B, orc, report):
    """h grows fast (n_target far above the initial counts), so many rows
    outgrow the space reserved from the previous step's row lengths and are
    searched again into a second reservation; the trajectory must not notice."""
    f = inputs.random_cloud(2000, seed=31, h_lo=0.07, h_hi=0.09, vscale=0.5)
    n = len(f["x"])
    kw = dict(n_target=150.0)
    ref = orc.Sim(f, **kw)
    counts = []
    for step in range(3):
        nb = orc.neighbors(ref["x"], ref["y"], ref["z"], ref["h"], 1.0)
        counts.append(np.diff(nb.off).astype(np.int64))
        ref.step(1)
    # precondition, from the oracle alone: some rows exceed c + c/3 + 8
    c0, c1 = counts[0], counts[1]
    assert np.sum(c1 > ((c0 + c0 // 3 + 8 + 7) // 8) * 8) > n // 20
    sim = B.SPH(n, precision="fp64", max_pairs=cap_pairs(n), **kw)
    sim.set_particles(f)
    sim.step(3)
    g = {k: sim.field(k) for k in ("x", "y", "z", "vx", "vy", "vz", "u", "h", "nown", "rho", "ax", "ay", "az")}
    sim.close()
    assert np.array_equal(g["nown"], ref["nown"])
    report["outgrow/fp64"] = _compare_state(g, ref, 1e-12, "outgrow")


def test_batched_patches_match_single(B, orc):
    rng = np.random.default_rng(3)
    edges = [6, 9, 7, 11]
    omegas = rng.uniform(2, 8, len(edges))
    parts = [inputs.square_patch(e, w) for e, w in zip(edges, omegas)]
    f = {k: np.concatenate([p[k] for p in parts]) for k in parts[0]}
    offs = np.concatenate([[0], np.cumsum([e ** 3 for e in edges])])
    sim = B.SPH(len(f["x"]), precision="fp64", max_patches=len(edges))
    sim.set_particles(f)
    sim.set_patches(offs)
    refs = [orc.Sim(p) for p in parts]
    for step in range(4):
        sim.step(1)
        for r in refs:
            r.step(1)
        x = sim.field("x")
        u = sim.field("u")
        for p, r in enumerate(refs):
            sl = slice(offs[p], offs[p + 1])
            assert normwise(x[sl], r["x"]) < 1e-12
            assert normwise(u[sl], r["u"]) < 1e-12
            dt, _, nst = sim.dt(p)
            assert dt == pytest.approx(r.dt, rel=1e-12) and nst == step + 1
        vx, vy, vz, y, m = (sim.field(k) for k in ("vx", "vy", "vz", "y", "m"))
        for p, r in enumerate(refs):
            ce = conserved_errors(sim.conserved(p), r.conserved(),
                                  conserved_scales(*[r[k] for k in ("x", "y", "vx", "vy", "vz", "m", "u")]))
            for k, v in ce.items():
                assert v < 1e-12, (step, p, k, v)
        # all patches at once: the sums over the whole particle set
        ce = conserved_errors(sim.conserved(-1), sum(r.conserved() for r in refs),
                              conserved_scales(x, y, vx, vy, vz, m, u))
        for k, v in ce.items():
            assert v < 1e-12, (step, "all", k, v)
    sim.close()


@pytest.mark.parametrize("precision,tol_p,tol_l", [("fp64", 1e-12, 1e-12), ("mixed", 2e-6, 1e-7)])
def test_long_run_momentum_and_lz(B, precision, tol_p, tol_l, report):
    """200 steps of the 40^3 patch on the GPU alone: every pair force is
    central and enters both particles with opposite signs, so the total
    momentum (zero by the lattice's symmetry) and L_z stay at their initial
    values to rounding through the leapfrog (P = sum m v_{n+1/2}, L_z likewise).  In FP64
    that rounding is ~1e-16.  The mixed path evaluates each pair term as the
    exact negative of its mirror (equal masses; the kernel factor is
    symmetric in i and j, and a separation across the periodic z boundary
    takes the negated cell shift from both sides) but sums each particle's
    row in FP32 (four terms plainly, then a Kahan step).  Along the periodic,
    gradient-free z axis of the lattice every particle sums nearly the same
    cancelling terms in the same order, so that rounding is the same for all
    of them and adds up to a net z force instead of averaging out: P_z drifts
    by 3e-7 of sum m |v| over the run (P_x, P_y ~1e-9, measured; 1e-5 when
    the wrapped separations were rounded differently from the two sides),
    while L_z keeps ~1e-8."""
    f = inputs.square_patch(40)
    sim = B.SPH(len(f["x"]), precision=precision)
    sim.set_particles(f)
    sim.step(1)
    c0 = sim.conserved()
    scale = float(np.sum(f["m"] * np.hypot(f["vx"], f["vy"])))
    sim.step(199)
    c = sim.conserved()
    sim.close()
    dp = max(abs(c[1]), abs(c[2]), abs(c[3])) / scale
    dl = abs(c[4] - c0[4]) / abs(c0[4])
    report["long200/%s" % precision] = dict(momentum=dp, lz=dl, p=[float(v) / scale for v in c[1:4]])
    assert c[0] == pytest.approx(c0[0], rel=1e-14)
    assert dp <= tol_p and dl <= tol_l, (dp, dl)
