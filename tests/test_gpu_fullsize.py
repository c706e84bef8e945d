"""The CUDA path at the benchmark's full sizes, in the launch shape the bench
times (the autotuned cell factor and threads per particle), against the FP64
oracle run on all host cores:

  - the 200^3 square patch (8,000,000 particles) and the 159^3 irregular
    patch (4,019,679 particles, neighbour counts spread over ~50-400):
    per-particle neighbour counts and n_i bit-exact for every particle, a
    seeded sample of 2000 rows bit-exact as sets, and density, pressure,
    sound speed, acceleration and du/dt of every particle within the mixed
    path's tolerance (1e-5, normwise and per particle against the sum of
    term magnitudes);
  - 64 independent patches advanced together (edges 10..60, omega 2..8):
    the same checks per patch, and one FP64 step per patch against the
    oracle's step of that patch (positions, h and the per-patch dt).
"""
import os

import numpy as np
import pytest

from paper_1905_03344_gb300 import inputs
from gpu_common import conserved_errors, conserved_scales, normwise, normwise_vec, scaled

pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 1
TOL_MIXED = 1e-5


@pytest.fixture(scope="module")
def B():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1905_03344_gb300 import binding, build
    build.build()
    binding.lib()
    return binding


def oracle_forces(orc, f, lz=1.0):
    nb = orc.neighbors(f["x"], f["y"], f["z"], f["h"], lz, nthreads=THREADS)
    rho = orc.density(f["x"], f["y"], f["z"], f["m"], f["h"], nb, lz, nthreads=THREADS)
    P, c = orc.eos(rho, f["u"])
    ax, ay, az, du, sa, sdu = orc.momentum_energy(f["x"], f["y"], f["z"], f["vx"], f["vy"], f["vz"],
                                                  f["m"], f["h"], rho, P, c, nb, lz, nthreads=THREADS)
    return nb, dict(rho=rho, P=P, c=c, ax=ax, ay=ay, az=az, du=du, sa=sa, sdu=sdu)


def force_errors(g, o):
    errs = {k: normwise(g[k], o[k]) for k in ("rho", "P", "c")}
    errs["a"] = normwise_vec([g["ax"], g["ay"], g["az"]], [o["ax"], o["ay"], o["az"]])
    for k in ("ax", "ay", "az"):
        errs[k + "/sa"] = scaled(g[k], o[k], o["sa"])
    errs["du/sdu"] = scaled(g["du"], o["du"], o["sdu"])
    return errs


def sampled_rows_match(B, sim, nb, n, count, seed):
    """count seeded rows of the GPU lists, as sets of original indices,
    against the oracle's rows (read on the device, only the sampled rows
    copied back)."""
    import torch
    off, col, perm = B.sph_copy_neighbors(sim.ctx, n, device="cuda")
    inv = torch.empty_like(perm)
    inv[perm.long()] = torch.arange(n, dtype=perm.dtype, device=perm.device)
    rng = np.random.default_rng(seed)
    picks = rng.choice(n, size=min(count, n), replace=False)
    ks = inv[torch.as_tensor(picks, device=perm.device).long()].long()
    offs = off.cpu().numpy()
    for p, k in zip(picks, ks.cpu().numpy()):
        row = perm[col[offs[k]:offs[k + 1]].long()].cpu().numpy().astype(np.int64)
        ref = nb.col[nb.off[p]:nb.off[p + 1]].astype(np.int64)
        if not np.array_equal(np.sort(row), ref):
            return p
    return None


def run_tuned(B, f, lz=1.0):
    n = len(f["x"])
    sim = B.SPH(n, precision="mixed", max_pairs=160 * n, lz=lz)
    sim.set_particles(f)
    sim.autotune()
    sim.set_particles(f)
    sim.find_neighbors()
    return sim


@pytest.mark.parametrize("name", ["c3", "c5"])
def test_full_size_patch(B, orc, name, report):
    f = inputs.config_patch(name)
    n = len(f["x"])
    sim = run_tuned(B, f)
    nown = sim.field("nown").astype(np.int64)
    nnb = sim.field("nnb").astype(np.int64)
    nb, o = oracle_forces(orc, f)
    assert np.array_equal(nnb, np.diff(nb.off))
    assert np.array_equal(nown, nb.nown.astype(np.int64))
    bad = sampled_rows_match(B, sim, nb, n, 2000, seed=7)
    assert bad is None, "row of particle %d differs" % bad
    sim.density()
    sim.momentum_energy()
    g = {k: sim.field(k) for k in ("rho", "P", "c", "ax", "ay", "az", "du")}
    tpp, cf = B.sph_get_tuning(sim.ctx)
    bins = sim.pair_bins()
    sim.close()
    errs = force_errors(g, o)
    report["fullsize/%s" % name] = dict(errs, tpp=tpp, cell_factor=cf, bins=bins, n=n, nnz=int(nb.off[-1]))
    for k, v in errs.items():
        assert v < TOL_MIXED, (name, k, v)
    if name == "c5":
        # row-length bins with 16 words per lane: the irregular patch's rows
        # (~50-400) fill the octaves of 4, 8, 16 and 32 lanes per particle
        rows = np.diff(nb.off)
        tpps = {min(32, max(1, 1 << int(np.ceil(np.log2(max(c, 1) / 16.0))))) for c in np.unique(rows)}
        assert {4, 8, 16, 32} <= tpps, sorted(tpps)
        sb = B.SPH(n, precision="mixed", max_pairs=160 * n, pair_bins=16)
        sb.set_particles(f)
        sb.find_neighbors()
        sb.density()
        sb.momentum_energy()
        gb = {k: sb.field(k) for k in ("rho", "P", "c", "ax", "ay", "az", "du")}
        assert sb.pair_bins() == (16, 16)
        sb.close()
        errs = force_errors(gb, o)
        report["fullsize/c5/bins16"] = errs
        for k, v in errs.items():
            assert v < TOL_MIXED, ("c5 bins", k, v)


def test_batched_64_patches(B, orc, report):
    f, offsets, edges, omegas = inputs.batch_patches(64, seed=0)
    n = len(f["x"])
    sim = B.SPH(n, precision="mixed", max_pairs=160 * n, max_patches=64)
    sim.set_particles(f)
    sim.set_patches(offsets)
    sim.find_neighbors()
    nnb = sim.field("nnb").astype(np.int64)
    nown = sim.field("nown").astype(np.int64)
    sim.density()
    sim.momentum_energy()
    g = {k: sim.field(k) for k in ("rho", "P", "c", "ax", "ay", "az", "du")}
    sim.close()
    worst = {}
    for p in range(64):
        a, b = int(offsets[p]), int(offsets[p + 1])
        part = {k: v[a:b] for k, v in f.items()}
        nb, o = oracle_forces(orc, part)
        assert np.array_equal(nnb[a:b], np.diff(nb.off)), p
        assert np.array_equal(nown[a:b], nb.nown.astype(np.int64)), p
        errs = force_errors({k: v[a:b] for k, v in g.items()}, o)
        for k, v in errs.items():
            worst[k] = max(worst.get(k, 0.0), v)
            assert v < TOL_MIXED, (p, k, v)
    report["fullsize/batched64"] = dict(worst, n=n)

    # one FP64 step: every patch takes its own dt
    s64 = B.SPH(n, precision="fp64", max_pairs=160 * n, max_patches=64)
    s64.set_particles(f)
    s64.set_patches(offsets)
    s64.step(1)
    x, hh = s64.field("x"), s64.field("h")
    dts = [s64.dt(p)[0] for p in range(64)]
    cons = [s64.conserved(p) for p in range(64)]
    s64.close()
    worst_c = 0.0
    for p in range(64):
        a, b = int(offsets[p]), int(offsets[p + 1])
        ref = orc.Sim({k: v[a:b] for k, v in f.items()}, nthreads=THREADS)
        ref.step(1)
        assert abs(dts[p] - ref.dt) <= 1e-12 * ref.dt, (p, dts[p], ref.dt)
        assert np.abs(x[a:b] - ref["x"]).max() <= 1e-12 * max(1.0, np.abs(ref["x"]).max()), p
        assert np.abs(hh[a:b] - ref["h"]).max() <= 1e-12 * np.abs(ref["h"]).max(), p
        # all 7 conserved sums of each patch after its own step
        ce = conserved_errors(cons[p], ref.conserved(),
                              conserved_scales(*[ref[k] for k in ("x", "y", "vx", "vy", "vz", "m", "u")]))
        for k, v in ce.items():
            assert v < 1e-12, (p, k, v)
        worst_c = max(worst_c, max(ce.values()))
    report["fullsize/batched64"]["conserved_fp64"] = worst_c


def test_full_size_fused_matches_lists(B):
    """The 200^3 patch in the list-free mode at the benchmark's cell factor:
    every force field, |N(i)| and n_i the same bits as the lists with one lane
    per particle."""
    f = inputs.config_patch("c3")
    n = len(f["x"])
    out = {}
    keys = ("rho", "P", "c", "ax", "ay", "az", "du", "nnb", "nown")
    for mode in ("fused", "lists"):
        sim = B.SPH(n, precision="mixed", max_pairs=160 * n, pair_mode=mode, threads_per_particle=1,
                    cell_factor=0.5)
        sim.set_particles(f)
        sim.find_neighbors()
        sim.density()
        sim.momentum_energy()
        out[mode] = {k: sim.field(k) for k in keys}
        sim.close()
    for k in keys:
        assert np.array_equal(out["fused"][k].view(np.uint64), out["lists"][k].view(np.uint64)), k
