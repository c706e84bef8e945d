"""The list-free pair sums (SPH_PAIRS_FUSED): the density and momentum passes
run the neighbour search themselves.

They take the lists' pairs in the lists' order and call the same per-pair
arithmetic, so with one lane per particle on the list side the two modes give
the same bits: every force field, |N(i)| and n_i, and (the update being
shared) whole trajectories.  They are also checked against the oracle.
"""
import numpy as np
import pytest

from paper_1905_03344_gb300 import inputs
from gpu_common import normwise
from test_gpu_parity import (FORCE_CASES, _check_forces, _compare_state, _oracle_forces, cap_pairs)

pytestmark = pytest.mark.gpu

FIELDS = ("rho", "P", "c", "ax", "ay", "az", "du", "nnb", "nown")


@pytest.fixture(scope="module")
def B():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1905_03344_gb300 import binding, build
    build.build()
    binding.lib()
    return binding


def _forces(B, f, mode, precision, **kw):
    n = len(f["x"])
    sim = B.SPH(n, precision=precision, max_pairs=cap_pairs(n), pair_mode=mode, **kw)
    sim.set_particles(f)
    sim.find_neighbors()
    sim.density()
    sim.momentum_energy()
    assert sim.pair_mode() == mode
    out = {k: sim.field(k) for k in FIELDS}
    sim.close()
    return out


def _same_bits(g, h, what):
    for k in FIELDS:
        assert np.array_equal(g[k].view(np.uint64), h[k].view(np.uint64)), (what, k)


@pytest.mark.parametrize("case", sorted(FORCE_CASES))
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("cf", [1.0 / 3.0, 0.4, 0.5, 1.0])
def test_fused_equals_lists(B, case, precision, cf):
    f = FORCE_CASES[case]()
    lz = f.pop("lz", 1.0)
    kw = dict(lz=lz, cell_factor=cf, threads_per_particle=1)
    _same_bits(_forces(B, f, "fused", precision, **kw), _forces(B, f, "lists", precision, **kw),
               "%s/%s/cf%.2f" % (case, precision, cf))


@pytest.mark.parametrize("kernel,grad_h", [("sinc", 0), ("wendland", 1), ("sinc", 1)])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", ["patch20", "htail_near"])
def test_fused_equals_lists_other_forms(B, kernel, grad_h, precision, case):
    f = FORCE_CASES[case]()
    lz = f.pop("lz", 1.0)
    kw = dict(lz=lz, threads_per_particle=1, kernel=kernel, kernel_n=6, grad_h=grad_h)
    _same_bits(_forces(B, f, "fused", precision, **kw), _forces(B, f, "lists", precision, **kw),
               "%s/%s/%s/gh%d" % (case, kernel, precision, grad_h))


@pytest.mark.parametrize("case", sorted(FORCE_CASES))
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
def test_fused_pair_sums_match_oracle(B, orc, case, precision, tol, report):
    f = FORCE_CASES[case]()
    lz = f.pop("lz", 1.0)
    g = _forces(B, f, "fused", precision, lz=lz)
    o = _oracle_forces(orc, f, lz)
    nb = orc.neighbors(f["x"], f["y"], f["z"], f["h"], lz)
    assert np.array_equal(g["nnb"].astype(np.int64), np.diff(nb.off))
    assert np.array_equal(g["nown"].astype(np.int64), nb.nown.astype(np.int64))
    _check_forces(g, o, tol, report, "fused/%s/%s" % (precision, case))


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
def test_fused_ten_steps(B, orc, precision, tol, report):
    """Ten steps without any list: against the oracle, and bit for bit
    against the list mode with one lane per particle."""
    f = inputs.square_patch(20)
    n = len(f["x"])
    fused = B.SPH(n, precision=precision, pair_mode="fused")
    lists = B.SPH(n, precision=precision, pair_mode="lists", threads_per_particle=1)
    fused.set_particles(f)
    lists.set_particles(f)
    ref = orc.Sim(f)
    hist = []
    keys = ("x", "y", "z", "vx", "vy", "vz", "u", "h", "nown", "rho", "ax", "ay", "az")
    for step in range(10):
        dt = fused.step(1)
        dt_l = lists.step(1)
        ref.step(1)
        assert dt == dt_l, step
        assert abs(dt - ref.dt) <= tol * ref.dt, (step, dt, ref.dt)
        g = {k: fused.field(k) for k in keys}
        h = {k: lists.field(k) for k in keys}
        for k in keys:
            assert np.array_equal(g[k].view(np.uint64), h[k].view(np.uint64)), (step, k)
        hist.append(_compare_state(g, ref, tol, "fused step %d" % step))
    report["fused_steps10/%s" % precision] = hist
    assert fused.pair_count() == lists.pair_count()
    fused.close()
    lists.close()


def test_fused_graph_replay_same_bits(B):
    f = inputs.irregular_patch(16, seed_pos=6, seed_mass=7)
    n = len(f["x"])
    out = []
    for graph in (0, 1):
        sim = B.SPH(n, pair_mode="fused", use_graph=graph)
        sim.set_particles(f)
        sim.step(4)
        out.append({k: sim.field(k) for k in ("x", "vx", "u", "h", "rho", "ax")})
        sim.close()
    for k in out[0]:
        assert np.array_equal(out[0][k].view(np.uint64), out[1][k].view(np.uint64)), k


def test_fused_batched_patches(B, orc):
    f, offsets, edges, omegas = inputs.batch_patches(6, seed=3)
    n = len(f["x"])
    g = {}
    for mode in ("fused", "lists"):
        sim = B.SPH(n, max_patches=6, pair_mode=mode, threads_per_particle=1)
        sim.set_particles(f)
        sim.set_patches(offsets)
        sim.find_neighbors()
        sim.density()
        sim.momentum_energy()
        g[mode] = {k: sim.field(k) for k in FIELDS}
        sim.close()
    _same_bits(g["fused"], g["lists"], "batched")


def test_autotune_chooses_a_mode(B, orc):
    f = inputs.square_patch(24)
    n = len(f["x"])
    sim = B.SPH(n, pair_mode="auto")
    sim.set_particles(f)
    assert sim.pair_mode() == "lists"
    sim.autotune()
    mode = sim.pair_mode()
    assert mode in ("lists", "fused")
    sim.set_particles(f)
    sim.step(1)
    ref = orc.Sim(f)
    ref.step(1)
    assert normwise(sim.field("rho"), ref["rho"]) < 1e-5
    assert np.array_equal(sim.field("nown"), ref["nown"])
    sim.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_fused_empty_and_single(B, precision):
    sim = B.SPH(4, precision=precision, pair_mode="fused")
    z = {k: np.zeros(0) for k in ("x", "y", "z", "vx", "vy", "vz", "m", "h", "u")}
    sim.set_particles(z)
    sim.step(2)
    one = {k: np.zeros(1) for k in ("x", "y", "z", "vx", "vy", "vz")}
    one.update(m=np.full(1, 0.5), h=np.full(1, 0.1), u=np.ones(1))
    sim.set_particles(one)
    sim.find_neighbors()
    sim.density()
    sim.momentum_energy()
    assert sim.field("nnb")[0] == 0 and sim.field("nown")[0] == 0
    assert sim.field("ax")[0] == 0
    sim.close()
