"""Edge and degenerate cases of the CUDA path through the C ABI: empty and
single-particle inputs, coincident particles, list overflow, bad inputs and
configurations, call-order errors, checkpoint/resume and graph replay."""
import math

import numpy as np
import pytest

from paper_1905_03344_gb300 import inputs

pytestmark = pytest.mark.gpu

SIGMA = 21.0 / (16.0 * math.pi)


@pytest.fixture(scope="module")
def B():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1905_03344_gb300 import binding, build
    build.build()
    binding.lib()
    return binding


def _fields(n, **over):
    f = {k: np.zeros(n) for k in ("x", "y", "z", "vx", "vy", "vz")}
    f.update(m=np.full(n, 0.5), h=np.full(n, 0.1), u=np.ones(n))
    f.update(over)
    return f


@pytest.mark.parametrize("bins", [0, 8])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_empty(B, precision, bins):
    sim = B.SPH(16, precision=precision, pair_bins=bins)
    sim.set_particles(_fields(0))
    sim.find_neighbors()
    off, col, perm = sim.neighbors()
    assert len(col) == 0 and off[0] == 0
    sim.step(2)
    assert np.all(sim.conserved() == 0)
    sim.close()


@pytest.mark.parametrize("bins", [0, 8])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_single_particle(B, precision, bins):
    # with bins: one particle is no sort; it is summed by the last octave's launch
    sim = B.SPH(4, precision=precision, pair_bins=bins)
    sim.set_particles(_fields(1, x=np.array([0.1]), vx=np.array([1.0])))
    sim.find_neighbors()
    sim.density()
    sim.momentum_energy()
    rho = sim.field("rho")[0]
    assert rho == pytest.approx(0.5 * SIGMA / 0.1 ** 3, rel=1e-6 if precision == "mixed" else 1e-14)
    assert sim.field("ax")[0] == 0 and sim.field("du")[0] == 0
    assert sim.field("nown")[0] == 0
    sim.step(1)
    assert sim.field("h")[0] == pytest.approx(0.2)   # n_i = 0 doubles h
    sim.close()


@pytest.mark.parametrize("bins", [0, 8])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_coincident_pair(B, precision, bins):
    sim = B.SPH(4, precision=precision, pair_bins=bins)
    sim.set_particles(_fields(2))
    sim.find_neighbors()
    off, col, perm = sim.neighbors()
    assert list(np.diff(off)) == [1, 1]
    sim.density()
    sim.momentum_energy()
    rho = sim.field("rho")
    assert np.allclose(rho, 2 * 0.5 * SIGMA / 0.1 ** 3, rtol=1e-6)
    assert np.all(sim.field("ax") == 0) and np.all(np.isfinite(sim.field("du")))
    sim.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_grad_h_isolated_particle(B, precision):
    """A particle with no neighbour inside its support has Omega = 0 in the
    grad-h form: the density call reports SPH_ENONFINITE."""
    sim = B.SPH(4, precision=precision, grad_h=1)
    sim.set_particles(_fields(2, x=np.array([0.1, 0.7])))
    sim.find_neighbors()
    with pytest.raises(B.SphError) as e:
        sim.density()
    assert e.value.status == B.SPH_ENONFINITE
    sim.close()


def test_overflow_leaves_state(B):
    f = inputs.square_patch(10)
    n = len(f["x"])
    sim = B.SPH(n, precision="fp64", max_pairs=10 * n)
    sim.set_particles(f)
    with pytest.raises(B.SphError) as e:
        sim.find_neighbors()
    assert e.value.status == B.SPH_EOVERFLOW
    x0 = sim.field("x")
    with pytest.raises(B.SphError) as e:
        sim.step(2)
    assert e.value.status == B.SPH_EOVERFLOW
    assert np.array_equal(sim.field("x"), x0)
    assert sim.dt()[2] == 0
    sim.close()


def test_overflow_of_long_rows_with_guard_band_words(B):
    """Rows of ~700 neighbours in a random cloud (many of them with words in
    the guard band, decided after the walk) against a pool far too small:
    the warps whose reservations do not fit must leave the pool alone, so the
    call reports the overflow and the context stays usable."""
    f = inputs.random_cloud(20000, seed=3)
    n = len(f["x"])
    sim = B.SPH(n, precision="fp64", max_pairs=10 * n)
    sim.set_particles(f)
    for _ in range(2):
        with pytest.raises(B.SphError) as e:
            sim.find_neighbors()
        assert e.value.status == B.SPH_EOVERFLOW
    assert np.array_equal(sim.field("x"), f["x"])
    sim.close()


def test_bad_inputs(B):
    sim = B.SPH(8)
    f = _fields(3)
    f["x"][1] = np.nan
    with pytest.raises(B.SphError) as e:
        sim.set_particles(f)
    assert e.value.status == B.SPH_EINVAL
    f = _fields(3)
    f["h"][0] = 0.0
    with pytest.raises(B.SphError):
        sim.set_particles(f)
    with pytest.raises(B.SphError):
        sim.set_particles(_fields(9))      # beyond max_particles
    sim.close()


@pytest.mark.parametrize("kw", [dict(cell_factor=0.3), dict(threads_per_particle=3),
                                dict(max_particles=0), dict(gamma=1.0), dict(max_patches=300),
                                dict(kernel=2), dict(kernel=1, kernel_n=1), dict(kernel=1, kernel_n=17),
                                dict(grad_h=2), dict(grad_h=-1), dict(pair_mode=3), dict(pair_mode=-1),
                                dict(list_skin=-0.1), dict(list_skin=1.5), dict(pair_bins=12), dict(pair_bins=-2),
                                dict(pair_bins=512), dict(pair_bins=4)])
def test_bad_config(B, kw):
    mp = kw.pop("max_particles", 8)
    with pytest.raises(B.SphError) as e:
        B.SPH(mp, **kw)
    assert e.value.status == B.SPH_EINVAL


def test_call_order(B):
    f = inputs.square_patch(6)
    sim = B.SPH(len(f["x"]))
    sim.set_particles(f)
    with pytest.raises(B.SphError) as e:
        sim.density()
    assert e.value.status == B.SPH_ESTATE
    with pytest.raises(B.SphError):
        sim.field("rho")
    sim.find_neighbors()
    with pytest.raises(B.SphError):
        sim.momentum_energy()
    sim.step(1)
    with pytest.raises(B.SphError) as e:
        sim.set_patches([0, len(f["x"])])
    assert e.value.status == B.SPH_ESTATE
    sim.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_checkpoint_resume_bitwise(B, precision):
    f = inputs.square_patch(12)
    sim = B.SPH(len(f["x"]), precision=precision)
    sim.set_particles(f)
    sim.step(3)
    blob = sim.get_state()
    sim.step(3)
    a = {k: sim.field(k) for k in ("x", "y", "z", "vx", "u", "h", "du_prev")}
    sim2 = B.SPH(len(f["x"]), precision=precision)
    sim2.set_state(blob)
    sim2.step(3)
    b = {k: sim2.field(k) for k in a}
    for k in a:
        assert np.array_equal(a[k], b[k]), k
    assert sim.dt() == sim2.dt()
    sim.close()
    sim2.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_host_state_round_trip_every_step_bitwise(B, precision):
    """The end-to-end use of the C ABI: each step uploads the whole state from
    a pinned host buffer (sph_set_state, which carries the context's last row
    lengths into the restored order as reservation hints), steps once and
    reads the state back (sph_get_state).  Bit for bit the same as stepping on
    the device; the first restore into a context that has stepped a different
    state gets foreign hints, which only cost a repair."""
    import torch
    f = inputs.square_patch(14)
    n = len(f["x"])
    ref = B.SPH(n, precision=precision)
    ref.set_particles(f)
    ref.step(2)
    buf = torch.empty(ref.state_bytes(), dtype=torch.uint8).pin_memory()
    assert ref.get_state(buf) == buf.numel()
    sim = B.SPH(n, precision=precision)
    sim.set_particles(inputs.random_cloud(n, seed=3))     # other lists, other hints
    sim.step(1)
    for _ in range(4):
        sim.set_state(buf)
        sim.step(1)
        sim.get_state(buf)
        ref.step(1)
    for k in ("x", "y", "z", "vx", "vy", "vz", "u", "h", "du_prev", "nown", "nnb"):
        assert np.array_equal(sim.field(k), ref.field(k)), k
    assert sim.dt() == ref.dt()
    sim.close()
    ref.close()


@pytest.mark.parametrize("bins", [0, 16])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_graph_replay_bitwise(B, precision, bins):
    """Replaying the captured step gives the same bits as launching it, also
    with row-length bins (their bounds stay on the device)."""
    f = inputs.square_patch(12)
    n = len(f["x"])
    runs = []
    for graph in (0, 1):
        sim = B.SPH(n, precision=precision, use_graph=graph, pair_bins=bins)
        sim.set_particles(f)
        sim.step(5)
        runs.append({k: sim.field(k) for k in ("x", "vy", "u", "h")})
        if graph:
            assert sim.launches() > 0
        sim.close()
    for k in runs[0]:
        assert np.array_equal(runs[0][k], runs[1][k]), k


def test_autotune_keeps_physics(B, orc):
    f = inputs.square_patch(14)
    sim = B.SPH(len(f["x"]), precision="fp64")
    sim.set_particles(f)
    tpp, cf = sim.autotune()
    assert tpp in (1, 2, 4, 8, 16, 32) and 0.5 <= cf <= 4
    sim.set_particles(f)
    sim.step(1)
    ref = orc.Sim(f)
    ref.step(1)
    assert np.abs(sim.field("x") - ref["x"]).max() < 1e-12
    sim.close()


def test_profile_and_launch_counts(B):
    f = inputs.square_patch(10)
    sim = B.SPH(len(f["x"]))
    sim.set_particles(f)
    sim.profile(True)
    l0 = sim.launches()
    sim.step(2)
    prof = sim.profile()
    assert sim.launches() > l0
    assert all(v[0] >= 0 for v in prof.values())
    assert prof["momentum"][1] == 2 and prof["density"][1] == 2
    assert sim.pair_count() > 0
    sim.close()


@pytest.mark.gpu
def test_fma_peak_plausible(B):
    """The FMA-chain rate: FP32 at least a few tens of TFLOP/s on a GB300 and
    FP64 far below it (the reduced FP64 pipe); a rate above the SM count x
    lanes x 2 x 3 GHz would mean the chains were optimised away."""
    f32 = B.sph_fma_peak("mixed")
    f64 = B.sph_fma_peak("fp64")
    assert 10e12 < f32 < 152 * 128 * 2 * 3.0e9
    assert 0.05e12 < f64 < f32 / 4


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_reupload_same_results(B, precision):
    """Uploading the same particles again carries the last row lengths over as
    reservation hints; they only place rows in the pool, so the steps that
    follow give the bits of a fresh context."""
    f = inputs.irregular_patch(14, seed_pos=6, seed_mass=7)
    n = len(f["x"])
    a = B.SPH(n, precision=precision)
    a.set_particles(f)
    a.step(3)
    a.set_particles(f)
    a.step(2)
    b = B.SPH(n, precision=precision)
    b.set_particles(f)
    b.step(2)
    for k in ("x", "vx", "u", "h", "rho", "ax", "nown", "nnb"):
        assert np.array_equal(a.field(k).view(np.uint64), b.field(k).view(np.uint64)), k
    a.close()
    b.close()
