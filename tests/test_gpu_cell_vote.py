"""The cell grid's vote, which moves an automatic cell factor between 1/2
(cells of edge h_s, a 2-cell stencil) and 0.4 (a 3-cell stencil over cells
down to 1.3 h_median) from one step call to the next:

  - a lattice patch whose h rises smoothly towards one face (a wide spread
    of h, smooth in space) switches to 0.4 after one step, and the lists on
    the new grid are bit-exact against the oracle's on the same state, the
    density within the mixed path's 1e-5;
  - a cloud whose h is drawn per particle (a wide spread, but no smooth
    region) keeps 1/2;
  - a cell factor set by the caller is kept.
"""
import numpy as np
import pytest

from paper_1905_03344_gb300 import inputs
from gpu_common import normwise

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1905_03344_gb300 import binding, build
    build.build()
    binding.lib()
    return binding


def graded_patch(n):
    """The n^3 square patch with h growing smoothly from h0 (x below 0.2) to
    2 h0 at the face x = 1/2: median h0, class threshold about 2 h0."""
    f = inputs.square_patch(n)
    t = np.clip((f["x"] - 0.2) / 0.3, 0.0, 1.0)
    f["h"] = f["h"] * (1.0 + t * t)
    return f


def cell_factor(B, sim):
    return B.sph_get_tuning(sim.ctx)[1]


def gpu_rows(B, sim, n):
    """The lists as a sorted array of original-index pairs (i, j)."""
    off, col, perm = B.sph_copy_neighbors(sim.ctx, n)
    off = np.asarray(off, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    perm = np.asarray(perm, dtype=np.int64)
    i = perm[np.repeat(np.arange(n), np.diff(off))]
    return np.sort(i * n + perm[col])


def test_smooth_wide_spread_switches_to_the_three_cell_stencil(B, orc):
    f = graded_patch(30)
    n = len(f["x"])
    sim = B.SPH(n, precision="mixed", max_pairs=400 * n, adapt_h=0)
    sim.set_particles(f)
    assert cell_factor(B, sim) == 0.5
    sim.step(1)
    assert cell_factor(B, sim) == 0.4
    # the next search runs on the 3-cell grid: lists, density and forces
    # against the oracle on the state after the step
    sim.find_neighbors()
    st = {k: sim.field(k) for k in ("x", "y", "z", "vx", "vy", "vz", "m", "h", "u")}
    nb = orc.neighbors(st["x"], st["y"], st["z"], st["h"], 1.0)
    ref = np.sort(np.repeat(np.arange(n), np.diff(nb.off)).astype(np.int64) * n + nb.col.astype(np.int64))
    assert np.array_equal(gpu_rows(B, sim, n), ref)
    assert np.array_equal(sim.field("nown").astype(np.int64), nb.nown.astype(np.int64))
    sim.density()
    rho_o = orc.density(st["x"], st["y"], st["z"], st["m"], st["h"], nb, 1.0)
    assert normwise(sim.field("rho"), rho_o) < 1e-5
    sim.close()


def test_per_particle_spread_and_caller_factor_keep_one_half(B):
    g = inputs.random_cloud(4000, seed=5, h_lo=0.04, h_hi=0.09)
    sim = B.SPH(len(g["x"]), precision="mixed", max_pairs=400 * len(g["x"]), adapt_h=0)
    sim.set_particles(g)
    sim.step(2)
    assert cell_factor(B, sim) == 0.5
    sim.close()
    f = graded_patch(30)
    n = len(f["x"])
    sim = B.SPH(n, precision="mixed", max_pairs=400 * n, adapt_h=0, cell_factor=0.5)
    sim.set_particles(f)
    sim.step(2)
    assert cell_factor(B, sim) == 0.5
    sim.close()
