"""sph_conserved_noalloc: the conserved sums without any device allocation,
for callers that cannot call cudaMalloc (work recorded into a CUDA graph, host
frameworks that own the allocator).  Its scratch is a fixed array inside the
library.  Checked through the C ABI against sph_conserved, the entry point
that uses the context's allocated scratch, and against the oracle's sums, on
calls in a row whose sizes shrink: a later call finds the array holding the
slots of a larger earlier call, which it must not read.  This file is named
to be collected last."""
import numpy as np
import pytest

from paper_1905_03344_gb300 import inputs

pytestmark = pytest.mark.gpu

NAMES = ("x", "y", "vx", "vy", "vz", "m", "u")


@pytest.fixture(scope="module")
def B():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1905_03344_gb300 import binding, build
    build.build()
    binding.lib()
    return binding


def _fields(n, seed):
    f = inputs.random_cloud(n, seed=seed, vscale=2.0)
    f["x"] = f["x"] + 0.25     # nonzero angular momentum and linear momentum
    return f


def _scales(f):
    """Per sum, the sum of its terms' magnitudes: the scale of its rounding."""
    m = f["m"]
    pv = (m * np.sqrt(f["vx"] ** 2 + f["vy"] ** 2 + f["vz"] ** 2)).sum()
    return np.array([m.sum(), pv, pv, pv,
                     (m * (np.abs(f["x"] * f["vy"]) + np.abs(f["y"] * f["vx"]))).sum(),
                     (0.5 * m * (f["vx"] ** 2 + f["vy"] ** 2 + f["vz"] ** 2)).sum(),
                     (m * np.abs(f["u"])).sum()])


def _noalloc(B, f):
    import torch
    dev = {k: torch.tensor(f[k], dtype=torch.float64, device="cuda") for k in NAMES}
    out = torch.full((7,), np.nan, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    B.sph_conserved_noalloc(dev, out, stream.cuda_stream)
    stream.synchronize()
    return out.cpu().numpy()


def test_noalloc_matches_allocating_entry_point_and_oracle(B, orc):
    # 60000 particles fill 15 scratch slots; the calls after it use 5 and 2
    for call, (n, seed) in enumerate(((60000, 0), (20000, 1), (5000, 2))):
        f = _fields(n, seed)
        sim = B.SPH(n, precision="fp64")
        sim.set_particles(f)
        ref = sim.conserved()
        sim.close()
        got = _noalloc(B, f)
        want = orc.conserved(*[f[k] for k in NAMES])
        tol = 1e-12 * _scales(f)
        assert np.all(np.isfinite(got)), call
        assert np.all(np.abs(got - ref) <= tol), (call, got, ref)
        assert np.all(np.abs(got - want) <= tol), (call, got, want)


def test_noalloc_of_no_particles_is_zero(B):
    import torch
    # after a call that filled slots, n = 0 reads none of them
    _noalloc(B, _fields(30000, 3))
    dev = {k: torch.zeros(0, dtype=torch.float64, device="cuda") for k in NAMES}
    out = torch.full((7,), np.nan, dtype=torch.float64, device="cuda")
    B.sph_conserved_noalloc(dev, out, torch.cuda.current_stream().cuda_stream)
    torch.cuda.current_stream().synchronize()
    assert np.all(out.cpu().numpy() == 0.0)


def test_noalloc_rejects_beyond_its_fixed_scratch(B):
    import torch
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    out = torch.zeros(7, dtype=torch.float64, device="cuda")
    import ctypes
    st = B.lib().sph_conserved_noalloc(16777217, *[ctypes.c_void_p(x.data_ptr())] * 7,
                                       ctypes.c_void_p(out.data_ptr()), None)
    assert st == B.SPH_EINVAL
    assert b"16777216" in B.lib().sph_noalloc_last_error()
