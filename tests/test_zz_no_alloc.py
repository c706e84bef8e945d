"""sph_conserved_noalloc: the conserved sums without any device allocation,
for callers that cannot call cudaMalloc (work recorded into a CUDA graph, host
frameworks that own the allocator).  Its scratch is a fixed array inside the
library.  Checked through the C ABI against sph_conserved, the entry point
that uses the context's allocated scratch, on two calls in a row (the second
call finds the array holding the first call's values).  This file is named to
be collected last."""
import numpy as np
import pytest

from paper_1905_03344_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1905_03344_gb300 import binding, build
    build.build()
    binding.lib()
    return binding


def _fields(seed):
    f = inputs.random_cloud(20000, seed=seed, vscale=2.0)
    f["x"] = f["x"] + 0.25     # nonzero angular momentum and linear momentum
    return f


def test_noalloc_matches_allocating_entry_point(B):
    import torch
    for call, seed in enumerate((0, 1)):
        f = _fields(seed)
        n = len(f["x"])
        sim = B.SPH(n, precision="fp64")
        sim.set_particles(f)
        ref = sim.conserved()
        sim.close()
        dev = {k: torch.tensor(f[k], dtype=torch.float64, device="cuda") for k in
               ("x", "y", "vx", "vy", "vz", "m", "u")}
        out = torch.full((7,), np.nan, dtype=torch.float64, device="cuda")
        stream = torch.cuda.current_stream()
        B.sph_conserved_noalloc(dev, out, stream.cuda_stream)
        stream.synchronize()
        got = out.cpu().numpy()
        scale = np.abs(ref).max()
        assert np.all(np.isfinite(got)), call
        assert np.allclose(got, ref, rtol=1e-12, atol=1e-12 * scale), (call, got, ref)


def test_noalloc_rejects_beyond_its_fixed_scratch(B):
    import torch
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    out = torch.zeros(7, dtype=torch.float64, device="cuda")
    import ctypes
    st = B.lib().sph_conserved_noalloc(16777217, *[ctypes.c_void_p(x.data_ptr())] * 7,
                                       ctypes.c_void_p(out.data_ptr()), None)
    assert st == B.SPH_EINVAL
    assert b"16777216" in B.lib().sph_noalloc_last_error()
