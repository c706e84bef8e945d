"""Argument checks of the Python binding, run on the CPU: every refusal
happens before the library is called, so nothing is launched and no device
is needed.  A wrong dtype, a short field or a short output buffer would
otherwise let a kernel or a copy read or write past an array: the
no-allocation conserved sums, sph_set_particles and sph_get_field."""
import pytest

torch = pytest.importorskip("torch")

from paper_1905_03344_gb300 import binding

NAMES = ("x", "y", "vx", "vy", "vz", "m", "u")


def _fields(n=10, dtype=torch.float64):
    return {k: torch.zeros(n, dtype=dtype) for k in NAMES}


def _refused(fields, out, match):
    with pytest.raises(ValueError, match=match):
        binding.sph_conserved_noalloc(fields, out)


def test_refuses_float32_field():
    f = _fields()
    f["vy"] = torch.zeros(10, dtype=torch.float32)
    _refused(f, torch.zeros(7, dtype=torch.float64), "vy must be float64")


def test_refuses_float32_out():
    _refused(_fields(), torch.zeros(7, dtype=torch.float32), "out must be float64")


@pytest.mark.parametrize("k", ["y", "m", "u"])
def test_refuses_fields_of_unequal_length(k):
    f = _fields()
    f[k] = torch.zeros(9, dtype=torch.float64)
    _refused(f, torch.zeros(7, dtype=torch.float64), "%s has 9 elements" % k)


def test_refuses_short_out():
    _refused(_fields(), torch.zeros(6, dtype=torch.float64), "out must hold 7")


def test_refuses_missing_field():
    f = _fields()
    del f["vz"]
    _refused(f, torch.zeros(7, dtype=torch.float64), "missing fields")


def test_refuses_host_tensors():
    _refused(_fields(), torch.zeros(7, dtype=torch.float64), "contiguous CUDA tensor")


def test_refuses_non_tensors():
    import numpy as np
    f = {k: np.zeros(10) for k in NAMES}
    _refused(f, torch.zeros(7, dtype=torch.float64), "must be a torch tensor")


# ---- the same kind of checks on sph_set_particles and sph_get_field ---------

FIELDS9 = ("x", "y", "z", "vx", "vy", "vz", "m", "h", "u")


def test_set_particles_refuses_float32_tensor():
    f = {k: torch.zeros(10, dtype=torch.float64) for k in FIELDS9}
    f["h"] = torch.zeros(10, dtype=torch.float32)
    with pytest.raises(ValueError, match="h must be float64"):
        binding.sph_set_particles(None, f)


def test_set_particles_refuses_unequal_lengths():
    f = {k: torch.zeros(10, dtype=torch.float64) for k in FIELDS9}
    f["u"] = torch.zeros(12, dtype=torch.float64)
    with pytest.raises(ValueError, match="u has 12 elements"):
        binding.sph_set_particles(None, f)
    import numpy as np
    g = {k: np.zeros(10) for k in FIELDS9}
    g["m"] = np.zeros(9)
    with pytest.raises(ValueError, match="m has 9 elements"):
        binding.sph_set_particles(None, g)


def test_set_particles_refuses_missing_field():
    f = {k: torch.zeros(4, dtype=torch.float64) for k in FIELDS9 if k != "vz"}
    with pytest.raises(ValueError, match="missing fields"):
        binding.sph_set_particles(None, f)


def test_get_field_refuses_short_or_float32_out():
    with pytest.raises(ValueError, match="at least 10"):
        binding.sph_get_field(None, "rho", 10, out=torch.zeros(9, dtype=torch.float64))
    with pytest.raises(ValueError, match="must be float64"):
        binding.sph_get_field(None, "rho", 10, out=torch.zeros(10, dtype=torch.float32))
