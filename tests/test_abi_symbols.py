"""The C ABI library loads and exports every entry point include/sph.h
declares; the Python binding marshals exactly those.  No GPU calls."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "sph.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:sph_status|void|const char\s*\*)\s+(sph_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_1905_03344_gb300 import build
    build.build()
    from paper_1905_03344_gb300 import binding
    return binding.lib()


def test_header_declares_the_entry_points():
    names = _declared()
    for n in ("sph_create", "sph_set_particles", "sph_find_neighbors", "sph_density",
              "sph_momentum_energy", "sph_step", "sph_conserved", "sph_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    from paper_1905_03344_gb300 import binding
    assert sorted(binding.SIGNATURES) == _declared()


def test_config_struct_matches_header_defaults(lib):
    from paper_1905_03344_gb300 import binding
    c = binding.sph_config_default()
    assert c.precision == binding.SPH_MIXED
    assert c.gamma == pytest.approx(5.0 / 3.0)
    assert c.courant == 0.2 and c.dt_growth == 1.1 and c.n_target == 100.0
    assert c.av_alpha == 1.0 and c.av_beta == 2.0 and c.av_eps == 0.01
    assert c.lz == 1.0 and c.adapt_h == 1 and c.cell_factor == 0.0


def test_status_strings(lib):
    from paper_1905_03344_gb300 import binding
    for k, v in binding.STATUS_NAMES.items():
        assert lib.sph_status_string(k).decode() == v


def test_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1905_03344_gb300 import binding
    with pytest.raises(binding.SphError) as e:
        binding.sph_create()
    assert e.value.status == binding.SPH_ECUDA


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No fallback: without the built library every call path raises."""
    from paper_1905_03344_gb300 import binding
    monkeypatch.setattr(binding._build, "LIB", str(tmp_path / "libsph_gb300.so"))
    monkeypatch.setattr(binding, "_lib", None)
    with pytest.raises(ImportError):
        binding.lib()
    with pytest.raises(ImportError):
        binding.SPH(8)
