"""CPU checks of the C ABI: the library builds for sm_103a, loads, exports every
symbol the headers in include/ declare, and rejects bad arguments before
touching CUDA."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


@pytest.fixture(scope="module")
def lib():
    from paper_2305_19400_gb300 import build as B, bte
    B.build()
    return bte.lib()


def declared_symbols():
    src = "".join(open(h).read() for h in HEADERS)
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bte_[a-zA-Z_]+)\s*\(", src)))


def test_header_declares_the_boundary_calls():
    names = declared_symbols()
    for must in ("bte_init_mesh", "bte_set_bands", "bte_set_bc", "bte_step", "bte_get_T", "bte_get_flux"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2305_19400_gb300 import bte
    for name in declared_symbols():
        assert hasattr(lib, name), name
        assert name in bte.SIGNATURES, f"binding lacks {name}"


def test_default_opts(lib):
    from paper_2305_19400_gb300 import bte
    o = bte.bte_default_opts()
    assert o.n_gauss == 16 and o.newton_maxit == 50 and o.precision == bte.BTE_FP64
    assert lib.bte_default_opts(None) == -1


@pytest.mark.parametrize("geom", [(2, 0, 4, 1), (2, 4, 4, 2), (4, 4, 4, 4), (3, 4, 4, 0)])
def test_init_mesh_rejects_bad_geometry(lib, geom):
    from paper_2305_19400_gb300 import bte
    g = bte.bte_geom(*geom, 1e-8, 1e-8, 1e-8)
    with pytest.raises(bte.BTEError) as e:
        bte.bte_init_mesh([g])
    assert e.value.code == -1


def test_init_mesh_rejects_mixed_dimensions(lib):
    from paper_2305_19400_gb300 import bte
    g2 = bte.bte_geom(2, 4, 4, 1, 1e-8, 1e-8, 1e-8)
    g3 = bte.bte_geom(3, 4, 4, 4, 1e-8, 1e-8, 1e-8)
    with pytest.raises(bte.BTEError) as e:
        bte.bte_init_mesh([g2, g3])
    assert e.value.code == -1 and "same dim" in str(e.value)


def test_init_mesh_rejects_bad_direction_sets_and_options(lib):
    from paper_2305_19400_gb300 import bte
    g = bte.bte_geom(2, 4, 4, 1, 1e-8, 1e-8, 1e-8)
    for field, val in (("n_gauss", 0), ("n_gauss", 99), ("newton_rtol", 0.0), ("newton_maxit", 0),
                       ("beta_T_exp", 17.0), ("beta_T_exp", float("nan")), ("T_ref", 0.5)):
        o = bte.bte_default_opts()
        setattr(o, field, val)
        with pytest.raises(bte.BTEError):
            bte.bte_init_mesh([g], o)
    h = C.c_void_p()
    assert lib.bte_init_mesh(None, 1, None, None) == -1
    assert lib.bte_init_mesh(C.byref(h), 0, None, None) == -1
    assert "n_geom" in bte.bte_last_error(None)


def test_null_handle_is_an_argument_error(lib):
    assert lib.bte_step(None, 1e-12, 1, 1, 0, None) == -1
    assert lib.bte_destroy(None) == -1
    assert lib.bte_workspace_bytes(None) == 0
    assert lib.bte_set_band_range(None, 0, 1) == -1
    from paper_2305_19400_gb300 import bte
    assert lib.bte_set_exchange(None, bte.bte_allreduce_fn(), None, None) == -1
