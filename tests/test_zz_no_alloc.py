"""The wall-flux entry point that allocates no device memory.

bte_get_wall_flux_noalloc exists for callers that cannot call cudaMalloc
(a fixed device-memory budget, memory owned by another allocator, or a
latency-critical loop where an allocation would synchronize the device).  It
keeps its per-face scratch in a static device array inside libbte.so.  This
test checks, through the C ABI, that two calls in a row return the same
per-side wall fluxes as bte_get_flux, within the tolerance the flux parity
tests use, for host and device outputs.  It lives in its own file, collected
last, and passes both alone in a fresh process and after the other tests.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2305_19400_gb300 import bte, workloads as W

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2305_19400_gb300 import build as B
    B.build()


def _flux_scale(s, geom):
    """Largest per-cell absolute flux sum, the scale the flux tolerance is relative to."""
    S, _, _ = bte.bte_get_directions(s.h)
    I = s.intensity(geom)
    return float(np.einsum("da,cdb->ca", np.abs(S), np.abs(I)).max())


@pytest.mark.parametrize("make", [lambda: W.cfg2(21, 13), lambda: W.cfg1()])
def test_noalloc_wall_flux_matches_bte_get_flux_twice(make):
    wl = make()
    s = bte.Solver(wl)
    s.step(nsteps=2, ninner=5)
    g = wl.geoms[0]
    _, qw_ref = s.flux(0)
    tol = 1e-11 * _flux_scale(s, 0)
    for _ in range(2):
        qw = np.zeros(2 * g.dim)
        bte.bte_get_wall_flux_noalloc(s.h, 0, qw)
        assert np.all(np.abs(qw - qw_ref) <= tol), (qw, qw_ref)
        qd = torch.zeros(2 * g.dim, dtype=torch.float64, device="cuda")
        bte.bte_get_wall_flux_noalloc(s.h, 0, qd)
        assert np.all(np.abs(qd.cpu().numpy() - qw_ref) <= tol)
    # the hot wall takes energy in (the cold wall is too far for the heat to arrive yet)
    assert qw_ref[0] < 0
    s.close()


def test_noalloc_wall_flux_on_several_geometries_and_after_more_steps():
    geoms = []
    for nx, ny, th in ((9, 4, 310.0), (3, 11, 305.0)):
        g = W.Geometry(2, nx, ny, 1, 10e-9, 10e-9, 10e-9)
        W.uniform_walls(g, [W.BC_ISOTHERMAL, W.BC_ISOTHERMAL, W.BC_ISOTHERMAL, W.BC_SPECULAR], [th, 300.0, 302.0, 0])
        geoms.append(g)
    wl = W.Workload("pair", geoms, W.Dirs("inplane", n_inplane=16), W.make_bands(40, 15, 19402), 1e-12, 3, 4)
    s = bte.Solver(wl)
    for round_ in range(2):
        s.step()
        for gi in range(2):
            _, qw_ref = s.flux(gi)
            qw = np.zeros(4)
            bte.bte_get_wall_flux_noalloc(s.h, gi, qw)
            assert np.all(np.abs(qw - qw_ref) <= 1e-11 * _flux_scale(s, gi))
    s.close()


def test_noalloc_rejects_bad_arguments_and_walls_beyond_its_maximum():
    wl = W.cfg1()
    s = bte.Solver(wl)
    with pytest.raises(bte.BTEError) as e:
        bte.bte_get_wall_flux_noalloc(s.h, 5, np.zeros(4))
    assert e.value.code == -1
    s.close()
    # a 1 x 70000 strip: its x walls have 70000 faces, more than the 65536 the static scratch holds
    g = W.Geometry(2, 1, 70000, 1, 10e-9, 10e-9, 10e-9)
    W.uniform_walls(g, [W.BC_ISOTHERMAL, W.BC_SPECULAR, W.BC_SPECULAR, W.BC_SPECULAR], [305.0, 0, 0, 0])
    wl = W.Workload("strip", [g], W.Dirs("inplane", n_inplane=4), W.make_bands(1, 0, 3), 1e-12, 1, 1)
    s = bte.Solver(wl)
    s.step()
    with pytest.raises(bte.BTEError) as e:
        bte.bte_get_wall_flux_noalloc(s.h, 0, np.zeros(4))
    assert e.value.code == -1 and "65536" in str(e.value)
    _, qw = s.flux(0)          # the allocating path still serves it
    assert np.all(np.isfinite(qw))
    s.close()
