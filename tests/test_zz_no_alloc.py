"""The wall-flux entry point that allocates no device memory.

bte_get_wall_flux_noalloc exists for callers that cannot call cudaMalloc
(a fixed device-memory budget, memory owned by another allocator, or a
latency-critical loop where an allocation would synchronize the device).  It
keeps its per-face scratch in a static device array inside libbte.so.  This
test checks, through the C ABI, that two calls in a row return the same
per-side wall fluxes as bte_get_flux, for host and device outputs, on every
wall kind (isothermal, mirror, diffuse, partially specular) and on the z
walls of a 3-D geometry.  Both paths add each face's terms in the same order
and reduce them with the same 256-thread tree, so the results must agree bit
for bit.  It lives in its own file, collected last, and passes both alone in
a fresh process and after the other tests.
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


def _check_twice(s, gi, dim):
    """Two calls in a row, host and device outputs, each equal to bte_get_flux bit for bit."""
    _, qw_ref = s.flux(gi)
    for _ in range(2):
        qw = np.zeros(dim * 2)
        bte.bte_get_wall_flux_noalloc(s.h, gi, qw)
        assert np.array_equal(qw, qw_ref), (qw, qw_ref)
        qd = torch.zeros(2 * dim, dtype=torch.float64, device="cuda")
        bte.bte_get_wall_flux_noalloc(s.h, gi, qd)
        assert np.array_equal(qd.cpu().numpy(), qw_ref)
    return qw_ref


@pytest.mark.parametrize("make", [lambda: W.cfg2(21, 13), lambda: W.cfg1()])
def test_noalloc_wall_flux_matches_bte_get_flux_twice(make):
    wl = make()
    s = bte.Solver(wl)
    s.step(nsteps=2, ninner=5)
    qw_ref = _check_twice(s, 0, wl.geoms[0].dim)
    # the hot wall takes energy in (the cold wall is too far for the heat to arrive yet)
    assert qw_ref[0] < 0
    s.close()


def test_noalloc_wall_flux_on_diffuse_and_partially_specular_walls():
    """-y diffuse (ghost rows refreshed from the current state first), +y
    partially specular (per-direction ghost rows), x walls isothermal."""
    g = W.Geometry(2, 11, 7, 1, 10e-9, 10e-9, 10e-9)
    W.uniform_walls(g, [W.BC_ISOTHERMAL, W.BC_ISOTHERMAL, W.BC_DIFFUSE, W.BC_PARTIAL], [312.0, 300.0, 0, 0.35])
    wl = W.Workload("diffuse+partial", [g], W.Dirs("polar_azim", n_polar=4, n_azim=8), W.make_bands(8, 3, 61),
                    1e-12, 3, 4)
    s = bte.Solver(wl)
    s.step()
    qw = _check_twice(s, 0, 2)
    assert qw[0] < 0 and np.all(np.isfinite(qw))
    s.step()
    _check_twice(s, 0, 2)
    s.close()


def test_noalloc_wall_flux_on_the_z_walls_of_a_3d_geometry():
    """5 x 4 x 3 cells; z walls isothermal (hot, cold) and the others mixed, so
    every side index 0..5 is served."""
    g = W.Geometry(3, 5, 4, 3, 10e-9, 10e-9, 10e-9)
    W.uniform_walls(g, [W.BC_SPECULAR, W.BC_DIFFUSE, W.BC_PARTIAL, W.BC_SPECULAR, W.BC_ISOTHERMAL, W.BC_ISOTHERMAL],
                    [0, 0, 0.6, 0, 309.0, 301.0])
    wl = W.Workload("3d z walls", [g], W.Dirs("polar_azim", n_polar=4, n_azim=8), W.make_bands(6, 2, 62),
                    1e-12, 2, 5)
    s = bte.Solver(wl)
    s.step()
    qw = _check_twice(s, 0, 3)
    assert qw[4] < 0 and np.all(np.isfinite(qw))   # the hot -z wall takes energy in
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
            assert np.array_equal(qw, qw_ref)
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
