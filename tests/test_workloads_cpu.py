"""The seeded input recipes: shapes and values the paper states (Sec. 3.1-3.2)
and the determinism both sides rely on."""
import math

import numpy as np

from paper_2305_19400_gb300 import workloads as W


def test_paper_device_has_the_stated_shape():
    wl = W.paper_hot_spot()
    g = wl.geoms[0]
    assert (g.dim, g.nx, g.ny, g.nz) == (2, 120, 120, 1)
    assert math.isclose(g.nx * g.dx, 525e-6, rel_tol=1e-15)       # 525 um square
    assert wl.dirs.nd == 20 and wl.bands.nb == 55                # 20 directions, 40 bands -> 55 band-pols
    assert wl.dof == 120 * 120 * 20 * 55                         # "about 1.6e7" degrees of freedom
    assert math.isclose(wl.dt * wl.nsteps, 100e-9, rel_tol=1e-15)  # 100 steps = 100 ns
    assert g.T_init == 300.0
    kinds = [k for k, _ in g.bc]
    assert kinds == [W.BC_ISOTHERMAL, W.BC_ISOTHERMAL, W.BC_SPECULAR, W.BC_SPECULAR]
    assert np.all(g.bc[1][1] == 300.0)                           # the cold wall


def test_hot_spot_profile_is_the_stated_gaussian():
    """Peak 350 K at the wall centre and 300 + 50/e^2 K at 10 um from it."""
    n, d = 120, 525e-6 / 120
    r = 10e-6 / d
    T = W.hot_spot_profile(n, 300.0, 50.0, r)
    y = (np.arange(n) + 0.5) * d - 60 * d                        # face centre minus the wall centre
    ref = 300.0 + 50.0 * np.exp(-2.0 * (y / 10e-6) ** 2)
    assert np.allclose(T, ref, rtol=0, atol=1e-12)
    assert np.isclose(300.0 + 50.0 * np.exp(-2.0 * (10e-6 / 10e-6) ** 2), 300.0 + 50.0 / math.e ** 2)
    assert T.max() < 350.0 and T.max() > 345.0                   # sampled half a cell off the peak
    assert np.allclose(T, T[::-1], rtol=0, atol=1e-12)           # centred


def test_band_tables_are_deterministic_and_in_the_stated_ranges():
    a = W.make_bands(40, 15, 19406)
    b = W.make_bands(40, 15, 19406)
    assert np.array_equal(a.vg, b.vg) and np.array_equal(a.beta, b.beta)
    assert np.all((a.vg >= 1e3) & (a.vg <= 8e3))
    tau = 1.0 / a.beta
    assert np.all((tau >= 1e-12 * (1 - 1e-12)) & (tau <= 1e-9 * (1 + 1e-12)))
    assert np.all(a.omega_hi > a.omega_lo) and a.omega_hi.max() == 1e14
