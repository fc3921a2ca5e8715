"""Pins of the FP64 CPU oracle against facts fixed by mathematics and physics.

Each check is chosen so that a plausible slip in the oracle -- a dropped term,
a wrong sign or index, a transposed operand -- fails at least one of them.
None of them re-types the oracle's own formula; they use closed forms,
independent library routines (scipy adaptive quadrature, root bracketing,
dense LU), hand-worked steps and conservation laws.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate, optimize

from oracle import oracle as O
from paper_2305_19400_gb300 import workloads as W

HBAR = 1.054571817e-34
KB = 1.380649e-23
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- quadrature
def test_gauss_legendre_exact_to_degree_31():
    x, w = O.gauss_legendre(16)
    assert np.all(np.diff(x) > 0)
    for k in range(32):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.sum(w * x ** k) - exact) < 1e-14, k
    # degree 32 is the first one a 16-point rule cannot integrate exactly
    assert abs(np.sum(w * x ** 32) - 2.0 / 33) > 1e-12


def _be_integral(lo, hi, T):
    f = lambda om: om ** 3 / math.expm1(HBAR * om / (KB * T))
    val, err = integrate.quad(f, lo, hi, epsabs=0.0, epsrel=1.2e-14, limit=200)
    return val


@pytest.mark.parametrize("T", [250.0, 300.0, 400.0])
def test_I0_against_adaptive_quadrature(T):
    bands = W.make_bands(40, 15, 19402)
    I0, _ = O.I0(bands, T)
    for b in range(bands.nb):
        ref = bands.degeneracy[b] * HBAR / (8 * math.pi ** 3 * bands.vg[b] ** 2) * \
            _be_integral(bands.omega_lo[b], bands.omega_hi[b], T)
        assert abs(I0[b] - ref) <= 1e-12 * ref, (b, I0[b], ref)


def test_I0_wide_bands_against_adaptive_quadrature():
    bands = W.make_bands(4, 0, 19401)
    for T in (250.0, 300.0, 400.0):
        I0, _ = O.I0(bands, T)
        for b in range(bands.nb):
            ref = HBAR / (8 * math.pi ** 3 * bands.vg[b] ** 2) * _be_integral(bands.omega_lo[b], bands.omega_hi[b], T)
            assert abs(I0[b] - ref) <= 1e-10 * ref


def test_I0_bands_add_up_to_the_planck_closed_form():
    """Many narrow bands with v = 1, g = 1 covering [0, 60 kT/hbar] sum to
    hbar/(8 pi^3) * (kT/hbar)^4 * pi^4/15 (the Bose-Einstein integral)."""
    T = 300.0
    top = 60.0 * KB * T / HBAR
    n = 300
    edges = np.linspace(0.0, top, n + 1)
    bands = W.Bands(edges[:-1], edges[1:], np.ones(n), np.ones(n), np.ones(n))
    I0, _ = O.I0(bands, T)
    exact = HBAR / (8 * math.pi ** 3) * (KB * T / HBAR) ** 4 * math.pi ** 4 / 15.0
    assert abs(I0.sum() - exact) <= 1e-13 * exact


def test_dI0_dT_against_central_difference():
    bands = W.make_bands(40, 15, 19402)
    T, h = 300.0, 1e-3
    _, d = O.I0(bands, T)
    up, _ = O.I0(bands, T + h)
    dn, _ = O.I0(bands, T - h)
    fd = (up - dn) / (2 * h)
    assert np.all(np.abs(d - fd) <= 1e-7 * np.abs(fd))


# ------------------------------------------------------------ direction sets
@pytest.mark.parametrize("kind", ["inplane16", "inplane20", "pa20x20", "pa4x8"])
def test_direction_set_moments_and_reflections(kind):
    if kind.startswith("inplane"):
        n = int(kind[7:])
        S, w, r = O.dirs_inplane(n)
        half = (4 * math.pi / n) / math.sin(math.pi / n)    # sum over S_x > 0 of S_x, closed form
    else:
        nt, nph = map(int, kind[2:].split("x"))
        S, w, r = O.dirs_polar_azim(nt, nph)
        half = math.pi                                       # int_{s_x>0} s_x dOmega
        # z half-range moment is pi as well, and the z-reflection flips S_z
        assert abs(S[S[:, 2] > 0, 2].sum() - math.pi) < 1e-13
    assert abs(w.sum() - 4 * math.pi) < 1e-13
    assert np.all(np.abs(S.sum(axis=0)) < 1e-13)
    assert abs(S[S[:, 0] > 0, 0].sum() - half) < 1e-13
    assert abs(S[S[:, 1] > 0, 1].sum() - half) < 1e-13
    nd = len(w)
    for ax in range(3):
        rr = r[ax]
        assert np.array_equal(rr[rr], np.arange(nd))                  # involution
        assert np.allclose(w[rr], w, rtol=1e-13, atol=0)               # weights kept (to rounding)
        assert np.allclose(S[rr, ax], -S[:, ax], atol=1e-14)          # normal part flips
        other = [a for a in range(3) if a != ax]
        assert np.allclose(S[rr][:, other], S[:, other], atol=1e-14)   # tangential part kept
    # no direction lies in a wall plane (upwind side always defined)
    assert np.all(S[:, 0] != 0) and np.all(S[:, 1] != 0)


# ---------------------------------------------------------------- Newton
def test_newton_matches_bracketing_root():
    wl = W.cfg2(4, 4)
    p = O.Problem(wl.geoms[0], O.dirs_for(wl.dirs), wl.bands)
    Wt = 4 * math.pi
    a = Wt * wl.bands.beta / wl.bands.vg
    for Ttrue in (251.3, 300.0, 333.3, 399.9):
        I0, _ = O.I0(wl.bands, Ttrue)
        E = float(np.dot(a, I0))
        f = lambda T: float(np.dot(a, O.I0(wl.bands, T)[0])) - E
        ref = optimize.brentq(f, 200.0, 500.0, xtol=1e-13, rtol=4 * np.finfo(float).eps, maxiter=500)
        for guess in (300.0, 250.0, 4999.0, 1.5):
            T, status = p.solve_T(a, E, guess)
            assert status in (0, 1)
            assert abs(T - ref) <= 1e-12 * ref, (Ttrue, guess, T, ref)
            assert abs(T - Ttrue) <= 1e-12 * Ttrue
    # an energy with no temperature in [1, 5000] K is reported, not invented
    T, status = p.solve_T(a, -1.0, 300.0)
    assert status == -1


def test_energy_is_monotone_so_the_root_is_unique():
    bands = W.make_bands(40, 15, 19402)
    a = 4 * math.pi / bands.vg
    Ts = np.linspace(5.0, 4000.0, 400)
    E = np.array([np.dot(a, O.I0(bands, T)[0]) for T in Ts])
    assert np.all(np.diff(E) > 0)


# ------------------------------------------------------ hand-worked update
def _two_cell_problem(dt, v, beta, T_hot, T_cold):
    g = W.Geometry(2, 2, 1, 1, 10e-9, 10e-9, 10e-9)
    g.bc = [(W.BC_ISOTHERMAL, np.array([T_hot])), (W.BC_ISOTHERMAL, np.array([T_cold])),
            (W.BC_SPECULAR, None), (W.BC_SPECULAR, None)]
    S = np.array([[2 * math.pi, 0, 0], [-2 * math.pi, 0, 0]])
    w = np.array([2 * math.pi, 2 * math.pi])
    r = np.array([[1, 0], [0, 1], [0, 1]], dtype=np.int32)
    bands = W.Bands(np.array([0.0]), np.array([5e13]), np.array([v]), np.array([beta]), np.array([1.0]))
    return O.Problem(g, (S, w, r), bands), bands


def test_two_cell_step_by_hand():
    gold = json.load(open(os.path.join(GOLDEN, "two_cell_step.json")))
    Th, Tc, dt = gold["T_hot"], gold["T_cold"], gold["dt_imp"]
    dx = 10e-9
    # v c = v |S_x| / (w dx) = v / dx = 2/dt ; beta = 1/dt
    v = 2.0 / dt * dx
    p, bands = _two_cell_problem(dt, v, 1.0 / dt, Th, Tc)
    A = O.I0(bands, Tc)[0][0]
    B = O.I0(bands, Th)[0][0]
    st = p.init_state(Tc)
    I0w = p.wall_I0()
    for key, (ca, cb) in gold["expected_implicit_in_units_of_A_B"].items():
        P, d = int(key[1]), int(key[3])
        got = p.update_one(dt, O.IMPLICIT, st["I"], st["I"], st["I0"], I0w, P, d, 0)
        assert abs(got - (ca * A + cb * B)) <= 1e-14 * A, key
    # explicit: beta = 0 and dt * v * c = 1/2
    p2, _ = _two_cell_problem(dt, v, 0.0, Th, Tc)
    dt_e = 0.5 / (v / dx)
    st2 = p2.init_state(Tc)
    I0w2 = p2.wall_I0()
    for key, (ca, cb) in gold["expected_explicit_in_units_of_A_B"].items():
        P, d = int(key[1]), int(key[3])
        got = p2.update_one(dt_e, O.EXPLICIT, st2["I"], st2["I"], st2["I0"], I0w2, P, d, 0)
        assert abs(got - (ca * A + cb * B)) <= 1e-14 * A, key


# ------------------------------------------------------ Jacobi vs dense LU
def _assemble_backward_euler(geom, S, w, r, bands, dt, In, I0wall_by_side):
    """Dense system of one backward-Euler step with beta = 0, written from Eq. 5/6:
    (1/dt) I_P + v sum_faces (s.n A/V) I_face = (1/dt) I^n_P, I_face upwind."""
    nx, ny = geom.nx, geom.ny
    nd, nb = len(w), len(bands.vg)
    N = nx * ny * nd * nb
    idx = lambda i, j, d, b: ((j * nx + i) * nd + d) * nb + b
    A = np.zeros((N, N))
    rhs = np.zeros(N)
    delta = (geom.dx, geom.dy)
    for j in range(ny):
        for i in range(nx):
            for d in range(nd):
                sdir = S[d] / w[d]
                for b in range(nb):
                    row = idx(i, j, d, b)
                    v = bands.vg[b]
                    A[row, row] += 1.0 / dt
                    rhs[row] += In[(j * nx + i), d, b] / dt
                    for ax, (lo_side, hi_side) in enumerate(((0, 1), (2, 3))):
                        # two faces along this axis: low (n = -e) and high (n = +e)
                        for side, nsgn in ((lo_side, -1.0), (hi_side, +1.0)):
                            sn = sdir[ax] * nsgn
                            coef = v * sn / delta[ax]
                            if sn > 0:            # outflow through this face: own value
                                A[row, row] += coef
                                continue
                            ci = [i, j]
                            ci[ax] += int(nsgn)
                            inside = 0 <= ci[0] < nx and 0 <= ci[1] < ny
                            if inside:
                                A[row, idx(ci[0], ci[1], d, b)] += coef
                            elif geom.bc[side][0] == W.BC_ISOTHERMAL:
                                rhs[row] -= coef * I0wall_by_side[side][b]
                            else:
                                A[row, idx(i, j, r[ax][d], b)] += coef
    return A, rhs


def test_jacobi_iterations_converge_to_dense_lu_solution():
    g = W.Geometry(2, 4, 3, 1, 10e-9, 7e-9, 10e-9)
    g.bc = [(W.BC_ISOTHERMAL, np.full(3, 310.0)), (W.BC_ISOTHERMAL, np.full(3, 300.0)),
            (W.BC_SPECULAR, None), (W.BC_SPECULAR, None)]
    S, w, r = O.dirs_inplane(8)
    bands = W.make_bands(2, 0, 7)
    bands.beta[:] = 0.0
    p = O.Problem(g, (S, w, r), bands)
    T0 = W.random_temperatures(12, 99, 295.0, 305.0)
    st = p.init_state(T0)
    In = st["I"].copy()
    I0w = {s: O.I0(bands, 310.0 if s == 0 else 300.0)[0] for s in (0, 1)}
    dt = 2e-12
    A, rhs = _assemble_backward_euler(g, S, w, r, bands, dt, In, I0w)
    x = np.linalg.solve(A, rhs).reshape(In.shape)
    p.run(st, dt, 1, 400)
    assert np.max(np.abs(st["I"] - x) / np.abs(x)) < 1e-13


def _small_lu_case(all_isothermal):
    g = W.Geometry(2, 4, 3, 1, 10e-9, 7e-9, 10e-9)
    side = [(W.BC_ISOTHERMAL, np.full(3, 310.0)), (W.BC_ISOTHERMAL, np.full(3, 300.0))]
    if all_isothermal:
        g.bc = side + [(W.BC_ISOTHERMAL, np.full(4, 305.0)), (W.BC_ISOTHERMAL, np.full(4, 295.0))]
    else:
        g.bc = side + [(W.BC_SPECULAR, None), (W.BC_SPECULAR, None)]
    S, w, r = O.dirs_inplane(8)
    bands = W.make_bands(2, 0, 7)
    bands.beta[:] = 0.0
    p = O.Problem(g, (S, w, r), bands)
    st = p.init_state(W.random_temperatures(12, 99, 295.0, 305.0))
    I0w = {s: O.I0(bands, T)[0] for s, T in zip(range(4), (310.0, 300.0, 305.0, 295.0))}
    dt = 2e-12
    A, rhs = _assemble_backward_euler(g, S, w, r, bands, dt, st["I"].copy(), I0w)
    return p, st, dt, np.linalg.solve(A, rhs).reshape(st["I"].shape)


def test_gauss_seidel_iterations_converge_to_dense_lu_solution():
    """The sweep-ordered form solves the same backward-Euler system."""
    p, st, dt, x = _small_lu_case(all_isothermal=False)
    p.run(st, dt, 1, 200, O.GAUSS_SEIDEL)
    assert np.max(np.abs(st["I"] - x) / np.abs(x)) < 1e-13


def test_one_gauss_seidel_pass_is_exact_when_every_ghost_is_fixed():
    """Isothermal walls and beta = 0: in upwind order the system is triangular,
    so one pass is the exact solution; one Jacobi pass is not."""
    p, st, dt, x = _small_lu_case(all_isothermal=True)
    stj = {k: v.copy() for k, v in st.items()}
    p.run(st, dt, 1, 1, O.GAUSS_SEIDEL)
    assert np.max(np.abs(st["I"] - x) / np.abs(x)) < 1e-13
    p.run(stj, dt, 1, 1, O.IMPLICIT)
    assert np.max(np.abs(stj["I"] - x) / np.abs(x)) > 1e-4


def test_gauss_seidel_converges_faster_than_jacobi():
    """Same fixed point; after a few inner iterations the sweep-ordered error
    is the smaller one (mirror walls, scattering on)."""
    wl = W.cfg2(9, 7)
    g = wl.geoms[0]
    p = O.Problem(g, O.dirs_for(wl.dirs), wl.bands)
    ref = p.init_state(g.T_init)
    p.run(ref, wl.dt, 1, 200, O.GAUSS_SEIDEL)
    ref_j = p.init_state(g.T_init)
    p.run(ref_j, wl.dt, 1, 200, O.IMPLICIT)
    assert np.max(np.abs(ref["Tp"] - ref_j["Tp"]) / ref["Tp"]) < 1e-13
    for m in (2, 4, 6):
        a = p.init_state(g.T_init)
        b = p.init_state(g.T_init)
        p.run(a, wl.dt, 1, m, O.GAUSS_SEIDEL)
        p.run(b, wl.dt, 1, m, O.IMPLICIT)
        err_gs = np.max(np.abs(a["I"] - ref["I"]))
        err_j = np.max(np.abs(b["I"] - ref["I"]))
        assert err_gs < 0.5 * err_j, (m, err_gs, err_j)


# ------------------------------------------------------ physics invariants
def test_uniform_equilibrium_stays_at_round_off():
    wl = W.cfg1()
    g = wl.geoms[0]
    W.uniform_walls(g, [W.BC_ISOTHERMAL, W.BC_SPECULAR, W.BC_ISOTHERMAL, W.BC_SPECULAR], [300.0, 0, 300.0, 0])
    p = O.Problem(g, O.dirs_for(wl.dirs), wl.bands)
    st = p.init_state(300.0)
    I_init = st["I"].copy()
    p.run(st, wl.dt, 20, 5)
    assert np.max(np.abs(st["I"] - I_init) / I_init) < 1e-14
    assert np.max(np.abs(st["TL"] - 300.0)) < 1e-14 * 300
    assert np.max(np.abs(st["Tp"] - 300.0)) < 1e-14 * 300
    p.run(st, 2e-13, 50, 1, O.EXPLICIT)
    assert np.max(np.abs(st["I"] - I_init) / I_init) < 1e-14


def _specular_box(nx, ny, ndir, nbands, seed):
    g = W.Geometry(2, nx, ny, 1, 10e-9, 10e-9, 10e-9)
    W.uniform_walls(g, [W.BC_SPECULAR] * 4, [0] * 4)
    bands = W.make_bands(nbands, 0, seed)
    p = O.Problem(g, O.dirs_inplane(ndir), bands)
    T0 = W.random_temperatures(nx * ny, seed + 1, 290.0, 310.0)
    return p, p.init_state(T0)


def _total_energy(p, I):
    return sum(p.cell_energy(I[P])[0] for P in range(p.nc))


def test_specular_enclosure_conserves_energy_explicit():
    p, st = _specular_box(8, 6, 8, 3, 11)
    E0 = _total_energy(p, st["I"])
    T0 = st["TL"].copy()
    p.run(st, 2e-13, 500, 1, O.EXPLICIT)
    E1 = _total_energy(p, st["I"])
    assert abs(E1 - E0) <= 1e-13 * E0
    assert np.max(np.abs(st["TL"] - T0)) > 0.5      # the field did evolve


def test_specular_enclosure_conserves_energy_implicit_converged():
    p, st = _specular_box(6, 5, 8, 3, 12)
    E0 = _total_energy(p, st["I"])
    p.run(st, 1e-12, 10, 80)
    E1 = _total_energy(p, st["I"])
    assert abs(E1 - E0) <= 1e-11 * E0


def _slab(nx, dx, dirs, bands, Th, Tc):
    g = W.Geometry(2, nx, 1, 1, dx, dx, dx)
    g.bc = [(W.BC_ISOTHERMAL, np.array([Th])), (W.BC_ISOTHERMAL, np.array([Tc])),
            (W.BC_SPECULAR, None), (W.BC_SPECULAR, None)]
    return O.Problem(g, dirs, bands)


@pytest.mark.parametrize("dirset", ["inplane16", "pa4x8"])
def test_ballistic_slab_matches_casimir_flux(dirset):
    if dirset == "inplane16":
        dirs = O.dirs_inplane(16)
        Mplus = (4 * math.pi / 16) / math.sin(math.pi / 16)
    else:
        dirs = O.dirs_polar_azim(4, 8)
        Mplus = math.pi
    bands = W.make_bands(4, 0, 5)
    bands.beta[:] = 0.0
    Th, Tc = 310.0, 300.0
    p = _slab(5, 10e-9, dirs, bands, Th, Tc)
    st = p.init_state(Tc)
    p.run(st, 1e-6, 4, 300)
    q, qw = p.flux(st["I"])
    exact = float(np.sum(O.I0(bands, Th)[0] - O.I0(bands, Tc)[0])) * Mplus
    assert np.all(np.abs(q[:, 0] - exact) <= 1e-10 * exact)
    assert abs(-qw[0] - exact) <= 1e-10 * exact      # into the domain at the hot wall
    assert abs(qw[1] - exact) <= 1e-10 * exact       # out at the cold wall


def test_diffusive_slab_matches_fourier_conduction():
    """Gray band with mean free path far below the slab: interior flux = -k dT/dx,
    k = tau v dI0/dT sum_d S_x^2 / w_d (Chapman-Enskog on the discrete set)."""
    v, tau = 1e3, 1e-11
    lam = v * tau
    dx = lam / 2
    nx = 80
    bands = W.Bands(np.array([0.0]), np.array([4e13]), np.array([v]), np.array([1.0 / tau]), np.array([1.0]))
    dirs = O.dirs_inplane(16)
    S, w, _ = dirs
    Th, Tc = 302.0, 298.0
    p = _slab(nx, dx, dirs, bands, Th, Tc)
    x = (np.arange(nx) + 0.5) / nx
    st = p.init_state(Th + (Tc - Th) * x)
    p.run(st, 5e-11, 240, 60)
    q, _ = p.flux(st["I"])
    T = st["TL"]
    inner = slice(nx // 4, 3 * nx // 4)
    xc = (np.arange(nx) + 0.5) * dx
    slope, icpt = np.polyfit(xc[inner], T[inner], 1)
    fit = slope * xc[inner] + icpt
    r2 = 1 - np.sum((T[inner] - fit) ** 2) / np.sum((T[inner] - T[inner].mean()) ** 2)
    assert r2 > 0.999
    Tm = float(T[inner].mean())
    dI0 = O.I0(bands, Tm)[1][0]
    k = tau * v * dI0 * float(np.sum(S[:, 0] ** 2 / w))
    qint = float(np.mean(q[inner, 0]))
    assert np.max(np.abs(q[inner, 0] - qint)) <= 1e-4 * abs(qint)       # steady: flux uniform
    assert abs(qint - (-k * slope)) <= 0.02 * abs(qint), (qint, -k * slope)


# ------------------------------------------------------ relabelling symmetry
def test_direction_relabelling_leaves_temperature_unchanged():
    wl = W.cfg1()
    g = wl.geoms[0]
    g.nx, g.ny = 7, 5
    W.uniform_walls(g, [W.BC_ISOTHERMAL, W.BC_SPECULAR, W.BC_ISOTHERMAL, W.BC_SPECULAR], [310.0, 0, 300.0, 0])
    S, w, r = O.dirs_inplane(16)
    perm = np.random.default_rng(3).permutation(16)
    inv = np.argsort(perm)
    S2, w2 = S[perm], w[perm]
    r2 = np.stack([inv[r[a][perm]] for a in range(3)]).astype(np.int32)
    T0 = W.random_temperatures(35, 4, 295.0, 305.0)
    out = []
    for dirs in ((S, w, r), (S2, w2, r2)):
        p = O.Problem(g, dirs, wl.bands)
        st = p.init_state(T0)
        p.run(st, wl.dt, 5, 4)
        out.append((st["TL"].copy(), st["Tp"].copy(), st["I"][:, inv if dirs[0] is S2 else slice(None)].copy()))
    assert np.max(np.abs(out[0][0] - out[1][0])) <= 1e-13 * 300
    assert np.max(np.abs(out[0][1] - out[1][1])) <= 1e-13 * 300
    assert np.max(np.abs(out[0][2] - out[1][2]) / out[0][2]) <= 1e-13


def test_mirrored_geometry_gives_mirrored_temperature():
    wl = W.cfg1()
    bands = wl.bands
    S, w, r = O.dirs_inplane(16)
    nx, ny = 6, 4
    T0 = W.random_temperatures(nx * ny, 8, 295.0, 305.0).reshape(ny, nx)
    res = []
    for mirror in (False, True):
        g = W.Geometry(2, nx, ny, 1, 10e-9, 10e-9, 10e-9)
        hot, cold = (W.BC_ISOTHERMAL, np.full(ny, 310.0)), (W.BC_SPECULAR, None)
        g.bc = [cold, hot] if mirror else [hot, cold]
        g.bc += [(W.BC_ISOTHERMAL, np.full(nx, 300.0)), (W.BC_SPECULAR, None)]
        p = O.Problem(g, (S, w, r), bands)
        st = p.init_state((T0[:, ::-1] if mirror else T0).ravel())
        p.run(st, wl.dt, 4, 4)
        T = st["TL"].reshape(ny, nx)
        res.append(T[:, ::-1] if mirror else T)
    assert np.max(np.abs(res[0] - res[1])) <= 1e-12 * 300


def test_temperature_dependent_relaxation_rate_is_measured_from_one_step():
    """beta_b(T) = beta_b (T_p / T_ref)^p (Sec. 2.2, tau depends on T): one
    explicit step of a single mirror-walled cell with an isotropic perturbation
    is pure relaxation, so each band's measured rate (I1 - I)/(dt (I0 - I))
    must equal beta_b (T_p/T_ref)^p at the cell's T_p (not at T_L, which
    differs here)."""
    g = W.Geometry(2, 1, 1, 1, 10e-9, 10e-9, 10e-9)
    W.uniform_walls(g, [W.BC_SPECULAR] * 4, [0.0] * 4)
    bands = W.make_bands(4, 1, 47)
    dirs = O.dirs_for(W.Dirs("inplane", n_inplane=8))
    p_exp, Tref, dt = 2.0, 300.0, 1e-13   # dt beta ~ 3e-4: stable, and I1 - I well above round-off
    prob = O.Problem(g, dirs, bands, beta_exp=p_exp, beta_Tref=Tref)
    st = prob.init_state(320.0)
    st["I"][0, :, 0] *= 1.01            # band 0 above its equilibrium, the same in every direction
    st["I"][0, :, 2] *= 0.995
    Tp, TL = prob.cell_temperatures(st["I"][0], 320.0, 320.0)
    assert abs(Tp - TL) > 1e-3            # the two temperatures differ, so the law's argument is checked
    st["Tp"][0], st["TL"][0] = Tp, TL
    st["I0"][0] = O.I0(bands, Tp)[0]
    I_before = st["I"].copy()
    prob.run(st, dt, 1, 1, O.EXPLICIT)
    for b in range(bands.nb):
        dI = st["I"][0, 3, b] - I_before[0, 3, b]
        drive = O.I0(bands, Tp)[0][b] - I_before[0, 3, b]
        if abs(drive) < 1e-12 * I_before[0, 3, b]:
            continue                        # bands at equilibrium do not move
        rate = dI / (dt * drive)
        assert abs(rate / (bands.beta[b] * (Tp / Tref) ** p_exp) - 1.0) <= 1e-10, b


def test_temperature_dependent_relaxation_conserves_energy():
    """Relaxation with beta_b(T_p) still conserves energy in a mirror box (the
    law's factor is common to all bands, so the T_p balance holds)."""
    g = W.Geometry(2, 5, 4, 1, 10e-9, 10e-9, 10e-9)
    W.uniform_walls(g, [W.BC_SPECULAR] * 4, [0.0] * 4)
    bands = W.make_bands(6, 2, 48)
    prob = O.Problem(g, O.dirs_for(W.Dirs("inplane", n_inplane=8)), bands, beta_exp=1.5, beta_Tref=300.0)
    st = prob.init_state(W.random_temperatures(20, 11, 280.0, 330.0))
    E0 = sum(prob.cell_energy(r)[0] for r in st["I"])
    prob.run(st, 2e-13, 50, 1, O.EXPLICIT)
    E1 = sum(prob.cell_energy(r)[0] for r in st["I"])
    assert abs(E1 - E0) <= 1e-13 * E0


def _diffuse_box(nx, ny, kinds):
    g = W.Geometry(2, nx, ny, 1, 10e-9, 10e-9, 10e-9)
    g.bc = [(k, None if k != W.BC_ISOTHERMAL else np.full(ny if s < 2 else nx, T)) for s, (k, T) in enumerate(kinds)]
    return g


def test_diffuse_enclosure_conserves_energy_and_its_walls_carry_no_net_flux():
    """A diffuse wall returns each band's whole outgoing energy flux, spread
    evenly over the incoming directions: a box of such walls conserves energy
    and every wall's net flux vanishes."""
    g = _diffuse_box(5, 4, [(W.BC_DIFFUSE, None)] * 4)
    bands = W.make_bands(5, 2, 49)
    prob = O.Problem(g, O.dirs_for(W.Dirs("polar_azim", n_polar=4, n_azim=8)), bands)
    st = prob.init_state(W.random_temperatures(20, 12, 280.0, 330.0))
    E0 = sum(prob.cell_energy(r)[0] for r in st["I"])
    prob.run(st, 2e-13, 40, 1, O.EXPLICIT)
    E1 = sum(prob.cell_energy(r)[0] for r in st["I"])
    assert abs(E1 - E0) <= 1e-13 * E0
    q, qw = prob.flux(st["I"])
    scale = np.max(np.abs(q))
    assert scale > 0 and np.all(np.abs(qw) <= 1e-12 * scale)


def test_diffuse_walls_keep_an_isotropic_equilibrium():
    g = _diffuse_box(4, 3, [(W.BC_DIFFUSE, None), (W.BC_ISOTHERMAL, 300.0), (W.BC_DIFFUSE, None), (W.BC_DIFFUSE, None)])
    g.bc[1] = (W.BC_ISOTHERMAL, np.full(3, 300.0))
    bands = W.make_bands(4, 1, 50)
    prob = O.Problem(g, O.dirs_for(W.Dirs("inplane", n_inplane=12)), bands)
    st = prob.init_state(300.0)
    I_start = st["I"].copy()
    prob.run(st, 1e-12, 5, 4)
    assert np.max(np.abs(st["I"] - I_start) / I_start) <= 1e-14


def test_diffuse_side_walls_scatter_heat_back():
    """Ballistic channel between a hot and a cold wall: rough (diffuse) side
    walls send phonons back, so less heat reaches the cold wall than with
    mirror side walls."""
    q_out = {}
    for side_kind in (W.BC_SPECULAR, W.BC_DIFFUSE):
        g = _diffuse_box(8, 3, [(W.BC_ISOTHERMAL, 310.0), (W.BC_ISOTHERMAL, 300.0), (side_kind, None), (side_kind, None)])
        bands = W.make_bands(3, 1, 51)
        bands.beta[:] = 1e6                     # nearly ballistic
        prob = O.Problem(g, O.dirs_for(W.Dirs("inplane", n_inplane=16)), bands)
        st = prob.init_state(300.0)
        prob.run(st, 1e-12, 60, 8)
        q_out[side_kind] = prob.flux(st["I"])[1][1]     # heat leaving through the cold +x wall
    assert q_out[W.BC_SPECULAR] > 0 and 0 < q_out[W.BC_DIFFUSE] < 0.9 * q_out[W.BC_SPECULAR], q_out


# ------------------------------------------------------ partially specular walls
def _partial_box(p_spec, nx=6, ny=5, seed=71):
    g = W.Geometry(2, nx, ny, 1, 10e-9, 10e-9, 10e-9)
    W.uniform_walls(g, [W.BC_PARTIAL] * 4, [p_spec] * 4)
    return g


def test_partial_specularity_reduces_to_mirror_and_diffuse_walls():
    """p = 1 is the mirror wall and p = 0 the diffuse wall, to the last bit."""
    bands = W.make_bands(4, 1, 72)
    dirs = O.dirs_inplane(12)
    T0 = W.random_temperatures(30, 73, 290.0, 310.0)
    for p_spec, kind in ((1.0, W.BC_SPECULAR), (0.0, W.BC_DIFFUSE)):
        a = O.Problem(_partial_box(p_spec), dirs, bands)
        gb = W.Geometry(2, 6, 5, 1, 10e-9, 10e-9, 10e-9)
        W.uniform_walls(gb, [kind] * 4, [0.0] * 4)
        b = O.Problem(gb, dirs, bands)
        sa, sb = a.init_state(T0), b.init_state(T0)
        a.run(sa, 1e-12, 3, 4)
        b.run(sb, 1e-12, 3, 4)
        assert np.array_equal(sa["I"], sb["I"]), p_spec


def test_one_explicit_step_is_the_specularity_mix_of_its_limits():
    """For one explicit step from a fixed state the update is linear in the
    ghost, and the ghost is p x mirror + (1 - p) x diffuse."""
    bands = W.make_bands(4, 1, 74)
    dirs = O.dirs_inplane(12)
    T0 = W.random_temperatures(30, 75, 290.0, 310.0)
    warm = O.Problem(_partial_box(0.5), dirs, bands)     # an anisotropic start: a few steps first
    start = warm.init_state(T0)
    warm.run(start, 2e-13, 5, 1, O.EXPLICIT)
    out = {}
    for p_spec in (0.0, 0.3, 1.0):
        pr = O.Problem(_partial_box(p_spec), dirs, bands)
        st = {k: v.copy() for k, v in start.items()}
        pr.run(st, 2e-13, 1, 1, O.EXPLICIT)
        out[p_spec] = st["I"]
    mix = 0.3 * out[1.0] + 0.7 * out[0.0]
    assert np.max(np.abs(out[0.3] - mix) / out[0.3]) < 1e-14
    assert np.max(np.abs(out[1.0] - out[0.0]) / out[0.3]) > 1e-6     # the limits differ


def test_partially_specular_enclosure_conserves_energy_with_no_net_wall_flux():
    pr = O.Problem(_partial_box(0.4), O.dirs_inplane(12), W.make_bands(4, 1, 76))
    st = pr.init_state(W.random_temperatures(30, 77, 290.0, 310.0))
    E0 = _total_energy(pr, st["I"])
    T0 = st["TL"].copy()
    pr.run(st, 2e-13, 200, 1, O.EXPLICIT)
    assert abs(_total_energy(pr, st["I"]) - E0) <= 1e-13 * E0
    assert np.max(np.abs(st["TL"] - T0)) > 0.1
    q, qw = pr.flux(st["I"])
    assert np.all(np.abs(qw) <= 1e-12 * np.max(np.abs(q)))
