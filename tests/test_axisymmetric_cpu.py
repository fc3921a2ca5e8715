"""Axisymmetric problems (the reduced configurations Sec. 3.1 mentions for
problems with axial symmetry): one wedge of a body of revolution about the z
axis, one cell thick in the azimuth, whose two side faces are rotationally
periodic.  Across a side face lies the wedge itself rotated by the wedge
angle alpha, so by symmetry the ghost of direction s there is the cell's own
intensity in s rotated back by alpha; when alpha is the azimuthal bin width
of the direction set, that is the neighbouring azimuthal bin, and the flux
through the side faces is the discrete angular-redistribution term of the
axisymmetric transport equation.

The oracle's rotational faces are pinned against a computation that does not
use them: the full ring of wedges (every wedge a rotated copy, joined by
interior faces) solved by the already pinned unstructured update.  The
wedge's temperatures must equal those of every wedge of the ring, and its
intensities those of wedge k after rotating the directions by k bins; planted
mistakes (the rotation's sense reversed, no rotation) move T by about 1e-4.
Also pinned: equilibrium, energy conservation in a closed wedge, and the
refusal of a wedge angle that is no symmetry of the direction set."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2305_19400_gb300 import mesh as M, workloads as W


def _case(nphi, ntheta=4, nr=3, nz=4):
    alpha = 2 * np.pi / nphi
    dirs = W.Dirs("polar_azim", n_polar=ntheta, n_azim=nphi)
    args = (nr, nz, 20e-9, 60e-9, 40e-9, alpha)
    return alpha, dirs, M.wedge_ring(*args), M.wedge_ring(*args, nwedge=nphi)


@pytest.mark.parametrize("nphi,ntheta", [(8, 4), (12, 6)])
@pytest.mark.parametrize("scheme,dt,nsteps,ninner", [(O.IMPLICIT, 1e-12, 3, 5), (O.EXPLICIT, 2e-13, 15, 1)])
def test_wedge_with_rotational_sides_equals_the_full_ring(nphi, ntheta, scheme, dt, nsteps, ninner):
    alpha, dirs, wedge, ring = _case(nphi, ntheta)
    bands = W.make_bands(6, 2, 71)
    # hot inner surface, cold outer one, a mirror floor and a diffuse lid
    bc = {0: (O.ISOTHERMAL, 310.0), 1: (O.ISOTHERMAL, 300.0), 2: (O.SPECULAR, None), 3: (O.DIFFUSE, None)}
    D = O.dirs_for(dirs)
    pw = O.UMeshProblem(wedge, D, bands, {**bc, 4: (O.ROTATIONAL, alpha), 5: (O.ROTATIONAL, alpha)})
    sw = pw.init_state(300.0)
    pw.run(sw, dt, nsteps, ninner, scheme)
    pr = O.UMeshProblem(ring, D, bands, bc)
    sr = pr.init_state(300.0)
    pr.run(sr, dt, nsteps, ninner, scheme)
    nc = wedge.ncells
    assert sw["TL"].max() > 300.05          # heat has entered from the inner surface
    for k in range(nphi):
        for key in ("TL", "Tp"):
            assert np.max(np.abs(sr[key][k * nc:(k + 1) * nc] - sw[key]) / sw[key]) <= 1e-13
        rot = np.array([i * nphi + (j - k) % nphi for i in range(ntheta) for j in range(nphi)])
        Ik = sr["I"][k * nc:(k + 1) * nc]
        assert np.max(np.abs(Ik - sw["I"][:, rot, :]) / np.abs(Ik)) <= 1e-13


def test_uniform_equilibrium_in_a_wedge_stays_put():
    alpha, dirs, wedge, _ = _case(8)
    bands = W.make_bands(5, 2, 72)
    bc = {0: (O.ISOTHERMAL, 300.0), 1: (O.DIFFUSE, None), 2: (O.SPECULAR, None), 3: (O.ISOTHERMAL, 300.0),
          4: (O.ROTATIONAL, alpha), 5: (O.ROTATIONAL, alpha)}
    p = O.UMeshProblem(wedge, O.dirs_for(dirs), bands, bc)
    st = p.init_state(300.0)
    I0 = st["I"].copy()
    p.run(st, 1e-12, 10, 4)
    assert np.max(np.abs(st["I"] - I0) / I0) <= 1e-13
    assert np.max(np.abs(st["TL"] - 300.0)) <= 1e-12 * 300


def test_closed_wedge_conserves_energy():
    """Diffuse inner and outer surfaces, mirror floor and lid, rotational sides:
    no energy crosses any face, so sum_P V_P E_L(P) stays fixed (explicit scheme)."""
    alpha, dirs, wedge, _ = _case(8)
    bands = W.make_bands(8, 3, 73)
    bc = {0: (O.DIFFUSE, None), 1: (O.DIFFUSE, None), 2: (O.SPECULAR, None), 3: (O.SPECULAR, None),
          4: (O.ROTATIONAL, alpha), 5: (O.ROTATIONAL, alpha)}
    p = O.UMeshProblem(wedge, O.dirs_for(dirs), bands, bc)
    st = p.init_state(W.random_temperatures(wedge.ncells, 74, 290.0, 315.0))

    def energy():
        return sum(wedge.volume[P] * p.cell_energy(st["I"][P])[0] for P in range(wedge.ncells))

    E0 = energy()
    p.run(st, 2e-13, 60, 1, O.EXPLICIT)
    assert abs(energy() - E0) <= 1e-13 * E0
    assert np.ptp(st["TL"]) > 0.1            # the field is far from uniform: the walls really exchanged energy


def test_a_wedge_angle_that_is_no_rotation_of_the_direction_set_is_refused():
    alpha, dirs, wedge, _ = _case(8)
    bad = 2 * np.pi / 7
    wedge7 = M.wedge_ring(3, 4, 20e-9, 60e-9, 40e-9, bad)
    bc = {0: (O.ISOTHERMAL, 305.0), 1: (O.ISOTHERMAL, 300.0), 2: (O.SPECULAR, None), 3: (O.SPECULAR, None),
          4: (O.ROTATIONAL, bad), 5: (O.ROTATIONAL, bad)}
    p = O.UMeshProblem(wedge7, O.dirs_for(dirs), W.make_bands(4, 1, 75), bc)
    st = p.init_state(300.0)
    with pytest.raises(RuntimeError, match="rotation"):
        p.run(st, 1e-12, 1, 1)


def test_wedge_mesh_volumes_and_faces():
    """The generator's cells are the planar-faced trapezoidal prisms of the
    wedge: volumes from the trapezoid area times the height, side faces through
    the axis at -+alpha/2, inner and outer faces normal to +x."""
    alpha, _, wedge, ring = _case(8)
    half = 0.5 * alpha
    r = np.linspace(20e-9, 60e-9, 4)
    dz = 10e-9
    area = 0.5 * np.sin(alpha) * (r[1:] ** 2 - r[:-1] ** 2)
    assert np.allclose(wedge.volume.reshape(4, 3), (area * dz)[None, :], rtol=1e-12, atol=0)
    assert np.isclose(ring.volume.sum(), 8 * wedge.volume.sum(), rtol=1e-13)
    for t, ang in ((4, -half), (5, half)):
        f = wedge.boundary_faces(t)
        n = wedge.nA[f] / np.linalg.norm(wedge.nA[f], axis=1)[:, None]
        sgn = 1.0 if t == 5 else -1.0
        assert np.allclose(n, sgn * np.array([-np.sin(ang), np.cos(ang), 0.0])[None, :], atol=1e-12)
        assert np.allclose(np.einsum("ij,ij->i", wedge.face_center[f], n), 0.0, atol=1e-20)   # planes through the axis
    for t, sgn in ((0, -1.0), (1, 1.0)):
        f = wedge.boundary_faces(t)
        n = wedge.nA[f] / np.linalg.norm(wedge.nA[f], axis=1)[:, None]
        assert np.allclose(n, [[sgn, 0.0, 0.0]], atol=1e-12)
