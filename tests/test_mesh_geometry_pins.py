"""Pins of the mesh geometry that the oracle's unstructured update and the CUDA
path both consume (cell volumes V and face area vectors n A of Eq. 5's face
sum).  Each expected value here comes from a formula that mesh.py does not
use: hand-worked single elements, element volumes by determinants (mesh.py
uses the divergence theorem over the facets), facet area vectors from the
element's own vertices with the orientation taken from the vertex opposite
the facet (mesh.py orients by the cell centroid), per-cell closure summed
here from the face list, and the Gmsh and MEDIT readings of one mesh."""
import numpy as np
import pytest

from paper_2305_19400_gb300 import mesh as M


def _face_index(m):
    """{frozenset of owner/neighbour cells and rounded face centre: face id}."""
    return {tuple(np.round(m.face_center[f] * 1e12).astype(np.int64)): f for f in range(m.nfaces)}


def test_hand_worked_triangle():
    # right triangle (0,0) (3,0) (0,4): area 6; edges of length 3, 5, 4 with
    # outward normals (0,-1), (4,3)/5, (-1,0)
    m = M.from_elements(np.array([[0.0, 0.0], [3.0, 0.0], [0.0, 4.0]]), [("tri", (0, 1, 2))])
    assert m.dim == 2 and m.ncells == 1 and m.nfaces == 3
    assert m.volume[0] == pytest.approx(6.0, rel=1e-15)
    got = {tuple(np.round(c, 12)): v for c, v in zip(m.face_center, m.nA)}
    want = {(1.5, 0.0, 0.0): (0.0, -3.0, 0.0), (1.5, 2.0, 0.0): (4.0, 3.0, 0.0), (0.0, 2.0, 0.0): (-4.0, 0.0, 0.0)}
    assert set(got) == set(want)
    for k, v in want.items():
        assert np.allclose(got[k], v, rtol=0, atol=1e-14), (k, got[k], v)


def test_hand_worked_tetrahedron():
    # corner tetrahedron (0,0,0) (1,0,0) (0,2,0) (0,0,3): volume 1 x 2 x 3 / 6 = 1;
    # faces z=0 (area 1), y=0 (1.5), x=0 (3) and the slanted face x + y/2 + z/3 = 1,
    # whose area vector is half the cross product of two edges: (3, 1.5, 1)
    pts = np.array([[0, 0, 0], [1, 0, 0], [0, 2, 0], [0, 0, 3]], dtype=float)
    m = M.from_elements(pts, [("tet", (0, 1, 2, 3))])
    assert m.dim == 3 and m.nfaces == 4
    assert m.volume[0] == pytest.approx(1.0, rel=1e-15)
    want = {(1 / 3, 2 / 3, 0.0): (0, 0, -1.0), (1 / 3, 0.0, 1.0): (0, -1.5, 0), (0.0, 2 / 3, 1.0): (-3.0, 0, 0),
            (1 / 3, 2 / 3, 1.0): (3.0, 1.5, 1.0)}
    got = {tuple(np.round(c, 12)): v for c, v in zip(m.face_center, m.nA)}
    assert set(got) == {tuple(np.round(k, 12)) for k in want}
    for k, v in want.items():
        assert np.allclose(got[tuple(np.round(k, 12))], v, rtol=0, atol=1e-14)
    # the same tetrahedron listed with the other vertex order (negative orientation)
    m2 = M.from_elements(pts, [("tet", (0, 2, 1, 3))])
    assert m2.volume[0] == pytest.approx(1.0, rel=1e-15)


def _jittered_elements(kind, seed):
    """A small jittered mesh as (points, elements); kinds tri (2-D) or tet (3-D)."""
    rng = np.random.default_rng(seed)
    if kind == "tri":
        nx, ny, L = 5, 4, 1e-7
        x, y = np.meshgrid(np.linspace(0, L, nx + 1), np.linspace(0, L, ny + 1))
        pts = np.stack([x.ravel(), y.ravel(), np.zeros(x.size)], 1)
        inner = (pts[:, 0] > 0) & (pts[:, 0] < L) & (pts[:, 1] > 0) & (pts[:, 1] < L)
        pts[inner, :2] += rng.uniform(-0.3, 0.3, (inner.sum(), 2)) * L / 5
        vid = lambda i, j: j * (nx + 1) + i
        el = []
        for j in range(ny):
            for i in range(nx):
                a, b, c, d = vid(i, j), vid(i + 1, j), vid(i + 1, j + 1), vid(i, j + 1)
                el += [("tri", (a, b, c)), ("tri", (a, c, d))] if (i + j) % 2 else [("tri", (a, b, d)), ("tri", (b, c, d))]
        return pts, el, L * L
    n, L = 2, 1e-7
    g = np.linspace(0, L, n + 1)
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    inner = np.all((pts > 0) & (pts < L), axis=1)
    pts[inner] += rng.uniform(-0.2, 0.2, (inner.sum(), 3)) * L / n
    vid = lambda i, j, k: (k * (n + 1) + j) * (n + 1) + i
    el = []
    for k in range(n):
        for j in range(n):
            for i in range(n):
                c = [vid(i + a, j + b, k + e) for e in (0, 1) for b in (0, 1) for a in (0, 1)]
                for p, q in ((1, 3), (3, 2), (2, 6), (6, 4), (4, 5), (5, 1)):
                    el.append(("tet", (c[0], c[p], c[q], c[7])))
    return pts, el, L ** 3


@pytest.mark.parametrize("kind,seed", [("tri", 3), ("tri", 4), ("tet", 5)])
def test_volumes_and_area_vectors_against_determinants(kind, seed):
    pts, el, total = _jittered_elements(kind, seed)
    m = M.from_elements(pts, el)
    # cell volumes: |det| / 2 (triangle) or |det| / 6 (tetrahedron) of the edge vectors
    for ci, (_, v) in enumerate(el):
        P = pts[list(v)]
        E = (P[1:] - P[0])[:, :2] if kind == "tri" else P[1:] - P[0]
        vol = abs(np.linalg.det(E)) / (2.0 if kind == "tri" else 6.0)
        assert m.volume[ci] == pytest.approx(vol, rel=1e-12)
    assert m.volume.sum() == pytest.approx(total, rel=1e-12)
    # every facet of every element: the area vector from the vertices, pointing
    # away from the element's vertex that is not on the facet
    idx = _face_index(m)
    nfacet = 3 if kind == "tri" else 4
    for ci, (_, v) in enumerate(el):
        for skip in range(nfacet):
            fv = [v[i] for i in range(nfacet) if i != skip]
            P = pts[fv]
            if kind == "tri":
                d = P[1] - P[0]
                vec = np.array([d[1], -d[0], 0.0])
            else:
                vec = 0.5 * np.cross(P[1] - P[0], P[2] - P[0])
            if np.dot(pts[v[skip]] - P[0], vec) > 0:
                vec = -vec  # outward from this element
            f = idx[tuple(np.round(P.mean(0) * 1e12).astype(np.int64))]
            assert ci in (m.owner[f], m.neighbor[f])
            sign = 1.0 if m.owner[f] == ci else -1.0  # nA points out of the owner
            scale = np.linalg.norm(vec)
            assert np.allclose(sign * m.nA[f], vec, rtol=0, atol=1e-12 * scale)


@pytest.mark.parametrize("kind,seed", [("tri", 6), ("tet", 7)])
def test_every_cell_is_closed(kind, seed):
    """sum over a cell's faces of its outward area vectors is zero (summed here
    from the face list, with the neighbour's sign flipped)."""
    pts, el, _ = _jittered_elements(kind, seed)
    m = M.from_elements(pts, el)
    s = np.zeros((m.ncells, 3))
    area = np.zeros(m.ncells)
    for f in range(m.nfaces):
        s[m.owner[f]] += m.nA[f]
        area[m.owner[f]] += np.linalg.norm(m.nA[f])
        if m.neighbor[f] >= 0:
            s[m.neighbor[f]] -= m.nA[f]
            area[m.neighbor[f]] += np.linalg.norm(m.nA[f])
    assert np.max(np.linalg.norm(s, axis=1) / area) < 1e-14
    # the boundary's area vectors close the domain as well
    b = m.neighbor < 0
    assert np.linalg.norm(m.nA[b].sum(0)) < 1e-14 * np.linalg.norm(m.nA[b], axis=1).sum()


def test_gmsh_and_medit_readings_of_one_tetrahedral_mesh_are_identical(tmp_path):
    pts, el, _ = _jittered_elements("tet", 8)
    ref = M.from_elements(pts, el)
    # the boundary triangles, tagged by the box side they lie on
    bf = []
    L = pts.max()
    for f in ref.boundary_faces():
        c = ref.face_center[f]
        side = int(np.argmax(np.abs(ref.nA[f])))
        t = 2 * side + (1 if c[side] > 0.5 * L else 0)
        cell = el[ref.owner[f]][1]
        fv = [w for w in cell if np.isclose(pts[w][side], c[side], rtol=0, atol=1e-20)]
        assert len(fv) == 3
        bf.append((t, tuple(fv)))
    g, md = str(tmp_path / "m.msh"), str(tmp_path / "m.mesh")
    M.write_gmsh(g, pts, el, bf)
    M.write_medit(md, pts, el, bf, 3)
    a, b = M.read_gmsh(g), M.read_medit(md)
    for m in (a, b):
        assert m.ncells == ref.ncells and m.nfaces == ref.nfaces
        assert np.array_equal(m.volume, ref.volume)
        assert np.array_equal(m.nA, ref.nA)
    assert np.array_equal(a.owner, b.owner) and np.array_equal(a.neighbor, b.neighbor)
    assert np.array_equal(a.tag, b.tag) and a.tags == [0, 1, 2, 3, 4, 5]
