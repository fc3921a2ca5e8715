"""Unstructured meshes as face lists: construction, generators and import
(Gmsh 2.2 ASCII ``.msh``, MEDIT ASCII ``.mesh``), the mesh inputs the method
accepts besides its internal structured generator (Sec. 3.3, mesh setup).

A mesh is held in the form the finite-volume update of Eq. 5 consumes:
cells with volumes (areas per unit depth in 2-D) and faces with an owner
cell, a neighbour cell (-1 on the boundary), the area vector n A pointing
out of the owner (edge length times unit normal in 2-D) and, on the boundary,
an integer tag (the physical group of the boundary element).  This module is
geometry only: it holds none of the transport arithmetic, so the oracle and
the CUDA path both take their mesh input from it.

Element vertex orders follow the Gmsh convention (line 1, triangle 2,
quadrangle 3, tetrahedron 4, hexahedron 5); MEDIT uses the same orders for
these elements.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# faces of each element kind as vertex-index tuples (Gmsh orders)
_FACETS = {
    "tri": ((0, 1), (1, 2), (2, 0)),
    "quad": ((0, 1), (1, 2), (2, 3), (3, 0)),
    "tet": ((0, 2, 1), (0, 1, 3), (0, 3, 2), (1, 2, 3)),
    "hex": ((0, 3, 2, 1), (0, 1, 5, 4), (0, 4, 7, 3), (1, 2, 6, 5), (2, 3, 7, 6), (4, 5, 6, 7)),
}
_GMSH_KIND = {2: "tri", 3: "quad", 4: "tet", 5: "hex"}
_GMSH_NVERT = {1: 2, 2: 3, 3: 4, 4: 4, 5: 8, 15: 1}
_DIM_OF = {"tri": 2, "quad": 2, "tet": 3, "hex": 3}


@dataclass
class UMesh:
    """Face-based unstructured mesh (see the module docstring)."""
    dim: int
    volume: np.ndarray          # [ncells]
    owner: np.ndarray           # [nfaces] int64
    neighbor: np.ndarray        # [nfaces] int64, -1 on the boundary
    nA: np.ndarray              # [nfaces, 3] area vector out of the owner
    tag: np.ndarray             # [nfaces] int32, boundary tag (-1 on interior faces)
    centroid: np.ndarray        # [ncells, 3] vertex mean of each cell
    face_center: np.ndarray     # [nfaces, 3]
    T_init: float = 300.0
    bc: dict = field(default_factory=dict)   # tag -> (kind, T or None), filled by the caller

    @property
    def ncells(self) -> int:
        return int(self.volume.shape[0])

    @property
    def nfaces(self) -> int:
        return int(self.owner.shape[0])

    @property
    def tags(self):
        return sorted(int(t) for t in np.unique(self.tag[self.neighbor < 0]))

    def boundary_faces(self, tag=None) -> np.ndarray:
        b = self.neighbor < 0
        if tag is not None:
            b &= self.tag == tag
        return np.nonzero(b)[0]

    def closure_residual(self) -> float:
        """max over cells of |sum of outward area vectors| / sum of areas (0 for closed cells)."""
        s = np.zeros((self.ncells, 3))
        a = np.zeros(self.ncells)
        area = np.linalg.norm(self.nA, axis=1)
        np.add.at(s, self.owner, self.nA)
        np.add.at(a, self.owner, area)
        inner = self.neighbor >= 0
        np.add.at(s, self.neighbor[inner], -self.nA[inner])
        np.add.at(a, self.neighbor[inner], area[inner])
        return float(np.max(np.linalg.norm(s, axis=1) / a))


def _facet_vector(pts: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Area vector (any orientation) and centre of a facet: a 2-D edge (two
    points, length times normal) or a 3-D polygon (vector area)."""
    c = pts.mean(axis=0)
    if len(pts) == 2:
        d = pts[1] - pts[0]
        return np.array([d[1], -d[0], 0.0]), c
    v = np.zeros(3)
    for i in range(len(pts)):
        v += np.cross(pts[i], pts[(i + 1) % len(pts)])
    return 0.5 * v, c


def from_elements(points: np.ndarray, elements: list[tuple[str, tuple]], boundary: dict | None = None,
                  default_tag: int = 0) -> UMesh:
    """Build the face list of a conforming mesh.

    points: [npts, 3] (z = 0 in 2-D); elements: (kind, vertex tuple) per cell,
    kind in tri/quad/tet/hex; boundary: {frozenset(facet vertices): tag} for the
    tagged boundary facets (other boundary facets get default_tag).  Each face
    gets its area vector oriented out of the owner (the cell that lists it
    first); the cell volume follows from the divergence theorem,
    V = (1/dim) sum_f x_f . (n A)_f, exact for planar facets."""
    points = np.asarray(points, dtype=np.float64)
    if points.shape[1] == 2:
        points = np.hstack([points, np.zeros((len(points), 1))])
    dims = {_DIM_OF[k] for k, _ in elements}
    if len(dims) != 1:
        raise ValueError("all cells of a mesh must have one dimension")
    dim = dims.pop()
    nc = len(elements)
    centroid = np.zeros((nc, 3))
    faces = {}
    owner, neighbor, nA, fc, tag = [], [], [], [], []
    for ci, (kind, verts) in enumerate(elements):
        v = np.asarray(verts, dtype=np.int64)
        centroid[ci] = points[v].mean(axis=0)
        for fac in _FACETS[kind]:
            key = frozenset(int(v[i]) for i in fac)
            if key in faces:
                fi = faces.pop(key)
                if neighbor[fi] != -1:
                    raise ValueError("a facet is shared by more than two cells")
                neighbor[fi] = ci
                continue
            vec, c = _facet_vector(points[v[list(fac)]])
            faces[key] = len(owner)
            owner.append(ci)
            neighbor.append(-1)
            nA.append(vec)
            fc.append(c)
            tag.append(-1)
    owner = np.asarray(owner, dtype=np.int64)
    neighbor = np.asarray(neighbor, dtype=np.int64)
    nA = np.asarray(nA)
    fc = np.asarray(fc)
    # orientation: out of the owner (its centroid lies behind the face)
    flip = np.einsum("ij,ij->i", fc - centroid[owner], nA) < 0
    nA[flip] *= -1.0
    tag = np.asarray(tag, dtype=np.int32)
    boundary = boundary or {}
    for key, fi in faces.items():  # facets left unmatched are the boundary
        tag[fi] = boundary.get(key, default_tag)
    # volumes by the divergence theorem
    vol = np.zeros(nc)
    contrib = np.einsum("ij,ij->i", fc, nA) / dim
    np.add.at(vol, owner, contrib)
    inner = neighbor >= 0
    np.add.at(vol, neighbor[inner], -contrib[inner])
    if np.any(vol <= 0):
        raise ValueError("a cell has a non-positive volume")
    return UMesh(dim, vol, owner, neighbor, nA, tag, centroid, fc)


# ---------------------------------------------------------------- generators
def _grid_points(nx, ny, Lx, Ly):
    x = np.linspace(0.0, Lx, nx + 1)
    y = np.linspace(0.0, Ly, ny + 1)
    X, Y = np.meshgrid(x, y)  # [ny+1][nx+1]
    return np.stack([X.ravel(), Y.ravel(), np.zeros(X.size)], axis=1)


def _rect_boundary(nx, ny):
    """Tags 0..3 = x-low, x-high, y-low, y-high edges of a rectangle grid."""
    vid = lambda i, j: j * (nx + 1) + i
    b = {}
    for j in range(ny):
        b[frozenset((vid(0, j), vid(0, j + 1)))] = 0
        b[frozenset((vid(nx, j), vid(nx, j + 1)))] = 1
    for i in range(nx):
        b[frozenset((vid(i, 0), vid(i + 1, 0)))] = 2
        b[frozenset((vid(i, ny), vid(i + 1, ny)))] = 3
    return b


def quad_grid(nx: int, ny: int, Lx: float, Ly: float) -> UMesh:
    """nx x ny rectangles, cells numbered x fastest (the structured order)."""
    vid = lambda i, j: j * (nx + 1) + i
    el = [("quad", (vid(i, j), vid(i + 1, j), vid(i + 1, j + 1), vid(i, j + 1))) for j in range(ny) for i in range(nx)]
    return from_elements(_grid_points(nx, ny, Lx, Ly), el, _rect_boundary(nx, ny))


def tri_grid(nx: int, ny: int, Lx: float, Ly: float, jitter: float = 0.0, seed: int = 0) -> UMesh:
    """Each rectangle of an nx x ny grid split into two triangles (alternating
    diagonals); interior vertices moved by up to jitter x the spacing."""
    pts = _grid_points(nx, ny, Lx, Ly)
    if jitter:
        rng = np.random.default_rng(seed)
        inner = np.array([0 < i < nx and 0 < j < ny for j in range(ny + 1) for i in range(nx + 1)])
        d = rng.uniform(-jitter, jitter, (inner.sum(), 2)) * np.array([Lx / nx, Ly / ny])
        pts[inner, :2] += d
    vid = lambda i, j: j * (nx + 1) + i
    el = []
    for j in range(ny):
        for i in range(nx):
            a, b, c, d = vid(i, j), vid(i + 1, j), vid(i + 1, j + 1), vid(i, j + 1)
            if (i + j) % 2 == 0:
                el += [("tri", (a, b, c)), ("tri", (a, c, d))]
            else:
                el += [("tri", (a, b, d)), ("tri", (b, c, d))]
    return from_elements(pts, el, _rect_boundary(nx, ny))


def tet_box(nx: int, ny: int, nz: int, Lx: float, Ly: float, Lz: float) -> UMesh:
    """Each box of an nx x ny x nz grid split into six tetrahedra around its
    main diagonal; tags 0..5 = x-low, x-high, y-low, y-high, z-low, z-high."""
    x, y, z = np.linspace(0, Lx, nx + 1), np.linspace(0, Ly, ny + 1), np.linspace(0, Lz, nz + 1)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    vid = lambda i, j, k: (k * (ny + 1) + j) * (nx + 1) + i
    el = []
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                c = [vid(i + a, j + b, k + e) for e in (0, 1) for b in (0, 1) for a in (0, 1)]  # c[a + 2b + 4e]
                v0, v7 = c[0], c[7]
                for p, q in ((1, 3), (3, 2), (2, 6), (6, 4), (4, 5), (5, 1)):
                    el.append(("tet", (v0, c[p], c[q], v7)))
    b = {}
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                c = [vid(i + a, j + bb, k + e) for e in (0, 1) for bb in (0, 1) for a in (0, 1)]
                if i == 0: b.update(_box_face_tris(c, (0, 2, 6, 4), 0))
                if i == nx - 1: b.update(_box_face_tris(c, (1, 3, 7, 5), 1))
                if j == 0: b.update(_box_face_tris(c, (0, 1, 5, 4), 2))
                if j == ny - 1: b.update(_box_face_tris(c, (2, 3, 7, 6), 3))
                if k == 0: b.update(_box_face_tris(c, (0, 1, 3, 2), 4))
                if k == nz - 1: b.update(_box_face_tris(c, (4, 5, 7, 6), 5))
    return from_elements(pts, el, b)


def wedge_ring(nr: int, nz: int, r_in: float, r_out: float, Lz: float, alpha: float, nwedge: int = 1) -> UMesh:
    """A hollow cylinder about the z axis cut into wedges of angle alpha, each
    wedge nr x nz hexahedral cells in (r, z) with planar faces; the first wedge
    spans theta in [-alpha/2, alpha/2] (centred on +x) and wedge k is the first
    rotated by k alpha.  nwedge = 1 gives the one-cell-thick wedge of an
    axisymmetric problem; nwedge * alpha = 2 pi the full ring.  Cells are
    numbered (wedge, iz, ir) with ir fastest.  Tags: 0 the inner surface
    (r = r_in), 1 the outer one, 2 z = 0, 3 z = Lz, and on an open ring 4 the
    side at theta = -alpha/2 and 5 the side at theta = -alpha/2 + nwedge alpha."""
    if not (0.0 < r_in < r_out) or nr < 1 or nz < 1 or nwedge < 1 or not (0.0 < alpha * nwedge <= 2.0 * np.pi + 1e-12):
        raise ValueError("need 0 < r_in < r_out, nr, nz, nwedge >= 1 and nwedge * alpha <= 2 pi")
    closed = abs(alpha * nwedge - 2.0 * np.pi) < 1e-9
    nk = nwedge if closed else nwedge + 1        # distinct angle lines
    r = np.linspace(r_in, r_out, nr + 1)
    z = np.linspace(0.0, Lz, nz + 1)
    pts = []
    for k in range(nk):
        th = -0.5 * alpha + k * alpha
        for iz in range(nz + 1):
            for ir in range(nr + 1):
                pts.append((r[ir] * np.cos(th), r[ir] * np.sin(th), z[iz]))
    vid = lambda k, ir, iz: ((k % nk) * (nz + 1) + iz) * (nr + 1) + ir
    el, b = [], {}
    for k in range(nwedge):
        for iz in range(nz):
            for ir in range(nr):
                el.append(("hex", (vid(k, ir, iz), vid(k, ir + 1, iz), vid(k + 1, ir + 1, iz), vid(k + 1, ir, iz),
                                   vid(k, ir, iz + 1), vid(k, ir + 1, iz + 1), vid(k + 1, ir + 1, iz + 1),
                                   vid(k + 1, ir, iz + 1))))
        for iz in range(nz):
            b[frozenset((vid(k, 0, iz), vid(k + 1, 0, iz), vid(k + 1, 0, iz + 1), vid(k, 0, iz + 1)))] = 0
            b[frozenset((vid(k, nr, iz), vid(k + 1, nr, iz), vid(k + 1, nr, iz + 1), vid(k, nr, iz + 1)))] = 1
        for ir in range(nr):
            b[frozenset((vid(k, ir, 0), vid(k, ir + 1, 0), vid(k + 1, ir + 1, 0), vid(k + 1, ir, 0)))] = 2
            b[frozenset((vid(k, ir, nz), vid(k, ir + 1, nz), vid(k + 1, ir + 1, nz), vid(k + 1, ir, nz)))] = 3
    if not closed:
        for iz in range(nz):
            for ir in range(nr):
                b[frozenset((vid(0, ir, iz), vid(0, ir + 1, iz), vid(0, ir + 1, iz + 1), vid(0, ir, iz + 1)))] = 4
                b[frozenset((vid(nwedge, ir, iz), vid(nwedge, ir + 1, iz), vid(nwedge, ir + 1, iz + 1),
                             vid(nwedge, ir, iz + 1)))] = 5
    return from_elements(np.array(pts), el, b)


def _box_face_tris(c, quad, t):
    """Both triangulations of a box face (the split around the main diagonal
    uses one of them); each triangle keyed to tag t."""
    a, b_, cc, d = (c[q] for q in quad)
    return {frozenset((a, b_, cc)): t, frozenset((a, cc, d)): t, frozenset((a, b_, d)): t, frozenset((b_, cc, d)): t}


# ---------------------------------------------------------------- file import
def read_gmsh(path: str) -> UMesh:
    """Gmsh 2.2 ASCII: $Nodes and $Elements; cells are the elements of the
    highest dimension (triangles/quadrangles or tetrahedra/hexahedra), boundary
    tags the first (physical) tag of the lower-dimensional elements."""
    with open(path) as f:
        lines = [ln.strip() for ln in f]
    i = 0
    nodes, elems = {}, []
    while i < len(lines):
        if lines[i] == "$MeshFormat":
            ver = lines[i + 1].split()
            if not ver[0].startswith("2") or ver[1] != "0":
                raise ValueError("only Gmsh 2.x ASCII files are read")
            i += 3
        elif lines[i] == "$Nodes":
            n = int(lines[i + 1])
            for k in range(n):
                p = lines[i + 2 + k].split()
                nodes[int(p[0])] = [float(p[1]), float(p[2]), float(p[3])]
            i += n + 3
        elif lines[i] == "$Elements":
            n = int(lines[i + 1])
            for k in range(n):
                p = [int(x) for x in lines[i + 2 + k].split()]
                etype, ntags = p[1], p[2]
                tags = p[3:3 + ntags]
                verts = tuple(p[3 + ntags:3 + ntags + _GMSH_NVERT.get(etype, 0)])
                elems.append((etype, tags[0] if tags else 0, verts))
            i += n + 3
        else:
            i += 1
    ids = sorted(nodes)
    index = {v: k for k, v in enumerate(ids)}
    pts = np.array([nodes[v] for v in ids])
    cell_types = [t for t, _, _ in elems if t in _GMSH_KIND]
    if not cell_types:
        raise ValueError("no cells in the file")
    top = max(_DIM_OF[_GMSH_KIND[t]] for t in cell_types)
    cells = [(_GMSH_KIND[t], tuple(index[v] for v in vs)) for t, _, vs in elems
             if t in _GMSH_KIND and _DIM_OF[_GMSH_KIND[t]] == top]
    facet_types = (1,) if top == 2 else (2, 3)
    boundary = {frozenset(index[v] for v in vs): tg for t, tg, vs in elems if t in facet_types}
    return from_elements(pts, cells, boundary)


def write_gmsh(path: str, points: np.ndarray, elements: list[tuple[str, tuple]], boundary_facets: list[tuple[int, tuple]]):
    """Gmsh 2.2 ASCII writer for the same element kinds (1-based node ids)."""
    code = {v: k for k, v in _GMSH_KIND.items()}
    with open(path, "w") as f:
        f.write("$MeshFormat\n2.2 0 8\n$EndMeshFormat\n$Nodes\n%d\n" % len(points))
        for k, p in enumerate(points):
            f.write("%d %.17g %.17g %.17g\n" % (k + 1, p[0], p[1], p[2] if len(p) > 2 else 0.0))
        f.write("$EndNodes\n$Elements\n%d\n" % (len(elements) + len(boundary_facets)))
        n = 0
        for tg, vs in boundary_facets:
            n += 1
            t = 1 if len(vs) == 2 else (2 if len(vs) == 3 else 3)
            f.write("%d %d 2 %d %d %s\n" % (n, t, tg, tg, " ".join(str(v + 1) for v in vs)))
        for kind, vs in elements:
            n += 1
            f.write("%d %d 2 1 1 %s\n" % (n, code[kind], " ".join(str(v + 1) for v in vs)))
        f.write("$EndElements\n")


def read_medit(path: str) -> UMesh:
    """MEDIT ASCII (.mesh): Dimension, Vertices, and Edges / Triangles /
    Quadrilaterals / Tetrahedra / Hexahedra with a trailing reference each;
    the references of the boundary facets become the tags."""
    with open(path) as f:
        tok = f.read().split()
    i = 0
    dim, pts = 3, None
    blocks = {}
    nv = {"Edges": 2, "Triangles": 3, "Quadrilaterals": 4, "Tetrahedra": 4, "Hexahedra": 8}
    while i < len(tok):
        w = tok[i]
        if w == "Dimension":
            dim = int(tok[i + 1]); i += 2
        elif w == "Vertices":
            n = int(tok[i + 1]); i += 2
            pts = np.zeros((n, 3))
            for k in range(n):
                pts[k, :dim] = [float(x) for x in tok[i:i + dim]]
                i += dim + 1
        elif w in nv:
            n = int(tok[i + 1]); i += 2
            m = nv[w]
            rows = []
            for k in range(n):
                rows.append(([int(x) - 1 for x in tok[i:i + m]], int(tok[i + m])))
                i += m + 1
            blocks[w] = rows
        else:
            i += 1
    if pts is None:
        raise ValueError("no vertices in the file")
    kinds3 = (("Tetrahedra", "tet"), ("Hexahedra", "hex"))
    kinds2 = (("Triangles", "tri"), ("Quadrilaterals", "quad"))
    cell_kinds = kinds3 if any(k in blocks for k, _ in kinds3) else kinds2
    cells = [(kind, tuple(v)) for name, kind in cell_kinds for v, _ in blocks.get(name, [])]
    facet_names = ("Triangles", "Quadrilaterals") if cell_kinds is kinds3 else ("Edges",)
    boundary = {frozenset(v): ref for name in facet_names for v, ref in blocks.get(name, [])}
    return from_elements(pts, cells, boundary)


def write_medit(path: str, points: np.ndarray, elements: list[tuple[str, tuple]],
                boundary_facets: list[tuple[int, tuple]], dim: int):
    names = {"tri": "Triangles", "quad": "Quadrilaterals", "tet": "Tetrahedra", "hex": "Hexahedra"}
    with open(path, "w") as f:
        f.write("MeshVersionFormatted 2\nDimension %d\nVertices\n%d\n" % (dim, len(points)))
        for p in points:
            f.write(" ".join("%.17g" % x for x in p[:dim]) + " 0\n")
        facets = {}
        for tg, vs in boundary_facets:
            name = "Edges" if len(vs) == 2 else ("Triangles" if len(vs) == 3 else "Quadrilaterals")
            facets.setdefault(name, []).append((vs, tg))
        for name, rows in facets.items():
            f.write("%s\n%d\n" % (name, len(rows)))
            for vs, tg in rows:
                f.write(" ".join(str(v + 1) for v in vs) + " %d\n" % tg)
        by = {}
        for kind, vs in elements:
            by.setdefault(names[kind], []).append(vs)
        for name, rows in by.items():
            f.write("%s\n%d\n" % (name, len(rows)))
            for vs in rows:
                f.write(" ".join(str(v + 1) for v in vs) + " 1\n")
        f.write("End\n")
