"""Seeded polyhedral meshes of the unit cube and subdomain partitions.

Mesh layout (the one the library's ``vem_mesh`` takes):

* ``xyz``      float64 [nV, 3]  vertex coordinates.
* ``face_ptr`` int32 [nF+1], ``face_vtx`` int32: each face is a planar
  vertex loop; its orientation (right-hand rule) fixes the global face
  normal.
* ``elem_ptr`` int32 [nE+1], ``elem_face`` int32: signed face references,
  ``+(f+1)`` if the global normal of face ``f`` points out of the element,
  ``-(f+1)`` otherwise.

The CUBE family is an ``n x n x n`` grid of hexahedra (each a VEM polyhedron
with 6 quadrilateral faces).  Interior vertices may be moved by i.i.d.
uniform offsets in ``[-a h, a h]^3`` drawn in lexicographic vertex order
(x, then y, then z of each vertex).  A moved hexahedron has non-planar
quadrilaterals, so every quadrilateral is then split into two triangles
along the diagonal through its smallest-index vertex, giving polyhedra with
8 vertices, 18 edges and 12 triangular faces.

The OCTA family (``octa_mesh``) embeds an octahedron at the centre of every
``2 x 2 x 2`` block of grid cubes; its vertex, edge and face counts
reproduce the DOF counts the paper prints for its OCTA meshes.  The CVT
family (``cvt_mesh``) is a seeded, Lloyd-relaxed centroidal Voronoi
tessellation of the cube (general convex polyhedra, faces of up to about 9
vertices).
"""
import numpy as np


def _vid(n, i, j, l):
    return i + (n + 1) * (j + (n + 1) * l)


def cube_mesh(n, perturb=0.0, seed=None, split_quads=None):
    """Uniform ``n^3`` hexahedral mesh of [0,1]^3, optionally perturbed.

    ``perturb`` is the offset bound as a fraction of h = 1/n.  ``split_quads``
    defaults to ``perturb > 0``.
    """
    if split_quads is None:
        split_quads = perturb > 0.0
    h = 1.0 / n
    idx = np.arange(n + 1)
    L, J, I = np.meshgrid(idx, idx, idx, indexing="ij")
    xyz = np.stack([I.ravel(), J.ravel(), L.ravel()], axis=1).astype(np.float64) * h
    if perturb > 0.0:
        rng = np.random.default_rng(seed)
        off = rng.uniform(-perturb * h, perturb * h, size=xyz.shape)
        ii, jj, ll = I.ravel(), J.ravel(), L.ravel()
        interior = (ii > 0) & (ii < n) & (jj > 0) & (jj < n) & (ll > 0) & (ll < n)
        xyz[interior] += off[interior]

    quads = []
    # x-normal faces at i = 0..n, normal +x
    fx = {}
    for l in range(n):
        for j in range(n):
            for i in range(n + 1):
                fx[(i, j, l)] = len(quads)
                quads.append((_vid(n, i, j, l), _vid(n, i, j + 1, l),
                              _vid(n, i, j + 1, l + 1), _vid(n, i, j, l + 1)))
    fy = {}
    for l in range(n):
        for j in range(n + 1):
            for i in range(n):
                fy[(i, j, l)] = len(quads)
                quads.append((_vid(n, i, j, l), _vid(n, i, j, l + 1),
                              _vid(n, i + 1, j, l + 1), _vid(n, i + 1, j, l)))
    fz = {}
    for l in range(n + 1):
        for j in range(n):
            for i in range(n):
                fz[(i, j, l)] = len(quads)
                quads.append((_vid(n, i, j, l), _vid(n, i + 1, j, l),
                              _vid(n, i + 1, j + 1, l), _vid(n, i, j + 1, l)))

    faces = []
    quad_to_faces = []
    for q in quads:
        if split_quads:
            p = int(np.argmin(q))
            a, b, c, d = q[p], q[(p + 1) % 4], q[(p + 2) % 4], q[(p + 3) % 4]
            quad_to_faces.append((len(faces), len(faces) + 1))
            faces.append((a, b, c))
            faces.append((a, c, d))
        else:
            quad_to_faces.append((len(faces),))
            faces.append(tuple(q))

    elem_faces = []
    elem_ijk = []
    for l in range(n):
        for j in range(n):
            for i in range(n):
                ef = []
                for q, s in ((fx[(i, j, l)], -1), (fx[(i + 1, j, l)], 1),
                             (fy[(i, j, l)], -1), (fy[(i, j + 1, l)], 1),
                             (fz[(i, j, l)], -1), (fz[(i, j, l + 1)], 1)):
                    for f in quad_to_faces[q]:
                        ef.append(s * (f + 1))
                elem_faces.append(ef)
                elem_ijk.append((i, j, l))

    face_ptr = np.zeros(len(faces) + 1, dtype=np.int32)
    face_ptr[1:] = np.cumsum([len(f) for f in faces])
    face_vtx = np.array([v for f in faces for v in f], dtype=np.int32)
    elem_ptr = np.zeros(len(elem_faces) + 1, dtype=np.int32)
    elem_ptr[1:] = np.cumsum([len(e) for e in elem_faces])
    elem_face = np.array([f for e in elem_faces for f in e], dtype=np.int32)
    return {
        "n": n, "h": h, "xyz": xyz,
        "face_ptr": face_ptr, "face_vtx": face_vtx,
        "elem_ptr": elem_ptr, "elem_face": elem_face,
        "elem_ijk": np.array(elem_ijk, dtype=np.int32),
    }


def octa_mesh(m, cut=0.5):
    """OCTA family: the ``(2m)^3`` grid of cubes of [0,1]^3 in which the
    common vertex of every ``2 x 2 x 2`` block of cubes is cut away by an
    octahedron whose six vertices lie on the six grid edges at that vertex,
    at distance ``cut * h`` from it (h = 1/(2m)).  Elements: ``m^3``
    octahedra and ``8 m^3`` cubes with one corner truncated (3
    quadrilaterals, 3 pentagons, 1 triangle), ``9 m^3`` in all; grid faces
    through a removed vertex become pentagons.  Element order: the cubes in
    lexicographic order (x fastest), then the octahedra by block.
    ``elem_ijk`` gives each cube its grid cell and each octahedron the
    lowest cell of its block, so that ``box_partition`` with box edges on
    block boundaries keeps every block in one box.
    """
    n = 2 * m
    h = 1.0 / n

    def centre(i, j, l):
        return i % 2 == 1 and j % 2 == 1 and l % 2 == 1

    vid, xyz = {}, []
    for l in range(n + 1):
        for j in range(n + 1):
            for i in range(n + 1):
                if not centre(i, j, l):
                    vid[(i, j, l)] = len(xyz)
                    xyz.append((i * h, j * h, l * h))
    blocks = [(2 * a + 1, 2 * b + 1, 2 * c + 1) for c in range(m) for b in range(m) for a in range(m)]
    ov = {}   # (block centre, axis, sign) -> octahedron vertex
    for ctr in blocks:
        for axis in range(3):
            for sg in (-1, 1):
                p = [ctr[0] * h, ctr[1] * h, ctr[2] * h]
                p[axis] += sg * cut * h
                ov[(ctr, axis, sg)] = len(xyz)
                xyz.append(tuple(p))

    def toward(ctr, q):
        d = [q[t] - ctr[t] for t in range(3)]
        axis = int(np.nonzero(d)[0][0])
        return ov[(ctr, axis, int(np.sign(d[axis])))]

    def loop(corners):
        out = []
        for t, q in enumerate(corners):
            if centre(*q):
                out.append(toward(q, corners[t - 1]))
                out.append(toward(q, corners[(t + 1) % len(corners)]))
            else:
                out.append(vid[q])
        return tuple(out)

    faces, fx, fy, fz = [], {}, {}, {}
    for l in range(n):
        for j in range(n):
            for i in range(n + 1):
                fx[(i, j, l)] = len(faces)
                faces.append(loop([(i, j, l), (i, j + 1, l), (i, j + 1, l + 1), (i, j, l + 1)]))
    for l in range(n):
        for j in range(n + 1):
            for i in range(n):
                fy[(i, j, l)] = len(faces)
                faces.append(loop([(i, j, l), (i, j, l + 1), (i + 1, j, l + 1), (i + 1, j, l)]))
    for l in range(n + 1):
        for j in range(n):
            for i in range(n):
                fz[(i, j, l)] = len(faces)
                faces.append(loop([(i, j, l), (i + 1, j, l), (i + 1, j + 1, l), (i, j + 1, l)]))
    # octahedron faces, oriented outward from the octahedron (normal along
    # the sign vector s; the loop x, y, z has normal sx sy sz * s)
    tri = {}
    for ctr in blocks:
        for sz in (-1, 1):
            for sy in (-1, 1):
                for sx in (-1, 1):
                    t = [ov[(ctr, 0, sx)], ov[(ctr, 1, sy)], ov[(ctr, 2, sz)]]
                    if sx * sy * sz < 0:
                        t = t[::-1]
                    tri[(ctr, sx, sy, sz)] = len(faces)
                    faces.append(tuple(t))

    elem_faces, elem_ijk = [], []
    for l in range(n):
        for j in range(n):
            for i in range(n):
                ef = [-(fx[(i, j, l)] + 1), fx[(i + 1, j, l)] + 1, -(fy[(i, j, l)] + 1), fy[(i, j + 1, l)] + 1,
                      -(fz[(i, j, l)] + 1), fz[(i, j, l + 1)] + 1]
                ci, cj, cl = (i if i % 2 else i + 1), (j if j % 2 else j + 1), (l if l % 2 else l + 1)
                s = (1 if i == ci else -1, 1 if j == cj else -1, 1 if l == cl else -1)
                ef.append(-(tri[((ci, cj, cl),) + s] + 1))
                elem_faces.append(ef)
                elem_ijk.append((i, j, l))
    for ctr in blocks:
        elem_faces.append([tri[(ctr, sx, sy, sz)] + 1 for sz in (-1, 1) for sy in (-1, 1) for sx in (-1, 1)])
        elem_ijk.append((ctr[0] - 1, ctr[1] - 1, ctr[2] - 1))

    face_ptr = np.zeros(len(faces) + 1, dtype=np.int32)
    face_ptr[1:] = np.cumsum([len(f) for f in faces])
    face_vtx = np.array([v for f in faces for v in f], dtype=np.int32)
    elem_ptr = np.zeros(len(elem_faces) + 1, dtype=np.int32)
    elem_ptr[1:] = np.cumsum([len(e) for e in elem_faces])
    elem_face = np.array([f for e in elem_faces for f in e], dtype=np.int32)
    return {
        "n": n, "h": h, "xyz": np.array(xyz, dtype=np.float64),
        "face_ptr": face_ptr, "face_vtx": face_vtx,
        "elem_ptr": elem_ptr, "elem_face": elem_face,
        "elem_ijk": np.array(elem_ijk, dtype=np.int32),
    }


def _clipped_cells(pts):
    """Voronoi cells of ``pts`` clipped to [0,1]^3: per cell, the vertices
    (halfspace intersection) and the polygons on its bounding planes, each
    tagged with the neighbour (>= 0) or the cube face (-1 - axis*2 - side)."""
    from scipy.spatial import Voronoi, HalfspaceIntersection
    vor = Voronoi(pts)
    nbr = [[] for _ in range(len(pts))]
    for a, b in vor.ridge_points:
        nbr[a].append(int(b))
        nbr[b].append(int(a))
    cells = []
    for i, p in enumerate(pts):
        hs, tags = [], []
        for j in nbr[i]:
            d = pts[j] - p
            hs.append(np.concatenate([d, [-(pts[j] @ pts[j] - p @ p) / 2.0]]))
            tags.append(j)
        for axis in range(3):
            for side in range(2):
                n = np.zeros(3)
                n[axis] = 1.0 if side else -1.0
                hs.append(np.concatenate([n, [-1.0 if side else 0.0]]))
                tags.append(-1 - 2 * axis - side)
        hs = np.array(hs)
        V = HalfspaceIntersection(hs, p).intersections
        polys = []
        for h, tag in zip(hs, tags):
            nrm = np.linalg.norm(h[:3])
            on = np.nonzero(np.abs(V @ h[:3] + h[3]) <= 1e-10 * nrm)[0]
            if len(on) < 3:
                continue
            polys.append((tag, h[:3] / nrm, on))
        cells.append((V, polys))
    return cells


def cvt_mesh(ncells, seed, iters=30, weld=1e-9):
    """CVT family: a centroidal Voronoi tessellation of [0,1]^3 from
    ``ncells`` seeds drawn U(0,1)^3 by ``numpy.random.default_rng(seed)``,
    relaxed by ``iters`` Lloyd steps (each seed moved to the centroid of its
    clipped cell).  Vertices closer than ``weld`` are merged; every interior
    face is the polygon of the lower-numbered cell, referenced with opposite
    signs by the two cells; faces are planar and convex, elements convex.
    """
    rng = np.random.default_rng(seed)
    pts = rng.uniform(0.0, 1.0, size=(ncells, 3))
    for _ in range(iters):
        cells = _clipped_cells(pts)
        newp = np.empty_like(pts)
        for i, (V, polys) in enumerate(cells):
            # centroid of the convex cell: tetrahedra from the vertex mean
            c0 = V.mean(0)
            vol, cm = 0.0, np.zeros(3)
            for _, n, on in polys:
                P = _ordered(V[on], n)
                for a in range(1, len(P) - 1):
                    t = abs(np.linalg.det(np.array([P[0] - c0, P[a] - c0, P[a + 1] - c0]))) / 6.0
                    vol += t
                    cm += t * (c0 + P[0] + P[a] + P[a + 1]) / 4.0
            newp[i] = cm / vol
        pts = newp
    cells = _clipped_cells(pts)
    # weld vertices
    allv = np.concatenate([V for V, _ in cells])
    key = np.round(allv / weld).astype(np.int64)
    uniq, inv = np.unique(key, axis=0, return_inverse=True)
    inv = inv.ravel()
    xyz = np.zeros((len(uniq), 3))
    cnt = np.zeros(len(uniq))
    np.add.at(xyz, inv, allv)
    np.add.at(cnt, inv, 1.0)
    xyz /= cnt[:, None]
    base = np.cumsum([0] + [len(V) for V, _ in cells])
    faces, fkey, elem_faces = [], {}, []
    for i, (V, polys) in enumerate(cells):
        ef = []
        for tag, n, on in polys:
            order = _order_idx(V[on], n)
            loop = []
            for q in on[order]:
                g = int(inv[base[i] + q])
                if not loop or loop[-1] != g:
                    loop.append(g)
            if len(loop) > 1 and loop[0] == loop[-1]:
                loop.pop()
            if len(loop) < 3:
                continue
            if tag >= 0:
                k = (min(i, tag), max(i, tag))
                if k in fkey:
                    f = fkey[k]
                    if set(faces[f]) != set(loop):
                        raise ValueError("cvt_mesh: the two sides of a face differ after welding")
                    ef.append(-(f + 1))
                    continue
                fkey[k] = len(faces)
            ef.append(len(faces) + 1)
            faces.append(tuple(loop))
        elem_faces.append(ef)
    face_ptr = np.zeros(len(faces) + 1, dtype=np.int32)
    face_ptr[1:] = np.cumsum([len(f) for f in faces])
    face_vtx = np.array([v for f in faces for v in f], dtype=np.int32)
    elem_ptr = np.zeros(len(elem_faces) + 1, dtype=np.int32)
    elem_ptr[1:] = np.cumsum([len(e) for e in elem_faces])
    elem_face = np.array([f for e in elem_faces for f in e], dtype=np.int32)
    return {"xyz": xyz, "face_ptr": face_ptr, "face_vtx": face_vtx, "elem_ptr": elem_ptr,
            "elem_face": elem_face, "seeds": pts}


def _order_idx(P, n):
    """Indices ordering the coplanar points P counter-clockwise about n."""
    c = P.mean(0)
    a = P[0] - c
    a = a - n * (a @ n)
    a /= np.linalg.norm(a)
    b = np.cross(n, a)
    return np.argsort(np.arctan2((P - c) @ b, (P - c) @ a))


def _ordered(P, n):
    return P[_order_idx(P, n)]


def element_vertex_average(mesh):
    """Vertex average of each element (used to sample fields per element)."""
    fp, fv = mesh["face_ptr"], mesh["face_vtx"]
    ep, ef = mesh["elem_ptr"], mesh["elem_face"]
    out = np.zeros((len(ep) - 1, 3))
    for e in range(len(ep) - 1):
        vs = set()
        for sf in ef[ep[e]:ep[e + 1]]:
            f = abs(int(sf)) - 1
            vs.update(int(v) for v in fv[fp[f]:fp[f + 1]])
        out[e] = mesh["xyz"][sorted(vs)].mean(axis=0)
    return out


def box_partition(mesh, parts):
    """Split the element grid into ``px x py x pz`` boxes of whole elements."""
    n = mesh["n"]
    px, py, pz = parts
    ijk = mesh["elem_ijk"]
    bi = ijk[:, 0] * px // n
    bj = ijk[:, 1] * py // n
    bl = ijk[:, 2] * pz // n
    return (bi + px * (bj + py * bl)).astype(np.int32)


def _grid_neighbours(n):
    nb = [[] for _ in range(n ** 3)]
    for l in range(n):
        for j in range(n):
            for i in range(n):
                e = i + n * (j + n * l)
                for di, dj, dl in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
                    a, b, c = i + di, j + dj, l + dl
                    if 0 <= a < n and 0 <= b < n and 0 <= c < n:
                        nb[e].append(a + n * (b + n * c))
    return nb


def greedy_partition(mesh, nparts, seed, size_range=(0.5, 2.0)):
    """Seeded greedy graph-growing partition with uneven target sizes.

    Targets are drawn U(size_range) times the mean size and rescaled to sum
    to the element count.  Seeds: one random element, then farthest-point
    picks over element centres.  Subdomains grow round-robin by breadth-first
    search over face neighbours until they reach their target; elements left
    over join the smallest adjacent subdomain; disconnected pieces of a
    subdomain other than its largest join the smallest adjacent subdomain.
    """
    n = mesh["n"]
    ne = n ** 3
    rng = np.random.default_rng(seed)
    t = rng.uniform(size_range[0], size_range[1], size=nparts)
    target = np.maximum(1, np.round(t / t.sum() * ne)).astype(np.int64)
    ijk = mesh["elem_ijk"].astype(np.float64)
    nb = _grid_neighbours(n)
    seeds = [int(rng.integers(ne))]
    d = np.linalg.norm(ijk - ijk[seeds[0]], axis=1)
    for _ in range(1, nparts):
        s = int(np.argmax(d))
        seeds.append(s)
        d = np.minimum(d, np.linalg.norm(ijk - ijk[s], axis=1))
    part = -np.ones(ne, dtype=np.int64)
    fronts = []
    size = np.zeros(nparts, dtype=np.int64)
    for p, s in enumerate(seeds):
        part[s] = p
        size[p] = 1
        fronts.append([s])
    active = True
    while active:
        active = False
        for p in range(nparts):
            if size[p] >= target[p] or not fronts[p]:
                continue
            newf = []
            grown = False
            for e in fronts[p]:
                for q in nb[e]:
                    if part[q] < 0 and size[p] < target[p]:
                        part[q] = p
                        size[p] += 1
                        newf.append(q)
                        grown = True
            fronts[p] = newf
            active = active or grown
    while (part < 0).any():
        changed = False
        for e in np.nonzero(part < 0)[0]:
            cand = [part[q] for q in nb[e] if part[q] >= 0]
            if cand:
                p = min(cand, key=lambda c: (size[c], c))
                part[e] = p
                size[p] += 1
                changed = True
        if not changed:
            break
    # merge disconnected pieces into a neighbour
    for p in range(nparts):
        members = np.nonzero(part == p)[0]
        if len(members) == 0:
            continue
        seen = {}
        comps = []
        for e in members:
            if e in seen:
                continue
            comp = [e]
            seen[e] = True
            stack = [e]
            while stack:
                x = stack.pop()
                for q in nb[x]:
                    if part[q] == p and q not in seen:
                        seen[q] = True
                        comp.append(q)
                        stack.append(q)
            comps.append(comp)
        if len(comps) > 1:
            comps.sort(key=len, reverse=True)
            for comp in comps[1:]:
                cand = [part[q] for x in comp for q in nb[x] if part[q] != p]
                r = min(cand, key=lambda c: (size[c], c))
                for x in comp:
                    part[x] = r
                size[r] += len(comp)
                size[p] -= len(comp)
    # relabel to consecutive ids
    used = np.unique(part)
    remap = -np.ones(nparts, dtype=np.int64)
    remap[used] = np.arange(len(used))
    return remap[part].astype(np.int32)
