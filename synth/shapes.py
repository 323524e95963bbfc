"""Procedural non-convex shapes and area-uniform surface samples.

A shape is a union of closed, outward-oriented triangle meshes ("components").
The paper samples K points uniformly on each object's mesh surface and takes the
object centre to be the centre of the mesh's axis-aligned bounding box
(Sec. III and Sec. IV-A); the generators below do the same on procedural meshes:

* ``l_bracket``: three overlapping boxes, 400 triangles;
* ``torus_mesh``: R = 1, r = 0.3, 32 x 8 quads = 512 triangles;
* ``random_union``: 2-5 random boxes / ellipsoids, 300-2000 triangles.

Every mesh is translated so that its AABB centre is the body-frame origin.
"""

from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence

import numpy as np

N_POINTS = 2048


@dataclasses.dataclass
class Mesh:
    """Union of closed components.

    vertices: float64 [V, 3]; faces: int32 [T, 3] (outward, counter-clockwise
    seen from outside); comp: int32 [T] component id of each face;
    prims: analytic description of each component (used only to reject surface
    samples that fall inside another component).
    """

    vertices: np.ndarray
    faces: np.ndarray
    comp: np.ndarray
    prims: List[dict]

    @property
    def n_tris(self) -> int:
        return int(self.faces.shape[0])

    def translated(self, d: np.ndarray) -> "Mesh":
        prims = []
        for p in self.prims:
            q = dict(p)
            q["centre"] = np.asarray(p["centre"], np.float64) + d
            prims.append(q)
        return Mesh(self.vertices + d, self.faces.copy(), self.comp.copy(), prims)


def _rot_about(axis: Sequence[float], angle: float) -> np.ndarray:
    a = np.asarray(axis, np.float64)
    a = a / np.linalg.norm(a)
    k = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + np.sin(angle) * k + (1 - np.cos(angle)) * (k @ k)


def _random_rotation(rng: np.random.Generator) -> np.ndarray:
    q, r = np.linalg.qr(rng.normal(size=(3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def _merge(parts: Sequence[Mesh]) -> Mesh:
    verts, faces, comp, prims = [], [], [], []
    off = 0
    c0 = 0
    for m in parts:
        verts.append(m.vertices)
        faces.append(m.faces + off)
        comp.append(m.comp + c0)
        prims.extend(m.prims)
        off += m.vertices.shape[0]
        c0 += int(m.comp.max()) + 1
    return Mesh(np.concatenate(verts), np.concatenate(faces).astype(np.int32),
                np.concatenate(comp).astype(np.int32), prims)


def box_mesh(half: Sequence[float], segs: Sequence[int],
             centre: Sequence[float] = (0, 0, 0),
             rot: Optional[np.ndarray] = None) -> Mesh:
    """Closed box with half extents ``half`` and (nx, ny, nz) segments per axis.

    Triangle count 4 (nx ny + ny nz + nz nx).
    """
    h = np.asarray(half, np.float64)
    n = [int(s) for s in segs]
    rot = np.eye(3) if rot is None else np.asarray(rot, np.float64)
    c = np.asarray(centre, np.float64)
    e = np.eye(3)
    # (normal axis, sign, U axis, V axis) with U x V = sign * normal
    faces_def = [(0, +1, 1, 2), (0, -1, 2, 1), (1, +1, 2, 0), (1, -1, 0, 2),
                 (2, +1, 0, 1), (2, -1, 1, 0)]
    verts, tris = [], []
    for ax, sg, ua, va in faces_def:
        nu, nv = n[ua], n[va]
        base = len(verts)
        for i in range(nu + 1):
            for j in range(nv + 1):
                p = sg * h[ax] * e[ax] + (-h[ua] + 2 * h[ua] * i / nu) * e[ua] \
                    + (-h[va] + 2 * h[va] * j / nv) * e[va]
                verts.append(p)
        for i in range(nu):
            for j in range(nv):
                p00 = base + i * (nv + 1) + j
                p10 = p00 + (nv + 1)
                p11 = p10 + 1
                p01 = p00 + 1
                tris.append((p00, p10, p11))
                tris.append((p00, p11, p01))
    v = np.asarray(verts) @ rot.T + c
    f = np.asarray(tris, np.int32)
    prim = {"kind": "box", "centre": c, "rot": rot, "half": h}
    return Mesh(v, f, np.zeros(len(f), np.int32), [prim])


def ellipsoid_mesh(radii: Sequence[float], n_lat: int, n_lon: int,
                   centre: Sequence[float] = (0, 0, 0),
                   rot: Optional[np.ndarray] = None) -> Mesh:
    """UV ellipsoid: n_lat latitude bands, n_lon longitude segments.

    Triangle count 2 n_lon (n_lat - 1).
    """
    a = np.asarray(radii, np.float64)
    rot = np.eye(3) if rot is None else np.asarray(rot, np.float64)
    c = np.asarray(centre, np.float64)
    verts = [(0.0, 0.0, a[2])]
    for i in range(1, n_lat):
        th = np.pi * i / n_lat
        for j in range(n_lon):
            ph = 2 * np.pi * j / n_lon
            verts.append((a[0] * np.sin(th) * np.cos(ph),
                          a[1] * np.sin(th) * np.sin(ph), a[2] * np.cos(th)))
    verts.append((0.0, 0.0, -a[2]))
    south = len(verts) - 1

    def ring(i, j):  # i in 1..n_lat-1
        return 1 + (i - 1) * n_lon + (j % n_lon)

    tris = []
    for j in range(n_lon):
        tris.append((0, ring(1, j), ring(1, j + 1)))
    for i in range(1, n_lat - 1):
        for j in range(n_lon):
            p00, p10 = ring(i, j), ring(i + 1, j)
            p11, p01 = ring(i + 1, j + 1), ring(i, j + 1)
            tris.append((p00, p10, p11))
            tris.append((p00, p11, p01))
    for j in range(n_lon):
        tris.append((ring(n_lat - 1, j), south, ring(n_lat - 1, j + 1)))
    v = np.asarray(verts) @ rot.T + c
    f = np.asarray(tris, np.int32)
    prim = {"kind": "ellipsoid", "centre": c, "rot": rot, "half": a}
    return Mesh(v, f, np.zeros(len(f), np.int32), [prim])


def torus_mesh(R: float = 1.0, r: float = 0.3, n_u: int = 32,
               n_v: int = 8) -> Mesh:
    """Torus about the z axis; 2 n_u n_v triangles (512 at 32 x 8)."""
    verts = []
    for i in range(n_u):
        u = 2 * np.pi * i / n_u
        for j in range(n_v):
            v = 2 * np.pi * j / n_v
            verts.append(((R + r * np.cos(v)) * np.cos(u),
                          (R + r * np.cos(v)) * np.sin(u), r * np.sin(v)))

    def idx(i, j):
        return (i % n_u) * n_v + (j % n_v)

    tris = []
    for i in range(n_u):
        for j in range(n_v):
            tris.append((idx(i, j), idx(i + 1, j), idx(i + 1, j + 1)))
            tris.append((idx(i, j), idx(i + 1, j + 1), idx(i, j + 1)))
    prim = {"kind": "torus", "centre": np.zeros(3), "rot": np.eye(3),
            "half": np.array([R, r, 0.0])}
    return Mesh(np.asarray(verts, np.float64), np.asarray(tris, np.int32),
                np.zeros(len(tris), np.int32), [prim])


def l_bracket() -> Mesh:
    """Two 1.0 x 0.2 x 0.2 bars meeting at a corner plus a 0.6 x 0.2 x 0.5
    gusset block: 96 + 96 + 208 = 400 triangles."""
    bar_x = box_mesh((0.5, 0.1, 0.1), (5, 2, 2), centre=(0.4, 0.0, 0.0))
    bar_y = box_mesh((0.1, 0.5, 0.1), (2, 5, 2), centre=(0.0, 0.4, 0.0))
    block = box_mesh((0.3, 0.1, 0.25), (6, 2, 5), centre=(0.3, 0.0, 0.25))
    return _merge([bar_x, bar_y, block])


def _box_segs(half: np.ndarray, budget: int) -> tuple:
    # 4 (nx ny + ny nz + nz nx) ~ budget with n_i proportional to extents
    e = half / half.max()
    s = np.sqrt(budget / (4.0 * (e[0] * e[1] + e[1] * e[2] + e[2] * e[0])))
    return tuple(int(max(1, round(s * ei))) for ei in e)


def random_union(rng: np.random.Generator, min_tris: int = 300,
                 max_tris: int = 2000) -> Mesh:
    """Union of 2-5 random boxes / ellipsoids with 300-2000 triangles."""
    while True:
        k = int(rng.integers(2, 6))
        target = int(rng.integers(min_tris, max_tris + 1))
        budget = max(48, target // k)
        parts = []
        centre = np.zeros(3)
        for _ in range(k):
            half = rng.uniform(0.08, 0.35, size=3)
            rot = _random_rotation(rng)
            if rng.random() < 0.5:
                parts.append(box_mesh(half, _box_segs(half, budget), centre, rot))
            else:
                n_lat = max(3, int(round(np.sqrt(budget / 4.0))))
                n_lon = max(4, int(round(budget / (2.0 * (n_lat - 1)))))
                parts.append(ellipsoid_mesh(half, n_lat, n_lon, centre, rot))
            # next primitive starts near this one so the union stays compact
            centre = centre + rng.uniform(-0.25, 0.25, size=3)
        m = _merge(parts)
        if min_tris <= m.n_tris <= max_tris:
            return m


def _inside_prim(p: np.ndarray, prim: dict, tol: float = 1e-9) -> np.ndarray:
    loc = (p - prim["centre"]) @ prim["rot"]
    h = prim["half"]
    if prim["kind"] == "box":
        return np.all(np.abs(loc) < h - tol, axis=1)
    if prim["kind"] == "ellipsoid":
        return np.sum((loc / h) ** 2, axis=1) < 1.0 - tol
    raise ValueError(prim["kind"])


def sample_surface(mesh: Mesh, n: int, rng: np.random.Generator) -> np.ndarray:
    """n points uniform by area on the union's outer surface (float64 [n,3]).

    A sample on one component that lies strictly inside another component is
    not on the union's surface and is redrawn.
    """
    v = mesh.vertices[mesh.faces]
    area = 0.5 * np.linalg.norm(np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 0]),
                                axis=1)
    prob = area / area.sum()
    out = []
    have = 0
    while have < n:
        m = 2 * (n - have) + 64
        t = rng.choice(len(prob), size=m, p=prob)
        r1 = np.sqrt(rng.random(m))
        r2 = rng.random(m)
        p = ((1 - r1)[:, None] * v[t, 0] + (r1 * (1 - r2))[:, None] * v[t, 1]
             + (r1 * r2)[:, None] * v[t, 2])
        keep = np.ones(m, bool)
        if len(mesh.prims) > 1:
            for ci, prim in enumerate(mesh.prims):
                other = mesh.comp[t] != ci
                keep &= ~(other & _inside_prim(p, prim))
        p = p[keep]
        out.append(p)
        have += len(p)
    return np.concatenate(out)[:n]


def _centre_on_aabb(mesh: Mesh) -> Mesh:
    lo = mesh.vertices.min(axis=0)
    hi = mesh.vertices.max(axis=0)
    return mesh.translated(-(lo + hi) * 0.5)


@dataclasses.dataclass
class ShapeLibrary:
    """Meshes plus the arrays the contact detector consumes.

    points: float32 [S, n_points, 3] body-frame surface samples;
    aabb:   float32 [S, 6] body-frame (lo.xyz, hi.xyz) of each mesh.
    """

    meshes: List[Mesh]
    points: np.ndarray
    aabb: np.ndarray
    names: List[str]

    @property
    def n_shapes(self) -> int:
        return len(self.meshes)

    @property
    def n_points(self) -> int:
        return int(self.points.shape[1])


def _finish(meshes: List[Mesh], names: List[str], n_points: int,
            rng: np.random.Generator) -> ShapeLibrary:
    cm = [_centre_on_aabb(m) for m in meshes]
    pts = np.stack([sample_surface(m, n_points, rng) for m in cm])
    aabb = np.stack([np.concatenate([m.vertices.min(0), m.vertices.max(0)])
                     for m in cm])
    return ShapeLibrary(cm, pts.astype(np.float32), aabb.astype(np.float32),
                        names)


def tiny_library(n_points: int = N_POINTS, seed: int = 0) -> ShapeLibrary:
    """L-bracket (400 tris) and torus (512 tris), n_points samples each."""
    rng = np.random.default_rng(seed)
    return _finish([l_bracket(), torus_mesh()], ["l_bracket", "torus"],
                   n_points, rng)


def make_library(n_shapes: int, seed: int, n_points: int = N_POINTS,
                 min_tris: int = 300, max_tris: int = 2000) -> ShapeLibrary:
    """``n_shapes`` random unions of 2-5 boxes / ellipsoids."""
    rng = np.random.default_rng(seed)
    meshes = [random_union(rng, min_tris, max_tris) for _ in range(n_shapes)]
    return _finish(meshes, [f"union{i}" for i in range(n_shapes)], n_points,
                   rng)


def convex_elements(lib: "ShapeLibrary", max_vertices: int = 0, max_elements: int = 0):
    """Convex decomposition of every library shape from its components (each
    component of a procedural shape is a box or an ellipsoid, so convex):
    element e of shape s is the vertex set of one component, cut to
    ``max_vertices`` by farthest-point sampling when > 0 (the convex hull of
    the kept vertices is then an inner approximation), and at most
    ``max_elements`` elements per shape (the largest, by vertex spread) when
    > 0.  Returns elem_off int32 [S + 1], vert_off int32 [E + 1] and verts
    float32 [V, 3] (body frame)."""
    elem_off, vert_off, verts = [0], [0], []
    for m in lib.meshes:
        elems = []
        for c in np.unique(m.comp):
            v = m.vertices[np.unique(m.faces[m.comp == c].ravel())]
            if max_vertices and len(v) > max_vertices:
                keep = [int(np.argmax(np.linalg.norm(v - v.mean(0), axis=1)))]
                d = np.linalg.norm(v - v[keep[0]], axis=1)
                while len(keep) < max_vertices:
                    i = int(np.argmax(d))
                    keep.append(i)
                    d = np.minimum(d, np.linalg.norm(v - v[i], axis=1))
                v = v[keep]
            elems.append(v)
        if max_elements and len(elems) > max_elements:
            spread = [np.ptp(e, axis=0).prod() for e in elems]
            elems = [elems[i] for i in np.argsort(spread)[::-1][:max_elements]]
        for e in elems:
            verts.append(e.astype(np.float32))
            vert_off.append(vert_off[-1] + len(e))
        elem_off.append(elem_off[-1] + len(elems))
    return (np.asarray(elem_off, np.int32), np.asarray(vert_off, np.int32),
            np.concatenate(verts).astype(np.float32))
