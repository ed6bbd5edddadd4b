"""Seeded synthetic inputs for the Ginzburg-Landau Jacobian-solve workloads.

This module only draws random numbers and picks sizes. It holds none of the
method's arithmetic (no operator, no phase, no solver), so both the CPU
oracle's tests and the CUDA path's tests and benchmark may take their inputs
from here.

Every generator uses numpy's PCG64 with an explicit seed, so a given
(size, seed) pair always yields the same array on every machine.

Workloads (the paper's domains are the square and the cube, Section 4; the
sizes below are structured node lattices of those domains):

* ``square64``   2D, 64 x 64 nodes, mu = 1, field along z, psi uniform in the
                 unit disk (seed 1), b complex normal (seed 1).
* ``square1024`` 2D, 1024 x 1024 nodes, mu = 2, psi = (Newton steps from
                 psi = 1, at most five, until ||GL||_R <= 1e-7) + 0.1 * (uniform
                 in the unit disk) (seed 2); the solve is that state's Newton
                 system.
* ``cube128``    3D, 128^3 nodes, mu = 1, field along (1,1,1)/sqrt(3),
                 psi == 1 (the state the paper's Section 4 experiments use) or
                 psi uniform in the unit disk (seed 4); b complex normal (seed 5).
* ``batch64``    64 squares with N_s = round(exp(U(ln 32, ln 512))) (seed 6),
                 mu_s = 2 s / 63, psi_s = 1 + 0.1 * disk noise (seed 7 + s).
* ``cube256``    3D, 256^3 nodes, continuation over mu in [0, 1.5].
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "rng",
    "disk",
    "complex_normal",
    "psi_noisy_one",
    "batch_sizes",
    "warmstart_init",
    "WORKLOADS",
]


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def disk(n: int, seed: int) -> np.ndarray:
    """n complex numbers uniform in the closed unit disk: r = sqrt(U), arg = 2 pi U.

    Radii are drawn first (all n), then arguments (all n).
    """
    g = rng(seed)
    r = np.sqrt(g.random(n))
    a = 2.0 * math.pi * g.random(n)
    return (r * np.cos(a) + 1j * (r * np.sin(a))).astype(np.complex128)


def complex_normal(n: int, seed: int) -> np.ndarray:
    """n draws of CN(0, 1): real and imaginary parts N(0, 1/2), real parts first."""
    g = rng(seed)
    re = g.standard_normal(n)
    im = g.standard_normal(n)
    return ((re + 1j * im) / math.sqrt(2.0)).astype(np.complex128)


def psi_noisy_one(n: int, seed: int, amplitude: float = 0.1) -> np.ndarray:
    """1 + amplitude * (uniform in the unit disk)."""
    return (1.0 + amplitude * disk(n, seed)).astype(np.complex128)


def batch_sizes(count: int = 64, seed: int = 6, lo: int = 32, hi: int = 512) -> list[int]:
    """Log-uniform node counts per side: N_s = round(exp(U(ln lo, ln hi)))."""
    g = rng(seed)
    u = g.random(count)
    return [int(round(math.exp(math.log(lo) + (math.log(hi) - math.log(lo)) * x))) for x in u]


INV_SQRT3 = 1.0 / math.sqrt(3.0)

# name -> (dim, nodes per side, mu, unit field direction)
WORKLOADS = {
    "square64": (2, 64, 1.0, (0.0, 0.0, 1.0)),
    "square1024": (2, 1024, 2.0, (0.0, 0.0, 1.0)),
    "cube128": (3, 128, 1.0, (INV_SQRT3, INV_SQRT3, INV_SQRT3)),
    "cube256": (3, 256, 1.5, (0.0, 0.0, 1.0)),
}


def warmstart_init(seed: int = 11, layers: int = 4, channels: int = 64) -> np.ndarray:
    """Random initial parameters of the warm-start network, one flat float32
    vector: layers matrices of channels x (2 channels) drawn N(0, 2 / fan_in)
    (He initialisation, fan_in = 2 channels), then a 2 x channels head drawn
    N(0, 1 / channels) scaled by 0.1."""
    g = rng(seed)
    cin = 2 * channels
    ws = [g.standard_normal(channels * cin) * math.sqrt(2.0 / cin) for _ in range(layers)]
    head = g.standard_normal(2 * channels) * (0.1 / math.sqrt(channels))
    return np.concatenate(ws + [head]).astype(np.float32)


# ---------------------------------------------------------------- unstructured meshes
# The paper's test domains (Sec. 4), all centred at the origin with circumradius 5:
# the regular triangle, square and disc in 2D, the regular tetrahedron, cube and
# ball in 3D.  A mesh is the Delaunay triangulation (scipy's Qhull) of a point set:
# boundary points at spacing about h and a lattice of spacing h inside, jittered by
# up to 0.2 h (seeded), kept at least h/2 from the boundary.  Only input
# generation: the method takes any conforming simplicial mesh.
R_DOMAIN = 5.0


def _tet_vertices():
    s2, s23 = math.sqrt(2.0), math.sqrt(2.0 / 3.0)
    return R_DOMAIN * np.array([[0.0, 0.0, 1.0], [2 * s2 / 3, 0.0, -1.0 / 3], [-s2 / 3, s23, -1.0 / 3],
                                [-s2 / 3, -s23, -1.0 / 3]])


def _tri_vertices():
    r = R_DOMAIN
    return np.array([[0.0, r], [-r * math.sqrt(3.0) / 2, -r / 2], [r * math.sqrt(3.0) / 2, -r / 2]])


def _inside_distance(name: str, p: np.ndarray) -> np.ndarray:
    """Distance from each point to the boundary (negative outside)."""
    if name in ("circ", "ball"):
        return R_DOMAIN - np.linalg.norm(p, axis=1)
    if name == "sq":
        return R_DOMAIN / math.sqrt(2.0) - np.max(np.abs(p), axis=1)
    if name == "cube":
        return R_DOMAIN / math.sqrt(3.0) - np.max(np.abs(p), axis=1)
    # triangle / tetrahedron: the inradius minus the largest signed distance to a face plane
    v = _tri_vertices() if name == "tri" else _tet_vertices()
    d = v.shape[1]
    best = np.full(p.shape[0], np.inf)
    for i in range(d + 1):
        opp = np.delete(v, i, axis=0)
        if d == 2:
            t = opp[1] - opp[0]
            nrm = np.array([t[1], -t[0]])
        else:
            nrm = np.cross(opp[1] - opp[0], opp[2] - opp[0])
        nrm = nrm / np.linalg.norm(nrm)
        if np.dot(v[i] - opp[0], nrm) < 0:
            nrm = -nrm  # pointing inward
        best = np.minimum(best, (p - opp[0]) @ nrm)
    return best


def _segment_points(a, b, h):
    k = max(1, int(math.ceil(np.linalg.norm(b - a) / h)))
    t = np.arange(k)[:, None] / k
    return a[None, :] + t * (b - a)[None, :]


def _triangle_face_points(a, b, c, h):
    k = max(1, int(math.ceil(max(np.linalg.norm(b - a), np.linalg.norm(c - a)) / h)))
    pts = [a + (i / k) * (b - a) + (j / k) * (c - a) for i in range(k + 1) for j in range(k + 1 - i)]
    return np.array(pts)


def _boundary_points(name: str, h: float) -> np.ndarray:
    r = R_DOMAIN
    if name == "circ":
        k = max(8, int(math.ceil(2 * math.pi * r / h)))
        t = 2 * math.pi * np.arange(k) / k
        return np.stack([r * np.cos(t), r * np.sin(t)], axis=1)
    if name == "ball":
        k = max(20, int(math.ceil(4 * math.pi * r * r / (h * h) * 1.15)))
        i = np.arange(k) + 0.5
        phi = np.arccos(1 - 2 * i / k)
        th = math.pi * (1 + math.sqrt(5.0)) * i
        return r * np.stack([np.cos(th) * np.sin(phi), np.sin(th) * np.sin(phi), np.cos(phi)], axis=1)
    if name in ("tri", "sq"):
        v = _tri_vertices() if name == "tri" else (r / math.sqrt(2.0)) * np.array([[1, 1], [-1, 1], [-1, -1], [1, -1.0]])
        return np.concatenate([_segment_points(v[i], v[(i + 1) % len(v)], h) for i in range(len(v))])
    if name == "tet":
        v = _tet_vertices()
        faces = [(0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3)]
        return np.concatenate([_triangle_face_points(v[a], v[b], v[c], h) for a, b, c in faces])
    if name == "cube":
        s = r / math.sqrt(3.0)
        k = max(1, int(math.ceil(2 * s / h)))
        g = np.linspace(-s, s, k + 1)
        pts = []
        for ax in range(3):
            for side in (-s, s):
                u, w = np.meshgrid(g, g, indexing="ij")
                q = np.zeros((u.size, 3))
                q[:, ax] = side
                q[:, (ax + 1) % 3] = u.ravel()
                q[:, (ax + 2) % 3] = w.ravel()
                pts.append(q)
        return np.concatenate(pts)
    raise ValueError(f"unknown domain {name}")


def delaunay_domain(name: str, h: float, seed: int = 0):
    """(dim, x (n x 3, z = 0 in 2D), simplices (m x (dim + 1), int32)) of a Delaunay
    mesh of test domain `name` in {"tri", "sq", "circ", "tet", "cube", "ball"}."""
    from scipy.spatial import Delaunay

    dim = 2 if name in ("tri", "sq", "circ") else 3
    b = _boundary_points(name, h)
    k = int(math.ceil(R_DOMAIN / h)) + 1
    g = np.arange(-k, k + 1) * h
    grid = np.stack(np.meshgrid(*([g] * dim), indexing="ij"), axis=-1).reshape(-1, dim)
    grid = grid + rng(seed).uniform(-0.2 * h, 0.2 * h, size=grid.shape)
    inner = grid[_inside_distance(name, grid) >= 0.5 * h]
    pts = np.unique(np.round(np.concatenate([b, inner]), 12), axis=0)
    tri = Delaunay(pts)
    simp = tri.simplices.astype(np.int64)
    # drop flat simplices Qhull can leave along the hull
    e = pts[simp[:, 1:]] - pts[simp[:, :1]]
    vol = np.abs(np.linalg.det(e)) / math.factorial(dim)
    simp = simp[vol > 1e-9 * h ** dim]
    used = np.unique(simp)
    remap = -np.ones(len(pts), np.int64)
    remap[used] = np.arange(len(used))
    x = np.zeros((len(used), 3))
    x[:, :dim] = pts[used]
    return dim, x, remap[simp].astype(np.int32)
