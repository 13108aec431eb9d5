"""Seeded tetrahedral box meshes for the synthetic FEM workloads.

The paper studies unstructured tetrahedral FEM models (Section II, Section III)
without giving the meshes, so the inputs here are synthetic: the unit cube cut
into n^3 cubes, each cube split into six tetrahedra along its main diagonal
(Kuhn / Freudenthal split: one tetrahedron per ordering of the three axes;
the same orientation in every cube makes the mesh conforming), with every
interior vertex moved by a seeded uniform jitter so that no two elements are
congruent.  Boundary vertices stay on the cube faces, so the boundary stays
planar and the absorbing boundary faces are exact planes.

Edges are oriented from the lower to the higher global vertex index; that
orientation fixes the sign of every edge degree of freedom.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass

import numpy as np

# local edges of a tetrahedron with sorted vertices: (a, b) with a < b
TET_EDGES = np.array([(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)], dtype=np.int64)
# local faces of a tetrahedron: the three vertices it keeps
TET_FACES = np.array([(0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3)], dtype=np.int64)


@dataclass
class Mesh:
    n: int                  # cubes per side
    coords: np.ndarray      # (V, 3) float64 vertex coordinates
    grid: np.ndarray        # (V, 3) int64 integer lattice coordinates of each vertex
    tets: np.ndarray        # (T, 4) int64 vertex ids, sorted ascending in each row
    tet_cell: np.ndarray    # (T,) int64 cube index c = ci + n*(cj + n*ck)
    edges: np.ndarray       # (E, 2) int64 vertex ids (a < b)
    tet_edges: np.ndarray   # (T, 6) int64 global edge id of each local edge
    bface_tet: np.ndarray   # (F,) tet owning each boundary triangle
    bface_local: np.ndarray  # (F,) local face index (row of TET_FACES)
    bface_normal: np.ndarray  # (F, 3) outward unit normal

    @property
    def n_edges(self) -> int:
        return int(self.edges.shape[0])

    @property
    def h(self) -> float:
        return 1.0 / self.n


def kuhn_edge_count(a: int, b: int, c: int) -> int:
    """Number of edges of an a x b x c block of Kuhn-split cubes.

    Axis edges + one diagonal per lattice square + one body diagonal per cube.
    """
    axis = a * (b + 1) * (c + 1) + b * (a + 1) * (c + 1) + c * (a + 1) * (b + 1)
    face = a * b * (c + 1) + b * c * (a + 1) + c * a * (b + 1)
    return axis + face + a * b * c


def tet_volumes(coords: np.ndarray, tets: np.ndarray) -> np.ndarray:
    p = coords[tets]
    d = p[:, 1:, :] - p[:, 0:1, :]
    return np.linalg.det(d) / 6.0


def box_mesh(n: int, jitter: float = 0.15, seed: int = 0, min_vol_frac: float = 0.05,
             max_tries: int = 50) -> Mesh:
    """Kuhn-split unit-cube mesh with n^3 cubes and seeded interior jitter.

    Interior vertices move by U[-jitter*h, jitter*h]^3 drawn from
    numpy.random.default_rng(seed).  A draw that leaves any tetrahedron with
    volume <= min_vol_frac * h^3 / 6 is rejected and redrawn from the same
    generator (the stream continues, so the result stays a function of seed).
    """
    if n < 1:
        raise ValueError("n must be >= 1")
    h = 1.0 / n
    m = n + 1
    ii, jj, kk = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij")
    # vertex id v = i + m*(j + m*k)
    grid = np.stack([ii.transpose(2, 1, 0).ravel(), jj.transpose(2, 1, 0).ravel(),
                     kk.transpose(2, 1, 0).ravel()], axis=1).astype(np.int64)
    base = grid.astype(np.float64) * h
    interior = np.all((grid > 0) & (grid < n), axis=1)

    # six Kuhn tetrahedra per cube, one per permutation of the axes
    ci, cj, ck = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    ci = ci.transpose(2, 1, 0).ravel()
    cj = cj.transpose(2, 1, 0).ravel()
    ck = ck.transpose(2, 1, 0).ravel()
    cell = ci + n * (cj + n * ck)

    def vid(di, dj, dk):
        return (ci + di) + m * ((cj + dj) + m * (ck + dk))

    tets = []
    cells = []
    for perm in itertools.permutations(range(3)):
        step = np.zeros(3, dtype=np.int64)
        path = [vid(0, 0, 0)]
        for ax in perm:
            step[ax] = 1
            path.append(vid(*step))
        tets.append(np.stack(path, axis=1))
        cells.append(cell)
    tets = np.concatenate(tets, axis=0)
    tet_cell = np.concatenate(cells, axis=0)
    order = np.lexsort((np.repeat(np.arange(6), n ** 3), tet_cell))
    tets = np.sort(tets[order], axis=1)
    tet_cell = tet_cell[order]

    rng = np.random.default_rng(seed)
    vmin = min_vol_frac * h ** 3 / 6.0
    for _ in range(max_tries):
        jit = rng.uniform(-jitter * h, jitter * h, size=base.shape)
        coords = base.copy()
        coords[interior] += jit[interior]
        vol = np.abs(tet_volumes(coords, tets))
        if np.all(vol > vmin):
            break
    else:  # pragma: no cover - never reached for jitter <= 0.2
        raise RuntimeError("could not draw a valid jittered mesh")

    # global edges, oriented low -> high vertex id
    V = coords.shape[0]
    loc = tets[:, TET_EDGES]            # (T, 6, 2)
    keys = loc[:, :, 0] * V + loc[:, :, 1]
    ukeys, inv = np.unique(keys.ravel(), return_inverse=True)
    edges = np.stack([ukeys // V, ukeys % V], axis=1)
    tet_edges = inv.reshape(-1, 6)

    # boundary triangles: all three vertices on the same cube face
    fverts = tets[:, TET_FACES]          # (T, 4, 3)
    g = grid[fverts]                     # (T, 4, 3, 3)
    bt, bl, bn = [], [], []
    for ax in range(3):
        for side, val in ((-1.0, 0), (1.0, n)):
            on = np.all(g[:, :, :, ax] == val, axis=2)  # (T, 4)
            t_idx, f_idx = np.nonzero(on)
            nrm = np.zeros((t_idx.size, 3))
            nrm[:, ax] = side
            bt.append(t_idx)
            bl.append(f_idx)
            bn.append(nrm)
    bface_tet = np.concatenate(bt).astype(np.int64)
    bface_local = np.concatenate(bl).astype(np.int64)
    bface_normal = np.concatenate(bn)
    o = np.lexsort((bface_local, bface_tet))
    return Mesh(n=n, coords=coords, grid=grid, tets=tets, tet_cell=tet_cell, edges=edges,
                tet_edges=tet_edges, bface_tet=bface_tet[o], bface_local=bface_local[o],
                bface_normal=bface_normal[o])


def boundary_edge_mask(mesh: Mesh) -> np.ndarray:
    """True for edges lying on the boundary of the unit cube."""
    g = mesh.grid[mesh.edges]            # (E, 2, 3)
    n = mesh.n
    on = np.zeros(mesh.n_edges, dtype=bool)
    for ax in range(3):
        for val in (0, n):
            on |= np.all(g[:, :, ax] == val, axis=1)
    return on
