"""Seeded synthetic FEM problems: assembled global system plus its torn form.

A problem holds the global system A x = b (complex symmetric, A = A^T) and the
torn arrowhead data [blkdiag(A_i) B^T; B 0][u; lambda] = [f; 0]: for each domain
its local matrix A_i (CSR, caller ordering = ascending global edge id), its
load f_i and the signed-selection entries of B_i.  Nothing here factors or
solves anything: this module only generates inputs.

Workloads (sizes follow the scaled-up versions of the paper's test problems,
Section III; the paper's own meshes are not available):
  * "plain"    n = 8 cubes per side, 8 equal domains (2x2x2), eps_r = 2 - 0.1j;
  * "batched"  n = 41, 512 domains by jittered bisection (500..2500 edges per
               domain, roughly lognormal), eps_r per domain Re U[1,4], -Im U[0.05,0.2];
  * "large"    n = 65, 2048 domains, same recipe;
  * "tiny"     n = 1..6 with 2..16 domains, for brute-force checks.
k0 = 2 pi everywhere; first-order absorbing boundary on all six cube faces.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

from .decompose import RcbTree, Tearing, rcb_cells, tear
from .mesh import Mesh, boundary_edge_mask, box_mesh
from .nedelec import element_matrices, face_load, face_matrices, interpolate, volume_load

K0 = 2.0 * np.pi
EPS_UNIFORM = 2.0 - 0.1j
SOURCE_POINT = np.array([0.31, 0.37, 0.43])


@dataclass
class Subdomain:
    l2g: np.ndarray            # local -> global edge id (ascending)
    indptr: np.ndarray         # CSR of A_i, int32, full symmetric pattern, sorted columns
    indices: np.ndarray
    data: np.ndarray           # complex128
    f: np.ndarray              # (n_i, nrhs) complex128 local load
    b_dual: np.ndarray         # int32 multiplier id of each B_i entry
    b_local: np.ndarray        # int32 local row of each B_i entry
    b_sign: np.ndarray         # int8 +1/-1

    @property
    def n(self) -> int:
        return int(self.l2g.size)

    def dense(self) -> np.ndarray:
        return sp.csr_matrix((self.data, self.indices, self.indptr), shape=(self.n, self.n)).toarray()


@dataclass
class Problem:
    name: str
    mesh: Mesh
    k0: float
    eps_tet: np.ndarray        # (T,) complex relative permittivity per tetrahedron
    tet_sub: np.ndarray        # (T,) domain of every tetrahedron
    rcb: RcbTree
    tearing: Tearing
    A_indptr: np.ndarray       # global CSR
    A_indices: np.ndarray
    A_data: np.ndarray
    b: np.ndarray              # (n, nrhs)
    subs: list = field(default_factory=list)
    x_exact: np.ndarray | None = None   # set when the discrete solution is known in closed form
    rhs_edges: np.ndarray | None = None

    @property
    def n(self) -> int:
        return self.mesh.n_edges

    @property
    def n_sub(self) -> int:
        return len(self.subs)

    @property
    def n_dual(self) -> int:
        return self.tearing.n_dual

    @property
    def nrhs(self) -> int:
        return int(self.b.shape[1])

    def A_csr(self) -> sp.csr_matrix:
        return sp.csr_matrix((self.A_data, self.A_indices, self.A_indptr), shape=(self.n, self.n))

    def centroids(self) -> np.ndarray:
        c = np.empty((self.n_sub, 3))
        for s, (lo, hi) in enumerate(self.rcb.boxes):
            c[s] = 0.5 * (lo + hi) / self.mesh.n
        return c


# ----------------------------------------------------------------------------
# right-hand sides
# ----------------------------------------------------------------------------
def linear_field(a: np.ndarray, bvec: np.ndarray):
    """E(r) = a + b x r: in the lowest-order Nedelec space, curl E = 2 b."""
    def E(x):
        return a + np.cross(np.broadcast_to(bvec, x.shape), x)
    return E


def sine_field():
    """E = (sin py sin pz, sin pz sin px, sin px sin py) (p = pi); curl curl E = 2 pi^2 E."""
    p = np.pi

    def E(x):
        sx, sy, sz = np.sin(p * x[..., 0]), np.sin(p * x[..., 1]), np.sin(p * x[..., 2])
        return np.stack([sy * sz, sz * sx, sx * sy], axis=-1).astype(complex)

    def curlE(x):
        sx, sy, sz = np.sin(p * x[..., 0]), np.sin(p * x[..., 1]), np.sin(p * x[..., 2])
        cx, cy, cz = np.cos(p * x[..., 0]), np.cos(p * x[..., 1]), np.cos(p * x[..., 2])
        return p * np.stack([sx * (cy - cz), sy * (cz - cx), sz * (cx - cy)], axis=-1).astype(complex)
    return E, curlE


def plane_wave(p_vec: np.ndarray, k_hat: np.ndarray, k0: float):
    """Incident plane wave E = p exp(-j k0 k.r) (p perpendicular to k) and its curl -j k0 (k x p) exp(...)."""
    def E(x):
        ph = np.exp(-1j * k0 * (x @ k_hat))
        return ph[..., None] * p_vec
    kxp = np.cross(k_hat, p_vec)

    def curlE(x):
        ph = np.exp(-1j * k0 * (x @ k_hat))
        return (-1j * k0) * ph[..., None] * kxp
    return E, curlE


def seeded_plane_waves(count: int, seed: int):
    """Directions uniform on the sphere and unit polarisations perpendicular to them."""
    r = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        k = r.normal(size=3)
        k /= np.linalg.norm(k)
        t = r.normal(size=3)
        t -= (t @ k) * k
        t /= np.linalg.norm(t)
        out.append((t.astype(complex), k))
    return out


def _abc_data(E, curlE, k0):
    """U = n x curl E + j k0 n x (n x E) for the absorbing boundary condition."""
    def U(x, nrm):
        Ex = E(x)
        return np.cross(nrm, curlE(x)) + 1j * k0 * np.cross(nrm, np.cross(nrm, Ex))
    return U


# ----------------------------------------------------------------------------
# assembly
# ----------------------------------------------------------------------------
def _csr(rows, cols, vals, n):
    A = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    A.sum_duplicates()
    A.sort_indices()
    return A.indptr.astype(np.int32), A.indices.astype(np.int32), A.data.astype(np.complex128)


def build_problem(name: str, n: int, levels: int, *, jitter=0.15, mesh_seed=0,
                  split_range=None, split_seed=1, size_range=None,
                  eps="uniform", eps_seed=2, rhs="edge", rhs_seed=3, n_rhs_edges=1,
                  n_waves=0, wave_seed=4, field_seed=5, k0=K0) -> Problem:
    mesh = box_mesh(n, jitter=jitter, seed=mesh_seed)
    rng_split = np.random.default_rng(split_seed)
    rcb = rcb_cells(n, levels, split_range=split_range, rng=rng_split, size_range=size_range)
    ns = len(rcb.boxes)
    tet_sub = rcb.cell_sub[mesh.tet_cell]
    if eps == "uniform":
        eps_sub = np.full(ns, EPS_UNIFORM)
    else:
        r = np.random.default_rng(eps_seed)
        eps_sub = r.uniform(1.0, 4.0, ns) - 1j * r.uniform(0.05, 0.2, ns)
    eps_tet = eps_sub[tet_sub]

    K, M = element_matrices(mesh)
    Ae = K - (k0 ** 2) * eps_tet[:, None, None] * M
    Tf, feid = face_matrices(mesh)
    Af = 1j * k0 * Tf
    ftet = mesh.bface_tet

    te = mesh.tet_edges
    nE = mesh.n_edges
    rows = np.concatenate([np.repeat(te, 6, axis=1).ravel(), np.repeat(feid, 3, axis=1).ravel()])
    cols = np.concatenate([np.tile(te, (1, 6)).ravel(), np.tile(feid, (1, 3)).ravel()])
    vals = np.concatenate([Ae.ravel(), Af.ravel()])
    A_indptr, A_indices, A_data = _csr(rows, cols, vals, nE)

    tr = tear(te, tet_sub, nE, ns)

    # right-hand side (global) and its element / face pieces for the local loads
    x_exact = None
    rhs_edges = None
    elem_load = face_ld = None
    wave_loads = []
    if rhs == "edges+waves":
        # plane-wave sources enter through the absorbing boundary: b -= int U . N dS
        for p_vec, k_hat in seeded_plane_waves(n_waves, wave_seed):
            E, curlE = plane_wave(p_vec, k_hat, k0)
            fl, _ = face_load(mesh, _abc_data(E, curlE, k0), s=3)
            wave_loads.append(-fl)
        rhs = "edges"
    if rhs in ("edge", "edges"):
        interior = ~boundary_edge_mask(mesh)
        free = interior & (tr.edge_mult == 1)
        cand = np.nonzero(free)[0]
        if rhs == "edge":
            mid = 0.5 * (mesh.coords[mesh.edges[cand, 0]] + mesh.coords[mesh.edges[cand, 1]])
            d = np.linalg.norm(mid - SOURCE_POINT, axis=1)
            rhs_edges = np.array([cand[np.argmin(d)]])      # argmin returns the lowest index on ties
        else:
            rhs_edges = np.random.default_rng(rhs_seed).choice(cand, size=n_rhs_edges, replace=False)
        b = np.zeros((nE, rhs_edges.size + len(wave_loads)), dtype=np.complex128)
        b[rhs_edges, np.arange(rhs_edges.size)] = 1.0
        for c, fl in enumerate(wave_loads):
            b[:, rhs_edges.size + c] = _assemble_load(te[:0], np.zeros((0, 6)), feid, fl, nE)
    elif rhs == "linear":
        elem_load, face_ld, x_exact = _linear_pieces(mesh, eps_tet, k0, field_seed)
        b = _assemble_load(te, elem_load, feid, face_ld, nE)[:, None]
    elif rhs == "sine":
        E, curlE = sine_field()
        elem_load = volume_load(mesh, E, s=3) * ((2 * np.pi ** 2) - (k0 ** 2) * eps_tet[:, None])
        fl, _ = face_load(mesh, _abc_data(E, curlE, k0), s=3)
        face_ld = -fl
        b = _assemble_load(te, elem_load, feid, face_ld, nE)[:, None]
    else:
        raise ValueError(rhs)

    subs = []
    fmap_tet = ftet
    for s in range(ns):
        g = tr.l2g[s]
        tmask = tet_sub == s
        fmask = tet_sub[fmap_tet] == s
        lt = np.searchsorted(g, te[tmask])
        lf = np.searchsorted(g, feid[fmask])
        r_ = np.concatenate([np.repeat(lt, 6, axis=1).ravel(), np.repeat(lf, 3, axis=1).ravel()])
        c_ = np.concatenate([np.tile(lt, (1, 6)).ravel(), np.tile(lf, (1, 3)).ravel()])
        v_ = np.concatenate([Ae[tmask].ravel(), Af[fmask].ravel()])
        ip, ix, dv = _csr(r_, c_, v_, g.size)
        if elem_load is not None:
            f = _assemble_load(lt, elem_load[tmask], lf, face_ld[fmask], g.size)[:, None]
        else:
            f = np.zeros((g.size, b.shape[1]), dtype=np.complex128)
            for c, e in enumerate(rhs_edges):
                if tr.edge_mult[e] >= 1:
                    k = np.searchsorted(g, e)
                    if k < g.size and g[k] == e and s == _lowest_owner(tr, e, s):
                        f[k, c] = 1.0
            for c, fl in enumerate(wave_loads):
                f[:, rhs_edges.size + c] = _assemble_load(lt[:0], np.zeros((0, 6)), lf, fl[fmask], g.size)
        subs.append(Subdomain(l2g=g, indptr=ip, indices=ix, data=dv, f=f,
                              b_dual=tr.b_dual[s], b_local=tr.b_local[s], b_sign=tr.b_sign[s]))
    return Problem(name=name, mesh=mesh, k0=k0, eps_tet=eps_tet, tet_sub=tet_sub, rcb=rcb,
                   tearing=tr, A_indptr=A_indptr, A_indices=A_indices, A_data=A_data, b=b,
                   subs=subs, x_exact=x_exact, rhs_edges=rhs_edges)


def _linear_pieces(mesh: Mesh, eps_tet, k0, field_seed):
    """Element and face loads of the linear field E = a + b x r (seeded a, b)
    and its edge interpolant, the exact discrete solution."""
    r = np.random.default_rng(field_seed)
    a = r.normal(size=3) + 1j * r.normal(size=3)
    bb = r.normal(size=3) + 1j * r.normal(size=3)
    E = linear_field(a, bb)
    # curl curl E = 0, so F = -k0^2 eps_r E with each tetrahedron's own eps_r
    elem_load = volume_load(mesh, E, s=1) * (-(k0 ** 2) * eps_tet[:, None])
    U = _abc_data(E, lambda x: np.broadcast_to(2.0 * bb, x.shape).astype(complex), k0)
    fl, _ = face_load(mesh, U, s=1)
    return elem_load, -fl, interpolate(mesh, E)[:, None]


def linear_field_loads(p: Problem, field_seed=5):
    """Local loads f_i (list of (n_i, 1)) and the exact solution (n, 1) of the
    linear-field problem on p's mesh, materials and partition: the same A_i
    as p, so one factorization of p serves both.  Equal to the loads of
    build_problem(..., rhs="linear") with the same seeds."""
    mesh = p.mesh
    elem_load, face_ld, x_exact = _linear_pieces(mesh, p.eps_tet, p.k0, field_seed)
    _, feid = face_matrices(mesh)
    te = mesh.tet_edges
    f = []
    for s, sub in enumerate(p.subs):
        g = sub.l2g
        tmask = p.tet_sub == s
        fmask = p.tet_sub[mesh.bface_tet] == s
        lt = np.searchsorted(g, te[tmask])
        lf = np.searchsorted(g, feid[fmask])
        f.append(_assemble_load(lt, elem_load[tmask], lf, face_ld[fmask], g.size)[:, None])
    return f, x_exact


def _lowest_owner(tr: Tearing, e: int, s: int) -> int:
    """Lowest-index domain holding edge e (a point source goes to that copy)."""
    hits = tr.dual_pair[tr.dual_edge == e]
    return int(hits[0, 0]) if hits.size else s


def _assemble_load(te, elem_load, feid, face_ld, n):
    b = np.zeros(n, dtype=np.complex128)
    np.add.at(b, te.ravel(), elem_load.ravel())
    np.add.at(b, feid.ravel(), face_ld.ravel())
    return b


# ----------------------------------------------------------------------------
# named workloads
# ----------------------------------------------------------------------------
def plain_c1(rhs="edge", **kw) -> Problem:
    """n = 8, 8 equal domains (2x2x2), eps_r = 2 - 0.1j, 1 edge current: 4,184 DoFs."""
    return build_problem("plain-n8-s8", 8, 3, rhs=rhs, **kw)


def batched_c2(rhs="edge", **kw) -> Problem:
    """n = 41, 512 jittered-bisection domains of 500..2500 edges: 497,699 DoFs."""
    return build_problem("batched-n41-s512", 41, 9, split_range=(0.37, 0.63), size_range=(500, 2500),
                         eps="random", rhs=rhs, **kw)


def medium(rhs="edge", **kw) -> Problem:
    """n = 24, 64 jittered-bisection domains of 500..2500 edges (profiling-sized)."""
    return build_problem("medium-n24-s64", 24, 6, split_range=(0.37, 0.63), size_range=(500, 2500),
                         eps="random", rhs=rhs, **kw)


def big_domains(n: int = 24, rhs="edge", **kw) -> Problem:
    """8 equal domains (2x2x2) of an n^3 mesh: 13,428 edges each at n = 24
    (102,024 DoFs), 2,863 at n = 14 -- domains above the dense-front range,
    for the sparse-domain route."""
    return build_problem(f"big-n{n}-s8", n, 3, rhs=rhs, **kw)


def large_c4(rhs="edge", **kw) -> Problem:
    """n = 65, 2048 jittered-bisection domains of 500..2500 edges: 1,960,595 DoFs."""
    return build_problem("large-n65-s2048", 65, 11, split_range=(0.37, 0.63), size_range=(500, 2500),
                         eps="random", rhs=rhs, **kw)


def multi_rhs_c5(n_edges=56, n_waves=8, **kw) -> Problem:
    """8-domain mesh with many excitations: unit edge currents at seeded random
    interior edges (seed 3) followed by plane-wave sources through the
    absorbing boundary (seed 4); 56 + 8 = 64 right-hand sides by default."""
    if n_waves:
        return build_problem("multirhs-n8-s8", 8, 3, rhs="edges+waves", n_rhs_edges=n_edges, n_waves=n_waves, **kw)
    return build_problem("multirhs-n8-s8", 8, 3, rhs="edges", n_rhs_edges=n_edges, **kw)


def tiny(n: int, levels: int, rhs="edge", jittered=False, eps="uniform", **kw) -> Problem:
    """Small meshes for brute-force checks (n = 1..6, 2**levels domains)."""
    return build_problem(f"tiny-n{n}-l{levels}", n, levels, rhs=rhs,
                         split_range=(0.37, 0.63) if jittered else None, eps=eps, **kw)
