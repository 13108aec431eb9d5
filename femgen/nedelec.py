"""Lowest-order Nedelec (Whitney edge) elements on tetrahedra.

The paper's FEM models are curl-curl Maxwell boundary value problems
discretised with edge elements (Section I, Section II).  It gives no element
formulas, so this module writes the textbook ones:

* basis of edge e = (a, b), a < b:  N_e = l_a grad(l_b) - l_b grad(l_a),
  with curl N_e = 2 grad(l_a) x grad(l_b)   (l = barycentric coordinates);
* stiffness  K_ef = V (curl N_e) . (curl N_f);
* mass       M_ef = int N_e . N_f, using int l_p l_q dV = V (1 + d_pq) / 20;
* absorbing-boundary face matrix T_ef = int (n x N_e).(n x N_f) dS
  = int N_e,t . N_f,t dS, using int l_p l_q dS = A (1 + d_pq) / 12.

Time convention exp(+j w t).  The element matrix of the lossy, first-order
absorbing-boundary problem is K - k0^2 eps_r M (+ j k0 T on outer faces): from
curl curl E - k0^2 eps_r E = F with n x curl E + j k0 n x n x E = U on the
outer boundary, the weak form is
    a(E, v) = int curl E . curl v - k0^2 eps_r E . v dV + j k0 int E_t . v_t dS
    l(v)    = int F . v dV - int U . v dS.
"""
from __future__ import annotations

import math
from functools import lru_cache
from itertools import combinations_with_replacement

import numpy as np

from .mesh import TET_EDGES, TET_FACES, Mesh

# edges of a triangle with sorted vertices (local to the face)
TRI_EDGES = np.array([(0, 1), (0, 2), (1, 2)], dtype=np.int64)


def barycentric_gradients(P: np.ndarray):
    """P: (T, 4, 3) vertex coordinates -> (grads (T, 4, 3), signed volume (T,))."""
    J = np.transpose(P[:, 1:, :] - P[:, 0:1, :], (0, 2, 1))  # columns = edge vectors
    det = np.linalg.det(J)
    Jinv = np.linalg.inv(J)                                   # rows = grad l_1..l_3
    g = np.empty((P.shape[0], 4, 3))
    g[:, 1:, :] = Jinv
    g[:, 0, :] = -Jinv.sum(axis=1)
    return g, det / 6.0


def _four_term(Ml: np.ndarray, GG: np.ndarray, pairs: np.ndarray) -> np.ndarray:
    """sum of int l_p l_q * (grad . grad) over the four terms of N_e . N_f.

    Ml: (..., k, k) integrals of l_p l_q; GG: (..., k, k) gradient dots;
    pairs: (m, 2) local vertex pairs of the m edges.  Returns (..., m, m).
    """
    a = pairs[:, 0]
    b = pairs[:, 1]
    A = a[:, None]
    B = b[:, None]
    C = a[None, :]
    D = b[None, :]
    return (Ml[..., A, C] * GG[..., B, D] - Ml[..., A, D] * GG[..., B, C]
            - Ml[..., B, C] * GG[..., A, D] + Ml[..., B, D] * GG[..., A, C])


def element_matrices(mesh: Mesh):
    """Stiffness and mass matrices of every tetrahedron: (T, 6, 6) each, real."""
    P = mesh.coords[mesh.tets]
    g, vol = barycentric_gradients(P)
    V = np.abs(vol)
    curl = 2.0 * np.cross(g[:, TET_EDGES[:, 0], :], g[:, TET_EDGES[:, 1], :])   # (T, 6, 3)
    K = V[:, None, None] * np.einsum("tei,tfi->tef", curl, curl)
    GG = np.einsum("tpi,tqi->tpq", g, g)
    Ml = (np.ones((4, 4)) + np.eye(4)) / 20.0
    M = V[:, None, None] * _four_term(Ml[None], GG, TET_EDGES)
    return K, M


def face_geometry(mesh: Mesh):
    """Vertices (F, 3, 3), surface barycentric gradients (F, 3, 3), areas (F,)."""
    tv = mesh.tets[mesh.bface_tet]                     # (F, 4)
    fv = np.take_along_axis(tv, TET_FACES[mesh.bface_local], axis=1)  # (F, 3) sorted
    X = mesh.coords[fv]
    e1 = X[:, 1] - X[:, 0]
    e2 = X[:, 2] - X[:, 0]
    nrm = np.cross(e1, e2)
    area2 = np.linalg.norm(nrm, axis=1)
    nh = nrm / area2[:, None]
    # in-plane gradients: grad l_1 = (e2 x n)/(2A) ... via the metric tensor
    G = np.stack([e1, e2], axis=1)                      # (F, 2, 3)
    Gm = np.einsum("fai,fbi->fab", G, G)
    Ginv = np.linalg.inv(Gm)
    g12 = np.einsum("fab,fbi->fai", Ginv, G)            # grads of l_1, l_2
    gs = np.empty((X.shape[0], 3, 3))
    gs[:, 1:, :] = g12
    gs[:, 0, :] = -g12.sum(axis=1)
    return fv, X, gs, 0.5 * area2, nh


def face_matrices(mesh: Mesh):
    """ABC face matrices T (F, 3, 3) and the global edge ids of the face edges (F, 3)."""
    fv, X, gs, area, _ = face_geometry(mesh)
    GG = np.einsum("fpi,fqi->fpq", gs, gs)
    Ml = (np.ones((3, 3)) + np.eye(3)) / 12.0
    T = area[:, None, None] * _four_term(Ml[None], GG, TRI_EDGES)
    return T, face_edge_ids(mesh, fv)


def face_edge_ids(mesh: Mesh, fv: np.ndarray) -> np.ndarray:
    """Global edge ids (F, 3) of the edges of triangles with sorted vertices fv (F, 3)."""
    V = mesh.coords.shape[0]
    keys = fv[:, TRI_EDGES[:, 0]] * V + fv[:, TRI_EDGES[:, 1]]
    ekeys = mesh.edges[:, 0] * V + mesh.edges[:, 1]
    eid = np.searchsorted(ekeys, keys)
    assert np.all(ekeys[eid] == keys)
    return eid


# ----------------------------------------------------------------------------
# quadrature: Grundmann-Moeller rules on the n-simplex (Grundmann & Moeller,
# SIAM J. Numer. Anal. 15 (1978) 282-290), degree d = 2 s + 1.
# ----------------------------------------------------------------------------
def _compositions(total: int, parts: int):
    """All tuples of `parts` non-negative ints summing to `total`."""
    for c in combinations_with_replacement(range(parts), total):
        out = [0] * parts
        for k in c:
            out[k] += 1
        yield out


@lru_cache(maxsize=None)
def grundmann_moeller(dim: int, s: int):
    """Barycentric points (Q, dim+1) and weights (Q,) summing to 1 (unit measure).

    Rule of degree 2s+1 on the dim-simplex.  Weights are normalised to the
    simplex measure, so integral = measure * sum_q w_q f(x_q).
    """
    d = 2 * s + 1
    pts, wts = [], []
    for i in range(s + 1):
        denom = d + dim - 2 * i
        w = ((-1) ** i) * 2.0 ** (-2 * s) * denom ** d / (math.factorial(i) * math.factorial(d + dim - i))
        seen = set()
        for beta in _compositions(s - i, dim + 1):
            key = tuple(beta)
            if key in seen:
                continue
            seen.add(key)
            pts.append([(2 * bj + 1) / denom for bj in beta])
            wts.append(w)
    pts = np.array(pts)
    wts = np.array(wts) * math.factorial(dim)   # standard simplex has measure 1/dim!
    return pts, wts


def whitney_values(lam: np.ndarray, g: np.ndarray, pairs: np.ndarray) -> np.ndarray:
    """N_e at barycentric points.  lam (T, Q, k), g (T, k, 3) -> (T, Q, m, 3)."""
    a = pairs[:, 0]
    b = pairs[:, 1]
    return (lam[:, :, a, None] * g[:, None, b, :] - lam[:, :, b, None] * g[:, None, a, :])


def volume_load(mesh: Mesh, F, s: int = 2) -> np.ndarray:
    """Element loads int F . N_e dV: (T, 6) complex.  F(x) maps (..., 3) points to complex (..., 3)."""
    lam, w = grundmann_moeller(3, s)
    P = mesh.coords[mesh.tets]
    g, vol = barycentric_gradients(P)
    V = np.abs(vol)
    X = np.einsum("qk,tki->tqi", lam, P)
    Fx = F(X)                                             # (T, Q, 3)
    N = whitney_values(np.broadcast_to(lam, (P.shape[0],) + lam.shape), g, TET_EDGES)
    return V[:, None] * np.einsum("q,tqi,tqei->te", w, Fx, N)


def face_load(mesh: Mesh, U, s: int = 2):
    """Face loads int U . N_e dS: (F, 3) complex and the face edge ids (F, 3).

    U(x, n) maps points (..., 3) and outward normals (..., 3) to complex (..., 3).
    """
    lam, w = grundmann_moeller(2, s)
    fv, X, gs, area, _ = face_geometry(mesh)
    nrm = mesh.bface_normal
    Xq = np.einsum("qk,fki->fqi", lam, X)
    Ux = U(Xq, np.broadcast_to(nrm[:, None, :], Xq.shape))
    N = whitney_values(np.broadcast_to(lam, (X.shape[0],) + lam.shape), gs, TRI_EDGES)
    return area[:, None] * np.einsum("q,fqi,fqei->fe", w, Ux, N), face_edge_ids(mesh, fv)


def interpolate(mesh: Mesh, E, s: int = 3) -> np.ndarray:
    """Edge degrees of freedom x_e = int_e E . t ds (t from vertex a to b)."""
    # Gauss-Legendre on the segment (exact for polynomials of degree 2s+1)
    t, w = np.polynomial.legendre.leggauss(s + 1)
    t = 0.5 * (t + 1.0)
    w = 0.5 * w
    xa = mesh.coords[mesh.edges[:, 0]]
    xb = mesh.coords[mesh.edges[:, 1]]
    d = xb - xa
    pts = xa[:, None, :] + t[None, :, None] * d[:, None, :]
    Ex = E(pts)                                           # (E, Q, 3)
    return np.einsum("q,eqi,ei->e", w, Ex, d)


def evaluate(mesh: Mesh, x: np.ndarray, lam: np.ndarray):
    """Field and curl of sum_e x_e N_e at barycentric points lam (Q, 4) of every tet.

    Returns points (T, Q, 3), field (T, Q, 3), curl (T, 3) (constant per tet).
    """
    P = mesh.coords[mesh.tets]
    g, _ = barycentric_gradients(P)
    xe = x[mesh.tet_edges]                                # (T, 6)
    N = whitney_values(np.broadcast_to(lam, (P.shape[0],) + lam.shape), g, TET_EDGES)
    field = np.einsum("te,tqei->tqi", xe, N)
    curl = 2.0 * np.einsum("te,tei->ti", xe,
                           np.cross(g[:, TET_EDGES[:, 0], :], g[:, TET_EDGES[:, 1], :]))
    X = np.einsum("qk,tki->tqi", lam, P)
    return X, field, curl
