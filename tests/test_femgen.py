"""Pins of the seeded input generator (mesh, Whitney elements, tearing).

The paper gives no element formulas or meshes, so these checks rest on
closed forms: edge counts of the Kuhn split, the curl of a gradient being
zero, exact reproduction of constant and linear fields, and first-order
convergence on a smooth manufactured solution.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import femgen
from femgen.mesh import box_mesh, kuhn_edge_count, tet_volumes, TET_EDGES
from femgen.nedelec import (barycentric_gradients, element_matrices, evaluate, face_geometry,
                            face_matrices, grundmann_moeller, whitney_values, TRI_EDGES)
from femgen.problems import sine_field


@pytest.mark.parametrize("n,expected", [(1, 19), (2, 98), (3, 279), (8, 4184), (41, 497699), (65, 1960595)])
def test_edge_count_closed_form(n, expected):
    assert kuhn_edge_count(n, n, n) == expected
    if n <= 8:
        assert box_mesh(n).n_edges == expected


def test_mesh_valid_and_conforming():
    m = box_mesh(5, seed=3)
    vol = tet_volumes(m.coords, m.tets)
    assert np.all(np.abs(vol) > 0.05 * m.h ** 3 / 6)
    assert np.isclose(np.abs(vol).sum(), 1.0, rtol=0, atol=1e-13)
    # every interior triangle is shared by exactly two tets, boundary ones by one
    faces = np.sort(m.tets[:, [[0, 1, 2], [0, 1, 3], [0, 2, 3], [1, 2, 3]]].reshape(-1, 3), axis=1)
    _, cnt = np.unique(faces, axis=0, return_counts=True)
    assert set(np.unique(cnt)) <= {1, 2}
    assert (cnt == 1).sum() == m.bface_tet.size == 6 * 2 * 25
    # the boundary is unjittered
    on = np.any((m.grid == 0) | (m.grid == m.n), axis=1)
    assert np.array_equal(m.coords[on], m.grid[on] * m.h)


def test_gm_quadrature_exact_on_monomials():
    # integral over the unit tetrahedron of x^a y^b z^c = a! b! c! / (a+b+c+3)!
    from math import factorial
    lam, w = grundmann_moeller(3, 3)          # degree 7
    pts = lam[:, 1:]
    for a, b, c in [(0, 0, 0), (1, 0, 0), (2, 1, 0), (3, 2, 2), (1, 1, 1), (4, 0, 3)]:
        exact = factorial(a) * factorial(b) * factorial(c) / factorial(a + b + c + 3)
        approx = (1.0 / 6.0) * np.sum(w * pts[:, 0] ** a * pts[:, 1] ** b * pts[:, 2] ** c)
        assert abs(approx - exact) < 1e-15
    lam2, w2 = grundmann_moeller(2, 2)        # degree 5 on the triangle
    for a, b in [(0, 0), (2, 3), (1, 4), (5, 0)]:
        exact = factorial(a) * factorial(b) / factorial(a + b + 2)
        approx = 0.5 * np.sum(w2 * lam2[:, 1] ** a * lam2[:, 2] ** b)
        assert abs(approx - exact) < 1e-15


def test_curl_of_gradient_is_zero():
    m = box_mesh(3, seed=1)
    K, M = element_matrices(m)
    phi = np.random.default_rng(0).normal(size=m.coords.shape[0])
    xg = phi[m.edges[:, 1]] - phi[m.edges[:, 0]]             # edge dofs of grad(phi)
    Kx = np.einsum("tef,tf->te", K, xg[m.tet_edges])
    assert np.abs(Kx).max() < 1e-12 * np.abs(K).max()
    # but the mass matrix sees it
    assert np.abs(np.einsum("tef,tf->te", M, xg[m.tet_edges])).max() > 1e-3


def test_constant_field_reproduction():
    m = box_mesh(3, seed=2)
    K, M = element_matrices(m)
    P = m.coords[m.tets]
    g, vol = barycentric_gradients(P)
    V = np.abs(vol)
    c = np.array([0.3, -1.2, 0.7])
    u = (m.coords[m.edges[:, 1]] - m.coords[m.edges[:, 0]]) @ c
    ue = u[m.tet_edges]
    # pointwise reproduction at random barycentric points
    lam = np.random.default_rng(1).dirichlet(np.ones(4), size=5)
    N = whitney_values(np.broadcast_to(lam, (P.shape[0],) + lam.shape), g, TET_EDGES)
    field = np.einsum("te,tqei->tqi", ue, N)
    assert np.abs(field - c).max() < 1e-12
    assert np.allclose(np.einsum("te,tef,tf->t", ue, M, ue), V * (c @ c), rtol=1e-12, atol=0)
    assert np.abs(np.einsum("te,tef,tf->t", ue, K, ue)).max() < 1e-12
    # absorbing-boundary face matrix: u^T T u = area * |c_t|^2
    T, eid = face_matrices(m)
    _, _, _, area, nh = face_geometry(m)
    uf = u[eid]
    ct = c[None, :] - (nh @ c)[:, None] * nh
    assert np.allclose(np.einsum("fe,fek,fk->f", uf, T, uf), area * np.sum(ct ** 2, axis=1), rtol=1e-12)


def test_global_matrix_symmetric_and_lossy(c1):
    A = c1.A_csr()
    assert abs(A - A.T).max() <= 1e-14 * abs(A).max()
    # Im(x^H A x) > 0 on random vectors (lossy material + absorbing boundary)
    rng = np.random.default_rng(4)
    for _ in range(5):
        x = rng.normal(size=c1.n) + 1j * rng.normal(size=c1.n)
        assert (x.conj() @ (A @ x)).imag > 0


def test_c1_sizes(c1):
    assert c1.n == 4184 and c1.n_sub == 8 and c1.n_dual == 648
    assert all(s.n == 604 for s in c1.subs)
    assert int((c1.tearing.edge_mult > 1).sum()) == 600
    assert int((c1.tearing.edge_mult == 4).sum()) == 24


def test_tearing_invariants(c1):
    p = c1
    n_tot = sum(s.n for s in p.subs)
    R = sp.csr_matrix((np.ones(n_tot), (np.arange(n_tot), np.concatenate([s.l2g for s in p.subs]))),
                      shape=(n_tot, p.n))
    Ablk = sp.block_diag([sp.csr_matrix((s.data, s.indices, s.indptr), shape=(s.n, s.n)) for s in p.subs])
    # sum_i R_i^T A_i R_i = A, sum_i R_i^T f_i = b
    assert abs(R.T @ Ablk @ R - p.A_csr()).max() < 1e-12 * abs(p.A_csr()).max()
    f = np.concatenate([s.f for s in p.subs])
    assert np.abs(R.T @ f - p.b).max() == 0
    # B (R x) = 0 for a continuous x and B has full row rank
    offs = np.cumsum([0] + [s.n for s in p.subs])
    rows = np.concatenate([s.b_dual for s in p.subs])
    cols = np.concatenate([o + s.b_local for o, s in zip(offs, p.subs)])
    vals = np.concatenate([s.b_sign for s in p.subs]).astype(float)
    B = sp.csr_matrix((vals, (rows, cols)), shape=(p.n_dual, n_tot))
    x = np.random.default_rng(0).normal(size=p.n)
    assert np.abs(B @ (R @ x)).max() < 1e-14
    assert np.linalg.matrix_rank(B.toarray()) == p.n_dual
    # every multiplier couples exactly two domains with opposite signs
    per = np.bincount(rows, minlength=p.n_dual)
    assert np.all(per == 2) and np.all(np.bincount(rows, weights=vals, minlength=p.n_dual) == 0)


def test_batched_partition_sizes():
    """512 domains of 500..2500 edges, spread out (roughly lognormal)."""
    from femgen.decompose import rcb_cells
    tree = rcb_cells(41, 9, split_range=(0.37, 0.63), rng=np.random.default_rng(1), size_range=(500, 2500))
    sizes = np.array([kuhn_edge_count(*(hi - lo)) for lo, hi in tree.boxes])
    assert sizes.size == 512 and sizes.min() >= 500 and sizes.max() <= 2500
    assert np.std(np.log(sizes)) > 0.3
    # binary tree in post-order: leaves 0..511, every parent after its children, root last
    assert tree.parent[-1] == -1
    assert np.all(tree.parent[:-1] > np.arange(1022))
    assert np.all(np.bincount(tree.parent[:-1], minlength=1023)[512:] == 2)


@pytest.mark.parametrize("n,levels", [(2, 1), (3, 2), (8, 3)])
def test_exact_in_space_linear_field(n, levels):
    """E = a + b x r lies in the Nedelec space, so the Galerkin solution is its interpolant."""
    p = femgen.build_problem("lin", n, levels, rhs="linear")
    x = spla.spsolve(p.A_csr().tocsc(), p.b[:, 0])
    assert np.linalg.norm(x - p.x_exact[:, 0]) <= 1e-12 * np.linalg.norm(p.x_exact)


def test_convergence_rate_sine_field():
    """First-order H(curl) convergence on the manufactured smooth field."""
    E, curlE = sine_field()
    lam, w = grundmann_moeller(3, 3)
    errs = []
    for n in (4, 8, 16):
        p = femgen.build_problem("sin", n, 1, rhs="sine")
        x = spla.spsolve(p.A_csr().tocsc(), p.b[:, 0])
        X, fld, crl = evaluate(p.mesh, x, lam)
        _, vol = barycentric_gradients(p.mesh.coords[p.mesh.tets])
        V = np.abs(vol)
        e2 = np.sum(V * np.einsum("q,tq->t", w, np.sum(np.abs(E(X) - fld) ** 2, -1)))
        c2 = np.sum(V * np.einsum("q,tq->t", w, np.sum(np.abs(curlE(X) - crl[:, None, :]) ** 2, -1)))
        errs.append((np.sqrt(e2), np.sqrt(c2)))
    errs = np.array(errs)
    rates = np.log2(errs[:-1] / errs[1:])
    assert np.all(rates >= 0.9), rates


def test_plane_wave_curl_and_boundary_load():
    """curl of the incident plane wave matches central differences, and the
    64-excitation set splits exactly into domain loads (sum R_i^T f_i = b)."""
    from femgen.problems import plane_wave, seeded_plane_waves
    (p_vec, k_hat), = seeded_plane_waves(1, 4)
    assert abs(p_vec @ k_hat) < 1e-14
    E, curlE = plane_wave(p_vec, k_hat, 2 * np.pi)
    x = np.random.default_rng(0).uniform(size=(5, 3))
    h = 1e-6
    num = np.zeros((5, 3), dtype=complex)
    d = lambda i: np.eye(3)[i] * h
    dE = [(E(x + d(i)) - E(x - d(i))) / (2 * h) for i in range(3)]   # dE/dx_i
    num[:, 0] = dE[1][:, 2] - dE[2][:, 1]
    num[:, 1] = dE[2][:, 0] - dE[0][:, 2]
    num[:, 2] = dE[0][:, 1] - dE[1][:, 0]
    assert np.abs(num - curlE(x)).max() < 1e-6
    p = femgen.multi_rhs_c5()
    assert p.b.shape == (p.n, 64)
    n_tot = sum(s.n for s in p.subs)
    R = sp.csr_matrix((np.ones(n_tot), (np.arange(n_tot), np.concatenate([s.l2g for s in p.subs]))),
                      shape=(n_tot, p.n))
    f = np.concatenate([s.f for s in p.subs])
    assert np.abs(R.T @ f - p.b).max() <= 1e-15 * np.abs(p.b).max()
    assert np.all(np.abs(p.b[:, 56:]).max(axis=0) > 0.1)


def test_linear_field_loads_match_the_linear_problem():
    """linear_field_loads on an edge-current problem gives the loads and exact
    solution of the same mesh built with rhs="linear" (same matrices)."""
    a = femgen.tiny(4, 3, jittered=True, eps="random", rhs="linear")
    b = femgen.tiny(4, 3, jittered=True, eps="random")
    f, x = femgen.linear_field_loads(b)
    for sa, sb, fb in zip(a.subs, b.subs, f):
        assert np.array_equal(sa.data, sb.data)
        assert np.array_equal(sa.f, fb)
    assert np.array_equal(a.x_exact, x)
