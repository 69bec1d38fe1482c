"""Pins of the oracle's red refinement (Section 2.3): the paper's element
counts, the new-vertex numbering against the worked example's edge table,
exact geometry of the children, and the same refined geometry as the input
generator's independent refinement (which numbers vertices its own way)."""
import numpy as np
import pytest

from conftest import read_golden_sections
from oracle import phfem_oracle as O
from paper_2401_15557_gb300 import inputs as I


def _area2(P):
    return (P[:, 1, 0] - P[:, 0, 0]) * (P[:, 2, 1] - P[:, 0, 1]) - (P[:, 2, 0] - P[:, 0, 0]) * (P[:, 1, 1] - P[:, 0, 1])


def test_level_counts_match_the_paper():
    """Level n of the criss-cross square has 4^(n+1) elements (Section 2.3)."""
    m = I.criss_cross_level0()
    xy, tri, d, n = m.xy, m.tri, m.dirichlet, m.neumann
    for level in range(1, 6):
        nV, nE = xy.shape[0], O.edge_tables(tri, xy.shape[0])["nE"]
        nD, nN = len(d), len(n)
        xy, tri, d, n = O.redrefine(xy, tri, d, n)
        assert tri.shape[0] == 4 ** (level + 1)
        assert xy.shape[0] == nV + nE
        assert len(d) == 2 * nD and len(n) == 2 * nN


def test_new_vertices_follow_the_printed_edge_numbering():
    """Vertex nV + e is the midpoint of edge e of the worked example's table."""
    g = read_golden_sections("paper_level0_tables.txt")
    e2e = np.array(g["edge2element"], dtype=np.int64)
    m = I.criss_cross_level0()
    xy, tri, d, n = O.redrefine(m.xy, m.tri, m.dirichlet, m.neumann)
    for e, row in enumerate(e2e):
        a, b = row[0] - 1, row[1] - 1
        assert np.array_equal(xy[m.nV + e], (m.xy[a] + m.xy[b]) / 2)
    # the middle child of element 1 joins the midpoints of its three edges
    mid = tri[0]
    P = m.xy[m.tri[0]]
    want = {tuple((P[(k + 1) % 3] + P[(k + 2) % 3]) / 2) for k in range(3)}
    assert {tuple(xy[v]) for v in mid} == want


@pytest.mark.parametrize("mk", ["crisscross", "lshape", "square"])
def test_children_geometry(mk):
    m = {"crisscross": lambda: I.criss_cross(1), "lshape": lambda: I.lshape_mesh(n=3, seed=I.seed_for(1, 4)),
         "square": lambda: I.square_mesh(3)}[mk]()
    xy, tri, d, n = O.redrefine(m.xy, m.tri, m.dirichlet, m.neumann)
    nT = m.nT
    Pp = m.xy[m.tri]
    Pc = xy[tri]
    A = _area2(Pp)
    Ac = _area2(Pc)
    assert np.all(Ac > 0)  # counter-clockwise children
    for k in range(4):
        idx = np.arange(nT) if k == 0 else nT + 3 * np.arange(nT) + (k - 1)
        assert np.allclose(Ac[idx], A / 4, rtol=1e-13, atol=0)
        if k > 0:  # corner child k keeps parent vertex P_k first
            assert np.array_equal(tri[idx, 0], m.tri[:, k - 1])
    # the refined mesh is a valid mesh with the refined boundary lists
    st = O.setup(I.Mesh(xy=xy, tri=tri.astype(np.int32), dirichlet=d.astype(np.int32),
                        neumann=n.astype(np.int32), name="refined"))
    assert st["bsets"]["Dbed"].size == 2 * len(m.dirichlet)
    # each half keeps the listed orientation: (a, m) then (m, b) are collinear
    k = len(m.dirichlet)
    a, mm, b = xy[d[:k, 0]], xy[d[:k, 1]], xy[d[k:, 1]]
    assert np.array_equal(d[:k, 1], d[k:, 0])
    assert np.allclose(mm, (a + b) / 2, rtol=0, atol=1e-15)


@pytest.mark.parametrize("levels", [1, 2])
def test_same_geometry_as_the_generator(levels):
    """The generator's refinement (independent code, own vertex numbering)
    yields the same set of triangles and boundary segments."""
    m = I.lshape_mesh(n=3, seed=I.seed_for(1, 11))
    xy, tri, d, n = m.xy, m.tri, m.dirichlet, m.neumann
    g = m
    for _ in range(levels):
        xy, tri, d, n = O.redrefine(xy, tri, d, n)
        g = I.red_refine(g)

    def tris(X, T):
        return sorted(tuple(map(tuple, X[t])) for t in T)

    def segs(X, D):
        return sorted(tuple(sorted((tuple(X[a]), tuple(X[b])))) for a, b in D)

    assert tris(xy, tri) == tris(g.xy, g.tri)
    assert segs(xy, d) == segs(g.xy, g.dirichlet)
    assert segs(xy, n) == segs(g.xy, g.neumann)


def _refined(m):
    xy, tri, d, n = O.redrefine(m.xy, m.tri, m.dirichlet, m.neumann)
    return xy, tri


@pytest.mark.parametrize("mk", ["lshape", "crisscross"])
def test_prolongation_reproduces_affine_functions(mk):
    """An affine function sampled at the coarse midpoints is prolongated to the
    same function at the fine midpoints (a closed form)."""
    m = {"lshape": lambda: I.lshape_mesh(n=3, seed=I.seed_for(1, 12)), "crisscross": lambda: I.criss_cross(1)}[mk]()
    xy, tri = _refined(m)
    P = O.cr_prolongation(m.xy, m.tri, xy, tri)
    g = lambda X: 0.3 - 1.7 * X[:, 0] + 0.9 * X[:, 1]
    ec = O.edge_tables(m.tri, m.nV)["ed2el"]
    ef = O.edge_tables(tri, xy.shape[0])["ed2el"]
    mc = 0.5 * (m.xy[ec[:, 0]] + m.xy[ec[:, 1]])
    mf = 0.5 * (xy[ef[:, 0]] + xy[ef[:, 1]])
    assert np.max(np.abs(P @ g(mc) - g(mf))) < 1e-13
    # constants: every row sums to one
    assert np.allclose(np.asarray(P.sum(axis=1)).ravel(), 1.0, rtol=0, atol=1e-14)


def test_prolongation_of_a_basis_function_by_hand():
    """Two triangles of the unit square, split by the diagonal (0,0)-(1,1):
    the basis function of the diagonal is 1 at its midpoint and 0 at the
    other midpoints; on each triangle it is 1 - 2 lambda of the opposite
    vertex.  At the fine midpoints: 1 on the diagonal's halves, 1/2 on the
    four interior edges that touch its midpoint, 0 on the two interior edges
    that do not, and +1/2 / -1/2 on the halves of the outer edges near a
    vertex on / off the diagonal (at the quarter point next to the vertex P
    off the diagonal, lambda_P = 3/4)."""
    m = I.square_mesh(1)
    xy, tri = _refined(m)
    P = O.cr_prolongation(m.xy, m.tri, xy, tri).toarray()
    ec = O.edge_tables(m.tri, m.nV)["ed2el"]
    diag = [e for e in range(ec.shape[0]) if {tuple(m.xy[ec[e, 0]]), tuple(m.xy[ec[e, 1]])} == {(0.0, 0.0), (1.0, 1.0)}]
    assert len(diag) == 1
    col = P[:, diag[0]]
    ef = O.edge_tables(tri, xy.shape[0])["ed2el"]
    mid = 0.5 * (xy[ef[:, 0]] + xy[ef[:, 1]])
    for f in range(ef.shape[0]):
        x, y = mid[f]
        on_diag = abs(x - y) < 1e-15
        a, b = xy[ef[f, 0]], xy[ef[f, 1]]
        outer = any(abs(c) < 1e-15 or abs(c - 1) < 1e-15 for c in (x, y)) and not on_diag
        if on_diag and (abs(x - 0.25) < 1e-15 or abs(x - 0.75) < 1e-15) and (0.5 in (a[0], b[0])):
            assert col[f] == 1.0            # halves of the diagonal
        elif outer:
            # half of an outer edge near a diagonal vertex (0,0) or (1,1): +1/2, else -1/2
            near_diag_vertex = max(x, y) < 0.5 or min(x, y) > 0.5
            assert col[f] == (0.5 if near_diag_vertex else -0.5), (x, y, col[f])
        else:
            touches = any(np.allclose(v, (0.5, 0.5)) for v in (a, b))
            assert col[f] == (0.5 if touches else 0.0), (x, y, col[f])
