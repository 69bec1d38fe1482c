"""Pins of the oracle's topology (Section 2.2) against the paper's worked
example and against invariants that any correct edge table satisfies."""
import numpy as np
import pytest

from conftest import read_golden_sections
from oracle import phfem_oracle as O
from paper_2401_15557_gb300 import inputs as I


def test_paper_worked_example_tables():
    g = read_golden_sections("paper_level0_tables.txt")
    m = I.criss_cross_level0()
    topo = O.edge_tables(m.tri, m.nV)
    n2el = O.nodes2element(m.tri.astype(np.int64), m.nV).toarray()
    assert np.array_equal(n2el, np.array(g["nodes2element"], dtype=np.int64))
    assert np.array_equal(topo["n2ed"].toarray(), np.array(g["nodes2edge"], dtype=np.int64))
    ed2el = topo["ed2el"].copy()
    ed2el[:, :3] += 1
    ed2el[:, 3] = np.where(ed2el[:, 3] >= 0, ed2el[:, 3] + 1, 0)
    assert np.array_equal(ed2el, np.array(g["edge2element"], dtype=np.int64))


def test_paper_example_boundary_sets():
    m = I.criss_cross_level0()
    st = O.setup(m)
    # Dirichlet pairs (1,2),(2,4) are edges 1 and 3; Neumann (4,3),(3,1) edges 4 and 2
    assert sorted((st["bsets"]["Dbed"] + 1).tolist()) == [1, 3]
    assert sorted((st["bsets"]["Nbed"] + 1).tolist()) == [2, 4]
    assert (st["bsets"]["Redges"] + 1).tolist() == [1, 3, 5, 6, 7, 8]


def _random_meshes():
    yield I.square_mesh(5)
    yield I.criss_cross(2)
    yield I.lshape_mesh(n=4, seed=I.seed_for(1, 7))
    yield I.red_refine(I.lshape_mesh(n=3, seed=I.seed_for(1, 8)))


@pytest.mark.parametrize("mesh", list(_random_meshes()), ids=lambda m: m.name)
def test_edge_table_invariants(mesh):
    topo = O.edge_tables(mesh.tri, mesh.nV)
    tri = mesh.tri.astype(np.int64)
    ed2el, t2e, sigma = topo["ed2el"], topo["t2e"], topo["sigma"]
    nT, nE = tri.shape[0], topo["nE"]
    # Euler: V - E + F = 1 for a simply connected planar triangulation
    assert mesh.nV - nE + nT == 1
    # edges numbered by (max vertex, min vertex) lexicographically
    lo = np.minimum(ed2el[:, 0], ed2el[:, 1])
    hi = np.maximum(ed2el[:, 0], ed2el[:, 1])
    key = hi * mesh.nV + lo
    assert np.all(np.diff(key) > 0)
    # every edge appears in t2e once per owner, with sigma +1 in T+ and -1 in T-
    owners = np.bincount(t2e.ravel(), minlength=nE)
    assert np.array_equal(owners, np.where(ed2el[:, 3] >= 0, 2, 1))
    for m in range(nT):
        for k in range(3):
            e = t2e[m, k]
            a, b = tri[m, (k + 1) % 3], tri[m, (k + 2) % 3]
            assert {a, b} == {ed2el[e, 0], ed2el[e, 1]}
            if sigma[m, k] > 0:
                assert ed2el[e, 2] == m
                # (initial, end) is the counter-clockwise direction in T+
                assert (ed2el[e, 0], ed2el[e, 1]) == (a, b)
            else:
                assert ed2el[e, 3] == m
    # T+ is the lower element index of the two
    inter = ed2el[:, 3] >= 0
    assert np.all(ed2el[inter, 2] < ed2el[inter, 3])
    # boundary edges are exactly the listed Dirichlet and Neumann pairs
    st = O.setup(mesh)
    assert st["bsets"]["Dbed"].size + st["bsets"]["Nbed"].size == int((~inter).sum())


def test_invalid_meshes_rejected():
    m = I.square_mesh(2)
    bad = m.tri.copy()
    bad[0] = bad[0, [0, 2, 1]]        # clockwise triangle
    with pytest.raises(ValueError):
        O.element_geometry(m.xy, bad.astype(np.int64))
    with pytest.raises(ValueError):   # the same directed edge in two elements
        O.nodes2element(np.vstack([m.tri, m.tri[:1]]).astype(np.int64), m.nV)
    with pytest.raises(ValueError):   # an unlisted boundary edge
        O.boundary_sets(O.edge_tables(m.tri, m.nV), m.dirichlet, m.neumann[1:])
    with pytest.raises(ValueError):   # an edge both Dirichlet and Neumann
        O.boundary_sets(O.edge_tables(m.tri, m.nV), m.dirichlet, np.vstack([m.neumann, m.dirichlet[:1]]))
