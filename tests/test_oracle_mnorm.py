"""Pins of the oracle's multiplier error norm (m_norm_error).

The paper measures kappa - kappa_h in the mesh norm of Section 3.1 but does not
print how; the oracle computes sqrt(sum over multiplier edges E of |E| times
the integral over E of (kappa - Lambda_E)^2).  These cases fix that formula with
values worked out by hand on the two-triangle unit square (Dirichlet x = 0, 1;
Neumann y = 0, 1; diagonal from (0, 0) to (1, 1)), so that a dropped edge class,
a wrong power of |E|, a wrong quadrature or a wrong normal fails one of them.
They pin the formula, not the paper's M-norm column, which no variant
reproduces.
"""
import numpy as np
import pytest

from oracle import phfem_oracle as O
from paper_2401_15557_gb300 import inputs as I


def _two_triangles():
    mesh = I.square_mesh(1)
    st = O.setup(mesh, I.problem_sine_exp())
    red = st["bsets"]["Redges"]
    ends = st["xy"][st["topo"]["ed2el"][red, :2]]
    lengths = np.hypot(*(ends[:, 1] - ends[:, 0]).T)
    return st, red, lengths


def test_multiplier_edges_of_the_two_triangle_square():
    _, red, lengths = _two_triangles()
    # x = 0 and x = 1 (Dirichlet) and the interior diagonal; the Neumann sides carry no multiplier
    assert len(red) == 3
    assert sorted(lengths) == pytest.approx([1.0, 1.0, np.sqrt(2.0)], abs=1e-15)


@pytest.mark.parametrize("shift", [(1.0, 1.0, 1.0), (0.5, -2.0, 3.0)])
def test_constant_offsets_from_the_exact_flux(shift):
    """Linear u: kappa is constant on every edge; Lambda = kappa + c_E gives
    sum_E |E| * |E| c_E^2 exactly."""
    st, red, lengths = _two_triangles()
    grad = lambda x, y: (2.0 + 0 * x, -3.0 + 0 * y)
    kappa = O.exact_flux(st, grad)
    c = np.array(shift)
    got = O.m_norm_error(st, kappa + c, grad)
    want = np.sqrt(np.sum(lengths ** 2 * c ** 2))
    assert got == pytest.approx(want, rel=1e-14)


def test_flux_linear_along_the_diagonal():
    """u = x^2, Lambda = 0: on x = 1 kappa = 2 (1 * 1 * 4 = 4); on x = 0 kappa = 0;
    on the diagonal kappa = +-sqrt(2) s at (s, s), so |E| int_E kappa^2 =
    sqrt(2) * sqrt(2) * int_0^1 2 s^2 ds = 4/3.  Total 16/3."""
    st, red, _ = _two_triangles()
    grad = lambda x, y: (2.0 * x, 0 * y)
    got = O.m_norm_error(st, np.zeros(len(red)), grad)
    assert got == pytest.approx(4.0 / np.sqrt(3.0), rel=1e-14)


def test_neumann_edges_are_left_out():
    """u = x^2 + y^2, Lambda = 0: kappa = 2 on x = 1 (4), 0 on x = 0 and on the
    diagonal (grad u is parallel to it); the Neumann side y = 1 has kappa = 2 as
    well but carries no multiplier, so the norm is 2, not sqrt(8)."""
    st, red, _ = _two_triangles()
    grad = lambda x, y: (2.0 * x, 2.0 * y)
    got = O.m_norm_error(st, np.zeros(len(red)), grad)
    assert got == pytest.approx(2.0, rel=1e-14)


def test_scaling_with_the_mesh():
    """On the n x n square an offset of 1 on every multiplier edge gives
    sqrt(sum over multiplier edges of |E|^2), with the edge counts of the
    structured mesh written out below."""
    n = 4
    mesh = I.square_mesh(n)
    st = O.setup(mesh, I.problem_sine_exp())
    grad = lambda x, y: (0 * x + 1.0, 0 * y)
    kappa = O.exact_flux(st, grad)
    got = O.m_norm_error(st, kappa + 1.0, grad)
    h = 1.0 / n
    # multiplier edges: vertical edges x = i h for i = 0..n (all Dirichlet or
    # interior): (n + 1) n of length h; interior horizontal edges: (n - 1) n of
    # length h; diagonals: n^2 of length sqrt(2) h
    want2 = ((n + 1) * n + (n - 1) * n) * h ** 2 + n * n * 2.0 * h ** 2
    assert got == pytest.approx(np.sqrt(want2), rel=1e-13)
