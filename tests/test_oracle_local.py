"""Pins of the oracle's local matrices (Definition 3.1) against closed forms
and quadrature computed independently of the oracle's formulas."""
import numpy as np
import pytest

from oracle import phfem_oracle as O


def cross2(u, v):
    return u[0] * v[1] - u[1] * v[0]



def _geo(P):
    xy = np.asarray(P, dtype=np.float64)
    return O.element_geometry(xy, np.array([[0, 1, 2]]))


def _quad_points():
    # 7-point rule built from the vertices, edge midpoints and centroid
    # (exact for cubics): weights 1/20, 2/15, 9/20 of |T|.
    bary = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (0, .5, .5), (.5, 0, .5), (.5, .5, 0), (1 / 3, 1 / 3, 1 / 3)]
    w = [1 / 20] * 3 + [2 / 15] * 3 + [9 / 20]
    return np.array(bary), np.array(w)


def test_right_isoceles_stiffness_closed_form():
    # right angle at P1: B = 1/2 [[2,-1,-1],[-1,1,0],[-1,0,1]] for A = I
    geo = _geo([[0, 0], [1, 0], [0, 1]])
    loc = O.local_matrices(geo)
    ref = 0.5 * np.array([[2, -1, -1], [-1, 1, 0], [-1, 0, 1]])
    assert np.allclose(loc["B"][0], ref, atol=1e-15)
    # scaling by a and the stiffness does not depend on size
    geo2 = _geo([[3, 3], [3.5, 3], [3, 3.5]])
    assert np.allclose(O.local_matrices(geo2, aT=2.5)["B"][0], 2.5 * ref, atol=1e-14)


def test_general_triangle_invariants():
    rng = np.random.default_rng(0)
    for _ in range(20):
        P = rng.uniform(-1, 1, (3, 2))
        if cross2(P[1] - P[0], P[2] - P[0]) < 0:
            P = P[[0, 2, 1]]
        geo = _geo(P)
        area = 0.5 * abs(cross2(P[1] - P[0], P[2] - P[0]))
        assert np.isclose(geo["area"][0], area)
        loc = O.local_matrices(geo, aT=1.7, p=(0.3, -0.8), delta=0.9)
        B, M0, D = loc["B"][0], loc["M0"][0], loc["D"][0]
        assert np.allclose(B, B.T)
        assert np.allclose(B.sum(axis=1), 0, atol=1e-12)      # constants are in the kernel
        w = np.linalg.eigvalsh(B)
        assert w[0] > -1e-12 and w[1] > 1e-8                  # PSD, one-dimensional kernel
        assert np.isclose(M0.sum(), area)                     # sum of int lambda_i lambda_j = |T|
        assert np.allclose(loc["M"][0], 0.9 * M0)
        # mass and convection against quadrature of the barycentric functions
        bary, wq = _quad_points()
        Mq = area * np.einsum("q,qi,qj->ij", wq, bary, bary)
        assert np.allclose(M0, Mq, atol=1e-14)
        # D[r, c] = int lambda_r p.grad lambda_c
        G = geo["grads"][0]
        Dq = area * np.einsum("q,qr,c->rc", wq, bary, G @ np.array([0.3, -0.8]))
        assert np.allclose(D, Dq, atol=1e-13)
        # stiffness against the classical cotangent formula of P1 elements
        cot = []
        for k in range(3):
            a, b, c = P[k], P[(k + 1) % 3], P[(k + 2) % 3]
            u, v = b - a, c - a
            cot.append(np.dot(u, v) / abs(cross2(u, v)))
        for i in range(3):
            for j in range(3):
                if i != j:
                    k = 3 - i - j
                    assert np.isclose(B[i, j], -0.5 * 1.7 * cot[k], atol=1e-12)


def test_R_rows_are_lambda_at_midpoints_and_C_rows():
    rng = np.random.default_rng(1)
    P = np.array([[0.1, 0.2], [1.3, 0.4], [0.5, 1.1]])
    geo = _geo(P)
    coef = geo["coef"][0]
    for k in range(3):
        m = geo["mid"][0, k]
        lam = coef[0] + coef[1] * m[0] + coef[2] * m[1]
        assert np.allclose(lam, O.R[k], atol=1e-15)
        # |E_k| is the length of the edge opposite P_k
        a, b = P[(k + 1) % 3], P[(k + 2) % 3]
        assert np.isclose(geo["elen"][0, k], np.linalg.norm(b - a))
    sigma = np.array([[1, -1, 1]])
    C = O.local_C(geo, sigma)[0]
    assert np.allclose(C.sum(axis=1), sigma[0] * geo["elen"][0])
    # C_T[l, j] = int_{E_l} psi_l lambda_j: exact by 2-point Gauss on the edge
    g = np.array([0.5 - 0.5 / np.sqrt(3), 0.5 + 0.5 / np.sqrt(3)])
    for k in range(3):
        a, b = P[(k + 1) % 3], P[(k + 2) % 3]
        pts = a[None] + g[:, None] * (b - a)[None]
        lam = coef[0][None] + pts[:, :1] * coef[1][None] + pts[:, 1:] * coef[2][None]
        integ = 0.5 * np.linalg.norm(b - a) * lam.sum(axis=0)
        assert np.allclose(C[k], sigma[0, k] * integ, atol=1e-14)


@pytest.mark.parametrize("delta", [0.0, 1.3])
def test_condensed_block_closed_form(delta):
    # R^{-T} (a B + delta M0) R^{-1} = 4 a B + delta |T|/3 I (rows of B sum to 0,
    # and (J - 2I)(I + J)(J - 2I) = 4 I)
    P = np.array([[0.0, 0.0], [1.2, 0.1], [0.3, 0.9]])
    xy = P
    tri = np.array([[0, 1, 2]])

    class Pb:
        p = (0.0, 0.0)
        A = None
    Pb.delta = delta
    st = dict(xy=xy, tri=tri, geo=O.element_geometry(xy, tri))
    st["loc"] = O.local_matrices(st["geo"], aT=0.8, delta=delta)
    cl = O.condensed_local(st)
    ref = 4 * st["loc"]["B"][0] + delta * st["geo"]["area"][0] / 3 * np.eye(3)
    assert np.allclose(cl["KCR"][0], ref, atol=1e-13)
    assert np.allclose(cl["Rinv"], np.ones((3, 3)) - 2 * np.eye(3))
    # CR basis: int grad(1-2 lambda_i).grad(1-2 lambda_j) = 4 |T| grad lambda_i . grad lambda_j
    G = st["geo"]["grads"][0]
    assert np.allclose(cl["KCR"][0] - delta * st["geo"]["area"][0] / 3 * np.eye(3),
                       0.8 * 4 * st["geo"]["area"][0] * G @ G.T, atol=1e-13)
