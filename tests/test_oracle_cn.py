"""Pins of the oracle's Crank-Nicolson stepping (Section 4)."""
import numpy as np
import pytest

from conftest import read_golden_rows
from oracle import phfem_oracle as O
from paper_2401_15557_gb300 import inputs as I


def test_example2_orders_against_printed_orders():
    """Convergence orders with h = k (the printed errors themselves include a
    contribution of the paper's unprinted main program; with a solution linear in t the
    scheme as printed has no time error, so only the orders are compared)."""
    rows = read_golden_rows("paper_example2_orders.txt")
    pb = I.problem_paper_example2()
    errs, merr = [], []
    for lev in range(1, 6):
        mesh = I.criss_cross(lev)
        k = 2.0 ** -lev
        r = O.cn_solve(mesh, pb, k, 2 ** lev)
        errs.append(O.errors(r["st"], r["U"], pb.u, pb.grad, t=1.0))
        merr.append(O.m_norm_error(r["st"], r["Lambda_half"], pb.grad, t=1.0 - k / 2))
    for i, (lev, hk, o_h1, o_l2, o_m) in enumerate(rows):
        j = int(lev) - 1
        oh1 = np.log2(errs[j - 1]["H1semi"] / errs[j]["H1semi"])
        ol2 = np.log2(errs[j - 1]["L2"] / errs[j]["L2"])
        assert abs(oh1 - o_h1) < 0.2, (lev, oh1, o_h1)
        assert abs(ol2 - o_l2) < 0.2, (lev, ol2, o_l2)
    om = np.log2(np.array(merr[1:-1]) / np.array(merr[2:]))
    assert np.all(np.abs(om - 1.0) < 0.2), om


def test_second_order_in_time():
    """u = sin(3t)^2 sin(pi x) sin(pi y): u0 = 0 and f(0) = 0, so no stiff
    component of the initial state survives (Crank-Nicolson is not L-stable);
    the error against a fine-step reference at fixed h falls by 4 per halving
    of k (the remark after the scheme in Section 4)."""
    pi = np.pi
    s = lambda x, y: np.sin(pi * x) * np.sin(pi * y)
    phi = lambda t: np.sin(3 * t) ** 2
    dphi = lambda t: 6 * np.sin(3 * t) * np.cos(3 * t)
    pb = I.Problem(f=lambda x, y, t: (dphi(t) + 2 * pi * pi * phi(t)) * s(x, y),
                   g=lambda x, y, nx, ny, t: phi(t) * pi * (np.cos(pi * x) * np.sin(pi * y) * nx
                                                            + np.sin(pi * x) * np.cos(pi * y) * ny),
                   uD=lambda x, y, t: 0 * x, delta=0.0, u0=lambda x, y: 0 * x)
    mesh = I.square_mesh(6)
    ref = O.cn_solve(mesh, pb, 1.0 / 1024, 1024)["U"]
    err = [np.linalg.norm(O.cn_solve(mesh, pb, 1.0 / n, n)["U"] - ref) for n in (8, 16, 32, 64)]
    ratios = np.array(err[:-1]) / np.array(err[1:])
    assert np.all((ratios > 3.8) & (ratios < 4.4)), ratios


def test_steady_state_is_elliptic_solution():
    base = I.problem_sine_exp()
    pb = I.Problem(f=lambda x, y, t: base.f(x, y), g=lambda x, y, nx, ny, t: base.g(x, y, nx, ny),
                   uD=lambda x, y, t: base.uD(x, y), u=None, grad=None, delta=0.4,
                   u0=lambda x, y: 0 * x)
    ell = I.Problem(f=lambda x, y: base.f(x, y) + 0 * x, g=base.g, uD=base.uD, delta=0.4)
    mesh = I.square_mesh(4)
    r = O.cn_solve(mesh, pb, 0.05, 800)
    re = O.solve_saddle(mesh, ell)
    assert np.max(np.abs(r["U"] - re["U"])) < 1e-10
    assert np.max(np.abs(r["Lambda_half"] - re["Lambda"])) < 1e-8


def test_constraint_holds_at_every_step_and_lambda0_does_not_change_u():
    pb = I.problem_heat_sine()
    mesh = I.square_mesh(5)
    k = 0.1
    r = O.cn_solve(mesh, pb, k, 6, keep_history=True)
    st = r["st"]
    glob = O.global_blocks(st["tri"], st["topo"], st["bsets"], st["geo"], st["loc"])
    N = 3 * mesh.nT
    for n, W in enumerate(r["history"], start=1):
        lv = O.load_vectors(st["xy"], st["tri"], st["topo"], st["bsets"], st["geo"],
                            pb.f, pb.g, pb.uD, n * k)
        # C U^n = -b_D^n: midpoint continuity and Dirichlet midpoint values at t_n
        assert np.max(np.abs(glob["C"] @ W[:N] + lv["bD"])) < 1e-12
    L = st["bsets"]["Redges"].size
    r2 = O.cn_solve(mesh, pb, k, 6, Lambda0=np.linspace(-3, 3, L))
    assert np.max(np.abs(r2["U"] - r["U"])) < 1e-12
    assert np.max(np.abs(r2["Lambda_half"] - r["Lambda_half"])) < 1e-10
