"""Crank-Nicolson stepping of the CUDA path against the oracle's stepping of
the paper's saddle-point system (Section 4)."""
import numpy as np
import pytest
import torch

from oracle import phfem_oracle as O
from paper_2401_15557_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2401_15557_gb300 import phfem as P
    c = P.phfem_ctx_create()
    yield c
    P.phfem_ctx_destroy(c)


def _run_gpu(ctx, mesh, terms, phi_fn, dt, nsteps, u0, delta, aT=None, precision=0, rtol=1e-13, Lambda0=None,
             graph=False):
    """terms: list of (f_q, g_q, uD_q) spatial functions; phi_fn(t) -> [Q]."""
    from paper_2401_15557_gb300 import phfem as P
    from phfem_gpu import GpuMesh, dev
    gm = GpuMesh(mesh, ctx)
    fs, bcs = [], []
    for fq, gq, uq in terms:
        fm, bc = gm.edge_data(fq, gq, uq)
        fs.append(fm)
        bcs.append(bc)
    F = torch.stack(fs).contiguous()
    B = torch.stack(bcs).contiguous()
    phi = np.array([phi_fn(n * dt) for n in range(nsteps + 1)]).T.copy()
    sysh = P.phfem_assemble(gm.h, None, None, a_T=None if aT is None else dev(aT, torch.float64), delta=delta,
                            dt=dt, precision=precision)
    w0, _ = gm.edge_data(u0)
    cn = P.phfem_cn_create(sysh, F, B, phi, w0, Lambda0=None if Lambda0 is None else dev(Lambda0, torch.float64))
    if graph:  # two launches of the captured step sequence
        st = P.phfem_cn_step_graph(cn, nsteps // 2, P.solve_opts(rtol=rtol))
        st2 = P.phfem_cn_step_graph(cn, nsteps - nsteps // 2, P.solve_opts(rtol=rtol))
        st["iterations"] += st2["iterations"]
    else:
        st = P.phfem_cn_step(cn, nsteps, P.solve_opts(rtol=rtol))
    I_ = gm.info
    U = torch.empty(3 * I_["nT"], dtype=torch.float64, device="cuda")
    Ln = torch.empty(I_["nL"], dtype=torch.float64, device="cuda")
    Lh = torch.empty(I_["nL"], dtype=torch.float64, device="cuda")
    step = P.phfem_cn_read(cn, U=U, Lambda_n=Ln, Lambda_half=Lh)
    P.phfem_cn_destroy(cn)
    P.phfem_sys_destroy(sysh)
    gm.close()
    return dict(U=U.cpu().numpy(), Lambda=Ln.cpu().numpy(), Lambda_half=Lh.cpu().numpy(), step=step, stats=st)


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32ir"])
def test_heat_sine_matches_oracle(ctx, precision):
    pi = np.pi
    s = lambda x, y: np.sin(pi * x) * np.sin(pi * y)
    pb = I.problem_heat_sine()
    mesh = I.square_mesh(10)
    dt, n = 1.0 / 10, 10
    terms = [(lambda x, y: (2 * pi * pi - 1.0) * s(x, y),
              lambda x, y, nx, ny: pi * (np.cos(pi * x) * np.sin(pi * y) * nx + np.sin(pi * x) * np.cos(pi * y) * ny),
              lambda x, y: 0 * x)]
    out = _run_gpu(ctx, mesh, terms, lambda t: [np.exp(-t)], dt, n, s, 0.0, precision=precision,
                   rtol=1e-13 if precision == 0 else 1e-10)
    ref = O.cn_solve(mesh, pb, dt, n)
    assert out["step"] == n
    tol = 1e-10 if precision == 0 else 1e-7
    assert np.max(np.abs(out["U"] - ref["U"])) <= tol * np.max(np.abs(ref["U"]))
    assert np.max(np.abs(out["Lambda_half"] - ref["Lambda_half"])) <= 10 * tol * np.max(np.abs(ref["Lambda_half"]))
    assert np.max(np.abs(out["Lambda"] - ref["Lambda"])) <= 100 * tol * np.max(np.abs(ref["Lambda"]))


def test_two_term_source_reaction_variable_coefficient(ctx):
    """u = t s(x) with s = (x - x^2)(y - y^2) + 0.2 x: f = s + t (L s) has two
    separable terms; Dirichlet on x = 0, 1, Neumann elsewhere, delta > 0,
    variable a_T (the oracle gets the same a_T)."""
    mesh = I.lshape_mesh(n=4, seed=I.seed_for(1, 51))
    delta = 0.7
    aT = I.element_mean_at_midpoints(mesh.xy, mesh.tri, I.coeff_lshape)
    s = lambda x, y: (x - x * x) * (y - y * y) + 0.2 * x
    # L s = -div(a grad s) + delta s evaluated with the element coefficient is
    # not needed: any smooth f is a valid source; use f1 = sin(x) cos(y)
    f1 = lambda x, y: np.sin(x) * np.cos(y)
    g1 = lambda x, y, nx, ny: 0.3 * nx - 0.1 * ny
    uD1 = lambda x, y: 0.2 * x + 0.1
    terms = [(s, lambda x, y, nx, ny: 0 * x, lambda x, y: 0 * x), (f1, g1, uD1)]
    phi = lambda t: [1.0, t]
    pb = I.Problem(f=lambda x, y, t: s(x, y) + t * f1(x, y), g=lambda x, y, nx, ny, t: t * g1(x, y, nx, ny),
                   uD=lambda x, y, t: t * uD1(x, y), delta=delta, u0=lambda x, y: 0 * x)
    dt, n = 0.05, 8
    L0 = np.linspace(-1, 1, O.setup(mesh)["bsets"]["Redges"].size)
    out = _run_gpu(ctx, mesh, terms, phi, dt, n, lambda x, y: 0 * x, delta, aT=aT, Lambda0=L0)
    ref = O.cn_solve(mesh, pb, dt, n, aT=aT, Lambda0=L0)
    assert np.max(np.abs(out["U"] - ref["U"])) <= 1e-10 * np.max(np.abs(ref["U"]))
    assert np.max(np.abs(out["Lambda_half"] - ref["Lambda_half"])) <= 1e-8 * np.max(np.abs(ref["Lambda_half"]))
    assert np.max(np.abs(out["Lambda"] - ref["Lambda"])) <= 1e-7 * np.max(np.abs(ref["Lambda"]))


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32ir"])
def test_graph_steps_equal_host_steps(ctx, precision):
    """Steps replayed from the captured graph (device-controlled solve loop)
    give bitwise the results of the host-driven steps."""
    pi = np.pi
    s = lambda x, y: np.sin(pi * x) * np.sin(pi * y)
    mesh = I.lshape_mesh(n=6, seed=I.seed_for(1, 81), levels=1)
    aT = I.element_mean_at_midpoints(mesh.xy, mesh.tri, I.coeff_lshape)
    terms = [(lambda x, y: (2 * pi * pi - 1.0) * s(x, y),
              lambda x, y, nx, ny: pi * (np.cos(pi * x) * np.sin(pi * y) * nx + np.sin(pi * x) * np.cos(pi * y) * ny),
              lambda x, y: 0 * x)]
    kw = dict(aT=aT, precision=precision, rtol=1e-10)
    a = _run_gpu(ctx, mesh, terms, lambda t: [np.exp(-t)], 1.0 / 24, 12, s, 0.3, **kw)
    b = _run_gpu(ctx, mesh, terms, lambda t: [np.exp(-t)], 1.0 / 24, 12, s, 0.3, graph=True, **kw)
    assert b["step"] == 12
    assert np.array_equal(a["U"], b["U"]) and np.array_equal(a["Lambda"], b["Lambda"])
    assert np.array_equal(a["Lambda_half"], b["Lambda_half"])
    assert a["stats"]["iterations"] == b["stats"]["iterations"]


def _problem_nonseparable():
    """u = sin(pi y) exp(-x t), which no finite sum of f_q(x) phi_q(t) gives:
    u_t = -x u, -Lap u = (pi^2 - t^2) u, so f = (pi^2 - t^2 - x) u; u_D on x = 0
    (sin(pi y)) and x = 1 (e^-t sin(pi y)) varies in time; g = grad u . n on
    y = 0, 1."""
    pi = np.pi
    u = lambda x, y, t: np.sin(pi * y) * np.exp(-x * t)
    grad = lambda x, y, t: (-t * u(x, y, t), pi * np.cos(pi * y) * np.exp(-x * t))
    f = lambda x, y, t: (pi * pi - t * t - x) * u(x, y, t)

    def g(x, y, nx, ny, t):
        gx, gy = grad(x, y, t)
        return gx * nx + gy * ny

    return I.Problem(f=f, g=g, uD=u, u=u, grad=grad, delta=0.0, u0=lambda x, y: u(x, y, 0.0))


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32ir"])
def test_general_source_matches_oracle(ctx, precision):
    """Per-step data (phfem_cn_create_data / phfem_cn_step_data) for a source,
    flux and Dirichlet datum that are not separable in x and t, against the
    oracle's stepping of the saddle-point system with the same functions."""
    from paper_2401_15557_gb300 import phfem as P
    from phfem_gpu import GpuMesh
    pb = _problem_nonseparable()
    mesh = I.square_mesh(8)
    dt, nsteps = 0.05, 6
    gm = GpuMesh(mesh, ctx)
    data = lambda t: gm.edge_data(lambda x, y: pb.f(x, y, t), lambda x, y, nx, ny: pb.g(x, y, nx, ny, t),
                                  lambda x, y: pb.uD(x, y, t))
    f0, bc0 = data(0.0)
    w0, _ = gm.edge_data(pb.u0)
    sysh = P.phfem_assemble(gm.h, None, None, delta=0.0, dt=dt, precision=precision)
    cn = P.phfem_cn_create_data(sysh, f0, bc0, w0, nsteps)
    with pytest.raises(P.PhfemError):
        P.phfem_cn_step(cn, 1, P.solve_opts(rtol=1e-13))
    for n in range(1, nsteps + 1):
        fn, bcn = data(n * dt)
        st = P.phfem_cn_step_data(cn, fn, bcn, P.solve_opts(rtol=1e-12))
        assert st["converged"] == 1, (n, st)
    with pytest.raises(P.PhfemError):  # max_steps reached
        P.phfem_cn_step_data(cn, fn, bcn, P.solve_opts(rtol=1e-12))
    I_ = gm.info
    U = torch.empty(3 * I_["nT"], dtype=torch.float64, device="cuda")
    Lh = torch.empty(I_["nL"], dtype=torch.float64, device="cuda")
    P.phfem_cn_read(cn, U=U, Lambda_half=Lh)
    ref = O.cn_solve(mesh, pb, dt, nsteps)
    Ug, Lg = U.cpu().numpy(), Lh.cpu().numpy()
    assert np.max(np.abs(Ug - ref["U"])) <= 1e-9 * np.max(np.abs(ref["U"]))
    assert np.max(np.abs(Lg - ref["Lambda_half"])) <= 1e-8 * np.max(np.abs(ref["Lambda_half"]))
    P.phfem_cn_destroy(cn)
    P.phfem_sys_destroy(sysh)
    gm.close()
