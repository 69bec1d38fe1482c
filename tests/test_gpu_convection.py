"""Convection and a constant tensor A on the GPU: BiCGStab solves against the
oracle's saddle-point solve, the paper's Example 1 error table reproduced
from the GPU solution and the GPU error report, the patch test with a full
SPD tensor, Crank-Nicolson with convection (Example 2's data), and the
cases the library rejects."""
import numpy as np
import pytest
import torch

from conftest import read_golden_rows
from oracle import phfem_oracle as O
from paper_2401_15557_gb300 import inputs as I

pytestmark = pytest.mark.gpu

A_SPD = np.array([[1.4, 0.3], [0.3, 0.8]])


@pytest.fixture(scope="module")
def ctx():
    from paper_2401_15557_gb300 import phfem as P
    c = P.phfem_ctx_create()
    yield c
    P.phfem_ctx_destroy(c)


def _solve(gm, pb, precision, A=None, rtol=1e-10):
    from phfem_gpu import dev
    from paper_2401_15557_gb300 import phfem as P
    fm, bc = gm.edge_data(pb.f, pb.g, pb.uD)
    In = gm.info
    sysh = P.phfem_assemble(gm.h, fm, bc, delta=pb.delta, precision=precision, A=A,
                            p=pb.p if any(pb.p) else None)
    U = torch.empty(3 * In["nT"], dtype=torch.float64, device="cuda")
    L = torch.empty(max(In["nL"], 1), dtype=torch.float64, device="cuda")
    st = P.phfem_solve(sysh, P.solve_opts(rtol=rtol), U=U, Lambda=L)
    torch.cuda.synchronize()
    P.phfem_sys_destroy(sysh)
    return st, U, L[:In["nL"]]


@pytest.mark.parametrize("level", [1, 2, 3])
@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32ir"])
def test_example1_matches_saddle_solve(ctx, level, precision):
    from phfem_gpu import GpuMesh
    mesh = I.criss_cross(level)
    pb = I.problem_paper_example1()
    ref = O.solve_saddle(mesh, pb)
    gm = GpuMesh(mesh, ctx)
    st, U, L = _solve(gm, pb, precision)
    assert st["converged"] >= 1 and st["rel_residual"] <= 1e-10, st
    assert np.max(np.abs(U.cpu().numpy() - ref["U"])) <= 1e-8 * np.max(np.abs(ref["U"]))
    assert np.max(np.abs(L.cpu().numpy() - ref["Lambda"])) <= 1e-7 * np.max(np.abs(ref["Lambda"]))
    gm.close()


def test_example1_error_table_on_the_gpu(ctx):
    """The printed H1 errors (to their 4 decimals) and L2 errors of Example 1,
    from the GPU solution and the GPU error report."""
    from phfem_gpu import GpuMesh, dev
    from paper_2401_15557_gb300 import phfem as P
    rows = read_golden_rows("paper_example1_errors.txt")
    pb = I.problem_paper_example1()
    for lev, h1, l2, _m in rows[:4]:
        gm = GpuMesh(I.criss_cross(int(lev)), ctx)
        st, U, L = _solve(gm, pb, P.PHFEM_FP64, rtol=1e-12)
        nq = 6
        X = torch.empty((gm.info["nT"], nq * nq, 2), dtype=torch.float64, device="cuda")
        P.phfem_error_points(gm.h, nq, tri_xy=X)
        Xh = X.cpu().numpy()
        gx, gy = pb.grad(Xh[..., 0], Xh[..., 1])
        e = P.phfem_error_norms(gm.h, nq, U=U, u_q=dev(pb.u(Xh[..., 0], Xh[..., 1]), torch.float64),
                                grad_q=dev(np.stack([gx, gy], axis=-1), torch.float64))
        assert round(e["H1semi"], 4) == pytest.approx(h1, abs=1e-12), (lev, e)
        assert abs(e["L2"] - l2) <= 0.006 * l2 + 5e-5 * (l2 >= 1e-3), (lev, e)
        gm.close()


@pytest.mark.parametrize("mk", ["lshape", "square"])
def test_patch_test_with_a_full_tensor(ctx, mk):
    """A linear solution with a full SPD tensor A is reproduced exactly, and
    the multipliers are its exact normal flux (A grad u).nu."""
    from phfem_gpu import GpuMesh
    mesh = {"lshape": lambda: I.lshape_mesh(n=4, seed=I.seed_for(1, 3)), "square": lambda: I.square_mesh(6)}[mk]()
    c0, cx, cy = 0.3, 0.7, -0.4
    flux = A_SPD @ np.array([cx, cy])
    pb = I.Problem(f=lambda x, y: 0.7 * (c0 + cx * x + cy * y), g=lambda x, y, nx, ny: flux[0] * nx + flux[1] * ny,
                   uD=lambda x, y: c0 + cx * x + cy * y, u=lambda x, y: c0 + cx * x + cy * y,
                   grad=lambda x, y: (cx + 0 * x, cy + 0 * y), delta=0.7, A=A_SPD)
    gm = GpuMesh(mesh, ctx)
    st, U, L = _solve(gm, pb, 0, A=A_SPD, rtol=1e-13)
    st_o = O.setup(mesh, pb)
    P_ = st_o["geo"]["P"]
    assert np.max(np.abs(U.cpu().numpy() - pb.u(P_[..., 0], P_[..., 1]).reshape(-1))) < 1e-10
    kappa = O.exact_flux(st_o, pb.grad, A=A_SPD)
    assert np.max(np.abs(L.cpu().numpy() - kappa)) < 1e-9
    # and a non-polynomial problem against the oracle's saddle solve with the same A
    pb2 = I.problem_sine_exp()
    pb2.delta, pb2.A = 0.4, A_SPD
    ref = O.solve_saddle(mesh, pb2)
    st2, U2, L2 = _solve(gm, pb2, 1, A=A_SPD)
    assert np.max(np.abs(U2.cpu().numpy() - ref["U"])) <= 1e-7 * np.max(np.abs(ref["U"]))
    assert np.max(np.abs(L2.cpu().numpy() - ref["Lambda"])) <= 1e-6 * np.max(np.abs(ref["Lambda"]))
    gm.close()


def test_crank_nicolson_with_convection(ctx):
    """Example 2's data (convection p = (1, 1), reaction 1): host-driven steps
    against the oracle's Crank-Nicolson; the graph-captured step refuses."""
    from phfem_gpu import GpuMesh, dev
    from paper_2401_15557_gb300 import phfem as P
    mesh = I.criss_cross(3)
    pb = I.problem_paper_example2()
    gm = GpuMesh(mesh, ctx)
    tb = gm.tables
    s = lambda x, y: (x - x * x) * (y - y * y)
    f0 = lambda x, y: s(x, y)
    f1 = lambda x, y: (2 * (y - y * y) + 2 * (x - x * x) + (1 - 2 * x) * (y - y * y)
                       + (x - x * x) * (1 - 2 * y) + s(x, y))
    g1 = lambda x, y, nx, ny: (1 - x - x * x) * (y - y * y) * nx + (x - x * x) * (1 - y - y * y) * ny
    zero_g = lambda x, y, nx, ny: 0 * x
    zero = lambda x, y: 0 * x
    fa, ba = I.edge_data(mesh.xy, tb["ed2el"], tb["eclass"], f0, zero_g, zero)
    fb, bb = I.edge_data(mesh.xy, tb["ed2el"], tb["eclass"], f1, g1, zero)
    k, n = 1.0 / 16, 8
    t = k * np.arange(n + 1)
    phi = np.stack([np.ones_like(t), t])
    sysh = P.phfem_assemble(gm.h, None, None, delta=pb.delta, dt=k, precision=P.PHFEM_FP64, p=pb.p)
    F = dev(np.stack([fa, fb]), torch.float64)
    G = dev(np.stack([ba, bb]), torch.float64)
    cn = P.phfem_cn_create(sysh, F, G, phi, dev(np.zeros(gm.info["nE"]), torch.float64))
    with pytest.raises(P.PhfemError) as ei:
        P.phfem_cn_step_graph(cn, 1, P.solve_opts(rtol=1e-12))
    assert ei.value.status == P.PHFEM_EINVAL
    P.phfem_cn_step(cn, n, P.solve_opts(rtol=1e-12))
    U = torch.empty(3 * mesh.nT, dtype=torch.float64, device="cuda")
    P.phfem_cn_read(cn, U=U)
    ref = O.cn_solve(mesh, pb, k, n)
    assert np.max(np.abs(U.cpu().numpy() - ref["U"])) <= 1e-9 * np.max(np.abs(ref["U"]))
    P.phfem_cn_destroy(cn)
    P.phfem_sys_destroy(sysh)
    gm.close()


def test_rejections(ctx):
    from phfem_gpu import GpuMesh
    from paper_2401_15557_gb300 import phfem as P
    gm = GpuMesh(I.square_mesh(4), ctx)
    fm, bc = gm.edge_data(lambda x, y: 1.0 + 0 * x, lambda x, y, nx, ny: 0 * x, lambda x, y: 0 * x)
    cases = [dict(delta=1.0, p=(1.0, 0.5), form=P.PHFEM_FORM_FLUX),       # convection needs the trace form
             dict(delta=1.0, A=((1.0, 2.0), (2.0, 1.0))),                # indefinite tensor
             dict(delta=1.0, A=((-1.0, 0.0), (0.0, 1.0)))]
    for kw in cases:
        with pytest.raises(P.PhfemError) as ei:
            P.phfem_assemble(gm.h, fm, bc, **kw)
        assert ei.value.status == P.PHFEM_EINVAL
    H = P.phfem_mesh_refine(gm.h)
    info = P.phfem_mesh_info_get(H)
    ff = torch.ones(info["nE"], dtype=torch.float64, device="cuda")
    s = P.phfem_assemble(H, ff, torch.zeros_like(ff), delta=1.0, p=(1.0, 1.0))
    with pytest.raises(P.PhfemError) as ei:
        P.phfem_mg_create(s, [gm.h, H])
    assert ei.value.status == P.PHFEM_EINVAL
    P.phfem_sys_destroy(s)
    P.phfem_mesh_destroy(H)
    gm.close()
