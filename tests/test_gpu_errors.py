"""Error report on the GPU (L2, broken H1, multiplier mesh norm) against the
oracle's quadrature of the same solution, and against closed forms."""
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


def _points(gm, nq):
    from paper_2401_15557_gb300 import phfem as P
    In = gm.info
    txy = torch.empty((In["nT"], nq * nq, 2), dtype=torch.float64, device="cuda")
    exy = torch.empty((max(In["nL"], 1), nq, 2), dtype=torch.float64, device="cuda")
    nu = torch.empty((max(In["nL"], 1), 2), dtype=torch.float64, device="cuda")
    P.phfem_error_points(gm.h, nq, txy, exy, nu)
    torch.cuda.synchronize()
    return txy.cpu().numpy(), exy.cpu().numpy()[:In["nL"]], nu.cpu().numpy()[:In["nL"]]


def _report(gm, nq, U, Lam, u, grad):
    """Exact data evaluated at the library's points, then the GPU norms."""
    from phfem_gpu import dev
    from paper_2401_15557_gb300 import phfem as P
    txy, exy, nu = _points(gm, nq)
    uq = u(txy[..., 0], txy[..., 1])
    gx, gy = grad(txy[..., 0], txy[..., 1])
    ex, ey = grad(exy[..., 0], exy[..., 1])
    kq = ex * nu[:, None, 0] + ey * nu[:, None, 1]
    return P.phfem_error_norms(gm.h, nq, U=dev(U, torch.float64), u_q=dev(uq, torch.float64),
                               grad_q=dev(np.stack([gx, gy], axis=-1), torch.float64),
                               Lambda=dev(Lam, torch.float64) if Lam is not None else None,
                               kappa_q=dev(kq, torch.float64) if Lam is not None else None)


def test_error_report_matches_oracle_on_the_32_square(ctx):
    """Config 0: -Lap u = f, u = sin(pi x) e^y, 32 x 32 squares, mixed boundary."""
    from phfem_gpu import GpuMesh, solve
    mesh = I.square_mesh(32)
    pb = I.problem_sine_exp()
    gm = GpuMesh(mesh, ctx)
    out = solve(gm, pb, rtol=1e-12)
    st = O.setup(mesh, pb)
    ref = O.errors(st, out["U"], pb.u, pb.grad, nq=6)
    ref_m = O.m_norm_error(st, out["Lambda"], pb.grad, nq=6)
    got = _report(gm, 6, out["U"], out["Lambda"], pb.u, pb.grad)
    for k in ("L2", "H1semi", "H1"):
        assert abs(got[k] - ref[k]) <= 1e-12 * ref[k], (k, got[k], ref[k])
    assert abs(got["M"] - ref_m) <= 1e-12 * ref_m
    # the paper's lowest-order rates: L2 ~ h^2, energy ~ h (h = 1/32)
    assert got["L2"] < 2e-3 and got["H1semi"] < 2e-1
    gm.close()


def test_points_are_the_oracle_rule(ctx):
    """Triangle points are the barycentric combinations of the Duffy rule."""
    from phfem_gpu import GpuMesh
    mesh = I.lshape_mesh(n=4, seed=I.seed_for(1, 9))
    gm = GpuMesh(mesh, ctx)
    nq = 4
    txy, exy, nu = _points(gm, nq)
    xi, _ = np.polynomial.legendre.leggauss(nq)
    xi = 0.5 * (xi + 1.0)
    s = np.repeat(xi, nq)
    t = np.tile(xi, nq) * (1.0 - s)
    P = mesh.xy[mesh.tri]                                       # (nT, 3, 2)
    X = (1 - s - t)[None, :, None] * P[:, None, 0] + s[None, :, None] * P[:, None, 1] + t[None, :, None] * P[:, None, 2]
    assert np.max(np.abs(txy - X)) <= 1e-15
    st = O.setup(mesh)
    Redges = st["bsets"]["Redges"]
    ed2el = st["topo"]["ed2el"]
    a, b = mesh.xy[ed2el[Redges, 0]], mesh.xy[ed2el[Redges, 1]]
    assert np.max(np.abs(exy - (a[:, None, :] + xi[None, :, None] * (b - a)[:, None, :]))) <= 1e-15
    _, _, nrm = O.edge_midpoints(mesh.xy, ed2el)
    assert np.max(np.abs(nu - nrm[Redges])) <= 1e-15
    gm.close()


@pytest.mark.parametrize("nq", [1, 2, 3, 5, 8, 16])
def test_closed_forms(ctx, nq):
    """U = 0 against u = x^a y^b: L2^2 = int x^2a y^2b over the unit square,
    exact once the collapsed rule has the degree; a linear u reproduced by U
    gives zero errors."""
    from phfem_gpu import GpuMesh
    gm = GpuMesh(I.square_mesh(5), ctx)
    nT = gm.info["nT"]
    zero = np.zeros(3 * nT)
    a, b = (1, 1) if nq >= 3 else (0, 0)
    u = lambda x, y: x ** a * y ** b
    grad = lambda x, y: (a * x ** max(a - 1, 0) * y ** b, b * x ** a * y ** max(b - 1, 0))
    got = _report(gm, nq, zero, None, u, grad)
    exact_l2 = 1.0 / ((2 * a + 1) * (2 * b + 1))
    assert abs(got["L2"] ** 2 - exact_l2) <= 1e-14
    exact_h1 = (a * a / ((2 * a - 1) * (2 * b + 1)) if a else 0.0) + (b * b / ((2 * a + 1) * (2 * b - 1)) if b else 0.0)
    assert abs(got["H1semi"] ** 2 - exact_h1) <= 1e-14
    assert got["M"] == 0.0
    lin = lambda x, y: 0.3 + 0.7 * x - 0.4 * y
    lgrad = lambda x, y: (0.7 + 0 * x, -0.4 + 0 * y)
    Uv = lin(gm.mesh.xy[gm.mesh.tri][..., 0], gm.mesh.xy[gm.mesh.tri][..., 1]).reshape(-1)
    z = _report(gm, nq, Uv, None, lin, lgrad)
    assert z["L2"] <= 1e-15 and z["H1semi"] <= 1e-14
    gm.close()


def test_rejections(ctx):
    from phfem_gpu import GpuMesh, dev
    from paper_2401_15557_gb300 import phfem as P
    gm = GpuMesh(I.square_mesh(2), ctx)
    for nq in (0, 17):
        with pytest.raises(P.PhfemError) as ei:
            P.phfem_error_norms(gm.h, nq)
        assert ei.value.status == P.PHFEM_EINVAL
    U = dev(np.zeros(3 * gm.info["nT"]), torch.float64)
    with pytest.raises(P.PhfemError) as ei:
        P.phfem_error_norms(gm.h, 3, U=U)  # U without u_q and grad_q
    assert ei.value.status == P.PHFEM_EINVAL
    gm.close()
