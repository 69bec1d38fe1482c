"""The multiplier ("flux") Schur form on the GPU: its multipliers and the
recovered element values against the oracle's saddle-point solve, its residual
against the oracle's C K^-1 C' system, and the cases it rejects."""
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


def _solve_flux(gm, pb, aT, precision, rtol=1e-10):
    from phfem_gpu import dev
    from paper_2401_15557_gb300 import phfem as P
    fm, bc = gm.edge_data(pb.f, pb.g, pb.uD)
    In = gm.info
    sysh = P.phfem_assemble(gm.h, fm, bc, a_T=None if aT is None else dev(aT, torch.float64), delta=pb.delta,
                            precision=precision, form=P.PHFEM_FORM_FLUX)
    w = torch.empty(In["nE"], dtype=torch.float64, device="cuda")
    U = torch.empty(3 * In["nT"], dtype=torch.float64, device="cuda")
    Lam = torch.empty(max(In["nL"], 1), dtype=torch.float64, device="cuda")
    st = P.phfem_solve(sysh, P.solve_opts(rtol=rtol), w=w, U=U, Lambda=Lam)
    torch.cuda.synchronize()
    out = dict(w=w.cpu().numpy(), U=U.cpu().numpy(), Lambda=Lam.cpu().numpy()[:In["nL"]], stats=st)
    P.phfem_sys_destroy(sysh)
    return out


CASES = [
    ("two", lambda: I.square_mesh(1), False),
    ("crisscross3", lambda: I.criss_cross(3), True),
    ("square40", lambda: I.square_mesh(40), False),
    ("lshape8r1", lambda: I.lshape_mesh(n=8, seed=I.seed_for(1, 31), levels=1), True),
    ("alldirichlet", lambda: I.square_mesh(9, dirichlet_sides=("left", "right", "top", "bottom")), True),
    ("allneumann", lambda: I.square_mesh(9, dirichlet_sides=()), False),
]


@pytest.mark.parametrize("name,mk,var", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32ir"])
def test_flux_form_matches_saddle_solve(ctx, name, mk, var, precision):
    from phfem_gpu import GpuMesh
    mesh = mk()
    pb = I.problem_sine_exp()
    pb.delta = 0.6
    aT = I.element_mean_at_midpoints(mesh.xy, mesh.tri, I.coeff_lshape) if var else None
    ref = O.solve_saddle(mesh, pb, aT=aT)
    fs = O.flux_system(mesh, pb, aT=aT)
    gm = GpuMesh(mesh, ctx)
    out = _solve_flux(gm, pb, aT, precision)
    st = out["stats"]
    assert st["converged"] in (1, 2) and st["rel_residual"] <= max(1e-10, 2 * st["fp64_floor"]), st
    if fs["rhs"].size:
        assert O.relative_residual(fs["S"], fs["rhs"], out["Lambda"]) <= 1.2e-10
    lam_id = gm.tables["lam_id"]
    # w holds the multiplier of every edge: Lambda on interior and Dirichlet
    # edges, zero on Neumann edges (bit-exact placement)
    assert np.array_equal(out["w"][lam_id >= 0], out["Lambda"][lam_id[lam_id >= 0]])
    assert np.all(out["w"][lam_id < 0] == 0.0)
    scale_l = max(1.0, np.max(np.abs(ref["Lambda"]))) if ref["Lambda"].size else 1.0
    assert np.max(np.abs(out["Lambda"] - ref["Lambda"]), initial=0.0) <= 1e-7 * scale_l
    assert np.max(np.abs(out["U"] - ref["U"])) <= 1e-7 * max(1.0, np.max(np.abs(ref["U"])))
    gm.close()


def test_flux_and_trace_forms_agree(ctx):
    """Both condensations of the same saddle system give the same solution."""
    from phfem_gpu import GpuMesh, solve
    mesh = I.lshape_mesh(n=10, seed=I.seed_for(1, 77), levels=1)
    pb = I.problem_sine_exp()
    pb.delta = 1.3
    aT = I.element_mean_at_midpoints(mesh.xy, mesh.tri, I.coeff_lshape)
    gm = GpuMesh(mesh, ctx)
    tr = solve(gm, pb, aT=aT, rtol=1e-12)
    fl = _solve_flux(gm, pb, aT, 0, rtol=1e-12)
    assert np.max(np.abs(tr["U"] - fl["U"])) <= 1e-9 * np.max(np.abs(tr["U"]))
    assert np.max(np.abs(tr["Lambda"] - fl["Lambda"])) <= 1e-8 * np.max(np.abs(tr["Lambda"]))
    gm.close()


def test_flux_form_rejections(ctx):
    from phfem_gpu import GpuMesh
    from paper_2401_15557_gb300 import phfem as P
    gm = GpuMesh(I.square_mesh(4), ctx)
    fm, bc = gm.edge_data(lambda x, y: 1.0 + 0 * x, lambda x, y, nx, ny: 0 * x, lambda x, y: 0 * x)
    for kw, msg in [(dict(delta=0.0), "delta > 0"), (dict(delta=1.0, dt=0.1), "dt = 0"),
                    (dict(delta=1.0, form=7), "form")]:
        kw.setdefault("form", P.PHFEM_FORM_FLUX)
        with pytest.raises(P.PhfemError) as ei:
            P.phfem_assemble(gm.h, fm, bc, **kw)
        assert ei.value.status == P.PHFEM_EINVAL and msg in str(ei.value)
    sysh = P.phfem_assemble(gm.h, fm, bc, delta=1.0, form=P.PHFEM_FORM_FLUX)
    In = gm.info
    val = torch.empty(max(In["nnz"], 1), dtype=torch.float64, device="cuda")
    rhs = torch.empty(max(In["nF"], 1), dtype=torch.float64, device="cuda")
    with pytest.raises(P.PhfemError) as ei:
        P.phfem_sys_csr(sysh, val, rhs)
    assert ei.value.status == P.PHFEM_EINVAL
    P.phfem_sys_destroy(sysh)
    gm.close()
