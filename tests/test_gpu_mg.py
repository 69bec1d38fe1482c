"""Multigrid preconditioner over device-refined hierarchies: transfer
operators against the oracle's Crouzeix-Raviart prolongation, solutions
against the oracle's saddle-point solve, level-independent iteration counts,
determinism, Crank-Nicolson, and rejections."""
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


class Hierarchy:
    """Level 0 built from host arrays, then refined on the device; the oracle's
    refinement of the same arrays gives the host copies of every level."""

    def __init__(self, ctx, m0, levels):
        from phfem_gpu import dev
        from paper_2401_15557_gb300 import phfem as P
        self.P = P
        h = P.phfem_mesh_build(ctx, dev(m0.xy, torch.float64), dev(m0.tri, torch.int32),
                               dev(m0.dirichlet, torch.int32) if len(m0.dirichlet) else None,
                               dev(m0.neumann, torch.int32) if len(m0.neumann) else None)
        self.handles = [h]
        self.meshes = [m0]
        xy, tri, d, n = m0.xy, m0.tri, m0.dirichlet, m0.neumann
        for _ in range(levels):
            self.handles.append(P.phfem_mesh_refine(self.handles[-1]))
            xy, tri, d, n = O.redrefine(xy, tri, d, n)
            self.meshes.append(I.Mesh(xy=xy, tri=tri.astype(np.int32), dirichlet=d.astype(np.int32),
                                      neumann=n.astype(np.int32), name=f"level{len(self.meshes)}"))
        self.tables = [{k: v.cpu().numpy() for k, v in P.phfem_mesh_tables(h).items()} for h in self.handles]

    def close(self):
        for h in self.handles:
            self.P.phfem_mesh_destroy(h)


def _system(H, pb, aT, precision, dt=0.0):
    from phfem_gpu import dev
    P = H.P
    tf = H.tables[-1]
    fm, bc = I.edge_data(H.meshes[-1].xy, tf["ed2el"], tf["eclass"], pb.f, pb.g, pb.uD)
    return P.phfem_assemble(H.handles[-1], dev(fm, torch.float64) if dt == 0 else None,
                            dev(bc, torch.float64) if dt == 0 else None,
                            a_T=dev(aT, torch.float64), delta=pb.delta, dt=dt, precision=precision)


def _solve(P, sysh, info, rtol=1e-10):
    U = torch.empty(3 * info["nT"], dtype=torch.float64, device="cuda")
    L = torch.empty(max(info["nL"], 1), dtype=torch.float64, device="cuda")
    w = torch.empty(info["nE"], dtype=torch.float64, device="cuda")
    st = P.phfem_solve(sysh, P.solve_opts(rtol=rtol), w=w, U=U, Lambda=L)
    torch.cuda.synchronize()
    return st, U.cpu().numpy(), L.cpu().numpy()[:info["nL"]], w.cpu().numpy()


@pytest.mark.parametrize("mk", ["lshape", "square_alldirichlet"])
def test_transfer_matches_oracle_prolongation(ctx, mk):
    from phfem_gpu import dev
    m0 = {"lshape": lambda: I.lshape_mesh(n=4, seed=I.seed_for(1, 41)),
          "square_alldirichlet": lambda: I.square_mesh(3, dirichlet_sides=("left", "right", "top", "bottom"))}[mk]()
    H = Hierarchy(ctx, m0, 2)
    P = H.P
    pb = I.problem_sine_exp()
    pb.delta = 0.5
    aT = I.element_mean_at_midpoints(H.meshes[-1].xy, H.meshes[-1].tri, I.coeff_lshape)
    sysh = _system(H, pb, aT, P.PHFEM_FP64)
    mg = P.phfem_mg_create(sysh, H.handles, a_T=dev(aT, torch.float64))
    rng = np.random.default_rng(7)
    for lev in range(2):
        mc, mf = H.meshes[lev], H.meshes[lev + 1]
        Pm = O.cr_prolongation(mc.xy, mc.tri, mf.xy, mf.tri)
        dc = H.tables[lev]["eclass"] == 1
        df = H.tables[lev + 1]["eclass"] == 1
        zc = rng.standard_normal(Pm.shape[1])
        zc[dc] = 0.0
        out = torch.empty(Pm.shape[0], dtype=torch.float64, device="cuda")
        P.phfem_mg_transfer(mg, lev, 0, dev(zc, torch.float64), out)
        want = Pm @ zc
        want[df] = 0.0
        assert np.max(np.abs(out.cpu().numpy() - want)) <= 1e-14 * np.max(np.abs(want))
        rf = rng.standard_normal(Pm.shape[0])
        rf[df] = 0.0
        outc = torch.empty(Pm.shape[1], dtype=torch.float64, device="cuda")
        P.phfem_mg_transfer(mg, lev, 1, dev(rf, torch.float64), outc)
        want = Pm.T @ rf
        want[dc] = 0.0
        assert np.max(np.abs(outc.cpu().numpy() - want)) <= 1e-14 * np.max(np.abs(want))
    P.phfem_mg_destroy(mg)
    P.phfem_sys_destroy(sysh)
    H.close()


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32ir"])
def test_mg_solve_matches_saddle_solve(ctx, precision):
    from phfem_gpu import dev
    H = Hierarchy(ctx, I.lshape_mesh(n=6, seed=I.seed_for(1, 43)), 3)
    P = H.P
    pb = I.problem_sine_exp()
    pb.delta = 1.0
    mesh = H.meshes[-1]
    aT = I.element_mean_at_midpoints(mesh.xy, mesh.tri, I.coeff_lshape)
    sysh = _system(H, pb, aT, precision)
    info = P.phfem_mesh_info_get(H.handles[-1])
    st_j, U_j, L_j, _ = _solve(P, sysh, info)
    mg = P.phfem_mg_create(sysh, H.handles, a_T=dev(aT, torch.float64))
    P.phfem_sys_set_mg(sysh, mg)
    st, U, L, w = _solve(P, sysh, info)
    st2, U2, L2, w2 = _solve(P, sysh, info)
    assert st["converged"] == 1 and st["rel_residual"] <= 1e-10, st
    assert st["iterations"] * 10 < st_j["iterations"], (st, st_j)
    # deterministic
    assert np.array_equal(w, w2) and st["iterations"] == st2["iterations"]
    ref = O.solve_saddle(mesh, pb, aT=aT)
    assert np.max(np.abs(U - ref["U"])) <= 1e-7 * np.max(np.abs(ref["U"]))
    assert np.max(np.abs(L - ref["Lambda"])) <= 1e-6 * np.max(np.abs(ref["Lambda"]))
    cs = O.condensed_system(mesh, pb, aT=aT)
    assert O.relative_residual(cs["S"], cs["rhs"], w[cs["st"]["bsets"]["free"]]) <= 1.2e-10
    # the coarsest iteration one launch per step: the same arithmetic per row as
    # the default single cluster launch (the coarse rows spread over its 8 CTAs,
    # neighbours read across them), so bitwise the same solve
    mg_s = P.phfem_mg_create(sysh, H.handles, a_T=dev(aT, torch.float64), flags=P.PHFEM_MG_COARSE_STEPWISE)
    P.phfem_sys_set_mg(sysh, mg_s)
    st4, U4, _, w4 = _solve(P, sysh, info)
    assert np.array_equal(w, w4) and st4["iterations"] == st["iterations"]
    P.phfem_mg_destroy(mg_s)
    # detached: back to Jacobi with the same answer
    P.phfem_sys_set_mg(sysh, None)
    st3, U3, _, _ = _solve(P, sysh, info)
    assert st3["iterations"] == st_j["iterations"] and np.array_equal(U3, U_j)
    P.phfem_mg_destroy(mg)
    P.phfem_sys_destroy(sysh)
    H.close()


def test_iterations_do_not_grow_with_refinement(ctx):
    from phfem_gpu import dev
    counts = []
    for levels in (1, 2, 3, 4):
        H = Hierarchy(ctx, I.lshape_mesh(n=4, seed=I.seed_for(1, 45)), levels)
        P = H.P
        pb = I.problem_sine_exp()
        pb.delta = 1.0
        mesh = H.meshes[-1]
        aT = I.element_mean_at_midpoints(mesh.xy, mesh.tri, I.coeff_lshape)
        sysh = _system(H, pb, aT, P.PHFEM_FP32_IR)
        mg = P.phfem_mg_create(sysh, H.handles, a_T=dev(aT, torch.float64))
        P.phfem_sys_set_mg(sysh, mg)
        st, _, _, _ = _solve(P, sysh, P.phfem_mesh_info_get(H.handles[-1]))
        assert st["converged"] >= 1
        counts.append(st["iterations"])
        P.phfem_mg_destroy(mg)
        P.phfem_sys_destroy(sysh)
        H.close()
    assert max(counts) <= 40 and max(counts) <= 1.6 * min(counts), counts


def test_crank_nicolson_with_multigrid(ctx):
    """Graph-captured and host-driven steps under multigrid agree with the
    Jacobi steps to the solver tolerance."""
    from phfem_gpu import dev
    from paper_2401_15557_gb300 import phfem as P
    H = Hierarchy(ctx, I.square_mesh(4), 3)
    sq = H.meshes[-1]
    tf = H.tables[-1]
    pi = np.pi
    s_fn = lambda x, y: np.sin(pi * x) * np.sin(pi * y)
    f0, g0 = I.edge_data(sq.xy, tf["ed2el"], tf["eclass"], lambda x, y: (2 * pi * pi - 1) * s_fn(x, y),
                         lambda x, y, nx, ny: pi * (np.cos(pi * x) * np.sin(pi * y) * nx
                                                    + np.sin(pi * x) * np.cos(pi * y) * ny),
                         lambda x, y: 0 * x)
    w0, _ = I.edge_data(sq.xy, tf["ed2el"], tf["eclass"], s_fn)
    dt, steps = 1.0 / 32, 6
    phi = np.exp(-dt * np.arange(steps + 1))[None]
    outs = {}
    for mode in ("jacobi", "mg_host", "mg_graph"):
        s2 = P.phfem_assemble(H.handles[-1], None, None, delta=0.0, dt=dt, precision=P.PHFEM_FP32_IR)
        mg = None
        if mode != "jacobi":
            mg = P.phfem_mg_create(s2, H.handles)
            P.phfem_sys_set_mg(s2, mg)
        cn = P.phfem_cn_create(s2, dev(f0[None], torch.float64), dev(g0[None], torch.float64), phi,
                               dev(w0, torch.float64))
        opts = P.solve_opts(rtol=1e-11)
        st = P.phfem_cn_step_graph(cn, steps, opts) if mode == "mg_graph" else P.phfem_cn_step(cn, steps, opts)
        U = torch.empty(3 * sq.nT, dtype=torch.float64, device="cuda")
        P.phfem_cn_read(cn, U=U)
        outs[mode] = (U.cpu().numpy(), st)
        P.phfem_cn_destroy(cn)
        if mg is not None:
            P.phfem_mg_destroy(mg)
        P.phfem_sys_destroy(s2)
    Uj = outs["jacobi"][0]
    for mode in ("mg_host", "mg_graph"):
        assert np.max(np.abs(outs[mode][0] - Uj)) <= 1e-8 * np.max(np.abs(Uj)), mode
        assert outs[mode][1]["iterations"] < outs["jacobi"][1]["iterations"]
    assert np.array_equal(outs["mg_host"][0], outs["mg_graph"][0])
    H.close()


def test_rejections(ctx):
    from phfem_gpu import GpuMesh
    from paper_2401_15557_gb300 import phfem as P
    H = Hierarchy(ctx, I.square_mesh(3), 1)
    other = GpuMesh(I.square_mesh(6), ctx)  # the refinement's counts, not the system's mesh
    m3 = I.square_mesh(3)
    perm = np.roll(np.arange(m3.nT), 5)
    shuffled = GpuMesh(I.Mesh(xy=m3.xy, tri=m3.tri[perm], dirichlet=m3.dirichlet, neumann=m3.neumann, name="perm"),
                       ctx)  # the coarse counts, but the fine mesh is not its refinement
    pb = I.problem_sine_exp()
    pb.delta = 1.0
    tf = H.tables[-1]
    fm, bc = I.edge_data(H.meshes[-1].xy, tf["ed2el"], tf["eclass"], pb.f, pb.g, pb.uD)
    from phfem_gpu import dev
    sysh = P.phfem_assemble(H.handles[-1], dev(fm, torch.float64), dev(bc, torch.float64), delta=1.0)
    for meshes in ([H.handles[-1]], [other.h, H.handles[-1]], [H.handles[0], other.h],
                   [shuffled.h, H.handles[-1]]):
        with pytest.raises(P.PhfemError) as ei:
            P.phfem_mg_create(sysh, meshes)
        assert ei.value.status == P.PHFEM_EINVAL
    flux = P.phfem_assemble(H.handles[-1], dev(fm, torch.float64), dev(bc, torch.float64), delta=1.0,
                            form=P.PHFEM_FORM_FLUX)
    with pytest.raises(P.PhfemError):
        P.phfem_mg_create(flux, H.handles)
    P.phfem_sys_destroy(flux)
    P.phfem_sys_destroy(sysh)
    other.close()
    shuffled.close()
    H.close()


def test_system_destroyed_before_its_multigrid(ctx):
    from phfem_gpu import dev
    H = Hierarchy(ctx, I.square_mesh(3), 2)
    P = H.P
    pb = I.problem_sine_exp()
    pb.delta = 1.0
    aT = np.ones(H.meshes[-1].nT)
    sysh = _system(H, pb, aT, P.PHFEM_FP64)
    mg = P.phfem_mg_create(sysh, H.handles, a_T=dev(aT, torch.float64))
    P.phfem_sys_set_mg(sysh, mg)
    P.phfem_sys_destroy(sysh)
    out = torch.empty(H.tables[1]["eclass"].size, dtype=torch.float64, device="cuda")
    inp = torch.zeros(H.tables[0]["eclass"].size, dtype=torch.float64, device="cuda")
    P.phfem_mg_transfer(mg, 0, 0, inp, out)  # level 1 is not the finest: still valid
    with pytest.raises(P.PhfemError):
        P.phfem_mg_transfer(mg, 1, 0, torch.zeros_like(out), torch.empty(H.tables[2]["eclass"].size,
                                                                        dtype=torch.float64, device="cuda"))
    P.phfem_mg_destroy(mg)
    H.close()


def test_full_size_lshape_multigrid(ctx):
    """The benchmark's multigrid step at full size (level 0 refined five times on
    the device, 6.3M triangles): the FP64 residual of the exported CSR system
    meets the target, the iteration count stays small, and U equals the
    element-major U of the Jacobi solve on the generator's level-5 mesh (the
    same triangles in the same order)."""
    import scipy.sparse as sp
    from phfem_gpu import GpuMesh, dev, solve
    from paper_2401_15557_gb300 import phfem as P
    m0 = I.lshape_mesh(n=32, seed=I.seed_for(1, 0), levels=0)
    h0 = P.phfem_mesh_build(ctx, dev(m0.xy, torch.float64), dev(m0.tri, torch.int32),
                            dev(m0.dirichlet, torch.int32), dev(m0.neumann, torch.int32))
    hs = [h0]
    for _ in range(5):
        hs.append(P.phfem_mesh_refine(hs[-1]))
    fine = I.lshape_mesh(n=32, seed=I.seed_for(1, 0), levels=5)
    aT = I.element_mean_at_midpoints(fine.xy, fine.tri, I.coeff_lshape)
    info = P.phfem_mesh_info_get(hs[-1])
    ones = torch.ones(info["nE"], dtype=torch.float64, device="cuda")
    sysh = P.phfem_assemble(hs[-1], ones, torch.zeros_like(ones), a_T=dev(aT, torch.float64), delta=1.0,
                            precision=P.PHFEM_FP32_IR)
    mg = P.phfem_mg_create(sysh, hs, a_T=dev(aT, torch.float64))
    P.phfem_sys_set_mg(sysh, mg)
    U = torch.empty(3 * info["nT"], dtype=torch.float64, device="cuda")
    w = torch.empty(info["nE"], dtype=torch.float64, device="cuda")
    st = P.phfem_solve(sysh, P.solve_opts(rtol=1e-10), w=w, U=U)
    # the solver's iterate (an FP64 pair plus the last correction) meets 1e-10
    assert st["converged"] == 1 and st["iterations"] <= 60 and st["rel_residual"] <= 1e-10, st
    T = {k: v.cpu().numpy() for k, v in P.phfem_mesh_tables(hs[-1]).items()}
    val = torch.empty(info["nnz"], dtype=torch.float64, device="cuda")
    rhs = torch.empty(info["nF"], dtype=torch.float64, device="cuda")
    P.phfem_sys_csr(sysh, val, rhs)
    S = sp.csr_matrix((val.cpu().numpy(), T["col"], T["row_ptr"]), shape=(info["nF"], info["nF"]))
    wf = w.cpu().numpy()[T["free_id"] >= 0]
    bf = rhs.cpu().numpy()
    # its rounding to FP64 (the exported w) may add up to 2^-53 || |S| |w| || / ||b||
    rounding = 2.0 ** -53 * np.linalg.norm(abs(S) @ np.abs(wf)) / np.linalg.norm(bf)
    assert O.relative_residual(S, bf, wf) <= 1e-10 + rounding
    # the same solution as Jacobi-PCG on the generator's numbering of the mesh
    pb = I.Problem(f=lambda x, y: 1.0 + 0 * x, g=lambda x, y, nx, ny: 0 * x, uD=lambda x, y: 0 * x, delta=1.0)
    gm = GpuMesh(fine, ctx)
    out = solve(gm, pb, aT=aT, precision=1, rtol=1e-10)
    Uj = out["U"]
    assert np.max(np.abs(U.cpu().numpy() - Uj)) <= 1e-8 * np.max(np.abs(Uj))
    gm.close()
    P.phfem_mg_destroy(mg)
    P.phfem_sys_destroy(sysh)
    for h in reversed(hs):
        P.phfem_mesh_destroy(h)


@pytest.mark.parametrize("n0", [3, 30, 60], ids=["one_block", "cluster4", "cluster8"])
def test_coarse_iteration_in_one_launch(ctx, n0):
    """The coarsest Chebyshev iteration in one launch (one block for a few
    hundred rows, a cluster of 4 or 8 CTAs reading neighbours across them for
    thousands) against the step-per-launch iteration: bitwise the same solve."""
    H = Hierarchy(ctx, I.square_mesh(n0), 2)
    P = H.P
    pb = I.problem_sine_exp()
    pb.delta = 0.5
    mesh = H.meshes[-1]
    sysh = _system(H, pb, np.ones(mesh.nT), P.PHFEM_FP32_IR)
    info = P.phfem_mesh_info_get(H.handles[-1])
    coarse = P.phfem_mesh_info_get(H.handles[0])["nE"]
    assert coarse == 3 * n0 * n0 + 2 * n0
    ws, its = [], []
    for flags in (0, P.PHFEM_MG_COARSE_STEPWISE):
        mg = P.phfem_mg_create(sysh, H.handles, flags=flags)
        P.phfem_sys_set_mg(sysh, mg)
        st, _, _, w = _solve(P, sysh, info)
        assert st["converged"] == 1 and st["rel_residual"] <= 1e-10, st
        ws.append(w)
        its.append(st["iterations"])
        P.phfem_sys_set_mg(sysh, None)
        P.phfem_mg_destroy(mg)
    assert np.array_equal(ws[0], ws[1]) and its[0] == its[1]
    P.phfem_sys_destroy(sysh)
    H.close()
