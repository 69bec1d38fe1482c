"""Batched solve (one persistent launch) against the oracle and against the
single-mesh path."""
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


def _members():
    """Meshes of uneven size with varied data: (mesh, aT, delta, problem)."""
    out = []
    sizes = [1, 3, 17, 5, 9, 24, 2, 12]
    for i, n in enumerate(sizes):
        m = I.square_mesh(n)
        aT = I.element_mean_at_midpoints(m.xy, m.tri, I.fourier_field(I.seed_for(3, 100 + i)).a)
        pb = I.problem_sine_exp()
        pb.delta = 0.3 * (i % 3)
        out.append((m, aT, pb.delta, pb))
    lsh = I.lshape_mesh(n=6, seed=I.seed_for(1, 71), levels=1)
    pb = I.problem_sine_exp()
    pb.delta = 1.0
    out.append((lsh, I.element_mean_at_midpoints(lsh.xy, lsh.tri, I.coeff_lshape), 1.0, pb))
    cc = I.criss_cross(3)
    pb = I.problem_sine_exp()
    pb.delta = 0.0
    out.append((cc, np.ones(cc.nT), 0.0, pb))
    nd = I.square_mesh(6, dirichlet_sides=())
    pb = I.problem_sine_exp()
    pb.delta = 0.7
    out.append((nd, np.full(nd.nT, 1.3), 0.7, pb))
    return out


def _build(ctx, members):
    from paper_2401_15557_gb300 import phfem as P
    from phfem_gpu import GpuMesh
    gms = [GpuMesh(m, ctx) for m, _, _, _ in members]
    fs, bcs = [], []
    for gm, (m, aT, d, pb) in zip(gms, members):
        f, bc = I.edge_data(m.xy, gm.tables["ed2el"], gm.tables["eclass"], pb.f, pb.g, pb.uD)
        fs.append(f)
        bcs.append(bc)
    batch = P.phfem_batch_create(ctx, [gm.h for gm in gms])
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    data = dict(aT=dev(np.concatenate([mb[1] for mb in members])),
                delta=dev(np.array([mb[2] for mb in members])),
                f=dev(np.concatenate(fs)), bc=dev(np.concatenate(bcs)))
    return gms, batch, data


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32ir"])
def test_batch_matches_oracle_and_single_mesh(ctx, precision):
    from paper_2401_15557_gb300 import phfem as P
    from phfem_gpu import solve
    members = _members()
    gms, batch, data = _build(ctx, members)
    count = len(members)
    toff, eoff, loff = P.phfem_batch_offsets(batch, count)
    U = torch.empty(3 * int(toff[-1]), dtype=torch.float64, device="cuda")
    L = torch.empty(int(loff[-1]), dtype=torch.float64, device="cuda")
    w = torch.empty(int(eoff[-1]), dtype=torch.float64, device="cuda")
    res = P.phfem_batch_solve(batch, count, data["delta"], a_T=data["aT"], f_mid=data["f"], bc_mid=data["bc"],
                              precision=precision, opts=P.solve_opts(rtol=1e-10), w=w, U=U, Lambda=L)
    torch.cuda.synchronize()
    assert np.all(res["converged"] == 1), res
    assert np.all(res["rel_residual"] <= 1e-10)
    Uh, Lh, wh = U.cpu().numpy(), L.cpu().numpy(), w.cpu().numpy()
    for i, (gm, (m, aT, d, pb)) in enumerate(zip(gms, members)):
        ref = O.solve_saddle(m, pb, aT=aT)
        Ui = Uh[3 * toff[i]:3 * toff[i + 1]]
        Li = Lh[loff[i]:loff[i + 1]]
        assert np.max(np.abs(Ui - ref["U"])) <= 1e-7 * max(1.0, np.max(np.abs(ref["U"]))), i
        assert np.max(np.abs(Li - ref["Lambda"])) <= 1e-6 * max(1.0, np.max(np.abs(ref["Lambda"]))), i
        cs = O.condensed_system(m, pb, aT=aT)
        wi = wh[eoff[i]:eoff[i + 1]]
        assert O.relative_residual(cs["S"], cs["rhs"], wi[cs["st"]["bsets"]["free"]]) <= 1.2e-10, i
        single = solve(gm, pb, aT=aT, precision=precision, rtol=1e-10)
        assert np.max(np.abs(Ui - single["U"])) <= 1e-7 * max(1.0, np.max(np.abs(single["U"]))), i
    # every launch shape (threads per block, CTAs per mesh as a thread-block
    # cluster) gives a converged, consistent answer; a shape's result does not
    # depend on the batch's other meshes (the same mesh alone, bitwise); the
    # tuner picks one shape
    for bs, cl in P.BATCH_SHAPES:
        U2 = torch.empty_like(U)
        r2 = P.phfem_batch_solve(batch, count, data["delta"], a_T=data["aT"], f_mid=data["f"], bc_mid=data["bc"],
                                 precision=precision, U=U2, block=bs, cluster=cl)
        assert np.all(r2["converged"] == 1), (bs, cl)
        assert np.max(np.abs(U2.cpu().numpy() - Uh)) <= 1e-7 * np.max(np.abs(Uh)), (bs, cl)
        if (bs, cl) in ((256, 1), (512, 4)):
            one = P.phfem_batch_create(ctx, [gms[1].h])
            U1 = torch.empty(3 * int(toff[2] - toff[1]), dtype=torch.float64, device="cuda")
            P.phfem_batch_solve(one, 1, data["delta"][1:2], a_T=data["aT"][toff[1]:toff[2]],
                                f_mid=data["f"][eoff[1]:eoff[2]], bc_mid=data["bc"][eoff[1]:eoff[2]],
                                precision=precision, U=U1, block=bs, cluster=cl)
            assert np.array_equal(U1.cpu().numpy(), U2.cpu().numpy()[3 * toff[1]:3 * toff[2]]), (bs, cl)
            P.phfem_batch_destroy(one)
    chosen, ms = P.phfem_batch_tune(batch, data["delta"], a_T=data["aT"], f_mid=data["f"], bc_mid=data["bc"],
                                    precision=precision)
    assert chosen in P.BATCH_SHAPES and len(ms) == len(P.BATCH_SHAPES) and all(v > 0 for v in ms.values())
    P.phfem_batch_destroy(batch)
    for gm in gms:
        gm.close()


def test_batch_refuses_singular_member(ctx):
    from paper_2401_15557_gb300 import phfem as P
    from phfem_gpu import GpuMesh
    gm = GpuMesh(I.square_mesh(4, dirichlet_sides=()), ctx)
    batch = P.phfem_batch_create(ctx, [gm.h])
    with pytest.raises(P.PhfemError) as ei:
        P.phfem_batch_solve(batch, 1, torch.zeros(1, dtype=torch.float64, device="cuda"))
    assert ei.value.status == -1
    P.phfem_batch_destroy(batch)
    gm.close()


def test_batched_workload_sample(ctx):
    """64 members of the batched workload (sides log-uniform in [8, 256],
    a = exp(0.5 z), delta ~ U[0, 2], f = 1, homogeneous data): all converge
    and sampled members match the single-mesh solve."""
    from paper_2401_15557_gb300 import phfem as P
    from phfem_gpu import GpuMesh, solve
    sides = I.batch_sides(64)
    members = [I.batch_member(i, n) for i, n in enumerate(sides)]
    gms = [GpuMesh(m, ctx) for m, _, _ in members]
    batch = P.phfem_batch_create(ctx, [g.h for g in gms])
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    aT = dev(np.concatenate([a for _, a, _ in members]))
    delta = dev(np.array([d for _, _, d in members]))
    toff, eoff, loff = P.phfem_batch_offsets(batch, len(members))
    f = torch.ones(int(eoff[-1]), dtype=torch.float64, device="cuda")
    U = torch.empty(3 * int(toff[-1]), dtype=torch.float64, device="cuda")
    res = P.phfem_batch_solve(batch, len(members), delta, a_T=aT, f_mid=f, precision=1, U=U)
    assert np.all(res["converged"] >= 1) and np.all(res["rel_residual"] <= 1e-10)
    Uh = U.cpu().numpy()
    one = I.Problem(f=lambda x, y: 1.0 + 0 * x, g=lambda x, y, nx, ny: 0 * x, uD=lambda x, y: 0 * x)
    for i in (0, 7, 31, 63):
        m, a, d = members[i]
        one.delta = d
        single = solve(gms[i], one, aT=a, precision=1)
        Ui = Uh[3 * toff[i]:3 * toff[i + 1]]
        assert np.max(np.abs(Ui - single["U"])) <= 1e-7 * np.max(np.abs(single["U"])), i
    P.phfem_batch_destroy(batch)
    for g in gms:
        g.close()
