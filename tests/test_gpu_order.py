"""The locality order of the Jacobi iteration (Morton order of the edge
midpoints, a stable device radix sort) and the solve that runs in it, against
the paper-order solve and the oracle's direct saddle-point solve."""
import numpy as np
import pytest

from oracle import phfem_oracle as O
from paper_2401_15557_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _morton_keys(xy, ed2el, nE):
    """Keys of the documented rule: midpoints on a 2^q x 2^q grid over the
    vertices' bounding box, 4 nE <= 4^q, q <= 15, bits interleaved x first."""
    q = 4
    while q < 15 and (1 << (2 * q)) < 4 * nE:
        q += 1
    x0, y0 = xy[:, 0].min(), xy[:, 1].min()
    span = max(xy[:, 0].max() - x0, xy[:, 1].max() - y0)
    scale = (1 << q) / span
    mid = 0.5 * (xy[ed2el[:, 0]] + xy[ed2el[:, 1]])
    top = (1 << q) - 1
    qx = np.floor(np.clip((mid[:, 0] - x0) * scale, 0, top)).astype(np.uint64)
    qy = np.floor(np.clip((mid[:, 1] - y0) * scale, 0, top)).astype(np.uint64)
    key = np.zeros(nE, np.uint64)
    for b in range(q):
        key |= ((qx >> b) & 1) << (2 * b)
        key |= ((qy >> b) & 1) << (2 * b + 1)
    return key


MESHES = {
    "square8": lambda: I.square_mesh(8),
    "lshape_l1": lambda: I.lshape_mesh(n=12, jitter=0.2, seed=I.seed_for(1, 71), levels=1),
    "lshape_l2": lambda: I.lshape_mesh(n=32, jitter=0.2, seed=I.seed_for(1, 72), levels=2),
}


@pytest.mark.parametrize("name", sorted(MESHES))
def test_order_is_the_stable_morton_sort(name):
    from paper_2401_15557_gb300 import phfem as P
    from phfem_gpu import GpuMesh

    ctx = P.phfem_ctx_create()
    mesh = MESHES[name]()
    gm = GpuMesh(mesh, ctx)
    out = P.phfem_mesh_order(gm.h)
    perm = out["perm"].cpu().numpy()
    nE = gm.info["nE"]
    assert np.array_equal(np.sort(perm), np.arange(nE))
    key = _morton_keys(mesh.xy, gm.tables["ed2el"], nE)[perm]
    assert np.all(key[1:] >= key[:-1])
    ties = key[1:] == key[:-1]
    assert np.all(perm[1:][ties] > perm[:-1][ties])  # ties keep the paper's order
    if name == "lshape_l2":
        assert out["overflow_rows"] > 0  # rows with far neighbours exist, and take the full-index path
    gm.close()
    P.phfem_ctx_destroy(ctx)


@pytest.mark.parametrize("name", ["lshape_l1", "lshape_l2"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_locality_order_solve_matches_paper_order_and_oracle(name, prec):
    from paper_2401_15557_gb300 import phfem as P
    from phfem_gpu import GpuMesh, dev
    import torch

    precision = P.PHFEM_FP64 if prec == "fp64" else P.PHFEM_FP32_IR
    ctx = P.phfem_ctx_create()
    mesh = MESHES[name]()
    aT = I.element_mean_at_midpoints(mesh.xy, mesh.tri, I.coeff_lshape)
    pb = I.problem_sine_exp()
    pb.delta = 1.0
    gm = GpuMesh(mesh, ctx)
    fm, bc = gm.edge_data(pb.f, pb.g, pb.uD)
    sysh = P.phfem_assemble(gm.h, fm, bc, a_T=dev(aT, torch.float64), delta=pb.delta, precision=precision)
    nE, nT, nL = gm.info["nE"], gm.info["nT"], gm.info["nL"]
    res = {}
    for order in (0, 1, 0):
        w = torch.empty(nE, dtype=torch.float64, device="cuda")
        U = torch.empty(3 * nT, dtype=torch.float64, device="cuda")
        L = torch.empty(nL, dtype=torch.float64, device="cuda")
        st = P.phfem_solve(sysh, P.solve_opts(rtol=1e-10, order=order), w=w, U=U, Lambda=L)
        assert st["converged"] == 1 and st["rel_residual"] <= 1e-10, (order, st)
        r = (w.cpu().numpy(), U.cpu().numpy(), L.cpu().numpy(), st)
        if order in res:  # the same solve twice: bitwise the same
            assert np.array_equal(res[order][0], r[0]) and res[order][3]["iterations"] == st["iterations"]
        res[order] = r
    ref = O.solve_saddle(mesh, pb, aT=aT)
    for order, (w, U, L, st) in res.items():
        eu = np.max(np.abs(U - ref["U"])) / np.max(np.abs(ref["U"]))
        el = np.max(np.abs(L - ref["Lambda"])) / np.max(np.abs(ref["Lambda"]))
        assert eu < 1e-7 and el < 1e-6, (order, eu, el)
    w0, w1 = res[0][0], res[1][0]
    assert np.max(np.abs(w0 - w1)) <= 1e-8 * np.max(np.abs(w1))
    P.phfem_sys_destroy(sysh)
    gm.close()
    P.phfem_ctx_destroy(ctx)


def test_unfused_fp32_iteration_matches_fused():
    """The FP32 iteration's kernel variants (phfem_ctx_set_cg_kernel): the
    default fused product with the rows staged in shared memory (0) and the
    fused product reading them through L1/L2 (2) visit the same rows in the same
    order with the same arithmetic, so their solutions are bitwise equal; with
    the direction update as a kernel of its own (1) the solve converges to the
    same solution within the solve tolerance.  The mesh (85,069 edges) spans
    332 tiles of 256 rows and a ragged last one of 77."""
    from paper_2401_15557_gb300 import phfem as P
    from phfem_gpu import GpuMesh, dev
    import torch

    ctx = P.phfem_ctx_create()
    mesh = I.lshape_mesh(n=97, jitter=0.2, seed=I.seed_for(1, 73))
    aT = I.element_mean_at_midpoints(mesh.xy, mesh.tri, I.coeff_lshape)
    pb = I.problem_sine_exp()
    pb.delta = 1.0
    gm = GpuMesh(mesh, ctx)
    fm, bc = gm.edge_data(pb.f, pb.g, pb.uD)
    sysh = P.phfem_assemble(gm.h, fm, bc, a_T=dev(aT, torch.float64), delta=pb.delta, precision=P.PHFEM_FP32_IR)
    assert gm.info["nE"] == 85069
    ws, its = [], []
    for variant in (0, 1, 2):
        P.phfem_ctx_set_cg_kernel(ctx, variant)
        w = torch.empty(gm.info["nE"], dtype=torch.float64, device="cuda")
        st = P.phfem_solve(sysh, P.solve_opts(rtol=1e-10), w=w)
        assert st["converged"] == 1 and st["rel_residual"] <= 1e-10, (variant, st)
        ws.append(w.cpu().numpy())
        its.append(st["iterations"])
    assert np.array_equal(ws[0], ws[2]) and its[0] == its[2]
    assert np.max(np.abs(ws[0] - ws[1])) <= 1e-8 * np.max(np.abs(ws[1]))
    for bad in (-1, 3):
        with pytest.raises(P.PhfemError):
            P.phfem_ctx_set_cg_kernel(ctx, bad)
    P.phfem_sys_destroy(sysh)
    gm.close()
    P.phfem_ctx_destroy(ctx)


def test_fp32_solve_of_tiny_data():
    """The square scaled by 2^-45 with the sine data: u ~ 1e-13, so FP32 squares
    of the residual would underflow without the power-of-two scaling of the
    inner vectors at each true residual.  FP32 + refinement converges to the
    FP64 solution and to the oracle's."""
    import dataclasses
    from paper_2401_15557_gb300 import phfem as P
    from phfem_gpu import GpuMesh, solve

    ctx = P.phfem_ctx_create()
    base = I.square_mesh(6)
    mesh = dataclasses.replace(base, xy=np.ascontiguousarray(base.xy * 2.0 ** -45))
    pb = I.problem_sine_exp()
    pb.delta = 1.0
    gm = GpuMesh(mesh, ctx)
    out = {}
    for prec in (P.PHFEM_FP64, P.PHFEM_FP32_IR):
        r = solve(gm, pb, precision=prec, rtol=1e-10)
        assert r["stats"]["converged"] == 1 and r["stats"]["rel_residual"] <= 1e-10, (prec, r["stats"])
        out[prec] = r
        P.phfem_sys_destroy(r["sys"])
    w64, w32 = out[P.PHFEM_FP64]["w"], out[P.PHFEM_FP32_IR]["w"]
    assert np.max(np.abs(w64)) < 1e-12  # the data really are tiny
    assert np.max(np.abs(w32 - w64)) <= 1e-8 * np.max(np.abs(w64))
    ref = O.solve_saddle(mesh, pb)
    U = out[P.PHFEM_FP32_IR]["U"]
    assert np.max(np.abs(U - ref["U"])) <= 1e-7 * np.max(np.abs(ref["U"]))
    gm.close()
    P.phfem_ctx_destroy(ctx)
