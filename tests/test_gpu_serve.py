"""Request server: results are the same alone and in the mix; admission obeys
the HBM budget in arrival order."""
import numpy as np
import pytest
import torch

from oracle import phfem_oracle as O
from paper_2401_15557_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _requests():
    """Uneven elliptic and Crank-Nicolson requests with their device inputs."""
    from paper_2401_15557_gb300 import phfem as P
    dev = lambda a, t: torch.as_tensor(np.ascontiguousarray(a), dtype=t, device="cuda")
    specs = []
    sizes = [6, 40, 12, 60, 9, 25, 16, 33]
    for i, n in enumerate(sizes):
        m = I.square_mesh(n)
        fld = I.fourier_field(I.seed_for(4, 200 + i))
        aT = I.element_mean_at_midpoints(m.xy, m.tri, fld.a)
        kind = 1 if i % 3 == 2 else 0
        specs.append(dict(mesh=m, aT=aT, kind=kind, delta=0.25 * (i % 4), steps=16 + 4 * (i % 3),
                          dt=1.0 / n, precision=i % 2))
    lsh = I.lshape_mesh(n=8, seed=I.seed_for(1, 91), levels=1)
    specs.append(dict(mesh=lsh, aT=I.element_mean_at_midpoints(lsh.xy, lsh.tri, I.coeff_lshape), kind=0, delta=1.0,
                      steps=0, dt=0.0, precision=1))
    out = []
    for sp in specs:
        m = sp["mesh"]
        nE = m.nV + m.nT - 1
        t = dict(xy=dev(m.xy, torch.float64), tri=dev(m.tri, torch.int32),
                 d=dev(m.dirichlet, torch.int32), nn=dev(m.neumann, torch.int32), aT=dev(sp["aT"], torch.float64))
        t["U"] = torch.full((3 * m.nT,), np.nan, dtype=torch.float64, device="cuda")
        t["L"] = torch.full((nE,), np.nan, dtype=torch.float64, device="cuda")
        req = P.make_request(t["xy"], t["tri"], t["d"], t["nn"], kind=sp["kind"], a_T=t["aT"], delta=sp["delta"],
                             f=1.0, uD=0.2, g=0.1, dt=sp["dt"], u0=0.0, steps=sp["steps"],
                             precision=sp["precision"], U_out=t["U"], Lambda_out=t["L"])
        out.append((sp, t, req))
    return out


def _collect(reqs, results):
    return [(t["U"].cpu().numpy().copy(), t["L"].cpu().numpy()[:r["nL"]].copy(), r) for (_, t, _), r in
            zip(reqs, results)]


def test_same_result_alone_and_in_the_mix():
    from paper_2401_15557_gb300 import phfem as P
    reqs = _requests()
    # alone: one slot, one request at a time
    srv = P.phfem_server_create(1, 64e9, P.solve_opts(rtol=1e-10))
    alone = []
    for _, _, rq in reqs:
        rid = P.phfem_server_submit(srv, rq)
        alone.append(P.phfem_server_poll(srv, rid, wait=True))
    P.phfem_server_destroy(srv)
    A = _collect(reqs, alone)
    for _, t, _ in reqs:
        t["U"].fill_(np.nan)
        t["L"].fill_(np.nan)
    # in the mix: four slots, everything submitted at once
    srv = P.phfem_server_create(4, 64e9, P.solve_opts(rtol=1e-10))
    ids = [P.phfem_server_submit(srv, rq) for _, _, rq in reqs]
    P.phfem_server_drain(srv)
    mixed = [P.phfem_server_poll(srv, i, wait=False) for i in ids]
    P.phfem_server_destroy(srv)
    B = _collect(reqs, mixed)
    slots = {r["slot"] for r in mixed}
    assert len(slots) > 1  # the work was spread over several slots
    overlap = any(mixed[i]["t_admit"] < mixed[j]["t_finish"] and mixed[j]["t_admit"] < mixed[i]["t_finish"]
                  for i in range(len(mixed)) for j in range(i + 1, len(mixed)))
    assert overlap  # admitted while others were running
    # and on the device: the event windows of two requests on different slots intersect
    assert all(0.0 <= r["t_dev_start"] < r["t_dev_end"] for r in mixed)
    dev_overlap = any(mixed[i]["slot"] != mixed[j]["slot"] and mixed[i]["t_dev_start"] < mixed[j]["t_dev_end"]
                      and mixed[j]["t_dev_start"] < mixed[i]["t_dev_end"]
                      for i in range(len(mixed)) for j in range(i + 1, len(mixed)))
    assert dev_overlap
    for (Ua, La, ra), (Ub, Lb, rb) in zip(A, B):
        assert ra["status"] == 0 and rb["status"] == 0
        assert ra["rel_residual"] <= 1e-10 and rb["rel_residual"] <= 1e-10
        # deterministic kernels: bitwise the same alone and in the mix
        assert np.array_equal(Ua, Ub) and np.array_equal(La, Lb)
        assert ra["iterations"] == rb["iterations"]
    # an elliptic request against the oracle's saddle-point solve
    sp, t, _ = reqs[1]
    m = sp["mesh"]
    pb = I.Problem(f=lambda x, y: 1.0 + 0 * x, g=lambda x, y, nx, ny: 0.1 + 0 * x, uD=lambda x, y: 0.2 + 0 * x,
                   delta=sp["delta"])
    ref = O.solve_saddle(m, pb, aT=sp["aT"])
    assert np.max(np.abs(B[1][0] - ref["U"])) <= 1e-7 * np.max(np.abs(ref["U"]))
    assert np.max(np.abs(B[1][1] - ref["Lambda"])) <= 1e-6 * np.max(np.abs(ref["Lambda"]))


def test_budget_admission_in_arrival_order():
    from paper_2401_15557_gb300 import phfem as P
    reqs = _requests()[:5]
    srv = P.phfem_server_create(4, 1.0, P.solve_opts(rtol=1e-10))  # every request exceeds the budget
    ids = [P.phfem_server_submit(srv, rq) for _, _, rq in reqs]
    P.phfem_server_drain(srv)
    res = [P.phfem_server_poll(srv, i, wait=False) for i in ids]
    P.phfem_server_destroy(srv)
    for a, b in zip(res, res[1:]):
        assert b["t_admit"] >= a["t_finish"] - 1e-9  # one at a time, first in first out
        assert b["t_admit"] >= a["t_admit"]
    assert all(r["status"] == 0 for r in res)


def test_refined_requests_use_multigrid():
    """Requests with refinement levels: the server refines on the device and
    solves with the multigrid preconditioner; the result matches the oracle's
    saddle solve on the oracle-refined mesh, bitwise the same alone and in a mix
    with plain requests, in far fewer iterations than Jacobi."""
    from paper_2401_15557_gb300 import phfem as P
    dev = lambda a, t: torch.as_tensor(np.ascontiguousarray(a), dtype=t, device="cuda")
    reqs = []
    for i, (n0, levels, kind) in enumerate([(3, 3, 0), (4, 2, 1), (5, 3, 0), (2, 4, 1)]):
        m0 = I.square_mesh(n0)
        xy, tri, d, nn = m0.xy, m0.tri, m0.dirichlet, m0.neumann
        for _ in range(levels):
            xy, tri, d, nn = O.redrefine(xy, tri, d, nn)
        fine = I.Mesh(xy=xy, tri=tri.astype(np.int32), dirichlet=d.astype(np.int32), neumann=nn.astype(np.int32),
                      name="fine")
        fld = I.fourier_field(I.seed_for(4, 300 + i))
        aT = I.element_mean_at_midpoints(fine.xy, fine.tri, fld.a)
        t = dict(xy=dev(m0.xy, torch.float64), tri=dev(m0.tri, torch.int32), d=dev(m0.dirichlet, torch.int32),
                 nn=dev(m0.neumann, torch.int32), aT=dev(aT, torch.float64),
                 U=torch.full((3 * fine.nT,), np.nan, dtype=torch.float64, device="cuda"))
        rq = P.make_request(t["xy"], t["tri"], t["d"], t["nn"], kind=kind, a_T=t["aT"], delta=0.5, f=1.0, uD=0.2,
                            g=0.1, dt=1.0 / (n0 * 2 ** levels), steps=12, precision=P.PHFEM_FP32_IR, U_out=t["U"],
                            levels=levels)
        reqs.append((fine, aT, kind, t, rq))
    srv = P.phfem_server_create(1, 64e9, P.solve_opts(rtol=1e-10))
    alone = []
    for _, _, _, t, rq in reqs:
        r = P.phfem_server_poll(srv, P.phfem_server_submit(srv, rq), wait=True)
        alone.append((t["U"].cpu().numpy().copy(), r))
        t["U"].fill_(np.nan)
    P.phfem_server_destroy(srv)
    plain = _requests()[:3]
    srv = P.phfem_server_create(4, 64e9, P.solve_opts(rtol=1e-10))
    ids = [P.phfem_server_submit(srv, rq) for *_, rq in reqs] + [P.phfem_server_submit(srv, rq) for _, _, rq in plain]
    P.phfem_server_drain(srv)
    mixed = [P.phfem_server_poll(srv, i, wait=False) for i in ids]
    P.phfem_server_destroy(srv)
    for (fine, aT, kind, t, _), (Ua, ra), rb in zip(reqs, alone, mixed):
        assert ra["status"] == 0 and rb["status"] == 0
        assert np.array_equal(Ua, t["U"].cpu().numpy()) and ra["iterations"] == rb["iterations"]
        if kind == 0:
            assert ra["iterations"] < 60, ra
            pb = I.Problem(f=lambda x, y: 1.0 + 0 * x, g=lambda x, y, nx, ny: 0.1 + 0 * x,
                           uD=lambda x, y: 0.2 + 0 * x, delta=0.5)
            ref = O.solve_saddle(fine, pb, aT=aT)
            assert np.max(np.abs(Ua - ref["U"])) <= 1e-7 * np.max(np.abs(ref["U"]))
    assert all(r["status"] == 0 for r in mixed)


def test_midpoint_data_requests():
    """Requests with midpoint arrays instead of constants: arrays holding the
    constants give bitwise the request with the constants (both kinds); an
    elliptic request with the sine data of a manufactured problem matches the
    oracle's saddle solve with that data."""
    from paper_2401_15557_gb300 import phfem as P
    from phfem_gpu import GpuMesh
    dev = lambda a, t: torch.as_tensor(np.ascontiguousarray(a), dtype=t, device="cuda")
    ctx = P.phfem_ctx_create()
    srv = P.phfem_server_create(2, 64e9, P.solve_opts(rtol=1e-10))
    for kind, n in ((0, 24), (1, 20)):
        m = I.square_mesh(n)
        gm = GpuMesh(m, ctx)
        nE, cls = gm.info["nE"], gm.tables["eclass"]
        t = dict(xy=dev(m.xy, torch.float64), tri=dev(m.tri, torch.int32), d=dev(m.dirichlet, torch.int32),
                 nn=dev(m.neumann, torch.int32))
        fm = torch.ones(nE, dtype=torch.float64, device="cuda")
        # edge classes: 1 Dirichlet, 2 Neumann
        bcm = dev(np.where(cls == 1, 0.2, np.where(cls == 2, 0.1, 0.0)), torch.float64)
        u0m = dev(np.where(cls == 1, 0.2, 0.0), torch.float64)
        outs = []
        for arrays in (False, True):
            U = torch.full((3 * m.nT,), np.nan, dtype=torch.float64, device="cuda")
            kw = dict(f_mid=fm, bc_mid=bcm, u0_mid=u0m if kind == 1 else None) if arrays else {}
            rq = P.make_request(t["xy"], t["tri"], t["d"], t["nn"], kind=kind, delta=0.5, f=1.0, uD=0.2, g=0.1,
                                dt=1.0 / n, u0=0.0, steps=8, precision=P.PHFEM_FP32_IR, U_out=U, **kw)
            r = P.phfem_server_poll(srv, P.phfem_server_submit(srv, rq), wait=True)
            assert r["status"] == 0 and r["rel_residual"] <= 1e-10, r
            outs.append((U.cpu().numpy(), r["iterations"]))
        assert np.array_equal(outs[0][0], outs[1][0]) and outs[0][1] == outs[1][1]
        gm.close()
    # non-constant data against the oracle
    m = I.lshape_mesh(n=10, seed=I.seed_for(1, 92))
    pb = I.problem_sine_exp()
    pb.delta = 1.0
    gm = GpuMesh(m, ctx)
    fm, bcm = gm.edge_data(pb.f, pb.g, pb.uD)
    U = torch.full((3 * m.nT,), np.nan, dtype=torch.float64, device="cuda")
    t = dict(xy=dev(m.xy, torch.float64), tri=dev(m.tri, torch.int32), d=dev(m.dirichlet, torch.int32),
             nn=dev(m.neumann, torch.int32))
    rq = P.make_request(t["xy"], t["tri"], t["d"], t["nn"], kind=0, delta=pb.delta, precision=P.PHFEM_FP64,
                        U_out=U, f_mid=fm, bc_mid=bcm)
    r = P.phfem_server_poll(srv, P.phfem_server_submit(srv, rq), wait=True)
    assert r["status"] == 0, r
    ref = O.solve_saddle(m, pb)
    assert np.max(np.abs(U.cpu().numpy() - ref["U"])) <= 1e-7 * np.max(np.abs(ref["U"]))
    gm.close()
    P.phfem_server_destroy(srv)
    P.phfem_ctx_destroy(ctx)


def test_memory_accounting_and_measured_admission():
    """The context counts its own allocations (back to where it was once the
    objects are destroyed); a served request records its peak, and the next
    request of the same class is reserved the measured bytes per triangle
    (+10 %, + 4 MB) instead of the static guess."""
    from paper_2401_15557_gb300 import phfem as P
    from phfem_gpu import GpuMesh
    dev = lambda a, t: torch.as_tensor(np.ascontiguousarray(a), dtype=t, device="cuda")
    ctx = P.phfem_ctx_create()
    now0, _ = P.phfem_ctx_memory(ctx, reset_peak=True)
    m = I.square_mesh(64)
    gm = GpuMesh(m, ctx)
    fm, bcm = gm.edge_data(lambda x, y: 1.0 + 0 * x, lambda x, y, nx, ny: 0 * x, lambda x, y: 0 * x)
    sysh = P.phfem_assemble(gm.h, fm, bcm, precision=P.PHFEM_FP32_IR)
    P.phfem_solve(sysh, P.solve_opts(rtol=1e-10))
    now1, peak1 = P.phfem_ctx_memory(ctx)
    assert now1 > now0 and peak1 >= now1
    P.phfem_sys_destroy(sysh)
    gm.close()
    now2, _ = P.phfem_ctx_memory(ctx)
    assert now2 == now0
    P.phfem_ctx_destroy(ctx)

    srv = P.phfem_server_create(1, 64e9, P.solve_opts(rtol=1e-10))
    res = []
    for n in (256, 200):  # 131,072 and 80,000 triangles: both learn
        mm = I.square_mesh(n)
        t = dict(xy=dev(mm.xy, torch.float64), tri=dev(mm.tri, torch.int32), d=dev(mm.dirichlet, torch.int32),
                 nn=dev(mm.neumann, torch.int32))
        rq = P.make_request(t["xy"], t["tri"], t["d"], t["nn"], kind=0, delta=0.5, f=1.0,
                            precision=P.PHFEM_FP32_IR)
        res.append((mm.nT, P.phfem_server_poll(srv, P.phfem_server_submit(srv, rq), wait=True)))
    P.phfem_server_destroy(srv)
    (n1, r1), (n2, r2) = res
    assert r1["status"] == 0 and r2["status"] == 0
    assert r1["bytes_peak"] > 0 and r2["bytes_peak"] > 0
    # stream priority by size: 131,072 triangles run in the middle class, 80,000 in the highest
    assert r1["priority_class"] == 1 and r2["priority_class"] == 0
    assert r1["bytes_reserved"] == pytest.approx(400.0 * n1 + 4 * 2 ** 20)  # nothing measured yet
    assert r2["bytes_reserved"] == pytest.approx(1.1 * r1["bytes_peak"] / n1 * n2 + 4 * 2 ** 20)
    assert r2["bytes_peak"] <= r2["bytes_reserved"]
