"""The allocation-free solve (phfem_csr_pcg_noalloc) against the regular solve.

Some callers of this library cannot allocate device memory while they call
it: programs whose device memory is owned by another framework's pool or a
fixed arena, and loops with a latency or memory budget, where cudaMalloc may
synchronise the device or fail part-way.  They use this entry point, whose
temporaries live in one fixed device array of the library.  These tests call
it through the C ABI and through the Python binding, check it against the
regular phfem_solve on the same system on two calls in a row, check that a
warm call changes the device's free memory by nothing, and check its errors.
The file is collected last, so that a run stopping at the first failure has
already run every other test; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from oracle import phfem_oracle as O
from paper_2401_15557_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def system():
    import torch
    from paper_2401_15557_gb300 import phfem as P
    from phfem_gpu import GpuMesh, solve

    ctx = P.phfem_ctx_create()
    mesh = I.lshape_mesh(n=10, seed=I.seed_for(1, 61), levels=1)
    aT = I.element_mean_at_midpoints(mesh.xy, mesh.tri, I.coeff_lshape)
    pb = I.problem_sine_exp()
    pb.delta = 0.5
    gm = GpuMesh(mesh, ctx)
    ref = solve(gm, pb, aT=aT, precision=P.PHFEM_FP64, rtol=1e-12)   # the regular entry point
    T = gm.tables
    nF = gm.info["nF"]
    assert nF <= P.NOALLOC_MAX_ROWS
    out = dict(nF=nF, rp=torch.as_tensor(T["row_ptr"], device="cuda"), col=torch.as_tensor(T["col"], device="cuda"),
               val=torch.as_tensor(ref["val"], device="cuda"), rhs=torch.as_tensor(ref["rhs"], device="cuda"),
               w_ref=ref["w"][T["free_id"] >= 0], ref=ref, T=T)
    yield out
    P.phfem_sys_destroy(ref["sys"])
    gm.close()
    P.phfem_ctx_destroy(ctx)


def _check_solution(s, xs):
    import scipy.sparse as sp
    S = sp.csr_matrix((s["ref"]["val"], s["T"]["col"], s["T"]["row_ptr"]), shape=(s["nF"], s["nF"]))
    # same tolerances as the other solve tests: residual and forward error
    assert O.relative_residual(S, s["ref"]["rhs"], xs) <= 1.2e-10
    assert np.max(np.abs(xs - s["w_ref"])) <= 1e-7 * np.max(np.abs(s["w_ref"]))


def test_noalloc_matches_regular_solve_twice(system):
    import torch
    from paper_2401_15557_gb300 import phfem as P

    s = system
    L = P.lib()
    for call in range(2):
        x = torch.zeros(s["nF"], dtype=torch.float64, device="cuda")
        it, rel = ctypes.c_int32(), ctypes.c_double()
        status = L.phfem_csr_pcg_noalloc(None, s["nF"], s["rp"].data_ptr(), s["col"].data_ptr(), s["val"].data_ptr(),
                                         s["rhs"].data_ptr(), x.data_ptr(), 1e-12, 0, ctypes.byref(it),
                                         ctypes.byref(rel))
        torch.cuda.synchronize()
        assert status == 0, (call, P.phfem_last_error())
        assert rel.value <= 1e-12 and it.value > 0
        _check_solution(s, x.cpu().numpy())
    # sizes beyond the fixed scratch are refused with a clear message
    big = P.NOALLOC_MAX_ROWS + 1
    status = L.phfem_csr_pcg_noalloc(None, big, s["rp"].data_ptr(), s["col"].data_ptr(), s["val"].data_ptr(),
                                     s["rhs"].data_ptr(), x.data_ptr(), 1e-10, 0, None, None)
    assert status == P.PHFEM_EINVAL and "exceed" in P.phfem_last_error()


def test_binding_call_leaves_free_memory_unchanged(system):
    import torch
    from paper_2401_15557_gb300 import phfem as P

    s = system
    x = torch.zeros(s["nF"], dtype=torch.float64, device="cuda")
    P.phfem_csr_pcg_noalloc(s["rp"], s["col"], s["val"], s["rhs"], x, rtol=1e-12)   # warm: kernels loaded
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    x.zero_()
    r = P.phfem_csr_pcg_noalloc(s["rp"], s["col"], s["val"], s["rhs"], x, rtol=1e-12)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    assert r["iterations"] > 0 and r["rel_residual"] <= 1e-12
    _check_solution(s, x.cpu().numpy())


def test_errors_missing_diagonal_and_iteration_limit(system):
    import torch
    from paper_2401_15557_gb300 import phfem as P

    s = system
    rp = s["T"]["row_ptr"]
    col = s["T"]["col"]
    row = s["nF"] // 2
    k = rp[row] + int(np.nonzero(col[rp[row]:rp[row + 1]] == row)[0][0])
    bad = s["val"].clone()
    bad[k] = 0.0
    x = torch.zeros(s["nF"], dtype=torch.float64, device="cuda")
    with pytest.raises(P.PhfemError) as e:
        P.phfem_csr_pcg_noalloc(s["rp"], s["col"], bad, s["rhs"], x)
    assert e.value.status == P.PHFEM_EINVAL and "diagonal" in str(e.value)
    x.zero_()
    with pytest.raises(P.PhfemError) as e:
        P.phfem_csr_pcg_noalloc(s["rp"], s["col"], s["val"], s["rhs"], x, rtol=1e-12, max_iter=1)
    assert e.value.status == P.PHFEM_ENOCONV
    # the shared scratch is usable again right after the failures
    x.zero_()
    P.phfem_csr_pcg_noalloc(s["rp"], s["col"], s["val"], s["rhs"], x, rtol=1e-12)
    torch.cuda.synchronize()
    _check_solution(s, x.cpu().numpy())
