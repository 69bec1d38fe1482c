"""The allocation-free solve (phfem_csr_pcg_noalloc) against the regular solve.

Callers that cannot allocate device memory during a call (graph capture,
memory owned by another framework, allocation-free loops) use the entry point
with the library's fixed device scratch.  This file is collected last so that
a run stopping at the first failure has already run every other test; it also
passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from oracle import phfem_oracle as O
from paper_2401_15557_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_noalloc_matches_regular_solve_twice():
    import scipy.sparse as sp
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
    rp = torch.as_tensor(T["row_ptr"], device="cuda")
    col = torch.as_tensor(T["col"], device="cuda")
    val = torch.as_tensor(ref["val"], device="cuda")
    rhs = torch.as_tensor(ref["rhs"], device="cuda")
    w_ref = ref["w"][T["free_id"] >= 0]
    S = sp.csr_matrix((ref["val"], T["col"], T["row_ptr"]), shape=(nF, nF))
    L = P.lib()
    for call in range(2):
        x = torch.zeros(nF, dtype=torch.float64, device="cuda")
        it, rel = ctypes.c_int32(), ctypes.c_double()
        status = L.phfem_csr_pcg_noalloc(None, nF, rp.data_ptr(), col.data_ptr(), val.data_ptr(), rhs.data_ptr(),
                                         x.data_ptr(), 1e-12, 0, ctypes.byref(it), ctypes.byref(rel))
        torch.cuda.synchronize()
        assert status == 0, (call, P.phfem_last_error())
        xs = x.cpu().numpy()
        assert rel.value <= 1e-12 and it.value > 0
        # same tolerance as the other solve tests: residual and forward error
        assert O.relative_residual(S, ref["rhs"], xs) <= 1.2e-10
        assert np.max(np.abs(xs - w_ref)) <= 1e-7 * np.max(np.abs(w_ref)), call
    # sizes beyond the fixed scratch are refused with a clear message
    big = P.NOALLOC_MAX_ROWS + 1
    status = L.phfem_csr_pcg_noalloc(None, big, rp.data_ptr(), col.data_ptr(), val.data_ptr(), rhs.data_ptr(),
                                     x.data_ptr(), 1e-10, 0, None, None)
    assert status == -1 and "exceed" in P.phfem_last_error()
    gm.close()
    P.phfem_ctx_destroy(ctx)
