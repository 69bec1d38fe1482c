"""Assembled values of the CUDA path against the oracle's condensed system
(FP64, within 1e-12 of the row scale)."""
import numpy as np
import pytest

from oracle import phfem_oracle as O
from paper_2401_15557_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2401_15557_gb300 import phfem as P
    c = P.phfem_ctx_create()
    yield c
    P.phfem_ctx_destroy(c)


def _rowscaled_err(row_ptr, val_a, val_b):
    err = 0.0
    for r in range(row_ptr.size - 1):
        s, e = row_ptr[r], row_ptr[r + 1]
        scale = np.max(np.abs(val_b[s:e]))
        err = max(err, np.max(np.abs(val_a[s:e] - val_b[s:e])) / scale)
    return err


CASES = [
    ("square17", lambda: I.square_mesh(17), 0.0, False),
    ("lshape6", lambda: I.lshape_mesh(n=6, seed=I.seed_for(1, 21)), 0.7, True),
    ("lshape5r1", lambda: I.lshape_mesh(n=5, seed=I.seed_for(1, 22), levels=1), 1.0, True),
    ("crisscross3", lambda: I.criss_cross(3), 0.3, True),
    ("two", lambda: I.square_mesh(1), 0.0, False),
]


@pytest.mark.parametrize("name,mk,delta,var", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32ir"])
def test_assembled_values(ctx, name, mk, delta, var, precision):
    from phfem_gpu import GpuMesh, solve
    mesh = mk()
    pb = I.problem_sine_exp()
    pb.delta = delta
    aT = I.element_mean_at_midpoints(mesh.xy, mesh.tri, I.coeff_lshape) if var else None
    cs = O.condensed_system(mesh, pb, aT=aT)
    gm = GpuMesh(mesh, ctx)
    out = solve(gm, pb, aT=aT, precision=precision)
    assert np.array_equal(gm.tables["row_ptr"], cs["row_ptr"])
    assert _rowscaled_err(cs["row_ptr"], out["val"], cs["val"]) <= 1e-12
    scale = np.max(np.abs(cs["rhs"]))
    assert np.max(np.abs(out["rhs"] - cs["rhs"])) <= 1e-12 * scale
    # symmetric pattern and values
    import scipy.sparse as sp
    S = sp.csr_matrix((out["val"], cs["col"], cs["row_ptr"]), shape=(cs["rhs"].size,) * 2)
    assert abs(S - S.T).max() <= 1e-14 * abs(S).max()
    gm.close()
