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


def _scaled(m, sx, sy):
    """The mesh with its coordinates scaled by (sx, sy)."""
    import dataclasses
    return dataclasses.replace(m, xy=np.ascontiguousarray(m.xy * np.array([sx, sy])))


# stretched8: triangles (ll, lr, ur) have a 2.9-degree angle at P0, so FP32 systems take
# the FP64 element records for them (and compensated FP32 for the others); tiny6: edges
# below 2^-40, every triangle takes the FP64 records.  tiny6 solves a linear u of size
# one here; the sine data on it (u ~ 1e-13) are solved in test_gpu_order.py, where the
# scaling of the FP32 inner vectors keeps them in range.
SINE, LINEAR = I.problem_sine_exp, I.problem_linear
CASES = [
    ("square17", lambda: I.square_mesh(17), 0.0, False, SINE),
    ("stretched8", lambda: _scaled(I.square_mesh(8), 1.0, 1.0 / 20.0), 0.5, False, SINE),
    ("tiny6", lambda: _scaled(I.square_mesh(6), 2.0 ** -45, 2.0 ** -45), 1.0, False, LINEAR),
    ("lshape6", lambda: I.lshape_mesh(n=6, seed=I.seed_for(1, 21)), 0.7, True, SINE),
    ("lshape5r1", lambda: I.lshape_mesh(n=5, seed=I.seed_for(1, 22), levels=1), 1.0, True, SINE),
    ("crisscross3", lambda: I.criss_cross(3), 0.3, True, SINE),
    ("two", lambda: I.square_mesh(1), 0.0, False, SINE),
]


@pytest.mark.parametrize("name,mk,delta,var,problem", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32ir"])
def test_assembled_values(ctx, name, mk, delta, var, problem, precision):
    from phfem_gpu import GpuMesh, solve
    mesh = mk()
    pb = problem()
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
