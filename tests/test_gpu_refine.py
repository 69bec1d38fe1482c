"""Red refinement on the GPU: refined coordinates, elements and boundary lists
bit-exact against the oracle's refinement, over several levels, and the
refined mesh's tables bit-exact against the oracle's topology."""
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


MESHES = {
    "crisscross0": lambda: I.criss_cross_level0(),
    "lshape": lambda: I.lshape_mesh(n=5, seed=I.seed_for(1, 21)),
    "square_alldirichlet": lambda: I.square_mesh(3, dirichlet_sides=("left", "right", "top", "bottom")),
    "square_allneumann": lambda: I.square_mesh(4, dirichlet_sides=()),
}


@pytest.mark.parametrize("name", list(MESHES))
def test_refinement_matches_oracle(ctx, name):
    from phfem_gpu import GpuMesh
    from paper_2401_15557_gb300 import phfem as P
    m = MESHES[name]()
    gm = GpuMesh(m, ctx)
    h = gm.h
    xy, tri, d, n = m.xy, m.tri, m.dirichlet, m.neumann
    for level in range(3):
        fine, arr = P.phfem_mesh_refine(h, build=True, arrays=True)
        xy, tri, d, n = O.redrefine(xy, tri, d, n)
        assert np.array_equal(arr["xy"].cpu().numpy(), xy)  # (a + b) / 2 is exact the same way
        assert np.array_equal(arr["tri"].cpu().numpy(), tri)
        assert np.array_equal(arr["dirichlet"].cpu().numpy().reshape(-1, 2), d.reshape(-1, 2))
        assert np.array_equal(arr["neumann"].cpu().numpy().reshape(-1, 2), n.reshape(-1, 2))
        topo = O.edge_tables(tri, xy.shape[0])
        tabs = {k: v.cpu().numpy() for k, v in P.phfem_mesh_tables(fine).items()}
        assert np.array_equal(tabs["ed2el"], topo["ed2el"])
        assert np.array_equal(tabs["t2e"], topo["t2e"])
        if h is not gm.h:
            P.phfem_mesh_destroy(h)
        h = fine
    P.phfem_mesh_destroy(h)
    gm.close()


def test_refined_solve_matches_oracle(ctx):
    """A solve on a device-refined mesh equals the oracle's saddle solve on the
    oracle-refined mesh."""
    from phfem_gpu import GpuMesh, dev
    from paper_2401_15557_gb300 import phfem as P
    m = I.lshape_mesh(n=4, seed=I.seed_for(1, 23))
    gm = GpuMesh(m, ctx)
    fine, arr = P.phfem_mesh_refine(gm.h, build=True, arrays=True)
    xy, tri, d, n = O.redrefine(m.xy, m.tri, m.dirichlet, m.neumann)
    mf = I.Mesh(xy=xy, tri=tri.astype(np.int32), dirichlet=d.astype(np.int32), neumann=n.astype(np.int32),
                name="refined")
    pb = I.problem_sine_exp()
    pb.delta = 1.0
    tabs = {k: v.cpu().numpy() for k, v in P.phfem_mesh_tables(fine).items()}
    fm, bc = I.edge_data(xy, tabs["ed2el"], tabs["eclass"], pb.f, pb.g, pb.uD)
    sysh = P.phfem_assemble(fine, dev(fm, torch.float64), dev(bc, torch.float64), delta=pb.delta)
    info = P.phfem_mesh_info_get(fine)
    U = torch.empty(3 * info["nT"], dtype=torch.float64, device="cuda")
    st = P.phfem_solve(sysh, P.solve_opts(rtol=1e-12), U=U)
    ref = O.solve_saddle(mf, pb)
    assert st["converged"] >= 1
    assert np.max(np.abs(U.cpu().numpy() - ref["U"])) <= 1e-9 * np.max(np.abs(ref["U"]))
    P.phfem_sys_destroy(sysh)
    P.phfem_mesh_destroy(fine)
    gm.close()


def test_arrays_only_and_rejections(ctx):
    from phfem_gpu import GpuMesh
    from paper_2401_15557_gb300 import phfem as P
    m = I.square_mesh(2)
    gm = GpuMesh(m, ctx)
    arr = P.phfem_mesh_refine(gm.h, build=False, arrays=True)
    xy, tri, _, _ = O.redrefine(m.xy, m.tri, m.dirichlet, m.neumann)
    assert np.array_equal(arr["tri"].cpu().numpy(), tri)
    with pytest.raises(P.PhfemError) as ei:
        P.phfem_mesh_refine(gm.h, build=False, arrays=False)  # nothing to write to
    assert ei.value.status == P.PHFEM_EINVAL
    gm.close()


@pytest.mark.parametrize("name", list(MESHES))
def test_closed_form_tables_equal_the_sorted_build(ctx, name):
    """The refined mesh's tables derived from the coarse ones equal, array by
    array, those of phfem_mesh_build on the refined arrays (three levels)."""
    from phfem_gpu import GpuMesh
    from paper_2401_15557_gb300 import phfem as P
    gm = GpuMesh(MESHES[name](), ctx)
    h = gm.h
    for level in range(3):
        fine, arr = P.phfem_mesh_refine(h, build=True, arrays=True)
        ref = P.phfem_mesh_build(ctx, arr["xy"], arr["tri"], arr["dirichlet"] if arr["dirichlet"].numel() else None,
                                 arr["neumann"] if arr["neumann"].numel() else None)
        a = {k: v.cpu().numpy() for k, v in P.phfem_mesh_tables(fine).items()}
        b = {k: v.cpu().numpy() for k, v in P.phfem_mesh_tables(ref).items()}
        assert P.phfem_mesh_info_get(fine) == P.phfem_mesh_info_get(ref)
        for k in b:
            assert np.array_equal(a[k], b[k]), (name, level, k)
        P.phfem_mesh_destroy(ref)
        if h is not gm.h:
            P.phfem_mesh_destroy(h)
        h = fine
    P.phfem_mesh_destroy(h)
    gm.close()
