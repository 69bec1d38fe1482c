"""Mesh tables of the CUDA path against the oracle: bit-exact integers."""
import numpy as np
import pytest

from oracle import phfem_oracle as O
from paper_2401_15557_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _meshes():
    yield I.criss_cross_level0()
    yield I.square_mesh(1)
    yield I.square_mesh(7)
    yield I.criss_cross(3)
    yield I.lshape_mesh(n=6, seed=I.seed_for(1, 11))
    yield I.lshape_mesh(n=5, seed=I.seed_for(1, 12), levels=1)
    yield I.square_mesh(64, dirichlet_sides=("left", "bottom", "top"))


@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_2401_15557_gb300 import phfem as P
    torch.cuda.init()
    c = P.phfem_ctx_create()
    yield c
    P.phfem_ctx_destroy(c)


@pytest.mark.parametrize("mesh", list(_meshes()), ids=lambda m: f"{m.name}-{m.nT}")
def test_tables_bit_exact(ctx, mesh):
    from phfem_gpu import GpuMesh
    gm = GpuMesh(mesh, ctx)
    T = gm.tables
    topo = O.edge_tables(mesh.tri, mesh.nV)
    bs = O.boundary_sets(topo, mesh.dirichlet, mesh.neumann)
    cs = O.condensed_system(mesh, I.problem_sine_exp())
    assert gm.info["nE"] == topo["nE"]
    assert np.array_equal(T["ed2el"], topo["ed2el"])
    assert np.array_equal(T["t2e"], topo["t2e"])
    assert np.array_equal(T["sigma"], topo["sigma"])
    assert np.array_equal(T["eclass"], bs["eclass"])
    assert np.array_equal(T["free_id"], bs["free_id"])
    assert np.array_equal(T["lam_id"], bs["lam_id"])
    assert gm.info["nF"] == bs["free"].size and gm.info["nL"] == bs["Redges"].size
    assert np.array_equal(T["row_ptr"], cs["row_ptr"])
    assert np.array_equal(T["col"], cs["col"])
    gm.close()


def test_high_valence_vertex(ctx):
    """A fan of 10,000 triangles around one vertex (valence 10,000, the larger
    vertex of all its spokes): tables bit-exact against the oracle, and the
    build takes no longer per triangle than on a regular mesh of about the
    same size (up to 2x)."""
    import time
    import torch
    from paper_2401_15557_gb300 import phfem as P
    from phfem_gpu import GpuMesh, dev
    fan = I.fan_mesh(10000)
    gm = GpuMesh(fan, ctx)
    topo = O.edge_tables(fan.tri, fan.nV)
    assert gm.info["nE"] == topo["nE"] == 20000
    assert np.array_equal(gm.tables["ed2el"], topo["ed2el"])
    assert np.array_equal(gm.tables["t2e"], topo["t2e"])
    assert np.array_equal(gm.tables["sigma"], topo["sigma"])
    gm.close()

    def build_ms(mesh):
        args = (dev(mesh.xy, torch.float64), dev(mesh.tri, torch.int32), dev(mesh.dirichlet, torch.int32),
                dev(mesh.neumann, torch.int32) if len(mesh.neumann) else None)
        P.phfem_mesh_destroy(P.phfem_mesh_build(ctx, *args))  # warm
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(5):
            P.phfem_mesh_destroy(P.phfem_mesh_build(ctx, *args))
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / 5 * 1e3 / mesh.nT

    square = I.square_mesh(71)  # 10,082 triangles
    assert build_ms(fan) <= 2.0 * build_ms(square)


def _expect_emesh(ctx, mesh):
    from paper_2401_15557_gb300 import phfem as P
    from phfem_gpu import GpuMesh
    with pytest.raises(P.PhfemError) as ei:
        GpuMesh(mesh, ctx)
    assert ei.value.status == -2, str(ei.value)


def test_invalid_meshes_rejected(ctx):
    base = I.square_mesh(4)
    cw = I.Mesh(base.xy, base.tri.copy(), base.dirichlet, base.neumann)
    cw.tri[3] = cw.tri[3, [0, 2, 1]]
    _expect_emesh(ctx, cw)
    unlisted = I.Mesh(base.xy, base.tri, base.dirichlet, base.neumann[1:])
    _expect_emesh(ctx, unlisted)
    twice = I.Mesh(base.xy, base.tri, np.vstack([base.dirichlet, base.dirichlet[:1]]), base.neumann)
    _expect_emesh(ctx, twice)
    both = I.Mesh(base.xy, base.tri, base.dirichlet, np.vstack([base.neumann, base.dirichlet[:1]]))
    _expect_emesh(ctx, both)
    interior = I.Mesh(base.xy, base.tri, np.vstack([base.dirichlet, base.tri[5, :2][None]]), base.neumann)
    _expect_emesh(ctx, interior)
    bad = I.Mesh(base.xy, base.tri.copy(), base.dirichlet, base.neumann)
    bad.tri[0, 0] = base.nV + 3
    _expect_emesh(ctx, bad)
    dup = I.Mesh(base.xy, np.vstack([base.tri, base.tri[:1]]), base.dirichlet, base.neumann)
    _expect_emesh(ctx, dup)


def test_full_size_lshape_tables_properties(ctx):
    """6.3M triangles (the L-shaped workload's finest level): properties that
    hold at any size, checked on the device."""
    import torch
    from phfem_gpu import GpuMesh
    mesh = I.lshape_mesh(levels=5)
    gm = GpuMesh(mesh, ctx)
    dev = "cuda"
    tri = torch.as_tensor(mesh.tri, device=dev).long()
    ed = torch.as_tensor(gm.tables["ed2el"], device=dev).long()
    t2e = torch.as_tensor(gm.tables["t2e"], device=dev).long()
    sig = torch.as_tensor(gm.tables["sigma"], device=dev).long()
    nV, nT, nE = mesh.nV, mesh.nT, gm.info["nE"]
    assert nV - nE + nT == 1
    lo = torch.minimum(ed[:, 0], ed[:, 1])
    hi = torch.maximum(ed[:, 0], ed[:, 1])
    key = hi * nV + lo
    assert bool((key[1:] > key[:-1]).all())
    # (initial, end) is the directed edge P_{k+1} -> P_{k+2} of T+ at the local index of t2e
    ar = torch.arange(nT, device=dev)
    for k in range(3):
        e = t2e[:, k]
        a, b = tri[:, (k + 1) % 3], tri[:, (k + 2) % 3]
        plus = sig[:, k] > 0
        assert bool((ed[e[plus], 2] == ar[plus]).all())
        assert bool((ed[e[plus], 0] == a[plus]).all()) and bool((ed[e[plus], 1] == b[plus]).all())
        assert bool((ed[e[~plus], 3] == ar[~plus]).all())
        assert bool((ed[e[~plus], 0] == b[~plus]).all()) and bool((ed[e[~plus], 1] == a[~plus]).all())
    inter = ed[:, 3] >= 0
    assert bool((ed[inter, 2] < ed[inter, 3]).all())
    assert int((~inter).sum()) == len(mesh.dirichlet) + len(mesh.neumann)
    # CSR rows: sorted, diagonal present, length 1 + free neighbours
    rp = torch.as_tensor(gm.tables["row_ptr"], device=dev).long()
    col = torch.as_tensor(gm.tables["col"], device=dev).long()
    lens = rp[1:] - rp[:-1]
    assert int(lens.min()) >= 1 and int(lens.max()) <= 5
    rows = torch.repeat_interleave(torch.arange(lens.numel(), device=dev), lens)
    same_row = rows[1:] == rows[:-1]
    assert bool((col[1:][same_row] > col[:-1][same_row]).all())
    assert int((col == rows).sum()) == lens.numel()
    gm.close()
