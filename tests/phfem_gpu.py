"""Helpers of the GPU tests: run a mesh/problem through the C ABI."""
import numpy as np
import torch

from paper_2401_15557_gb300 import inputs as I
from paper_2401_15557_gb300 import phfem as P


def dev(a, dtype):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


class GpuMesh:
    def __init__(self, mesh, ctx):
        self.mesh = mesh
        self.ctx = ctx
        self.xy = dev(mesh.xy, torch.float64)
        self.h = P.phfem_mesh_build(ctx, self.xy, dev(mesh.tri, torch.int32),
                                    dev(mesh.dirichlet, torch.int32) if len(mesh.dirichlet) else None,
                                    dev(mesh.neumann, torch.int32) if len(mesh.neumann) else None)
        self.info = P.phfem_mesh_info_get(self.h)
        self.tables = {k: v.cpu().numpy() for k, v in P.phfem_mesh_tables(self.h).items()}

    def edge_data(self, f, g=None, uD=None, t=None):
        fm, bc = I.edge_data(self.mesh.xy, self.tables["ed2el"], self.tables["eclass"], f, g, uD, t)
        return dev(fm, torch.float64), dev(bc, torch.float64)

    def close(self):
        P.phfem_mesh_destroy(self.h)


def solve(gm, problem, aT=None, precision=P.PHFEM_FP64, rtol=1e-10, inner_rtol=0.0, w0=None):
    fm, bc = gm.edge_data(problem.f, problem.g, problem.uD)
    I_ = gm.info
    sysh = P.phfem_assemble(gm.h, fm, bc, a_T=None if aT is None else dev(aT, torch.float64),
                            delta=problem.delta, precision=precision)
    w = torch.empty(I_["nE"], dtype=torch.float64, device="cuda")
    U = torch.empty(3 * I_["nT"], dtype=torch.float64, device="cuda")
    Lam = torch.empty(max(I_["nL"], 1), dtype=torch.float64, device="cuda")
    st = P.phfem_solve(sysh, P.solve_opts(rtol=rtol, inner_rtol=inner_rtol), w0=w0, w=w, U=U, Lambda=Lam)
    val = torch.empty(max(I_["nnz"], 1), dtype=torch.float64, device="cuda")
    rhs = torch.empty(max(I_["nF"], 1), dtype=torch.float64, device="cuda")
    P.phfem_sys_csr(sysh, val, rhs)
    torch.cuda.synchronize()
    out = dict(w=w.cpu().numpy(), U=U.cpu().numpy(), Lambda=Lam.cpu().numpy()[:I_["nL"]], stats=st,
               val=val.cpu().numpy()[:I_["nnz"]], rhs=rhs.cpu().numpy()[:I_["nF"]], sys=sysh)
    return out
