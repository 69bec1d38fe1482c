// Uniform red refinement (Section 2.3, redrefine_vec) on the device.
//
// Everything is closed-form from the coarse mesh's tables: new vertex nV + e
// sits at the midpoint of edge e, the children of triangle t reference its
// vertices and the new vertices of its edges t2e[t][k], and a listed boundary
// pair splits at the new vertex of its edge (recorded by phfem_mesh_build).
// The refined tables are then built by phfem_mesh_build.
#include "internal.cuh"

namespace phfem {
namespace {

__global__ void k_refine_xy(int nV, int nE, const double2* __restrict__ xy, const int32_t* __restrict__ ed2el,
                            double2* __restrict__ out) {
  const int n = nV + nE;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (i < nV) {
      out[i] = xy[i];
    } else {
      const int e = i - nV;
      const double2 a = xy[ed2el[4 * e]], b = xy[ed2el[4 * e + 1]];
      out[i] = make_double2((a.x + b.x) / 2, (a.y + b.y) / 2);
    }
  }
}

__global__ void k_refine_tri(int nT, int nV, const int32_t* __restrict__ tri, const int32_t* __restrict__ t2e,
                             int32_t* __restrict__ out) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nT; t += gridDim.x * blockDim.x) {
    const int P1 = tri[3 * t], P2 = tri[3 * t + 1], P3 = tri[3 * t + 2];
    const int M1 = nV + t2e[3 * t], M2 = nV + t2e[3 * t + 1], M3 = nV + t2e[3 * t + 2];
    int32_t* mid = out + 3 * (size_t)t;
    mid[0] = M1;
    mid[1] = M2;
    mid[2] = M3;
    int32_t* c = out + 3 * ((size_t)nT + 3 * (size_t)t);
    c[0] = P1;
    c[1] = M3;
    c[2] = M2;
    c[3] = P2;
    c[4] = M1;
    c[5] = M3;
    c[6] = P3;
    c[7] = M2;
    c[8] = M1;
  }
}

__global__ void k_refine_pairs(int nB, int nV, const int32_t* __restrict__ pairs, const int32_t* __restrict__ bedge,
                               int32_t* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nB; i += gridDim.x * blockDim.x) {
    const int a = pairs[2 * i], b = pairs[2 * i + 1], m = nV + bedge[i];
    out[2 * i] = a;
    out[2 * i + 1] = m;
    out[2 * ((size_t)nB + i)] = m;
    out[2 * ((size_t)nB + i) + 1] = b;
  }
}

}  // namespace
}  // namespace phfem

using namespace phfem;

extern "C" {

PHFEM_API int phfem_mesh_refine(phfem_mesh coarse, double* xy, int32_t* tri, int32_t* dirichlet, int32_t* neumann,
                                phfem_mesh* fine) {
  if (fine) *fine = nullptr;
  if (!coarse) return fail(PHFEM_EINVAL, "phfem_mesh_refine: NULL mesh");
  if (!fine && (!xy || !tri)) return fail(PHFEM_EINVAL, "phfem_mesh_refine: xy and tri are needed without a fine mesh");
  const phfem_mesh_info I = coarse->info;
  const int64_t nV2 = (int64_t)I.nV + I.nE, nT2 = 4 * (int64_t)I.nT;
  const int64_t nD2 = 2 * (int64_t)I.nD, nN2 = 2 * (int64_t)I.nN;
  if (nV2 > INT32_MAX || 3 * nT2 > INT32_MAX || 2 * nD2 > INT32_MAX || 2 * nN2 > INT32_MAX)
    return fail(PHFEM_EINVAL, "phfem_mesh_refine: the refined mesh exceeds the int32 index range");
  phfem_ctx ctx = coarse->ctx;
  cudaStream_t s = ctx->stream;
  double* txy = nullptr;
  int32_t *ttri = nullptr, *tdir = nullptr, *tneu = nullptr;
  int st = PHFEM_OK;
  if (!xy) {
    st = dalloc_n(ctx, &txy, 2 * (size_t)nV2);
    xy = txy;
  }
  if (st == PHFEM_OK && !tri) {
    st = dalloc_n(ctx, &ttri, 3 * (size_t)nT2);
    tri = ttri;
  }
  if (st == PHFEM_OK && !dirichlet && nD2 > 0) {
    st = dalloc_n(ctx, &tdir, 2 * (size_t)nD2);
    dirichlet = tdir;
  }
  if (st == PHFEM_OK && !neumann && nN2 > 0) {
    st = dalloc_n(ctx, &tneu, 2 * (size_t)nN2);
    neumann = tneu;
  }
  if (st == PHFEM_OK) {
    k_refine_xy<<<grid_for(ctx, nV2), kBlock, 0, s>>>(I.nV, I.nE, reinterpret_cast<const double2*>(coarse->xy),
                                                      coarse->ed2el, reinterpret_cast<double2*>(xy));
    st = check_launch(ctx, "k_refine_xy");
  }
  if (st == PHFEM_OK && I.nT > 0) {
    k_refine_tri<<<grid_for(ctx, I.nT), kBlock, 0, s>>>(I.nT, I.nV, coarse->tri, coarse->t2e, tri);
    st = check_launch(ctx, "k_refine_tri");
  }
  if (st == PHFEM_OK && I.nD > 0) {
    k_refine_pairs<<<grid_for(ctx, I.nD), kBlock, 0, s>>>(I.nD, I.nV, coarse->bpairs, coarse->bedge, dirichlet);
    st = check_launch(ctx, "k_refine_pairs");
  }
  if (st == PHFEM_OK && I.nN > 0) {
    k_refine_pairs<<<grid_for(ctx, I.nN), kBlock, 0, s>>>(I.nN, I.nV, coarse->bpairs + 2 * (size_t)I.nD,
                                                           coarse->bedge + I.nD, neumann);
    st = check_launch(ctx, "k_refine_pairs");
  }
  if (st == PHFEM_OK && fine)
    st = phfem_mesh_build(ctx, (int32_t)nV2, xy, (int32_t)nT2, tri, (int32_t)nD2, nD2 ? dirichlet : nullptr,
                          (int32_t)nN2, nN2 ? neumann : nullptr, fine);
  dfree(ctx, txy);
  dfree(ctx, ttri);
  dfree(ctx, tdir);
  dfree(ctx, tneu);
  return st;
}

}  // extern "C"
