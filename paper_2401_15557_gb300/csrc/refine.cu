// Uniform red refinement (Section 2.3, redrefine_vec) on the device.
//
// Everything is closed-form from the coarse mesh's tables: new vertex nV + e
// sits at the midpoint of edge e, the children of triangle t reference its
// vertices and the new vertices of its edges t2e[t][k], and a listed boundary
// pair splits at the new vertex of its edge (recorded by phfem_mesh_build).
// The refined tables (edge numbering, T+/T-, directions, classes) follow from
// the coarse ones as well, with one scan and no sort.
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

// ---- refined tables in closed form ------------------------------------------
// Every fine edge has a midpoint for its larger vertex, so in the edge numbering
// (by larger, then smaller vertex) the fine edges come grouped by coarse edge E
// (larger vertex nV + E): first its two halves (smaller vertex: the coarse
// ends, in increasing order), then the middle-child edges joining M_E to the
// midpoint of a smaller neighbouring edge E' (in increasing E').  T+ of a half
// is the corner child, at that end, of the coarse T+; T+ of a middle-child
// edge is the middle child (it precedes every corner child).

__device__ __forceinline__ int nbr_edges(const int32_t* t2e, int t, int k, int out[2]) {
  out[0] = t2e[3 * t + (k + 1) % 3];
  out[1] = t2e[3 * t + (k + 2) % 3];
  return 2;
}

__global__ void k_ref_group(int nEc, const int32_t* __restrict__ ed2el, const uint8_t* __restrict__ lk,
                            const int32_t* __restrict__ t2e, int32_t* __restrict__ gsize) {
  for (int E = blockIdx.x * blockDim.x + threadIdx.x; E < nEc; E += gridDim.x * blockDim.x) {
    const int tp = ed2el[4 * E + 2], tm = ed2el[4 * E + 3];
    int n[2], c = 0;
    nbr_edges(t2e, tp, lk[E] & 3, n);
    c += (n[0] < E) + (n[1] < E);
    if (tm >= 0) {
      nbr_edges(t2e, tm, (lk[E] >> 2) & 3, n);
      c += (n[0] < E) + (n[1] < E);
    }
    gsize[E] = 2 + c;
  }
}

__device__ __forceinline__ int local_of(const int32_t* tri, int t, int v) {
  return tri[3 * t] == v ? 0 : (tri[3 * t + 1] == v ? 1 : 2);
}

__global__ void k_ref_edges(int nVc, int nTc, int nEc, const int32_t* __restrict__ tri, const int32_t* __restrict__ ed2el,
                            const uint8_t* __restrict__ lk, const int32_t* __restrict__ t2e,
                            const uint8_t* __restrict__ eclass, const int32_t* __restrict__ base,
                            int32_t* __restrict__ ed2el_f, uint8_t* __restrict__ lk_f, uint8_t* __restrict__ eclass_f,
                            int32_t* __restrict__ half_at, int32_t* __restrict__ g_id) {
  for (int E = blockIdx.x * blockDim.x + threadIdx.x; E < nEc; E += gridDim.x * blockDim.x) {
    const int I = ed2el[4 * E], J = ed2el[4 * E + 1], tp = ed2el[4 * E + 2], tm = ed2el[4 * E + 3];
    const int kp = lk[E] & 3, km = (lk[E] >> 2) & 3;
    const int b0 = base[E], mid = nVc + E;
    // the two halves, the one at the smaller coarse vertex first
    for (int h = 0; h < 2; ++h) {
      const int v = h == 0 ? I : J;
      const int f = b0 + ((v == I) == (I < J) ? 0 : 1);
      half_at[2 * E + h] = f;
      const int jp = local_of(tri, tp, v);
      const bool to_mid = kp == (jp + 2) % 3;  // E = E_{j+2}: P_j -> M in the corner child
      int4 row;
      row.x = to_mid ? v : mid;
      row.y = to_mid ? mid : v;
      row.z = nTc + 3 * tp + jp;
      int lkp = to_mid ? 2 : 1, lkm = 0;
      if (tm >= 0) {
        const int jm = local_of(tri, tm, v);
        row.w = nTc + 3 * tm + jm;
        lkm = km == (jm + 2) % 3 ? 2 : 1;
      } else {
        row.w = -1;
      }
      reinterpret_cast<int4*>(ed2el_f)[f] = row;
      lk_f[f] = (uint8_t)(lkp | (lkm << 2));
      eclass_f[f] = eclass[E];
    }
    // middle-child edges from M_E to the midpoints of smaller neighbours
    int nb[4], nt[4], nk[4], cnt = 0;
    {
      int n2[2];
      nbr_edges(t2e, tp, kp, n2);
      for (int q = 0; q < 2; ++q) {
        if (n2[q] < E) {
          nb[cnt] = n2[q];
          nt[cnt] = tp;
          nk[cnt] = 3 - kp - (q == 0 ? (kp + 1) % 3 : (kp + 2) % 3);  // the third edge of tp
          ++cnt;
        }
      }
      if (tm >= 0) {
        nbr_edges(t2e, tm, km, n2);
        for (int q = 0; q < 2; ++q) {
          if (n2[q] < E) {
            nb[cnt] = n2[q];
            nt[cnt] = tm;
            nk[cnt] = 3 - km - (q == 0 ? (km + 1) % 3 : (km + 2) % 3);
            ++cnt;
          }
        }
      }
    }
    for (int a = 0; a < cnt; ++a) {
      int rank = 0;
      for (int b = 0; b < cnt; ++b) rank += nb[b] < nb[a];
      const int f = b0 + 2 + rank;
      const int t = nt[a], k3 = nk[a];
      int4 row;
      row.x = nVc + t2e[3 * t + (k3 + 1) % 3];
      row.y = nVc + t2e[3 * t + (k3 + 2) % 3];
      row.z = t;
      row.w = nTc + 3 * t + k3;
      reinterpret_cast<int4*>(ed2el_f)[f] = row;
      lk_f[f] = (uint8_t)k3;  // edge k3 of the middle child, edge 0 of the corner child
      eclass_f[f] = PHFEM_EDGE_INTERIOR;
      g_id[3 * t + k3] = f;
    }
  }
}

__global__ void k_ref_t2e(int nTc, const int32_t* __restrict__ tri, const int32_t* __restrict__ ed2el,
                          const int32_t* __restrict__ t2e, const int32_t* __restrict__ half_at,
                          const int32_t* __restrict__ g_id, int32_t* __restrict__ t2e_f, int8_t* __restrict__ sigma_f) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nTc; t += gridDim.x * blockDim.x) {
    for (int k = 0; k < 3; ++k) {
      t2e_f[3 * t + k] = g_id[3 * t + k];
      sigma_f[3 * t + k] = 1;
    }
    for (int j = 0; j < 3; ++j) {
      const size_t c = (size_t)nTc + 3 * (size_t)t + j;
      const int Pj = tri[3 * t + j];
      t2e_f[3 * c] = g_id[3 * t + j];
      sigma_f[3 * c] = -1;
      for (int q = 1; q <= 2; ++q) {  // local edge q: the half of E_{j+q} next to P_j
        const int E = t2e[3 * t + (j + q) % 3];
        const int f = half_at[2 * E + (ed2el[4 * E] == Pj ? 0 : 1)];
        t2e_f[3 * c + q] = f;
        sigma_f[3 * c + q] = ed2el[4 * E + 2] == t ? 1 : -1;
      }
    }
  }
}

// Edge ids of the refined boundary lists: (a, m) is the half at a, (m, b) the half at b.
__global__ void k_ref_bedge(int nB, const int32_t* __restrict__ pairs, const int32_t* __restrict__ bedge,
                            const int32_t* __restrict__ ed2el, const int32_t* __restrict__ half_at,
                            int32_t* __restrict__ bedge_f) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nB; i += gridDim.x * blockDim.x) {
    const int E = bedge[i], a = pairs[2 * i], b = pairs[2 * i + 1];
    bedge_f[i] = half_at[2 * E + (ed2el[4 * E] == a ? 0 : 1)];
    bedge_f[nB + i] = half_at[2 * E + (ed2el[4 * E] == b ? 0 : 1)];
  }
}

// The refined mesh, tables derived from the coarse ones (no sort).
int refine_tables(phfem_mesh c, phfem_mesh* out) {
  phfem_ctx ctx = c->ctx;
  cudaStream_t s = ctx->stream;
  const phfem_mesh_info I = c->info;
  phfem_mesh m = new phfem_mesh_s();
  m->ctx = ctx;
  m->info.nV = I.nV + I.nE;
  m->info.nT = 4 * I.nT;
  m->info.nE = 2 * I.nE + 3 * I.nT;
  const int nB = I.nD + I.nN;
  int32_t *gsize = nullptr, *base = nullptr, *half_at = nullptr, *g_id = nullptr;
  int st = PHFEM_OK;
  auto chk = [&](int r) {
    if (st == PHFEM_OK) st = r;
  };
  chk(dalloc_n(ctx, &m->xy, 2 * (size_t)m->info.nV));
  chk(dalloc_n(ctx, &m->tri, 3 * (size_t)m->info.nT));
  chk(dalloc_n(ctx, &m->ed2el, 4 * (size_t)m->info.nE));
  chk(dalloc_n(ctx, &m->t2e, 3 * (size_t)m->info.nT));
  chk(dalloc_n(ctx, &m->sigma, 3 * (size_t)m->info.nT));
  chk(dalloc_n(ctx, &m->lk, (size_t)m->info.nE));
  chk(dalloc_n(ctx, &m->eclass, (size_t)m->info.nE));
  chk(dalloc_n(ctx, &m->bpairs, 4 * (size_t)nB));
  chk(dalloc_n(ctx, &m->bedge, 2 * (size_t)nB));
  chk(dalloc_n(ctx, &gsize, (size_t)I.nE + 1));
  chk(dalloc_n(ctx, &base, (size_t)I.nE + 1));
  chk(dalloc_n(ctx, &half_at, 2 * (size_t)I.nE));
  chk(dalloc_n(ctx, &g_id, 3 * (size_t)I.nT));
  if (st == PHFEM_OK) {
    k_refine_xy<<<grid_for(ctx, m->info.nV), kBlock, 0, s>>>(I.nV, I.nE, reinterpret_cast<const double2*>(c->xy),
                                                             c->ed2el, reinterpret_cast<double2*>(m->xy));
    chk(check_launch(ctx, "k_refine_xy"));
    k_refine_tri<<<grid_for(ctx, I.nT), kBlock, 0, s>>>(I.nT, I.nV, c->tri, c->t2e, m->tri);
    chk(check_launch(ctx, "k_refine_tri"));
    k_ref_group<<<grid_for(ctx, I.nE), kBlock, 0, s>>>(I.nE, c->ed2el, c->lk, c->t2e, gsize);
    chk(check_launch(ctx, "k_ref_group"));
  }
  if (st == PHFEM_OK) chk(exclusive_scan(ctx, gsize, base, I.nE, base + I.nE));
  if (st == PHFEM_OK) {
    k_ref_edges<<<grid_for(ctx, I.nE), kBlock, 0, s>>>(I.nV, I.nT, I.nE, c->tri, c->ed2el, c->lk, c->t2e, c->eclass,
                                                       base, m->ed2el, m->lk, m->eclass, half_at, g_id);
    chk(check_launch(ctx, "k_ref_edges"));
    k_ref_t2e<<<grid_for(ctx, I.nT), kBlock, 0, s>>>(I.nT, c->tri, c->ed2el, c->t2e, half_at, g_id, m->t2e,
                                                     m->sigma);
    chk(check_launch(ctx, "k_ref_t2e"));
    if (I.nD > 0) {
      k_refine_pairs<<<grid_for(ctx, I.nD), kBlock, 0, s>>>(I.nD, I.nV, c->bpairs, c->bedge, m->bpairs);
      k_ref_bedge<<<grid_for(ctx, I.nD), kBlock, 0, s>>>(I.nD, c->bpairs, c->bedge, c->ed2el, half_at, m->bedge);
      chk(check_launch(ctx, "k_ref_bedge"));
    }
    if (I.nN > 0) {
      k_refine_pairs<<<grid_for(ctx, I.nN), kBlock, 0, s>>>(I.nN, I.nV, c->bpairs + 2 * (size_t)I.nD,
                                                             c->bedge + I.nD, m->bpairs + 4 * (size_t)I.nD);
      k_ref_bedge<<<grid_for(ctx, I.nN), kBlock, 0, s>>>(I.nN, c->bpairs + 2 * (size_t)I.nD, c->bedge + I.nD,
                                                         c->ed2el, half_at, m->bedge + 2 * I.nD);
      chk(check_launch(ctx, "k_ref_bedge"));
    }
  }
  dfree(ctx, gsize);
  dfree(ctx, base);
  dfree(ctx, half_at);
  dfree(ctx, g_id);
  if (st == PHFEM_OK) st = mesh_finish(m);
  if (st != PHFEM_OK) {
    cudaStreamSynchronize(s);
    phfem_mesh_destroy(m);
    return st;
  }
  *out = m;
  return PHFEM_OK;
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
  if (fine) {  // tables in closed form; the arrays, if asked for, are copies of the mesh's
    PH_TRY(refine_tables(coarse, fine));
    const phfem_mesh m = *fine;
    cudaError_t e = cudaSuccess;
    if (xy) e = cudaMemcpyAsync(xy, m->xy, sizeof(double) * 2 * (size_t)nV2, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && tri)
      e = cudaMemcpyAsync(tri, m->tri, sizeof(int32_t) * 3 * (size_t)nT2, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && dirichlet && nD2)
      e = cudaMemcpyAsync(dirichlet, m->bpairs, sizeof(int32_t) * 2 * (size_t)nD2, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && neumann && nN2)
      e = cudaMemcpyAsync(neumann, m->bpairs + 2 * (size_t)nD2, sizeof(int32_t) * 2 * (size_t)nN2,
                          cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) {
      phfem_mesh_destroy(m);
      *fine = nullptr;
      return cuda_fail(e, "phfem_mesh_refine: copies", __FILE__, __LINE__);
    }
    return PHFEM_OK;
  }
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
  dfree(ctx, txy);
  dfree(ctx, ttri);
  dfree(ctx, tdir);
  dfree(ctx, tneu);
  return st;
}

}  // extern "C"
