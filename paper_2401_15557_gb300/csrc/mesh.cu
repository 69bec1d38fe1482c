// Mesh tables on the device (Section 2.2: nodes2element, nodes2edge,
// edge2element, led/ledTN of Listings 1-3) and the CSR pattern of the
// free-edge system.
//
// Edge numbering of nodes2edge = column-major order of the nonzeros of
// triu(B): edges sorted by (larger vertex, smaller vertex).  The directed edge
// occurrences o = 3t + j (edge P_{j+1} -> P_{j+2} of triangle t, element-major
// as in Listing 3) are put in (larger vertex, smaller vertex, occurrence)
// order by two stable radix sorts (by the smaller vertex, then by the larger
// one; equal keys keep the occurrence order); an entry that differs from the
// previous one starts an edge, and a scan of those starts numbers the edges.
// Every step runs one thread per entry, so the cost does not depend on vertex
// valence.  The first occurrence of an edge is its T+ (Eq. ed2el), the second
// its T-.
#include <algorithm>
#include <vector>

#include "internal.cuh"

namespace phfem {
namespace {

__device__ __forceinline__ void record(DevStatus* s, int code, int index, int detail) {
  if (atomicCAS(&s->code, 0, code) == 0) {
    s->index = index;
    s->detail = detail;
  }
}

// detail codes of PHFEM_EMESH
enum {
  kBadVertex = 1, kClockwise = 2, kDegenerateEdge = 3, kEdgeInThree = 4, kSameDirection = 5,
  kNotAnEdge = 6, kInteriorListed = 7, kBoundaryClass = 8
};

__global__ void k_count(int nT, int nV, const int32_t* __restrict__ tri, const double* __restrict__ xy,
                        int32_t* __restrict__ cnt, DevStatus* err) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nT; t += gridDim.x * blockDim.x) {
    int v[3] = {tri[3 * t], tri[3 * t + 1], tri[3 * t + 2]};
    bool ok = true;
    for (int j = 0; j < 3; ++j)
      if (v[j] < 0 || v[j] >= nV) ok = false;
    if (!ok) {
      record(err, PHFEM_EMESH, t, kBadVertex);
      continue;
    }
    const double x0 = xy[2 * v[0]], y0 = xy[2 * v[0] + 1];
    const double x1 = xy[2 * v[1]], y1 = xy[2 * v[1] + 1];
    const double x2 = xy[2 * v[2]], y2 = xy[2 * v[2] + 1];
    const double area2 = (x1 - x0) * (y2 - y0) - (y1 - y0) * (x2 - x0);
    if (!(area2 > 0.0)) record(err, PHFEM_EMESH, t, kClockwise);
    for (int j = 0; j < 3; ++j) {
      int a = v[j], b = v[(j + 1) % 3];
      if (a == b) {
        record(err, PHFEM_EMESH, t, kDegenerateEdge);
        continue;
      }
      atomicAdd(&cnt[max(a, b)], 1);
    }
  }
}

// Keys of the directed edges in occurrence order: smaller and larger vertex.
__global__ void k_keys(int nT, const int32_t* __restrict__ tri, uint32_t* __restrict__ lo_o,
                       uint32_t* __restrict__ hi_o, uint32_t* __restrict__ key, int32_t* __restrict__ occ) {
  const int n = 3 * nT;
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < n; o += gridDim.x * blockDim.x) {
    const int t = o / 3, j = o - 3 * t;
    const int a = tri[o], b = tri[3 * t + (j == 2 ? 0 : j + 1)];
    const uint32_t lo = (uint32_t)min(a, b), hi = (uint32_t)max(a, b);
    lo_o[o] = lo;
    hi_o[o] = hi;
    key[o] = lo;
    occ[o] = o;
  }
}

// key[i] = larger vertex of the entry now at position i (for the second sort).
__global__ void k_hi_key(int n, const uint32_t* __restrict__ hi_o, const int32_t* __restrict__ occ,
                         uint32_t* __restrict__ key) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) key[i] = hi_o[occ[i]];
}

// Entries in (larger, smaller, occurrence) order: the packed entry
// (smaller << 32 | occurrence), whether it starts an edge, and the checks that
// an edge has at most two occurrences of opposite direction.
__global__ void k_entries(int n, const int32_t* __restrict__ tri, const uint32_t* __restrict__ lo_o,
                          const uint32_t* __restrict__ hi_o, const int32_t* __restrict__ occ,
                          unsigned long long* __restrict__ buf, int32_t* __restrict__ start, DevStatus* err) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int o = occ[i];
    const uint32_t lo = lo_o[o], hi = hi_o[o];
    buf[i] = ((unsigned long long)lo << 32) | (unsigned)o;
    bool same = false;
    if (i > 0) {
      const int op = occ[i - 1];
      same = lo_o[op] == lo && hi_o[op] == hi;
      if (same) {
        if (tri[op] == tri[o]) record(err, PHFEM_EMESH, (int)hi, kSameDirection);  // same initial vertex
        if (i > 1) {
          const int oq = occ[i - 2];
          if (lo_o[oq] == lo && hi_o[oq] == hi) record(err, PHFEM_EMESH, (int)hi, kEdgeInThree);
        }
      }
    }
    start[i] = same ? 0 : 1;
  }
}

__device__ __forceinline__ int next3(int j) { return j == 2 ? 0 : j + 1; }

// One thread per entry that starts an edge: edge number = number of starts
// before it; T+ is this occurrence, T- the next entry's if it is the same edge.
__global__ void k_edges(int n, const int32_t* __restrict__ tri, const unsigned long long* __restrict__ buf,
                        const int32_t* __restrict__ start, const int32_t* __restrict__ enr,
                        int32_t* __restrict__ ed2el, int32_t* __restrict__ t2e, int8_t* __restrict__ sigma,
                        uint8_t* __restrict__ lk, int32_t* __restrict__ pos_edge) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (!start[i]) continue;
    const int edge = enr[i];
    const int run = (i + 1 < n && !start[i + 1]) ? 2 : 1;
    const int op = (int)(unsigned)buf[i];
    const int tp = op / 3, jp = op - 3 * tp;
    const int kp = (jp + 2) % 3;  // directed edge P_{j+1}P_{j+2} is E_{j+3 mod 3}
    ed2el[4 * edge + 0] = tri[3 * tp + jp];
    ed2el[4 * edge + 1] = tri[3 * tp + next3(jp)];
    ed2el[4 * edge + 2] = tp;
    t2e[3 * tp + kp] = edge;
    sigma[3 * tp + kp] = 1;
    int km = 0;
    if (run == 2) {
      const int om = (int)(unsigned)buf[i + 1];
      const int tm = om / 3, jm = om - 3 * tm;
      km = (jm + 2) % 3;
      ed2el[4 * edge + 3] = tm;
      t2e[3 * tm + km] = edge;
      sigma[3 * tm + km] = -1;
    } else {
      ed2el[4 * edge + 3] = -1;
    }
    lk[edge] = (uint8_t)(kp | (km << 2));
    for (int r = 0; r < run; ++r) pos_edge[i + r] = edge;
  }
}

// Listed boundary pairs -> edge ids; adds `code` to the edge's class word.
__global__ void k_bclass(int nB, const int32_t* __restrict__ pairs, int code, int nV,
                         const int32_t* __restrict__ bstart, const unsigned long long* __restrict__ buf,
                         const int32_t* __restrict__ pos_edge, const int32_t* __restrict__ ed2el,
                         int32_t* __restrict__ ecode, int32_t* __restrict__ bedge, DevStatus* err) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nB; i += gridDim.x * blockDim.x) {
    int a = pairs[2 * i], b = pairs[2 * i + 1];
    if (a < 0 || b < 0 || a >= nV || b >= nV || a == b) {
      record(err, PHFEM_EMESH, i, kNotAnEdge);
      continue;
    }
    int hi = max(a, b), lo = min(a, b);
    int found = -1;  // the bucket of hi is sorted by the smaller vertex: binary search
    int l0 = bstart[hi], l1 = bstart[hi + 1];
    while (l0 < l1) {
      const int mid = (l0 + l1) >> 1;
      if ((int)(buf[mid] >> 32) < lo) l0 = mid + 1;
      else l1 = mid;
    }
    if (l0 < bstart[hi + 1] && (int)(buf[l0] >> 32) == lo) found = l0;
    if (found < 0) {
      record(err, PHFEM_EMESH, i, kNotAnEdge);
      continue;
    }
    int e = pos_edge[found];
    bedge[i] = e;
    if (ed2el[4 * e + 3] >= 0) {
      record(err, PHFEM_EMESH, i, kInteriorListed);
      continue;
    }
    atomicAdd(&ecode[e], code);
  }
}

__global__ void k_class(int nE, const int32_t* __restrict__ ed2el, const int32_t* __restrict__ ecode,
                        uint8_t* __restrict__ eclass, int32_t* __restrict__ isfree,
                        int32_t* __restrict__ islam, DevStatus* err) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nE; e += gridDim.x * blockDim.x) {
    int c = ecode[e];
    uint8_t cls = PHFEM_EDGE_INTERIOR;
    if (ed2el[4 * e + 3] < 0) {
      if (c == 1) cls = PHFEM_EDGE_DIRICHLET;
      else if (c == 16) cls = PHFEM_EDGE_NEUMANN;
      else record(err, PHFEM_EMESH, e, kBoundaryClass);
    }
    eclass[e] = cls;
    isfree[e] = cls != PHFEM_EDGE_DIRICHLET;
    islam[e] = cls != PHFEM_EDGE_NEUMANN;
  }
}

__global__ void k_flags(int nE, const uint8_t* __restrict__ eclass, int32_t* __restrict__ isfree,
                        int32_t* __restrict__ islam) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nE; e += gridDim.x * blockDim.x) {
    const uint8_t c = eclass[e];
    isfree[e] = c != PHFEM_EDGE_DIRICHLET;
    islam[e] = c != PHFEM_EDGE_NEUMANN;
  }
}

__global__ void k_ids(int nE, const int32_t* __restrict__ flag_free, const int32_t* __restrict__ flag_lam,
                      int32_t* __restrict__ free_id, int32_t* __restrict__ lam_id, const uint8_t* __restrict__ eclass) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nE; e += gridDim.x * blockDim.x) {
    uint8_t c = eclass[e];
    if (c == PHFEM_EDGE_DIRICHLET) free_id[e] = -1;
    if (c == PHFEM_EDGE_NEUMANN) lam_id[e] = -1;
  }
}

__global__ void k_nbr(int nE, const int32_t* __restrict__ ed2el, const uint8_t* __restrict__ lk,
                      const int32_t* __restrict__ t2e, const int32_t* __restrict__ free_id,
                      const double* __restrict__ xy, int32_t* __restrict__ nbr, double* __restrict__ elen,
                      int32_t* __restrict__ rowlen) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nE; e += gridDim.x * blockDim.x) {
    const int tp = ed2el[4 * e + 2], tm = ed2el[4 * e + 3];
    const int kp = lk[e] & 3, km = (lk[e] >> 2) & 3;
    int n[4];
    n[0] = t2e[3 * tp + next3(kp)];
    n[1] = t2e[3 * tp + next3(next3(kp))];
    if (tm >= 0) {
      n[2] = t2e[3 * tm + next3(km)];
      n[3] = t2e[3 * tm + next3(next3(km))];
    } else {
      n[2] = n[3] = e;
    }
#pragma unroll
    for (int s = 0; s < 4; ++s) nbr[(size_t)s * nE + e] = n[s];
    const int a = ed2el[4 * e], b = ed2el[4 * e + 1];
    const double dx = xy[2 * b] - xy[2 * a], dy = xy[2 * b + 1] - xy[2 * a + 1];
    elen[e] = sqrt(dx * dx + dy * dy);
    const int r = free_id[e];
    if (r >= 0) {
      int len = 1;
#pragma unroll
      for (int s = 0; s < 4; ++s)
        if (n[s] != e && free_id[n[s]] >= 0) ++len;
      rowlen[r] = len;
    }
  }
}

__global__ void k_col(int nE, const int32_t* __restrict__ nbr, const int32_t* __restrict__ free_id,
                      const int32_t* __restrict__ row_ptr, int32_t* __restrict__ col) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nE; e += gridDim.x * blockDim.x) {
    const int r = free_id[e];
    if (r < 0) continue;
    int c[5];
    int len = 0;
    c[len++] = r;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      int n = nbr[(size_t)s * nE + e];
      if (n != e) {
        int f = free_id[n];
        if (f >= 0) c[len++] = f;
      }
    }
    for (int i = 1; i < len; ++i) {
      int k = c[i], j = i - 1;
      while (j >= 0 && c[j] > k) {
        c[j + 1] = c[j];
        --j;
      }
      c[j + 1] = k;
    }
    const int base = row_ptr[r];
    for (int i = 0; i < len; ++i) col[base + i] = c[i];
  }
}

const char* mesh_detail(int d) {
  switch (d) {
    case kBadVertex: return "vertex index out of range";
    case kClockwise: return "clockwise or degenerate triangle";
    case kDegenerateEdge: return "triangle with a repeated vertex";
    case kEdgeInThree: return "edge shared by more than two triangles";
    case kSameDirection: return "two triangles traverse a shared edge in the same direction";
    case kNotAnEdge: return "listed boundary pair is not an edge of the mesh";
    case kInteriorListed: return "listed boundary pair is an interior edge";
    case kBoundaryClass: return "boundary edge listed in neither or both lists, or twice";
    default: return "mesh error";
  }
}

int check_status(phfem_ctx ctx, DevStatus* d_err, const char* where) {
  DevStatus h;
  PH_CUDA(cudaMemcpyAsync(&h, d_err, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
  PH_CUDA(cudaStreamSynchronize(ctx->stream));
  if (h.code != 0) {
    std::string msg = std::string(where) + ": " + mesh_detail(h.detail) + " (index " + std::to_string(h.index) + ")";
    return fail(h.code, msg);
  }
  return PHFEM_OK;
}

struct Temps {
  phfem_ctx ctx;
  std::vector<void*> ptrs;
  ~Temps() {
    for (void* p : ptrs) dfree(ctx, p);
  }
  template <typename T>
  int get(T** p, size_t n) {
    int s = dalloc_n(ctx, p, n);
    if (s == PHFEM_OK) ptrs.push_back(*p);
    return s;
  }
};

void mesh_free(phfem_mesh m) {
  phfem_ctx c = m->ctx;
  dfree(c, m->xy);
  dfree(c, m->tri);
  dfree(c, m->ed2el);
  dfree(c, m->t2e);
  dfree(c, m->sigma);
  dfree(c, m->eclass);
  dfree(c, m->lk);
  dfree(c, m->free_id);
  dfree(c, m->lam_id);
  dfree(c, m->nbr);
  dfree(c, m->elen);
  dfree(c, m->row_ptr);
  dfree(c, m->col);
  dfree(c, m->bpairs);
  dfree(c, m->bedge);
  mesh_order_free(m);
  delete m;
}

int read_int(phfem_ctx ctx, const int32_t* d, int32_t* h) {
  PH_CUDA(cudaMemcpyAsync(h, d, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
  PH_CUDA(cudaStreamSynchronize(ctx->stream));
  return PHFEM_OK;
}

int build(phfem_ctx ctx, int nV, const double* xy, int nT, const int32_t* tri, int nD,
          const int32_t* dir, int nN, const int32_t* neu, phfem_mesh m) {
  cudaStream_t s = ctx->stream;
  Temps tmp{ctx, {}};
  PH_TRY(dalloc_n(ctx, &m->xy, 2 * (size_t)nV));
  PH_TRY(dalloc_n(ctx, &m->tri, 3 * (size_t)nT));
  PH_CUDA(cudaMemcpyAsync(m->xy, xy, sizeof(double) * 2 * (size_t)nV, cudaMemcpyDeviceToDevice, s));
  PH_CUDA(cudaMemcpyAsync(m->tri, tri, sizeof(int32_t) * 3 * (size_t)nT, cudaMemcpyDeviceToDevice, s));

  DevStatus* err;
  PH_TRY(tmp.get(&err, 1));
  PH_CUDA(cudaMemsetAsync(err, 0, sizeof(DevStatus), s));
  int32_t *cnt, *bstart;
  PH_TRY(tmp.get(&cnt, nV));
  PH_TRY(tmp.get(&bstart, (size_t)nV + 1));
  PH_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * nV, s));

  k_count<<<grid_for(ctx, nT), kBlock, 0, s>>>(nT, nV, m->tri, m->xy, cnt, err);
  PH_TRY(check_launch(ctx, "k_count"));
  PH_TRY(check_status(ctx, err, "phfem_mesh_build"));
  PH_TRY(exclusive_scan(ctx, cnt, bstart, nV, bstart + nV));  // bucket of each larger vertex

  // directed edges in (larger vertex, smaller vertex, occurrence) order
  const int n = 3 * nT;
  uint32_t *lo_o, *hi_o, *key, *key2;
  int32_t *occ, *occ2, *start, *enr;
  unsigned long long* buf;
  PH_TRY(tmp.get(&lo_o, (size_t)n));
  PH_TRY(tmp.get(&hi_o, (size_t)n));
  PH_TRY(tmp.get(&key, (size_t)n));
  PH_TRY(tmp.get(&key2, (size_t)n));
  PH_TRY(tmp.get(&occ, (size_t)n));
  PH_TRY(tmp.get(&occ2, (size_t)n));
  PH_TRY(tmp.get(&start, (size_t)n + 1));
  PH_TRY(tmp.get(&enr, (size_t)n + 1));
  PH_TRY(tmp.get(&buf, (size_t)n));
  int vbits = 1;
  while (vbits < 31 && (1ll << vbits) < (long long)nV) ++vbits;
  k_keys<<<grid_for(ctx, n), kBlock, 0, s>>>(nT, m->tri, lo_o, hi_o, key, occ);
  PH_TRY(check_launch(ctx, "k_keys"));
  PH_TRY(radix_sort_pairs(ctx, key, occ, key2, occ2, n, vbits));   // by the smaller vertex
  k_hi_key<<<grid_for(ctx, n), kBlock, 0, s>>>(n, hi_o, occ, key);
  PH_TRY(check_launch(ctx, "k_hi_key"));
  PH_TRY(radix_sort_pairs(ctx, key, occ, key2, occ2, n, vbits));   // then, stably, by the larger one
  k_entries<<<grid_for(ctx, n), kBlock, 0, s>>>(n, m->tri, lo_o, hi_o, occ, buf, start, err);
  PH_TRY(check_launch(ctx, "k_entries"));
  PH_TRY(check_status(ctx, err, "phfem_mesh_build"));
  PH_TRY(exclusive_scan(ctx, start, enr, n, enr + n));
  int32_t nE = 0;
  PH_TRY(read_int(ctx, enr + n, &nE));
  m->info.nE = nE;

  int32_t* pos_edge;
  PH_TRY(tmp.get(&pos_edge, 3 * (size_t)nT));
  PH_TRY(dalloc_n(ctx, &m->ed2el, 4 * (size_t)nE));
  PH_TRY(dalloc_n(ctx, &m->t2e, 3 * (size_t)nT));
  PH_TRY(dalloc_n(ctx, &m->sigma, 3 * (size_t)nT));
  PH_TRY(dalloc_n(ctx, &m->lk, (size_t)nE));
  k_edges<<<grid_for(ctx, n), kBlock, 0, s>>>(n, m->tri, buf, start, enr, m->ed2el, m->t2e, m->sigma, m->lk,
                                              pos_edge);
  PH_TRY(check_launch(ctx, "k_edges"));

  int32_t *ecode, *isfree, *islam;
  PH_TRY(tmp.get(&ecode, nE));
  PH_TRY(tmp.get(&isfree, (size_t)nE + 1));
  PH_TRY(tmp.get(&islam, (size_t)nE + 1));
  PH_CUDA(cudaMemsetAsync(ecode, 0, sizeof(int32_t) * nE, s));
  PH_TRY(dalloc_n(ctx, &m->bpairs, 2 * ((size_t)nD + nN)));
  PH_TRY(dalloc_n(ctx, &m->bedge, (size_t)nD + nN));
  if (nD > 0) {
    PH_CUDA(cudaMemcpyAsync(m->bpairs, dir, sizeof(int32_t) * 2 * (size_t)nD, cudaMemcpyDeviceToDevice, s));
    k_bclass<<<grid_for(ctx, nD), kBlock, 0, s>>>(nD, dir, 1, nV, bstart, buf, pos_edge, m->ed2el, ecode, m->bedge,
                                                  err);
    PH_TRY(check_launch(ctx, "k_bclass"));
  }
  if (nN > 0) {
    PH_CUDA(cudaMemcpyAsync(m->bpairs + 2 * (size_t)nD, neu, sizeof(int32_t) * 2 * (size_t)nN,
                            cudaMemcpyDeviceToDevice, s));
    k_bclass<<<grid_for(ctx, nN), kBlock, 0, s>>>(nN, neu, 16, nV, bstart, buf, pos_edge, m->ed2el, ecode,
                                                  m->bedge + nD, err);
    PH_TRY(check_launch(ctx, "k_bclass"));
  }
  PH_TRY(dalloc_n(ctx, &m->eclass, (size_t)nE));
  k_class<<<grid_for(ctx, nE), kBlock, 0, s>>>(nE, m->ed2el, ecode, m->eclass, isfree, islam, err);
  PH_TRY(check_launch(ctx, "k_class"));
  PH_TRY(check_status(ctx, err, "phfem_mesh_build"));

  return mesh_finish(m);
}

}  // namespace

// Free and multiplier numbering, neighbour slots, edge lengths and the CSR
// pattern, from ed2el, lk, t2e, eclass and xy.
int mesh_finish(phfem_mesh m) {
  phfem_ctx ctx = m->ctx;
  cudaStream_t s = ctx->stream;
  const int nE = m->info.nE;
  Temps tmp{ctx, {}};
  int32_t *isfree, *islam;
  PH_TRY(tmp.get(&isfree, (size_t)nE + 1));
  PH_TRY(tmp.get(&islam, (size_t)nE + 1));
  k_flags<<<grid_for(ctx, nE), kBlock, 0, s>>>(nE, m->eclass, isfree, islam);
  PH_TRY(check_launch(ctx, "k_flags"));
  PH_TRY(dalloc_n(ctx, &m->free_id, (size_t)nE));
  PH_TRY(dalloc_n(ctx, &m->lam_id, (size_t)nE));
  int32_t* totals;
  PH_TRY(tmp.get(&totals, 2));
  PH_TRY(exclusive_scan(ctx, isfree, m->free_id, nE, totals));
  PH_TRY(exclusive_scan(ctx, islam, m->lam_id, nE, totals + 1));
  k_ids<<<grid_for(ctx, nE), kBlock, 0, s>>>(nE, isfree, islam, m->free_id, m->lam_id, m->eclass);
  PH_TRY(check_launch(ctx, "k_ids"));
  int32_t ht[2];
  PH_CUDA(cudaMemcpyAsync(ht, totals, sizeof(ht), cudaMemcpyDeviceToHost, s));
  PH_CUDA(cudaStreamSynchronize(s));
  const int nF = ht[0], nL = ht[1];
  m->info.nF = nF;
  m->info.nL = nL;
  m->info.nD = nE - nF;
  m->info.nN = nE - nL;

  PH_TRY(dalloc_n(ctx, &m->nbr, 4 * (size_t)nE));
  PH_TRY(dalloc_n(ctx, &m->elen, (size_t)nE));
  PH_TRY(dalloc_n(ctx, &m->row_ptr, (size_t)nF + 1));
  int32_t* rowlen;
  PH_TRY(tmp.get(&rowlen, (size_t)nF + 1));
  k_nbr<<<grid_for(ctx, nE), kBlock, 0, s>>>(nE, m->ed2el, m->lk, m->t2e, m->free_id, m->xy, m->nbr, m->elen,
                                             rowlen);
  PH_TRY(check_launch(ctx, "k_nbr"));
  PH_TRY(exclusive_scan(ctx, rowlen, m->row_ptr, nF, m->row_ptr + nF));
  int32_t nnz = 0;
  PH_TRY(read_int(ctx, m->row_ptr + nF, &nnz));
  m->info.nnz = nnz;
  PH_TRY(dalloc_n(ctx, &m->col, (size_t)nnz));
  k_col<<<grid_for(ctx, nE), kBlock, 0, s>>>(nE, m->nbr, m->free_id, m->row_ptr, m->col);
  PH_TRY(check_launch(ctx, "k_col"));
  PH_CUDA(cudaStreamSynchronize(s));
  return PHFEM_OK;
}

}  // namespace phfem

using namespace phfem;

extern "C" {

PHFEM_API int phfem_mesh_build(phfem_ctx ctx, int32_t nV, const double* xy, int32_t nT, const int32_t* tri,
                               int32_t nD, const int32_t* dirichlet, int32_t nN, const int32_t* neumann,
                               phfem_mesh* out) {
  if (!out) return fail(PHFEM_EINVAL, "phfem_mesh_build: out is NULL");
  *out = nullptr;
  if (!ctx) return fail(PHFEM_EINVAL, "phfem_mesh_build: NULL context");
  if (nV < 3 || nT < 1 || !xy || !tri) return fail(PHFEM_EINVAL, "phfem_mesh_build: empty mesh or NULL arrays");
  if (nD < 0 || nN < 0 || (nD > 0 && !dirichlet) || (nN > 0 && !neumann))
    return fail(PHFEM_EINVAL, "phfem_mesh_build: bad boundary lists");
  if ((int64_t)nT * 3 >= (int64_t)INT32_MAX) return fail(PHFEM_EINVAL, "phfem_mesh_build: too many triangles");
  phfem_mesh m = new phfem_mesh_s();
  m->ctx = ctx;
  m->info.nV = nV;
  m->info.nT = nT;
  int st = build(ctx, nV, xy, nT, tri, nD, dirichlet, nN, neumann, m);
  if (st != PHFEM_OK) {
    cudaStreamSynchronize(ctx->stream);
    mesh_free(m);
    return st;
  }
  *out = m;
  return PHFEM_OK;
}

PHFEM_API int phfem_mesh_info_get(phfem_mesh mesh, phfem_mesh_info* out) {
  if (!mesh || !out) return fail(PHFEM_EINVAL, "phfem_mesh_info_get: NULL argument");
  *out = mesh->info;
  return PHFEM_OK;
}

PHFEM_API int phfem_mesh_tables(phfem_mesh m, int32_t* ed2el, int32_t* t2e, int8_t* sigma, uint8_t* eclass,
                                int32_t* free_id, int32_t* lam_id, int32_t* row_ptr, int32_t* col) {
  if (!m) return fail(PHFEM_EINVAL, "phfem_mesh_tables: NULL mesh");
  cudaStream_t s = m->ctx->stream;
  const phfem_mesh_info& I = m->info;
  auto cp = [&](void* dst, const void* src, size_t bytes) -> int {
    if (dst && bytes) PH_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, s));
    return PHFEM_OK;
  };
  PH_TRY(cp(ed2el, m->ed2el, sizeof(int32_t) * 4 * (size_t)I.nE));
  PH_TRY(cp(t2e, m->t2e, sizeof(int32_t) * 3 * (size_t)I.nT));
  PH_TRY(cp(sigma, m->sigma, sizeof(int8_t) * 3 * (size_t)I.nT));
  PH_TRY(cp(eclass, m->eclass, sizeof(uint8_t) * (size_t)I.nE));
  PH_TRY(cp(free_id, m->free_id, sizeof(int32_t) * (size_t)I.nE));
  PH_TRY(cp(lam_id, m->lam_id, sizeof(int32_t) * (size_t)I.nE));
  PH_TRY(cp(row_ptr, m->row_ptr, sizeof(int32_t) * ((size_t)I.nF + 1)));
  PH_TRY(cp(col, m->col, sizeof(int32_t) * (size_t)I.nnz));
  return PHFEM_OK;
}

PHFEM_API int phfem_mesh_destroy(phfem_mesh mesh) {
  if (!mesh) return fail(PHFEM_EINVAL, "phfem_mesh_destroy: NULL mesh");
  mesh_free(mesh);
  return PHFEM_OK;
}

}  // extern "C"
