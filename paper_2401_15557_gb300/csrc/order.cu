// Locality order of the edges for the iteration kernels.
//
// The paper numbers edges by (larger vertex, smaller vertex) (Listing 2).  On
// red-refined meshes that order scatters the neighbours of an edge row: about
// a third of the references of the edge system's rows point hundreds of
// thousands of rows away, so every operator product re-fetches the gathered
// vector from DRAM and needs 32-bit column indices.  The iteration kernels
// therefore run on an internal numbering: edges sorted by the Morton (Z-order)
// code of their midpoints, ties kept in the paper's order (a stable sort, so
// the numbering is deterministic).  In that order ~95 % of the neighbour
// references lie within 256 rows and ~99 % of the rows have all four
// neighbours within +-32767 rows, so a row's neighbours are stored as four
// 16-bit differences; the few other rows are marked (first difference
// -32768) and keep their four 32-bit indices in an overflow table.  The paper's
// numbering stays the one every entry point reads and writes.
//
// The sort is a least-significant-digit radix sort with 8-bit digits: per
// pass, a per-block digit histogram, one exclusive scan of the histograms in
// digit-major order, and a stable scatter that ranks equal digits within a
// block warp by warp (match masks) and across warps through shared memory.
#include <cstdio>

#include "internal.cuh"

namespace phfem {
namespace {

constexpr int kRsItems = 16;
constexpr int kRsTile = kBlock * kRsItems;  // elements per block and pass
constexpr int kRsDigits = 256;
static_assert(kBlock == kRsDigits, "the scatter gives every thread one digit");

// Bounding box of the vertices: min x, min y, -max x, -max y (all minima).
__global__ void k_bbox(int nV, const double2* __restrict__ xy, double* partials, unsigned int* counter,
                       double* box) {
  __shared__ double smem[kBlock / 32];
  double m[4] = {INFINITY, INFINITY, INFINITY, INFINITY};
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nV; v += gridDim.x * blockDim.x) {
    const double2 p = xy[v];
    m[0] = fmin(m[0], p.x);
    m[1] = fmin(m[1], p.y);
    m[2] = fmin(m[2], -p.x);
    m[3] = fmin(m[3], -p.y);
  }
  for (int k = 0; k < 4; ++k) {
    double v = m[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_down_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) smem[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      double b = smem[0];
      for (int i = 1; i < kBlock / 32; ++i) b = fmin(b, smem[i]);
      partials[k * kMaxGrid + blockIdx.x] = b;
    }
    __syncthreads();
  }
  if (!arrive_last(counter)) return;
  if (threadIdx.x < 4) {
    double b = INFINITY;
    for (int i = 0; i < (int)gridDim.x; ++i) b = fmin(b, __ldcg(partials + threadIdx.x * kMaxGrid + i));
    box[threadIdx.x] = b;
  }
  if (threadIdx.x == 0) *counter = 0;
}

__device__ __forceinline__ uint32_t spread16(uint32_t v) {
  v &= 0xFFFFu;
  v = (v | (v << 8)) & 0x00FF00FFu;
  v = (v | (v << 4)) & 0x0F0F0F0Fu;
  v = (v | (v << 2)) & 0x33333333u;
  v = (v | (v << 1)) & 0x55555555u;
  return v;
}

// Morton code of every edge midpoint on a 2^qbits x 2^qbits grid over the
// bounding box; the value is the edge id.
__global__ void k_morton(int nE, const int32_t* __restrict__ ed2el, const double2* __restrict__ xy,
                         const double* __restrict__ box, int qbits, uint32_t* __restrict__ key,
                         int32_t* __restrict__ val) {
  const double x0 = box[0], y0 = box[1];
  const double span = fmax(-box[2] - x0, -box[3] - y0);
  const double cells = (double)(1u << qbits);
  const double scale = span > 0.0 ? cells / span : 0.0;
  const uint32_t top = (1u << qbits) - 1u;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nE; e += gridDim.x * blockDim.x) {
    const int4 E = reinterpret_cast<const int4*>(ed2el)[e];
    const double2 a = xy[E.x], b = xy[E.y];
    const double mx = 0.5 * (a.x + b.x), my = 0.5 * (a.y + b.y);
    uint32_t qx = (uint32_t)fmin(fmax((mx - x0) * scale, 0.0), (double)top);
    uint32_t qy = (uint32_t)fmin(fmax((my - y0) * scale, 0.0), (double)top);
    key[e] = spread16(qx) | (spread16(qy) << 1);
    val[e] = e;
  }
}

// Morton key of each tile of kBlock consecutive edges (one block per tile):
// the mean of its edge midpoints on a 2^16 x 2^16 grid over the bounding box;
// the value is the tile.
__global__ void __launch_bounds__(kBlock) k_tile_key(int nE, const int32_t* __restrict__ ed2el,
                                                     const double2* __restrict__ xy, const double* __restrict__ box,
                                                     uint32_t* __restrict__ key, int32_t* __restrict__ val) {
  __shared__ double sm[2][kBlock / 32];
  const int t = blockIdx.x, e = t * kBlock + threadIdx.x;
  double mx = 0.0, my = 0.0;
  if (e < nE) {
    const int4 E = reinterpret_cast<const int4*>(ed2el)[e];
    const double2 a = xy[E.x], b = xy[E.y];
    mx = 0.5 * (a.x + b.x);
    my = 0.5 * (a.y + b.y);
  }
  mx = warp_sum(mx);
  my = warp_sum(my);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    sm[0][w] = mx;
    sm[1][w] = my;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  double sx = 0.0, sy = 0.0;
  for (int i = 0; i < kBlock / 32; ++i) {
    sx += sm[0][i];
    sy += sm[1][i];
  }
  const int cnt = min(kBlock, nE - t * kBlock);
  const double x0 = box[0], y0 = box[1];
  const double span = fmax(-box[2] - x0, -box[3] - y0);
  const double scale = span > 0.0 ? 65536.0 / span : 0.0;
  const uint32_t qx = (uint32_t)fmin(fmax((sx / cnt - x0) * scale, 0.0), 65535.0);
  const uint32_t qy = (uint32_t)fmin(fmax((sy / cnt - y0) * scale, 0.0), 65535.0);
  key[t] = spread16(qx) | (spread16(qy) << 1);
  val[t] = t;
}

// Per-block digit histogram, stored digit-major: counts[d * nb + block].
__global__ void __launch_bounds__(kBlock) k_rs_hist(int n, const uint32_t* __restrict__ key, int shift,
                                                    int32_t* __restrict__ counts, int nb) {
  __shared__ int h[kRsDigits];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kRsTile;
  for (int r = 0; r < kRsItems; ++r) {
    const int64_t j = base + (int64_t)r * kBlock + threadIdx.x;
    if (j < n) atomicAdd(&h[(key[j] >> shift) & 0xFF], 1);
  }
  __syncthreads();
  counts[(size_t)threadIdx.x * nb + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter of one pass: element j of a block's tile goes to
// offs[d * nb + block] + (number of earlier tile elements with digit d).
__global__ void __launch_bounds__(kBlock) k_rs_scatter(int n, const uint32_t* __restrict__ kin,
                                                       const int32_t* __restrict__ vin, uint32_t* __restrict__ kout,
                                                       int32_t* __restrict__ vout, int shift,
                                                       const int32_t* __restrict__ offs, int nb) {
  __shared__ int run[kRsDigits];                // tile elements of each digit placed so far
  __shared__ int wcnt[kBlock / 32][kRsDigits];  // this round: per-warp counts, then per-warp starts
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  run[threadIdx.x] = offs[(size_t)threadIdx.x * nb + blockIdx.x];
  const unsigned lt = (1u << lane) - 1u;
  const int64_t base = (int64_t)blockIdx.x * kRsTile;
  for (int r = 0; r < kRsItems; ++r) {
#pragma unroll
    for (int k = 0; k < kBlock / 32; ++k) wcnt[k][threadIdx.x] = 0;
    __syncthreads();
    const int64_t j = base + (int64_t)r * kBlock + threadIdx.x;
    const bool valid = j < n;
    uint32_t kv = 0;
    int32_t vv = 0;
    int d = kRsDigits;  // invalid lanes form their own group
    if (valid) {
      kv = kin[j];
      vv = vin[j];
      d = (kv >> shift) & 0xFF;
    }
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int rank = __popc(peers & lt);
    if (valid && rank == 0) wcnt[w][d] = __popc(peers);
    __syncthreads();
    {  // thread t: starts of digit t for every warp of this round
      int acc = run[threadIdx.x];
#pragma unroll
      for (int k = 0; k < kBlock / 32; ++k) {
        const int c = wcnt[k][threadIdx.x];
        wcnt[k][threadIdx.x] = acc;
        acc += c;
      }
      run[threadIdx.x] = acc;
    }
    __syncthreads();
    if (valid) {
      const int pos = wcnt[w][d] + rank;
      kout[pos] = kv;
      vout[pos] = vv;
    }
    __syncthreads();
  }
}

__global__ void k_inverse(int n, const int32_t* __restrict__ perm, int32_t* __restrict__ iperm) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) iperm[perm[i]] = i;
}

// Internal neighbours of internal row i; flags rows whose neighbours are not
// all within +-32767 rows.
__global__ void k_nbr_flag(int nE, const int32_t* __restrict__ perm, const int32_t* __restrict__ iperm,
                           const int32_t* __restrict__ nbr, int32_t* __restrict__ flag) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nE; i += gridDim.x * blockDim.x) {
    const int e = perm[i];
    int far = 0;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int d = iperm[nbr[(size_t)s * nE + e]] - i;
      far |= (d < -32767 || d > 32767);
    }
    flag[i] = far;
  }
}

__global__ void k_nbr16(int nE, const int32_t* __restrict__ perm, const int32_t* __restrict__ iperm,
                        const int32_t* __restrict__ nbr, const int32_t* __restrict__ flag,
                        const int32_t* __restrict__ slot, const uint8_t* __restrict__ eclass, short4* __restrict__ nb,
                        int4* __restrict__ ovf, uint8_t* __restrict__ eclass_i) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nE; i += gridDim.x * blockDim.x) {
    const int e = perm[i];
    int c[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) c[s] = iperm[nbr[(size_t)s * nE + e]];
    if (flag[i]) {
      const int k = slot[i];
      ovf[k] = make_int4(c[0], c[1], c[2], c[3]);
      nb[i] = make_short4((short)-32768, (short)(uint16_t)(k & 0xFFFF), (short)(uint16_t)((unsigned)k >> 16), 0);
    } else {
      nb[i] = make_short4((short)(c[0] - i), (short)(c[1] - i), (short)(c[2] - i), (short)(c[3] - i));
    }
    eclass_i[i] = eclass[e];
  }
}

}  // namespace

// Stable sort of (key, value) pairs by the low `bits` bits of the key.  The
// result is in (k0, v0); (k1, v1) are scratch of the same size.
int radix_sort_pairs(phfem_ctx ctx, uint32_t* k0, int32_t* v0, uint32_t* k1, int32_t* v1, int n, int bits) {
  if (n <= 1) return PHFEM_OK;
  cudaStream_t s = ctx->stream;
  const int nb = (n + kRsTile - 1) / kRsTile;
  int32_t* counts = nullptr;
  PH_TRY(dalloc_n(ctx, &counts, (size_t)kRsDigits * nb));
  int st = PHFEM_OK;
  int passes = (bits + 7) / 8;
  uint32_t *ka = k0, *kb = k1;
  int32_t *va = v0, *vb = v1;
  for (int p = 0; p < passes && st == PHFEM_OK; ++p) {
    k_rs_hist<<<nb, kBlock, 0, s>>>(n, ka, 8 * p, counts, nb);
    st = check_launch(ctx, "k_rs_hist");
    if (st == PHFEM_OK) st = exclusive_scan(ctx, counts, counts, kRsDigits * nb, nullptr);
    if (st == PHFEM_OK) {
      k_rs_scatter<<<nb, kBlock, 0, s>>>(n, ka, va, kb, vb, 8 * p, counts, nb);
      st = check_launch(ctx, "k_rs_scatter");
    }
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  if (st == PHFEM_OK && ka != k0) {  // an odd number of passes: the result is in the scratch
    cudaError_t e = cudaMemcpyAsync(k0, ka, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(v0, va, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) st = cuda_fail(e, "radix_sort_pairs copy", __FILE__, __LINE__);
  }
  dfree(ctx, counts);
  return st;
}

// Builds the mesh's locality order (perm, iperm), the 16-bit neighbour
// differences with their overflow table and the class of each internal row,
// once per mesh.
int mesh_order(phfem_mesh m) {
  if (m->perm) return PHFEM_OK;
  phfem_ctx ctx = m->ctx;
  cudaStream_t s = ctx->stream;
  const int nE = m->info.nE, nV = m->info.nV;
  int qbits = 4;
  while (qbits < 15 && (1ll << (2 * qbits)) < 4ll * nE) ++qbits;
  uint32_t *key = nullptr, *key2 = nullptr;
  int32_t *val2 = nullptr, *flag = nullptr, *slot = nullptr;
  double* scratch = nullptr;  // partials [4][kMaxGrid], box [4], counter
  int st = PHFEM_OK;
  auto chk = [&](int r) {
    if (st == PHFEM_OK) st = r;
  };
  chk(dalloc_n(ctx, &m->perm, (size_t)nE));
  chk(dalloc_n(ctx, &m->iperm, (size_t)nE));
  chk(dalloc_n(ctx, &m->nbr16, (size_t)nE + 2));  // + 16 bytes: tiles are copied in 16-byte units
  chk(dalloc_n(ctx, &m->eclass_i, (size_t)nE));
  chk(dalloc_n(ctx, &key, (size_t)nE));
  chk(dalloc_n(ctx, &key2, (size_t)nE));
  chk(dalloc_n(ctx, &val2, (size_t)nE));
  chk(dalloc_n(ctx, &flag, (size_t)nE + 1));
  chk(dalloc_n(ctx, &slot, (size_t)nE + 1));
  chk(dalloc_n(ctx, &scratch, 4 * (size_t)kMaxGrid + 8));
  if (st == PHFEM_OK) {
    double* box = scratch + 4 * kMaxGrid;
    unsigned int* counter = reinterpret_cast<unsigned int*>(box + 4);
    cudaMemsetAsync(counter, 0, sizeof(unsigned int), s);
    k_bbox<<<grid_for(ctx, nV), kBlock, 0, s>>>(nV, reinterpret_cast<const double2*>(m->xy), scratch, counter, box);
    chk(check_launch(ctx, "k_bbox"));
    k_morton<<<grid_for(ctx, nE), kBlock, 0, s>>>(nE, m->ed2el, reinterpret_cast<const double2*>(m->xy), box, qbits,
                                                  key, m->perm);
    chk(check_launch(ctx, "k_morton"));
  }
  if (st == PHFEM_OK) chk(radix_sort_pairs(ctx, key, m->perm, key2, val2, nE, 2 * qbits));
  if (st == PHFEM_OK) {
    k_inverse<<<grid_for(ctx, nE), kBlock, 0, s>>>(nE, m->perm, m->iperm);
    chk(check_launch(ctx, "k_inverse"));
    k_nbr_flag<<<grid_for(ctx, nE), kBlock, 0, s>>>(nE, m->perm, m->iperm, m->nbr, flag);
    chk(check_launch(ctx, "k_nbr_flag"));
  }
  if (st == PHFEM_OK) chk(exclusive_scan(ctx, flag, slot, nE, slot + nE));
  int32_t novf = 0;
  if (st == PHFEM_OK) {
    cudaError_t e = cudaMemcpyAsync(&novf, slot + nE, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_fail(e, "mesh_order", __FILE__, __LINE__);
  }
  if (st == PHFEM_OK) chk(dalloc_n(ctx, &m->nbr_ovf, (size_t)(novf > 0 ? novf : 1)));
  if (st == PHFEM_OK) {
    m->novf = novf;
    k_nbr16<<<grid_for(ctx, nE), kBlock, 0, s>>>(nE, m->perm, m->iperm, m->nbr, flag, slot, m->eclass, m->nbr16,
                                                 m->nbr_ovf, m->eclass_i);
    chk(check_launch(ctx, "k_nbr16"));
  }
  dfree(ctx, key);
  dfree(ctx, key2);
  dfree(ctx, val2);
  dfree(ctx, flag);
  dfree(ctx, slot);
  dfree(ctx, scratch);
  if (st != PHFEM_OK) {
    dfree(ctx, m->perm);
    dfree(ctx, m->iperm);
    dfree(ctx, m->nbr16);
    dfree(ctx, m->nbr_ovf);
    dfree(ctx, m->eclass_i);
    m->perm = m->iperm = nullptr;
    m->nbr16 = nullptr;
    m->nbr_ovf = nullptr;
    m->eclass_i = nullptr;
  }
  return st;
}

// Builds the visit order of the edge-row assembly pass, once per mesh: the
// tiles of kBlock consecutive edges (the paper's numbering, so each tile's
// rows are written coalesced) sorted by the Morton code of their mean
// midpoint.  An edge row reads the element records of its two triangles, and
// each record is read by the triangle's three edges; in the paper's edge
// order those three lie far apart (edges are numbered by their larger vertex,
// and red refinement numbers new vertices by coarse edge), so a record is
// fetched again from DRAM for most of its uses.  Visited in this order the
// three uses fall close together in time (a CPU model of the level-4
// L-shaped mesh: record lines fetched 2.6x their size in the paper's order,
// 1.07x in this one).
int mesh_row_tiles(phfem_mesh m) {
  if (m->row_tiles) return PHFEM_OK;
  phfem_ctx ctx = m->ctx;
  cudaStream_t s = ctx->stream;
  const int nE = m->info.nE, nV = m->info.nV;
  const int nt = (nE + kBlock - 1) / kBlock;
  uint32_t *key = nullptr, *key2 = nullptr;
  int32_t* val2 = nullptr;
  double* scratch = nullptr;  // partials [4][kMaxGrid], box [4], counter
  int st = PHFEM_OK;
  auto chk = [&](int r) {
    if (st == PHFEM_OK) st = r;
  };
  chk(dalloc_n(ctx, &m->row_tiles, (size_t)nt));
  chk(dalloc_n(ctx, &key, (size_t)nt));
  chk(dalloc_n(ctx, &key2, (size_t)nt));
  chk(dalloc_n(ctx, &val2, (size_t)nt));
  chk(dalloc_n(ctx, &scratch, 4 * (size_t)kMaxGrid + 8));
  if (st == PHFEM_OK) {
    double* box = scratch + 4 * kMaxGrid;
    unsigned int* counter = reinterpret_cast<unsigned int*>(box + 4);
    cudaMemsetAsync(counter, 0, sizeof(unsigned int), s);
    k_bbox<<<grid_for(ctx, nV), kBlock, 0, s>>>(nV, reinterpret_cast<const double2*>(m->xy), scratch, counter, box);
    chk(check_launch(ctx, "k_bbox"));
    k_tile_key<<<nt, kBlock, 0, s>>>(nE, m->ed2el, reinterpret_cast<const double2*>(m->xy), box, key, m->row_tiles);
    chk(check_launch(ctx, "k_tile_key"));
  }
  if (st == PHFEM_OK) chk(radix_sort_pairs(ctx, key, m->row_tiles, key2, val2, nt, 32));
  dfree(ctx, key);
  dfree(ctx, key2);
  dfree(ctx, val2);
  dfree(ctx, scratch);
  if (st != PHFEM_OK) {
    dfree(ctx, m->row_tiles);
    m->row_tiles = nullptr;
  }
  return st;
}

void mesh_order_free(phfem_mesh m) {
  phfem_ctx c = m->ctx;
  dfree(c, m->row_tiles);
  m->row_tiles = nullptr;
  dfree(c, m->perm);
  dfree(c, m->iperm);
  dfree(c, m->nbr16);
  dfree(c, m->nbr_ovf);
  dfree(c, m->eclass_i);
  m->perm = m->iperm = nullptr;
}

}  // namespace phfem

using namespace phfem;

extern "C" {

PHFEM_API int phfem_mesh_order(phfem_mesh mesh, int32_t* perm, int32_t* n_overflow) {
  if (!mesh) return fail(PHFEM_EINVAL, "phfem_mesh_order: NULL mesh");
  PH_TRY(mesh_order(mesh));
  cudaStream_t s = mesh->ctx->stream;
  if (perm)
    PH_CUDA(cudaMemcpyAsync(perm, mesh->perm, sizeof(int32_t) * mesh->info.nE, cudaMemcpyDeviceToDevice, s));
  if (n_overflow) *n_overflow = mesh->novf;
  PH_CUDA(cudaStreamSynchronize(s));
  return PHFEM_OK;
}

}  // extern "C"
