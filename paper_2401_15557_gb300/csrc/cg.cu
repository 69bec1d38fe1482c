// Jacobi-preconditioned conjugate gradients on the condensed trace-form edge
// system (Section 3.5 after elimination of the element unknowns) in the
// locality order of the edges (order.cu), two kernels per iteration; the
// product kernel stages each tile's own row data in shared memory with bulk
// copies (k_fcg_spmv_staged, the default for FP32 systems).
//
// Same method as the paper-order iteration of solve.cu (Jacobi-PCG with
// reliable updates: FP32 or FP64 inner vectors, FP64 true residual in
// difference form replacing the recursive one whenever it has fallen by
// inner_rtol, the direction kept with a line search or restarted), arranged
// to move fewer bytes per iteration:
//   * the operator rows are stored in the locality order: four l_es as one
//     16-byte (FP32) vector, the reaction part, and the neighbours as four
//     16-bit differences, so an operator product reads 28 bytes of matrix per
//     row in FP32 and its gathers hit lines that neighbouring rows just read;
//   * the preconditioned residual u = D^-1 r is the stored vector (r = u / d
//     is never needed), and the direction update p = u + beta p is folded
//     into the operator product: each row forms p at itself and at its four
//     neighbours from u and the previous p (four buffers in rotation), writes
//     its own p and q = S p, and sums p.q;
//   * the second kernel updates u and sums r.z = u.u / D^-1; every fourth
//     iteration it also adds alpha p of the last four directions (still in
//     their buffers) to the solution correction y, so y is read and written
//     once per four iterations;
//   * the solution is x = (xh + xl) + y: xh + xl an unevaluated FP64 pair
//     ("double-double"), y the correction since the last reliable update,
//     accumulated as an unevaluated pair of floats (FP32 systems: about 48
//     bits with FP32 arithmetic only) or in FP64.  At every reliable update
//     y (and any pending terms) is added into the pair and cleared, and the true
//     residual b - S x is evaluated from the pair: the solution then carries
//     more than FP64 precision, which the relative residual 1e-10 needs on
//     fine meshes, where b scales like h^2 while S does not and no FP64 vector
//     has a residual below ~1.3e-10 (L-shaped domain, h = 1/1024).
// The true residual evaluates (x_e - x_s) from the pairs (TwoSum on the
// leading parts), so its own rounding is ~2^-53 of sum |l_es (x_e - x_s)| per
// row; that estimate is the floor reported with the result.
#include <cmath>
#include <cstdio>
#include <cstdlib>

#include "kernels.cuh"

namespace phfem {

template <typename T>
struct Inner;
template <>
struct Inner<float> {
  using L4 = float4;  // the four l_es of a row
  using Y = float2;   // solution correction: unevaluated pair of floats
};
template <>
struct Inner<double> {
  struct __align__(32) L4 {
    double x, y, z, w;
  };
  using Y = double;
};

// Direction buffers of the iteration.  The fused FP32 iteration rotates
// through all four: the product kernel writes the direction after the
// newest, and the update kernel adds alpha p of four iterations to y at once
// every fourth iteration (the three before stay pending in their buffers).
// The unfused iteration uses buffer 0 only.
constexpr int kDirs = 4;
template <typename T>
struct Dirs {
  T* base;        // buffer 0
  size_t stride;  // elements from one buffer to the next
  __host__ __device__ T* b(int k) const { return base + (size_t)k * stride; }
};

struct FastCG {
  int n = 0;
  bool fp32 = true;
  void* l4 = nullptr;     // [n] Inner<T>::L4
  void* rd = nullptr;     // [n] T: reaction/mass part of the diagonal
  void* di = nullptr;     // [n] T: 1 / S_ee
  void* dg = nullptr;     // [n] T: S_ee (FP64 systems only)
  double* val = nullptr;  // [5][n] FP64 rows in difference form
  double* b = nullptr;    // [n] right-hand side of the current solve
  double* xh = nullptr;   // [n] solution, leading part
  double* xl = nullptr;   // [n] solution, trailing part
  void* y = nullptr;      // [n] Inner<T>::Y correction since the last reliable update
  void* vec = nullptr;    // u, q, the kDirs direction buffers: slots of `slot` bytes (256-aligned)
  size_t slot = 0;
  // resident blocks per SM of the iteration kernels, [F] (fused or not): the
  // grids are one wave of resident blocks, so no kernel runs a partial last
  // wave (the FP32 update kernel holds 3 blocks per SM, the product kernel 8)
  int per_spmv[2] = {1, 1}, per_update[2] = {1, 1}, per_dir = 1, per_staged = 1;
  void* u() const { return vec; }
  void* q() const { return (char*)vec + slot; }
  void* pk(int k) const { return (char*)vec + (2 + k) * slot; }
  template <typename T>
  Dirs<T> dirs() const {
    return Dirs<T>{(T*)pk(0), slot / sizeof(T)};
  }
};

namespace {

__device__ __forceinline__ void row_nbrs(const short4* __restrict__ nb, const int4* __restrict__ ovf, int i,
                                         int c[4]) {
  const short4 s = __ldg(nb + i);
  if (s.x != (short)-32768) {
    c[0] = i + s.x;
    c[1] = i + s.y;
    c[2] = i + s.z;
    c[3] = i + s.w;
  } else {
    const int k = (int)(uint16_t)s.y | ((int)(uint16_t)s.z << 16);
    const int4 o = __ldg(ovf + k);
    c[0] = o.x;
    c[1] = o.y;
    c[2] = o.z;
    c[3] = o.w;
  }
}

__device__ __forceinline__ void load_l4(const float4* __restrict__ l, int i, float v[4]) {
  const float4 a = __ldg(l + i);
  v[0] = a.x;
  v[1] = a.y;
  v[2] = a.z;
  v[3] = a.w;
}
__device__ __forceinline__ void load_l4(const Inner<double>::L4* __restrict__ l, int i, double v[4]) {
  const double2* p = reinterpret_cast<const double2*>(l + i);
  const double2 a = __ldg(p), b = __ldg(p + 1);
  v[0] = a.x;
  v[1] = a.y;
  v[2] = b.x;
  v[3] = b.y;
}

// Tiles the product kernel prefetches into L2 ahead of the one it processes:
// one tile is a visit later, ~3 us at level 5, several DRAM latencies;
// 2 and 4 were slower (the prefetched lines are evicted before use).
constexpr int kPrefetchAhead = 1;

// L2 prefetch of bytes (rounded down to 16) from a 16-byte aligned address
// by the bulk-copy engine; no registers, no completion to wait for.
__device__ __forceinline__ void prefetch_l2(const void* a, int bytes) {
  bytes &= ~15;
  if (bytes > 0) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"(bytes) : "memory");
}


__device__ __forceinline__ double y_value(float2 y) { return (double)y.x + (double)y.y; }
__device__ __forceinline__ double y_value(double y) { return y; }
__device__ __forceinline__ void y_zero(float2& y) { y = make_float2(0.f, 0.f); }
__device__ __forceinline__ void y_zero(double& y) { y = 0.0; }

// Operator rows in the locality order (once per system).
template <typename T>
__global__ void k_fcg_op(int n, const int32_t* __restrict__ perm, const T* __restrict__ lval,
                         const T* __restrict__ rdiag, const T* __restrict__ dinv, const double* __restrict__ val,
                         typename Inner<T>::L4* __restrict__ l4, T* __restrict__ rd, T* __restrict__ di,
                         T* __restrict__ dg, double* __restrict__ vi) {
  const size_t m = (size_t)n;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int e = perm[i];
    typename Inner<T>::L4 l;
    l.x = lval[e];
    l.y = lval[m + e];
    l.z = lval[2 * m + e];
    l.w = lval[3 * m + e];
    l4[i] = l;
    rd[i] = rdiag[e];
    di[i] = dinv[e];
    double v[5];
#pragma unroll
    for (int s = 0; s < 5; ++s) {
      v[s] = val[s * m + e];
      vi[s * m + i] = v[s];
    }
    if (dg) dg[i] = (T)((((v[0] + v[1]) + v[2]) + v[3]) + v[4]);  // the diagonal, summed as assembled
  }
}

// Start of a solve: b and x from the paper's order, y = 0.
template <typename Y>
__global__ void k_fcg_in(int n, const int32_t* __restrict__ perm, const double* __restrict__ b_paper,
                         const double* __restrict__ x_paper, double* __restrict__ b, double* __restrict__ xh,
                         double* __restrict__ xl, Y* __restrict__ y, SolveState* st) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->ypend = 0;
    st->sc = 1.0;
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int e = perm[i];
    b[i] = b_paper[e];
    xh[i] = x_paper[e];
    xl[i] = 0.0;
    Y z;
    y_zero(z);
    y[i] = z;
  }
}

// The pending terms of the fused FP32 iteration: alpha p of the newest
// ypend directions, oldest first (the update adds four iterations' terms to
// y at once), or 0.
template <typename T>
__device__ __forceinline__ double pending_terms(const SolveState* st, const Dirs<const T>& d, int i) {
  double s = 0.0;
  for (int j = st->ypend - 1; j >= 0; --j) {
    const int k = (st->par - j) & (kDirs - 1);
    s += st->alpha_dir[k] * (double)d.b(k)[i];
  }
  return s;
}

// y and the pending terms carry the scale of the inner vectors (a power of
// two): dividing by it is exact.
template <typename Y, typename T>
__device__ __forceinline__ double correction(const SolveState* st, const Y& y, const Dirs<const T>& d, int i) {
  return (y_value(y) + pending_terms(st, d, i)) / st->sc;
}

// End of a solve: x = (xh + xl) + y (+ pending terms), rounded to FP64, in
// the paper's order.
template <typename Y, typename T>
__global__ void k_fcg_out(int n, const int32_t* __restrict__ perm, const double* __restrict__ xh,
                          const double* __restrict__ xl, const Y* __restrict__ y, Dirs<const T> d,
                          const SolveState* st, double* __restrict__ x_paper) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double h = xh[i], l = xl[i];
    dd_add(h, l, correction(st, y[i], d, i));
    x_paper[perm[i]] = h + l;
  }
}

// (xh, xl) += y (+ pending terms), y = 0; with cond only when the iteration
// asked for a reliable update (done == 1).  The residual kernel that follows
// clears the pending count.
template <typename Y, typename T>
__global__ void k_fcg_fold(int n, double* __restrict__ xh, double* __restrict__ xl, Y* __restrict__ y,
                           Dirs<const T> d, const SolveState* st, int cond) {
  if (cond && st->done != 1) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double h = xh[i], l = xl[i];
    Y v = y[i];
    dd_add(h, l, correction(st, v, d, i));
    xh[i] = h;
    xl[i] = l;
    y_zero(v);
    y[i] = v;
  }
}

// The kernels take F (fused): true folds the direction update p = u + beta p
// into the operator product (FP32 systems may choose it); false runs it as a
// kernel of its own after the update, which FP64 systems always do: on GB300
// FP64 arithmetic, not memory, bounds their iteration, and forming p at the
// four neighbours would add four FP64 operations per row.

__device__ __forceinline__ float fmadd(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmadd(double a, double b, double c) { return __fma_rn(a, b, c); }

// True residual r = b - S x (FP64, difference form, x = xh + xl) and the
// start of the inner iteration from it: u = D^-1 r, r.z, r.p for the line
// search, ||r||^2 and the evaluation floor.  Modes as in solve.cu: 0 the norm
// of the free-edge right-hand side with the Dirichlet lifting, 1 start, 2
// reliable update, 3 = 2 only if the iteration asked for it.
// Directions: at the start p = u (unfused: written here; fused: by the next
// product kernel in restart mode).  At a reliable update the kept direction
// is the one the next iteration would have taken, p = u + beta p with the
// recursive u: the unfused iteration already formed it before pausing, the
// fused one forms it here from the recursive u before u is replaced.
// Scaling: the inner vectors of the next cycle carry sc, a power of two that
// brings the previous true residual (or b at the start) to an RMS of about
// one per row, so FP32 quantities and their squares stay in range whatever
// the size of the data; alpha and beta do not depend on it, the kept
// direction is rescaled by sc_new / sc_old (exact), and y is divided by sc
// when it is folded into the solution.
template <typename T, bool F>
__global__ void k_fcg_residual(int n, const short4* __restrict__ nb, const int4* __restrict__ ovf,
                               const double* __restrict__ val, const double* __restrict__ b,
                               const double* __restrict__ xh, const double* __restrict__ xl,
                               const uint8_t* __restrict__ ecl, uint8_t ident, const T* __restrict__ di,
                               const T* __restrict__ dg, T* __restrict__ u, Dirs<T> dirs, double* partials,
                               SolveState* st, double rtol2, double inner_rtol2, int mode) {
  if (mode == 3) {
    if (st->done != 1) return;  // every block reads done before the last block rewrites it
    mode = 2;
  }
  __shared__ double smem[kBlock / 32];
  const size_t m = (size_t)n;
  T* __restrict__ pc = dirs.b(F ? st->par & (kDirs - 1) : 0);
  const T beta = (T)st->beta;
  double sc = 1.0;  // scale of the next cycle's inner vectors
  if (mode != 0) {
    const double prev = mode == 1 ? st->bb : st->rr64;
    if (prev > 0.0 && isfinite(prev)) {
      const int ex = ilogb(sqrt(prev / (double)n));
      sc = ldexp(1.0, -max(-900, min(900, ex)));
    }
  }
  const T ratio = (T)(sc / st->sc);  // a power of two
  double acc_r = 0.0, acc_z = 0.0, acc_f = 0.0, acc_p = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int c[4];
    row_nbrs(nb, ovf, i, c);
    if (mode == 0) {
      double r = 0.0;
      if (ecl[i] != ident) {
        r = b[i];
#pragma unroll
        for (int s = 0; s < 4; ++s)
          if (c[s] != i && ecl[c[s]] == ident) r += val[(s + 1) * m + i] * b[c[s]];
      }
      acc_r += r * r;
      continue;
    }
    const double he = xh[i], le = xl[i];
    const double rho = val[i];
    double sx = rho * he + rho * le;
    double fl = fabs(rho * he);
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const double l = val[(s + 1) * m + i];
      const double nh = -xh[c[s]];
      const double sh = he + nh;  // (x_e - x_s) from the pairs: TwoSum of the leading parts
      const double bb = sh - he;
      const double eh = (he - (sh - bb)) + (nh - bb);
      const double d = sh + (eh + (le - xl[c[s]]));
      sx += l * d;
      fl += fabs(l * d);
    }
    const double r = b[i] - sx;
    acc_r += r * r;
    fl *= 0x1p-53;
    acc_f += fl * fl;
    const double dd = (double)di[i];
    const double rs = sc * r;
    const T ue = (T)(dd * rs);
    if (mode == 1 && !F) pc[i] = ue;
    if (mode == 2) {
      T pk = pc[i];
      if (F) pk = fmadd(beta, pk, u[i]);
      pk *= ratio;
      pc[i] = pk;
      acc_p += rs * (double)pk;
    }
    u[i] = ue;
    if constexpr (sizeof(T) == sizeof(float)) acc_z += dd > 0.0 ? (double)ue * (double)ue / dd : 0.0;
    else acc_z += (double)ue * (double)ue * (double)dg[i];  // the stored diagonal: FP64 systems only
  }
  acc_r = block_sum(acc_r, smem);
  acc_z = block_sum(acc_z, smem);
  acc_f = block_sum(acc_f, smem);
  acc_p = block_sum(acc_p, smem);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = acc_r;
    partials[kMaxGrid + blockIdx.x] = acc_z;
    partials[2 * kMaxGrid + blockIdx.x] = acc_f;
    partials[3 * kMaxGrid + blockIdx.x] = acc_p;
  }
  if (!arrive_last(&st->counter[0])) return;
  const double rr = sum_partials(partials, smem);
  const double rz = sum_partials(partials + kMaxGrid, smem);
  const double ff = sum_partials(partials + 2 * kMaxGrid, smem);
  const double rp = sum_partials(partials + 3 * kMaxGrid, smem);
  if (threadIdx.x == 0) {
    st->counter[0] = 0;
    if (mode == 0) {
      st->bb = rr;
      return;
    }
    const double rsc = sc / st->sc;
    st->rz *= rsc * rsc;  // the recursive r.z in the new scale, for decide's comparison
    decide(st, rr, rz, ff, rp, mode, rtol2, inner_rtol2);
    st->sc = sc;
    st->ypend = 0;  // folded into the pair before this residual
    if (mode == 1 && F) st->restart = 1;  // the product kernel forms p = u
  }
}

// q = S p with, fused (F), the direction update folded in: p = u + beta
// p_old (restart: p = u; right after a reliable update that keeps the
// direction: p = p_old) at the row and at its four neighbours, the same
// rounded operation for every row, so all rows use the same p.  p_old is read
// from the newest direction buffer and p written to the next one; the last
// block advances the rotation.
// Unfused: the stored p (restart: p = u, each row writing its own p).  Then
// p.q -> alpha = r.z / p.q (or r.p / p.q after a reliable update).
// One row per thread and grid stride, at full occupancy; the gathers go
// through L1 and L2 (in the locality order most neighbours were just read by
// nearby rows); the bulk L2 prefetch of the next tile takes the DRAM latency
// out of the chain index load -> gathers (93 -> 83 us at level 5).  Measured
// variants without it (tiles staged in shared memory, with and without
// cp.async; several rows per thread; a software pipeline over rows;
// contiguous runs of tiles per block) were all slower on GB300.
template <typename T, bool F>
__global__ void __launch_bounds__(kBlock) k_fcg_spmv(int n, const short4* __restrict__ nb,
                                                     const int4* __restrict__ ovf,
                                                     const typename Inner<T>::L4* __restrict__ lv,
                                                     const T* __restrict__ rd, const T* __restrict__ u, Dirs<T> dirs,
                                                     T* __restrict__ q, double* partials, SolveState* st,
                                                     int ahead) {
  // The block visits tiles of kBlock rows, blockIdx.x + k gridDim.x.  The
  // five streamed arrays of the tile `ahead` visits on are prefetched into L2
  // by the bulk-copy engine (the neighbour differences are then an L2 hit,
  // and the gathers that depend on them wait for L2 instead of DRAM).  L2 is
  // the point of coherence, so the first tiles are prefetched before the wait
  // on the previous kernel.
  const int ntiles = (n + kBlock - 1) / kBlock;
  auto tile = [&](int k) { return blockIdx.x + k * (int)gridDim.x; };
  // the previous direction's buffer: before the wait a hint (a stale value
  // costs one useless prefetch), after it the value read below
  const T* pfo = dirs.b(F ? (*(volatile const int*)&st->par) & (kDirs - 1) : 0);
  auto prefetch = [&](int k) {
    const int t = tile(k);
    if (t >= ntiles || threadIdx.x >= 5) return;
    const int r0 = t * kBlock, cnt = min(kBlock, n - r0);
    switch (threadIdx.x) {
      case 0: prefetch_l2(nb + r0, cnt * sizeof(short4)); break;
      case 1: prefetch_l2(lv + r0, cnt * sizeof(typename Inner<T>::L4)); break;
      case 2: prefetch_l2(rd + r0, cnt * sizeof(T)); break;
      case 3: prefetch_l2(u + r0, cnt * sizeof(T)); break;
      default: prefetch_l2(pfo + r0, cnt * sizeof(T)); break;
    }
  };
  for (int k = 0; k < ahead; ++k) prefetch(k);
  pdl_enter();
  if (!F && blockIdx.x == 0 && threadIdx.x == 0) st->dir_pending = 0;  // no block of this kernel reads it
  if (st->done) return;
  const int par = F ? st->par & (kDirs - 1) : 0;
  const T* __restrict__ po = dirs.b(par);
  T* __restrict__ pn = dirs.b(F ? (par + 1) & (kDirs - 1) : 0);
  pfo = po;
  const int mode = st->restart ? 1 : (st->use_rp ? 2 : 0);
  const T beta = (T)st->beta;
  __shared__ double smem[kBlock / 32];
  auto pval = [&](T uv, T pv) -> T {
    if (mode == 1) return uv;
    if (F && mode == 0) return fmadd(beta, pv, uv);
    return pv;
  };
  T acc = (T)0;  // this thread's few rows in T; across threads and blocks in FP64
  for (int k = 0;; ++k) {
    const int t = tile(k);
    if (t >= ntiles) break;
    if (ahead) prefetch(k + ahead);
    const int i = t * kBlock + threadIdx.x;
    if (i >= n) continue;
    int c[4];
    row_nbrs(nb, ovf, i, c);
    T l[4];
    load_l4(lv, i, l);
    const T pe = pval(mode != 2 ? __ldg(u + i) : (T)0, mode != 1 ? __ldg(po + i) : (T)0);
    T gu[4], gp[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      gu[m] = mode != 2 ? __ldg(u + c[m]) : (T)0;
      gp[m] = mode != 1 ? __ldg(po + c[m]) : (T)0;
    }
    T s = __ldg(rd + i) * pe;
#pragma unroll
    for (int m = 0; m < 4; ++m) s = fmadd(l[m], pe - pval(gu[m], gp[m]), s);
    if (F || mode == 1) pn[i] = pe;
    q[i] = s;
    acc = fmadd(pe, s, acc);
  }
  const double accd = block_sum((double)acc, smem);
  if (threadIdx.x == 0) partials[blockIdx.x] = accd;
  if (!arrive_last(&st->counter[1])) return;
  const double pq = sum_partials(partials, smem);
  if (threadIdx.x == 0) {
    st->counter[1] = 0;
    if (F) st->par = (par + 1) & (kDirs - 1);
    if (!(pq > 0.0) || !isfinite(pq)) {
      st->done = 3;
      st->status = isfinite(pq) ? PHFEM_EBREAKDOWN : PHFEM_ENAN;
    } else {
      const double a = (st->use_rp ? st->rp : st->rz) / pq;
      st->alpha = a;
      st->alpha_f[0] = (float)a;  // the pair the FP32 update kernel uses (no FP64 work per thread there)
      st->alpha_f[1] = (float)(a - (double)(float)a);
      st->use_rp = 0;
      st->restart = 0;
    }
  }
}

// ---- product kernel with the tile's row data staged in shared memory ----
// One stage holds a tile's neighbour differences, l_es, reaction part, u and
// p_old, copied by the bulk-copy engine (one thread issues five
// cp.async.bulk copies, completion counted on an mbarrier); two stages, the
// copies of a tile issued two tiles ahead.
struct __align__(16) FStage {
  short4 nb[kBlock];
  float4 l4[kBlock];
  float rd[kBlock];
  float u[kBlock];
  float po[kBlock];
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes, uint64_t* b) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(b))
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
// Waits for the phase of parity `parity` to complete; false after a second
// (the copies of a tile take microseconds: a second means they never will).
__device__ __forceinline__ bool mbar_wait(uint64_t* b, unsigned parity) {
  const uint64_t t0 = global_ns();
  for (;;) {
    if (mbar_try_wait(b, parity)) return true;
    if (global_ns() - t0 > 1000000000ull) return false;
  }
}

// The fused FP32 product kernel of k_fcg_spmv<float, true>, the row's own data
// read from the staged tile: the neighbour differences are then a shared-memory
// load, and only the gathers of u and p_old at the neighbours go to L1 and L2.
// The copies are issued after the wait on the previous kernel (unlike an L2
// prefetch, a shared-memory copy is not updated by later writes).  If a copy
// never completes the block records PHFEM_ECUDA, waits (bounded) for the copies
// it still has in flight and leaves the tile loop.
__global__ void __launch_bounds__(kBlock) k_fcg_spmv_staged(int n, const short4* __restrict__ nb,
                                                            const int4* __restrict__ ovf,
                                                            const float4* __restrict__ lv,
                                                            const float* __restrict__ rd, const float* __restrict__ u,
                                                            Dirs<float> dirs, float* __restrict__ q, double* partials,
                                                            SolveState* st) {
  __shared__ FStage stage[2];
  __shared__ uint64_t bar[2];
  __shared__ double smem[kBlock / 32];
  __shared__ int s_fail;
  const int ntiles = (n + kBlock - 1) / kBlock;
  auto tile = [&](int k) { return blockIdx.x + k * (int)gridDim.x; };
  if (threadIdx.x < 3 && tile(0) < ntiles) {  // the first tile's static arrays into L2 before the wait
    const int r0 = tile(0) * kBlock, cnt = min(kBlock, n - r0);
    if (threadIdx.x == 0) prefetch_l2(nb + r0, cnt * (int)sizeof(short4));
    if (threadIdx.x == 1) prefetch_l2(lv + r0, cnt * (int)sizeof(float4));
    if (threadIdx.x == 2) prefetch_l2(rd + r0, cnt * (int)sizeof(float));
  }
  pdl_enter();
  if (st->done) return;
  const int par = st->par & (kDirs - 1);
  const float* __restrict__ po = dirs.b(par);
  float* __restrict__ pn = dirs.b((par + 1) & (kDirs - 1));
  const int mode = st->restart ? 1 : (st->use_rp ? 2 : 0);
  const float beta = (float)st->beta;
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  auto issue = [&](int k) {  // thread 0: the copies of the block's k-th tile into stage k & 1
    const int t = tile(k);
    if (t >= ntiles) return;
    const int r0 = t * kBlock, cnt = min(kBlock, n - r0);
    FStage& S = stage[k & 1];
    const unsigned b8 = (unsigned)(cnt * 8 + 15) & ~15u, b16 = (unsigned)cnt * 16u,
                   b4 = (unsigned)(cnt * 4 + 15) & ~15u;  // rounded up to 16: the arrays are padded for it
    mbar_expect_tx(&bar[k & 1], b8 + b16 + 3 * b4);
    bulk_copy_g2s(S.nb, nb + r0, b8, &bar[k & 1]);
    bulk_copy_g2s(S.l4, lv + r0, b16, &bar[k & 1]);
    bulk_copy_g2s(S.rd, rd + r0, b4, &bar[k & 1]);
    bulk_copy_g2s(S.u, u + r0, b4, &bar[k & 1]);
    bulk_copy_g2s(S.po, po + r0, b4, &bar[k & 1]);
  };
  if (threadIdx.x == 0) {
    issue(0);
    issue(1);
  }
  auto pval = [&](float uv, float pv) -> float {
    if (mode == 1) return uv;
    if (mode == 0) return fmadd(beta, pv, uv);
    return pv;
  };
  float acc = 0.f;
  int k = 0;
  for (;; ++k) {
    const int t = tile(k);
    if (t >= ntiles) break;
    if (!mbar_wait(&bar[k & 1], (k >> 1) & 1)) s_fail = 1;
    const FStage& S = stage[k & 1];
    const int i = t * kBlock + threadIdx.x;
    if (i < n && !s_fail) {
      const short4 s4 = S.nb[threadIdx.x];
      int c[4];
      if (s4.x != (short)-32768) {
        c[0] = i + s4.x;
        c[1] = i + s4.y;
        c[2] = i + s4.z;
        c[3] = i + s4.w;
      } else {
        const int4 o = __ldg(ovf + ((int)(uint16_t)s4.y | ((int)(uint16_t)s4.z << 16)));
        c[0] = o.x;
        c[1] = o.y;
        c[2] = o.z;
        c[3] = o.w;
      }
      float gu[4], gp[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        gu[m] = mode != 2 ? __ldg(u + c[m]) : 0.f;
        gp[m] = mode != 1 ? __ldg(po + c[m]) : 0.f;
      }
      const float4 l = S.l4[threadIdx.x];
      const float pe = pval(S.u[threadIdx.x], S.po[threadIdx.x]);
      float sv = S.rd[threadIdx.x] * pe;
      sv = fmadd(l.x, pe - pval(gu[0], gp[0]), sv);
      sv = fmadd(l.y, pe - pval(gu[1], gp[1]), sv);
      sv = fmadd(l.z, pe - pval(gu[2], gp[2]), sv);
      sv = fmadd(l.w, pe - pval(gu[3], gp[3]), sv);
      pn[i] = pe;
      q[i] = sv;
      acc = fmadd(pe, sv, acc);
    }
    __syncthreads();  // the stage is read: it may be refilled
    if (s_fail) break;
    if (threadIdx.x == 0) issue(k + 2);
  }
  if (s_fail && threadIdx.x == 0) {
    // the copies still in flight (tiles k and k + 1, issued before the
    // failure) land in this block's shared memory: wait for them, bounded,
    // before leaving
    mbar_wait(&bar[k & 1], (k >> 1) & 1);
    if (tile(k + 1) < ntiles) mbar_wait(&bar[(k + 1) & 1], ((k + 1) >> 1) & 1);
    st->status = PHFEM_ECUDA;
    st->done = 3;
  }
  const double accd = block_sum((double)acc, smem);
  if (threadIdx.x == 0) partials[blockIdx.x] = accd;
  if (!arrive_last(&st->counter[1])) return;
  const double pq = sum_partials(partials, smem);
  if (threadIdx.x == 0) {
    st->counter[1] = 0;
    st->par = (par + 1) & (kDirs - 1);
    if (st->done == 3) return;
    if (!(pq > 0.0) || !isfinite(pq)) {
      st->done = 3;
      st->status = isfinite(pq) ? PHFEM_EBREAKDOWN : PHFEM_ENAN;
    } else {
      const double a = (st->use_rp ? st->rp : st->rz) / pq;
      st->alpha = a;
      st->alpha_f[0] = (float)a;
      st->alpha_f[1] = (float)(a - (double)(float)a);
      st->use_rp = 0;
      st->restart = 0;
    }
  }
}

// One row of the update: u -= alpha D^-1 q and its r.z term.
__device__ __forceinline__ void update_u(float qe, float d, float& ue, float ah, float& acc) {
  ue = fmadd(-ah, d * qe, ue);
  acc += d > 0.f ? __fdividef(ue * ue, d) : 0.f;
}
__device__ __forceinline__ void update_u4(const float4& qv, const float4& dv, float4& uv, float ah, float& acc) {
  update_u(qv.x, dv.x, uv.x, ah, acc);
  update_u(qv.y, dv.y, uv.y, ah, acc);
  update_u(qv.z, dv.z, uv.z, ah, acc);
  update_u(qv.w, dv.w, uv.w, ah, acc);
}

// u -= alpha D^-1 q, r.z = u.u / D^-1 (FP32) or u.u D (FP64, with the stored
// diagonal: no FP64 division) -> beta, and the solution correction y.
// Fused FP32: the directions of the last kDirs iterations are still in their
// buffers, so every kDirs-th iteration y takes their kDirs terms alpha p at
// once, oldest first (the other iterations leave alpha p pending, which the
// fold and the end of the solve add); then the test of the recursive residual
// (done = 1 asks for a reliable update).  Unfused: y += alpha p every
// iteration, and the direction kernel follows and tests the residual.  FP32
// rows go four at a time through 16-byte loads and stores: two groups of four
// per thread and pass (all loads issued before the first store) when y is not
// touched, one group with its directions and y when it is.
template <typename T, bool F>
__global__ void __launch_bounds__(kBlock) k_fcg_update(int n, Dirs<const T> dirs, const T* __restrict__ q,
                                                       const T* __restrict__ di, const T* __restrict__ dg,
                                                       T* __restrict__ u, typename Inner<T>::Y* __restrict__ y,
                                                       double* partials, SolveState* st) {
  pdl_enter();
  if (st->done) return;
  const int par = F ? st->par & (kDirs - 1) : 0;
  const double a64 = st->alpha;
  T ah, al;
  if constexpr (sizeof(T) == sizeof(float)) {
    ah = st->alpha_f[0];
    al = st->alpha_f[1];
  } else {
    ah = a64;
    al = 0.0;
  }
  const int pend = F ? st->ypend : 0;
  __shared__ double smem[kBlock / 32];
  T acc = (T)0;
  if constexpr (sizeof(T) == sizeof(float)) {
    constexpr int NT = F ? kDirs : 1;  // terms added to y when it is touched
    const bool with_y = !F || pend == kDirs - 1;
    const int n4 = n / 4;
    const int stride = gridDim.x * blockDim.x;
    const float4* __restrict__ q4 = reinterpret_cast<const float4*>(q);
    const float4* __restrict__ d4 = reinterpret_cast<const float4*>(di);
    float4* __restrict__ u4 = reinterpret_cast<float4*>(u);
    // term t: the direction in buffer par + 1 + t (fused: oldest first, the
    // last one this iteration's), its alpha as a pair of floats
    const float* pt[NT];
    float th[NT], tl[NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      const int k = F ? (par + 1 + t) & (kDirs - 1) : 0;
      pt[t] = dirs.b(k);
      th[t] = t < NT - 1 ? st->alpha_dir_f[k][0] : ah;
      tl[t] = t < NT - 1 ? st->alpha_dir_f[k][1] : al;
    }
    if (!with_y) {
      for (int j0 = blockIdx.x * blockDim.x + threadIdx.x; j0 < n4; j0 += 2 * stride) {
        float4 qv[2], dv[2], uv[2];
        bool ok[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int j = j0 + h * stride;
          ok[h] = j < n4;
          if (ok[h]) {
            qv[h] = q4[j];
            dv[h] = d4[j];
            uv[h] = u4[j];
          }
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          if (!ok[h]) continue;
          update_u4(qv[h], dv[h], uv[h], ah, acc);
          u4[j0 + h * stride] = uv[h];
        }
      }
    } else {
      float4* __restrict__ y4 = reinterpret_cast<float4*>(y);  // two rows' pairs per float4
      for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n4; j += stride) {
        float4 pv[NT];
#pragma unroll
        for (int t = 0; t < NT; ++t) pv[t] = reinterpret_cast<const float4*>(pt[t])[j];
        const float4 qv = q4[j], dv = d4[j];
        float4 uv = u4[j];
        const float4 ya = y4[2 * j], yb = y4[2 * j + 1];
        float2 y0 = make_float2(ya.x, ya.y), y1 = make_float2(ya.z, ya.w);
        float2 y2 = make_float2(yb.x, yb.y), y3 = make_float2(yb.z, yb.w);
#pragma unroll
        for (int t = 0; t < NT; ++t) {
          y0 = y_add(y0, th[t], tl[t], pv[t].x);
          y1 = y_add(y1, th[t], tl[t], pv[t].y);
          y2 = y_add(y2, th[t], tl[t], pv[t].z);
          y3 = y_add(y3, th[t], tl[t], pv[t].w);
        }
        update_u4(qv, dv, uv, ah, acc);
        u4[j] = uv;
        y4[2 * j] = make_float4(y0.x, y0.y, y1.x, y1.y);
        y4[2 * j + 1] = make_float4(y2.x, y2.y, y3.x, y3.y);
      }
    }
    // the last n % 4 rows
    const int i = 4 * n4 + blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
      if (with_y) {
        float2 yi = y[i];
#pragma unroll
        for (int t = 0; t < NT; ++t) yi = y_add(yi, th[t], tl[t], pt[t][i]);
        y[i] = yi;
      }
      float ue = u[i];
      update_u(q[i], di[i], ue, ah, acc);
      u[i] = ue;
    }
  } else {
    const T* __restrict__ p = dirs.b(0);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
      y[i] = y_add(y[i], ah, al, p[i]);
      const T d = di[i];
      const T ue = fmadd(-ah, d * q[i], u[i]);
      u[i] = ue;
      acc = fmadd(ue * ue, dg[i], acc);
    }
  }
  const double accd = block_sum((double)acc, smem);
  if (threadIdx.x == 0) partials[kMaxGrid + blockIdx.x] = accd;
  if (!arrive_last(&st->counter[2])) return;
  const double rz = sum_partials(partials + kMaxGrid, smem);
  if (threadIdx.x == 0) {
    st->counter[2] = 0;
    st->beta = st->rz > 0.0 ? rz / st->rz : 0.0;
    st->rz = rz;
    st->it += 1;
    if (F) {  // alpha p of this iteration stays pending unless y took it
      st->alpha_dir[par] = a64;
      st->alpha_dir_f[par][0] = (float)ah;
      st->alpha_dir_f[par][1] = (float)al;
      st->ypend = pend == kDirs - 1 ? 0 : pend + 1;
    }
    if (!isfinite(rz)) {
      st->done = 3;
      st->status = PHFEM_ENAN;
    } else if (F && rz <= st->tol2) {
      st->done = 1;
    } else if (!F) {
      st->dir_pending = 1;
    }
  }
}

// Unfused: p = u + beta p, then the test of the recursive residual, so that
// the direction is complete when the iteration pauses for a reliable update.
// Runs only after an update kernel that did run (dir_pending).
template <typename T>
__global__ void __launch_bounds__(kBlock) k_fcg_dir(int n, const T* __restrict__ u, T* __restrict__ p,
                                                    SolveState* st) {
  pdl_enter();
  if (!st->dir_pending) return;
  const T beta = (T)st->beta;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = fmadd(beta, p[i], u[i]);
  if (blockIdx.x == 0 && threadIdx.x == 0 && st->done == 0 && st->rz <= st->tol2) st->done = 1;
}

__global__ void k_fcg_loop_control(SolveState* st, cudaGraphConditionalHandle handle, int max_iter,
                                   int max_bodies) {
  st->bodies += 1;
  const bool more = st->done == 0 && st->it < max_iter && st->bodies < max_bodies;
  cudaGraphSetConditional(handle, more ? 1u : 0u);
}

// The L2 window of the iteration: u, written by the update kernel and read
// (at every row and gathered at its neighbours) by the next product kernel,
// and read and written again by the next update, stays in L2 with the
// set-aside sized to it; the streamed operator, q, the directions and y pass
// through the rest of L2.  Measured at level 5 (FP32, us per iteration): no
// window 122.2, u 114.9, q 119.2, u and q 124.2 (a 75 MB set-aside leaves too
// little L2 for the gathers and the prefetched tiles).  Only when u fits the
// largest set-aside; while a graph is captured (capturing) the set-aside,
// which is device-wide, is not changed: the window is used only if the
// set-aside already has its size.
L2Window u_window(phfem_sys sys, bool capturing) {
  phfem_ctx ctx = sys->mesh->ctx;
  const FastCG* f = sys->fcg;
  L2Window w;
  const size_t want = f->slot;
  if (!ctx->l2_window || want > ctx->l2_persist_max || want > ctx->l2_window_max) {
    if (ctx->l2_window && !capturing) set_l2_limit(ctx, 0);
    return w;
  }
  if (capturing ? ctx->l2_limit != want : !set_l2_limit(ctx, want)) return w;
  w.base = f->u();
  w.bytes = want;
  w.hit_ratio = 1.0f;
  return w;
}

template <typename T, bool F>
struct FLaunch {
  using L4 = typename Inner<T>::L4;
  using Y = typename Inner<T>::Y;
  phfem_sys sys;
  cudaStream_t s;
  int g, n;
  double rtol2, irtol2;
  L2Window win;
  const FastCG* f() const { return sys->fcg; }
  int prologue() const {
    phfem_ctx ctx = sys->mesh->ctx;
    k_fcg_in<Y><<<g, kBlock, 0, s>>>(n, sys->mesh->perm, sys->b, sys->x, f()->b, f()->xh, f()->xl, (Y*)f()->y,
                                     sys->st);
    return check_launch(ctx, "k_fcg_in");
  }
  int epilogue() const {
    phfem_ctx ctx = sys->mesh->ctx;
    k_fcg_out<Y, T><<<g, kBlock, 0, s>>>(n, sys->mesh->perm, f()->xh, f()->xl, (const Y*)f()->y,
                                         f()->template dirs<const T>(), sys->st, sys->x);
    return check_launch(ctx, "k_fcg_out");
  }
  int residual(int mode) const {
    phfem_ctx ctx = sys->mesh->ctx;
    phfem_mesh m = sys->mesh;
    if (mode >= 2) {
      k_fcg_fold<Y, T><<<g, kBlock, 0, s>>>(n, f()->xh, f()->xl, (Y*)f()->y, f()->template dirs<const T>(), sys->st,
                                            mode == 3);
      PH_TRY(check_launch(ctx, "k_fcg_fold"));
    }
    prof_start(ctx, kProfResidual);
    k_fcg_residual<T, F><<<g, kBlock, 0, s>>>(n, m->nbr16, m->nbr_ovf, f()->val, f()->b, f()->xh, f()->xl,
                                           m->eclass_i, sys->ident_class, (const T*)f()->di, (const T*)f()->dg,
                                           (T*)f()->u(), f()->template dirs<T>(), sys->partials, sys->st,
                                           rtol2, irtol2, mode);
    prof_stop(ctx, kProfResidual);
    return check_launch(ctx, "k_fcg_residual");
  }
  int wave(int per) const {
    phfem_ctx ctx = sys->mesh->ctx;
    int64_t g = (int64_t)ctx->num_sms * per;
    const int64_t need = (n + kBlock - 1) / kBlock;
    if (g > kMaxGrid) g = kMaxGrid;
    if (g > need) g = need;
    return g < 1 ? 1 : (int)g;
  }
  int iteration() const {
    phfem_ctx ctx = sys->mesh->ctx;
    phfem_mesh m = sys->mesh;
    prof_start(ctx, kProfSpmv);
    bool staged = false;
    if constexpr (F && sizeof(T) == sizeof(float)) {
      if (sys->mesh->ctx->cg_variant == 0) {
        PH_CUDA(launch_pdl_w(win, k_fcg_spmv_staged, wave(f()->per_staged), s, n, (const short4*)m->nbr16,
                             (const int4*)m->nbr_ovf, (const float4*)f()->l4, (const float*)f()->rd,
                             (const float*)f()->u(), f()->template dirs<float>(), (float*)f()->q(), sys->partials,
                             sys->st));
        staged = true;
      }
    }
    if (!staged)
    PH_CUDA(launch_pdl_w(win, k_fcg_spmv<T, F>, wave(f()->per_spmv[F]), s, n, (const short4*)m->nbr16, (const int4*)m->nbr_ovf,
                       (const L4*)f()->l4, (const T*)f()->rd, (const T*)f()->u(), f()->template dirs<T>(),
                       (T*)f()->q(), sys->partials, sys->st, kPrefetchAhead));
    prof_stop(ctx, kProfSpmv);
    prof_start(ctx, kProfUpdate);
    PH_CUDA(launch_pdl_w(win, k_fcg_update<T, F>, wave(f()->per_update[F]), s, n, f()->template dirs<const T>(), (const T*)f()->q(),
                       (const T*)f()->di, (const T*)f()->dg, (T*)f()->u(), (Y*)f()->y, sys->partials, sys->st));
    prof_stop(ctx, kProfUpdate);
    ctx->launches += 1;
    if (!F) {
      prof_start(ctx, kProfDir);
      PH_CUDA(launch_pdl_w(win, k_fcg_dir<T>, wave(f()->per_dir), s, n, (const T*)f()->u(), (T*)f()->pk(0), sys->st));
      prof_stop(ctx, kProfDir);
      ctx->launches += 1;
    }
    return check_launch(ctx, "k_fcg");
  }
};

int read_state(phfem_sys sys) {
  cudaStream_t s = sys->mesh->ctx->stream;
  PH_CUDA(cudaMemcpyAsync(sys->st_host, sys->st, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
  PH_CUDA(cudaStreamSynchronize(s));
  return PHFEM_OK;
}

template <typename T, bool F>
int fcg_solve_typed(phfem_sys sys, const phfem_solve_opts& o, phfem_stats* stats) {
  phfem_ctx ctx = sys->mesh->ctx;
  const int n = sys->mesh->info.nE;
  const FLaunch<T, F> L{sys, ctx->stream, grid_for(ctx, n), n, o.rtol * o.rtol, o.inner_rtol * o.inner_rtol,
                        u_window(sys, false)};
  static const bool verbose = getenv("PHFEM_VERBOSE") != nullptr;
  PH_TRY(L.prologue());
  PH_TRY(L.residual(0));
  PH_TRY(L.residual(1));
  PH_TRY(read_state(sys));
  int status = PHFEM_OK, stagnant = 0, last_updates = 0;
  double best = 1e300;
  for (;;) {
    const SolveState& h = *sys->st_host;
    if (h.updates != last_updates) {  // a new true residual: progress bookkeeping
      last_updates = h.updates;
      const double rel = h.bb > 0 ? std::sqrt(h.rr64 / h.bb) : 0.0;
      if (verbose)
        fprintf(stderr, "phfem: update %d  iterations %d  relative residual %.3e  floor %.3e  restart %d\n", h.updates,
                h.it, rel, h.bb > 0 ? std::sqrt(h.floor2 / h.bb) : 0.0, h.restart);
      stagnant = (rel > 0.5 * best) ? stagnant + 1 : 0;
      best = rel < best ? rel : best;
    }
    if (h.done == 3) {
      status = h.status;
      break;
    }
    if (h.done == 2) break;
    if (h.it >= o.max_iter || h.updates > o.max_refine || stagnant >= 8) {
      status = PHFEM_ENOCONV;
      break;
    }
    if (h.done == 1) {  // reliable update requested by the iteration
      PH_TRY(L.residual(2));
      PH_TRY(read_state(sys));
      continue;
    }
    int chunk = o.check_every;
    if (h.it + chunk > o.max_iter) chunk = o.max_iter - h.it;
    for (int k = 0; k < chunk; ++k) PH_TRY(L.iteration());
    PH_TRY(read_state(sys));
  }
  PH_TRY(L.epilogue());
  if (L.win.bytes > 0) {  // the window's lines and the set-aside go back to normal L2 use
    cudaCtxResetPersistingL2Cache();
    cudaGetLastError();
    set_l2_limit(ctx, 0);
  }
  const SolveState& h = *sys->st_host;
  const double rel = h.bb > 0 ? std::sqrt(h.rr64 / h.bb) : 0.0;
  if (stats) {
    stats->iterations += h.it;
    stats->refinements += h.updates;
    stats->converged = h.done == 2 ? h.conv : 0;
    stats->rel_residual = rel;
    stats->fp64_floor = h.bb > 0 ? std::sqrt(h.floor2 / h.bb) : 0.0;
  }
  if (status != PHFEM_OK) {
    char buf[200];
    snprintf(buf, sizeof(buf), "solve: %s after %d iterations, %d residual updates, relative residual %.3e",
             phfem_status_str(status), h.it, h.updates, rel);
    return fail(status, buf);
  }
  return PHFEM_OK;
}

// The prologue and start kernels, a WHILE node whose body runs `per_body`
// iterations, the conditional reliable update and the loop control, then the
// epilogue.
template <typename T, bool F>
int fcg_capture_typed(phfem_sys sys, const phfem_solve_opts& o, cudaStream_t cs, int per_body) {
  phfem_ctx ctx = sys->mesh->ctx;
  const int n = sys->mesh->info.nE;
  const FLaunch<T, F> L{sys, cs, grid_for(ctx, n), n, o.rtol * o.rtol, o.inner_rtol * o.inner_rtol,
                        u_window(sys, true)};
  PH_TRY(L.prologue());
  PH_TRY(L.residual(0));
  PH_TRY(L.residual(1));
  cudaStreamCaptureStatus cst;
  cudaGraph_t graph;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  PH_CUDA(cudaStreamGetCaptureInfo(cs, &cst, nullptr, &graph, &deps, nullptr, &ndeps));
  if (cst != cudaStreamCaptureStatusActive) return fail(PHFEM_ECUDA, "capture_solve: stream is not capturing");
  cudaGraphConditionalHandle handle;
  PH_CUDA(cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = handle;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t cnode;
  PH_CUDA(cudaGraphAddNode(&cnode, graph, deps, nullptr, ndeps, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  PH_CUDA(cudaStreamUpdateCaptureDependencies(cs, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies));
  cudaStream_t bs;
  PH_CUDA(cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking));
  int st = PHFEM_OK;
  cudaError_t e = cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) st = cuda_fail(e, "cudaStreamBeginCaptureToGraph", __FILE__, __LINE__);
  if (st == PHFEM_OK) {
    const FLaunch<T, F> B{sys, bs, L.g, n, L.rtol2, L.irtol2, L.win};
    for (int k = 0; k < per_body && st == PHFEM_OK; ++k) st = B.iteration();
    if (st == PHFEM_OK) st = B.residual(3);
    if (st == PHFEM_OK) {
      const int max_bodies = o.max_iter / (per_body > 0 ? per_body : 1) + o.max_refine + 16;
      k_fcg_loop_control<<<1, 1, 0, bs>>>(sys->st, handle, o.max_iter, max_bodies);
      st = check_launch(ctx, "k_fcg_loop_control");
    }
    cudaGraph_t out;
    e = cudaStreamEndCapture(bs, &out);
    if (e != cudaSuccess && st == PHFEM_OK) st = cuda_fail(e, "cudaStreamEndCapture(body)", __FILE__, __LINE__);
  }
  cudaStreamDestroy(bs);
  if (st == PHFEM_OK) st = L.epilogue();
  return st;
}

}  // namespace

// FP32 systems fold the direction update into the product unless the
// context chose the unfused kernels.
static bool fused_fp32(phfem_sys sys) { return sys->mesh->ctx->cg_variant != 1; }  // 0 and 2

bool fcg_eligible(phfem_sys sys, const phfem_solve_opts& o) {
  return o.order == 0 && sys->form == PHFEM_FORM_TRACE && !sys->conv && !sys->mg;
}

template <typename K>
static int resident_blocks(K kernel) {
  int per = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, kBlock, 0) != cudaSuccess || per < 1) {
    (void)cudaGetLastError();
    per = 1;
  }
  return per;
}

int fcg_prepare(phfem_sys sys) {
  if (sys->fcg) return PHFEM_OK;
  phfem_mesh m = sys->mesh;
  phfem_ctx ctx = m->ctx;
  PH_TRY(mesh_order(m));
  const int n = m->info.nE;
  const size_t isz = sys->fp32 ? sizeof(float) : sizeof(double);
  FastCG* f = new FastCG();
  f->n = n;
  f->fp32 = sys->fp32;
  f->slot = ((size_t)n * isz + 255) / 256 * 256;
  int st = PHFEM_OK;
  auto chk = [&](int r) {
    if (st == PHFEM_OK) st = r;
  };
  chk(dalloc(ctx, &f->l4, (size_t)n * 4 * isz + 32));
  chk(dalloc(ctx, &f->rd, (size_t)n * isz + 16));
  chk(dalloc(ctx, &f->di, (size_t)n * isz + 16));
  if (!sys->fp32) chk(dalloc(ctx, &f->dg, (size_t)n * isz + 16));
  chk(dalloc_n(ctx, &f->val, 5 * (size_t)n));
  chk(dalloc_n(ctx, &f->b, (size_t)n));
  chk(dalloc_n(ctx, &f->xh, (size_t)n));
  chk(dalloc_n(ctx, &f->xl, (size_t)n));
  chk(dalloc(ctx, &f->y, (size_t)n * 8 + 16));
  chk(dalloc(ctx, &f->vec, (2 + kDirs) * f->slot + 16));
  sys->fcg = f;
  if (sys->fp32) {
    f->per_spmv[0] = resident_blocks(k_fcg_spmv<float, false>);
    f->per_spmv[1] = resident_blocks(k_fcg_spmv<float, true>);
    f->per_update[0] = resident_blocks(k_fcg_update<float, false>);
    f->per_update[1] = resident_blocks(k_fcg_update<float, true>);
    f->per_dir = resident_blocks(k_fcg_dir<float>);
    // The staged product kernel needs ~150 KB of shared memory per SM for 8
    // blocks; the update kernel almost none.  Left to choose, the two would
    // run under different L1 / shared-memory splits, and every switch between
    // them drains the SM (no overlap of consecutive launches): 125 us per
    // iteration at level 5 against 105 with one split for both.  Set once
    // per process: changing a kernel's attributes can wait for that kernel's
    // launches in flight on other streams (the request server's slots).
    static const bool split_set = [] {
      int smem_sm = 0, dev = 0;
      cudaFuncAttributes fa{};
      cudaGetDevice(&dev);
      if (cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) == cudaSuccess &&
          cudaFuncGetAttributes(&fa, k_fcg_spmv_staged) == cudaSuccess && smem_sm > 0) {
        const double need = (double)kBlocksPerSM * ((double)fa.sharedSizeBytes + 1024.0);  // + 1 KB per block reserved
        // The preference is a percentage of the SM's shared memory, and the
        // driver maps it to one of the sizes the SM supports (KB, compute
        // capability 9.0 and 10.x): a percentage between two sizes may map to
        // different sizes for kernels of different needs, so the request is
        // the smallest supported size that holds 8 staged blocks, exactly.
        static const int kSizesKB[] = {0, 8, 16, 32, 64, 100, 132, 164, 196, 228};
        for (int kb : kSizesKB) {
          if (kb * 1024.0 < need || kb * 1024 > smem_sm) continue;
          const int carve = (int)std::ceil(100.0 * kb * 1024.0 / smem_sm);
          cudaFuncSetAttribute(k_fcg_spmv_staged, cudaFuncAttributePreferredSharedMemoryCarveout, carve);
          cudaFuncSetAttribute(k_fcg_update<float, true>, cudaFuncAttributePreferredSharedMemoryCarveout, carve);
          if (resident_blocks(k_fcg_spmv_staged) >= kBlocksPerSM) break;
        }
      }
      cudaGetLastError();
      return true;
    }();
    (void)split_set;
    f->per_staged = resident_blocks(k_fcg_spmv_staged);
  } else {
    f->per_spmv[0] = resident_blocks(k_fcg_spmv<double, false>);
    f->per_update[0] = resident_blocks(k_fcg_update<double, false>);
    f->per_dir = resident_blocks(k_fcg_dir<double>);
  }
  if (st == PHFEM_OK) {
    const int g = grid_for(ctx, n);
    if (sys->fp32)
      k_fcg_op<float><<<g, kBlock, 0, ctx->stream>>>(n, m->perm, (const float*)sys->lval, (const float*)sys->rdiag,
                                                     (const float*)sys->dinv, sys->val, (float4*)f->l4,
                                                     (float*)f->rd, (float*)f->di, nullptr, f->val);
    else
      k_fcg_op<double><<<g, kBlock, 0, ctx->stream>>>(n, m->perm, (const double*)sys->lval,
                                                      (const double*)sys->rdiag, (const double*)sys->dinv, sys->val,
                                                      (Inner<double>::L4*)f->l4, (double*)f->rd, (double*)f->di,
                                                      (double*)f->dg, f->val);
    chk(check_launch(ctx, "k_fcg_op"));
  }
  if (st != PHFEM_OK) fcg_free(sys);
  return st;
}

void fcg_free(phfem_sys sys) {
  FastCG* f = sys->fcg;
  if (!f) return;
  phfem_ctx c = sys->mesh->ctx;
  dfree(c, f->l4);
  dfree(c, f->rd);
  dfree(c, f->di);
  dfree(c, f->dg);
  dfree(c, f->val);
  dfree(c, f->b);
  dfree(c, f->xh);
  dfree(c, f->xl);
  dfree(c, f->y);
  dfree(c, f->vec);
  delete f;
  sys->fcg = nullptr;
}

int fcg_solve(phfem_sys sys, const phfem_solve_opts& o, phfem_stats* stats) {
  PH_TRY(fcg_prepare(sys));
  if (!sys->fp32) return fcg_solve_typed<double, false>(sys, o, stats);
  return fused_fp32(sys) ? fcg_solve_typed<float, true>(sys, o, stats) : fcg_solve_typed<float, false>(sys, o, stats);
}

int fcg_capture(phfem_sys sys, const phfem_solve_opts& o, cudaStream_t cs, int per_body) {
  if (!sys->fcg) return fail(PHFEM_ECUDA, "capture_solve: the locality-order operator must be built before capture");
  if (!sys->fp32) return fcg_capture_typed<double, false>(sys, o, cs, per_body);
  return fused_fp32(sys) ? fcg_capture_typed<float, true>(sys, o, cs, per_body)
                         : fcg_capture_typed<float, false>(sys, o, cs, per_body);
}

}  // namespace phfem
