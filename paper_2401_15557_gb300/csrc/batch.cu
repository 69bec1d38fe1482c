// Batched assembly and solve of many independent meshes in one persistent
// launch.
//
// Each thread block takes the next mesh from a device work queue (meshes in
// decreasing size, so the largest start first) and runs the whole path for it:
// the triangle pass (condensed element blocks), the edge-row pass (difference
// form, FP64 and inner precision), Jacobi-PCG with reliable updates (FP32
// systems: the direction update folded into the product and the solution
// correction accumulated as a float pair; FP64 systems: three loops and the
// solution accumulated in FP64), and the recovery of U and Lambda.  Block-wide
// barriers replace the kernel boundaries of the single-mesh path, and dot
// products are block reductions (FP64 across threads), so one launch solves
// the whole batch.  The per-element and per-row arithmetic is the same code as
// the single-mesh kernels (kernels.cuh).
//
// A mesh can also be taken by a thread-block cluster of C CTAs (C = 2, 4, 8)
// instead of one block, so that the largest meshes, which set the launch's
// tail, run on C SMs: triangles and rows are split over the cluster's threads,
// cluster barriers replace the block barriers, and every reduction sums the C
// block totals read from the CTAs' shared memory (distributed shared memory,
// fixed rank order, so every CTA gets the same value and takes the same
// branch).  The tuner picks the block size and the cluster size.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <numeric>
#include <vector>

#include <cooperative_groups.h>

#include "kernels.cuh"

namespace phfem {
namespace {

struct MeshDesc {
  int nT, nE, nL, pad;
  long long t0, e0, l0, v0;  // offsets of the mesh's triangles, edges, multipliers, vertices
};

struct BatchParams {
  double rtol2, upd2;   // rtol^2, reliable-update factor^2
  int max_iter, max_updates;
  double a_const;
};

struct MeshStats {
  int iterations, updates, converged, status;
  double rel, floor_rel;
  int where, pad;      // failure site: 1 residual, 2 p.q, 3 r.z
  double dbg[4];       // pq, rz, rz of the last update, alpha at the failure
};

namespace cgr = cooperative_groups;

// Barrier over the mesh's threads: the block, or the whole cluster (which also
// orders the threads' global-memory writes for the cluster).
template <int C>
__device__ __forceinline__ void msync() {
  if constexpr (C == 1) __syncthreads();
  else cgr::this_cluster().sync();
}

// Sum of v over the mesh's threads, the same value in every thread: warp sums,
// then the block total by a butterfly over the warp totals; with a cluster, each CTA publishes its
// total in slot `slot` (alternating between consecutive reductions, so one
// barrier suffices) and every thread adds the C totals in rank order.
// Sum over the 32 lanes by a butterfly: every lane computes the same pairwise
// sums (a + b and b + a are the same IEEE result), so all lanes, and all
// warps given the same inputs, get the same value.
__device__ __forceinline__ double warp_allsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// num / den computed once per warp and broadcast: an FP64 division in every
// thread would hold GB300's FP64 pipe (num and den are uniform over the block).
__device__ __forceinline__ double warp_div(double num, double den) {
  double q = 0.0;
  if ((threadIdx.x & 31) == 0) q = num / den;
  return __shfl_sync(0xffffffffu, q, 0);
}

template <int BS, int C>
__device__ __forceinline__ double bsum(double v, double* smem, double* cl_part, int& slot) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();  // smem may still be read by the previous reduction
  if (lane == 0) smem[w] = v;
  __syncthreads();
  // every warp sums the BS / 32 warp totals by the same butterfly
  double t = warp_allsum(lane < BS / 32 ? smem[lane] : 0.0);
  if constexpr (C == 1) {
    return t;
  } else {
    cgr::cluster_group cl = cgr::this_cluster();
    if (threadIdx.x == 0) cl_part[slot] = t;
    cl.sync();
    double u = 0.0;
    for (unsigned r = 0; r < (unsigned)C; ++r) u += *cl.map_shared_rank(cl_part + slot, r);
    slot ^= 1;
    return u;
  }
}

template <typename T>
struct BatchArrays {
  const double2* xy;
  const int32_t* tri;
  const int32_t* ed2el;
  const uint8_t* lk;
  const uint8_t* eclass;
  const int32_t* nbr;
  const double* elen;
  const int32_t* t2e;
  const int8_t* sigma;
  const int32_t* lam_id;
  const double* aT;      // [sum nT] or NULL
  const double* delta;   // [count]
  const double* f_mid;   // [sum nE] or NULL
  const double* bc_mid;  // [sum nE] or NULL
  double* Kt;            // [sum nT][4] records (AoS)
  double* val;           // [5 sum nE]
  double* b;
  T* lval;               // [4 sum nE]
  T* rdiag;
  T* dinv;
  double* x;
  float2* y;             // [sum nE] FP32 systems: correction since the last reliable update (a float pair)
  T* r;
  T* p;
  T* p2;                 // FP32 systems: the second direction buffer of the fused iteration
  T* q;
  double* U;             // [3 sum nT] or NULL
  double* Lambda;        // [sum nL] or NULL
  double* w;             // [sum nE] or NULL
};

template <typename T, int BS, int C>
__global__ void __launch_bounds__(BS) k_batch(int count, const MeshDesc* __restrict__ desc,
                                              const int* __restrict__ order, int* next, BatchArrays<T> A,
                                              BatchParams P, MeshStats* stats) {
  __shared__ double smem[BS / 32];
  __shared__ double cl_part[2];
  __shared__ int s_mesh;
  int slot = 0;
  unsigned crank = 0;  // rank of this CTA in its cluster
  if constexpr (C > 1) crank = cgr::this_cluster().block_rank();
  const int tid0 = (int)crank * BS + threadIdx.x;  // thread index within the mesh's threads
  constexpr int STR = C * BS;                      // threads working on one mesh
  for (;;) {
    msync<C>();
    if (crank == 0 && threadIdx.x == 0) s_mesh = atomicAdd(next, 1);
    msync<C>();
    int k;
    if constexpr (C == 1) {
      k = s_mesh;
    } else {
      k = *cgr::this_cluster().map_shared_rank(&s_mesh, 0);
      msync<C>();  // no CTA leaves while another still reads rank 0's s_mesh
    }
    if (k >= count) return;
    const int id = order[k];
    const MeshDesc D = desc[id];
    const int nT = D.nT, nE = D.nE;
    const size_t m = (size_t)nE;
    const double2* xy = A.xy + D.v0;
    const int32_t* tri = A.tri + 3 * D.t0;
    const int32_t* ed2el = A.ed2el + 4 * D.e0;
    const uint8_t* lk = A.lk + D.e0;
    const uint8_t* ecl = A.eclass + D.e0;
    const int32_t* nbr = A.nbr + 4 * D.e0;
    const double* elen = A.elen + D.e0;
    double* Kt = A.Kt + (size_t)kRec * D.t0;
    double* val = A.val + 5 * D.e0;
    double* b = A.b + D.e0;
    T* lval = A.lval + 4 * D.e0;
    T* rdiag = A.rdiag + D.e0;
    T* dinv = A.dinv + D.e0;
    double* x = A.x + D.e0;
    float2* y = A.y + D.e0;
    // FP32 systems: the solution correction as a float pair, and the fused
    // iteration (r holds u = D^-1 r; the direction update is folded into the
    // product, which forms p at each row and its neighbours from u and the
    // previous p in the other buffer: two loops and two barriers per
    // iteration instead of three).  FP64 systems keep the three loops: GB300's
    // FP64 rate makes the four extra FP64 operations per row cost more.
    constexpr bool kPair = sizeof(T) == sizeof(float);
    constexpr bool kFused = kPair;
    T* r = A.r + D.e0;
    T* p = A.p + D.e0;
    T* q = A.q + D.e0;
    T* po = p;               // fused: the previous direction
    T* pn = A.p2 + D.e0;     // fused: the direction being formed (the two swap every iteration)
    const double delta = A.delta[id];
    const double* f = A.f_mid ? A.f_mid + D.e0 : nullptr;
    const double* bc = A.bc_mid ? A.bc_mid + D.e0 : nullptr;

    // 1. triangle pass
    for (int t = tid0; t < nT; t += STR) {
      const double a = A.aT ? A.aT[D.t0 + t] : P.a_const;
      const double2 p0 = xy[tri[3 * t]], p1 = xy[tri[3 * t + 1]], p2 = xy[tri[3 * t + 2]];
      // FP64 records in both precisions: the meshes are small and the time is
      // the iteration's; the compensated path's registers would cost occupancy
      double R[4];
      tri_record64(p0, p1, p2, a, R);
      store_record(Kt + (size_t)kRec * t, R);
    }
    msync<C>();
    // 2. edge rows; x starts at 0 on free edges and u_D on Dirichlet edges
    for (int e = tid0; e < nE; e += STR) {
      const int4 qd = reinterpret_cast<const int4*>(ed2el)[e];
      const int kk = lk[e];
      const uint8_t cls = ecl[e];
      const EdgeRow R = edge_row<false, true>(Kt, qd.z, kk & 3, qd.w, (kk >> 2) & 3, cls, f ? f[e] : 0.0,
                                              bc ? bc[e] : 0.0, cls == PHFEM_EDGE_NEUMANN ? elen[e] : 0.0, 1.0, 0.0,
                                              delta, f != nullptr, bc != nullptr);
      val[e] = R.rpart;
#pragma unroll
      for (int s = 0; s < 4; ++s) val[(s + 1) * m + e] = R.l[s];
      b[e] = R.rhs;
#pragma unroll
      for (int s = 0; s < 4; ++s) lval[s * m + e] = (T)R.l[s];
      rdiag[e] = (T)R.rpart;
      dinv[e] = (T)(1.0 / R.diag);
      x[e] = (cls == PHFEM_EDGE_DIRICHLET) ? R.rhs : 0.0;
      if constexpr (kPair) y[e] = make_float2(0.f, 0.f);
    }
    msync<C>();
    // ||b_free|| with the Dirichlet lifting (x is (0, u_D) now)
    double bb = 0.0;
    {
      double acc = 0.0;
      for (int e = tid0; e < nE; e += STR) {
        if (ecl[e] == PHFEM_EDGE_DIRICHLET) continue;
        double fl;
        const double rr = residual_row(nbr, val, b, x, m, e, fl);
        acc += rr * rr;
      }
      bb = bsum<BS, C>(acc, smem, cl_part, slot);
    }
    // 3. Jacobi-PCG with reliable updates
    int it = 0, updates = 0, converged = 0, status = 0, stagnant = 0, where = 0;
    double rel = 0.0, floor_rel = 0.0, best = 1e300, rz = 0.0, tol2 = 0.0, dpq = 0.0, dal = 0.0, drzt = 0.0;
    bool first = true;
    int mode = 1;      // fused: 1 restart (p = u), 2 keep the direction (p = p_old), 0 p = u + beta p_old
    T beta_f = (T)0;   // fused: the last beta
    for (;;) {
      if constexpr (kPair) {  // the correction into x before x is read at the neighbours
        if (!first) {
          for (int e = tid0; e < nE; e += STR) {
            const float2 v = y[e];
            x[e] += (double)v.x + (double)v.y;
            y[e] = make_float2(0.f, 0.f);
          }
          msync<C>();
        }
      }
      // true residual (FP64, difference form), inner residual replaced
      double a_r = 0.0, a_z = 0.0, a_f = 0.0, a_p = 0.0;
      for (int e = tid0; e < nE; e += STR) {
        double fl;
        const double rr = residual_row(nbr, val, b, x, m, e, fl);
        a_r += rr * rr;
        fl *= 0x1p-53;
        a_f += fl * fl;
        const T rs = (T)rr;
        const T zs = dinv[e] * rs;
        if constexpr (kFused) {
          // the kept direction is the one the next iteration would take,
          // p = u + beta p_old from the recursive u, formed before u is replaced
          if (!first) {
            const T pk = fmaf(beta_f, po[e], r[e]);
            po[e] = pk;
            a_p += (double)rs * (double)pk;
          }
          r[e] = zs;
        } else {
          r[e] = rs;
          if (first) p[e] = zs;
          else a_p += (double)rs * (double)p[e];
        }
        a_z += (double)rs * (double)zs;
      }
      const double rr64 = bsum<BS, C>(a_r, smem, cl_part, slot);
      const double rz_true = bsum<BS, C>(a_z, smem, cl_part, slot);
      const double ff = bsum<BS, C>(a_f, smem, cl_part, slot);
      const double rp = bsum<BS, C>(a_p, smem, cl_part, slot);
      ++updates;
      rel = bb > 0 ? sqrt(rr64 / bb) : 0.0;
      floor_rel = bb > 0 ? sqrt(ff / bb) : 0.0;
      drzt = rz_true;
      if (!isfinite(rr64) || !isfinite(rz_true)) {
        status = PHFEM_ENAN;
        where = 1;
        break;
      }
      if (rr64 <= P.rtol2 * bb || rr64 == 0.0) {
        converged = 1;
        break;
      }
      if (rel <= 2.0 * floor_rel) {
        converged = 2;
        break;
      }
      stagnant = (rel > 0.5 * best) ? stagnant + 1 : 0;
      best = rel < best ? rel : best;
      if (it >= P.max_iter || updates > P.max_updates || stagnant >= 8) {
        status = PHFEM_ENOCONV;
        break;
      }
      // the first step after the replacement is a line search alpha = r.p / p.Ap;
      // restart the direction if it no longer fits the replaced residual
      bool line_search = !first;
      if (!first && (rz_true > 4.0 * rz || !(rp > 0.0))) {
        if constexpr (!kFused)
          for (int e = tid0; e < nE; e += STR) p[e] = dinv[e] * r[e];
        line_search = false;
      }
      mode = line_search ? 2 : 1;
      first = false;
      rz = rz_true;
      tol2 = rz * fmax(P.upd2, fmin(bb > 0.0 ? 0.8 * P.rtol2 * bb / rr64 : 0.0, 1.0));  // as update_target
      msync<C>();
      // iterate until the recursive residual fell by the update factor
      while (it < P.max_iter) {
        T acc = (T)0;
        if constexpr (kFused) {
          const T bf = beta_f;
          const int md = mode;
          auto pval = [&](int i) -> T {
            if (md == 1) return r[i];
            if (md == 2) return po[i];
            return fmaf(bf, po[i], r[i]);
          };
          for (int e = tid0; e < nE; e += STR) {
            const int c0 = nbr[e], c1 = nbr[m + e], c2 = nbr[2 * m + e], c3 = nbr[3 * m + e];
            const T pe = pval(e);
            T sv = rdiag[e] * pe;
            sv += lval[e] * (pe - pval(c0));
            sv += lval[m + e] * (pe - pval(c1));
            sv += lval[2 * m + e] * (pe - pval(c2));
            sv += lval[3 * m + e] * (pe - pval(c3));
            pn[e] = pe;
            q[e] = sv;
            acc += pe * sv;
          }
        } else {
          for (int e = tid0; e < nE; e += STR) {
            const T sv = spmv_row<T, false>(nbr, lval, rdiag, p, m, e);
            q[e] = sv;
            acc += p[e] * sv;
          }
        }
        const double pq = bsum<BS, C>((double)acc, smem, cl_part, slot);
        dpq = pq;
        if (!(pq > 0.0) || !isfinite(pq)) {
          status = isfinite(pq) ? PHFEM_EBREAKDOWN : PHFEM_ENAN;
          where = 2;
          break;
        }
        const double alpha64 = warp_div(line_search ? rp : rz, pq);
        line_search = false;
        mode = 0;
        dal = alpha64;
        const T alpha = (T)alpha64;
        T acc2 = (T)0;
        if constexpr (kFused) {  // y += alpha p (float pair), u -= alpha D^-1 q, r.z = u.u / D^-1
          const float al = (float)(alpha64 - (double)alpha);
          for (int e = tid0; e < nE; e += STR) {
            y[e] = y_add(y[e], alpha, al, pn[e]);
            const T d = dinv[e];
            const T ue = fmaf(-alpha, d * q[e], r[e]);
            r[e] = ue;
            acc2 += d > (T)0 ? __fdividef(ue * ue, d) : (T)0;
          }
        } else {
          for (int e = tid0; e < nE; e += STR) {
            x[e] += alpha64 * (double)p[e];
            const T re = r[e] - alpha * q[e];
            r[e] = re;
            acc2 += re * (dinv[e] * re);
          }
        }
        const double rzn = bsum<BS, C>((double)acc2, smem, cl_part, slot);
        const T beta = (T)(rz > 0.0 ? warp_div(rzn, rz) : 0.0);
        rz = rzn;
        ++it;
        if constexpr (kFused) {
          // the reductions' barriers ordered this iteration's writes of p and u
          // before the next product reads them at the neighbours
          beta_f = beta;
          T* t = po;
          po = pn;
          pn = t;
        } else {
          for (int e = tid0; e < nE; e += STR) p[e] = dinv[e] * r[e] + beta * p[e];
          msync<C>();
        }
        if (!isfinite(rz)) {
          status = PHFEM_ENAN;
          where = 3;
          break;
        }
        if (rz <= tol2) break;
      }
      if (status) break;
      msync<C>();
    }
    msync<C>();
    // 4. recovery: U = R^-1 w per triangle, Lambda from the T+ rows
    if (A.U || A.Lambda) {
      const int32_t* t2e = A.t2e + 3 * D.t0;
      const int8_t* sg = A.sigma + 3 * D.t0;
      const int32_t* lam = A.lam_id + D.e0;
      for (int t = tid0; t < nT; t += STR) {
        const int e0 = t2e[3 * t], e1 = t2e[3 * t + 1], e2 = t2e[3 * t + 2];
        const double a0 = x[e0], a1 = x[e1], a2 = x[e2];
        if (A.U) {
          const double s = a0 + a1 + a2;
          double* U = A.U + 3 * D.t0;
          U[3 * t] = s - 2.0 * a0;
          U[3 * t + 1] = s - 2.0 * a1;
          U[3 * t + 2] = s - 2.0 * a2;
        }
        if (A.Lambda) {  // row k of K^CR_T x in difference form, from the record, per multiplier edge
          const int ee[3] = {e0, e1, e2};
          const double aa[3] = {a0, a1, a2};
          const double* rt = Kt + (size_t)kRec * t;
#pragma unroll
          for (int kk = 0; kk < 3; ++kk) {
            const int li = lam[ee[kk]];
            if (li < 0 || sg[3 * t + kk] < 0) continue;
            const int k1 = kk == 2 ? 0 : kk + 1, k2 = kk == 0 ? 2 : kk - 1;
            const double mT = rt[3];
            const double res = rt[kk] * (aa[kk] - aa[k1]) + rt[k2] * (aa[kk] - aa[k2]) + delta * mT * aa[kk];
            const double rr = res - mT * (f ? f[ee[kk]] : 0.0);
            A.Lambda[D.l0 + li] = rr / elen[ee[kk]];
          }
        }
      }
    }
    if (A.w)
      for (int e = tid0; e < nE; e += STR) A.w[D.e0 + e] = x[e];
    if (crank == 0 && threadIdx.x == 0) {
      MeshStats s;
      s.iterations = it;
      s.updates = updates;
      s.converged = converged;
      s.status = status;
      s.rel = rel;
      s.floor_rel = floor_rel;
      s.where = where;
      s.dbg[0] = dpq;
      s.dbg[1] = rz;
      s.dbg[2] = drzt;
      s.dbg[3] = dal;
      stats[id] = s;
    }
  }
}

}  // namespace
}  // namespace phfem

using namespace phfem;

struct phfem_batch_s {
  phfem_ctx ctx;
  int count;
  std::vector<long long> toff, eoff, loff, voff;  // count + 1
  MeshDesc* desc;
  int* order;
  int* next;
  MeshStats* stats;
  double2* xy;
  int32_t* tri;
  int32_t* ed2el;
  uint8_t* lk;
  uint8_t* eclass;
  int32_t* nbr;
  double* elen;
  int32_t* t2e;
  int8_t* sigma;
  int32_t* lam_id;
  int32_t nD_zero_count;  // meshes without a Dirichlet edge
  std::vector<int> nD;
  // system and workspace (allocated on the first solve, for both precisions)
  double* Kt = nullptr;
  double* val = nullptr;
  double* b = nullptr;
  double* x = nullptr;
  float2* y = nullptr;
  void* lval = nullptr;
  void* rdiag = nullptr;
  void* dinv = nullptr;
  void* r = nullptr;
  void* p = nullptr;
  void* p2 = nullptr;
  void* q = nullptr;
  int block = 0;    // 0: not tuned yet
  int cluster = 1;  // CTAs per mesh
};

namespace phfem {
namespace {

void batch_free(phfem_batch B) {
  phfem_ctx c = B->ctx;
  for (void* ptr : {(void*)B->desc, (void*)B->order, (void*)B->next, (void*)B->stats, (void*)B->xy, (void*)B->tri,
                    (void*)B->ed2el, (void*)B->lk, (void*)B->eclass, (void*)B->nbr, (void*)B->elen, (void*)B->t2e,
                    (void*)B->sigma, (void*)B->lam_id, (void*)B->Kt, (void*)B->val, (void*)B->b, (void*)B->x, (void*)B->y,
                    B->lval, B->rdiag, B->dinv, B->r, B->p, B->p2, B->q})
    dfree(c, ptr);
  delete B;
}

template <typename T, int BS, int C>
int launch_batch(phfem_batch B, const BatchArrays<T>& A, const BatchParams& P) {
  phfem_ctx ctx = B->ctx;
  PH_CUDA(cudaMemsetAsync(B->next, 0, sizeof(int), ctx->stream));
  auto K = k_batch<T, BS, C>;
  if constexpr (C == 1) {
    int per_sm = 0;
    PH_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, K, BS, 0));
    if (per_sm < 1) per_sm = 1;
    int grid = ctx->num_sms * per_sm;
    if (grid > B->count) grid = B->count;
    K<<<grid, BS, 0, ctx->stream>>>(B->count, B->desc, B->order, B->next, A, P, B->stats);
    return check_launch(ctx, "k_batch");
  } else {
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(BS);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = ctx->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3(C * ctx->num_sms);
    int clusters = 0;
    PH_CUDA(cudaOccupancyMaxActiveClusters(&clusters, K, &cfg));
    if (clusters < 1) clusters = 1;
    if (clusters > B->count) clusters = B->count;
    cfg.gridDim = dim3(C * clusters);
    PH_CUDA(cudaLaunchKernelEx(&cfg, K, B->count, (const MeshDesc*)B->desc, (const int*)B->order, B->next, A, P,
                               B->stats));
    return check_launch(ctx, "k_batch");
  }
}

// The launch shapes the tuner tries: threads per block, CTAs per cluster.
constexpr int kShapes = 10;
constexpr int kShapeBlock[kShapes] = {128, 256, 512, 1024, 256, 512, 1024, 256, 512, 1024};
constexpr int kShapeCluster[kShapes] = {1, 1, 1, 1, 4, 4, 4, 8, 8, 8};

template <typename T>
int run_batch(phfem_batch B, int block, int cluster, const BatchArrays<T>& A, const BatchParams& P) {
  switch (cluster * 10000 + block) {
    case 10128: return launch_batch<T, 128, 1>(B, A, P);
    case 10256: return launch_batch<T, 256, 1>(B, A, P);
    case 10512: return launch_batch<T, 512, 1>(B, A, P);
    case 11024: return launch_batch<T, 1024, 1>(B, A, P);
    case 40256: return launch_batch<T, 256, 4>(B, A, P);
    case 40512: return launch_batch<T, 512, 4>(B, A, P);
    case 41024: return launch_batch<T, 1024, 4>(B, A, P);
    case 80256: return launch_batch<T, 256, 8>(B, A, P);
    case 80512: return launch_batch<T, 512, 8>(B, A, P);
    case 81024: return launch_batch<T, 1024, 8>(B, A, P);
    default: return fail(PHFEM_EINVAL, "phfem_batch_solve: unsupported block/cluster shape");
  }
}

}  // namespace
}  // namespace phfem

extern "C" {

PHFEM_API int phfem_batch_create(phfem_ctx ctx, int32_t count, const phfem_mesh* meshes, phfem_batch* out) {
  if (!out) return fail(PHFEM_EINVAL, "phfem_batch_create: out is NULL");
  *out = nullptr;
  if (!ctx || count < 1 || !meshes) return fail(PHFEM_EINVAL, "phfem_batch_create: bad argument");
  phfem_batch B = new phfem_batch_s();
  B->ctx = ctx;
  B->count = count;
  B->toff.assign(count + 1, 0);
  B->eoff.assign(count + 1, 0);
  B->loff.assign(count + 1, 0);
  B->voff.assign(count + 1, 0);
  B->nD.resize(count);
  std::vector<MeshDesc> hd(count);
  for (int i = 0; i < count; ++i) {
    if (!meshes[i] || meshes[i]->ctx->device != ctx->device) {
      delete B;
      return fail(PHFEM_EINVAL, "phfem_batch_create: NULL mesh or mesh of another device");
    }
    const phfem_mesh_info& I = meshes[i]->info;
    hd[i] = MeshDesc{I.nT, I.nE, I.nL, 0, B->toff[i], B->eoff[i], B->loff[i], B->voff[i]};
    B->toff[i + 1] = B->toff[i] + I.nT;
    B->eoff[i + 1] = B->eoff[i] + I.nE;
    B->loff[i + 1] = B->loff[i] + I.nL;
    B->voff[i + 1] = B->voff[i] + I.nV;
    B->nD[i] = I.nD;
  }
  const size_t sT = B->toff[count], sE = B->eoff[count], sV = B->voff[count];
  int st = PHFEM_OK;
  auto chk = [&](int r) {
    if (st == PHFEM_OK) st = r;
  };
  chk(dalloc_n(ctx, &B->desc, count));
  chk(dalloc_n(ctx, &B->order, count));
  chk(dalloc_n(ctx, &B->next, 1));
  chk(dalloc_n(ctx, &B->stats, count));
  chk(dalloc_n(ctx, &B->xy, sV));
  chk(dalloc_n(ctx, &B->tri, 3 * sT));
  chk(dalloc_n(ctx, &B->ed2el, 4 * sE));
  chk(dalloc_n(ctx, &B->lk, sE));
  chk(dalloc_n(ctx, &B->eclass, sE));
  chk(dalloc_n(ctx, &B->nbr, 4 * sE));
  chk(dalloc_n(ctx, &B->elen, sE));
  chk(dalloc_n(ctx, &B->t2e, 3 * sT));
  chk(dalloc_n(ctx, &B->sigma, 3 * sT));
  chk(dalloc_n(ctx, &B->lam_id, sE));
  if (st != PHFEM_OK) {
    cudaStreamSynchronize(ctx->stream);
    batch_free(B);
    return st;
  }
  cudaStream_t s = ctx->stream;
  // largest meshes first
  std::vector<int> ord(count);
  std::iota(ord.begin(), ord.end(), 0);
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int c) { return hd[a].nE > hd[c].nE; });
  auto cp = [&](void* dst, const void* src, size_t bytes) {
    if (st == PHFEM_OK && bytes) {
      cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, s);
      if (e != cudaSuccess) st = cuda_fail(e, "phfem_batch_create copy", __FILE__, __LINE__);
    }
  };
  for (int i = 0; i < count; ++i) {
    phfem_mesh M = meshes[i];
    const phfem_mesh_info& I = M->info;
    const long long t0 = B->toff[i], e0 = B->eoff[i], v0 = B->voff[i];
    cp(B->xy + v0, M->xy, sizeof(double2) * I.nV);
    cp(B->tri + 3 * t0, M->tri, sizeof(int32_t) * 3 * I.nT);
    cp(B->ed2el + 4 * e0, M->ed2el, sizeof(int32_t) * 4 * I.nE);
    cp(B->lk + e0, M->lk, I.nE);
    cp(B->eclass + e0, M->eclass, I.nE);
    cp(B->nbr + 4 * e0, M->nbr, sizeof(int32_t) * 4 * I.nE);
    cp(B->elen + e0, M->elen, sizeof(double) * I.nE);
    cp(B->t2e + 3 * t0, M->t2e, sizeof(int32_t) * 3 * I.nT);
    cp(B->sigma + 3 * t0, M->sigma, 3 * I.nT);
    cp(B->lam_id + e0, M->lam_id, sizeof(int32_t) * I.nE);
  }
  if (st == PHFEM_OK) {
    cudaMemcpyAsync(B->desc, hd.data(), sizeof(MeshDesc) * count, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(B->order, ord.data(), sizeof(int) * count, cudaMemcpyHostToDevice, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) st = cuda_fail(cudaGetLastError(), "phfem_batch_create", __FILE__, __LINE__);
  }
  if (st != PHFEM_OK) {
    cudaStreamSynchronize(s);
    batch_free(B);
    return st;
  }
  *out = B;
  return PHFEM_OK;
}

PHFEM_API int phfem_batch_offsets(phfem_batch B, int64_t* tri_off, int64_t* edge_off, int64_t* lam_off) {
  if (!B) return fail(PHFEM_EINVAL, "phfem_batch_offsets: NULL batch");
  for (int i = 0; i <= B->count; ++i) {
    if (tri_off) tri_off[i] = B->toff[i];
    if (edge_off) edge_off[i] = B->eoff[i];
    if (lam_off) lam_off[i] = B->loff[i];
  }
  return PHFEM_OK;
}

PHFEM_API int phfem_batch_solve(phfem_batch B, const double* a_T, const double* delta, const double* f_mid,
                                const double* bc_mid, int32_t precision, const phfem_solve_opts* opts, double* w,
                                double* U, double* Lambda, int32_t block, int32_t cluster, int32_t* iterations,
                                int32_t* converged, double* rel_residual) {
  if (!B || !delta) return fail(PHFEM_EINVAL, "phfem_batch_solve: NULL argument");
  if (precision != PHFEM_FP64 && precision != PHFEM_FP32_IR)
    return fail(PHFEM_EINVAL, "phfem_batch_solve: unknown precision");
  {
    bool ok = block == 0 && cluster == 0;
    for (int i = 0; i < kShapes && !ok; ++i) ok = block == kShapeBlock[i] && cluster == kShapeCluster[i];
    if (!ok)
      return fail(PHFEM_EINVAL, "phfem_batch_solve: (block, cluster) must be (0, 0) or a tuner shape: (128|256|512|1024, 1), "
                                "(256|512|1024, 4|8)");
  }
  phfem_ctx ctx = B->ctx;
  cudaStream_t s = ctx->stream;
  // host copy of delta to check solvability (no Dirichlet edge needs delta > 0)
  std::vector<double> hdel(B->count);
  PH_CUDA(cudaMemcpyAsync(hdel.data(), delta, sizeof(double) * B->count, cudaMemcpyDeviceToHost, s));
  PH_CUDA(cudaStreamSynchronize(s));
  for (int i = 0; i < B->count; ++i) {
    if (!(hdel[i] >= 0.0) || !std::isfinite(hdel[i]))
      return fail(PHFEM_EINVAL, "phfem_batch_solve: delta must be finite and >= 0 (mesh " + std::to_string(i) + ")");
    if (hdel[i] == 0.0 && B->nD[i] == 0)
      return fail(PHFEM_EINVAL, "phfem_batch_solve: mesh " + std::to_string(i) +
                                    " has no Dirichlet edge and no reaction term (singular)");
  }
  const size_t sT = B->toff[B->count], sE = B->eoff[B->count];
  const bool fp32 = precision == PHFEM_FP32_IR;
  if (!B->Kt) {
    int st = PHFEM_OK;
    auto chk = [&](int r) {
      if (st == PHFEM_OK) st = r;
    };
    chk(dalloc_n(ctx, &B->Kt, (size_t)kRec * sT));
    chk(dalloc_n(ctx, &B->val, 5 * sE));
    chk(dalloc_n(ctx, &B->b, sE));
    chk(dalloc_n(ctx, &B->x, sE));
    chk(dalloc_n(ctx, &B->y, sE));
    chk(dalloc(ctx, &B->lval, 4 * sE * sizeof(double)));
    chk(dalloc(ctx, &B->rdiag, sE * sizeof(double)));
    chk(dalloc(ctx, &B->dinv, sE * sizeof(double)));
    chk(dalloc(ctx, &B->r, sE * sizeof(double)));
    chk(dalloc(ctx, &B->p, sE * sizeof(double)));
    chk(dalloc(ctx, &B->p2, sE * sizeof(float)));
    chk(dalloc(ctx, &B->q, sE * sizeof(double)));
    if (st != PHFEM_OK) return st;
  }
  phfem_solve_opts o{};
  if (opts) o = *opts;
  if (o.rtol <= 0) o.rtol = 1e-10;
  if (o.inner_rtol <= 0) o.inner_rtol = fp32 ? 0.1 : 0.01;
  if (o.max_iter <= 0) o.max_iter = 200000;
  if (o.max_refine <= 0) o.max_refine = 1000;
  BatchParams P{o.rtol * o.rtol, o.inner_rtol * o.inner_rtol, o.max_iter, o.max_refine, 1.0};
  const int bs = block ? block : (B->block ? B->block : 256);
  const int cs = block ? cluster : (B->block ? B->cluster : 1);
  int st;
  if (fp32) {
    BatchArrays<float> A{B->xy, B->tri, B->ed2el, B->lk, B->eclass, B->nbr, B->elen, B->t2e, B->sigma, B->lam_id,
                         a_T, delta, f_mid, bc_mid, B->Kt, B->val, B->b, (float*)B->lval, (float*)B->rdiag,
                         (float*)B->dinv, B->x, B->y, (float*)B->r, (float*)B->p, (float*)B->p2, (float*)B->q, U, Lambda, w};
    st = run_batch<float>(B, bs, cs, A, P);
  } else {
    BatchArrays<double> A{B->xy, B->tri, B->ed2el, B->lk, B->eclass, B->nbr, B->elen, B->t2e, B->sigma, B->lam_id,
                          a_T, delta, f_mid, bc_mid, B->Kt, B->val, B->b, (double*)B->lval, (double*)B->rdiag,
                          (double*)B->dinv, B->x, B->y, (double*)B->r, (double*)B->p, nullptr, (double*)B->q, U, Lambda, w};
    st = run_batch<double>(B, bs, cs, A, P);
  }
  if (st != PHFEM_OK) return st;
  std::vector<MeshStats> hs(B->count);
  PH_CUDA(cudaMemcpyAsync(hs.data(), B->stats, sizeof(MeshStats) * B->count, cudaMemcpyDeviceToHost, s));
  PH_CUDA(cudaStreamSynchronize(s));
  int worst = PHFEM_OK, bad = -1;
  for (int i = 0; i < B->count; ++i) {
    if (iterations) iterations[i] = hs[i].iterations;
    if (converged) converged[i] = hs[i].converged;
    if (rel_residual) rel_residual[i] = hs[i].rel;
    if (hs[i].status != 0 && worst == PHFEM_OK) {
      worst = hs[i].status;
      bad = i;
    }
  }
  if (worst != PHFEM_OK) {
    const MeshStats& w = hs[bad];
    char buf[320];
    snprintf(buf, sizeof(buf),
             "phfem_batch_solve: mesh %d: %s (site %d, iteration %d, update %d, p.q %.3e, r.z %.3e, "
             "last true r.z %.3e, alpha %.3e, relative residual %.3e)",
             bad, phfem_status_str(worst), w.where, w.iterations, w.updates, w.dbg[0], w.dbg[1], w.dbg[2], w.dbg[3],
             w.rel);
    return fail(worst, buf);
  }
  return PHFEM_OK;
}

PHFEM_API int phfem_batch_tune(phfem_batch B, const double* a_T, const double* delta, const double* f_mid,
                               const double* bc_mid, int32_t precision, const phfem_solve_opts* opts,
                               int32_t* chosen_block, int32_t* chosen_cluster, double* ms_per_shape) {
  if (!B) return fail(PHFEM_EINVAL, "phfem_batch_tune: NULL batch");
  double best = 1e300;
  int pick = 1;
  for (int i = 0; i < kShapes; ++i) {
    auto t0 = std::chrono::steady_clock::now();
    int st = phfem_batch_solve(B, a_T, delta, f_mid, bc_mid, precision, opts, nullptr, nullptr, nullptr,
                               kShapeBlock[i], kShapeCluster[i], nullptr, nullptr, nullptr);
    double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (st != PHFEM_OK && st != PHFEM_ENOCONV) return st;
    if (ms_per_shape) ms_per_shape[i] = ms;
    if (ms < best) {
      best = ms;
      pick = i;
    }
  }
  B->block = kShapeBlock[pick];
  B->cluster = kShapeCluster[pick];
  if (chosen_block) *chosen_block = B->block;
  if (chosen_cluster) *chosen_cluster = B->cluster;
  return PHFEM_OK;
}

PHFEM_API int phfem_batch_destroy(phfem_batch B) {
  if (!B) return fail(PHFEM_EINVAL, "phfem_batch_destroy: NULL batch");
  batch_free(B);
  return PHFEM_OK;
}

}  // extern "C"
