// Geometric multigrid preconditioner for the condensed edge system over a
// hierarchy of uniform red refinements (Section 2.3).
//
// Level l + 1 is the red refinement of level l, so every fine edge is either
// half of a coarse edge or one of the three edges of the middle child of a
// coarse triangle.  Unknowns are values at edge midpoints (the trace form), so
// the transfer between levels is that of Crouzeix-Raviart functions:
//   prolongation  the coarse function v = sum_k v_k (1 - 2 lambda_k) on each
//                 coarse triangle, evaluated at the fine midpoints: (v_a + v_b)/2
//                 on the middle child's edge joining the midpoints of coarse
//                 edges a and b; on the half of coarse edge E_k next to vertex
//                 P_i (other end P_j) v_k - v_i/2 + v_j/2 (v_i on the edge
//                 opposite P_i), averaged over the two coarse triangles of E_k;
//   restriction   its transpose.
// Identity rows (Dirichlet edges) carry zero corrections on every level.
// Coarse operators are rediscretisations (the same assembly, a_T averaged
// over the four children).  Smoothing is a Chebyshev polynomial in D^-1 A on
// [b/ratio, b] with b the Gershgorin bound of D^-1 A, the same polynomial
// before and after the coarse correction, so the V-cycle is a symmetric
// positive definite preconditioner; the coarsest level is solved
// approximately by a fixed Chebyshev polynomial on an interval estimated by
// Lanczos, which keeps the whole preconditioner linear.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include <cooperative_groups.h>

#include "kernels.cuh"

struct phfem_mg_s {
  struct Level {
    phfem_mesh mesh = nullptr;
    phfem_sys sys = nullptr;
    bool owned = false;
    int nE = 0, nT = 0;
    void* rhs = nullptr;  // restricted right-hand side (coarse levels)
    void* z = nullptr;
    void* zb = nullptr;
    size_t zbytes = 0;  // bytes of the z, zb allocation
    void* d = nullptr;
    void* res = nullptr;
    int32_t* ct = nullptr;  // [nT][9] fine edges of each triangle (levels below the finest)
    int32_t* parent = nullptr;  // [nE] parent codes of this level's edges (levels above the coarsest)
    double b = 0.0;         // Gershgorin bound of D^-1 A
  };
  phfem_sys fine = nullptr;
  bool fp32 = false;
  std::vector<Level> L;
  int nu = 2;
  double ratio = 6.0;
  double coarse_a = 0.0, coarse_b = 0.0;
  int coarse_deg = 0;
  // the coarsest iteration in one cluster launch (k_mg_coarse), when its rows
  // fit the cluster's shared memory and PHFEM_MG_COARSE_STEPWISE is not set
  bool coarse_fused = false;
  int coarse_ctas = 1;         // CTAs of the cluster (1: a plain one-block launch)
  int coarse_threads = 1024;   // threads per CTA
  int coarse_per = 0;          // rows per CTA
  size_t coarse_smem = 0;      // dynamic shared memory per CTA
  double* coarse_coef = nullptr;  // [2][coarse_deg]: cd, then cr
};

namespace phfem {
namespace {

__device__ __forceinline__ bool skip(const SolveState* st, int want) { return st && st->done != want; }

// Chebyshev step in D^-1 A (difference form):
//   mode 0: d = cr D^-1 rhs, zout = d                       (from zero)
//   mode 1: d = cr D^-1 (rhs - A zin), zout = zin + d        (from zin)
//   mode 2: d = cd d + cr D^-1 (rhs - A zin), zout = zin + d
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

// One row of a Chebyshev step after the first (mode 1 with cd = 0, mode 2):
// the residual rhs - (A z)_e in difference form and the new d, with explicit
// fused multiply-adds so that every kernel that takes a step rounds alike.
template <typename T>
__device__ __forceinline__ T cheb_d(T rd, T l0, T l1, T l2, T l3, T pe, T g0, T g1, T g2, T g3, T rhs, T di, T dprev,
                                    T cd, T cr) {
  T sv = rd * pe;
  sv = fma_rn(l0, pe - g0, sv);
  sv = fma_rn(l1, pe - g1, sv);
  sv = fma_rn(l2, pe - g2, sv);
  sv = fma_rn(l3, pe - g3, sv);
  const T res = rhs - sv;
  return fma_rn(cd, dprev, cr * (di * res));
}

template <typename T>
__global__ void k_mg_cheb(int nE, const int32_t* __restrict__ nbr, const T* __restrict__ lval,
                          const T* __restrict__ rdiag, const T* __restrict__ dinv, const T* __restrict__ rhs,
                          const T* __restrict__ zin, T* __restrict__ zout, T* __restrict__ d, T cd, T cr, int mode,
                          const SolveState* st, int want) {
  pdl_enter();
  if (skip(st, want)) return;
  const size_t m = (size_t)nE;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nE; e += gridDim.x * blockDim.x) {
    if (mode == 0) {
      const T de = cr * (dinv[e] * rhs[e]);
      d[e] = de;
      zout[e] = de;
    } else {
      const T pe = zin[e];
      const T de = cheb_d(rdiag[e], lval[e], lval[m + e], lval[2 * m + e], lval[3 * m + e], pe,
                          __ldg(zin + nbr[e]), __ldg(zin + nbr[m + e]), __ldg(zin + nbr[2 * m + e]),
                          __ldg(zin + nbr[3 * m + e]), rhs[e], dinv[e], mode == 1 ? (T)0 : d[e],
                          mode == 1 ? (T)0 : cd, cr);
      d[e] = de;
      zout[e] = pe + de;
    }
  }
}

// The coarsest level's whole Chebyshev iteration in one launch: one block, or
// one cluster of up to kCoarseCluster CTAs, CTA r owning rows [r per,
// (r + 1) per).  Each CTA copies
// its rows' operator, D^-1 and right-hand side into shared memory once and
// keeps their z (two buffers) and d there; a step reads z at the neighbours
// from the owning CTA's shared memory (distributed shared memory) and ends
// with a cluster barrier.  The per-row arithmetic is k_mg_cheb's (cheb_d: from
// zero, then mode 2), so the result is bitwise the step-per-launch iteration's;
// ~100 launches of a few microseconds each become one.
constexpr int kCoarseCluster = 8;
constexpr int kCoarseThreads = 1024;

template <typename T>
__global__ void __launch_bounds__(kCoarseThreads) k_mg_coarse(int nE, int per, const int32_t* __restrict__ nbr,
                                                              const T* __restrict__ lval,
                                                              const T* __restrict__ rdiag,
                                                              const T* __restrict__ dinv, const T* __restrict__ rhs,
                                                              T* __restrict__ zout, int deg,
                                                              const double* __restrict__ coef, const SolveState* st,
                                                              int want) {
  namespace cgr = cooperative_groups;
  cgr::cluster_group cl = cgr::this_cluster();
  extern __shared__ __align__(16) unsigned char coarse_smem[];
  pdl_enter();
  if (skip(st, want)) return;  // the same for every CTA of the cluster
  const size_t m = (size_t)nE;
  const int rank = (int)cl.block_rank();
  const int e0 = rank * per;
  const int cnt = max(0, min(per, nE - e0));
  int* snb = reinterpret_cast<int*>(coarse_smem);  // [4][per]
  T* sl = reinterpret_cast<T*>(snb + 4 * per);      // [4][per]
  T* srd = sl + 4 * per;
  T* sdi = srd + per;
  T* srh = sdi + per;
  T* sz = srh + per;  // [2][per]
  T* sd = sz + 2 * per;
  for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
    const int e = e0 + j;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      snb[k * per + j] = nbr[k * m + e];
      sl[k * per + j] = lval[k * m + e];
    }
    srd[j] = rdiag[e];
    sdi[j] = dinv[e];
    srh[j] = rhs[e];
  }
  __syncthreads();
  auto zat = [&](const T* zc, int c) -> T {  // z of row c, from the CTA that owns it
    const int owner = c / per, j = c - owner * per;
    if (owner == rank) return zc[j];
    return *cl.map_shared_rank(const_cast<T*>(zc) + j, owner);
  };
  int cur = 0;
  for (int k = 0; k < deg; ++k) {
    const T cd = (T)coef[k], cr = (T)coef[deg + k];
    T* zc = sz + cur * per;
    if (k == 0) {  // from zero: d = cr D^-1 rhs, z = d
      for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
        const T de = cr * (sdi[j] * srh[j]);
        sd[j] = de;
        zc[j] = de;
      }
    } else {
      T* zn = sz + (cur ^ 1) * per;
      for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
        const T pe = zc[j];
        const T de = cheb_d(srd[j], sl[j], sl[per + j], sl[2 * per + j], sl[3 * per + j], pe, zat(zc, snb[j]),
                            zat(zc, snb[per + j]), zat(zc, snb[2 * per + j]), zat(zc, snb[3 * per + j]), srh[j],
                            sdi[j], sd[j], cd, cr);
        sd[j] = de;
        zn[j] = pe + de;
      }
      cur ^= 1;
    }
    cl.sync();  // this step's z is complete in every CTA before the next reads it
  }
  const T* zc = sz + cur * per;
  for (int j = threadIdx.x; j < cnt; j += blockDim.x) zout[e0 + j] = zc[j];
}

template <typename T>
__global__ void k_mg_residual(int nE, const int32_t* __restrict__ nbr, const T* __restrict__ lval,
                              const T* __restrict__ rdiag, const T* __restrict__ rhs, const T* __restrict__ z,
                              T* __restrict__ res, const SolveState* st, int want) {
  pdl_enter();
  if (skip(st, want)) return;
  const size_t m = (size_t)nE;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nE; e += gridDim.x * blockDim.x)
    res[e] = rhs[e] - spmv_row(nbr, lval, rdiag, z, m, e);
}

// Parent of every fine edge (for the prolongation, one fine edge per thread):
// (3t + k) << 2 for the middle-child edge opposite M_k of coarse triangle t,
// (E << 2) | 1 and (E << 2) | 2 for the halves of coarse edge E next to
// P_{kp+1} and P_{kp+2} of its T+, and 3 for identity rows (no correction).
__global__ void k_mg_parent(int nTc, int nEc, const int32_t* __restrict__ ed2el, const uint8_t* __restrict__ lk,
                            const int32_t* __restrict__ ct, const uint8_t* __restrict__ eclass_f, uint8_t ident,
                            int32_t* __restrict__ parent) {
  const int n = nTc + nEc;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (i < nTc) {
      for (int k = 0; k < 3; ++k) parent[ct[9 * (size_t)i + k]] = (3 * i + k) << 2;
    } else {
      const int E = i - nTc;
      const int tp = ed2el[4 * E + 2], kp = lk[E] & 3;
      const int hA = ct[9 * (size_t)tp + 3 + 2 * kp], hB = ct[9 * (size_t)tp + 4 + 2 * kp];
      parent[hA] = eclass_f[hA] == ident ? 3 : ((E << 2) | 1);
      parent[hB] = eclass_f[hB] == ident ? 3 : ((E << 2) | 2);
    }
  }
}

// zf += P zc, one fine edge per thread (coalesced on the fine side).
template <typename T>
__global__ void k_mg_prolong_f(int nEf, const int32_t* __restrict__ parent, const int32_t* __restrict__ t2e,
                               const int32_t* __restrict__ ed2el, const uint8_t* __restrict__ lk,
                               const T* __restrict__ zc, T* __restrict__ zf, const SolveState* st, int want) {
  pdl_enter();
  if (skip(st, want)) return;
  for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < nEf; f += gridDim.x * blockDim.x) {
    const int code = parent[f], type = code & 3, id = code >> 2;
    if (type == 3) continue;
    T val;
    if (type == 0) {  // joins the midpoints of edges k + 1 and k + 2 of coarse triangle t
      const int t = id / 3, k = id - 3 * t;
      val = (T)0.5 * (zc[t2e[3 * t + (k + 1) % 3]] + zc[t2e[3 * t + (k + 2) % 3]]);
    } else {
      const int E = id;
      const int tp = ed2el[4 * E + 2], tm = ed2el[4 * E + 3];
      const int kp = lk[E] & 3, km = (lk[E] >> 2) & 3;
      const T v = zc[E];
      const T p1 = zc[t2e[3 * tp + (kp + 1) % 3]], p2 = zc[t2e[3 * tp + (kp + 2) % 3]];
      // A: next to P_{kp+1} of T+ (P_{km+2} of T-); B: next to P_{kp+2} (P_{km+1} of T-)
      val = type == 1 ? v - (T)0.5 * p1 + (T)0.5 * p2 : v - (T)0.5 * p2 + (T)0.5 * p1;
      if (tm >= 0) {
        const T m1 = zc[t2e[3 * tm + (km + 1) % 3]], m2 = zc[t2e[3 * tm + (km + 2) % 3]];
        val = (T)0.5 * (val + (type == 1 ? v - (T)0.5 * m2 + (T)0.5 * m1 : v - (T)0.5 * m1 + (T)0.5 * m2));
      }
    }
    zf[f] += val;
  }
}

// rc = P' rf, one coarse edge per thread (zero on identity rows).
template <typename T>
__global__ void k_mg_restrict(int nEc, const int32_t* __restrict__ t2e, const int32_t* __restrict__ ed2el,
                              const uint8_t* __restrict__ lk, const uint8_t* __restrict__ eclass_c, uint8_t ident,
                              const int32_t* __restrict__ ct, const T* __restrict__ rf, T* __restrict__ rc,
                              const SolveState* st, int want) {
  pdl_enter();
  if (skip(st, want)) return;
  for (int E = blockIdx.x * blockDim.x + threadIdx.x; E < nEc; E += gridDim.x * blockDim.x) {
    if (eclass_c[E] == ident) {
      rc[E] = (T)0;
      continue;
    }
    const int tp = ed2el[4 * E + 2], tm = ed2el[4 * E + 3];
    const int kp = lk[E] & 3, km = (lk[E] >> 2) & 3;
    // its own halves (weight 1)
    T acc = rf[ct[9 * (size_t)tp + 3 + 2 * kp]] + rf[ct[9 * (size_t)tp + 4 + 2 * kp]];
    for (int side = 0; side < 2; ++side) {
      const int t = side == 0 ? tp : tm;
      if (t < 0) break;
      const int mloc = side == 0 ? kp : km;
      const int32_t* c = ct + 9 * (size_t)t;
      const int k1 = (mloc + 1) % 3, k2 = (mloc + 2) % 3;
      // middle-child edges touching the midpoint of E (weight 1/2 each)
      acc += (T)0.5 * (rf[c[k1]] + rf[c[k2]]);
      // halves of the other two edges, averaged over their triangles
      const T w1 = ed2el[4 * t2e[3 * t + k1] + 3] >= 0 ? (T)0.25 : (T)0.5;
      const T w2 = ed2el[4 * t2e[3 * t + k2] + 3] >= 0 ? (T)0.25 : (T)0.5;
      acc += w1 * (rf[c[3 + 2 * k1]] - rf[c[4 + 2 * k1]]);  // E is edge k1 + 2 of t
      acc += w2 * (rf[c[4 + 2 * k2]] - rf[c[3 + 2 * k2]]);  // E is edge k2 + 1 of t
    }
    rc[E] = acc;
  }
}

// Fine edges of every coarse triangle from the refined mesh's t2e: the middle
// child t holds (opposite its vertex M_k) the edge joining the other two
// midpoints; corner child nT + 3t + j = [P_j, M_{j+2}, M_{j+1}] holds the half
// of edge j + 2 next to P_j as its edge 2 and the half of edge j + 1 next to
// P_j as its edge 1.  ct[t] = {g0, g1, g2, h00, h01, h10, h11, h20, h21} with
// hk0 / hk1 the half of edge k next to P_{k+1} / P_{k+2}.  Also checks that the
// fine mesh is the red refinement of the coarse one.
__global__ void k_mg_ct(int nTc, int nVc, const int32_t* __restrict__ tri_c, const int32_t* __restrict__ t2e_c,
                        const int32_t* __restrict__ tri_f, const int32_t* __restrict__ t2e_f, int32_t* __restrict__ ct,
                        int* __restrict__ bad) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nTc; t += gridDim.x * blockDim.x) {
    bool ok = true;
    for (int k = 0; k < 3; ++k) {
      ok = ok && tri_f[3 * t + k] == nVc + t2e_c[3 * t + k];
      ok = ok && tri_f[3 * ((size_t)nTc + 3 * t + k)] == tri_c[3 * t + k];
    }
    if (!ok) atomicOr(bad, 1);
    int32_t* c = ct + 9 * (size_t)t;
    for (int k = 0; k < 3; ++k) {
      c[k] = t2e_f[3 * t + k];
      c[3 + 2 * k] = t2e_f[3 * ((size_t)nTc + 3 * t + (k + 1) % 3) + 2];
      c[4 + 2 * k] = t2e_f[3 * ((size_t)nTc + 3 * t + (k + 2) % 3) + 1];
    }
  }
}

__global__ void k_mg_coarsen_a(int nTc, const double* __restrict__ af, double* __restrict__ ac) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nTc; t += gridDim.x * blockDim.x) {
    const size_t c = (size_t)nTc + 3 * (size_t)t;
    ac[t] = 0.25 * (af[t] + af[c] + af[c + 1] + af[c + 2]);
  }
}

// max over rows of (A_ee + sum |A_es|) / A_ee from the FP64 difference-form rows.
__global__ void k_mg_gershgorin(int nE, const int32_t* __restrict__ nbr, const double* __restrict__ val,
                                unsigned int* __restrict__ out) {
  const size_t m = (size_t)nE;
  float best = 0.0f;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nE; e += gridDim.x * blockDim.x) {
    double diag = val[e], off = 0.0;
    for (int s = 0; s < 4; ++s) {
      const double l = val[(s + 1) * m + e];
      if (nbr[s * m + e] != e) {
        diag += l;
        off += fabs(l);
      }
    }
    best = fmaxf(best, (float)((diag + off) / diag) * 1.0001f);
  }
  // block maximum, then one atomic per block (positive floats order like their bit patterns)
  for (int o = 16; o > 0; o >>= 1) best = fmaxf(best, __shfl_down_sync(0xffffffffu, best, o));
  __shared__ float wmax[kBlock / 32];
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x == 0) {
    float b = 0.0f;
    for (int w = 0; w < kBlock / 32; ++w) b = fmaxf(b, wmax[w]);
    atomicMax(out, __float_as_uint(b));
  }
}

// Largest and smallest eigenvalue of a symmetric tridiagonal matrix by
// bisection on Sturm sequence counts.
double tridiag_eig(const std::vector<double>& a, const std::vector<double>& b, int which_smallest) {
  const int n = (int)a.size();
  double lo = 1e300, hi = -1e300;
  for (int i = 0; i < n; ++i) {
    const double r = (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < n ? std::fabs(b[i]) : 0.0);
    lo = std::min(lo, a[i] - r);
    hi = std::max(hi, a[i] + r);
  }
  auto count_below = [&](double x) {  // eigenvalues < x
    int c = 0;
    double q = a[0] - x;
    if (q < 0) ++c;
    for (int i = 1; i < n; ++i) {
      const double qq = q == 0.0 ? 1e-300 : q;
      q = a[i] - x - b[i - 1] * b[i - 1] / qq;
      if (q < 0) ++c;
    }
    return c;
  };
  const int target = which_smallest ? 1 : n;  // the target-th eigenvalue
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (count_below(mid) >= target) hi = mid;
    else lo = mid;
  }
  return 0.5 * (lo + hi);
}

// Lanczos on B = D^-1/2 A D^-1/2 restricted to the rows that are not identity
// rows (FP64, on the host): extreme Ritz values.  In difference form
// B = I - W with W_es = l_es / sqrt(A_ee A_ss) on the neighbour slots.  Runs
// until the smallest Ritz value changes by less than 3 % over 20 steps, or
// `kmax` steps.
void lanczos_bounds(int nE, const std::vector<int32_t>& nbr, const std::vector<double>& val,
                    const std::vector<uint8_t>& eclass, uint8_t ident, int kmax, double& lmin, double& lmax) {
  const size_t m = (size_t)nE;
  std::vector<double> sq(nE);
  for (int e = 0; e < nE; ++e) {
    double d = val[e];
    for (int s = 0; s < 4; ++s)
      if (nbr[s * m + e] != e) d += val[(s + 1) * m + e];
    sq[e] = eclass[e] == ident ? 0.0 : 1.0 / std::sqrt(d);
  }
  std::vector<double> W(4 * m, 0.0);
  std::vector<int32_t> C(4 * m, 0);
  for (int e = 0; e < nE; ++e)
    for (int s = 0; s < 4; ++s) {
      const int c = nbr[s * m + e];
      C[s * m + e] = c;
      if (c != e) W[s * m + e] = val[(s + 1) * m + e] * sq[e] * sq[c];
    }
  // start from the constant vector on the free rows: it is smooth, so it holds
  // a large component along the lowest eigenvectors and the smallest Ritz value
  // settles in about half the steps a random start needs
  std::vector<double> v(nE), vp(nE, 0.0), w(nE);
  double nrm = 0.0;
  for (int e = 0; e < nE; ++e) {
    v[e] = sq[e] == 0.0 ? 0.0 : 1.0;
    nrm += v[e] * v[e];
  }
  lmin = lmax = 1.0;
  if (nrm == 0.0) return;  // identity rows only
  nrm = std::sqrt(nrm);
  for (double& x : v) x /= nrm;
  std::vector<double> al, be;
  double beta = 0.0, prev_min = 0.0;
  for (int j = 0; j < kmax; ++j) {
    double a = 0.0;
    for (int e = 0; e < nE; ++e) {
      double t = sq[e] == 0.0 ? 0.0 : v[e];
      for (int s = 0; s < 4; ++s) t -= W[s * m + e] * v[C[s * m + e]];
      t -= beta * vp[e];
      w[e] = t;
      a += t * v[e];
    }
    double bn = 0.0;
    for (int e = 0; e < nE; ++e) {
      w[e] -= a * v[e];
      bn += w[e] * w[e];
    }
    bn = std::sqrt(bn);
    al.push_back(a);
    const bool last = bn < 1e-300 || j + 1 == kmax;
    if ((j + 1) % 20 == 0 || last) {
      std::vector<double> bb(be.begin(), be.end());
      lmin = tridiag_eig(al, bb, 1);
      lmax = tridiag_eig(al, bb, 0);
      if (j + 1 >= 40 && std::fabs(lmin - prev_min) < 0.03 * lmin) break;
      prev_min = lmin;
    }
    if (last) break;
    be.push_back(bn);
    for (int e = 0; e < nE; ++e) {
      vp[e] = v[e];
      v[e] = w[e] / bn;
    }
    beta = bn;
  }
}

// Chebyshev coefficients (cd_k, cr_k) of degree `deg` on [a, b].
void cheb_coeffs(double a, double b, int deg, std::vector<double>& cd, std::vector<double>& cr) {
  const double th = 0.5 * (b + a), de = 0.5 * (b - a), sig = th / de;
  cd.assign(deg, 0.0);
  cr.assign(deg, 0.0);
  double rho = 1.0 / sig;
  cr[0] = 1.0 / th;
  for (int k = 1; k < deg; ++k) {
    const double rn = 1.0 / (2.0 * sig - rho);
    cd[k] = rn * rho;
    cr[k] = 2.0 * rn / de;
    rho = rn;
  }
}

template <typename T>
struct MgRun {
  phfem_mg mg;
  cudaStream_t s;
  const SolveState* st;
  int want;

  phfem_ctx ctx(int l) const { return mg->L[l].mesh->ctx; }

  // The finest level's z, zb stay in L2 when the set-aside reserved for the
  // iteration's window (r, p: the same size) can hold them.
  L2Window window(int l) const {
    L2Window w;
    const phfem_mg_s::Level& Lv = mg->L[l];
    phfem_ctx c = ctx(l);
    if (l + 1 != (int)mg->L.size() || !c->l2_window || Lv.zbytes == 0 || c->l2_limit < Lv.zbytes ||
        Lv.zbytes > c->l2_window_max)
      return w;
    w.base = Lv.z;
    w.bytes = Lv.zbytes;
    w.hit_ratio = 1.0f;
    return w;
  }

  int smooth(int l, const T* rhs, T* zin_out_first, T* zalt, bool from_zero, int deg, const double* cd,
             const double* cr, T** result) {
    // alternates between the two buffers; returns the buffer with the result
    phfem_mg_s::Level& Lv = mg->L[l];
    phfem_sys sy = Lv.sys;
    const int g = grid_for(ctx(l), Lv.nE);
    T* cur = zin_out_first;
    T* other = zalt;
    for (int k = 0; k < deg; ++k) {
      const int mode = k == 0 ? (from_zero ? 0 : 1) : 2;
      T* out = (k == 0 && from_zero) ? cur : other;
      PH_CUDA(launch_pdl_w(window(l), k_mg_cheb<T>, g, s, Lv.nE, Lv.mesh->nbr, (const T*)sy->lval, (const T*)sy->rdiag,
                         (const T*)sy->dinv, rhs, (const T*)cur, out, (T*)Lv.d, (T)cd[k], (T)cr[k], mode, st, want));
      PH_TRY(check_launch(ctx(l), "k_mg_cheb"));
      if (out != cur) std::swap(cur, other);
    }
    *result = cur;
    return PHFEM_OK;
  }

  // z_l = V(rhs_l); the result is written to `z_out`.
  int vcycle(int l, const T* rhs, T* z_out) {
    phfem_mg_s::Level& Lv = mg->L[l];
    T* zb = (T*)Lv.zb;
    T* res = nullptr;
    if (l == 0 && mg->coarse_fused) {
      phfem_sys sy = Lv.sys;
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(mg->coarse_ctas);
      cfg.blockDim = dim3(mg->coarse_threads);
      cfg.dynamicSmemBytes = mg->coarse_smem;
      cfg.stream = s;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = mg->coarse_ctas;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = mg->coarse_ctas > 1 ? 1 : 0;
      PH_CUDA(cudaLaunchKernelEx(&cfg, k_mg_coarse<T>, Lv.nE, mg->coarse_per, (const int32_t*)Lv.mesh->nbr,
                                 (const T*)sy->lval, (const T*)sy->rdiag, (const T*)sy->dinv, rhs, z_out,
                                 mg->coarse_deg, (const double*)mg->coarse_coef, st, want));
      return check_launch(ctx(l), "k_mg_coarse");
    }
    if (l == 0) {
      std::vector<double> cd, cr;
      cheb_coeffs(mg->coarse_a, mg->coarse_b, mg->coarse_deg, cd, cr);
      // writes alternate starting at the first buffer: start so that the last lands in z_out
      T* first = (mg->coarse_deg % 2 == 1) ? z_out : zb;
      T* second = first == z_out ? zb : z_out;
      T* outp = nullptr;
      PH_TRY(smooth(0, rhs, first, second, true, mg->coarse_deg, cd.data(), cr.data(), &outp));
      if (outp != z_out) return fail(PHFEM_ECUDA, "multigrid: coarse buffer parity");
      return PHFEM_OK;
    }
    std::vector<double> cd, cr;
    cheb_coeffs(Lv.b / mg->ratio, Lv.b, mg->nu, cd, cr);
    // pre-smoothing: nu writes starting in zb; the post-smoothing's nu writes
    // then end in z_out (2 nu writes alternate zb, z_out, ...)
    T* cur = nullptr;
    PH_TRY(smooth(l, rhs, zb, z_out, true, mg->nu, cd.data(), cr.data(), &cur));
    res = (T*)Lv.res;
    const int g = grid_for(ctx(l), Lv.nE);
    phfem_sys sy = Lv.sys;
    PH_CUDA(launch_pdl_w(window(l), k_mg_residual<T>, g, s, Lv.nE, Lv.mesh->nbr, (const T*)sy->lval,
                         (const T*)sy->rdiag, rhs,
                       (const T*)cur, res, st, want));
    PH_TRY(check_launch(ctx(l), "k_mg_residual"));
    phfem_mg_s::Level& C = mg->L[l - 1];
    PH_CUDA(launch_pdl(k_mg_restrict<T>, grid_for(ctx(l), C.nE), s, C.nE, C.mesh->t2e, C.mesh->ed2el, C.mesh->lk,
                       C.mesh->eclass, C.sys->ident_class, C.ct, (const T*)res, (T*)C.rhs, st, want));
    PH_TRY(check_launch(ctx(l), "k_mg_restrict"));
    PH_TRY(vcycle(l - 1, (const T*)C.rhs, (T*)C.z));
    PH_CUDA(launch_pdl_w(window(l), k_mg_prolong_f<T>, grid_for(ctx(l), Lv.nE), s, Lv.nE, Lv.parent, C.mesh->t2e,
                       C.mesh->ed2el, C.mesh->lk, (const T*)C.z, cur, st, want));
    PH_TRY(check_launch(ctx(l), "k_mg_prolong_f"));
    T* alt = cur == zb ? z_out : zb;
    T* outp = nullptr;
    PH_TRY(smooth(l, rhs, cur, alt, false, mg->nu, cd.data(), cr.data(), &outp));
    if (outp != z_out) return fail(PHFEM_ECUDA, "multigrid: buffer parity");
    return PHFEM_OK;
  }
};

void mg_free(phfem_mg mg) {
  for (size_t l = 0; l < mg->L.size(); ++l) {
    phfem_mg_s::Level& Lv = mg->L[l];
    if (!Lv.mesh) continue;
    phfem_ctx c = Lv.mesh->ctx;
    dfree(c, Lv.rhs);
    dfree(c, Lv.z);  // zb lives in the same allocation
    dfree(c, Lv.d);
    dfree(c, Lv.res);
    dfree(c, Lv.ct);
    dfree(c, Lv.parent);
    if (l == 0) dfree(c, mg->coarse_coef);
    if (Lv.owned && Lv.sys) phfem_sys_destroy(Lv.sys);
  }
  if (mg->fine && mg->fine->mg == mg) mg->fine->mg = nullptr;
  delete mg;
}

}  // namespace

int mg_apply(phfem_mg mg, cudaStream_t s, const void* r, const SolveState* st, int want) {
  const int top = (int)mg->L.size() - 1;
  if (mg->fp32) {
    MgRun<float> R{mg, s, st, want};
    return R.vcycle(top, (const float*)r, (float*)mg->L[top].z);
  }
  MgRun<double> R{mg, s, st, want};
  return R.vcycle(top, (const double*)r, (double*)mg->L[top].z);
}

void* mg_fine_z(phfem_mg mg) { return mg->L.back().z; }

void mg_forget_system(phfem_mg mg) {
  mg->fine = nullptr;
  if (!mg->L.empty()) mg->L.back().sys = nullptr;
}

}  // namespace phfem

using namespace phfem;

extern "C" {

PHFEM_API int phfem_mg_create(phfem_sys sys, int32_t nlevels, const phfem_mesh* meshes, const double* a_T,
                              const phfem_mg_opts* opts, phfem_mg* out) {
  if (!out) return fail(PHFEM_EINVAL, "phfem_mg_create: out is NULL");
  *out = nullptr;
  if (!sys || !meshes || nlevels < 2) return fail(PHFEM_EINVAL, "phfem_mg_create: a system and >= 2 levels");
  if (meshes[nlevels - 1] != sys->mesh)
    return fail(PHFEM_EINVAL, "phfem_mg_create: the finest mesh must be the system's mesh");
  if (sys->form != PHFEM_FORM_TRACE) return fail(PHFEM_EINVAL, "phfem_mg_create: the trace form only");
  if (sys->conv) return fail(PHFEM_EINVAL, "phfem_mg_create: symmetric systems only (no convection)");
  phfem_mg_opts o{};
  if (opts) o = *opts;
  if (o.nu <= 0) o.nu = 2;
  if (!(o.smooth_ratio > 1.0)) o.smooth_ratio = 6.0;
  if (!(o.coarse_eps > 0.0 && o.coarse_eps < 1.0)) o.coarse_eps = 0.3;
  if (o.nu > 16 || o.coarse_degree < 0 || o.coarse_degree > 2000)
    return fail(PHFEM_EINVAL, "phfem_mg_create: nu in 1..16, coarse_degree in 0..2000");
  phfem_ctx ctx = sys->mesh->ctx;
  cudaStream_t s = ctx->stream;
  for (int l = 0; l < nlevels; ++l)
    if (!meshes[l] || meshes[l]->ctx != ctx) return fail(PHFEM_EINVAL, "phfem_mg_create: NULL mesh or another context");
  for (int l = 0; l + 1 < nlevels; ++l) {
    const phfem_mesh_info& C = meshes[l]->info;
    const phfem_mesh_info& F = meshes[l + 1]->info;
    if (F.nT != 4 * (int64_t)C.nT || F.nV != (int64_t)C.nV + C.nE)
      return fail(PHFEM_EINVAL, "phfem_mg_create: level " + std::to_string(l + 1) +
                                    " is not the red refinement of level " + std::to_string(l));
    if (12 * (int64_t)C.nT >= (int64_t)INT32_MAX || 4 * (int64_t)C.nE >= (int64_t)INT32_MAX)
      return fail(PHFEM_EINVAL, "phfem_mg_create: a coarse level exceeds the transfer tables' index range");
  }
  phfem_mg mg = new phfem_mg_s();
  mg->fine = sys;
  mg->fp32 = sys->fp32;
  mg->nu = o.nu;
  mg->ratio = o.smooth_ratio;
  mg->L.resize(nlevels);
  const size_t es = sys->fp32 ? sizeof(float) : sizeof(double);
  int st = PHFEM_OK;
  auto chk = [&](int r) {
    if (st == PHFEM_OK) st = r;
  };
  // device scratch: [0] bad flag, [1 .. nlevels] Gershgorin bounds (float bits)
  unsigned int* flags = nullptr;
  chk(dalloc_n(ctx, &flags, (size_t)nlevels + 1));
  if (st == PHFEM_OK) {
    cudaError_t e = cudaMemsetAsync(flags, 0, sizeof(unsigned int) * (nlevels + 1), s);
    if (e != cudaSuccess) st = cuda_fail(e, "cudaMemsetAsync", __FILE__, __LINE__);
  }
  // transfer tables (checking the refinement structure) and vectors
  for (int l = 0; l < nlevels && st == PHFEM_OK; ++l) {
    phfem_mg_s::Level& Lv = mg->L[l];
    Lv.mesh = meshes[l];
    Lv.nE = meshes[l]->info.nE;
    Lv.nT = meshes[l]->info.nT;
    if (l + 1 < nlevels) {
      chk(dalloc_n(ctx, &Lv.ct, 9 * (size_t)Lv.nT));
      if (st != PHFEM_OK) break;
      k_mg_ct<<<grid_for(ctx, Lv.nT), kBlock, 0, s>>>(Lv.nT, meshes[l]->info.nV, meshes[l]->tri, meshes[l]->t2e,
                                                      meshes[l + 1]->tri, meshes[l + 1]->t2e, Lv.ct,
                                                      reinterpret_cast<int*>(flags));
      chk(check_launch(ctx, "k_mg_ct"));
    }
    chk(dalloc(ctx, &Lv.rhs, es * Lv.nE + 16));
    {  // z and zb in one allocation (one L2 window covers both on the finest level)
      const size_t vb = (es * Lv.nE + 255) / 256 * 256;
      chk(dalloc(ctx, &Lv.z, 2 * vb));
      Lv.zb = st == PHFEM_OK ? (void*)((char*)Lv.z + vb) : nullptr;
      Lv.zbytes = 2 * vb;
    }
    chk(dalloc(ctx, &Lv.d, es * Lv.nE + 16));
    if (l > 0) chk(dalloc(ctx, &Lv.res, es * Lv.nE + 16));
  }
  // coefficients of every level (the fine a_T averaged over children), then
  // the coarse systems (rediscretisation), with no host synchronisation
  std::vector<double*> aT(nlevels, nullptr);
  if (st == PHFEM_OK && a_T) {
    aT[nlevels - 1] = const_cast<double*>(a_T);
    for (int l = nlevels - 2; l >= 0 && st == PHFEM_OK; --l) {
      chk(dalloc_n(ctx, &aT[l], (size_t)mg->L[l].nT));
      if (st != PHFEM_OK) break;
      k_mg_coarsen_a<<<grid_for(ctx, mg->L[l].nT), kBlock, 0, s>>>(mg->L[l].nT, aT[l + 1], aT[l]);
      chk(check_launch(ctx, "k_mg_coarsen_a"));
    }
  }
  for (int l = 0; l < nlevels && st == PHFEM_OK; ++l) {
    phfem_mg_s::Level& Lv = mg->L[l];
    if (l == nlevels - 1) {
      Lv.sys = sys;
      Lv.owned = false;
    } else {
      phfem_coeffs c = sys->c;
      c.a_T = a_T ? aT[l] : nullptr;
      c.form = PHFEM_FORM_TRACE;
      chk(assemble_system(meshes[l], c, nullptr, nullptr, &Lv.sys, false));
      Lv.owned = true;
    }
  }
  for (int l = nlevels - 2; l >= 0; --l)
    if (aT[l]) dfree(ctx, aT[l]);
  for (int l = 1; l < nlevels && st == PHFEM_OK; ++l) {
    phfem_mg_s::Level& F = mg->L[l];
    phfem_mg_s::Level& Cl = mg->L[l - 1];
    chk(dalloc_n(ctx, &F.parent, (size_t)F.nE));
    if (st != PHFEM_OK) break;
    k_mg_parent<<<grid_for(ctx, (int64_t)Cl.nT + Cl.nE), kBlock, 0, s>>>(Cl.nT, Cl.nE, Cl.mesh->ed2el, Cl.mesh->lk,
                                                                         Cl.ct, F.mesh->eclass, F.sys->ident_class,
                                                                         F.parent);
    chk(check_launch(ctx, "k_mg_parent"));
  }
  for (int l = 0; l < nlevels && st == PHFEM_OK; ++l) {
    phfem_mg_s::Level& Lv = mg->L[l];
    k_mg_gershgorin<<<grid_for(ctx, Lv.nE), kBlock, 0, s>>>(Lv.nE, Lv.mesh->nbr, Lv.sys->val, flags + 1 + l);
    chk(check_launch(ctx, "k_mg_gershgorin"));
  }
  // one read-back: flags, bounds and the coarsest level for the Lanczos run
  std::vector<unsigned int> hflags(nlevels + 1, 0);
  phfem_mg_s::Level& C = mg->L[0];
  const int n = C.nE;
  std::vector<int32_t> nbr(4 * (size_t)n);
  std::vector<double> val(5 * (size_t)n);
  std::vector<uint8_t> ec(n);
  if (st == PHFEM_OK) {
    cudaError_t e = cudaMemcpyAsync(hflags.data(), flags, sizeof(unsigned int) * hflags.size(),
                                    cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(nbr.data(), C.mesh->nbr, sizeof(int32_t) * nbr.size(), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(val.data(), C.sys->val, sizeof(double) * val.size(), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ec.data(), C.mesh->eclass, n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_fail(e, "phfem_mg_create: read-back", __FILE__, __LINE__);
    else if (hflags[0]) st = fail(PHFEM_EINVAL, "phfem_mg_create: a level is not the red refinement of the one below");
  }
  if (st == PHFEM_OK) {
    for (int l = 0; l < nlevels; ++l) {
      float fb;
      std::memcpy(&fb, &hflags[1 + l], sizeof(fb));
      mg->L[l].b = fb > 1.0f ? (double)fb : 1.0;
    }
    // interval and degree of the coarsest polynomial
    const int steps = n <= 200000 ? std::min(n, 400) : 60;
    double lmin = 0.0, lmax = 0.0;
    const auto t0 = std::chrono::steady_clock::now();
    lanczos_bounds(n, nbr, val, ec, C.sys->ident_class, steps, lmin, lmax);
    if (getenv("PHFEM_VERBOSE"))
      fprintf(stderr, "phfem: multigrid coarsest level %d rows, Ritz interval [%.4e, %.4e], %.2f ms\n", n, lmin,
              lmax, std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count());
    // Ritz values lie inside the spectrum: widen both ends
    mg->coarse_b = std::min(1.02 * lmax, C.b);
    mg->coarse_a = (n <= 200000 ? 0.85 : 0.25) * lmin;
    if (!(mg->coarse_a > 0.0) || !(mg->coarse_a < mg->coarse_b)) mg->coarse_a = mg->coarse_b * 1e-4;
    if (o.coarse_degree > 0) {
      mg->coarse_deg = o.coarse_degree;
    } else {
      const double kap = mg->coarse_b / mg->coarse_a;
      const double rho = (std::sqrt(kap) - 1.0) / (std::sqrt(kap) + 1.0);
      const int deg = rho > 0.0 ? (int)std::ceil(std::log(2.0 / o.coarse_eps) / std::log(1.0 / rho)) : 1;
      mg->coarse_deg = std::max(1, std::min(deg, 2000));
    }
  }
  if (st == PHFEM_OK && !(o.flags & PHFEM_MG_COARSE_STEPWISE)) {
    // the coarsest iteration as one cluster launch, if its rows fit
    // CTAs: one row per thread where possible, the fewest CTAs that give it (a
    // coarse level of a few hundred rows takes one small block, which the GPU
    // can place at once while other work runs; a cluster waits for SMs of
    // one GPC with room for all its CTAs)
    const int n = mg->L[0].nE;
    int ctas = 1;
    while (ctas < kCoarseCluster && ctas * kCoarseThreads < n) ctas *= 2;
    const int per = (n + ctas - 1) / ctas;
    const int threads = ctas > 1 ? kCoarseThreads : std::max(32, std::min(kCoarseThreads, (per + 31) / 32 * 32));
    const size_t tsz = mg->fp32 ? sizeof(float) : sizeof(double);
    const size_t smem = (size_t)per * (16 + 10 * tsz);
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    auto kern = mg->fp32 ? (const void*)k_mg_coarse<float> : (const void*)k_mg_coarse<double>;
    // the kernel's shared-memory limit is set to the device's largest, once
    // per process: a limit sized to one hierarchy would race with another's
    // launch (the request server creates hierarchies concurrently), and
    // changing a kernel's attributes can wait for that kernel's launches in
    // flight on other streams
    static const bool limit_set = [optin] {
      const bool a = cudaFuncSetAttribute(k_mg_coarse<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin) ==
                     cudaSuccess;
      const bool b = cudaFuncSetAttribute(k_mg_coarse<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin) ==
                     cudaSuccess;
      cudaGetLastError();
      return a && b;
    }();
    bool ok = smem <= (size_t)optin && limit_set;
    if (ok && ctas > 1) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(ctas);
      cfg.blockDim = dim3(threads);
      cfg.dynamicSmemBytes = smem;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = ctas;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      int clusters = 0;
      ok = cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg) == cudaSuccess && clusters >= 1;
    }
    cudaGetLastError();
    if (ok) {
      std::vector<double> cd, cr;
      cheb_coeffs(mg->coarse_a, mg->coarse_b, mg->coarse_deg, cd, cr);
      cd.insert(cd.end(), cr.begin(), cr.end());
      st = dalloc_n(ctx, &mg->coarse_coef, cd.size());
      if (st == PHFEM_OK) {
        cudaError_t e = cudaMemcpyAsync(mg->coarse_coef, cd.data(), sizeof(double) * cd.size(),
                                        cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // cd is a host temporary
        if (e != cudaSuccess) st = cuda_fail(e, "phfem_mg_create coarse coefficients", __FILE__, __LINE__);
      }
      mg->coarse_fused = st == PHFEM_OK;
      mg->coarse_ctas = ctas;
      mg->coarse_threads = threads;
      mg->coarse_per = per;
      mg->coarse_smem = smem;
    }
  }
  dfree(ctx, flags);
  if (st != PHFEM_OK) {
    cudaStreamSynchronize(s);
    mg_free(mg);
    return st;
  }
  *out = mg;
  return PHFEM_OK;
}

PHFEM_API int phfem_mg_info(phfem_mg mg, phfem_mg_info_t* out) {
  if (!mg || !out) return fail(PHFEM_EINVAL, "phfem_mg_info: NULL argument");
  out->levels = (int32_t)mg->L.size();
  out->nu = mg->nu;
  out->coarse_degree = mg->coarse_deg;
  out->coarse_a = mg->coarse_a;
  out->coarse_b = mg->coarse_b;
  out->smooth_ratio = mg->ratio;
  return PHFEM_OK;
}

PHFEM_API int phfem_sys_set_mg(phfem_sys sys, phfem_mg mg) {
  if (!sys) return fail(PHFEM_EINVAL, "phfem_sys_set_mg: NULL system");
  if (mg && mg->fine != sys) return fail(PHFEM_EINVAL, "phfem_sys_set_mg: the multigrid belongs to another system");
  sys->mg = mg;
  return PHFEM_OK;
}

PHFEM_API int phfem_mg_transfer(phfem_mg mg, int32_t level, int32_t direction, const double* in, double* out) {
  if (!mg || !in || !out) return fail(PHFEM_EINVAL, "phfem_mg_transfer: NULL argument");
  if (level < 0 || level + 1 >= (int)mg->L.size() || (direction != 0 && direction != 1))
    return fail(PHFEM_EINVAL, "phfem_mg_transfer: level in 0..levels-2, direction 0 or 1");
  phfem_mg_s::Level& C = mg->L[level];
  phfem_mg_s::Level& F = mg->L[level + 1];
  if (!F.sys) return fail(PHFEM_EINVAL, "phfem_mg_transfer: the multigrid's system was destroyed");
  phfem_ctx ctx = C.mesh->ctx;
  cudaStream_t s = ctx->stream;
  if (direction == 0) {
    PH_CUDA(cudaMemsetAsync(out, 0, sizeof(double) * F.nE, s));
    k_mg_prolong_f<double><<<grid_for(ctx, F.nE), kBlock, 0, s>>>(F.nE, F.parent, C.mesh->t2e, C.mesh->ed2el,
                                                                   C.mesh->lk, in, out, nullptr, 0);
    return check_launch(ctx, "k_mg_prolong_f");
  }
  k_mg_restrict<double><<<grid_for(ctx, C.nE), kBlock, 0, s>>>(C.nE, C.mesh->t2e, C.mesh->ed2el, C.mesh->lk,
                                                                C.mesh->eclass, C.sys->ident_class, C.ct, in, out,
                                                                nullptr, 0);
  return check_launch(ctx, "k_mg_restrict");
}

PHFEM_API int phfem_mg_destroy(phfem_mg mg) {
  if (!mg) return fail(PHFEM_EINVAL, "phfem_mg_destroy: NULL multigrid");
  mg_free(mg);
  return PHFEM_OK;
}

}  // extern "C"
