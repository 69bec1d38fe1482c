// Jacobi-preconditioned conjugate gradients on the condensed edge system,
// with an FP64 iterative refinement around FP32 (or FP64) inner iterations,
// and the recovery of the paper's unknowns U and Lambda (Wvec of Main.m).
//
// The system is stored per edge row (all nE edges; Dirichlet rows are identity
// rows holding u_D) in difference form (S p)_e = r_e p_e + sum_s l_es (p_e -
// p[nbr_s]) with l_es = -S_{e,nbr_s} and r_e the reaction/mass part of the
// diagonal: in FP64 (val[5][nE]) for the outer residual, and in the inner
// precision with the Jacobi inverse diagonal for the inner iterations.  The inner search direction is
// zero on Dirichlet rows, so the Dirichlet columns (kept in the free rows for
// the lifting) never act inside the iteration.
//
// Jacobi-PCG with reliable updates: the residual, direction and operator
// product live in the inner precision (FP32, or FP64; dot products sum each
// thread's few rows in that precision and accumulate across threads and
// blocks in FP64) while the solution x is accumulated in FP64 at every
// iteration (rounding a correction vector to FP32 would leave a residual of
// 2^-24 |S| |d|, far above |b| ~ h^2 on fine meshes).  Whenever the recursive
// residual has fallen by the factor inner_rtol since the last update, the true
// residual r = b - S x is recomputed in FP64 (difference form) and replaces
// the recursive one while the search direction is kept, so the Krylov space is
// not lost as in restarted refinement.  The first step after a replacement is
// an exact line search alpha = r.p / p.Ap (in exact CG r.p = r.z; with the
// replaced residual the plain formula can diverge), and the direction is
// restarted (p = D^-1 r) when r.p <= 0 or when the true residual is far above
// the recursive one.  The solve stops when
// ||r|| <= rtol ||b_free||, or when ||r|| reaches the level that rounding x to
// FP64 alone leaves (estimated from |l| |x| per row), which on fine meshes can
// exceed rtol because b scales like h^2 while S does not.
// Every kernel is a grid-stride loop; reductions write one partial per block
// and the last block to arrive sums the partials in a fixed order
// (deterministic results, no floating-point atomics).
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>

#include "kernels.cuh"

namespace phfem {
namespace {

// The solution of a solve is x = (xh + xl) + y: an unevaluated FP64 pair
// and the FP64 correction y accumulated by the iterations since the last
// reliable update (the vector sys->x during the solve).  k_dd_begin moves the
// start vector into the pair, k_dd_fold adds y into it before every true
// residual, and k_dd_end leaves the rounded sum in sys->x.
__global__ void k_dd_begin(int nE, double* __restrict__ x, double* __restrict__ xh, double* __restrict__ xl) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nE; e += gridDim.x * blockDim.x) {
    xh[e] = x[e];
    xl[e] = 0.0;
    x[e] = 0.0;
  }
}

__global__ void k_dd_fold(int nE, double* __restrict__ x, double* __restrict__ xh, double* __restrict__ xl,
                          const SolveState* st, int cond) {
  if (cond && st->done != 1) return;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nE; e += gridDim.x * blockDim.x) {
    double h = xh[e], l = xl[e];
    dd_add(h, l, x[e]);
    xh[e] = h;
    xl[e] = l;
    x[e] = 0.0;
  }
}

__global__ void k_dd_end(int nE, double* __restrict__ x, const double* __restrict__ xh,
                         const double* __restrict__ xl) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nE; e += gridDim.x * blockDim.x) {
    double h = xh[e], l = xl[e];
    dd_add(h, l, x[e]);
    x[e] = h + l;
  }
}

// r = b - S x (FP64, x = xh + xl after the fold); inner start vectors;
// reductions ||r||^2, r.D^-1 r, the evaluation floor and (after an update)
// r.p.  Modes:
//   0  ||b_free||^2 with the Dirichlet lifting (x replaced by (0, u_D));
//   1  start: p = D^-1 r;
//   2  reliable update: the true residual replaces the recursive one, p kept;
//   3  as 2, but only if the iteration asked for an update (done == 1).
// The last block decides on the device (decide()): converged (rtol, or twice
// the evaluation floor), the line-search step, or a restart of the direction.
// With precond != 0 (multigrid) the kernel only forms r and the sums ||r||^2
// and the floor; the preconditioner and k_mg_finish complete the step.
template <typename T>
__global__ void k_residual(int nE, const int32_t* __restrict__ nbr, const double* __restrict__ val,
                           const double* __restrict__ b, const double* __restrict__ xh,
                           const double* __restrict__ xl, const uint8_t* __restrict__ eclass, uint8_t ident,
                           const T* __restrict__ dinv, T* __restrict__ ri, T* __restrict__ pi, double* partials,
                           SolveState* st, double rtol2, double inner_rtol2, int mode, int precond) {
  if (mode == 3) {
    if (st->done != 1) return;  // every block reads done before the last block rewrites it
    mode = 2;
  }
  __shared__ double smem[kBlock / 32];
  const size_t m = (size_t)nE;
  double acc_r = 0.0, acc_z = 0.0, acc_f = 0.0, acc_p = 0.0;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nE; e += gridDim.x * blockDim.x) {
    double r;
    if (mode == 0) {
      if (eclass[e] == ident) {  // identity rows hold their fixed value
        r = 0.0;
      } else {
        r = b[e];
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          const int c = nbr[s * m + e];
          if (c != e && eclass[c] == ident) r += val[(s + 1) * m + e] * b[c];
        }
      }
      acc_r += r * r;
    } else {
      double fl;  // scale of the row's own rounding
      r = residual_row(nbr, val, b, xh, xl, m, e, fl);
      acc_r += r * r;
      fl *= 0x1p-53;
      acc_f += fl * fl;
      const T rs = (T)r;
      ri[e] = rs;
      if (!precond) {
        const T zs = dinv[e] * rs;
        if (mode == 1) pi[e] = zs;
        else acc_p += (double)rs * (double)pi[e];
        acc_z += (double)rs * (double)zs;
      }
    }
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
    if (precond) {  // completed by k_mg_finish
      st->rr_pending = rr;
      st->ff_pending = ff;
      return;
    }
    decide(st, rr, rz, ff, rp, mode, rtol2, inner_rtol2);
  }
}

// Completes a true residual under the multigrid preconditioner: z = M^-1 r is
// in zi; rz = r.z, and p = z at the start (mode 1) or r.p for the line search
// (mode 2; mode 3 = mode 2 when the iteration asked for it).
template <typename T>
__global__ void k_mg_finish(int nE, const T* __restrict__ ri, const T* __restrict__ zi, T* __restrict__ pi,
                            double* partials, SolveState* st, double rtol2, double inner_rtol2, int mode) {
  pdl_enter();
  if (mode == 3) {
    if (st->done != 1) return;
    mode = 2;
  }
  __shared__ double smem[kBlock / 32];
  T acc_z = (T)0, acc_p = (T)0;  // this thread's few rows in T; across threads and blocks in FP64
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nE; e += gridDim.x * blockDim.x) {
    const T r = ri[e], z = zi[e];
    acc_z += r * z;
    if (mode == 1) pi[e] = z;
    else acc_p += r * pi[e];
  }
  const double sz = block_sum((double)acc_z, smem);
  const double sp = block_sum((double)acc_p, smem);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = sz;
    partials[kMaxGrid + blockIdx.x] = sp;
  }
  if (!arrive_last(&st->counter[3])) return;
  const double rz = sum_partials(partials, smem);
  const double rp = sum_partials(partials + kMaxGrid, smem);
  if (threadIdx.x == 0) {
    st->counter[3] = 0;
    decide(st, st->rr_pending, rz, st->ff_pending, rp, mode, rtol2, inner_rtol2);
  }
}

// q = S p in difference form, p.q -> alpha = rz / p.q (or r.p / p.q right
// after a reliable update).  In restart mode the direction is first set to
// p = D^-1 r, or to the stored z = M^-1 r (zsrc) under multigrid (each block
// writes its own rows and takes neighbours' values from r and D^-1 or from z,
// so no block reads p being written).
template <typename T>
__global__ void __launch_bounds__(kBlock) k_cg_spmv(int nE, const int32_t* __restrict__ nbr,
                                                    const T* __restrict__ lval, const T* __restrict__ rdiag,
                                                    T* __restrict__ p, T* __restrict__ q, const T* __restrict__ r,
                                                    const T* __restrict__ dinv, const T* __restrict__ zsrc,
                                                    double* partials, SolveState* st) {
  pdl_enter();
  if (blockIdx.x == 0 && threadIdx.x == 0) st->dir_pending = 0;  // no block of this kernel reads it
  if (st->done) return;
  __shared__ double smem[kBlock / 32];
  const size_t m = (size_t)nE;
  T acc = (T)0;  // this thread's few rows in T; across threads and blocks in FP64
  if (st->restart) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nE; e += gridDim.x * blockDim.x) {
      const T pe = zsrc ? zsrc[e] : dinv[e] * r[e];
      T s = rdiag[e] * pe;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int c = nbr[k * m + e];
        s += lval[k * m + e] * (pe - (zsrc ? zsrc[c] : dinv[c] * r[c]));
      }
      p[e] = pe;
      q[e] = s;
      acc += pe * s;
    }
  } else {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nE; e += gridDim.x * blockDim.x) {
      const T s = spmv_row(nbr, lval, rdiag, (const T*)p, m, e);
      q[e] = s;
      acc += p[e] * s;
    }
  }
  const double accd = block_sum((double)acc, smem);
  if (threadIdx.x == 0) partials[blockIdx.x] = accd;
  if (!arrive_last(&st->counter[1])) return;
  const double pq = sum_partials(partials, smem);
  if (threadIdx.x == 0) {
    st->counter[1] = 0;
    if (!(pq > 0.0) || !isfinite(pq)) {
      st->done = 3;
      st->status = isfinite(pq) ? PHFEM_EBREAKDOWN : PHFEM_ENAN;
    } else {
      st->alpha = (st->use_rp ? st->rp : st->rz) / pq;
      st->use_rp = 0;
      st->restart = 0;
    }
  }
}

// x += alpha p, r -= alpha q, r.D^-1 r -> beta
template <typename T>
__global__ void __launch_bounds__(kBlock) k_cg_update(int nE, double* __restrict__ x, const T* __restrict__ p,
                                                      T* __restrict__ r, const T* __restrict__ q,
                                                      const T* __restrict__ dinv, double* partials,
                                                      SolveState* st) {
  pdl_enter();
  if (st->done) return;
  __shared__ double smem[kBlock / 32];
  const double alpha64 = st->alpha;
  const T alpha = (T)alpha64;
  T acc = (T)0;  // this thread's few rows in T; across threads and blocks in FP64
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nE; e += gridDim.x * blockDim.x) {
    x[e] += alpha64 * (double)p[e];
    const T re = r[e] - alpha * q[e];
    r[e] = re;
    acc += re * (dinv[e] * re);
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
    st->dir_pending = 1;
    if (!isfinite(rz)) {
      st->done = 3;
      st->status = PHFEM_ENAN;
    }
  }
}

// Multigrid iteration: x += alpha p, r -= alpha q (the preconditioner then
// forms z), r.z -> beta, p = z + beta p.
template <typename T>
__global__ void __launch_bounds__(kBlock) k_cg_update_x(int nE, double* __restrict__ x, const T* __restrict__ p,
                                                        T* __restrict__ r, const T* __restrict__ q,
                                                        const SolveState* st) {
  pdl_enter();
  if (st->done) return;
  const double alpha64 = st->alpha;
  const T alpha = (T)alpha64;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nE; e += gridDim.x * blockDim.x) {
    x[e] += alpha64 * (double)p[e];
    r[e] = r[e] - alpha * q[e];
  }
}

template <typename T>
__global__ void __launch_bounds__(kBlock) k_cg_rz(int nE, const T* __restrict__ r, const T* __restrict__ z,
                                                  double* partials, SolveState* st) {
  pdl_enter();
  if (st->done) return;
  __shared__ double smem[kBlock / 32];
  T acc = (T)0;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nE; e += gridDim.x * blockDim.x) acc += r[e] * z[e];
  const double accd = block_sum((double)acc, smem);
  if (threadIdx.x == 0) partials[kMaxGrid + blockIdx.x] = accd;
  if (!arrive_last(&st->counter[2])) return;
  const double rz = sum_partials(partials + kMaxGrid, smem);
  if (threadIdx.x == 0) {
    st->counter[2] = 0;
    st->beta = st->rz > 0.0 ? rz / st->rz : 0.0;
    st->rz = rz;
    st->it += 1;
    st->dir_pending = 1;
    if (!isfinite(rz)) {
      st->done = 3;
      st->status = PHFEM_ENAN;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kBlock) k_cg_dir_z(int nE, const T* __restrict__ z, T* __restrict__ p,
                                                     SolveState* st) {
  pdl_enter();
  if (!st->dir_pending) return;
  const T beta = (T)st->beta;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nE; e += gridDim.x * blockDim.x)
    p[e] = z[e] + beta * p[e];
  if (blockIdx.x == 0 && threadIdx.x == 0 && st->done == 0 && st->rz <= st->tol2) st->done = 1;
}

// p = D^-1 r + beta p; then the test of the recursive residual, so that the
// direction is always complete when the iteration pauses for an update.  The
// kernel runs only after an update kernel that did run (dir_pending), and the
// done flag it sets is read only by later kernels.
template <typename T>
__global__ void __launch_bounds__(kBlock) k_cg_dir(int nE, const T* __restrict__ r, const T* __restrict__ dinv,
                                                   T* __restrict__ p, SolveState* st) {
  pdl_enter();
  if (!st->dir_pending) return;
  const T beta = (T)st->beta;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nE; e += gridDim.x * blockDim.x)
    p[e] = dinv[e] * r[e] + beta * p[e];
  if (blockIdx.x == 0 && threadIdx.x == 0 && st->done == 0 && st->rz <= st->tol2) st->done = 1;
}

// Graph loop control: continue while the iteration runs and stays within the
// iteration and body limits (every loop is bounded).
__global__ void k_loop_control(SolveState* st, cudaGraphConditionalHandle handle, int max_iter, int max_bodies) {
  st->bodies += 1;
  const bool more = st->done == 0 && st->it < max_iter && st->bodies < max_bodies;
  cudaGraphSetConditional(handle, more ? 1u : 0u);
}

__global__ void k_init_x(int nE, const uint8_t* __restrict__ eclass, uint8_t ident, const double* __restrict__ b,
                         const double* __restrict__ w0, double* __restrict__ x) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nE; e += gridDim.x * blockDim.x)
    x[e] = (eclass[e] == ident) ? b[e] : (w0 ? w0[e] : 0.0);
}

// Flux form: w_T = (K^CR_T)^-1 (F^CR_T + diag(sigma |E|) Lambda_T), U = R^-1 w_T.
__global__ void k_recover_flux(int nT, const int32_t* __restrict__ t2e, const int8_t* __restrict__ sigma,
                               const uint8_t* __restrict__ eclass, const double* __restrict__ elen,
                               const double* __restrict__ rec, double delta, const double* __restrict__ f,
                               const double* __restrict__ bc, const double* __restrict__ lam, double* __restrict__ U) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nT; t += gridDim.x * blockDim.x) {
    double r[4], K[6];
    load_record<true>(rec, t, r);
    record_block(r, delta, K);
    const double a = K[0], b = K[1], c = K[2], d = K[3], e = K[4], g = K[5], mT = r[3];
    const double C00 = b * c - e * e, C11 = a * c - g * g, C22 = a * b - d * d;
    const double C01 = e * g - d * c, C12 = d * g - a * e, C20 = d * e - b * g;
    const double inv = 1.0 / (a * C00 + d * C01 + g * C20);
    double rhs[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int ek = t2e[3 * t + k];
      const double L = elen[ek];
      rhs[k] = mT * f[ek] + (eclass[ek] == PHFEM_EDGE_NEUMANN ? L * bc[ek] : 0.0) + sigma[3 * t + k] * L * lam[ek];
    }
    const double w0 = (C00 * rhs[0] + C01 * rhs[1] + C20 * rhs[2]) * inv;
    const double w1 = (C01 * rhs[0] + C11 * rhs[1] + C12 * rhs[2]) * inv;
    const double w2 = (C20 * rhs[0] + C12 * rhs[1] + C22 * rhs[2]) * inv;
    const double sw = w0 + w1 + w2;
    U[3 * t] = sw - 2.0 * w0;
    U[3 * t + 1] = sw - 2.0 * w1;
    U[3 * t + 2] = sw - 2.0 * w2;
  }
}

__global__ void k_copy_lambda(int nE, const int32_t* __restrict__ lam_id, const double* __restrict__ x,
                              double* __restrict__ Lambda) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nE; e += gridDim.x * blockDim.x) {
    const int li = lam_id[e];
    if (li >= 0) Lambda[li] = x[e];
  }
}

// U = R^-1 w per triangle (u at the vertices); with Lambda: the element row
// residual mT (wa - wb)/dt + K^CR_T (theta wa + (1 - theta) wb) - mT f, divided
// by |E_k|, on the T+ side of every multiplier edge.  K^CR_T w is applied in
// difference form from the record; conv: [3][nT] convection columns or NULL.
__global__ void k_recover(int nT, const int32_t* __restrict__ t2e, const int8_t* __restrict__ sigma,
                          const int32_t* __restrict__ lam_id, const double* __restrict__ rec, double delta,
                          const double* __restrict__ conv, const double* __restrict__ elen,
                          const double* __restrict__ wa, const double* __restrict__ wb, const double* __restrict__ f,
                          double inv_dt, double theta, double* __restrict__ U, double* __restrict__ Lambda) {
  const size_t n = (size_t)nT;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nT; t += gridDim.x * blockDim.x) {
    const int e0 = t2e[3 * t], e1 = t2e[3 * t + 1], e2 = t2e[3 * t + 2];
    const double a0 = wa[e0], a1 = wa[e1], a2 = wa[e2];
    if (U) {
      const double s = a0 + a1 + a2;
      U[3 * t] = s - 2.0 * a0;
      U[3 * t + 1] = s - 2.0 * a1;
      U[3 * t + 2] = s - 2.0 * a2;
    }
    if (!Lambda) continue;
    double b0 = 0.0, b1 = 0.0, b2 = 0.0;
    if (wb) {
      b0 = wb[e0];
      b1 = wb[e1];
      b2 = wb[e2];
    }
    const double m0 = theta * a0 + (1.0 - theta) * b0;
    const double m1 = theta * a1 + (1.0 - theta) * b1;
    const double m2 = theta * a2 + (1.0 - theta) * b2;
    double r4[4], res[3];
    load_record<true>(rec, t, r4);
    record_apply(r4, delta, m0, m1, m2, res);
    const double mT = r4[3];
    if (conv) {  // convection adds the same sum_j c_j m_j to every row
      const double cv = conv[t] * m0 + conv[n + t] * m1 + conv[2 * n + t] * m2;
      res[0] += cv;
      res[1] += cv;
      res[2] += cv;
    }
    const double dw[3] = {a0 - b0, a1 - b1, a2 - b2};
    const int ee[3] = {e0, e1, e2};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int li = lam_id[ee[k]];
      if (li < 0 || sigma[3 * t + k] < 0) continue;
      double r = res[k] - mT * (f ? f[ee[k]] : 0.0);
      if (inv_dt > 0.0) r += mT * inv_dt * dw[k];
      Lambda[li] = r / elen[ee[k]];
    }
  }
}

// ---- BiCGStab (systems with convection) ------------------------------------
// Jacobi-preconditioned (on the right) BiCGStab in the inner precision with the
// solution accumulated in FP64 and the same reliable updates as the CG path:
// when the recursive residual has fallen by inner_rtol (or on a breakdown) the
// true FP64 residual replaces it and the iteration restarts with r^ = r.

// After a true residual (k_residual with precond = 1): r^ = p = r, rho = r.r,
// and the convergence decision.
template <typename T>
__global__ void k_bi_start(int nE, const T* __restrict__ r, T* __restrict__ rh, T* __restrict__ p, double* partials,
                           SolveState* st, double rtol2, double inner_rtol2, int mode) {
  if (mode == 3) {
    if (st->done != 1) return;
    mode = 2;
  }
  __shared__ double smem[kBlock / 32];
  T acc = (T)0;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nE; e += gridDim.x * blockDim.x) {
    const T re = r[e];
    rh[e] = re;
    p[e] = re;
    acc += re * re;
  }
  const double a = block_sum((double)acc, smem);
  if (threadIdx.x == 0) partials[blockIdx.x] = a;
  if (!arrive_last(&st->counter[3])) return;
  const double rho = sum_partials(partials, smem);
  if (threadIdx.x == 0) {
    st->counter[3] = 0;
    const double rr = st->rr_pending, ff = st->ff_pending;
    st->rr64 = rr;
    st->floor2 = ff;
    st->rho = rho;
    st->rz = rho;
    st->tol2 = inner_rtol2 * rho;
    st->status = 0;
    if (mode == 1) {
      st->it = 0;
      st->updates = 1;
      st->bodies = 0;
    } else {
      st->updates += 1;
    }
    st->conv = 0;
    if (!isfinite(rr) || !isfinite(rho)) {
      st->done = 3;
      st->status = PHFEM_ENAN;
    } else if (rr <= rtol2 * st->bb || rr == 0.0) {
      st->done = 2;
      st->conv = 1;
    } else if (rr <= 4.0 * ff) {
      st->done = 2;
      st->conv = 2;
    } else {
      st->done = 0;
    }
  }
}

// ph = D^-1 p, v = A ph (neighbours' ph from p and D^-1), alpha = rho / (r^, v).
template <typename T>
__global__ void __launch_bounds__(kBlock) k_bi_v(int nE, const int32_t* __restrict__ nbr,
                                                 const T* __restrict__ lval, const T* __restrict__ rdiag,
                                                 const T* __restrict__ dinv, const T* __restrict__ p,
                                                 T* __restrict__ ph, T* __restrict__ v, const T* __restrict__ rh,
                                                 double* partials, SolveState* st) {
  if (blockIdx.x == 0 && threadIdx.x == 0) st->dir_pending = 0;
  if (st->done) return;
  __shared__ double smem[kBlock / 32];
  const size_t m = (size_t)nE;
  T acc = (T)0;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nE; e += gridDim.x * blockDim.x) {
    const T pe = dinv[e] * p[e];
    T s = rdiag[e] * pe;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int c = nbr[k * m + e];
      s += lval[k * m + e] * (pe - dinv[c] * p[c]);
    }
    ph[e] = pe;
    v[e] = s;
    acc += rh[e] * s;
  }
  const double a = block_sum((double)acc, smem);
  if (threadIdx.x == 0) partials[blockIdx.x] = a;
  if (!arrive_last(&st->counter[1])) return;
  const double rv = sum_partials(partials, smem);
  if (threadIdx.x == 0) {
    st->counter[1] = 0;
    if (!isfinite(rv)) {
      st->done = 3;
      st->status = PHFEM_ENAN;
    } else if (rv == 0.0 || st->rho == 0.0) {
      st->done = 1;  // breakdown: restart from the true residual
    } else {
      st->alpha = st->rho / rv;
    }
  }
}

// s = r - alpha v, sh = D^-1 s.
template <typename T>
__global__ void __launch_bounds__(kBlock) k_bi_s(int nE, const T* __restrict__ r, const T* __restrict__ v,
                                                 const T* __restrict__ dinv, T* __restrict__ s, T* __restrict__ sh,
                                                 const SolveState* st) {
  if (st->done) return;
  const T alpha = (T)st->alpha;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nE; e += gridDim.x * blockDim.x) {
    const T se = r[e] - alpha * v[e];
    s[e] = se;
    sh[e] = dinv[e] * se;
  }
}

// t = A sh, omega = (t, s) / (t, t).
template <typename T>
__global__ void __launch_bounds__(kBlock) k_bi_t(int nE, const int32_t* __restrict__ nbr,
                                                 const T* __restrict__ lval, const T* __restrict__ rdiag,
                                                 const T* __restrict__ sh, const T* __restrict__ s, T* __restrict__ t,
                                                 double* partials, SolveState* st) {
  if (st->done) return;
  __shared__ double smem[kBlock / 32];
  const size_t m = (size_t)nE;
  T ats = (T)0, att = (T)0;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nE; e += gridDim.x * blockDim.x) {
    const T te = spmv_row(nbr, lval, rdiag, sh, m, e);
    t[e] = te;
    ats += te * s[e];
    att += te * te;
  }
  const double a = block_sum((double)ats, smem);
  const double b = block_sum((double)att, smem);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = a;
    partials[kMaxGrid + blockIdx.x] = b;
  }
  if (!arrive_last(&st->counter[2])) return;
  const double ts = sum_partials(partials, smem);
  const double tt = sum_partials(partials + kMaxGrid, smem);
  if (threadIdx.x == 0) {
    st->counter[2] = 0;
    st->omega = tt > 0.0 ? ts / tt : 0.0;
  }
}

// x += alpha ph + omega sh (FP64), r = s - omega t, rho' = (r^, r), ||r||^2.
template <typename T>
__global__ void __launch_bounds__(kBlock) k_bi_x(int nE, double* __restrict__ x, const T* __restrict__ ph,
                                                 const T* __restrict__ sh, const T* __restrict__ s,
                                                 const T* __restrict__ t, T* __restrict__ r, const T* __restrict__ rh,
                                                 double* partials, SolveState* st) {
  if (st->done) return;
  __shared__ double smem[kBlock / 32];
  const double alpha64 = st->alpha, omega64 = st->omega;
  const T omega = (T)omega64;
  T arr = (T)0, arh = (T)0;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nE; e += gridDim.x * blockDim.x) {
    x[e] += alpha64 * (double)ph[e] + omega64 * (double)sh[e];
    const T re = s[e] - omega * t[e];
    r[e] = re;
    arr += re * re;
    arh += rh[e] * re;
  }
  const double a = block_sum((double)arr, smem);
  const double b = block_sum((double)arh, smem);
  if (threadIdx.x == 0) {
    partials[2 * kMaxGrid + blockIdx.x] = a;
    partials[3 * kMaxGrid + blockIdx.x] = b;
  }
  if (!arrive_last(&st->counter[0])) return;
  const double rr = sum_partials(partials + 2 * kMaxGrid, smem);
  const double rho = sum_partials(partials + 3 * kMaxGrid, smem);
  if (threadIdx.x == 0) {
    st->counter[0] = 0;
    st->beta = (st->rho != 0.0 && omega64 != 0.0) ? (rho / st->rho) * (st->alpha / omega64) : 0.0;
    st->rho = rho;
    st->rz = rr;
    st->it += 1;
    st->dir_pending = 1;
    if (!isfinite(rr)) {
      st->done = 3;
      st->status = PHFEM_ENAN;
    } else if (omega64 == 0.0 || rho == 0.0) {
      st->done = 1;  // stagnation or breakdown: restart from the true residual
    }
  }
}

// p = r + beta (p - omega v); then the test of the recursive residual.
template <typename T>
__global__ void __launch_bounds__(kBlock) k_bi_p(int nE, const T* __restrict__ r, const T* __restrict__ v,
                                                 T* __restrict__ p, SolveState* st) {
  if (!st->dir_pending) return;
  const T beta = (T)st->beta, omega = (T)st->omega;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nE; e += gridDim.x * blockDim.x)
    p[e] = r[e] + beta * (p[e] - omega * v[e]);
  if (blockIdx.x == 0 && threadIdx.x == 0 && st->done == 0 && st->rz <= st->tol2) st->done = 1;
}

int read_state(phfem_sys sys) {
  cudaStream_t s = sys->mesh->ctx->stream;
  PH_CUDA(cudaMemcpyAsync(sys->st_host, sys->st, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
  PH_CUDA(cudaStreamSynchronize(s));
  return PHFEM_OK;
}

// The L2 window over the inner iteration's r and p (each read and written by
// the CG kernels every iteration), with the L2 set-aside sized to it.  Used only
// when both fit the largest set-aside: measured on the level-5 system, a window
// that covers more than the set-aside (r, p and q with a 0.75 hit ratio), or a
// set-aside larger than its window (r alone), is slower than no window at all.
L2Window rp_window(phfem_sys sys) {
  phfem_ctx ctx = sys->mesh->ctx;
  L2Window w;
  size_t want = 2 * sys->l2_vec;
  void* base = sys->ri;
  if (want > ctx->l2_persist_max || want > ctx->l2_window_max) {  // p alone (the gathered vector)
    want = sys->l2_vec;
    base = sys->pi;
  }
  if (!ctx->l2_window || want == 0 || want > ctx->l2_persist_max || want > ctx->l2_window_max) {
    // no window: a set-aside left from an earlier solve would only shrink L2
    if (ctx->l2_window) set_l2_limit(ctx, 0);
    return w;
  }
  if (!set_l2_limit(ctx, want)) return w;
  w.base = base;
  w.bytes = want;
  w.hit_ratio = 1.0f;
  static const bool verbose = getenv("PHFEM_VERBOSE") != nullptr;
  if (verbose)
    fprintf(stderr, "phfem: L2 window %.1f MB, set-aside max %.1f MB\n", w.bytes / 1e6, ctx->l2_persist_max / 1e6);
  return w;
}

template <typename T>
struct Launch {
  phfem_sys sys;
  cudaStream_t s;
  int g, nE;
  double rtol2, irtol2;
  L2Window win;
  int residual(int mode) const {
    phfem_ctx ctx = sys->mesh->ctx;
    const int pre = (sys->mg && mode != 0) ? 1 : 0;
    prof_start(ctx, kProfResidual);
    if (mode >= 2) {
      k_dd_fold<<<g, kBlock, 0, s>>>(nE, sys->x, sys->xh, sys->xl, sys->st, mode == 3);
      PH_TRY(check_launch(ctx, "k_dd_fold"));
    }
    k_residual<T><<<g, kBlock, 0, s>>>(nE, sys->mesh->nbr, sys->val, sys->b, sys->xh, sys->xl, sys->mesh->eclass,
                                       sys->ident_class, (const T*)sys->dinv, (T*)sys->ri, (T*)sys->pi,
                                       sys->partials, sys->st, rtol2, irtol2, mode, pre);
    prof_stop(ctx, kProfResidual);
    PH_TRY(check_launch(ctx, "k_residual"));
    if (!pre) return PHFEM_OK;
    // z = M^-1 r, then r.z (and p = z or r.p) and the decision
    prof_start(ctx, kProfMg);
    PH_TRY(mg_apply(sys->mg, s, sys->ri, mode == 3 ? sys->st : nullptr, 1));
    prof_stop(ctx, kProfMg);
    PH_CUDA(launch_pdl(k_mg_finish<T>, g, s, nE, (const T*)sys->ri, (const T*)mg_fine_z(sys->mg), (T*)sys->pi,
                       sys->partials, sys->st, rtol2, irtol2, mode));
    return check_launch(ctx, "k_mg_finish");
  }
  int iteration() const {
    phfem_ctx ctx = sys->mesh->ctx;
    const T* lval = (const T*)sys->lval;
    const T* rdiag = (const T*)sys->rdiag;
    const T* dinv = (const T*)sys->dinv;
    T* ri = (T*)sys->ri;
    T* pi = (T*)sys->pi;
    T* qi = (T*)sys->qi;
    const T* zmg = sys->mg ? (const T*)mg_fine_z(sys->mg) : nullptr;
    prof_start(ctx, kProfSpmv);
    PH_CUDA(launch_pdl_w(win, k_cg_spmv<T>, g, s, nE, sys->mesh->nbr, lval, rdiag, pi, qi, ri, dinv, zmg,
                         sys->partials, sys->st));
    prof_stop(ctx, kProfSpmv);
    if (sys->mg) {
      prof_start(ctx, kProfUpdate);
      PH_CUDA(launch_pdl_w(win, k_cg_update_x<T>, g, s, nE, sys->x, (const T*)pi, ri, (const T*)qi,
                           (const SolveState*)sys->st));
      prof_stop(ctx, kProfUpdate);
      PH_TRY(check_launch(ctx, "k_cg_update_x"));
      prof_start(ctx, kProfMg);
      PH_TRY(mg_apply(sys->mg, s, ri, sys->st, 0));
      prof_stop(ctx, kProfMg);
      prof_start(ctx, kProfDir);
      PH_CUDA(launch_pdl_w(win, k_cg_rz<T>, g, s, nE, (const T*)ri, zmg, sys->partials, sys->st));
      PH_CUDA(launch_pdl_w(win, k_cg_dir_z<T>, g, s, nE, zmg, pi, sys->st));
      prof_stop(ctx, kProfDir);
      ctx->launches += 2;  // spmv and rz (update_x and dir_z counted by check_launch)
      return check_launch(ctx, "k_cg");
    }
    prof_start(ctx, kProfUpdate);
    PH_CUDA(launch_pdl_w(win, k_cg_update<T>, g, s, nE, sys->x, (const T*)pi, ri, (const T*)qi, dinv,
                         sys->partials, sys->st));
    prof_stop(ctx, kProfUpdate);
    prof_start(ctx, kProfDir);
    PH_CUDA(launch_pdl_w(win, k_cg_dir<T>, g, s, nE, (const T*)ri, dinv, pi, sys->st));
    prof_stop(ctx, kProfDir);
    ctx->launches += 2;
    return check_launch(ctx, "k_cg");
  }
};

template <typename T>
int solve_typed(phfem_sys sys, const phfem_solve_opts& o, phfem_stats* stats) {
  phfem_mesh m = sys->mesh;
  phfem_ctx ctx = m->ctx;
  const int nE = m->info.nE;
  const Launch<T> L{sys, ctx->stream, grid_for(ctx, nE), nE, o.rtol * o.rtol, o.inner_rtol * o.inner_rtol,
                    rp_window(sys)};
  static const bool verbose = getenv("PHFEM_VERBOSE") != nullptr;
  // ||b|| of the free-edge system (with the Dirichlet lifting), then the start
  k_dd_begin<<<L.g, kBlock, 0, L.s>>>(nE, sys->x, sys->xh, sys->xl);
  PH_TRY(check_launch(ctx, "k_dd_begin"));
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
        fprintf(stderr, "phfem: update %d  iterations %d  relative residual %.3e  fp64 floor %.3e  restart %d\n",
                h.updates, h.it, rel, h.bb > 0 ? std::sqrt(h.floor2 / h.bb) : 0.0, h.restart);
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
  k_dd_end<<<L.g, kBlock, 0, L.s>>>(nE, sys->x, sys->xh, sys->xl);
  PH_TRY(check_launch(ctx, "k_dd_end"));
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

template <typename T>
int bicgstab_typed(phfem_sys sys, const phfem_solve_opts& o, phfem_stats* stats) {
  phfem_mesh m = sys->mesh;
  phfem_ctx ctx = m->ctx;
  cudaStream_t s = ctx->stream;
  const int nE = m->info.nE;
  const size_t mm = (size_t)nE;
  if (!sys->bw) PH_TRY(dalloc(ctx, &sys->bw, 7 * mm * sizeof(T) + 16));
  T* W = (T*)sys->bw;
  T *rh = W, *p = W + mm, *v = W + 2 * mm, *sv = W + 3 * mm, *tv = W + 4 * mm, *ph = W + 5 * mm, *sh = W + 6 * mm;
  T* r = (T*)sys->ri;
  const T* lval = (const T*)sys->lval;
  const T* rdiag = (const T*)sys->rdiag;
  const T* dinv = (const T*)sys->dinv;
  const int g = grid_for(ctx, nE);
  const double rtol2 = o.rtol * o.rtol, irtol2 = o.inner_rtol * o.inner_rtol;
  auto residual = [&](int mode) -> int {
    prof_start(ctx, kProfResidual);
    if (mode >= 2) {
      k_dd_fold<<<g, kBlock, 0, s>>>(nE, sys->x, sys->xh, sys->xl, sys->st, mode == 3);
      PH_TRY(check_launch(ctx, "k_dd_fold"));
    }
    k_residual<T><<<g, kBlock, 0, s>>>(nE, m->nbr, sys->val, sys->b, sys->xh, sys->xl, m->eclass, sys->ident_class, dinv, r,
                                       (T*)sys->pi, sys->partials, sys->st, rtol2, irtol2, mode, mode == 0 ? 0 : 1);
    prof_stop(ctx, kProfResidual);
    PH_TRY(check_launch(ctx, "k_residual"));
    if (mode == 0) return PHFEM_OK;
    k_bi_start<T><<<g, kBlock, 0, s>>>(nE, r, rh, p, sys->partials, sys->st, rtol2, irtol2, mode);
    return check_launch(ctx, "k_bi_start");
  };
  auto iteration = [&]() -> int {
    prof_start(ctx, kProfSpmv);
    k_bi_v<T><<<g, kBlock, 0, s>>>(nE, m->nbr, lval, rdiag, dinv, p, ph, v, rh, sys->partials, sys->st);
    k_bi_s<T><<<g, kBlock, 0, s>>>(nE, r, v, dinv, sv, sh, sys->st);
    k_bi_t<T><<<g, kBlock, 0, s>>>(nE, m->nbr, lval, rdiag, sh, sv, tv, sys->partials, sys->st);
    prof_stop(ctx, kProfSpmv);
    prof_start(ctx, kProfUpdate);
    k_bi_x<T><<<g, kBlock, 0, s>>>(nE, sys->x, ph, sh, sv, tv, r, rh, sys->partials, sys->st);
    k_bi_p<T><<<g, kBlock, 0, s>>>(nE, r, v, p, sys->st);
    prof_stop(ctx, kProfUpdate);
    ctx->launches += 4;
    return check_launch(ctx, "k_bi");
  };
  k_dd_begin<<<g, kBlock, 0, s>>>(nE, sys->x, sys->xh, sys->xl);
  PH_TRY(check_launch(ctx, "k_dd_begin"));
  PH_TRY(residual(0));
  PH_TRY(residual(1));
  PH_TRY(read_state(sys));
  int status = PHFEM_OK, stagnant = 0, last_updates = 0;
  double best = 1e300;
  for (;;) {
    const SolveState& h = *sys->st_host;
    if (h.updates != last_updates) {
      last_updates = h.updates;
      const double rel = h.bb > 0 ? std::sqrt(h.rr64 / h.bb) : 0.0;
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
    if (h.done == 1) {
      PH_TRY(residual(2));
      PH_TRY(read_state(sys));
      continue;
    }
    int chunk = o.check_every;
    if (h.it + chunk > o.max_iter) chunk = o.max_iter - h.it;
    for (int k = 0; k < chunk; ++k) PH_TRY(iteration());
    PH_TRY(read_state(sys));
  }
  k_dd_end<<<g, kBlock, 0, s>>>(nE, sys->x, sys->xh, sys->xl);
  PH_TRY(check_launch(ctx, "k_dd_end"));
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
    snprintf(buf, sizeof(buf), "BiCGStab: %s after %d iterations, %d residual updates, relative residual %.3e",
             phfem_status_str(status), h.it, h.updates, rel);
    return fail(status, buf);
  }
  return PHFEM_OK;
}

// The start kernels, then a WHILE node whose body runs `per_body` iterations,
// the conditional reliable update and the loop control.
template <typename T>
int capture_typed(phfem_sys sys, const phfem_solve_opts& o, cudaStream_t cs, int per_body) {
  phfem_ctx ctx = sys->mesh->ctx;
  const int nE = sys->mesh->info.nE;
  const Launch<T> L{sys, cs, grid_for(ctx, nE), nE, o.rtol * o.rtol, o.inner_rtol * o.inner_rtol, rp_window(sys)};
  k_dd_begin<<<L.g, kBlock, 0, cs>>>(nE, sys->x, sys->xh, sys->xl);
  PH_TRY(check_launch(ctx, "k_dd_begin"));
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
  // the body is captured on a second private stream
  cudaStream_t bs;
  PH_CUDA(cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking));
  int st = PHFEM_OK;
  cudaError_t e = cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) st = cuda_fail(e, "cudaStreamBeginCaptureToGraph", __FILE__, __LINE__);
  if (st == PHFEM_OK) {
    const Launch<T> B{sys, bs, L.g, nE, L.rtol2, L.irtol2, L.win};
    for (int k = 0; k < per_body && st == PHFEM_OK; ++k) st = B.iteration();
    if (st == PHFEM_OK) st = B.residual(3);
    if (st == PHFEM_OK) {
      const int max_bodies = o.max_iter / (per_body > 0 ? per_body : 1) + o.max_refine + 16;
      k_loop_control<<<1, 1, 0, bs>>>(sys->st, handle, o.max_iter, max_bodies);
      st = check_launch(ctx, "k_loop_control");
    }
    cudaGraph_t out;
    e = cudaStreamEndCapture(bs, &out);
    if (e != cudaSuccess && st == PHFEM_OK) st = cuda_fail(e, "cudaStreamEndCapture(body)", __FILE__, __LINE__);
  }
  cudaStreamDestroy(bs);
  if (st == PHFEM_OK) {
    k_dd_end<<<L.g, kBlock, 0, cs>>>(nE, sys->x, sys->xh, sys->xl);
    st = check_launch(ctx, "k_dd_end");
  }
  return st;
}

}  // namespace

void fill_opts(phfem_sys sys, phfem_solve_opts& o) {
  if (o.rtol <= 0) o.rtol = 1e-10;
  if (o.inner_rtol <= 0)
    o.inner_rtol = sys->conv ? (sys->fp32 ? 1e-2 : 1e-6)
                             : sys->mg ? (sys->fp32 ? 1e-3 : 1e-4) : (sys->fp32 ? 0.1 : 0.01);
  if (o.max_iter <= 0) o.max_iter = 200000;
  if (o.max_refine <= 0) o.max_refine = 1000;
  if (o.check_every <= 0) o.check_every = sys->mg ? 2 : (sys->conv ? 16 : 64);
}

int solve_bicgstab(phfem_sys sys, const phfem_solve_opts& o, phfem_stats* stats) {
  return sys->fp32 ? bicgstab_typed<float>(sys, o, stats) : bicgstab_typed<double>(sys, o, stats);
}

int capture_solve(phfem_sys sys, const phfem_solve_opts* opts, cudaStream_t capture, int iters_per_body) {
  if (sys->conv) return fail(PHFEM_EINVAL, "graph-captured steps: not with convection (use phfem_cn_step)");
  phfem_solve_opts o{};
  if (opts) o = *opts;
  fill_opts(sys, o);
  if (fcg_eligible(sys, o)) return fcg_capture(sys, o, capture, iters_per_body);
  return sys->fp32 ? capture_typed<float>(sys, o, capture, iters_per_body)
                   : capture_typed<double>(sys, o, capture, iters_per_body);
}

namespace {
}  // namespace

int sys_init_x(phfem_sys sys, const double* w0) {
  phfem_mesh m = sys->mesh;
  phfem_ctx ctx = m->ctx;
  const int nE = m->info.nE;
  k_init_x<<<grid_for(ctx, nE), kBlock, 0, ctx->stream>>>(nE, m->eclass, sys->ident_class, sys->b, w0, sys->x);
  return check_launch(ctx, "k_init_x");
}

int solve_system(phfem_sys sys, const phfem_solve_opts* opts, phfem_stats* stats, bool /*warm*/) {
  phfem_solve_opts o{};
  if (opts) o = *opts;
  fill_opts(sys, o);
  if (sys->conv) return solve_bicgstab(sys, o, stats);
  if (fcg_eligible(sys, o)) return fcg_solve(sys, o, stats);
  return sys->fp32 ? solve_typed<float>(sys, o, stats) : solve_typed<double>(sys, o, stats);
}

int recover(phfem_sys sys, const double* x_new, const double* x_old, const double* f_eff, double inv_dt,
            double theta, double* U, double* Lambda) {
  phfem_mesh m = sys->mesh;
  phfem_ctx ctx = m->ctx;
  const int nT = m->info.nT;
  if (!U && !Lambda) return PHFEM_OK;
  prof_start(ctx, kProfRecover);
  const double* conv = sys->conv ? sys->Kt + (size_t)kRec * nT : nullptr;
  k_recover<<<grid_for(ctx, nT), kBlock, 0, ctx->stream>>>(nT, m->t2e, m->sigma, m->lam_id, sys->Kt, sys->c.delta,
                                                           conv, m->elen, x_new, x_old, f_eff, inv_dt, theta, U,
                                                           Lambda);
  prof_stop(ctx, kProfRecover);
  return check_launch(ctx, "k_recover");
}

}  // namespace phfem

using namespace phfem;

extern "C" {

PHFEM_API int phfem_solve(phfem_sys sys, const phfem_solve_opts* opts, const double* w0, double* w, double* U,
                          double* Lambda, phfem_stats* stats) {
  if (!sys) return fail(PHFEM_EINVAL, "phfem_solve: NULL system");
  auto t0 = std::chrono::steady_clock::now();
  phfem_stats st{};
  PH_TRY(sys_init_x(sys, w0));
  int status = solve_system(sys, opts, &st, false);
  if (status == PHFEM_OK || status == PHFEM_ENOCONV) {
    phfem_mesh m = sys->mesh;
    cudaStream_t s = m->ctx->stream;
    if (w) PH_CUDA(cudaMemcpyAsync(w, sys->x, sizeof(double) * m->info.nE, cudaMemcpyDeviceToDevice, s));
    if (sys->form == PHFEM_FORM_FLUX) {
      phfem_ctx ctx = m->ctx;
      if (U) {
        k_recover_flux<<<grid_for(ctx, m->info.nT), kBlock, 0, s>>>(m->info.nT, m->t2e, m->sigma, m->eclass, m->elen,
                                                                    sys->Kt, sys->c.delta, sys->f, sys->bc, sys->x,
                                                                    U);
        PH_TRY(check_launch(ctx, "k_recover_flux"));
      }
      if (Lambda) {
        k_copy_lambda<<<grid_for(ctx, m->info.nE), kBlock, 0, s>>>(m->info.nE, m->lam_id, sys->x, Lambda);
        PH_TRY(check_launch(ctx, "k_copy_lambda"));
      }
    } else {
      PH_TRY(recover(sys, sys->x, nullptr, sys->f, 0.0, 1.0, U, Lambda));
    }
    PH_CUDA(cudaStreamSynchronize(s));
  }
  st.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (stats) *stats = st;
  return status;
}

}  // extern "C"
