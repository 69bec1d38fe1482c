// Crank-Nicolson stepping (Section 4, Eq. MatrixformParabolic) on the
// condensed edge system.
//
// Condensing M+ W^n = M- W^{n-1} + F element by element with u = R^-1 w gives,
// on every free edge,
//   (M^CR + dt/2 K^CR) w^n = (M^CR - dt/2 K^CR) w^{n-1} + dt (F^n + F^{n-1})/2,
// with M^CR = |T|/3 I per triangle (pure mass), K^CR the elliptic block
// (stiffness + delta reaction), F the edge load of Eqs. parabolicRight_b/_g and
// w^n = u_D(t_n) on Dirichlet edges.  The multiplier average follows from the
// element rows on the T+ side:
//   |E| Lambda^{n-1/2} = (M^CR (w^n - w^{n-1})/dt + K^CR (w^n + w^{n-1})/2 - F^{n-1/2})_k
// and Lambda^n = 2 Lambda^{n-1/2} - Lambda^{n-1}.
#include <chrono>
#include <vector>

#include "internal.cuh"

struct phfem_cn_s {
  phfem_sys sys;
  int Q;
  int nt;
  int step;
  double* fq;        // [Q][nE]
  double* bcq;       // [Q][nE]
  std::vector<double> phi;  // [Q][nt]
  double* xprev;     // [nE]
  double* f_eff;     // [nE]
  double* lam_half;  // [nL]
  double* lam_n;     // [nL]
};

namespace phfem {
namespace {

struct Phi {
  double now[PHFEM_MAX_TERMS];
  double avg[PHFEM_MAX_TERMS];
};

__global__ void k_cn_init(int nE, const uint8_t* __restrict__ eclass, const double* __restrict__ w0,
                          const double* __restrict__ bcq, int Q, Phi ph, double* __restrict__ x) {
  const size_t m = (size_t)nE;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nE; e += gridDim.x * blockDim.x) {
    if (eclass[e] == PHFEM_EDGE_DIRICHLET) {
      double v = 0.0;
      for (int q = 0; q < Q; ++q) v += ph.now[q] * bcq[q * m + e];
      x[e] = v;
    } else {
      x[e] = w0 ? w0[e] : 0.0;
    }
  }
}

// rhs = 2 M w^{n-1} - A+ w^{n-1} + dt (sum_q avg_q (m_e f_q + [Neumann] |E| g_q))
// on free rows (A+ = M + dt/2 K; w^{n-1} holds u_D(t_{n-1}) on Dirichlet rows),
// u_D(t_n) on Dirichlet rows; also the averaged source f^{n-1/2} per edge.
__global__ void k_cn_rhs(int nE, const int32_t* __restrict__ nbr, const double* __restrict__ val,
                         const double* __restrict__ x, const double* __restrict__ me,
                         const uint8_t* __restrict__ eclass, const double* __restrict__ elen,
                         const double* __restrict__ fq, const double* __restrict__ bcq, int Q, Phi ph, double dt,
                         double* __restrict__ b, double* __restrict__ f_eff) {
  const size_t m = (size_t)nE;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nE; e += gridDim.x * blockDim.x) {
    const uint8_t cls = eclass[e];
    double fav = 0.0;
    for (int q = 0; q < Q; ++q) fav += ph.avg[q] * fq[q * m + e];
    f_eff[e] = fav;
    if (cls == PHFEM_EDGE_DIRICHLET) {
      double v = 0.0;
      for (int q = 0; q < Q; ++q) v += ph.now[q] * bcq[q * m + e];
      b[e] = v;
      continue;
    }
    const double xe = x[e];
    double aw = val[e] * xe;  // (A+ w)_e in difference form
#pragma unroll
    for (int s = 0; s < 4; ++s) aw += val[(s + 1) * m + e] * (xe - x[nbr[s * m + e]]);
    double load = me[e] * fav;
    if (cls == PHFEM_EDGE_NEUMANN) {
      double g = 0.0;
      for (int q = 0; q < Q; ++q) g += ph.avg[q] * bcq[q * m + e];
      load += elen[e] * g;
    }
    b[e] = 2.0 * me[e] * x[e] - aw + dt * load;
  }
}

__global__ void k_set_dirichlet(int nE, const uint8_t* __restrict__ eclass, const double* __restrict__ b,
                                double* __restrict__ x) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nE; e += gridDim.x * blockDim.x)
    if (eclass[e] == PHFEM_EDGE_DIRICHLET) x[e] = b[e];
}

__global__ void k_lam_update(int nL, const double* __restrict__ half, double* __restrict__ lam) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nL; i += gridDim.x * blockDim.x)
    lam[i] = 2.0 * half[i] - lam[i];
}

void cn_free(phfem_cn cn) {
  phfem_ctx c = cn->sys->mesh->ctx;
  dfree(c, cn->fq);
  dfree(c, cn->bcq);
  dfree(c, cn->xprev);
  dfree(c, cn->f_eff);
  dfree(c, cn->lam_half);
  dfree(c, cn->lam_n);
  delete cn;
}

Phi phi_at(const phfem_cn_s* cn, int n) {
  Phi p{};
  for (int q = 0; q < cn->Q; ++q) {
    p.now[q] = cn->phi[(size_t)q * cn->nt + n];
    p.avg[q] = n > 0 ? 0.5 * (cn->phi[(size_t)q * cn->nt + n] + cn->phi[(size_t)q * cn->nt + n - 1]) : p.now[q];
  }
  return p;
}

}  // namespace
}  // namespace phfem

using namespace phfem;

extern "C" {

PHFEM_API int phfem_cn_create(phfem_sys sys, const phfem_source* src, const double* w0, const double* Lambda0,
                              phfem_cn* out) {
  if (!out) return fail(PHFEM_EINVAL, "phfem_cn_create: out is NULL");
  *out = nullptr;
  if (!sys || !src) return fail(PHFEM_EINVAL, "phfem_cn_create: NULL argument");
  if (!(sys->c.dt > 0)) return fail(PHFEM_EINVAL, "phfem_cn_create: the system was assembled with dt = 0");
  if (src->nterms < 1 || src->nterms > PHFEM_MAX_TERMS || src->nt < 1 || !src->phi || !src->f_mid || !src->bc_mid)
    return fail(PHFEM_EINVAL, "phfem_cn_create: bad source description");
  phfem_mesh m = sys->mesh;
  phfem_ctx ctx = m->ctx;
  cudaStream_t s = ctx->stream;
  const size_t nE = m->info.nE, nL = m->info.nL;
  phfem_cn cn = new phfem_cn_s();
  cn->sys = sys;
  cn->Q = src->nterms;
  cn->nt = src->nt;
  cn->step = 0;
  cn->phi.assign(src->phi, src->phi + (size_t)cn->Q * cn->nt);
  int st = PHFEM_OK;
  auto chk = [&](int r) {
    if (st == PHFEM_OK) st = r;
  };
  chk(dalloc_n(ctx, &cn->fq, cn->Q * nE));
  chk(dalloc_n(ctx, &cn->bcq, cn->Q * nE));
  chk(dalloc_n(ctx, &cn->xprev, nE));
  chk(dalloc_n(ctx, &cn->f_eff, nE));
  chk(dalloc_n(ctx, &cn->lam_half, nL));
  chk(dalloc_n(ctx, &cn->lam_n, nL));
  if (st == PHFEM_OK) {
    cudaMemcpyAsync(cn->fq, src->f_mid, sizeof(double) * cn->Q * nE, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(cn->bcq, src->bc_mid, sizeof(double) * cn->Q * nE, cudaMemcpyDeviceToDevice, s);
    if (Lambda0) cudaMemcpyAsync(cn->lam_n, Lambda0, sizeof(double) * nL, cudaMemcpyDeviceToDevice, s);
    else cudaMemsetAsync(cn->lam_n, 0, sizeof(double) * nL, s);
    cudaMemsetAsync(cn->lam_half, 0, sizeof(double) * nL, s);
    k_cn_init<<<grid_for(ctx, nE), kBlock, 0, s>>>((int)nE, m->eclass, w0, cn->bcq, cn->Q, phi_at(cn, 0), sys->x);
    st = check_launch(ctx, "k_cn_init");
  }
  if (st == PHFEM_OK && cudaStreamSynchronize(s) != cudaSuccess)
    st = cuda_fail(cudaGetLastError(), "phfem_cn_create", __FILE__, __LINE__);
  if (st != PHFEM_OK) {
    cudaStreamSynchronize(s);
    cn_free(cn);
    return st;
  }
  *out = cn;
  return PHFEM_OK;
}

PHFEM_API int phfem_cn_step(phfem_cn cn, int32_t nsteps, const phfem_solve_opts* opts, phfem_stats* stats) {
  if (!cn || nsteps < 0) return fail(PHFEM_EINVAL, "phfem_cn_step: bad argument");
  if (cn->step + nsteps >= cn->nt)
    return fail(PHFEM_EINVAL, "phfem_cn_step: the source has no time factors for the requested steps");
  auto t0 = std::chrono::steady_clock::now();
  phfem_sys sys = cn->sys;
  phfem_mesh m = sys->mesh;
  phfem_ctx ctx = m->ctx;
  cudaStream_t s = ctx->stream;
  const int nE = m->info.nE, nL = m->info.nL;
  const double dt = sys->c.dt;
  phfem_stats st{};
  int status = PHFEM_OK;
  for (int k = 0; k < nsteps; ++k) {
    const int n = cn->step + 1;
    const Phi ph = phi_at(cn, n);
    PH_CUDA(cudaMemcpyAsync(cn->xprev, sys->x, sizeof(double) * nE, cudaMemcpyDeviceToDevice, s));
    k_cn_rhs<<<grid_for(ctx, nE), kBlock, 0, s>>>(nE, m->nbr, sys->val, sys->x, sys->me, m->eclass, m->elen, cn->fq,
                                                  cn->bcq, cn->Q, ph, dt, sys->b, cn->f_eff);
    PH_TRY(check_launch(ctx, "k_cn_rhs"));
    k_set_dirichlet<<<grid_for(ctx, nE), kBlock, 0, s>>>(nE, m->eclass, sys->b, sys->x);
    PH_TRY(check_launch(ctx, "k_set_dirichlet"));
    status = solve_system(sys, opts, &st, true);
    if (status != PHFEM_OK) break;
    PH_TRY(recover(sys, sys->x, cn->xprev, cn->f_eff, 1.0 / dt, 0.5, nullptr, cn->lam_half));
    k_lam_update<<<grid_for(ctx, nL), kBlock, 0, s>>>(nL, cn->lam_half, cn->lam_n);
    PH_TRY(check_launch(ctx, "k_lam_update"));
    cn->step = n;
    st.steps += 1;
  }
  PH_CUDA(cudaStreamSynchronize(s));
  st.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (stats) *stats = st;
  return status;
}

PHFEM_API int phfem_cn_read(phfem_cn cn, double* w, double* U, double* Lambda_n, double* Lambda_half,
                            int32_t* step) {
  if (!cn) return fail(PHFEM_EINVAL, "phfem_cn_read: NULL handle");
  phfem_sys sys = cn->sys;
  phfem_mesh m = sys->mesh;
  cudaStream_t s = m->ctx->stream;
  if (w) PH_CUDA(cudaMemcpyAsync(w, sys->x, sizeof(double) * m->info.nE, cudaMemcpyDeviceToDevice, s));
  if (Lambda_n) PH_CUDA(cudaMemcpyAsync(Lambda_n, cn->lam_n, sizeof(double) * m->info.nL, cudaMemcpyDeviceToDevice, s));
  if (Lambda_half)
    PH_CUDA(cudaMemcpyAsync(Lambda_half, cn->lam_half, sizeof(double) * m->info.nL, cudaMemcpyDeviceToDevice, s));
  if (U) PH_TRY(recover(sys, sys->x, nullptr, nullptr, 0.0, 1.0, U, nullptr));
  if (step) *step = cn->step;
  PH_CUDA(cudaStreamSynchronize(s));
  return PHFEM_OK;
}

PHFEM_API int phfem_cn_destroy(phfem_cn cn) {
  if (!cn) return fail(PHFEM_EINVAL, "phfem_cn_destroy: NULL handle");
  cn_free(cn);
  return PHFEM_OK;
}

}  // extern "C"
