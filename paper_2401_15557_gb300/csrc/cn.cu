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
#include <algorithm>
#include <chrono>
#include <cstring>
#include <vector>

#include "internal.cuh"

struct phfem_cn_s {
  phfem_sys sys;
  int Q;             // separable terms; 0: per-step data (fq, bcq hold the previous step's arrays)
  int nt;
  int step;
  double* fq;        // [Q][nE]
  double* bcq;       // [Q][nE]
  std::vector<double> phi;  // [Q][nt]
  double* phi_dev;   // [Q][nt] (the graph reads the time factors on the device)
  int* step_dev;     // steps done, advanced on the device
  int* it_dev;       // [nt] iterations of every step
  int* conv_dev;     // [nt] convergence code of every step
  double* rel_dev;   // [nt] final relative residual of every step
  double* xprev;     // [nE]
  double* f_eff;     // [nE]
  double* lam_half;  // [nL]
  double* lam_n;     // [nL]
  // captured step
  cudaGraphExec_t exec = nullptr;
  phfem_solve_opts graph_opts{};
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

// Time factors of step n = *step + 1 from the device table.
__device__ __forceinline__ Phi phi_dev_at(const double* phi, int Q, int nt, int n) {
  Phi p;
  for (int q = 0; q < Q; ++q) {
    p.now[q] = phi[q * nt + n];
    p.avg[q] = 0.5 * (phi[q * nt + n] + phi[q * nt + n - 1]);
  }
  return p;
}

// rhs = 2 M w^{n-1} - A+ w^{n-1} + dt (sum_q avg_q (m_e f_q + [Neumann] |E| g_q))
// on free rows (A+ = M + dt/2 K; w^{n-1} holds u_D(t_{n-1}) on Dirichlet rows),
// u_D(t_n) on Dirichlet rows; also the averaged source f^{n-1/2} per edge.
__global__ void k_cn_rhs(int nE, const int32_t* __restrict__ nbr, const double* __restrict__ val,
                         const double* __restrict__ x, const double* __restrict__ me,
                         const uint8_t* __restrict__ eclass, const double* __restrict__ elen,
                         const double* __restrict__ fq, const double* __restrict__ bcq, int Q,
                         const double* __restrict__ phi, int nt, const int* __restrict__ step, double dt,
                         double* __restrict__ b, double* __restrict__ f_eff) {
  const size_t m = (size_t)nE;
  const Phi ph = phi_dev_at(phi, Q, nt, *step + 1);
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

// The same right-hand side from per-step data (general sources): f and g
// averaged over t_{n-1} and t_n from the two arrays, u_D(t_n) on Dirichlet rows.
__global__ void k_cn_rhs_data(int nE, const int32_t* __restrict__ nbr, const double* __restrict__ val,
                              const double* __restrict__ x, const double* __restrict__ me,
                              const uint8_t* __restrict__ eclass, const double* __restrict__ elen,
                              const double* __restrict__ f_now, const double* __restrict__ f_prev,
                              const double* __restrict__ bc_now, const double* __restrict__ bc_prev, double dt,
                              double* __restrict__ b, double* __restrict__ f_eff) {
  const size_t m = (size_t)nE;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nE; e += gridDim.x * blockDim.x) {
    const uint8_t cls = eclass[e];
    const double fav = 0.5 * ((f_now ? f_now[e] : 0.0) + f_prev[e]);
    f_eff[e] = fav;
    if (cls == PHFEM_EDGE_DIRICHLET) {
      b[e] = bc_now ? bc_now[e] : 0.0;
      continue;
    }
    const double xe = x[e];
    double aw = val[e] * xe;  // (A+ w)_e in difference form
#pragma unroll
    for (int s = 0; s < 4; ++s) aw += val[(s + 1) * m + e] * (xe - x[nbr[s * m + e]]);
    double load = me[e] * fav;
    if (cls == PHFEM_EDGE_NEUMANN) load += elen[e] * 0.5 * ((bc_now ? bc_now[e] : 0.0) + bc_prev[e]);
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

// Records the step's solve statistics and advances the step counter.
__global__ void k_cn_advance(int* step, const SolveState* st, int* it, int* conv, double* rel) {
  const int n = *step + 1;
  it[n] = st->it;
  conv[n] = st->done == 2 ? st->conv : (st->done == 3 ? st->status : PHFEM_ENOCONV);
  rel[n] = st->bb > 0 ? sqrt(st->rr64 / st->bb) : 0.0;
  *step = n;
}

void cn_free(phfem_cn cn) {
  phfem_ctx c = cn->sys->mesh->ctx;
  if (cn->exec) cudaGraphExecDestroy(cn->exec);
  dfree(c, cn->fq);
  dfree(c, cn->bcq);
  dfree(c, cn->phi_dev);
  dfree(c, cn->step_dev);
  dfree(c, cn->it_dev);
  dfree(c, cn->conv_dev);
  dfree(c, cn->rel_dev);
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

// One step's work up to the solve, on the context stream.
int enqueue_pre(phfem_cn cn) {
  phfem_sys sys = cn->sys;
  phfem_mesh m = sys->mesh;
  phfem_ctx ctx = m->ctx;
  cudaStream_t s = ctx->stream;
  const int nE = m->info.nE;
  PH_CUDA(cudaMemcpyAsync(cn->xprev, sys->x, sizeof(double) * nE, cudaMemcpyDeviceToDevice, s));
  k_cn_rhs<<<grid_for(ctx, nE), kBlock, 0, s>>>(nE, m->nbr, sys->val, sys->x, sys->me, m->eclass, m->elen, cn->fq,
                                                cn->bcq, cn->Q, cn->phi_dev, cn->nt, cn->step_dev, sys->c.dt, sys->b,
                                                cn->f_eff);
  PH_TRY(check_launch(ctx, "k_cn_rhs"));
  k_set_dirichlet<<<grid_for(ctx, nE), kBlock, 0, s>>>(nE, m->eclass, sys->b, sys->x);
  return check_launch(ctx, "k_set_dirichlet");
}

// One step's work after the solve: Lambda^{n-1/2}, Lambda^n, step statistics.
int enqueue_post(phfem_cn cn) {
  phfem_sys sys = cn->sys;
  phfem_mesh m = sys->mesh;
  phfem_ctx ctx = m->ctx;
  cudaStream_t s = ctx->stream;
  const int nL = m->info.nL;
  PH_TRY(recover(sys, sys->x, cn->xprev, cn->f_eff, 1.0 / sys->c.dt, 0.5, nullptr, cn->lam_half));
  k_lam_update<<<grid_for(ctx, nL), kBlock, 0, s>>>(nL, cn->lam_half, cn->lam_n);
  PH_TRY(check_launch(ctx, "k_lam_update"));
  k_cn_advance<<<1, 1, 0, s>>>(cn->step_dev, sys->st, cn->it_dev, cn->conv_dev, cn->rel_dev);
  return check_launch(ctx, "k_cn_advance");
}

// Captures one whole step into a graph: the solve loop runs in a conditional
// WHILE node controlled on the device, so a step needs no host round trip.
int build_step_graph(phfem_cn cn, const phfem_solve_opts& o) {
  phfem_ctx ctx = cn->sys->mesh->ctx;
  // the locality-order operator is allocated and built before the capture
  if (fcg_eligible(cn->sys, o)) PH_TRY(fcg_prepare(cn->sys));
  PH_CUDA(cudaStreamSynchronize(ctx->stream));
  cudaStream_t cs;
  PH_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  const cudaStream_t saved = ctx->stream;
  const bool saved_prof = ctx->profile;
  ctx->stream = cs;      // every helper enqueues on ctx->stream
  ctx->profile = false;  // no event nodes inside the graph
  int st = PHFEM_OK;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) st = cuda_fail(e, "cudaStreamBeginCapture", __FILE__, __LINE__);
  if (st == PHFEM_OK) st = enqueue_pre(cn);
  if (st == PHFEM_OK) st = capture_solve(cn->sys, &o, cs, cn->sys->mg ? 2 : 8);
  if (st == PHFEM_OK) st = enqueue_post(cn);
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(cs, &graph);
  if (e != cudaSuccess && st == PHFEM_OK) st = cuda_fail(e, "cudaStreamEndCapture", __FILE__, __LINE__);
  ctx->stream = saved;
  ctx->profile = saved_prof;
  if (st == PHFEM_OK) {
    if (cn->exec) cudaGraphExecDestroy(cn->exec);
    cn->exec = nullptr;
    e = cudaGraphInstantiate(&cn->exec, graph, 0);
    if (e != cudaSuccess) st = cuda_fail(e, "cudaGraphInstantiate", __FILE__, __LINE__);
  }
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(cs);
  cudaGetLastError();
  if (st == PHFEM_OK) cn->graph_opts = o;
  return st;
}

int read_steps(phfem_cn cn, int first, int count, phfem_stats* st) {
  if (count <= 0) return PHFEM_OK;
  cudaStream_t s = cn->sys->mesh->ctx->stream;
  std::vector<int> it(count), conv(count);
  std::vector<double> rel(count);
  PH_CUDA(cudaMemcpyAsync(it.data(), cn->it_dev + first, sizeof(int) * count, cudaMemcpyDeviceToHost, s));
  PH_CUDA(cudaMemcpyAsync(conv.data(), cn->conv_dev + first, sizeof(int) * count, cudaMemcpyDeviceToHost, s));
  PH_CUDA(cudaMemcpyAsync(rel.data(), cn->rel_dev + first, sizeof(double) * count, cudaMemcpyDeviceToHost, s));
  PH_CUDA(cudaStreamSynchronize(s));
  int worst = 1;
  for (int i = 0; i < count; ++i) {
    st->iterations += it[i];
    worst = std::min(worst, conv[i]);
    st->rel_residual = std::max(st->rel_residual, rel[i]);
  }
  st->converged = worst;
  return worst > 0 ? PHFEM_OK : worst;
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
  chk(dalloc_n(ctx, &cn->phi_dev, (size_t)cn->Q * cn->nt));
  chk(dalloc_n(ctx, &cn->step_dev, 1));
  chk(dalloc_n(ctx, &cn->it_dev, cn->nt));
  chk(dalloc_n(ctx, &cn->conv_dev, cn->nt));
  chk(dalloc_n(ctx, &cn->rel_dev, cn->nt));
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
    cudaMemcpyAsync(cn->phi_dev, cn->phi.data(), sizeof(double) * cn->phi.size(), cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(cn->step_dev, 0, sizeof(int), s);
    cudaMemsetAsync(cn->it_dev, 0, sizeof(int) * cn->nt, s);
    cudaMemsetAsync(cn->conv_dev, 0, sizeof(int) * cn->nt, s);
    cudaMemsetAsync(cn->rel_dev, 0, sizeof(double) * cn->nt, s);
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
  if (cn->Q == 0) return fail(PHFEM_EINVAL, "phfem_cn_step: created for per-step data (use phfem_cn_step_data)");
  if (cn->step + nsteps >= cn->nt)
    return fail(PHFEM_EINVAL, "phfem_cn_step: the source has no time factors for the requested steps");
  auto t0 = std::chrono::steady_clock::now();
  phfem_sys sys = cn->sys;
  phfem_mesh m = sys->mesh;
  phfem_ctx ctx = m->ctx;
  cudaStream_t s = ctx->stream;
  phfem_stats st{};
  int status = PHFEM_OK;
  for (int k = 0; k < nsteps; ++k) {
    PH_TRY(enqueue_pre(cn));
    status = solve_system(sys, opts, &st, true);
    if (status != PHFEM_OK) break;
    PH_TRY(enqueue_post(cn));
    cn->step += 1;
    st.steps += 1;
  }
  PH_CUDA(cudaStreamSynchronize(s));
  st.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (stats) *stats = st;
  return status;
}

PHFEM_API int phfem_cn_step_graph(phfem_cn cn, int32_t nsteps, const phfem_solve_opts* opts, phfem_stats* stats) {
  if (!cn || nsteps < 0) return fail(PHFEM_EINVAL, "phfem_cn_step_graph: bad argument");
  if (cn->Q == 0) return fail(PHFEM_EINVAL, "phfem_cn_step_graph: created for per-step data (use phfem_cn_step_data)");
  if (cn->step + nsteps >= cn->nt)
    return fail(PHFEM_EINVAL, "phfem_cn_step_graph: the source has no time factors for the requested steps");
  auto t0 = std::chrono::steady_clock::now();
  phfem_solve_opts o{};
  if (opts) o = *opts;
  fill_opts(cn->sys, o);
  if (!cn->exec || std::memcmp(&o, &cn->graph_opts, sizeof(o)) != 0) PH_TRY(build_step_graph(cn, o));
  phfem_ctx ctx = cn->sys->mesh->ctx;
  for (int k = 0; k < nsteps; ++k) PH_CUDA(cudaGraphLaunch(cn->exec, ctx->stream));
  ctx->launches += (int64_t)nsteps;
  phfem_stats st{};
  const int first = cn->step + 1;
  int status = read_steps(cn, first, nsteps, &st);
  cn->step += nsteps;
  st.steps = nsteps;
  st.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (stats) *stats = st;
  if (status != PHFEM_OK) return fail(status, "phfem_cn_step_graph: a step did not converge");
  return PHFEM_OK;
}

PHFEM_API int phfem_cn_create_data(phfem_sys sys, const double* f0_mid, const double* bc0_mid, const double* w0,
                                   const double* Lambda0, int32_t max_steps, phfem_cn* out) {
  if (!out) return fail(PHFEM_EINVAL, "phfem_cn_create_data: out is NULL");
  *out = nullptr;
  if (!sys || max_steps < 1) return fail(PHFEM_EINVAL, "phfem_cn_create_data: bad argument");
  if (!(sys->c.dt > 0)) return fail(PHFEM_EINVAL, "phfem_cn_create_data: the system was assembled with dt = 0");
  phfem_mesh m = sys->mesh;
  phfem_ctx ctx = m->ctx;
  cudaStream_t s = ctx->stream;
  const size_t nE = m->info.nE, nL = m->info.nL;
  phfem_cn cn = new phfem_cn_s();
  cn->sys = sys;
  cn->Q = 0;
  cn->nt = max_steps + 1;
  cn->step = 0;
  int st = PHFEM_OK;
  auto chk = [&](int r) {
    if (st == PHFEM_OK) st = r;
  };
  chk(dalloc_n(ctx, &cn->fq, nE));   // f and g / u_D of the previous step
  chk(dalloc_n(ctx, &cn->bcq, nE));
  chk(dalloc_n(ctx, &cn->step_dev, 1));
  chk(dalloc_n(ctx, &cn->it_dev, cn->nt));
  chk(dalloc_n(ctx, &cn->conv_dev, cn->nt));
  chk(dalloc_n(ctx, &cn->rel_dev, cn->nt));
  chk(dalloc_n(ctx, &cn->xprev, nE));
  chk(dalloc_n(ctx, &cn->f_eff, nE));
  chk(dalloc_n(ctx, &cn->lam_half, nL));
  chk(dalloc_n(ctx, &cn->lam_n, nL));
  if (st == PHFEM_OK) {
    if (f0_mid) cudaMemcpyAsync(cn->fq, f0_mid, sizeof(double) * nE, cudaMemcpyDeviceToDevice, s);
    else cudaMemsetAsync(cn->fq, 0, sizeof(double) * nE, s);
    if (bc0_mid) cudaMemcpyAsync(cn->bcq, bc0_mid, sizeof(double) * nE, cudaMemcpyDeviceToDevice, s);
    else cudaMemsetAsync(cn->bcq, 0, sizeof(double) * nE, s);
    if (Lambda0) cudaMemcpyAsync(cn->lam_n, Lambda0, sizeof(double) * nL, cudaMemcpyDeviceToDevice, s);
    else cudaMemsetAsync(cn->lam_n, 0, sizeof(double) * nL, s);
    cudaMemsetAsync(cn->lam_half, 0, sizeof(double) * nL, s);
    cudaMemsetAsync(cn->step_dev, 0, sizeof(int), s);
    cudaMemsetAsync(cn->it_dev, 0, sizeof(int) * cn->nt, s);
    cudaMemsetAsync(cn->conv_dev, 0, sizeof(int) * cn->nt, s);
    cudaMemsetAsync(cn->rel_dev, 0, sizeof(double) * cn->nt, s);
    Phi one{};
    one.now[0] = 1.0;  // x = w0, and u_D(t_0) on Dirichlet rows
    k_cn_init<<<grid_for(ctx, nE), kBlock, 0, s>>>((int)nE, m->eclass, w0, cn->bcq, 1, one, sys->x);
    st = check_launch(ctx, "k_cn_init");
  }
  if (st == PHFEM_OK && cudaStreamSynchronize(s) != cudaSuccess)
    st = cuda_fail(cudaGetLastError(), "phfem_cn_create_data", __FILE__, __LINE__);
  if (st != PHFEM_OK) {
    cudaStreamSynchronize(s);
    cn_free(cn);
    return st;
  }
  *out = cn;
  return PHFEM_OK;
}

PHFEM_API int phfem_cn_step_data(phfem_cn cn, const double* f_mid, const double* bc_mid,
                                 const phfem_solve_opts* opts, phfem_stats* stats) {
  if (!cn) return fail(PHFEM_EINVAL, "phfem_cn_step_data: NULL handle");
  if (cn->Q != 0) return fail(PHFEM_EINVAL, "phfem_cn_step_data: created for a separable source (use phfem_cn_step)");
  if (cn->step + 1 >= cn->nt) return fail(PHFEM_EINVAL, "phfem_cn_step_data: max_steps reached");
  auto t0 = std::chrono::steady_clock::now();
  phfem_sys sys = cn->sys;
  phfem_mesh m = sys->mesh;
  phfem_ctx ctx = m->ctx;
  cudaStream_t s = ctx->stream;
  const int nE = m->info.nE;
  PH_CUDA(cudaMemcpyAsync(cn->xprev, sys->x, sizeof(double) * nE, cudaMemcpyDeviceToDevice, s));
  k_cn_rhs_data<<<grid_for(ctx, nE), kBlock, 0, s>>>(nE, m->nbr, sys->val, sys->x, sys->me, m->eclass, m->elen, f_mid,
                                                     cn->fq, bc_mid, cn->bcq, sys->c.dt, sys->b, cn->f_eff);
  PH_TRY(check_launch(ctx, "k_cn_rhs_data"));
  k_set_dirichlet<<<grid_for(ctx, nE), kBlock, 0, s>>>(nE, m->eclass, sys->b, sys->x);
  PH_TRY(check_launch(ctx, "k_set_dirichlet"));
  phfem_stats st{};
  int status = solve_system(sys, opts, &st, true);
  if (status == PHFEM_OK) {
    PH_TRY(enqueue_post(cn));
    // this step's data become the previous step's
    if (f_mid) PH_CUDA(cudaMemcpyAsync(cn->fq, f_mid, sizeof(double) * nE, cudaMemcpyDeviceToDevice, s));
    else PH_CUDA(cudaMemsetAsync(cn->fq, 0, sizeof(double) * nE, s));
    if (bc_mid) PH_CUDA(cudaMemcpyAsync(cn->bcq, bc_mid, sizeof(double) * nE, cudaMemcpyDeviceToDevice, s));
    else PH_CUDA(cudaMemsetAsync(cn->bcq, 0, sizeof(double) * nE, s));
    cn->step += 1;
    st.steps = 1;
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
