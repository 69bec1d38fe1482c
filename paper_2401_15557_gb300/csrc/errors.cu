// Error report of a computed solution against an exact one (the error tables
// of Section 3.6: the L2 error, the broken H1 error and the mesh norm of the
// multiplier error).
//
// The library owns the quadrature: a Duffy-collapsed nq x nq Gauss-Legendre
// rule on every triangle (s = x_i, t = x_j (1 - x_i), weight w_i w_j (1 - x_i),
// Jacobian 2|T|) and an nq-point Gauss-Legendre rule on every multiplier edge.
// phfem_error_points writes the physical points, the caller evaluates the exact
// solution there (any way it likes, on the device), and phfem_error_norms
// integrates.  Sums are FP64, per thread then per block then over the blocks in
// a fixed order, so the report is deterministic.
#include <cmath>

#include "internal.cuh"

namespace phfem {
namespace {

constexpr int kMaxNq = 16;

struct Rule {
  double x[kMaxNq];  // nodes on [0, 1]
  double w[kMaxNq];  // weights, summing to 1
  int n;
};

// Gauss-Legendre nodes as roots of P_n by Newton's method on the three-term
// recurrence (n P_n = (2n-1) x P_{n-1} - (n-1) P_{n-2}), weights
// 2 / ((1 - x^2) P_n'(x)^2); mapped from [-1, 1] to [0, 1].
Rule gauss_legendre01(int n) {
  Rule r{};
  r.n = n;
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < n; ++i) {
    double x = std::cos(pi * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = x;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      const double pn = n == 1 ? x : p1;
      const double pm = n == 1 ? 1.0 : p0;
      dp = n * (x * pn - pm) / (x * x - 1.0);
      const double dx = pn / dp;
      x -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    {  // derivative at the converged root
      double p0 = 1.0, p1 = x;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      const double pn = n == 1 ? x : p1;
      const double pm = n == 1 ? 1.0 : p0;
      dp = n * (x * pn - pm) / (x * x - 1.0);
    }
    // ascending order on [0, 1]
    r.x[n - 1 - i] = 0.5 * (x + 1.0);
    r.w[n - 1 - i] = 1.0 / ((1.0 - x * x) * dp * dp);
  }
  return r;
}

__device__ __forceinline__ void duffy(const Rule& R, int q, double& s, double& t, double& w) {
  const int i = q / R.n, j = q - i * R.n;
  s = R.x[i];
  t = R.x[j] * (1.0 - R.x[i]);
  w = R.w[i] * R.w[j] * (1.0 - R.x[i]);
}

__global__ void k_tri_points(int nT, const int32_t* __restrict__ tri, const double2* __restrict__ xy, Rule R,
                             double2* __restrict__ out) {
  const int Q = R.n * R.n;
  const int64_t total = (int64_t)nT * Q;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
    const int t = (int)(k / Q), q = (int)(k - (int64_t)t * Q);
    const double2 P0 = xy[tri[3 * t]], P1 = xy[tri[3 * t + 1]], P2 = xy[tri[3 * t + 2]];
    double s, u, w;
    duffy(R, q, s, u, w);
    const double l0 = 1.0 - s - u;
    out[k] = make_double2(l0 * P0.x + s * P1.x + u * P2.x, l0 * P0.y + s * P1.y + u * P2.y);
  }
}

// Points and outward normals (of T+) of the multiplier edges, in multiplier order.
__global__ void k_edge_points(int nE, const int32_t* __restrict__ ed2el, const int32_t* __restrict__ lam_id,
                              const double2* __restrict__ xy, Rule R, double2* __restrict__ pts,
                              double2* __restrict__ nu) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nE; e += gridDim.x * blockDim.x) {
    const int li = lam_id[e];
    if (li < 0) continue;
    const double2 a = xy[ed2el[4 * e]], b = xy[ed2el[4 * e + 1]];
    const double dx = b.x - a.x, dy = b.y - a.y;
    if (nu) {
      const double L = sqrt(dx * dx + dy * dy);
      nu[li] = make_double2(dy / L, -dx / L);
    }
    if (pts)
      for (int q = 0; q < R.n; ++q) pts[(size_t)li * R.n + q] = make_double2(a.x + R.x[q] * dx, a.y + R.x[q] * dy);
  }
}

// Per triangle: sum over the points of 2|T| w (u - u_h)^2 and 2|T| w |grad u - grad u_h|^2,
// with u_h = sum_k lambda_k U_k and grad u_h = sum_k U_k grad lambda_k.
__global__ void k_tri_errors(int nT, const int32_t* __restrict__ tri, const double2* __restrict__ xy,
                             const double* __restrict__ U, const double* __restrict__ uq,
                             const double2* __restrict__ gq, Rule R, double* partials, unsigned int* counter,
                             double* result) {
  __shared__ double smem[kBlock / 32];
  const int Q = R.n * R.n;
  double acc_l2 = 0.0, acc_h1 = 0.0;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nT; t += gridDim.x * blockDim.x) {
    const double2 P0 = xy[tri[3 * t]], P1 = xy[tri[3 * t + 1]], P2 = xy[tri[3 * t + 2]];
    const double det = (P1.x - P0.x) * (P2.y - P0.y) - (P2.x - P0.x) * (P1.y - P0.y);  // 2|T|
    const double U0 = U[3 * t], U1 = U[3 * t + 1], U2 = U[3 * t + 2];
    // grad lambda_k = (y_{k+1} - y_{k+2}, x_{k+2} - x_{k+1}) / 2|T|
    const double gx = (U0 * (P1.y - P2.y) + U1 * (P2.y - P0.y) + U2 * (P0.y - P1.y)) / det;
    const double gy = (U0 * (P2.x - P1.x) + U1 * (P0.x - P2.x) + U2 * (P1.x - P0.x)) / det;
    double el2 = 0.0, eh1 = 0.0;
    for (int q = 0; q < Q; ++q) {
      double s, u, w;
      duffy(R, q, s, u, w);
      const double uh = (1.0 - s - u) * U0 + s * U1 + u * U2;
      const double d = uq[(size_t)t * Q + q] - uh;
      const double2 g = gq[(size_t)t * Q + q];
      el2 += w * d * d;
      eh1 += w * ((g.x - gx) * (g.x - gx) + (g.y - gy) * (g.y - gy));
    }
    acc_l2 += det * el2;
    acc_h1 += det * eh1;
  }
  acc_l2 = block_sum(acc_l2, smem);
  acc_h1 = block_sum(acc_h1, smem);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = acc_l2;
    partials[kMaxGrid + blockIdx.x] = acc_h1;
  }
  if (!arrive_last(counter)) return;
  const double l2 = sum_partials(partials, smem);
  const double h1 = sum_partials(partials + kMaxGrid, smem);
  if (threadIdx.x == 0) {
    *counter = 0;
    result[0] = l2;
    result[1] = h1;
  }
}

// Per multiplier edge: |E| * (|E| sum_q w_q (kappa_q - Lambda_E)^2).
__global__ void k_edge_errors(int nE, const int32_t* __restrict__ ed2el, const int32_t* __restrict__ lam_id,
                              const double2* __restrict__ xy, const double* __restrict__ Lambda,
                              const double* __restrict__ kq, Rule R, double* partials, unsigned int* counter,
                              double* result) {
  __shared__ double smem[kBlock / 32];
  double acc = 0.0;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nE; e += gridDim.x * blockDim.x) {
    const int li = lam_id[e];
    if (li < 0) continue;
    const double2 a = xy[ed2el[4 * e]], b = xy[ed2el[4 * e + 1]];
    const double L = sqrt((b.x - a.x) * (b.x - a.x) + (b.y - a.y) * (b.y - a.y));
    const double lam = Lambda[li];
    double s = 0.0;
    for (int q = 0; q < R.n; ++q) {
      const double d = kq[(size_t)li * R.n + q] - lam;
      s += R.w[q] * d * d;
    }
    acc += L * (s * L);
  }
  acc = block_sum(acc, smem);
  if (threadIdx.x == 0) partials[2 * kMaxGrid + blockIdx.x] = acc;
  if (!arrive_last(counter + 1)) return;
  const double m = sum_partials(partials + 2 * kMaxGrid, smem);
  if (threadIdx.x == 0) {
    counter[1] = 0;
    result[2] = m;
  }
}

int check_nq(int nq, const char* who) {
  if (nq < 1 || nq > kMaxNq) return fail(PHFEM_EINVAL, std::string(who) + ": nq must be in 1..16");
  return PHFEM_OK;
}

}  // namespace
}  // namespace phfem

using namespace phfem;

extern "C" {

PHFEM_API int phfem_error_points(phfem_mesh mesh, int32_t nq, double* tri_xy, double* edge_xy, double* edge_nu) {
  if (!mesh) return fail(PHFEM_EINVAL, "phfem_error_points: NULL mesh");
  PH_TRY(check_nq(nq, "phfem_error_points"));
  phfem_ctx ctx = mesh->ctx;
  const Rule R = gauss_legendre01(nq);
  const phfem_mesh_info& I = mesh->info;
  const double2* xy = reinterpret_cast<const double2*>(mesh->xy);
  if (tri_xy && I.nT > 0) {
    const int64_t total = (int64_t)I.nT * nq * nq;
    k_tri_points<<<grid_for(ctx, total), kBlock, 0, ctx->stream>>>(I.nT, mesh->tri, xy, R,
                                                                    reinterpret_cast<double2*>(tri_xy));
    PH_TRY(check_launch(ctx, "k_tri_points"));
  }
  if ((edge_xy || edge_nu) && I.nL > 0) {
    k_edge_points<<<grid_for(ctx, I.nE), kBlock, 0, ctx->stream>>>(I.nE, mesh->ed2el, mesh->lam_id, xy, R,
                                                                    reinterpret_cast<double2*>(edge_xy),
                                                                    reinterpret_cast<double2*>(edge_nu));
    PH_TRY(check_launch(ctx, "k_edge_points"));
  }
  return PHFEM_OK;
}

PHFEM_API int phfem_error_norms(phfem_mesh mesh, int32_t nq, const double* U, const double* u_q,
                                const double* grad_q, const double* Lambda, const double* kappa_q,
                                phfem_errors* out) {
  if (!mesh || !out) return fail(PHFEM_EINVAL, "phfem_error_norms: NULL argument");
  PH_TRY(check_nq(nq, "phfem_error_norms"));
  const bool tri_part = U && u_q && grad_q;
  const bool edge_part = Lambda && kappa_q;
  if (!tri_part && (U || u_q || grad_q))
    return fail(PHFEM_EINVAL, "phfem_error_norms: U, u_q and grad_q go together");
  if (!edge_part && (Lambda || kappa_q))
    return fail(PHFEM_EINVAL, "phfem_error_norms: Lambda and kappa_q go together");
  phfem_ctx ctx = mesh->ctx;
  cudaStream_t s = ctx->stream;
  const Rule R = gauss_legendre01(nq);
  const phfem_mesh_info& I = mesh->info;
  const double2* xy = reinterpret_cast<const double2*>(mesh->xy);
  double* scratch = nullptr;  // partials [3][kMaxGrid], results [3], counters
  const size_t n_d = 3 * (size_t)kMaxGrid + 4;
  PH_TRY(dalloc(ctx, reinterpret_cast<void**>(&scratch), n_d * sizeof(double) + 16));
  double* partials = scratch;
  double* result = scratch + 3 * kMaxGrid;
  unsigned int* counter = reinterpret_cast<unsigned int*>(scratch + n_d);
  int st = PHFEM_OK;
  cudaError_t e = cudaMemsetAsync(scratch, 0, n_d * sizeof(double) + 16, s);
  if (e != cudaSuccess) st = cuda_fail(e, "cudaMemsetAsync", __FILE__, __LINE__);
  if (st == PHFEM_OK && tri_part && I.nT > 0) {
    k_tri_errors<<<grid_for(ctx, I.nT), kBlock, 0, s>>>(I.nT, mesh->tri, xy, U, u_q,
                                                        reinterpret_cast<const double2*>(grad_q), R, partials,
                                                        counter, result);
    st = check_launch(ctx, "k_tri_errors");
  }
  if (st == PHFEM_OK && edge_part && I.nL > 0) {
    k_edge_errors<<<grid_for(ctx, I.nE), kBlock, 0, s>>>(I.nE, mesh->ed2el, mesh->lam_id, xy, Lambda, kappa_q, R,
                                                         partials, counter, result);
    st = check_launch(ctx, "k_edge_errors");
  }
  double h[3] = {0.0, 0.0, 0.0};
  if (st == PHFEM_OK) {
    e = cudaMemcpyAsync(h, result, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_fail(e, "phfem_error_norms: read back", __FILE__, __LINE__);
  }
  dfree(ctx, scratch);
  PH_TRY(st);
  out->L2 = std::sqrt(h[0]);
  out->H1semi = std::sqrt(h[1]);
  out->H1 = std::sqrt(h[0] + h[1]);
  out->M = std::sqrt(h[2]);
  return PHFEM_OK;
}

}  // extern "C"
