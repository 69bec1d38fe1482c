// Assembly of the condensed edge system (Definition 3.1 condensed to the edge
// midpoints; Eqs. right_b, right_g) and its CSR export.
//
// With u_T = R^-1 w_T (R of Definition 3.1, R^-1 = J - 2I), the element block
// a_T B_T + delta M_T becomes
//     K^CR_T[k][j] = (a_T / |T|) e_k . e_j + delta |T|/3 [k == j]
// where e_k = P_{k+2} - P_{k+1} is the edge vector opposite P_k (cyclic), since
// |T| grad(lambda_k) . grad(lambda_j) = e_k . e_j / (4 |T|) and
// R^-T M_T R^-1 = delta |T|/3 I.  The load |T|/3 sum_i f(m_i) R_i of Eq. right_b
// becomes |T|/3 f(m_k) on edge k, and the Neumann term |E| g(m_E) R_k of
// Eq. right_g becomes |E| g(m_E) on that edge.
//
// Two passes, none with atomics:
//   k_asm_tri   one thread per triangle: geometry and the record of K^CR_T
//               (its off-diagonal entries, negated, and |T|/3: the stiffness
//               rows sum to zero, e_0 + e_1 + e_2 = 0, so the diagonal
//               follows), 32 bytes AoS per triangle in FP64; FP32 systems
//               take compensated FP32 element arithmetic (c32.cuh), FP64
//               past an aspect bound;
//   k_asm_rows  one thread per edge: its row = the rows of K^CR_{T+} and
//               K^CR_{T-} at the edge, the rhs, and the operator, in FP64 and
//               in the inner precision, in difference form
//                 (S p)_e = r_e p_e + sum_s l_es (p_e - p_s),  l_es = -S_es,
//               with r_e the reaction/mass part of the diagonal.  The stiffness
//               rows of K^CR sum to zero, so the diagonal is sum_s l_es + r_e
//               exactly; storing l and r instead of S keeps constants in the
//               kernel of the rounded operator, and rounding l and r to FP32
//               perturbs S by a relative 2^-24 in the energy norm whatever its
//               condition number -- which is what lets the FP32 inner solve
//               drive an FP64 refinement on fine meshes.
#include <cmath>
#include <type_traits>

#include "kernels.cuh"

namespace phfem {
namespace {

// rec: [nT][4] records (C32: compensated FP32 element arithmetic, for FP32
// systems); conv: [3][nT] the column values c_j of the convection block, or NULL.
template <bool C32>
__global__ void k_asm_tri(int nT, const int32_t* __restrict__ tri, const double2* __restrict__ xy,
                          const double* __restrict__ aT, double a_const, double A11, double A12, double A22,
                          double px, double py, double* __restrict__ rec, double* __restrict__ conv,
                          int* __restrict__ bad) {
  const size_t n = (size_t)nT;
  const bool iso = A11 == 1.0 && A12 == 0.0 && A22 == 1.0;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nT; t += gridDim.x * blockDim.x) {
    const int v0 = tri[3 * t], v1 = tri[3 * t + 1], v2 = tri[3 * t + 2];
    const double a = aT ? aT[t] : a_const;
    // a > 0 and finite, tested on the 32-bit halves of its bits (integer
    // pipe): sign clear, not zero, and an exponent below the all-ones of Inf / NaN
    const int ahi = __double2hiint(a);
    const bool finite = ((ahi >> 20) & 0x7FF) != 0x7FF;
    if (!(ahi >= 0 && (ahi | __double2loint(a)) != 0 && finite)) atomicOr(bad, finite ? 1 : 2);
    const double2 p0 = __ldg(xy + v0), p1 = __ldg(xy + v1), p2 = __ldg(xy + v2);
    double* dst = rec + (size_t)kRec * t;
    if constexpr (C32) {
      tri_record32_store(p0, p1, p2, a, dst, iso, A11, A12, A22);
    } else {
      double R[4];
      tri_record64(p0, p1, p2, a, R, A11, A12, A22);
      store_record(dst, R);
    }
    if (conv) {
      double c[3];
      tri_conv(p0, p1, p2, px, py, c);
#pragma unroll
      for (int j = 0; j < 3; ++j) conv[j * n + t] = c[j];
    }
  }
}

// Adds the convection columns of T+ (tp, local kp) and T- to an edge row
// (slots: T+ (k+1, k+2), T- (k+1, k+2)); the row sums do not change.
__device__ __forceinline__ void add_conv(const double* c, size_t n, int tp, int kp, int tm, int km, double sK,
                                         EdgeRow& R) {
  R.diag += sK * c[(size_t)kp * n + tp];
  R.l[0] -= sK * c[(size_t)((kp + 1) % 3) * n + tp];
  R.l[1] -= sK * c[(size_t)((kp + 2) % 3) * n + tp];
  if (tm >= 0) {
    R.diag += sK * c[(size_t)km * n + tm];
    R.l[2] -= sK * c[(size_t)((km + 1) % 3) * n + tm];
    R.l[3] -= sK * c[(size_t)((km + 2) % 3) * n + tm];
  }
}

// sK scales K^CR and sM the mass |T|/3 (elliptic: 1, 0; Crank-Nicolson: dt/2, 1).
// The boundary data is read on boundary edges only; me (the mass diagonal,
// read by the Crank-Nicolson right-hand side) may be NULL.
template <typename T, bool ELLIPTIC>
__global__ void k_asm_rows(int nE, int nT, const int32_t* __restrict__ ed2el, const uint8_t* __restrict__ lk,
                           const uint8_t* __restrict__ eclass, const double* __restrict__ rec,
                           const double* __restrict__ conv, const double* __restrict__ f_mid,
                           const double* __restrict__ bc_mid, const double* __restrict__ elen, double sK, double sM,
                           double delta, double* __restrict__ val, double* __restrict__ b, double* __restrict__ me,
                           T* __restrict__ lval, T* __restrict__ rdiag, T* __restrict__ dinv,
                           const int32_t* __restrict__ tiles) {
  const size_t n = (size_t)nT, m = (size_t)nE;
  // tiles of kBlock consecutive rows, in the mesh's tile order when given
  const int ntiles = (nE + kBlock - 1) / kBlock;
  for (int v = blockIdx.x; v < ntiles; v += gridDim.x) {
    const int e = (tiles ? tiles[v] : v) * kBlock + threadIdx.x;
    if (e >= nE) continue;
    const int4 q = reinterpret_cast<const int4*>(ed2el)[e];
    const int kk = lk[e];
    const uint8_t cls = eclass[e];
    const int kp = kk & 3, km = (kk >> 2) & 3;
    const double bc = (bc_mid && cls != PHFEM_EDGE_INTERIOR) ? bc_mid[e] : 0.0;
    EdgeRow R = edge_row<true, ELLIPTIC>(rec, q.z, kp, q.w, km, cls, f_mid ? f_mid[e] : 0.0, bc,
                                         cls == PHFEM_EDGE_NEUMANN ? elen[e] : 0.0, sK, sM, delta,
                                         f_mid != nullptr, bc_mid != nullptr);
    if (conv && cls != PHFEM_EDGE_DIRICHLET) add_conv(conv, n, q.z, kp, q.w, km, sK, R);
    val[e] = R.rpart;
#pragma unroll
    for (int s = 0; s < 4; ++s) val[(s + 1) * m + e] = R.l[s];
    b[e] = R.rhs;
    if (me) me[e] = R.mass;
    store_inner(R, m, e, lval, rdiag, dinv);
  }
}

// Flux form, per triangle: S_T = D (K^CR_T)^-1 D with D = diag(sigma_k |E_k|)
// and the load term g_T = -D (K^CR_T)^-1 F^CR_T, F^CR_T[k] = |T|/3 f(m_k)
// + [edge k Neumann] |E_k| g(m_k) (C_T K_T^-1 C_T' and C_T K_T^-1 F_T written
// with C_T = D R and R K_T^-1 R' = (K^CR_T)^-1).  The inverse of the symmetric
// 3x3 block is its cofactor matrix over the determinant.
__global__ void k_asm_flux_tri(int nT, const int32_t* __restrict__ t2e, const int8_t* __restrict__ sigma,
                               const uint8_t* __restrict__ eclass, const double* __restrict__ elen,
                               const double* __restrict__ rec, double delta, const double* __restrict__ f_mid,
                               const double* __restrict__ bc_mid, double* __restrict__ St) {
  const size_t n = (size_t)nT;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nT; t += gridDim.x * blockDim.x) {
    double r[4], K[6];
    load_record<true>(rec, t, r);
    record_block(r, delta, K);
    const double a = K[0], b = K[1], c = K[2], d = K[3], e = K[4], f = K[5], mT = r[3];
    const double C00 = b * c - e * e, C11 = a * c - f * f, C22 = a * b - d * d;
    const double C01 = e * f - d * c, C12 = d * f - a * e, C20 = d * e - b * f;
    const double inv = 1.0 / (a * C00 + d * C01 + f * C20);
    const double I00 = C00 * inv, I11 = C11 * inv, I22 = C22 * inv, I01 = C01 * inv, I12 = C12 * inv,
                 I20 = C20 * inv;
    double D[3], F[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int ek = t2e[3 * t + k];
      D[k] = sigma[3 * t + k] * elen[ek];
      F[k] = (f_mid ? mT * f_mid[ek] : 0.0) +
             ((bc_mid && eclass[ek] == PHFEM_EDGE_NEUMANN) ? elen[ek] * bc_mid[ek] : 0.0);
    }
    St[0 * n + t] = D[0] * I00 * D[0];
    St[1 * n + t] = D[1] * I11 * D[1];
    St[2 * n + t] = D[2] * I22 * D[2];
    St[3 * n + t] = D[0] * I01 * D[1];
    St[4 * n + t] = D[1] * I12 * D[2];
    St[5 * n + t] = D[2] * I20 * D[0];
    const double y0 = I00 * F[0] + I01 * F[1] + I20 * F[2];
    const double y1 = I01 * F[0] + I11 * F[1] + I12 * F[2];
    const double y2 = I20 * F[0] + I12 * F[1] + I22 * F[2];
    St[6 * n + t] = -D[0] * y0;
    St[7 * n + t] = -D[1] * y1;
    St[8 * n + t] = -D[2] * y2;
  }
}

// Row k of S_T stored slot-major with stride n (00, 11, 22, 01, 12, 20):
// the diagonal, (k, k+1) and (k+2, k).
__device__ __forceinline__ void st_row(const double* St, size_t n, int t, int k, double& d, double& o1,
                                       double& o2) {
  const int k2 = (k == 0) ? 2 : k - 1;  // k + 2 mod 3
  d = __ldg(St + (size_t)k * n + t);
  o1 = __ldg(St + (size_t)(3 + k) * n + t);
  o2 = __ldg(St + (size_t)(3 + k2) * n + t);
}

// Flux-form rows: the rows of S_{T+} and S_{T-} at the edge, rhs = sum of the
// load terms + |E| u_D on Dirichlet edges (-b_D of Eq. DirichletEqn);
// Neumann edges are identity rows with Lambda = 0.
template <typename T>
__global__ void k_asm_rows_flux(int nE, int nT, const int32_t* __restrict__ ed2el, const uint8_t* __restrict__ lk,
                                const uint8_t* __restrict__ eclass, const double* __restrict__ St,
                                const double* __restrict__ bc_mid, const double* __restrict__ elen,
                                double* __restrict__ val, double* __restrict__ b, T* __restrict__ lval,
                                T* __restrict__ rdiag, T* __restrict__ dinv) {
  const size_t n = (size_t)nT, m = (size_t)nE;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nE; e += gridDim.x * blockDim.x) {
    const int4 q = reinterpret_cast<const int4*>(ed2el)[e];
    const int kk = lk[e];
    const uint8_t cls = eclass[e];
    double diag, v[4] = {0.0, 0.0, 0.0, 0.0}, rhs;
    if (cls == PHFEM_EDGE_NEUMANN) {
      diag = 1.0;
      rhs = 0.0;
    } else {
      double d, o1, o2;
      int k = kk & 3;
      st_row(St, n, q.z, k, d, o1, o2);
      diag = d;
      v[0] = o1;
      v[1] = o2;
      rhs = __ldg(St + (size_t)(6 + k) * n + q.z);
      if (q.w >= 0) {
        k = (kk >> 2) & 3;
        st_row(St, n, q.w, k, d, o1, o2);
        diag += d;
        v[2] = o1;
        v[3] = o2;
        rhs += __ldg(St + (size_t)(6 + k) * n + q.w);
      }
      if (cls == PHFEM_EDGE_DIRICHLET && bc_mid) rhs += elen[e] * bc_mid[e];
    }
    double rpart = diag;
#pragma unroll
    for (int s = 0; s < 4; ++s) rpart += v[s];  // diag = rpart + sum of l, l = -off
    val[e] = rpart;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      val[(s + 1) * m + e] = -v[s];
      lval[s * m + e] = (T)(-v[s]);
    }
    b[e] = rhs;
    rdiag[e] = (T)rpart;
    dinv[e] = (T)(1.0 / diag);
  }
}

// CSR export of the free-edge system: the row of free edge e lists (column,
// value) for e and its free neighbours, sorted by column; rhs subtracts the
// Dirichlet couplings times u_D (the lifting).
__global__ void k_export(int nE, const int32_t* __restrict__ nbr, const int32_t* __restrict__ free_id,
                         const uint8_t* __restrict__ eclass, const int32_t* __restrict__ row_ptr,
                         const double* __restrict__ val, const double* __restrict__ b, double* __restrict__ out_val,
                         double* __restrict__ out_rhs) {
  const size_t m = (size_t)nE;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nE; e += gridDim.x * blockDim.x) {
    const int r = free_id[e];
    if (r < 0) continue;
    int c[5];
    double v[5];
    int len = 0;
    double diag = val[e];  // r_e + sum of l_es over every neighbour slot
    for (int s = 0; s < 4; ++s) diag += val[(s + 1) * m + e];
    c[len] = r;
    v[len++] = diag;
    double rhs = b[e];
    for (int s = 0; s < 4; ++s) {
      const int n = nbr[s * m + e];
      if (n == e) continue;
      const double a = -val[(s + 1) * m + e];
      const int f = free_id[n];
      if (f >= 0) {
        c[len] = f;
        v[len++] = a;
      } else if (eclass[n] == PHFEM_EDGE_DIRICHLET) {
        rhs -= a * b[n];
      }
    }
    for (int i = 1; i < len; ++i) {
      int ck = c[i];
      double vk = v[i];
      int j = i - 1;
      while (j >= 0 && c[j] > ck) {
        c[j + 1] = c[j];
        v[j + 1] = v[j];
        --j;
      }
      c[j + 1] = ck;
      v[j + 1] = vk;
    }
    if (out_val) {
      const int base = row_ptr[r];
      for (int i = 0; i < len; ++i) out_val[base + i] = v[i];
    }
    if (out_rhs) out_rhs[r] = rhs;
  }
}

void sys_free(phfem_sys s) {
  phfem_ctx c = s->mesh->ctx;
  dfree(c, s->Kt);
  dfree(c, s->val);
  dfree(c, s->b);
  dfree(c, s->me);
  dfree(c, s->lval);
  dfree(c, s->rdiag);
  dfree(c, s->dinv);
  dfree(c, s->f);
  dfree(c, s->bc);
  dfree(c, s->St);
  dfree(c, s->bw);
  if (s->mg) mg_forget_system(s->mg);
  dfree(c, s->x);
  dfree(c, s->xh);
  dfree(c, s->xl);
  dfree(c, s->r64);
  dfree(c, s->ri);  // p and q live in the same allocation
  dfree(c, s->partials);
  dfree(c, s->st);
  fcg_free(s);
  delete s;
}

}  // namespace

// Runs the three assembly passes (also used to re-assemble in place).
int assemble_into(phfem_sys sys, const double* f_mid, const double* bc_mid, int* d_bad) {
  phfem_mesh m = sys->mesh;
  phfem_ctx ctx = m->ctx;
  cudaStream_t s = ctx->stream;
  const int nT = m->info.nT, nE = m->info.nE;
  const phfem_coeffs& c = sys->c;
  if (!m->row_tiles && sys->form == PHFEM_FORM_TRACE) {
    // the rows' visit order, once per mesh (not while a graph is captured: the
    // rows are then visited in the paper's order, with the same results)
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone) {
      if (mesh_row_tiles(m) != PHFEM_OK) cudaGetLastError();  // without it the paper's order is used
    } else {
      cudaGetLastError();
    }
  }
  prof_start(ctx, kProfAsmTri);
  const bool iso = c.A[0] == 0.0 && c.A[1] == 0.0 && c.A[2] == 0.0;
  double* conv = sys->conv ? sys->Kt + (size_t)kRec * nT : nullptr;
  auto tri_pass = sys->fp32 ? k_asm_tri<true> : k_asm_tri<false>;
  tri_pass<<<grid_for(ctx, nT), kBlock, 0, s>>>(nT, m->tri, reinterpret_cast<const double2*>(m->xy), c.a_T, c.a,
                                                iso ? 1.0 : c.A[0], iso ? 0.0 : c.A[1], iso ? 1.0 : c.A[2], c.p[0],
                                                c.p[1], sys->Kt, conv, d_bad);
  prof_stop(ctx, kProfAsmTri);
  PH_TRY(check_launch(ctx, "k_asm_tri"));
  if (sys->form == PHFEM_FORM_FLUX) {
    k_asm_flux_tri<<<grid_for(ctx, nT), kBlock, 0, s>>>(nT, m->t2e, m->sigma, m->eclass, m->elen, sys->Kt,
                                                        c.delta, f_mid, bc_mid, sys->St);
    PH_TRY(check_launch(ctx, "k_asm_flux_tri"));
    prof_start(ctx, kProfAsmRows);
    if (sys->fp32)
      k_asm_rows_flux<float><<<grid_for(ctx, nE), kBlock, 0, s>>>(nE, nT, m->ed2el, m->lk, m->eclass, sys->St,
                                                                  bc_mid, m->elen, sys->val, sys->b,
                                                                  (float*)sys->lval, (float*)sys->rdiag,
                                                                  (float*)sys->dinv);
    else
      k_asm_rows_flux<double><<<grid_for(ctx, nE), kBlock, 0, s>>>(nE, nT, m->ed2el, m->lk, m->eclass, sys->St,
                                                                   bc_mid, m->elen, sys->val, sys->b,
                                                                   (double*)sys->lval, (double*)sys->rdiag,
                                                                   (double*)sys->dinv);
    prof_stop(ctx, kProfAsmRows);
    return check_launch(ctx, "k_asm_rows_flux");
  }
  const double sK = c.dt > 0 ? 0.5 * c.dt : 1.0, sM = c.dt > 0 ? 1.0 : 0.0;
  prof_start(ctx, kProfAsmRows);
  const bool ell = c.dt == 0.0;
  auto rows = [&](auto kernel, auto* inner) {
    using T = std::remove_pointer_t<decltype(inner)>;
    kernel<<<grid_for(ctx, nE), kBlock, 0, s>>>(nE, nT, m->ed2el, m->lk, m->eclass, sys->Kt, conv, f_mid,
                                                bc_mid, m->elen, sK, sM, c.delta, sys->val, sys->b, sys->me,
                                                (T*)sys->lval, (T*)sys->rdiag, (T*)sys->dinv, m->row_tiles);
  };
  if (sys->fp32 && ell) rows(k_asm_rows<float, true>, (float*)nullptr);
  else if (!sys->fp32 && ell) rows(k_asm_rows<double, true>, (double*)nullptr);
  else if (sys->fp32) rows(k_asm_rows<float, false>, (float*)nullptr);
  else rows(k_asm_rows<double, false>, (double*)nullptr);
  prof_stop(ctx, kProfAsmRows);
  return check_launch(ctx, "k_asm_rows");
}

}  // namespace phfem

using namespace phfem;

extern "C" {

PHFEM_API int phfem_assemble(phfem_mesh mesh, const phfem_coeffs* coeffs, const double* f_mid,
                             const double* bc_mid, phfem_sys* out) {
  if (!out) return fail(PHFEM_EINVAL, "phfem_assemble: out is NULL");
  *out = nullptr;
  if (!mesh || !coeffs) return fail(PHFEM_EINVAL, "phfem_assemble: NULL argument");
  return assemble_system(mesh, *coeffs, f_mid, bc_mid, out, true);
}

}  // extern "C"

namespace phfem {

int assemble_system(phfem_mesh mesh, const phfem_coeffs& c, const double* f_mid, const double* bc_mid,
                    phfem_sys* out, bool check) {
  *out = nullptr;
  if (!(c.delta >= 0.0) || !(c.dt >= 0.0)) return fail(PHFEM_EINVAL, "phfem_assemble: delta and dt must be >= 0");
  if (!c.a_T && !(c.a > 0.0)) return fail(PHFEM_EINVAL, "phfem_assemble: coefficient a must be > 0");
  if (c.precision != PHFEM_FP64 && c.precision != PHFEM_FP32_IR)
    return fail(PHFEM_EINVAL, "phfem_assemble: unknown precision");
  if (c.delta == 0.0 && c.dt == 0.0 && mesh->info.nD == 0)
    return fail(PHFEM_EINVAL, "phfem_assemble: no Dirichlet edge and no reaction term (singular system)");
  if (c.form != PHFEM_FORM_TRACE && c.form != PHFEM_FORM_FLUX)
    return fail(PHFEM_EINVAL, "phfem_assemble: unknown form");
  if (c.form == PHFEM_FORM_FLUX && !(c.delta > 0.0))
    return fail(PHFEM_EINVAL, "phfem_assemble: the flux form needs delta > 0 (an invertible element block)");
  if (c.form == PHFEM_FORM_FLUX && c.dt != 0.0)
    return fail(PHFEM_EINVAL, "phfem_assemble: the flux form is elliptic only (dt = 0)");
  if (!std::isfinite(c.delta) || !std::isfinite(c.dt) || (!c.a_T && !std::isfinite(c.a)))
    return fail(PHFEM_ENAN, "phfem_assemble: non-finite coefficient");
  const bool iso = c.A[0] == 0.0 && c.A[1] == 0.0 && c.A[2] == 0.0;
  if (!iso && !(c.A[0] > 0.0 && c.A[2] > 0.0 && c.A[0] * c.A[2] - c.A[1] * c.A[1] > 0.0))
    return fail(PHFEM_EINVAL, "phfem_assemble: the tensor A must be symmetric positive definite");
  const bool conv = c.p[0] != 0.0 || c.p[1] != 0.0;
  if (!std::isfinite(c.p[0]) || !std::isfinite(c.p[1])) return fail(PHFEM_ENAN, "phfem_assemble: non-finite p");
  if (conv && c.form != PHFEM_FORM_TRACE)
    return fail(PHFEM_EINVAL, "phfem_assemble: convection needs the trace form");
  phfem_ctx ctx = mesh->ctx;
  cudaStream_t s = ctx->stream;
  const size_t nT = mesh->info.nT, nE = mesh->info.nE;
  phfem_sys sys = new phfem_sys_s();
  sys->mesh = mesh;
  sys->c = c;
  sys->c.a_T = nullptr;  // the pointer is only valid during this call
  sys->fp32 = c.precision == PHFEM_FP32_IR;
  sys->form = c.form;
  sys->conv = conv;
  sys->ident_class = c.form == PHFEM_FORM_FLUX ? PHFEM_EDGE_NEUMANN : PHFEM_EDGE_DIRICHLET;
  const size_t isz = sys->fp32 ? sizeof(float) : sizeof(double);
  int st = PHFEM_OK;
  int* d_bad = nullptr;
  auto chk = [&](int r) {
    if (st == PHFEM_OK) st = r;
  };
  chk(dalloc_n(ctx, &sys->Kt, (kRec + (conv ? 3 : 0)) * nT));
  chk(dalloc_n(ctx, &sys->val, 5 * nE));
  chk(dalloc_n(ctx, &sys->b, nE));
  if (c.dt > 0) chk(dalloc_n(ctx, &sys->me, nE));
  chk(dalloc(ctx, &sys->lval, 4 * nE * isz));
  chk(dalloc(ctx, &sys->rdiag, nE * isz));
  chk(dalloc(ctx, &sys->dinv, nE * isz));
  chk(dalloc_n(ctx, &sys->f, nE));
  chk(dalloc_n(ctx, &sys->bc, nE));
  if (c.form == PHFEM_FORM_FLUX) chk(dalloc_n(ctx, &sys->St, 9 * nT));
  chk(dalloc_n(ctx, &sys->x, nE));
  chk(dalloc_n(ctx, &sys->xh, nE));
  chk(dalloc_n(ctx, &sys->xl, nE));
  chk(dalloc_n(ctx, &sys->r64, nE));
  {  // r, p and q in one allocation: the iteration keeps them resident in L2 as one window
    const size_t vb = (nE * isz + 255) / 256 * 256;
    chk(dalloc(ctx, &sys->ri, 3 * vb));
    sys->pi = st == PHFEM_OK ? (void*)((char*)sys->ri + vb) : nullptr;
    sys->qi = st == PHFEM_OK ? (void*)((char*)sys->ri + 2 * vb) : nullptr;
    sys->l2_vec = vb;
  }
  chk(dalloc_n(ctx, &sys->partials, 4 * (size_t)kMaxGrid));
  chk(dalloc_n(ctx, &sys->st, 1));
  chk(dalloc_n(ctx, &d_bad, 1));
  sys->st_host = ctx->st_pinned;
  if (st == PHFEM_OK) {
    cudaMemsetAsync(sys->st, 0, sizeof(SolveState), s);
    cudaMemsetAsync(d_bad, 0, sizeof(int), s);
    if (f_mid) cudaMemcpyAsync(sys->f, f_mid, nE * sizeof(double), cudaMemcpyDeviceToDevice, s);
    else cudaMemsetAsync(sys->f, 0, nE * sizeof(double), s);
    if (bc_mid) cudaMemcpyAsync(sys->bc, bc_mid, nE * sizeof(double), cudaMemcpyDeviceToDevice, s);
    else cudaMemsetAsync(sys->bc, 0, nE * sizeof(double), s);
    sys->c.a_T = c.a_T;
    st = assemble_into(sys, f_mid, bc_mid, d_bad);
    sys->c.a_T = nullptr;
  }
  if (st == PHFEM_OK && check) {
    int bad = 0;
    cudaError_t e = cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_fail(e, "phfem_assemble", __FILE__, __LINE__);
    else if (bad & 2) st = fail(PHFEM_ENAN, "phfem_assemble: non-finite coefficient a_T");
    else if (bad & 1) st = fail(PHFEM_EINVAL, "phfem_assemble: coefficient a_T must be > 0");
  }
  dfree(ctx, d_bad);
  if (st != PHFEM_OK) {
    cudaStreamSynchronize(s);
    sys_free(sys);
    return st;
  }
  *out = sys;
  return PHFEM_OK;
}

}  // namespace phfem

extern "C" {

PHFEM_API int phfem_sys_csr(phfem_sys sys, double* val, double* rhs) {
  if (!sys) return fail(PHFEM_EINVAL, "phfem_sys_csr: NULL system");
  if (sys->form != PHFEM_FORM_TRACE) return fail(PHFEM_EINVAL, "phfem_sys_csr: only the trace form has a CSR export");
  phfem_mesh m = sys->mesh;
  phfem_ctx ctx = m->ctx;
  const int nE = m->info.nE;
  k_export<<<grid_for(ctx, nE), kBlock, 0, ctx->stream>>>(nE, m->nbr, m->free_id, m->eclass, m->row_ptr, sys->val,
                                                          sys->b, val, rhs);
  return check_launch(ctx, "k_export");
}

PHFEM_API int phfem_sys_destroy(phfem_sys sys) {
  if (!sys) return fail(PHFEM_EINVAL, "phfem_sys_destroy: NULL system");
  sys_free(sys);
  return PHFEM_OK;
}

}  // extern "C"
