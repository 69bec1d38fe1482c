// Per-triangle and per-edge arithmetic shared by the grid-wide kernels and the
// batched (one block per mesh) kernels.  FP64 systems compute bitwise the same
// values on both; FP32 systems take compensated FP32 element records on the
// grid and FP64 ones in the batch (within a few 1e-14 of each other).  See
// assemble.cu for the derivation of the condensed blocks.
#pragma once

#include "c32.cuh"
#include "internal.cuh"

namespace phfem {

// The helpers take plain pointers (no __restrict__, which would let the
// compiler choose non-coherent loads by itself); the grid kernels pass RO = true.
// Loads through the read-only (non-coherent) path are only valid for data that
// no thread writes during the kernel: the grid-wide kernels use them, the
// persistent batch kernel (which writes the records and p and reads them back after a
// block barrier) must use coherent loads.
template <bool RO, typename T>
__device__ __forceinline__ T ld(const T* ptr) {
  if constexpr (RO) return __ldg(ptr);
  else return *ptr;
}

// Programmatic dependent launch: iteration kernels are launched so that their
// blocks may be scheduled while the previous kernel drains; each waits for the
// previous grid to complete (and its writes to be visible) before it reads
// anything, and lets the next kernel be scheduled at once.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// An L2 access-policy window: accesses inside [base, base + bytes) persist in
// the L2 set-aside (with probability hit_ratio), others stream.  bytes == 0: none.
struct L2Window {
  void* base = nullptr;
  size_t bytes = 0;
  float hit_ratio = 0.f;
};

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl_w(const L2Window& w, void (*kernel)(KArgs...), int grid, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kBlock);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  int na = 1;
  if (w.bytes > 0) {
    attr[1].id = cudaLaunchAttributeAccessPolicyWindow;
    attr[1].val.accessPolicyWindow.base_ptr = w.base;
    attr[1].val.accessPolicyWindow.num_bytes = w.bytes;
    attr[1].val.accessPolicyWindow.hitRatio = w.hit_ratio;
    attr[1].val.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
    attr[1].val.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
    na = 2;
  }
  cfg.attrs = attr;
  cfg.numAttrs = na;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), int grid, cudaStream_t s, Args... args) {
  return launch_pdl_w(L2Window{}, kernel, grid, s, args...);
}

// Decision after a true residual (the last block of a residual kernel, thread
// 0): the iteration's state, convergence (rtol, or twice the estimated floor
// of the residual's evaluation), and for a reliable update the line-search
// step along the kept direction or a restart of the direction.
// mode 1 = start, 2 = reliable update.
// y += alpha p with alpha = ah + al (FP32 systems): the product as an exact
// pair plus al p, added to the pair y by TwoSum; FP32 arithmetic only.  The
// solution correction between reliable updates is accumulated this way
// (about 48 bits) instead of in FP64, whose rate on GB300 is ~1/64 of FP32's.
__device__ __forceinline__ float2 y_add(float2 y, float ah, float al, float p) {
  const c32::f2 pr = c32::two_prod(ah, p);
  const float pe = c32::ffma(al, p, pr.l);
  const c32::f2 s = c32::two_sum(y.x, pr.h);
  const float t = c32::fadd(c32::fadd(s.l, y.y), pe);
  const float hi = c32::fadd(s.h, t);
  return make_float2(hi, c32::fsub(t, c32::fsub(hi, s.h)));
}
__device__ __forceinline__ double y_add(double y, double a, double, double p) { return fma(a, p, y); }

// The value of the recursive r.z at which the next reliable update is taken:
// a fall by the update factor, or, when that comes sooner, the point where
// the true residual is predicted to meet the tolerance, r.r being taken to
// fall in proportion to r.z from the true residual just evaluated, aiming at
// 0.8 of the tolerance in the squares.  Without the second bound a solve whose
// true residual lands just above the tolerance iterates a further update
// factor; a prediction that falls short costs one more reliable update.
__device__ __forceinline__ double update_target(double rz, double rr, double bb, double rtol2, double inner_rtol2) {
  const double reach = rr > 0.0 ? 0.8 * rtol2 * bb / rr : 0.0;
  return rz * fmax(inner_rtol2, fmin(reach, 1.0));
}

__device__ inline void decide(SolveState* st, double rr, double rz, double ff, double rp, int mode, double rtol2,
                              double inner_rtol2) {
  const double rz_recursive = st->rz;
  st->rr64 = rr;
  st->floor2 = ff;
  st->rz = rz;
  st->rp = rp;
  st->tol2 = update_target(rz, rr, st->bb, rtol2, inner_rtol2);
  st->status = 0;
  if (mode == 1) {
    st->rz0 = rz;
    st->it = 0;
    st->updates = 1;
    st->bodies = 0;
    st->use_rp = 0;
    st->restart = 0;
  } else {
    st->updates += 1;
    // line search along the kept direction, or restart it when it no longer
    // fits the replaced residual
    const int restart = (rz > 4.0 * rz_recursive) || !(rp > 0.0);
    st->restart = restart;
    st->use_rp = !restart;
  }
  st->conv = 0;
  if (!isfinite(rr) || !isfinite(rz)) {
    st->done = 3;
    st->status = PHFEM_ENAN;
  } else if (rr <= rtol2 * st->bb || rr == 0.0) {
    st->done = 2;
    st->conv = 1;
  } else if (rr <= 4.0 * ff) {  // relative residual within twice the estimated floor
    st->done = 2;
    st->conv = 2;
  } else {
    st->done = 0;
  }
}

// Per-triangle record of the trace-form block K^CR_T = (a/|T|) e_i' A~ e_j +
// delta |T|/3 I, e_k = P_{k+2} - P_{k+1}, A~ = [[A22, -A12], [-A12, A11]]
// (|T| grad lambda_k is the edge vector e_k turned by a right angle, over 2).
// The stiffness rows sum to zero (e_0 + e_1 + e_2 = 0, for any A), so the
// block is fixed by its off-diagonal entries and |T|/3; the record holds
//   L01, L12, L20 = -K^CR_T off the diagonal, and |T|/3
// as four doubles (32 bytes, one sector, AoS), so an edge row reads one
// sector per owner triangle.  The diagonal is
// K_kk = L_{k,k+1} + L_{k+2,k} + delta |T|/3.
constexpr int kRec = 4;

// FP64 record of the triangle (p0, p1, p2).
__device__ __forceinline__ void tri_record64(double2 p0, double2 p1, double2 p2, double a, double out[4],
                                             double A11 = 1.0, double A12 = 0.0, double A22 = 1.0) {
  const double e0x = p2.x - p1.x, e0y = p2.y - p1.y;
  const double e1x = p0.x - p2.x, e1y = p0.y - p2.y;
  const double e2x = p1.x - p0.x, e2y = p1.y - p0.y;
  const double area2 = e1x * e2y - e1y * e2x;  // 2|T| = cross(P1 - P0, P2 - P0)
  const double nc = -(a + a) / area2;          // -a / |T|
  if (A11 == 1.0 && A12 == 0.0 && A22 == 1.0) {  // A = I (uniform across a launch)
    out[0] = nc * (e0x * e1x + e0y * e1y);
    out[1] = nc * (e1x * e2x + e1y * e2y);
    out[2] = nc * (e2x * e0x + e2y * e0y);
  } else {
    auto q = [&](double ux, double uy, double vx, double vy) {
      return A22 * ux * vx - A12 * (ux * vy + uy * vx) + A11 * uy * vy;
    };
    out[0] = nc * q(e0x, e0y, e1x, e1y);
    out[1] = nc * q(e1x, e1y, e2x, e2y);
    out[2] = nc * q(e2x, e2y, e0x, e0y);
  }
  out[3] = area2 * (1.0 / 6.0);
}

// Stores a record (two 16-byte stores; records are 32-byte aligned).
__device__ __forceinline__ void store_record(double* dst, const double R[4]) {
  double2* p = reinterpret_cast<double2*>(dst);
  p[0] = make_double2(R[0], R[1]);
  p[1] = make_double2(R[2], R[3]);
}

// The FP64 record computed and stored out of line: inlined next to the
// compensated path, the compiler evaluates part of it (the edge vectors are
// shared) ahead of that path's outcome.
static __device__ __noinline__ void tri_record64_store(double2 p0, double2 p1, double2 p2, double a, double* dst, double A11,
                                                double A12, double A22) {
  double R[4];
  tri_record64(p0, p1, p2, a, R, A11, A12, A22);
  store_record(dst, R);
}

// Record of an FP32 system, stored at dst: compensated FP32 for the isotropic
// case (within a few 1e-14 of the row scale), FP64 for triangles outside its
// range or shape bound and for a tensor A.
__device__ __forceinline__ void tri_record32_store(double2 p0, double2 p1, double2 p2, double a, double* dst, bool iso,
                                                   double A11 = 1.0, double A12 = 0.0, double A22 = 1.0) {
  double R[4];
  if (iso && c32::tri_record(p0.x, p0.y, p1.x, p1.y, p2.x, p2.y, a, R)) store_record(dst, R);
  else tri_record64_store(p0, p1, p2, a, dst, A11, A12, A22);
}

template <bool RO>
__device__ __forceinline__ void load_record(const double* rec, int t, double r[4]) {
  const double2* p = reinterpret_cast<const double2*>(rec + (size_t)kRec * t);
  const double2 a = ld<RO>(p), b = ld<RO>(p + 1);
  r[0] = a.x;
  r[1] = a.y;
  r[2] = b.x;
  r[3] = b.y;
}

// The full block of a record: K[0..2] diagonal, K[3] (0,1), K[4] (1,2),
// K[5] (2,0).
__device__ __forceinline__ void record_block(const double r[4], double delta, double K[6]) {
  const double dm = delta * r[3];
  K[0] = r[0] + r[2] + dm;
  K[1] = r[0] + r[1] + dm;
  K[2] = r[1] + r[2] + dm;
  K[3] = -r[0];
  K[4] = -r[1];
  K[5] = -r[2];
}

// (K^CR_T w)_k - the stiffness part in difference form,
// sum_{j != k} L_kj (w_k - w_j), plus delta |T|/3 w_k.
__device__ __forceinline__ void record_apply(const double r[4], double delta, double w0, double w1, double w2,
                                             double out[3]) {
  const double dm = delta * r[3];
  out[0] = r[0] * (w0 - w1) + r[2] * (w0 - w2) + dm * w0;
  out[1] = r[0] * (w1 - w0) + r[1] * (w1 - w2) + dm * w1;
  out[2] = r[1] * (w2 - w1) + r[2] * (w2 - w0) + dm * w2;
}

// Convection in the trace form: R^-T D_T R^-1 with the column-constant
// (D_T)_{rc} = |T|/3 p.grad(lambda_c) is column-constant as well,
// -2|T|/3 p.grad(lambda_j) = (p_x e_jy - p_y e_jx) / 3 in column j (rows sum to 0).
__device__ __forceinline__ void tri_conv(double2 p0, double2 p1, double2 p2, double px, double py, double out[3]) {
  out[0] = (px * (p2.y - p1.y) - py * (p2.x - p1.x)) * (1.0 / 3.0);
  out[1] = (px * (p0.y - p2.y) - py * (p0.x - p2.x)) * (1.0 / 3.0);
  out[2] = (px * (p1.y - p0.y) - py * (p1.x - p0.x)) * (1.0 / 3.0);
}

struct EdgeRow {
  double rpart;   // reaction/mass part of the diagonal (difference form)
  double l[4];    // -S_{e, nbr_s}
  double diag;    // S_ee
  double rhs;
  double mass;    // sum of |T|/3 over the owners
};

// Row of edge e from the records of T+ (tp, local kp) and T- (tm, km;
// tm < 0 on the boundary); sK scales K^CR and sM the mass (elliptic 1, 0;
// Crank-Nicolson dt/2, 1).  Dirichlet rows are identity rows holding u_D.
// The diagonal is rpart + sum of l.  ELLIPTIC: sK = 1 and sM = 0 (no
// scaling products).
// Row k of the record of triangle t: L_{k,k+1}, L_{k+2,k} and |T|/3, three
// loads from the record's one sector.
template <bool RO>
__device__ __forceinline__ void record_row(const double* rec, int t, int k, double& o1, double& o2, double& mT) {
  const double* r = rec + (size_t)kRec * t;
  o1 = ld<RO>(r + k);
  o2 = ld<RO>(r + (k == 0 ? 2 : k - 1));
  mT = ld<RO>(r + 3);
}

template <bool RO = true, bool ELLIPTIC = false>
__device__ __forceinline__ EdgeRow edge_row(const double* rec, int tp, int kp, int tm, int km, uint8_t cls,
                                            double f, double bc, double elen, double sK, double sM, double delta,
                                            bool have_f, bool have_bc) {
  EdgeRow R;
  double v1, v2, v3 = 0.0, v4 = 0.0, mass, m2;
  record_row<RO>(rec, tp, kp, v1, v2, mass);
  if (tm >= 0) {
    record_row<RO>(rec, tm, km, v3, v4, m2);
    mass += m2;
  }
  if (!ELLIPTIC) {
    v1 *= sK;
    v2 *= sK;
    v3 *= sK;
    v4 *= sK;
  }
  double rhs, rpart;
  if (cls == PHFEM_EDGE_DIRICHLET) {
    v1 = v2 = v3 = v4 = 0.0;
    rhs = have_bc ? bc : 0.0;
    rpart = 1.0;
  } else {
    rhs = have_f ? mass * f : 0.0;
    if (cls == PHFEM_EDGE_NEUMANN && have_bc) rhs += elen * bc;
    rpart = ELLIPTIC ? delta * mass : (sK * delta + sM) * mass;
  }
  R.rpart = rpart;
  R.l[0] = v1;
  R.l[1] = v2;
  R.l[2] = v3;
  R.l[3] = v4;
  R.diag = rpart + v1 + v2 + v3 + v4;
  R.rhs = rhs;
  R.mass = mass;
  return R;
}

// Inner-precision values of a row: the FP64 ones rounded to floats (integer
// operations, no conversion instructions) and the Jacobi inverse of their
// diagonal in FP32 arithmetic; float or double lval, rdiag, dinv.
template <typename T>
__device__ __forceinline__ void store_inner(const EdgeRow& R, size_t m, int e, T* lval, T* rdiag, T* dinv) {
  if constexpr (sizeof(T) == sizeof(float)) {
    float d = c32::narrow(R.rpart);
    rdiag[e] = d;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const float l = c32::narrow(R.l[s]);
      lval[s * m + e] = l;
      d += l;
    }
    dinv[e] = c32::frcp(d);  // to 2^-24; a Jacobi scaling needs no correct rounding
  } else {
#pragma unroll
    for (int s = 0; s < 4; ++s) lval[s * m + e] = R.l[s];
    rdiag[e] = R.rpart;
    dinv[e] = 1.0 / R.diag;
  }
}

// (S p)_e in difference form: rdiag_e p_e + sum_s l_es (p_e - p_s).
template <typename T, bool RO = true>
__device__ __forceinline__ T spmv_row(const int32_t* nbr, const T* lval,
                                      const T* rdiag, const T* p, size_t m, int e) {
  const int c0 = nbr[e], c1 = nbr[m + e], c2 = nbr[2 * m + e], c3 = nbr[3 * m + e];
  const T l0 = lval[e], l1 = lval[m + e], l2 = lval[2 * m + e], l3 = lval[3 * m + e];
  const T pe = p[e];
  T s = rdiag[e] * pe;
  s += l0 * (pe - ld<RO>(p + c0));
  s += l1 * (pe - ld<RO>(p + c1));
  s += l2 * (pe - ld<RO>(p + c2));
  s += l3 * (pe - ld<RO>(p + c3));
  return s;
}

// b_e - (S x)_e in FP64 difference form with x = xh + xl (an unevaluated
// FP64 pair): each difference x_e - x_s is formed from the pairs with TwoSum
// on the leading parts, so the row's own rounding is about 2^-53 of
// |rho x_e| + sum_s |l_es (x_e - x_s)|, returned in absrow (the evaluation
// floor).
__device__ __forceinline__ double residual_row(const int32_t* nbr, const double* val, const double* b,
                                               const double* xh, const double* xl, size_t m, int e,
                                               double& absrow) {
  const double he = xh[e], le = xl[e];
  const double rho = val[e];
  double sx = rho * he + rho * le;
  double fl = fabs(rho * he);
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const double l = val[(s + 1) * m + e];
    const int c = nbr[s * m + e];
    const double nh = -xh[c];
    const double sh = he + nh;
    const double bb = sh - he;
    const double eh = (he - (sh - bb)) + (nh - bb);
    const double d = sh + (eh + (le - xl[c]));
    sx += l * d;
    fl += fabs(l * d);
  }
  absrow = fl;
  return b[e] - sx;
}

// The same with x in plain FP64 (the batched kernel), absrow the scale of
// the FP64 rounding of x: sum |S_es| |x_s| over the row.
__device__ __forceinline__ double residual_row(const int32_t* nbr, const double* val, const double* b,
                                               const double* x, size_t m, int e, double& absrow) {
  const double xe = x[e];
  double sx = val[e] * xe;
  double fl = fabs(val[e] * xe);
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const double l = val[(s + 1) * m + e], xs = x[nbr[s * m + e]];
    sx += l * (xe - xs);
    fl += fabs(l) * (fabs(xe) + fabs(xs));
  }
  absrow = fl;
  return b[e] - sx;
}

// (h, l) += v in FP64: TwoSum of the leading parts, then renormalised.
__device__ __forceinline__ void dd_add(double& h, double& l, double v) {
  const double s = h + v;
  const double bb = s - h;
  const double e = (h - (s - bb)) + (v - bb);
  const double t = e + l;
  h = s + t;
  l = t - (h - s);
}

}  // namespace phfem
