// Per-triangle and per-edge arithmetic shared by the grid-wide kernels and the
// batched (one block per mesh) kernels, so both compute bitwise the same
// values.  See assemble.cu for the derivation of the condensed blocks.
#pragma once

#include "internal.cuh"

namespace phfem {

// The helpers take plain pointers (no __restrict__, which would let the
// compiler choose non-coherent loads by itself); the grid kernels pass RO = true.
// Loads through the read-only (non-coherent) path are only valid for data that
// no thread writes during the kernel: the grid-wide kernels use them, the
// persistent batch kernel (which writes Kt and p and reads them back after a
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

// K^CR_T = (a/|T|) e_k' A~ e_j + delta |T|/3 I for the triangle (p0, p1, p2),
// e_k = P_{k+2} - P_{k+1}, A~ = [[A22, -A12], [-A12, A11]] (since |T| grad
// lambda_k = the edge vector e_k turned by a right angle, over 2): out[0..2]
// diagonal, out[3] (0,1), out[4] (1,2), out[5] (2,0), out[6] = |T|/3.
__device__ __forceinline__ void tri_block(double2 p0, double2 p1, double2 p2, double a, double delta,
                                          double out[7], double A11 = 1.0, double A12 = 0.0, double A22 = 1.0) {
  const double e0x = p2.x - p1.x, e0y = p2.y - p1.y;
  const double e1x = p0.x - p2.x, e1y = p0.y - p2.y;
  const double e2x = p1.x - p0.x, e2y = p1.y - p0.y;
  const double area2 = e1x * e2y - e1y * e2x;  // 2|T| = cross(P1 - P0, P2 - P0)
  const double mT = area2 * (1.0 / 6.0);       // |T|/3
  const double c = (a + a) / area2;            // a / |T|
  const double dm = delta * mT;
  if (A11 == 1.0 && A12 == 0.0 && A22 == 1.0) {  // A = I (uniform across a launch)
    out[0] = c * (e0x * e0x + e0y * e0y) + dm;
    out[1] = c * (e1x * e1x + e1y * e1y) + dm;
    out[2] = c * (e2x * e2x + e2y * e2y) + dm;
    out[3] = c * (e0x * e1x + e0y * e1y);
    out[4] = c * (e1x * e2x + e1y * e2y);
    out[5] = c * (e2x * e0x + e2y * e0y);
  } else {
    auto q = [&](double ux, double uy, double vx, double vy) {
      return A22 * ux * vx - A12 * (ux * vy + uy * vx) + A11 * uy * vy;
    };
    out[0] = c * q(e0x, e0y, e0x, e0y) + dm;
    out[1] = c * q(e1x, e1y, e1x, e1y) + dm;
    out[2] = c * q(e2x, e2y, e2x, e2y) + dm;
    out[3] = c * q(e0x, e0y, e1x, e1y);
    out[4] = c * q(e1x, e1y, e2x, e2y);
    out[5] = c * q(e2x, e2y, e0x, e0y);
  }
  out[6] = mT;
}

// Convection in the trace form: R^-T D_T R^-1 with the column-constant
// (D_T)_{rc} = |T|/3 p.grad(lambda_c) is column-constant as well,
// -2|T|/3 p.grad(lambda_j) = (p_x e_jy - p_y e_jx) / 3 in column j (rows sum to 0).
__device__ __forceinline__ void tri_conv(double2 p0, double2 p1, double2 p2, double px, double py, double out[3]) {
  out[0] = (px * (p2.y - p1.y) - py * (p2.x - p1.x)) * (1.0 / 3.0);
  out[1] = (px * (p0.y - p2.y) - py * (p0.x - p2.x)) * (1.0 / 3.0);
  out[2] = (px * (p1.y - p0.y) - py * (p1.x - p0.x)) * (1.0 / 3.0);
}

// Entries of row k of K^CR_T stored slot-major with stride n: diagonal,
// (k, k+1), (k, k+2), and |T|/3.
template <bool RO = true>
__device__ __forceinline__ void tri_row(const double* Kt, size_t n, int t, int k, double& d,
                                        double& o1, double& o2, double& mT) {
  const int k2 = (k == 0) ? 2 : k - 1;  // k + 2 mod 3
  d = ld<RO>(Kt + (size_t)k * n + t);
  o1 = ld<RO>(Kt + (size_t)(3 + k) * n + t);   // pair (k, k+1)
  o2 = ld<RO>(Kt + (size_t)(3 + k2) * n + t);  // pair (k+2, k)
  mT = ld<RO>(Kt + 6 * n + t);
}

struct EdgeRow {
  double rpart;   // reaction/mass part of the diagonal (difference form)
  double l[4];    // -S_{e, nbr_s}
  double diag;    // S_ee
  double rhs;
  double mass;    // sum of |T|/3 over the owners
};

// Row of edge e from the element blocks of T+ (tp, local kp) and T- (tm, km;
// tm < 0 on the boundary); sK scales K^CR and sM the mass (elliptic 1, 0;
// Crank-Nicolson dt/2, 1).  Dirichlet rows are identity rows holding u_D.
// ELLIPTIC: sK = 1 and sM = 0 (no scaling products).
template <bool RO = true, bool ELLIPTIC = false>
__device__ __forceinline__ EdgeRow edge_row(const double* Kt, size_t n, int tp, int kp, int tm,
                                            int km, uint8_t cls, double f, double bc, double elen, double sK,
                                            double sM, double delta, bool have_f, bool have_bc) {
  EdgeRow R;
  double d, o1, o2, mT;
  tri_row<RO>(Kt, n, tp, kp, d, o1, o2, mT);
  double diag, v1, v2, v3 = 0.0, v4 = 0.0, mass = mT;
  if (ELLIPTIC) {
    diag = d;
    v1 = o1;
    v2 = o2;
  } else {
    diag = sK * d + sM * mT;
    v1 = sK * o1;
    v2 = sK * o2;
  }
  if (tm >= 0) {
    tri_row<RO>(Kt, n, tm, km, d, o1, o2, mT);
    if (ELLIPTIC) {
      diag += d;
      v3 = o1;
      v4 = o2;
    } else {
      diag += sK * d + sM * mT;
      v3 = sK * o1;
      v4 = sK * o2;
    }
    mass += mT;
  }
  double rhs, rpart;
  if (cls == PHFEM_EDGE_DIRICHLET) {
    diag = 1.0;
    v1 = v2 = v3 = v4 = 0.0;
    rhs = have_bc ? bc : 0.0;
    rpart = 1.0;
  } else {
    rhs = have_f ? mass * f : 0.0;
    if (cls == PHFEM_EDGE_NEUMANN && have_bc) rhs += elen * bc;
    rpart = ELLIPTIC ? delta * mass : (sK * delta + sM) * mass;
  }
  R.rpart = rpart;
  R.l[0] = -v1;
  R.l[1] = -v2;
  R.l[2] = -v3;
  R.l[3] = -v4;
  R.diag = diag;
  R.rhs = rhs;
  R.mass = mass;
  return R;
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

// b_e - (S x)_e in FP64 difference form, and the row's |S| |x| (the scale of
// the rounding of x to FP64).
__device__ __forceinline__ double residual_row(const int32_t* nbr, const double* val,
                                               const double* b, const double* x, size_t m,
                                               int e, double& absrow) {
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

}  // namespace phfem
