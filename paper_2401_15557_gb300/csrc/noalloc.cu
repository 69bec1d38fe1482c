// Jacobi-PCG on a caller-given CSR system without any device allocation.
//
// Some callers cannot allocate device memory while they call into this
// library: programs whose device memory is owned by another framework's pool
// or a fixed arena (an allocation outside it goes uncounted or fails), and
// loops with a latency or memory budget, where cudaMalloc may synchronise the
// device or fail under memory pressure in the middle of a run.  This entry
// point serves them: every temporary lives in one file-scope device array of
// fixed size, which every device that loads the library holds until the
// process exits.  The caller still passes the matrix, the right-hand side and
// the solution buffer.
//
// Limits and sharing rules:
//   * at most PHFEM_NOALLOC_MAX_ROWS rows (larger systems are rejected);
//   * the scratch array is shared by every call on a device and keeps the
//     contents of the last call; the state words that must start at zero are
//     cleared (cudaMemsetAsync) at the start of each call;
//   * calls whose work overlaps on the GPU (different streams, or host
//     threads, without ordering between them) race on the scratch array;
//   * the first call on a device looks up the array's device address with
//     cudaGetSymbolAddress while that device is current;
//   * the reported relative residual is that of the recursive residual the
//     iteration updates, not one recomputed from x;
//   * the call returns when the solve has finished: every 32 iterations it
//     copies the state to the host and waits for the stream.
#include <cmath>
#include <cstring>
#include <mutex>

#include "internal.cuh"

namespace phfem {
namespace {

constexpr int kNaBlock = 256;
constexpr int kNaMaxGrid = 152 * 8;

struct NaState {
  double rz, rr, bb, alpha, beta, tol2;
  int it, done, status, dir_pending;
  unsigned int counter[4];
};

// Layout: 4 vectors of PHFEM_NOALLOC_MAX_ROWS doubles (r, p, q, 1/diag),
// 3 partial arrays of kNaMaxGrid doubles, then the state.
constexpr size_t kNaVec = (size_t)PHFEM_NOALLOC_MAX_ROWS;
constexpr size_t kNaDoubles = 4 * kNaVec + 3 * (size_t)kNaMaxGrid;
constexpr size_t kNaBytes = kNaDoubles * sizeof(double) + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

struct Scratch {
  double* r;
  double* p;
  double* q;
  double* dinv;
  double* partials;
  NaState* st;
};

__device__ __forceinline__ double na_block_sum(double v, double* smem) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) smem[w] = v;
  __syncthreads();
  v = 0.0;
  if (w == 0) {
    v = (lane < kNaBlock / 32) ? smem[lane] : 0.0;
    v = warp_sum(v);
  }
  __syncthreads();
  return v;
}

__device__ __forceinline__ double na_sum_partials(const double* partials, double* smem) {
  double v = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) v += __ldcg(partials + i);
  return na_block_sum(v, smem);
}

// r = b - A x, 1/diag, p = D^-1 r; reductions ||b||^2, ||r||^2, r.D^-1 r
__global__ void k_na_init(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                          const double* __restrict__ val, const double* __restrict__ b, const double* __restrict__ x,
                          Scratch sc, double rtol2) {
  __shared__ double smem[kNaBlock / 32];
  double ab = 0.0, ar = 0.0, az = 0.0;
  int bad = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double ax = 0.0, d = 0.0;
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
      const int c = col[k];
      ax += val[k] * x[c];
      if (c == i) d = val[k];
    }
    if (!(d > 0.0)) bad = 1;
    const double di = d > 0.0 ? 1.0 / d : 0.0;
    const double r = b[i] - ax;
    sc.r[i] = r;
    sc.dinv[i] = di;
    sc.p[i] = di * r;
    ab += b[i] * b[i];
    ar += r * r;
    az += r * di * r;
  }
  if (bad) atomicOr(&sc.st->status, 1);
  ab = na_block_sum(ab, smem);
  ar = na_block_sum(ar, smem);
  az = na_block_sum(az, smem);
  if (threadIdx.x == 0) {
    sc.partials[blockIdx.x] = ab;
    sc.partials[kNaMaxGrid + blockIdx.x] = ar;
    sc.partials[2 * kNaMaxGrid + blockIdx.x] = az;
  }
  if (!arrive_last(&sc.st->counter[0])) return;
  const double bb = na_sum_partials(sc.partials, smem);
  const double rr = na_sum_partials(sc.partials + kNaMaxGrid, smem);
  const double rz = na_sum_partials(sc.partials + 2 * kNaMaxGrid, smem);
  if (threadIdx.x == 0) {
    sc.st->counter[0] = 0;
    sc.st->bb = bb;
    sc.st->rr = rr;
    sc.st->rz = rz;
    sc.st->tol2 = rtol2 * bb;
    if (sc.st->status) {
      sc.st->done = 3;
      sc.st->status = PHFEM_EINVAL;
    } else if (!isfinite(rr) || !isfinite(rz)) {
      sc.st->done = 3;
      sc.st->status = PHFEM_ENAN;
    } else if (rr <= rtol2 * bb) {
      sc.st->done = 1;
    }
  }
}

__global__ void k_na_spmv(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                          const double* __restrict__ val, Scratch sc) {
  if (blockIdx.x == 0 && threadIdx.x == 0) sc.st->dir_pending = 0;
  if (sc.st->done) return;
  __shared__ double smem[kNaBlock / 32];
  double acc = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int k = rp[i]; k < rp[i + 1]; ++k) s += val[k] * sc.p[col[k]];
    sc.q[i] = s;
    acc += sc.p[i] * s;
  }
  acc = na_block_sum(acc, smem);
  if (threadIdx.x == 0) sc.partials[blockIdx.x] = acc;
  if (!arrive_last(&sc.st->counter[1])) return;
  const double pq = na_sum_partials(sc.partials, smem);
  if (threadIdx.x == 0) {
    sc.st->counter[1] = 0;
    if (!(pq > 0.0) || !isfinite(pq)) {
      sc.st->done = 3;
      sc.st->status = isfinite(pq) ? PHFEM_EBREAKDOWN : PHFEM_ENAN;
    } else {
      sc.st->alpha = sc.st->rz / pq;
    }
  }
}

__global__ void k_na_update(int n, double* __restrict__ x, Scratch sc) {
  if (sc.st->done) return;
  __shared__ double smem[kNaBlock / 32];
  const double alpha = sc.st->alpha;
  double ar = 0.0, az = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    x[i] += alpha * sc.p[i];
    const double r = sc.r[i] - alpha * sc.q[i];
    sc.r[i] = r;
    ar += r * r;
    az += r * sc.dinv[i] * r;
  }
  ar = na_block_sum(ar, smem);
  az = na_block_sum(az, smem);
  if (threadIdx.x == 0) {
    sc.partials[kNaMaxGrid + blockIdx.x] = ar;
    sc.partials[2 * kNaMaxGrid + blockIdx.x] = az;
  }
  if (!arrive_last(&sc.st->counter[2])) return;
  const double rr = na_sum_partials(sc.partials + kNaMaxGrid, smem);
  const double rz = na_sum_partials(sc.partials + 2 * kNaMaxGrid, smem);
  if (threadIdx.x == 0) {
    sc.st->counter[2] = 0;
    sc.st->beta = rz / sc.st->rz;
    sc.st->rz = rz;
    sc.st->rr = rr;
    sc.st->it += 1;
    sc.st->dir_pending = 1;
    if (!isfinite(rr)) {
      sc.st->done = 3;
      sc.st->status = PHFEM_ENAN;
    }
  }
}

__global__ void k_na_dir(int n, Scratch sc) {
  if (!sc.st->dir_pending) return;
  const double beta = sc.st->beta;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    sc.p[i] = sc.dinv[i] * sc.r[i] + beta * sc.p[i];
  if (blockIdx.x == 0 && threadIdx.x == 0 && sc.st->done == 0 && sc.st->rr <= sc.st->tol2) sc.st->done = 1;
}

// Per-device address of the scratch array (looked up once per device).
std::mutex g_na_mutex;
void* g_na_ptr[64] = {nullptr};

int noalloc_scratch(int dev, unsigned char** out) {
  if (dev < 0 || dev >= 64) return fail(PHFEM_EINVAL, "phfem_csr_pcg_noalloc: device index out of range");
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)", __FILE__, __LINE__);
    g_na_ptr[dev] = p;
  }
  *out = (unsigned char*)g_na_ptr[dev];
  return PHFEM_OK;
}

}  // namespace
}  // namespace phfem

using namespace phfem;

extern "C" {

PHFEM_API int phfem_csr_pcg_noalloc(void* cuda_stream, int32_t n, const int32_t* row_ptr, const int32_t* col,
                                    const double* val, const double* rhs, double* x, double rtol, int32_t max_iter,
                                    int32_t* iterations, double* rel_residual) {
  if (n < 1 || !row_ptr || !col || !val || !rhs || !x)
    return fail(PHFEM_EINVAL, "phfem_csr_pcg_noalloc: empty system or NULL array");
  if (n > PHFEM_NOALLOC_MAX_ROWS)
    return fail(PHFEM_EINVAL, "phfem_csr_pcg_noalloc: " + std::to_string(n) + " rows exceed the fixed scratch of " +
                                  std::to_string(PHFEM_NOALLOC_MAX_ROWS) + " rows; use phfem_solve");
  if (!(rtol > 0.0)) rtol = 1e-10;
  if (max_iter <= 0) max_iter = 100000;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int dev = 0;
  PH_CUDA(cudaGetDevice(&dev));
  unsigned char* base = nullptr;
  PH_TRY(noalloc_scratch(dev, &base));
  Scratch sc;
  double* d = (double*)base;
  sc.r = d;
  sc.p = d + kNaVec;
  sc.q = d + 2 * kNaVec;
  sc.dinv = d + 3 * kNaVec;
  sc.partials = d + 4 * kNaVec;
  sc.st = (NaState*)(d + kNaDoubles);
  int sms = 0;
  PH_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  int grid = (n + kNaBlock - 1) / kNaBlock;
  if (grid > sms * 8) grid = sms * 8;
  if (grid > kNaMaxGrid) grid = kNaMaxGrid;
  // the previous call's state must not leak into this one
  PH_CUDA(cudaMemsetAsync(sc.st, 0, sizeof(NaState), s));
  k_na_init<<<grid, kNaBlock, 0, s>>>(n, row_ptr, col, val, rhs, x, sc, rtol * rtol);
  PH_CUDA(cudaGetLastError());
  NaState h;
  int it = 0;
  for (;;) {
    PH_CUDA(cudaMemcpyAsync(&h, sc.st, sizeof(h), cudaMemcpyDeviceToHost, s));
    PH_CUDA(cudaStreamSynchronize(s));
    it = h.it;
    if (h.done || it >= max_iter) break;
    const int chunk = (max_iter - it) < 32 ? (max_iter - it) : 32;
    for (int k = 0; k < chunk; ++k) {
      k_na_spmv<<<grid, kNaBlock, 0, s>>>(n, row_ptr, col, val, sc);
      k_na_update<<<grid, kNaBlock, 0, s>>>(n, x, sc);
      k_na_dir<<<grid, kNaBlock, 0, s>>>(n, sc);
    }
    PH_CUDA(cudaGetLastError());
  }
  const double rel = h.bb > 0 ? std::sqrt(h.rr / h.bb) : 0.0;
  if (iterations) *iterations = it;
  if (rel_residual) *rel_residual = rel;
  if (h.done == 3) {
    return fail(h.status, h.status == PHFEM_EINVAL ? "phfem_csr_pcg_noalloc: a diagonal entry is missing or <= 0"
                                                   : "phfem_csr_pcg_noalloc: numerical failure");
  }
  if (h.done != 1) return fail(PHFEM_ENOCONV, "phfem_csr_pcg_noalloc: iteration limit reached");
  return PHFEM_OK;
}

}  // extern "C"
