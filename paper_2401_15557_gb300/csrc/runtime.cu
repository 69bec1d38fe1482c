// Context, errors, stream-ordered allocation and the device-wide scan.
#include <cstdio>
#include <cstring>

#include "internal.cuh"

namespace phfem {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

int fail(int status, const std::string& msg) {
  set_error(msg);
  return status;
}

int cuda_fail(cudaError_t err, const char* what, const char* file, int line) {
  char buf[512];
  snprintf(buf, sizeof(buf), "%s failed: %s (%s:%d)", what, cudaGetErrorString(err), file, line);
  set_error(buf);
  return err == cudaErrorMemoryAllocation ? PHFEM_ENOMEM : PHFEM_ECUDA;
}

static void account(phfem_ctx ctx, void* p, size_t bytes) {
  ctx->live[p] = bytes;
  ctx->bytes_now += bytes;
  if (ctx->bytes_now > ctx->bytes_peak) ctx->bytes_peak = ctx->bytes_now;
}

int dalloc(phfem_ctx ctx, void** p, size_t bytes) {
  *p = nullptr;
  if (ctx->alloc) {
    *p = ctx->alloc(bytes, (void*)ctx->stream, ctx->alloc_user);
    if (!*p) return fail(PHFEM_ENOMEM, std::string("device allocation of ") + std::to_string(bytes) +
                                           " bytes failed (caller's allocator)");
    account(ctx, *p, bytes);
    return PHFEM_OK;
  }
  cudaError_t e = cudaMallocAsync(p, bytes, ctx->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(PHFEM_ENOMEM, std::string("device allocation of ") + std::to_string(bytes) +
                                  " bytes failed: " + cudaGetErrorString(e));
  }
  account(ctx, *p, bytes);
  return PHFEM_OK;
}

void dfree(phfem_ctx ctx, void* p) {
  if (!p) return;
  auto it = ctx->live.find(p);
  if (it != ctx->live.end()) {
    ctx->bytes_now -= it->second;
    ctx->live.erase(it);
  }
  if (ctx->free_fn) ctx->free_fn(p, (void*)ctx->stream, ctx->alloc_user);
  else cudaFreeAsync(p, ctx->stream);
}

bool set_l2_limit(phfem_ctx ctx, size_t bytes) {
  if (ctx->l2_limit == bytes) return true;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(ctx->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return false;
  }
  if (cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, bytes) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  ctx->l2_limit = bytes;
  return true;
}

int grid_for(phfem_ctx ctx, int64_t n) {
  int64_t need = (n + kBlock - 1) / kBlock;
  if (need < 1) need = 1;
  return (int)(need < ctx->grid ? need : ctx->grid);
}

static const char* kProfNames[kNumProf] = {"cg_spmv", "cg_update", "cg_dir", "residual",
                                           "asm_tri", "asm_rows", "recover", "mg_vcycle"};

void prof_start(phfem_ctx ctx, int k) {
  if (!ctx->profile) return;
  ProfSlot& p = ctx->prof[k];
  p.armed = (p.calls++ % ctx->profile_every) == 0;
  if (!p.armed) return;
  if (p.used + 2 > p.ev.size()) {
    for (int i = 0; i < 2; ++i) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return;
      p.ev.push_back(e);
    }
  }
  cudaEventRecord(p.ev[p.used], ctx->stream);
}

void prof_stop(phfem_ctx ctx, int k) {
  if (!ctx->profile) return;
  ProfSlot& p = ctx->prof[k];
  if (!p.armed || p.used + 2 > p.ev.size()) return;
  p.armed = false;
  cudaEventRecord(p.ev[p.used + 1], ctx->stream);
  p.used += 2;
}

int check_launch(phfem_ctx ctx, const char* what) {
  ctx->launches++;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, what, __FILE__, __LINE__);
  return PHFEM_OK;
}

// --- exclusive scan ---------------------------------------------------------
constexpr int kScanItems = 16;
constexpr int kScanTile = kBlock * kScanItems;

__device__ __forceinline__ int warp_incl_scan(int v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// Exclusive scan of one value per thread across the block; returns the block total.
__device__ __forceinline__ int block_excl_scan(int v, int* excl) {
  __shared__ int wsum[kBlock / 32];
  __shared__ int wtotal;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int inc = warp_incl_scan(v);
  if (lane == 31) wsum[w] = inc;
  __syncthreads();
  if (w == 0) {
    int s = (lane < kBlock / 32) ? wsum[lane] : 0;
    int si = warp_incl_scan(s);
    if (lane < kBlock / 32) wsum[lane] = si - s;
    if (lane == kBlock / 32 - 1) wtotal = si;
  }
  __syncthreads();
  *excl = inc - v + wsum[w];
  int total = wtotal;
  __syncthreads();
  return total;
}

__global__ void k_scan_reduce(const int32_t* __restrict__ in, int n, int32_t* __restrict__ sums) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  int s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    int64_t j = base + (int64_t)i * kBlock + threadIdx.x;
    if (j < n) s += in[j];
  }
  __shared__ double smem[kBlock / 32];
  double tot = block_sum((double)s, smem);
  if (threadIdx.x == 0) sums[blockIdx.x] = (int32_t)tot;
}

// Scans a tile; items are read in a blocked arrangement so that each thread
// owns kScanItems consecutive elements.
__global__ void k_scan_tile(const int32_t* __restrict__ in, int32_t* __restrict__ out, int n,
                            const int32_t* __restrict__ offsets, int32_t* __restrict__ total) {
  __shared__ int32_t tile[kScanTile];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  for (int i = threadIdx.x; i < kScanTile; i += kBlock) {
    int64_t j = base + i;
    tile[i] = (j < n) ? in[j] : 0;
  }
  __syncthreads();
  int local[kScanItems];
  int s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    local[i] = s;
    s += tile[threadIdx.x * kScanItems + i];
  }
  int excl;
  int btot = block_excl_scan(s, &excl);
  const int off = (offsets ? offsets[blockIdx.x] : 0) + excl;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) tile[threadIdx.x * kScanItems + i] = local[i] + off;
  __syncthreads();
  for (int i = threadIdx.x; i < kScanTile; i += kBlock) {
    int64_t j = base + i;
    if (j < n) out[j] = tile[i];
  }
  if (total && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0)
    *total = (offsets ? offsets[blockIdx.x] : 0) + btot;
}

int exclusive_scan(phfem_ctx ctx, const int32_t* in, int32_t* out, int n, int32_t* total_dev) {
  if (n <= 0) {
    if (total_dev) PH_CUDA(cudaMemsetAsync(total_dev, 0, sizeof(int32_t), ctx->stream));
    return PHFEM_OK;
  }
  int nb = (n + kScanTile - 1) / kScanTile;
  if (nb == 1) {
    k_scan_tile<<<1, kBlock, 0, ctx->stream>>>(in, out, n, nullptr, total_dev);
    return check_launch(ctx, "k_scan_tile");
  }
  int32_t* sums = nullptr;
  PH_TRY(dalloc_n(ctx, &sums, (size_t)nb));
  k_scan_reduce<<<nb, kBlock, 0, ctx->stream>>>(in, n, sums);
  int st = check_launch(ctx, "k_scan_reduce");
  if (st == PHFEM_OK) st = exclusive_scan(ctx, sums, sums, nb, nullptr);
  if (st == PHFEM_OK) {
    k_scan_tile<<<nb, kBlock, 0, ctx->stream>>>(in, out, n, sums, total_dev);
    st = check_launch(ctx, "k_scan_tile");
  }
  dfree(ctx, sums);
  return st;
}

}  // namespace phfem

using namespace phfem;

extern "C" {

PHFEM_API const char* phfem_status_str(int s) {
  switch (s) {
    case PHFEM_OK: return "ok";
    case PHFEM_EINVAL: return "invalid argument";
    case PHFEM_EMESH: return "invalid mesh";
    case PHFEM_ENOMEM: return "out of device memory";
    case PHFEM_ENOCONV: return "not converged";
    case PHFEM_EBREAKDOWN: return "conjugate gradient breakdown";
    case PHFEM_ENAN: return "non-finite value";
    case PHFEM_ECUDA: return "CUDA error";
    default: return "unknown status";
  }
}

PHFEM_API const char* phfem_last_error(void) { return g_last_error.c_str(); }

PHFEM_API int phfem_ctx_create(void* cuda_stream, phfem_ctx* out) {
  if (!out) return fail(PHFEM_EINVAL, "phfem_ctx_create: out is NULL");
  *out = nullptr;
  int dev = 0;
  PH_CUDA(cudaGetDevice(&dev));
  int sms = 0;
  PH_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  phfem::SolveState* pinned = nullptr;
  PH_CUDA(cudaMallocHost((void**)&pinned, sizeof(phfem::SolveState)));
  int persist = 0, window = 0;
  if (cudaDeviceGetAttribute(&persist, cudaDevAttrMaxPersistingL2CacheSize, dev) != cudaSuccess) persist = 0;
  if (cudaDeviceGetAttribute(&window, cudaDevAttrMaxAccessPolicyWindowSize, dev) != cudaSuccess) window = 0;
  cudaGetLastError();
  phfem_ctx c = new phfem_ctx_s();
  c->l2_persist_max = persist > 0 ? (size_t)persist : 0;
  c->l2_window_max = window > 0 ? (size_t)window : 0;
  c->st_pinned = pinned;
  c->stream = (cudaStream_t)cuda_stream;
  c->device = dev;
  c->num_sms = sms;
  c->grid = sms * kBlocksPerSM;
  if (c->grid > kMaxGrid) c->grid = kMaxGrid;
  c->launches = 0;
  *out = c;
  return PHFEM_OK;
}

PHFEM_API int phfem_ctx_create_with_allocator(void* cuda_stream, phfem_alloc_fn alloc, phfem_free_fn free_fn,
                                              void* user, phfem_ctx* out) {
  if (!out) return fail(PHFEM_EINVAL, "phfem_ctx_create_with_allocator: out is NULL");
  *out = nullptr;
  if (!alloc || !free_fn) return fail(PHFEM_EINVAL, "phfem_ctx_create_with_allocator: NULL callback");
  PH_TRY(phfem_ctx_create(cuda_stream, out));
  (*out)->alloc = alloc;
  (*out)->free_fn = free_fn;
  (*out)->alloc_user = user;
  return PHFEM_OK;
}

PHFEM_API int phfem_ctx_destroy(phfem_ctx ctx) {
  if (!ctx) return fail(PHFEM_EINVAL, "phfem_ctx_destroy: NULL context");
  for (auto& p : ctx->prof)
    for (cudaEvent_t e : p.ev) cudaEventDestroy(e);
  if (ctx->st_pinned) cudaFreeHost(ctx->st_pinned);
  delete ctx;
  return PHFEM_OK;
}

PHFEM_API int64_t phfem_ctx_launches(phfem_ctx ctx) { return ctx ? ctx->launches : -1; }

PHFEM_API int phfem_ctx_memory(phfem_ctx ctx, int64_t* bytes_now, int64_t* bytes_peak, int32_t reset_peak) {
  if (!ctx) return fail(PHFEM_EINVAL, "phfem_ctx_memory: NULL context");
  if (bytes_now) *bytes_now = (int64_t)ctx->bytes_now;
  if (bytes_peak) *bytes_peak = (int64_t)ctx->bytes_peak;
  if (reset_peak) ctx->bytes_peak = ctx->bytes_now;
  return PHFEM_OK;
}

PHFEM_API int phfem_ctx_set_cg_kernel(phfem_ctx ctx, int variant) {
  if (!ctx) return fail(PHFEM_EINVAL, "phfem_ctx_set_cg_kernel: NULL context");
  if (variant < 0 || variant > 2) return fail(PHFEM_EINVAL, "phfem_ctx_set_cg_kernel: variant must be 0, 1 or 2");
  ctx->cg_variant = variant;
  return PHFEM_OK;
}

PHFEM_API int phfem_ctx_set_l2_window(phfem_ctx ctx, int enable) {
  if (!ctx) return fail(PHFEM_EINVAL, "phfem_ctx_set_l2_window: NULL context");
  ctx->l2_window = enable != 0;
  return PHFEM_OK;
}

PHFEM_API int phfem_ctx_profile(phfem_ctx ctx, int enable) {
  if (!ctx) return fail(PHFEM_EINVAL, "phfem_ctx_profile: NULL context");
  ctx->profile = enable != 0;
  ctx->profile_every = enable > 1 ? enable : 1;
  return PHFEM_OK;
}

PHFEM_API int phfem_ctx_kernel_time(phfem_ctx ctx, const char* kernel, double* total_ms, int64_t* launches,
                                    int reset) {
  if (!ctx || !kernel) return fail(PHFEM_EINVAL, "phfem_ctx_kernel_time: NULL argument");
  int k = -1;
  for (int i = 0; i < kNumProf; ++i)
    if (std::strcmp(kernel, kProfNames[i]) == 0) k = i;
  if (k < 0) return fail(PHFEM_EINVAL, std::string("phfem_ctx_kernel_time: unknown kernel ") + kernel);
  ProfSlot& p = ctx->prof[k];
  double tot = 0.0;
  if (p.used) PH_CUDA(cudaEventSynchronize(p.ev[p.used - 1]));
  for (size_t i = 0; i + 1 < p.used; i += 2) {
    float ms = 0.f;
    PH_CUDA(cudaEventElapsedTime(&ms, p.ev[i], p.ev[i + 1]));
    tot += ms;
  }
  if (total_ms) *total_ms = tot;
  if (launches) *launches = (int64_t)(p.used / 2);
  if (reset) {
    p.used = 0;
    p.calls = 0;
  }
  return PHFEM_OK;
}

}  // extern "C"
