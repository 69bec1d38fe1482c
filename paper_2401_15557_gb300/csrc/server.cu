// Continuous-batching request server.
//
// Requests (elliptic solves and Crank-Nicolson runs on meshes of any size)
// are queued in arrival order.  Worker slots -- each a host thread owning a
// context on its own CUDA stream -- take the head of the queue as soon as they
// are free and the request's device-memory estimate fits in what remains of
// the HBM budget, so requests that arrive while others run are admitted as
// slots and memory free up and their kernels overlap on the GPU.  Mesh
// tables, the condensed system, the Jacobi preconditioner and the time-stepping
// state live on the device for the lifetime of a request.  Every request
// records its submit, admit and finish times (seconds since the server started).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "internal.cuh"

namespace phfem {
namespace {

// f at every edge, u_D on Dirichlet edges and g on Neumann edges (constants),
// and the initial values (u_D on Dirichlet edges) when w0 is given.
__global__ void k_fill_edge_data(int nE, const uint8_t* __restrict__ eclass, double f, double uD, double g,
                                 double* __restrict__ f_mid, double* __restrict__ bc_mid, double u0,
                                 double* __restrict__ w0) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nE; e += gridDim.x * blockDim.x) {
    const uint8_t c = eclass[e];
    f_mid[e] = f;
    bc_mid[e] = c == PHFEM_EDGE_DIRICHLET ? uD : (c == PHFEM_EDGE_NEUMANN ? g : 0.0);
    if (w0) w0[e] = c == PHFEM_EDGE_DIRICHLET ? uD : u0;
  }
}

// The GPU's global nanosecond timer, written by one thread.  (Timing CUDA
// events recorded on each request's stream, which this replaced, held small
// requests' host threads for hundreds of milliseconds while large requests
// ran: p50 77 ms against 16 ms at 8 requests/s.)
__global__ void k_stamp(uint64_t* out) {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  *out = t;
}

double now_since(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace
}  // namespace phfem

using namespace phfem;

struct phfem_server_s {
  int device;
  double budget;
  double reserved = 0.0;
  phfem_solve_opts opts;
  std::chrono::steady_clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::pair<int64_t, phfem_request>> queue;
  std::map<int64_t, phfem_result> results;
  int64_t next_id = 1;
  bool stop = false;
  std::vector<std::thread> workers;
  // per slot, kPrioClasses contexts, each on a stream of its own priority:
  // [slot * kPrioClasses + class]
  std::vector<phfem_ctx> ctxs;
  std::vector<cudaStream_t> streams;
  // device-time windows of the requests: the global timer (ns) written by a
  // one-thread kernel at the start and end of each request, per context
  // [2 * context], read back through pinned host memory; ref_ns is the
  // timer when the server was created
  uint64_t ref_ns = 0;
  uint64_t* stamp_dev = nullptr;
  uint64_t* stamp_host = nullptr;
  int64_t completed = 0;
  // largest device bytes per finest-mesh triangle that finished requests
  // allocated, by kind (elliptic, Crank-Nicolson) and refinement (none, some);
  // 0 until one has finished
  double per_tri[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
};

namespace phfem {
namespace {

double fine_triangles(const phfem_request& r) {
  return (double)r.nT * std::pow(4.0, (double)std::max(0, r.levels));
}

// Stream priority classes by request size: a small request's many short
// kernels would otherwise wait behind the full-GPU grids of a large one (a
// 50k-triangle multigrid solve took 36 ms beside a level-5 Jacobi solve on
// another stream, 5.5 ms on a higher-priority stream, 1.8 ms alone), so the
// block scheduler serves small requests first.
constexpr int kPrioClasses = 3;
int prio_class(const phfem_request& r) {
  const double fine = fine_triangles(r);
  return fine < 131072.0 ? 0 : (fine < 1048576.0 ? 1 : 2);
}

// The reservation of a request (the server's lock held): the measured bytes
// per triangle of its class, plus 10 %, once a request of the class has
// finished; before that a static guess (tables ~100 B/triangle, system ~150 B
// per edge at 1.5 edges per triangle, solver vectors and CN state: 400 B per
// triangle; a refinement hierarchy adds a third and the multigrid vectors),
// and 4 MB for what does not grow with the mesh.
double estimate_bytes(const phfem_server_s* S, const phfem_request& r) {
  const double fine = fine_triangles(r);
  const double learned = S->per_tri[r.kind == 1][r.levels > 0];
  if (learned > 0.0) return 1.1 * learned * fine + (double)(4 << 20);
  return (r.levels > 0 ? 600.0 : 400.0) * fine + (double)(4 << 20);
}
// Requests from which the bytes per triangle are learned: large enough that
// the allocations that do not grow with the mesh (reduction partials, sort
// scratch, the solver state) are a small part of the peak.
constexpr double kLearnFrom = 65536.0;

int run_request(phfem_ctx ctx, const phfem_request& r, const phfem_solve_opts& opts, phfem_result& out) {
  cudaStream_t s = ctx->stream;
  const size_t held0 = ctx->bytes_now;  // the request's own allocations are measured from here
  ctx->bytes_peak = held0;
  struct Peak {  // records the peak however the request ends
    phfem_ctx c;
    size_t base;
    phfem_result& o;
    ~Peak() { o.bytes_peak = (int64_t)(c->bytes_peak - base); }
  } peak{ctx, held0, out};
  std::vector<phfem_mesh> H;  // the hierarchy, coarsest first (one mesh without refinement)
  {
    phfem_mesh m0 = nullptr;
    PH_TRY(phfem_mesh_build(ctx, r.nV, r.xy, r.nT, r.tri, r.nD, r.dirichlet, r.nN, r.neumann, &m0));
    H.push_back(m0);
  }
  int st = PHFEM_OK;
  for (int l = 0; l < r.levels && st == PHFEM_OK; ++l) {
    phfem_mesh f = nullptr;
    st = phfem_mesh_refine(H.back(), nullptr, nullptr, nullptr, nullptr, &f);
    if (st == PHFEM_OK) H.push_back(f);
  }
  if (st != PHFEM_OK) {
    for (auto it = H.rbegin(); it != H.rend(); ++it) phfem_mesh_destroy(*it);
    return st;
  }
  phfem_mesh m = H.back();
  const phfem_mesh_info I = m->info;
  out.nL = I.nL;
  out.nE = I.nE;
  // the data: the caller's midpoint arrays, or constants filled in
  double *f = nullptr, *bc = nullptr, *w0 = nullptr;
  const bool fill_w0 = r.kind == 1 && !r.u0_mid;
  if (!r.f_mid || !r.bc_mid || fill_w0) {
    st = dalloc_n(ctx, &f, I.nE);
    if (st == PHFEM_OK) st = dalloc_n(ctx, &bc, I.nE);
    if (st == PHFEM_OK && fill_w0) st = dalloc_n(ctx, &w0, I.nE);
    if (st == PHFEM_OK) {
      k_fill_edge_data<<<grid_for(ctx, I.nE), kBlock, 0, s>>>(I.nE, m->eclass, r.f, r.uD, r.g, f, bc, r.u0, w0);
      st = check_launch(ctx, "k_fill_edge_data");
    }
  }
  const double* fe = r.f_mid ? r.f_mid : f;
  const double* be = r.bc_mid ? r.bc_mid : bc;
  const double* we = r.kind == 1 ? (r.u0_mid ? r.u0_mid : w0) : nullptr;
  phfem_sys sys = nullptr;
  phfem_mg mg = nullptr;
  if (st == PHFEM_OK) {
    phfem_coeffs c{r.a_T, 1.0, r.delta, r.kind == 1 ? r.dt : 0.0, r.precision, PHFEM_FORM_TRACE};
    st = phfem_assemble(m, &c, r.kind == 1 ? nullptr : fe, r.kind == 1 ? nullptr : be, &sys);
  }
  if (st == PHFEM_OK && H.size() > 1) {
    st = phfem_mg_create(sys, (int32_t)H.size(), H.data(), r.a_T, nullptr, &mg);
    if (st == PHFEM_OK) st = phfem_sys_set_mg(sys, mg);
  }
  if (st == PHFEM_OK && r.kind == 0) {
    phfem_stats stats{};
    st = phfem_solve(sys, &opts, nullptr, nullptr, r.U_out, r.Lambda_out, &stats);
    out.iterations = stats.iterations;
    out.rel_residual = stats.rel_residual;
  } else if (st == PHFEM_OK) {
    std::vector<double> phi((size_t)r.steps + 1, 1.0);  // constant-in-time data
    phfem_source src{1, r.steps + 1, fe, be, phi.data()};
    phfem_cn cn = nullptr;
    st = phfem_cn_create(sys, &src, we, nullptr, &cn);
    if (st == PHFEM_OK) {
      phfem_stats stats{};
      st = phfem_cn_step_graph(cn, r.steps, &opts, &stats);
      out.iterations = stats.iterations;
      out.rel_residual = stats.rel_residual;
      if (st == PHFEM_OK) st = phfem_cn_read(cn, nullptr, r.U_out, r.Lambda_out, nullptr, nullptr);
      phfem_cn_destroy(cn);
    }
  }
  if (mg) phfem_mg_destroy(mg);
  if (sys) phfem_sys_destroy(sys);
  dfree(ctx, f);
  dfree(ctx, bc);
  dfree(ctx, w0);
  for (auto it = H.rbegin(); it != H.rend(); ++it) phfem_mesh_destroy(*it);
  cudaError_t e = cudaStreamSynchronize(s);
  if (st == PHFEM_OK && e != cudaSuccess) st = cuda_fail(e, "server request", __FILE__, __LINE__);
  return st;
}

void worker(phfem_server S, int slot) {
  cudaSetDevice(S->device);
  for (;;) {
    std::pair<int64_t, phfem_request> job;
    double est = 0.0;
    {
      std::unique_lock<std::mutex> lock(S->mu);
      // FIFO admission: the head waits until its memory estimate fits
      S->cv_work.wait(lock, [&] {
        if (S->stop) return true;
        if (S->queue.empty()) return false;
        const double e = estimate_bytes(S, S->queue.front().second);
        return S->reserved + e <= S->budget || S->reserved == 0.0;
      });
      if (S->stop && S->queue.empty()) return;
      job = S->queue.front();
      S->queue.pop_front();
      est = estimate_bytes(S, job.second);
      S->reserved += est;
      S->results[job.first].t_admit = now_since(S->t0);
      S->results[job.first].slot = slot;
      S->results[job.first].bytes_reserved = est;
    }
    const int cls = prio_class(job.second);
    phfem_ctx ctx = S->ctxs[slot * kPrioClasses + cls];
    phfem_result res{};
    res.priority_class = cls;
    // the request's device-time window: timer stamps on its stream around its work
    const int ci = slot * kPrioClasses + cls;
    uint64_t* sd = S->stamp_dev + 2 * ci;
    uint64_t* sh = S->stamp_host + 2 * ci;
    k_stamp<<<1, 1, 0, ctx->stream>>>(sd);
    int st = run_request(ctx, job.second, S->opts, res);
    k_stamp<<<1, 1, 0, ctx->stream>>>(sd + 1);
    if (cudaMemcpyAsync(sh, sd, 2 * sizeof(uint64_t), cudaMemcpyDeviceToHost, ctx->stream) == cudaSuccess &&
        cudaStreamSynchronize(ctx->stream) == cudaSuccess) {
      res.t_dev_start = 1e-9 * (double)(int64_t)(sh[0] - S->ref_ns);
      res.t_dev_end = 1e-9 * (double)(int64_t)(sh[1] - S->ref_ns);
    }
    cudaGetLastError();
    {
      std::lock_guard<std::mutex> lock(S->mu);
      S->reserved -= est;
      phfem_result& R = S->results[job.first];
      R.status = st;
      R.done = 1;
      R.iterations = res.iterations;
      R.rel_residual = res.rel_residual;
      R.nL = res.nL;
      R.nE = res.nE;
      R.bytes_peak = res.bytes_peak;
      R.priority_class = res.priority_class;
      R.t_dev_start = res.t_dev_start;
      R.t_dev_end = res.t_dev_end;
      R.t_finish = now_since(S->t0);
      if (st == PHFEM_OK && res.bytes_peak > 0 && fine_triangles(job.second) >= kLearnFrom) {
        // what requests of this class actually allocate
        double& learned = S->per_tri[job.second.kind == 1][job.second.levels > 0];
        learned = std::max(learned, (double)res.bytes_peak / fine_triangles(job.second));
      }
      S->completed++;
    }
    S->cv_done.notify_all();
    S->cv_work.notify_all();
  }
}

}  // namespace
}  // namespace phfem

extern "C" {

PHFEM_API int phfem_server_create(int32_t slots, double hbm_budget_bytes, const phfem_solve_opts* opts,
                                  phfem_server* out) {
  if (!out) return fail(PHFEM_EINVAL, "phfem_server_create: out is NULL");
  *out = nullptr;
  if (slots < 1 || slots > 64 || !(hbm_budget_bytes > 0))
    return fail(PHFEM_EINVAL, "phfem_server_create: 1..64 slots and a positive budget");
  phfem_server S = new phfem_server_s();
  PH_CUDA(cudaGetDevice(&S->device));
  S->budget = hbm_budget_bytes;
  S->opts = opts ? *opts : phfem_solve_opts{};
  S->t0 = std::chrono::steady_clock::now();
  if (cudaMalloc((void**)&S->stamp_dev, sizeof(uint64_t) * 2 * (slots * kPrioClasses + 1)) != cudaSuccess ||
      cudaMallocHost((void**)&S->stamp_host, sizeof(uint64_t) * 2 * (slots * kPrioClasses + 1)) != cudaSuccess) {
    cudaGetLastError();
    if (S->stamp_dev) cudaFree(S->stamp_dev);
    delete S;
    return fail(PHFEM_ENOMEM, "phfem_server_create: timer stamps");
  }
  {  // the device-time origin, taken next to the host one
    uint64_t* last = S->stamp_dev + 2 * slots * kPrioClasses;
    k_stamp<<<1, 1>>>(last);
    if (cudaMemcpy(&S->ref_ns, last, sizeof(uint64_t), cudaMemcpyDeviceToHost) != cudaSuccess) {
      cudaFree(S->stamp_dev);
      cudaFreeHost(S->stamp_host);
      delete S;
      return fail(PHFEM_ECUDA, "phfem_server_create: timer origin");
    }
    S->t0 = std::chrono::steady_clock::now();
  }
  int least = 0, greatest = 0;  // numerically: greatest < least
  if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) least = greatest = 0;
  const int prio[kPrioClasses] = {greatest, (least + greatest) / 2, least};
  for (int i = 0; i < slots * kPrioClasses; ++i) {
    cudaStream_t s;
    cudaError_t e = cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, prio[i % kPrioClasses]);
    phfem_ctx c = nullptr;
    if (e != cudaSuccess || phfem_ctx_create(s, &c) != PHFEM_OK || phfem_ctx_set_l2_window(c, 0) != PHFEM_OK) {
      for (size_t j = 0; j < S->ctxs.size(); ++j) {
        phfem_ctx_destroy(S->ctxs[j]);
        cudaStreamDestroy(S->streams[j]);
      }
      cudaFree(S->stamp_dev);
      cudaFreeHost(S->stamp_host);
      delete S;
      return fail(PHFEM_ECUDA, "phfem_server_create: stream or context creation failed");
    }
    S->streams.push_back(s);
    S->ctxs.push_back(c);
  }
  for (int i = 0; i < slots; ++i) S->workers.emplace_back(worker, S, i);
  *out = S;
  return PHFEM_OK;
}

PHFEM_API int phfem_server_submit(phfem_server S, const phfem_request* req, int64_t* id) {
  if (!S || !req) return fail(PHFEM_EINVAL, "phfem_server_submit: NULL argument");
  if (req->kind != 0 && req->kind != 1) return fail(PHFEM_EINVAL, "phfem_server_submit: kind must be 0 or 1");
  if (req->kind == 1 && (!(req->dt > 0) || req->steps < 1))
    return fail(PHFEM_EINVAL, "phfem_server_submit: a Crank-Nicolson request needs dt > 0 and steps >= 1");
  if (req->levels < 0 || req->levels > 12 || (double)req->nT * std::pow(4.0, req->levels) > 5e8)
    return fail(PHFEM_EINVAL, "phfem_server_submit: levels in 0..12 and at most 5e8 refined triangles");
  int64_t my;
  {
    std::lock_guard<std::mutex> lock(S->mu);
    if (S->stop) return fail(PHFEM_EINVAL, "phfem_server_submit: server is stopping");
    my = S->next_id++;
    phfem_result r{};
    r.id = my;
    r.t_submit = now_since(S->t0);
    r.slot = -1;
    S->results[my] = r;
    S->queue.emplace_back(my, *req);
  }
  S->cv_work.notify_all();
  if (id) *id = my;
  return PHFEM_OK;
}

PHFEM_API int phfem_server_poll(phfem_server S, int64_t id, int32_t wait, phfem_result* out) {
  if (!S || !out) return fail(PHFEM_EINVAL, "phfem_server_poll: NULL argument");
  std::unique_lock<std::mutex> lock(S->mu);
  auto it = S->results.find(id);
  if (it == S->results.end()) return fail(PHFEM_EINVAL, "phfem_server_poll: unknown request id");
  if (wait) S->cv_done.wait(lock, [&] { return S->results[id].done != 0; });
  *out = S->results[id];
  return PHFEM_OK;
}

PHFEM_API int phfem_server_drain(phfem_server S) {
  if (!S) return fail(PHFEM_EINVAL, "phfem_server_drain: NULL server");
  std::unique_lock<std::mutex> lock(S->mu);
  S->cv_done.wait(lock, [&] { return S->queue.empty() && S->completed == S->next_id - 1; });
  return PHFEM_OK;
}

PHFEM_API int phfem_server_destroy(phfem_server S) {
  if (!S) return fail(PHFEM_EINVAL, "phfem_server_destroy: NULL server");
  {
    std::lock_guard<std::mutex> lock(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  for (auto& t : S->workers) t.join();
  for (size_t j = 0; j < S->ctxs.size(); ++j) {
    phfem_ctx_destroy(S->ctxs[j]);
    cudaStreamDestroy(S->streams[j]);
  }
  cudaFree(S->stamp_dev);
  cudaFreeHost(S->stamp_host);
  delete S;
  return PHFEM_OK;
}

}  // extern "C"
