// Internal declarations of the sm_103a primal hybrid FEM library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <unordered_map>
#include <vector>

#include "phfem.h"

namespace phfem {

constexpr int kBlock = 256;          // threads per block of every grid-stride kernel
constexpr int kBlocksPerSM = 8;      // resident blocks per SM targeted by the grids
constexpr int kMaxGrid = 152 * 16;   // upper bound of reduction partials per reduction

// Error plumbing ------------------------------------------------------------
void set_error(const std::string& msg);
int fail(int status, const std::string& msg);
int cuda_fail(cudaError_t err, const char* what, const char* file, int line);

#define PH_CUDA(call)                                                          \
  do {                                                                         \
    cudaError_t _e = (call);                                                   \
    if (_e != cudaSuccess) return ::phfem::cuda_fail(_e, #call, __FILE__, __LINE__); \
  } while (0)

#define PH_TRY(call)                \
  do {                              \
    int _s = (call);                \
    if (_s != PHFEM_OK) return _s;  \
  } while (0)

// Device-visible status word of a multi-kernel computation.
struct DevStatus {
  int code;      // 0 ok, else a negative phfem_status
  int index;     // first offending index (for messages)
  int detail;    // extra information
  int pad;
};

// Scalar state of one conjugate-gradient solve (device resident).
struct SolveState {
  double rz;       // r.r of the current inner residual (unit-diagonal system)
  double rz0;      // r.r at the start of the inner solve
  double tol2;     // inner stopping threshold on rz
  double alpha, beta;
  double rr64;     // ||b - S x||^2 of the outer FP64 residual
  double bb;       // ||b||^2 of the free-edge system (with lifting)
  double floor2;   // squared estimate of the residual that rounding x to FP64 alone leaves
  double rp;       // r.p right after a reliable update (p kept)
  double rr_pending, ff_pending;  // ||r||^2 and floor of a true residual awaiting the preconditioner
  double rho, omega;               // BiCGStab: (r^, r) and the stabilisation step
  int use_rp;      // 1: the next step is a line search alpha = r.p / p.Ap
  int restart;     // 1: the next SpMV restarts the direction, p = D^-1 r
  int conv;        // 1: rtol met, 2: stopped at the FP64 floor
  int updates;     // true-residual evaluations
  int bodies;      // executions of a graph loop body (bounded)
  int pad2;
  int it;          // inner iterations done
  int done;        // 1: inner converged, 2: outer converged, 3: failure
  int status;      // phfem_status of a failure
  int dir_pending; // set by the update kernel, cleared by the next SpMV: gates the direction kernel
  unsigned int counter[4];  // last-block counters of the reductions
  int par;         // locality-order CG: which of its direction buffers holds the current p
  int ypend;       // fused FP32 locality-order CG: the newest ypend directions' alpha p not yet in y
  double alpha_dir[4];  // locality-order CG: alpha of the direction held in each buffer
  double sc;       // locality-order CG: power-of-two scale of the inner vectors since the last true residual
  float alpha_f[2];          // alpha as an unevaluated pair of floats (set with alpha)
  float alpha_dir_f[4][2];   // alpha_dir likewise
};

}  // namespace phfem

namespace phfem {
// Kernels whose launches can be timed with CUDA events (phfem_ctx_profile).
enum ProfKernel { kProfSpmv = 0, kProfUpdate, kProfDir, kProfResidual, kProfAsmTri, kProfAsmRows,
                  kProfRecover, kProfMg, kNumProf };
struct ProfSlot {
  std::vector<cudaEvent_t> ev;  // start/stop pairs
  size_t used = 0;
  int64_t calls = 0;            // launches seen since the last reset
  bool armed = false;           // the current launch is being timed
};
}  // namespace phfem

// Handles --------------------------------------------------------------------
struct phfem_ctx_s {
  cudaStream_t stream;
  int device;
  int num_sms;
  int grid;              // blocks of the grid-stride kernels
  size_t l2_persist_max = 0;  // largest L2 set-aside for persisting accesses (0: none)
  size_t l2_window_max = 0;   // largest access-policy window
  size_t l2_limit = 0;        // the set-aside reserved now (cudaLimitPersistingL2CacheSize)
  bool l2_window = true;      // solves may use an L2 persistence window
  int cg_variant = 0;         // FP32 locality-order CG: 0 fused, rows staged in shared memory; 1 separate
                              // direction kernel; 2 fused, rows through L1/L2
  int64_t launches;
  bool profile = false;
  int profile_every = 1;   // time every n-th launch of each kernel
  phfem::ProfSlot prof[phfem::kNumProf];
  phfem_alloc_fn alloc = nullptr;          // caller's allocator (NULL: cudaMallocAsync)
  phfem_free_fn free_fn = nullptr;
  void* alloc_user = nullptr;
  phfem::SolveState* st_pinned = nullptr;  // pinned host mirror of a solver state, shared by the
                                           // context's systems (read right after each copy)
  // device memory the context holds (its allocations through dalloc, by
  // pointer), now and at the peak since the last reset
  std::unordered_map<void*, size_t> live;
  size_t bytes_now = 0, bytes_peak = 0;
};

struct phfem_mesh_s {
  phfem_ctx ctx;
  phfem_mesh_info info;
  double* xy;            // [nV][2]
  int32_t* tri;          // [nT][3]
  int32_t* ed2el;        // [nE][4]
  int32_t* t2e;          // [nT][3]
  int8_t* sigma;         // [nT][3]
  uint8_t* eclass;       // [nE]
  uint8_t* lk;           // [nE]: local index of the edge in T+ | (in T-) << 2
  int32_t* free_id;      // [nE]
  int32_t* lam_id;       // [nE]
  int32_t* nbr;          // [4][nE] neighbour edges: T+ (k+1, k+2), T- (k+1, k+2); self if absent
  double* elen;          // [nE] edge lengths
  int32_t* row_ptr;      // [nF + 1]
  int32_t* col;          // [nnz]
  int32_t* bpairs;       // [nD + nN][2] copies of the listed Dirichlet then Neumann pairs
  int32_t* bedge;        // [nD + nN] edge id of each listed pair
  // locality order of the iteration kernels (built on first use, mesh_order):
  int32_t* perm = nullptr;     // [nE] internal row -> edge (Morton order of the midpoints)
  int32_t* iperm = nullptr;    // [nE] edge -> internal row
  short4* nbr16 = nullptr;     // [nE] neighbours of internal row i as i + delta; x = -32768: see nbr_ovf
  int4* nbr_ovf = nullptr;     // [novf] the four internal neighbours of the marked rows
  uint8_t* eclass_i = nullptr; // [nE] class of internal row i
  int novf = 0;
  // visit order of the edge-row assembly pass (built on its first use,
  // mesh_row_tiles): the tiles of kBlock consecutive edges by the Morton code
  // of their mean midpoint
  int32_t* row_tiles = nullptr;
};

namespace phfem {
struct FastCG;  // the conjugate-gradient operator and vectors in the locality order (cg.cu)
}

struct phfem_sys_s {
  phfem_mesh mesh;
  phfem_coeffs c;
  bool fp32;
  int form;              // PHFEM_FORM_TRACE or PHFEM_FORM_FLUX
  bool conv;             // convection: nonsymmetric rows, its columns follow the records in Kt, BiCGStab
  void* bw;              // BiCGStab workspace [7][nE] in the inner precision (allocated on first use)
  uint8_t ident_class;   // class of the identity rows: Dirichlet (trace) or Neumann (flux)
  double* St;            // [9][nT] flux form: S_T (00, 11, 22, 01, 12, 20) and the load terms g_T
  double* bc;            // [nE] copy of the boundary data (flux-form recovery)
  double* Kt;            // [nT][4]: records of K^CR_T, AoS: -K01, -K12, -K20, |T|/3 (the
                         //          stiffness rows sum to zero, so the diagonal follows)
                         //          (+ [3][nT] convection columns c_j with convection)
  double* val;           // [5][nE]: FP64 row in difference form: slot 0 = r_e (reaction/mass
                         //          part of the diagonal), slots 1..4 = l_es = -S_{e,nbr_s}
  double* b;             // [nE]: right-hand side; u_D on Dirichlet rows
  double* me;            // [nE]: mass diagonal sum_T |T|/3 (dt > 0 only, else NULL)
  // inner operator in difference form (float or double):
  //   (S p)_e = rdiag_e p_e + sum_s lval[s][e] (p_e - p[nbr[s][e]])
  void* lval;            // [4][nE]: -S_{e, nbr_s}
  void* rdiag;           // [nE]: row sum (reaction / mass part)
  void* dinv;            // [nE]: 1 / S_ee (Jacobi)
  double* f;             // [nE]: copy of f at the midpoints (elliptic recovery)
  // solver workspace
  double* x;             // [nE] current midpoint values (FP64); during a paper-order solve the
                         //      correction since the last reliable update
  double* xh;            // [nE] paper-order solve: the solution as an FP64 pair xh + xl
  double* xl;            // [nE]
  double* r64;           // [nE]
  size_t l2_vec;         // bytes of one inner vector slot (r, p, q are consecutive slots)
  void* ri;              // [nE] inner vectors (float or double); pi and qi follow ri in one allocation
  void* pi;
  void* qi;
  double* partials;      // [4][kMaxGrid]
  phfem::SolveState* st;       // device
  phfem::SolveState* st_host;  // pinned host mirror (the context's)
  phfem_mg mg;                 // multigrid preconditioner (not owned), or NULL: Jacobi
  phfem::FastCG* fcg = nullptr;  // Jacobi-PCG in the locality order (built on the first solve)
};

namespace phfem {

// Allocation on the context stream (stream-ordered allocator).
int dalloc(phfem_ctx ctx, void** p, size_t bytes);
void dfree(phfem_ctx ctx, void* p);
template <typename T>
int dalloc_n(phfem_ctx ctx, T** p, size_t n) {
  return dalloc(ctx, reinterpret_cast<void**>(p), n * sizeof(T) + (n == 0 ? 16 : 0));
}

int grid_for(phfem_ctx ctx, int64_t n);
// Sets the device's persisting L2 set-aside (0 releases it); false under a
// stream capture (unless already that size) or when the call fails.
bool set_l2_limit(phfem_ctx ctx, size_t bytes);
// Event pair around one launch of kernel k when profiling is on (no-op otherwise).
void prof_start(phfem_ctx ctx, int k);
void prof_stop(phfem_ctx ctx, int k);
int check_launch(phfem_ctx ctx, const char* what);

// Device-wide exclusive scan of int32 (out may alias in); returns the total
// through *total_dev (device int) if non-NULL.
int exclusive_scan(phfem_ctx ctx, const int32_t* in, int32_t* out, int n, int32_t* total_dev);

// Solve helpers shared by the elliptic and Crank-Nicolson drivers.
int solve_system(phfem_sys sys, const phfem_solve_opts* opts, phfem_stats* stats, bool warm);
// Enqueues a whole solve (start, device-controlled iteration loop in a CUDA
// graph conditional WHILE node) into the graph being captured on `capture`.
int capture_solve(phfem_sys sys, const phfem_solve_opts* opts, cudaStream_t capture, int iters_per_body);
int sys_init_x(phfem_sys sys, const double* w0);
void fill_opts(phfem_sys sys, phfem_solve_opts& o);
// Numbering of free edges and multipliers, neighbour slots, edge lengths and
// the CSR pattern of a mesh whose xy, ed2el, lk, t2e and eclass are set.
int mesh_finish(phfem_mesh m);
// BiCGStab for systems with convection (same stopping rules and state).
int solve_bicgstab(phfem_sys sys, const phfem_solve_opts& o, phfem_stats* stats);
// phfem_assemble without the host synchronisation that checks a_T (for
// coefficients the library derived itself).
int assemble_system(phfem_mesh mesh, const phfem_coeffs& c, const double* f_mid, const double* bc_mid,
                    phfem_sys* out, bool check);
// Locality order of a mesh's edges for the iteration kernels (order.cu).
int mesh_order(phfem_mesh m);
int mesh_row_tiles(phfem_mesh m);
void mesh_order_free(phfem_mesh m);
int radix_sort_pairs(phfem_ctx ctx, uint32_t* k0, int32_t* v0, uint32_t* k1, int32_t* v1, int n, int bits);
// Jacobi-PCG on the trace-form system in the locality order (cg.cu): used for
// systems without convection and without multigrid.
bool fcg_eligible(phfem_sys sys, const phfem_solve_opts& o);
int fcg_solve(phfem_sys sys, const phfem_solve_opts& o, phfem_stats* stats);
int fcg_capture(phfem_sys sys, const phfem_solve_opts& o, cudaStream_t cs, int per_body);
int fcg_prepare(phfem_sys sys);
void fcg_free(phfem_sys sys);
int recover(phfem_sys sys, const double* x_new, const double* x_old, const double* f_eff,
            double inv_dt, double theta, double* U, double* Lambda);
// z = V-cycle(r) on the multigrid's finest level (into mg_fine_z(mg)); with
// st != NULL every kernel runs only while st->done == want.
int mg_apply(phfem_mg mg, cudaStream_t s, const void* r, const SolveState* st, int want);
void* mg_fine_z(phfem_mg mg);
// Called when the multigrid's system is destroyed first: the multigrid no
// longer refers to it.
void mg_forget_system(phfem_mg mg);

// Device helpers ---------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block sum of v (blockDim.x == kBlock); result valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double* smem) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) smem[w] = v;
  __syncthreads();
  v = 0.0;
  if (w == 0) {
    v = (lane < kBlock / 32) ? smem[lane] : 0.0;
    v = warp_sum(v);
  }
  __syncthreads();
  return v;
}

// Call after thread 0 wrote this block's partial(s): reports whether this is
// the last block to finish.  The last block can then read every partial (in a
// fixed order, hence a deterministic result) and must reset *counter to 0.
__device__ __forceinline__ bool arrive_last(unsigned int* counter) {
  __shared__ bool am_last;
  if (threadIdx.x == 0) {
    __threadfence();
    unsigned int t = atomicAdd(counter, 1u);
    am_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (am_last) __threadfence();
  return am_last;
}

// Sum of the partials in fixed order by the last block; result in thread 0.
__device__ __forceinline__ double sum_partials(const double* partials, double* smem) {
  double v = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) v += __ldcg(partials + i);
  return block_sum(v, smem);
}

}  // namespace phfem
