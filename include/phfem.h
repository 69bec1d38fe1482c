/*
 * phfem.h -- C ABI of the GB300 (sm_103a) primal hybrid finite element library.
 *
 * Lowest-order primal hybrid FEM for 2D second-order elliptic problems and
 * their Crank-Nicolson parabolic counterparts with mixed Dirichlet/Neumann
 * boundaries (Nagula Mallesham, Porwal, Valdman, Acharya, "Vectorized
 * implementation of primal hybrid FEM in MATLAB", arXiv 2401.15557):
 * discontinuous P1 unknowns on every triangle, one piecewise-constant Lagrange
 * multiplier per non-Neumann edge (Section 3.2, Eqs. ph21-ph22).
 *
 * The library eliminates every element's three P1 unknowns in favour of its
 * three edge-midpoint values w_T = R u_T (R from Definition 3.1: the rows R_k
 * of lambda_j at the midpoints).  The multiplier constraint (Eq. ph22) makes
 * these midpoint values single-valued, so the solve runs on one SPD system
 * over the edges; U and Lambda are recovered exactly from w per element.
 *
 * Conventions shared by every entry point:
 *   - Pointers to arrays are DEVICE pointers (CUDA global memory of the current
 *     device) unless the comment says "host".  Arrays are 0-based, row-major.
 *   - The caller owns every array it passes; the library reads inputs and
 *     writes outputs only during the call, ordered on the context's stream,
 *     and keeps no pointer to them after the call returns.
 *   - Handles (phfem_ctx/_mesh/_sys/_cn) own their device buffers (allocated
 *     stream-ordered on the context stream) until the matching *_destroy.
 *   - Every function returns a phfem_status (0 = success, < 0 = error); the
 *     message of the last error of the calling thread is phfem_last_error().
 *     On error no output is guaranteed to be written and no handle is created.
 *   - Edge numbering follows the paper's nodes2edge (Listing 2): edges are
 *     numbered by increasing (larger vertex, smaller vertex).
 *   - Local edge k of a triangle (P1, P2, P3) = (tri[t][0], tri[t][1],
 *     tri[t][2]) is the edge opposite P_{k+1} (E1, E2, E3 of Section 2).
 */
#ifndef PHFEM_H
#define PHFEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define PHFEM_API __attribute__((visibility("default")))
#else
#define PHFEM_API
#endif

typedef enum {
  PHFEM_OK = 0,
  PHFEM_EINVAL = -1,      /* bad argument (NULL handle, negative size, ...)        */
  PHFEM_EMESH = -2,       /* mesh rejected (see phfem_mesh_build)                   */
  PHFEM_ENOMEM = -3,      /* device allocation failed                                */
  PHFEM_ENOCONV = -4,     /* iteration limits reached before the tolerance           */
  PHFEM_EBREAKDOWN = -5,  /* conjugate gradients met p.Ap <= 0                       */
  PHFEM_ENAN = -6,        /* a NaN or Inf appeared in coefficients or iterates       */
  PHFEM_ECUDA = -7        /* a CUDA runtime call failed                               */
} phfem_status;

enum { PHFEM_FP64 = 0, PHFEM_FP32_IR = 1 };
enum { PHFEM_EDGE_INTERIOR = 0, PHFEM_EDGE_DIRICHLET = 1, PHFEM_EDGE_NEUMANN = 2 };

typedef struct phfem_ctx_s* phfem_ctx;
typedef struct phfem_mesh_s* phfem_mesh;
typedef struct phfem_sys_s* phfem_sys;
typedef struct phfem_cn_s* phfem_cn;

/* ------------------------------------------------------------------------ */
/* Context                                                                   */
/* ------------------------------------------------------------------------ */

/* Creates a context bound to the current CUDA device and to `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  All work of handles
 * made from this context is ordered on that stream. */
PHFEM_API int phfem_ctx_create(void* cuda_stream, phfem_ctx* out);
/* Device memory of the context's handles normally comes from the stream-ordered
 * allocator (cudaMallocAsync on the context stream).  With these callbacks it
 * comes from the caller's allocator instead (for instance a framework's caching
 * allocator, so that one pool owns all device memory): alloc returns `bytes` of
 * device memory usable on `stream` (NULL on failure -> PHFEM_ENOMEM), free
 * releases a pointer alloc returned, ordered on `stream`.  Both are called from
 * the thread that calls the library. */
typedef void* (*phfem_alloc_fn)(size_t bytes, void* stream, void* user);
typedef void (*phfem_free_fn)(void* ptr, void* stream, void* user);
PHFEM_API int phfem_ctx_create_with_allocator(void* cuda_stream, phfem_alloc_fn alloc, phfem_free_fn free_fn,
                                              void* user, phfem_ctx* out);
PHFEM_API int phfem_ctx_destroy(phfem_ctx ctx);
PHFEM_API const char* phfem_status_str(int status);
PHFEM_API const char* phfem_last_error(void);
/* Number of kernels the library launched on this context so far. */
PHFEM_API int64_t phfem_ctx_launches(phfem_ctx ctx);
/* Device memory held by the context's own allocations (meshes, systems,
 * solver workspaces: every buffer the library allocated through the context,
 * not the caller's arrays): now, and at the peak since the last reset;
 * reset_peak != 0 then sets the peak to the current value.  Either output may
 * be NULL. */
PHFEM_API int phfem_ctx_memory(phfem_ctx ctx, int64_t* bytes_now, int64_t* bytes_peak, int32_t reset_peak);
/* A context, and everything built on it, is used by one host thread at a time
 * (its systems share one pinned host mirror of the solver state). */
/* Solves keep the iteration's residual and direction resident in L2 with an
 * access-policy window when both fit the device's largest persisting set-aside;
 * the set-aside (cudaLimitPersistingL2CacheSize, a limit of the process's CUDA
 * context, released with it) is sized to the window, and the window's lines are
 * reset after each solve.  Contexts driven from several host threads at once
 * (the request server's) should turn the window off: the limit is shared. */
PHFEM_API int phfem_ctx_set_l2_window(phfem_ctx ctx, int enable);
/* Kernels of the FP32 Jacobi iteration in the locality order (a tuning choice,
 * not part of the method): 0 = the direction update p = u + beta p is folded
 * into the operator product, whose rows' own data are staged in shared memory
 * by bulk copies (two kernels per iteration, the default); 1 = the direction
 * update runs as a kernel of its own (three kernels); 2 = as 0 with the rows'
 * data read through L1/L2 after an L2 prefetch.  All compute the same p and q
 * per row; the sums are grouped alike, so results agree to rounding.  FP64
 * systems always use the separate direction kernel.  Other values:
 * PHFEM_EINVAL. */
PHFEM_API int phfem_ctx_set_cg_kernel(phfem_ctx ctx, int variant);
/* Instrumentation (not part of the method): when enabled, launches of the
 * kernels "cg_spmv", "cg_update", "cg_dir", "residual", "asm_tri", "asm_rows",
 * "recover" and of whole multigrid V-cycles ("mg_vcycle") are bracketed by
 * CUDA events on the context
 * stream; enable = n > 1 times only every n-th launch of each kernel (events
 * between two launches keep the second from overlapping the first's drain).
 * phfem_ctx_kernel_time synchronises on the last event and returns the summed
 * device time (ms) and the number of timed launches of one kernel;
 * reset != 0 starts a new accumulation. */
PHFEM_API int phfem_ctx_profile(phfem_ctx ctx, int enable);
PHFEM_API int phfem_ctx_kernel_time(phfem_ctx ctx, const char* kernel, double* total_ms,
                                    int64_t* launches, int reset);

/* ------------------------------------------------------------------------ */
/* Mesh tables (Section 2.2: edge_vec; Listings 1-3, Eqs. n2el/n2ed/ed2el)   */
/* ------------------------------------------------------------------------ */

typedef struct {
  int32_t nV, nT;  /* vertices, triangles                                   */
  int32_t nE;      /* edges (nrEdges of the paper)                           */
  int32_t nF;      /* free edges = interior + Neumann (unknowns of the solve) */
  int32_t nL;      /* multiplier edges = interior + Dirichlet (L, Sec. 2)   */
  int32_t nD, nN;  /* Dirichlet / Neumann edges                              */
  int32_t nnz;     /* nonzeros of the free-edge system (CSR pattern)         */
} phfem_mesh_info;

/* Builds every table of the mesh on the device.
 *   xy        [nV][2] double   vertex coordinates (coordinates.dat, Table 1)
 *   tri       [nT][3] int32    counter-clockwise triangles (elements.dat)
 *   dirichlet [nD][2] int32    vertex pairs of the Dirichlet edges (Dirichlet.dat)
 *   neumann   [nN][2] int32    vertex pairs of the Neumann edges (Neumann.dat)
 * Rules (the paper's definitions):
 *   - edge e's T+ is the first triangle, in the element-major order of the
 *     directed edges P1P2, P2P3, P3P1, that holds it; (initial, end) is its
 *     direction in T+; T- is the other triangle (ed2el, Eq. ed2el);
 *   - sigma = +1 on the T+ side of an edge and -1 on the T- side (psi_E, Sec. 3.2).
 * Returns PHFEM_EMESH when a vertex id is out of range, a triangle is
 * clockwise or degenerate, an edge lies in more than two triangles or twice in
 * the same direction, a boundary edge is listed in neither or both lists or
 * twice, or a listed pair is not a boundary edge.  The mesh handle copies xy
 * and tri (the caller's arrays may be freed after the call). */
PHFEM_API int phfem_mesh_build(phfem_ctx ctx, int32_t nV, const double* xy, int32_t nT,
                               const int32_t* tri, int32_t nD, const int32_t* dirichlet,
                               int32_t nN, const int32_t* neumann, phfem_mesh* out);
PHFEM_API int phfem_mesh_info_get(phfem_mesh mesh, phfem_mesh_info* out);
/* Copies tables into caller device buffers; any pointer may be NULL.
 *   ed2el   [nE][4] int32  initial node, end node, T+, T- (-1 on the boundary)
 *   t2e     [nT][3] int32  edge opposite local vertex k (E_{k+1})
 *   sigma   [nT][3] int8   +1 if the triangle is T+ of that edge, else -1
 *   eclass  [nE]    uint8  PHFEM_EDGE_INTERIOR / _DIRICHLET / _NEUMANN
 *   free_id [nE]    int32  row of the edge in the free-edge system, -1 on Dirichlet
 *   lam_id  [nE]    int32  index of the edge's multiplier (Redges order of
 *                          Main.m: non-Neumann edges by increasing number), -1 on Neumann
 *   row_ptr [nF+1]  int32  CSR row pointer of the free-edge system
 *   col     [nnz]   int32  CSR columns (sorted in each row; every pair of free
 *                          edges sharing a triangle, exact zeros kept) */
PHFEM_API int phfem_mesh_tables(phfem_mesh mesh, int32_t* ed2el, int32_t* t2e, int8_t* sigma,
                                uint8_t* eclass, int32_t* free_id, int32_t* lam_id,
                                int32_t* row_ptr, int32_t* col);
PHFEM_API int phfem_mesh_destroy(phfem_mesh mesh);

/* Uniform red refinement (Section 2.3, redrefine_vec) of a built mesh:
 *   - the midpoint of edge e (the mesh's edge numbering) becomes vertex nV + e,
 *     at (initial + end) / 2;
 *   - triangle t becomes its middle child [M1 M2 M3] at position t (Mk = the new
 *     vertex on the edge opposite Pk), and its corner children [P1 M3 M2],
 *     [P2 M1 M3], [P3 M2 M1] go to positions nT + 3t, nT + 3t + 1, nT + 3t + 2;
 *   - each listed boundary pair (a, b), in the order it was given to
 *     phfem_mesh_build, becomes (a, m) at its own position and (m, b) at
 *     position (list length + its own).
 * Outputs (caller device buffers; each may be NULL, then a temporary is used):
 *   xy [nV + nE][2] double, tri [4 nT][3] int32, dirichlet [2 nD][2] int32,
 *   neumann [2 nN][2] int32.
 * If fine != NULL, the refined mesh is also returned: its tables follow from the
 * coarse ones in closed form (one scan, no sort) and equal those that
 * phfem_mesh_build makes from the refined arrays; with fine == NULL, xy and
 * tri must be given.
 * PHFEM_EINVAL when a refined count exceeds the int32 range. */
PHFEM_API int phfem_mesh_refine(phfem_mesh coarse, double* xy, int32_t* tri, int32_t* dirichlet,
                                int32_t* neumann, phfem_mesh* fine);

/* ------------------------------------------------------------------------ */
/* Assembly (Definition 3.1; Eqs. right_b, right_g, DirichletEqn; Sec. 3.5)  */
/* ------------------------------------------------------------------------ */

typedef struct {
  const double* a_T;  /* [nT] per-triangle coefficient (A = a_T I), or NULL      */
  double a;           /* coefficient used when a_T == NULL                       */
  double delta;       /* reaction coefficient delta >= 0 (Eq. eq1)                */
  double dt;          /* 0: elliptic; > 0: Crank-Nicolson matrix M + dt/2 K (Sec. 4) */
  int32_t precision;  /* PHFEM_FP64, or PHFEM_FP32_IR: FP32 inner solve + FP64 refinement,
                         element arithmetic in compensated FP32 (the FP64 operator
                         within a few 1e-14 of the row scale; FP64 for triangles whose
                         angle at P0 has a sine below 1/4, for coordinates or a
                         coefficient outside [2^-40, 2^40], and for a tensor A)      */
  int32_t form;       /* PHFEM_FORM_TRACE (edge-midpoint values, default) or
                         PHFEM_FORM_FLUX (multipliers; elliptic with delta > 0)     */
  double A[3];        /* constant SPD tensor (A11, A12, A22) of Eq. eq1, scaled per
                         triangle by a_T (or a); all zero = identity               */
  double p[2];        /* constant convection velocity (the D_T block of Definition
                         3.1); nonzero makes the system nonsymmetric: phfem_solve
                         then uses BiCGStab (trace form; not with multigrid or the
                         graph-captured Crank-Nicolson step)                       */
} phfem_coeffs;

enum { PHFEM_FORM_TRACE = 0, PHFEM_FORM_FLUX = 1 };

/* Assembles, per triangle, the stiffness/reaction blocks of Definition 3.1
 * condensed to the edge midpoints, K^CR_T = R^-T (a_T B_T + D_T + delta M_T) R^-1
 * = a_T |T|^-1 (e_k' A~ e_j) + delta |T|/3 I + the convection columns
 * (p_x e_jy - p_y e_jx)/3 (e_k the edge vectors, A~ = [[A22, -A12], [-A12, A11]],
 * A = I unless given), and the
 * edge right-hand side of the midpoint quadrature of Eqs. right_b/right_g:
 *   rhs_e = sum_{T owning e} |T|/3 f(m_e) + [e Neumann] |E| g(m_e).
 * Dirichlet values enter through the matrix (lifting) at solve time.
 *   f_mid  [nE] double  f at the edge midpoints
 *   bc_mid [nE] double  u_D(m_E) on Dirichlet edges, g(m_E) (outward normal
 *                       flux) on Neumann edges, ignored elsewhere
 * For dt > 0 the matrix is M^CR + dt/2 K^CR (M^CR = |T|/3 I per triangle) and
 * f_mid/bc_mid may be NULL (the source comes with phfem_cn_create).
 * PHFEM_FORM_FLUX eliminates the element unknowns in favour of the multipliers
 * instead (Sec. 3.5 with U_T = K_T^-1 (F_T + C_T' Lambda_T)): the SPD system
 * S Lambda = -b_D - sum_T C_T K_T^-1 F_T over the non-Neumann edges, with
 * S_T = C_T K_T^-1 C_T' = diag(sigma|E|) (K^CR_T)^-1 diag(sigma|E|) per
 * triangle (Neumann edges become identity rows with Lambda = 0).  It needs an
 * invertible K_T (delta > 0) and is elliptic only (dt = 0); phfem_sys_csr is
 * not available for it (its rows are the multiplier edges).
 * Returns PHFEM_EINVAL for delta < 0, dt < 0, a nonpositive a, a tensor A that
 * is not positive definite, or convection with the flux form; PHFEM_ENAN when a
 * coefficient is not finite. */
PHFEM_API int phfem_assemble(phfem_mesh mesh, const phfem_coeffs* coeffs, const double* f_mid,
                             const double* bc_mid, phfem_sys* out);
/* The assembled free-edge system in CSR form (pattern of phfem_mesh_tables):
 *   val [nnz] double  matrix values; rhs [nF] double  right-hand side with
 *   the Dirichlet lifting applied.  Either pointer may be NULL. */
PHFEM_API int phfem_sys_csr(phfem_sys sys, double* val, double* rhs);
PHFEM_API int phfem_sys_destroy(phfem_sys sys);

/* ------------------------------------------------------------------------ */
/* Solve                                                                     */
/* ------------------------------------------------------------------------ */

typedef struct {
  double rtol;          /* stop when ||b - S w||_2 <= rtol ||b||_2 (FP64 S, free rows); 0 -> 1e-10 */
  double inner_rtol;    /* reliable-update factor: the true FP64 residual replaces the
                           recursive one whenever the latter fell by this factor;
                           0 -> 0.1 (FP32_IR) or 0.01 (FP64); with a multigrid
                           preconditioner 0 -> 1e-3 (FP32_IR) or 1e-4 (FP64); with
                           convection (BiCGStab) 0 -> 1e-2 (FP32_IR) or 1e-6 (FP64) */
  int32_t max_iter;     /* total inner iterations; 0 -> 200000                        */
  int32_t max_refine;   /* reliable updates (FP64 residual evaluations); 0 -> 1000    */
  int32_t check_every;  /* inner iterations between host convergence checks; 0 -> 64
                           (2 with a multigrid preconditioner, 16 with convection)  */
  int32_t order;        /* Jacobi iteration without multigrid or convection:
                           0 = in the locality order of the edges (Morton order of
                           their midpoints; solution kept as an FP64 pair plus the
                           correction since the last reliable update), 1 = in the
                           paper's edge order (FP64 solution); other solvers ignore it */
} phfem_solve_opts;

typedef struct {
  int32_t iterations;   /* conjugate-gradient iterations                            */
  int32_t refinements;  /* FP64 residual evaluations (reliable updates)             */
  int32_t converged;    /* 1: rtol met; 2: stopped at the FP64 floor (see below)   */
  int32_t steps;        /* time steps done (phfem_cn_step)                          */
  double rel_residual;  /* final ||b - S w|| / ||b|| in FP64 (difference form)      */
  double seconds;       /* host wall time of the call                               */
  double fp64_floor;    /* estimated ||b - S w|| / ||b|| that rounding w to FP64
                           alone leaves: 2^-53 ||(|S| |w|)|| / ||b||              */
} phfem_stats;

/* Solves the condensed system by Jacobi-preconditioned conjugate gradients
 * (FP64, or FP32 iterations with FP64-accumulated dot products whose residual
 * is replaced by the true FP64 residual at every reliable update, the FP64
 * solution accumulating the corrections), then recovers the paper's unknowns.
 * With a multigrid attached (phfem_sys_set_mg) the V-cycle replaces the Jacobi
 * step; with convection the iteration is BiCGStab (Jacobi on the right) with
 * the same reliable updates and stopping rules.
 * The solve stops when rtol is met, or when the residual reaches twice the
 * FP64 floor (converged = 2): on fine meshes b scales like h^2 while S does
 * not, and below that level no FP64 vector w satisfies the system better.
 *   w0     [nE] double  initial midpoint values (NULL = zero); Dirichlet
 *                       entries are ignored (u_D is imposed)
 *   w      [nE] double  out: midpoint values of u_h on every edge (or NULL);
 *                       with PHFEM_FORM_FLUX: the multiplier of every edge
 *                       (0 on Neumann edges)
 *   U      [3 nT] double out: u_h at the vertices, element-major (3t + k;
 *                       Wvec(1:N) of Main.m) (or NULL)
 *   Lambda [nL] double  out: multipliers in Redges order (Wvec(N+1:N+L)) (or NULL)
 * Recovery: u_T = R^-1 w_T and Lambda_E = (K^CR_T w_T - F^CR_T)_k / |E| read on
 * the T+ side.  Blocks until the result is known (one host synchronisation
 * per check).  Returns PHFEM_ENOCONV when the limits are reached (outputs are
 * still written), PHFEM_EBREAKDOWN or PHFEM_ENAN on numerical failure. */
PHFEM_API int phfem_solve(phfem_sys sys, const phfem_solve_opts* opts, const double* w0,
                          double* w, double* U, double* Lambda, phfem_stats* stats);

/* ------------------------------------------------------------------------ */
/* Multigrid preconditioner over a red-refinement hierarchy (Section 2.3)     */
/* ------------------------------------------------------------------------ */

/* The paper solves with a direct solver; this preconditioner replaces the
 * Jacobi one in phfem_solve (and phfem_cn_step / phfem_cn_step_graph) when
 * the mesh comes from uniform red refinements.  Level l + 1 must be the
 * phfem_mesh_refine of level l; the finest level is the system's mesh.
 * Transfer between levels is that of Crouzeix-Raviart functions (the coarse
 * piecewise-linear function evaluated at the fine edge midpoints, averaged
 * over the two coarse triangles on coarse edges) and its transpose; coarse
 * operators are assembled like the fine one with a_T averaged over the four
 * children.  Smoothing: a Chebyshev polynomial of degree nu in D^-1 A on
 * [b / smooth_ratio, b], b the Gershgorin bound, before and after the coarse
 * correction (a symmetric V-cycle); the coarsest level: a Chebyshev
 * polynomial on the interval of its extreme Ritz values (Lanczos), of the
 * degree that reduces the error by coarse_eps.  The preconditioner is a fixed
 * linear SPD operator, so the conjugate-gradient iteration is unchanged. */
typedef struct phfem_mg_s* phfem_mg;
typedef struct {
  int32_t nu;            /* smoothing degree before and after; 0 -> 2 (1..16)        */
  double smooth_ratio;   /* smoothing interval [b / ratio, b]; 0 -> 6                */
  double coarse_eps;     /* coarsest-level error reduction; 0 -> 0.3                 */
  int32_t coarse_degree; /* > 0: fixed coarsest degree instead (<= 2000)            */
  int32_t flags;         /* PHFEM_MG_COARSE_STEPWISE: the coarsest iteration one
                            launch per step (the default runs it in one launch of a
                            thread-block cluster when its rows fit; same results) */
} phfem_mg_opts;
#define PHFEM_MG_COARSE_STEPWISE 1
typedef struct {
  int32_t levels, nu, coarse_degree, reserved;
  double coarse_a, coarse_b, smooth_ratio;
} phfem_mg_info_t;

/* Builds the hierarchy for `sys` (assembled on meshes[nlevels-1]):
 *   meshes [nlevels]  coarsest first; each the phfem_mesh_refine of the one
 *                     before (checked; PHFEM_EINVAL otherwise); the caller keeps
 *                     them alive while the multigrid exists
 *   a_T [nT_finest]   the fine coefficient given to phfem_assemble (device), or
 *                     NULL for the scalar a of the system's coefficients
 * Trace form only.  Blocks the host (it reads level bounds back). */
PHFEM_API int phfem_mg_create(phfem_sys sys, int32_t nlevels, const phfem_mesh* meshes,
                              const double* a_T, const phfem_mg_opts* opts, phfem_mg* out);
PHFEM_API int phfem_mg_info(phfem_mg mg, phfem_mg_info_t* out);
/* Attaches the multigrid to its system (NULL: back to Jacobi). */
PHFEM_API int phfem_sys_set_mg(phfem_sys sys, phfem_mg mg);
/* The transfer operators in FP64 (device buffers), for level l and l + 1:
 *   direction 0: out [nE_{l+1}] = P in [nE_l]   (zero on Dirichlet edges of l + 1;
 *                in must vanish on the Dirichlet edges of l, as corrections do)
 *   direction 1: out [nE_l] = P' in [nE_{l+1}]  (zero on Dirichlet edges of l) */
PHFEM_API int phfem_mg_transfer(phfem_mg mg, int32_t level, int32_t direction, const double* in,
                                double* out);
/* Detaches the multigrid from its system and frees it.  Destroying the system
 * first is allowed once the multigrid is attached (the multigrid then only
 * frees its own levels). */
PHFEM_API int phfem_mg_destroy(phfem_mg mg);

/* ------------------------------------------------------------------------ */
/* Crank-Nicolson (Section 4, Eq. MatrixformParabolic)                       */
/* ------------------------------------------------------------------------ */

#define PHFEM_MAX_TERMS 4
/* Source of separable form f(x, t) = sum_q phi_q(t) f_q(x) (same for u_D and g):
 *   f_mid  [nterms][nE] double  f_q at the edge midpoints
 *   bc_mid [nterms][nE] double  u_D,q on Dirichlet edges, g_q on Neumann edges
 *   phi    host [nterms][nt] double  phi_q(t_n), t_n = n dt, n = 0 .. nt-1 */
typedef struct {
  int32_t nterms;
  int32_t nt;
  const double* f_mid;
  const double* bc_mid;
  const double* phi;
} phfem_source;

/* Starts a time integration with the system of phfem_assemble(dt > 0).
 *   w0      [nE] double  u0 at the edge midpoints (U^0 = R^-1 w0 per element)
 *   Lambda0 [nL] double  initial multipliers, or NULL for zero
 * The source arrays are copied. */
PHFEM_API int phfem_cn_create(phfem_sys sys, const phfem_source* src, const double* w0,
                              const double* Lambda0, phfem_cn* out);
/* Advances nsteps steps: per step the edge right-hand side
 * (M - dt/2 K) w^{n-1} + dt (F^n + F^{n-1})/2 (trapezoid average of the
 * sources, Sec. 4), the solve of (M + dt/2 K) w^n with w^n = u_D(t_n) on
 * Dirichlet edges (warm start w^{n-1}), and the recovery of Lambda^{n-1/2}
 * and Lambda^n = 2 Lambda^{n-1/2} - Lambda^{n-1}.  Fails with PHFEM_EINVAL if
 * the source has no phi for a requested step. */
PHFEM_API int phfem_cn_step(phfem_cn cn, int32_t nsteps, const phfem_solve_opts* opts,
                            phfem_stats* stats);
/* As phfem_cn_step, with every step replayed from a CUDA graph captured on
 * first use (and again when opts change): right-hand side, Dirichlet values,
 * the solve -- its iteration loop a conditional WHILE node whose body runs
 * eight iterations, the conditional reliable update and a one-thread control
 * kernel (bounded by max_iter) -- and the recovery.  The time index and the
 * time factors are read on the device, so the host only launches the graph
 * nsteps times and synchronises once.  Gives bitwise the results of
 * phfem_cn_step.  Requires a context stream other than the legacy default
 * stream for nothing: capture runs on a private stream. */
PHFEM_API int phfem_cn_step_graph(phfem_cn cn, int32_t nsteps, const phfem_solve_opts* opts,
                                  phfem_stats* stats);
/* Crank-Nicolson with general sources (Section 4, Eqs. parabolicRight_*):
 * instead of separable terms, every step supplies the data at its new time.
 *   f0_mid, bc0_mid [nE] double: f at the midpoints and the boundary datum
 *          (g on Neumann, u_D on Dirichlet edges) at t_0 (NULL = 0)
 *   w0, Lambda0 as in phfem_cn_create; max_steps: steps the handle may take
 * phfem_cn_step_data advances one step, t_{n-1} -> t_n = t_{n-1} + dt:
 *   f_mid, bc_mid [nE] double: the data at t_n (NULL = 0).  The load is the
 *   trapezoid average of the data at t_{n-1} (kept from the previous call or
 *   f0/bc0) and t_n, the Dirichlet rows hold u_D(t_n).  Blocks the host.
 * phfem_cn_step / phfem_cn_step_graph refuse such a handle (PHFEM_EINVAL),
 * and phfem_cn_step_data a separable one. */
PHFEM_API int phfem_cn_create_data(phfem_sys sys, const double* f0_mid, const double* bc0_mid,
                                   const double* w0, const double* Lambda0, int32_t max_steps,
                                   phfem_cn* out);
PHFEM_API int phfem_cn_step_data(phfem_cn cn, const double* f_mid, const double* bc_mid,
                                 const phfem_solve_opts* opts, phfem_stats* stats);
/* Reads the state after the last step (any pointer may be NULL):
 *   w [nE], U [3 nT], Lambda_n [nL], Lambda_half [nL] (Lambda^{n-1/2}),
 *   step: host int32, number of steps done. */
PHFEM_API int phfem_cn_read(phfem_cn cn, double* w, double* U, double* Lambda_n,
                            double* Lambda_half, int32_t* step);
PHFEM_API int phfem_cn_destroy(phfem_cn cn);

/* ------------------------------------------------------------------------ */
/* Batched assembly and solve of many meshes in one persistent launch       */
/* ------------------------------------------------------------------------ */

typedef struct phfem_batch_s* phfem_batch;

/* Gathers the tables of `count` meshes built by phfem_mesh_build on the same
 * device into one batch (the meshes may be destroyed afterwards).  Arrays of a
 * batch are the per-mesh arrays concatenated in mesh order; phfem_batch_offsets
 * gives the start of every mesh (count + 1 entries, host int64) in triangles,
 * edges and multipliers. */
PHFEM_API int phfem_batch_create(phfem_ctx ctx, int32_t count, const phfem_mesh* meshes,
                                 phfem_batch* out);
PHFEM_API int phfem_batch_offsets(phfem_batch batch, int64_t* tri_off, int64_t* edge_off,
                                  int64_t* lam_off);
/* Assembles and solves every mesh of the batch in ONE kernel launch: each
 * thread block (or thread-block cluster) takes the next mesh (largest first)
 * and runs the condensed assembly (as phfem_assemble), Jacobi-PCG with
 * reliable updates (as phfem_solve, reductions over the block or cluster) and
 * the recovery of U and Lambda.
 *   a_T    [sum nT] double per-triangle coefficient, or NULL for a = 1
 *   delta  [count] double reaction coefficient per mesh (device)
 *   f_mid, bc_mid [sum nE] double as in phfem_assemble (either may be NULL)
 *   precision PHFEM_FP64 or PHFEM_FP32_IR; opts as in phfem_solve
 *   w [sum nE], U [3 sum nT], Lambda [sum nL] double outputs (each may be NULL)
 *   block, cluster  launch shape: threads per block and CTAs per mesh (a
 *          thread-block cluster; its reductions read the CTAs' partial sums
 *          through distributed shared memory): (128|256|512|1024, 1) or
 *          (256|512|1024, 4|8); (0, 0) for the tuned shape (256, 1 before tuning)
 *   iterations, converged [count] int32, rel_residual [count] double: host
 *          outputs per mesh (each may be NULL)
 * Blocks until the batch is done.  Returns the first failing mesh's status. */
PHFEM_API int phfem_batch_solve(phfem_batch batch, const double* a_T, const double* delta,
                                const double* f_mid, const double* bc_mid, int32_t precision,
                                const phfem_solve_opts* opts, double* w, double* U, double* Lambda,
                                int32_t block, int32_t cluster, int32_t* iterations, int32_t* converged,
                                double* rel_residual);
/* Autotuner: times phfem_batch_solve on these inputs with the ten launch
 * shapes (block, cluster) = (128,1) (256,1) (512,1) (1024,1) (256,4) (512,4)
 * (1024,4) (256,8) (512,8) (1024,8), in that order, keeps the fastest for
 * (0, 0), and reports it (chosen_block, chosen_cluster, host) with the ten
 * host wall times in ms (ms_per_shape[10], host; may be NULL). */
#define PHFEM_BATCH_SHAPES 10
PHFEM_API int phfem_batch_tune(phfem_batch batch, const double* a_T, const double* delta,
                               const double* f_mid, const double* bc_mid, int32_t precision,
                               const phfem_solve_opts* opts, int32_t* chosen_block, int32_t* chosen_cluster,
                               double* ms_per_shape);
PHFEM_API int phfem_batch_destroy(phfem_batch batch);

/* ------------------------------------------------------------------------ */
/* Request server with continuous batching                                   */
/* ------------------------------------------------------------------------ */

typedef struct phfem_server_s* phfem_server;

/* One request: an elliptic solve (kind 0) or a Crank-Nicolson run (kind 1)
 * with data f, u_D, g (and u0 for kind 1) given as constants, or per edge
 * midpoint in f_mid, bc_mid and u0_mid (time-independent for kind 1; each may
 * be NULL, and the constant is then used).  Every pointer is device memory
 * owned by the caller and must stay valid until the request is done.  With
 * levels > 0 the mesh is a coarse mesh that the server refines `levels` times
 * (phfem_mesh_refine) and solves on the finest mesh with the multigrid
 * preconditioner; a_T, U_out, Lambda_out and the midpoint arrays then refer
 * to the finest mesh (nT 4^levels triangles, nE its edges, in the
 * refinement's order). */
typedef struct {
  int32_t kind;            /* 0 elliptic, 1 Crank-Nicolson                               */
  int32_t nV, nT, nD, nN;
  const double* xy;        /* [nV][2]                                                      */
  const int32_t* tri;      /* [nT][3] counter-clockwise                                    */
  const int32_t* dirichlet;/* [nD][2]                                                      */
  const int32_t* neumann;  /* [nN][2]                                                      */
  const double* a_T;       /* [nT] or NULL (a = 1)                                         */
  double delta, f, uD, g;  /* reaction, source, Dirichlet value, Neumann flux (constants)  */
  double dt, u0;           /* kind 1: time step and initial value                          */
  int32_t steps;           /* kind 1: number of time steps                                  */
  int32_t precision;       /* PHFEM_FP64 or PHFEM_FP32_IR                                   */
  double* U_out;           /* [3 nT] or NULL: u_h at the vertices (final time for kind 1)  */
  double* Lambda_out;      /* [nE] or NULL (room for nE, the first nL written)             */
  int32_t levels;          /* 0: solve on the given mesh (Jacobi-PCG); > 0: see above      */
  int32_t reserved;
  const double* f_mid;     /* [nE] or NULL: f at the edge midpoints                         */
  const double* bc_mid;    /* [nE] or NULL: u_D on Dirichlet edges, g on Neumann edges (as
                              phfem_assemble's bc_mid)                                     */
  const double* u0_mid;    /* kind 1, [nE] or NULL: the initial midpoint values (u_D on
                              Dirichlet edges)                                             */
} phfem_request;

typedef struct {
  int64_t id;
  int32_t status;          /* phfem_status of the request once done                      */
  int32_t done;            /* 1 when finished                                              */
  int32_t iterations;      /* conjugate-gradient iterations (all steps)                    */
  int32_t slot;            /* worker slot that ran it (-1 while queued)                    */
  int32_t nE, nL;
  double rel_residual;
  double t_submit, t_admit, t_finish;  /* seconds since the server was created          */
  double bytes_reserved;   /* device bytes the admission reserved for the request          */
  int64_t bytes_peak;      /* device bytes the request's own allocations held at their peak */
  double t_dev_start, t_dev_end;  /* device time of the request's first and last work on its
                                     stream (the GPU's global timer), seconds since the server
                                     was created                                            */
  int32_t priority_class;  /* stream priority the request ran at: 0 highest (under 131,072
                              finest-mesh triangles), 1 (under 1,048,576), 2 lowest         */
  int32_t pad;
} phfem_result;

/* Creates a server on the current device with `slots` workers, each a host
 * thread with its own context and CUDA stream, so admitted requests overlap on
 * the GPU.  A request is admitted (first in, first out) when a slot is free
 * and its device-memory reservation fits in hbm_budget_bytes minus what
 * admitted requests hold; a request larger than the whole budget runs alone.
 * The reservation is the bytes per (finest-mesh) triangle that finished
 * requests of the same kind (elliptic or Crank-Nicolson, with or without
 * refinement) of at least 65,536 triangles actually allocated at their peak,
 * the largest seen, plus 10 % and 4 MB; before any has finished, 400 bytes per
 * triangle (600 with refinement) + 4 MB.  Each slot runs a request on a
 * stream whose priority falls with the request's size (three classes, see
 * phfem_result), so small requests are not held up behind the kernels of
 * large ones.  opts apply to every solve. */
PHFEM_API int phfem_server_create(int32_t slots, double hbm_budget_bytes, const phfem_solve_opts* opts,
                                  phfem_server* out);
/* Queues a request (copied) and returns its id; never blocks on the GPU. */
PHFEM_API int phfem_server_submit(phfem_server server, const phfem_request* req, int64_t* id);
/* Reads a request's record; wait != 0 blocks until it is done. */
PHFEM_API int phfem_server_poll(phfem_server server, int64_t id, int32_t wait, phfem_result* out);
/* Blocks until every submitted request is done. */
PHFEM_API int phfem_server_drain(phfem_server server);
/* Finishes the queued requests, then stops the workers and frees the server. */
PHFEM_API int phfem_server_destroy(phfem_server server);

/* ------------------------------------------------------------------------ */
/* Error report (Sec. 3.6 tables: L2 error, broken H1 error, mesh norm)     */
/* ------------------------------------------------------------------------ */

/* Quadrature of the report.  Triangles: a Duffy-collapsed nq x nq
 * Gauss-Legendre rule, point q = i nq + j at barycentric coordinates
 * (1 - s - t, s, t), s = x_i, t = x_j (1 - x_i), weight w_i w_j (1 - x_i)
 * times 2|T|, with (x_i, w_i) the nq-point Gauss-Legendre rule on [0, 1].
 * Multiplier edges (interior and Dirichlet, in multiplier order): the nq
 * Gauss-Legendre points from the initial to the end vertex of the edge. */
typedef struct {
  double L2;      /* ||u - u_h||_{L2}                                            */
  double H1semi;  /* broken ||grad_h (u - u_h)||_{L2}                             */
  double H1;      /* sqrt(L2^2 + H1semi^2)                                        */
  double M;       /* sqrt(sum_E |E| int_E (kappa - Lambda_E)^2) over the multiplier
                     edges: the mesh norm of the multiplier error; 0 without kappa */
} phfem_errors;

/* Writes the physical quadrature points where the caller evaluates the exact
 * solution (device buffers, each may be NULL):
 *   tri_xy  [nT][nq*nq][2] double   triangle points (x, y)
 *   edge_xy [nL][nq][2]    double   edge points
 *   edge_nu [nL][2]        double   unit normal of the edge pointing out of T+
 *                                   (the direction of Lambda)
 * 1 <= nq <= 16 (else PHFEM_EINVAL).  Asynchronous on the context's stream. */
PHFEM_API int phfem_error_points(phfem_mesh mesh, int32_t nq, double* tri_xy, double* edge_xy,
                                 double* edge_nu);

/* Integrates the errors of a solution (all device buffers):
 *   U [3nT]              element values at the vertices (phfem_solve's U)
 *   u_q [nT][nq*nq]      exact u at tri_xy
 *   grad_q [nT][nq*nq][2]  exact grad u at tri_xy
 *   Lambda [nL]          multipliers (phfem_solve's Lambda)
 *   kappa_q [nL][nq]     exact normal flux (A grad u) . nu at edge_xy
 * U, u_q and grad_q come together (or are all NULL: L2 = H1semi = H1 = 0);
 * so do Lambda and kappa_q (or M = 0).  Sums are FP64 in a fixed order.
 * Blocks the host until *out (host) is written. */
PHFEM_API int phfem_error_norms(phfem_mesh mesh, int32_t nq, const double* U, const double* u_q,
                                const double* grad_q, const double* Lambda, const double* kappa_q,
                                phfem_errors* out);

/* The locality order in which the Jacobi iteration stores the edge system
 * (not in the paper, whose numbering every other entry point keeps): edges
 * sorted by the Morton code of their midpoints on a 2^q x 2^q grid over the
 * vertices' bounding box (4 nE <= 4^q, q <= 15), ties in the paper's order.
 *   perm [nE] int32 (device, may be NULL): perm[i] = edge of internal row i
 *   n_overflow (host, may be NULL): rows whose four neighbours are not all
 *                within 32767 rows, stored with full indices
 * Builds the order on first use (also done by the first solve); blocks the
 * host until it is built. */
PHFEM_API int phfem_mesh_order(phfem_mesh mesh, int32_t* perm, int32_t* n_overflow);

/* ------------------------------------------------------------------------ */
/* Solve without device allocation                                           */
/* ------------------------------------------------------------------------ */

/* The paper has no counterpart of this entry point.  It exists for callers
 * that cannot allocate device memory while they call the library: programs
 * whose device memory is owned by another framework's pool or a fixed arena
 * (an allocation outside it would go uncounted or fail), and loops with a
 * latency or memory budget, where cudaMalloc may synchronise the device or
 * fail under memory pressure in the middle of a run.
 *
 * Jacobi-preconditioned conjugate gradients (FP64) on a symmetric positive
 * definite CSR system A x = rhs given by the caller, for instance the export
 * of phfem_sys_csr.  It allocates nothing: its temporaries live in one
 * fixed-size file-scope device array of the library (about 8 MB per device,
 * which every device that loads the library holds until the process exits).
 *   cuda_stream  cudaStream_t the work is ordered on (NULL = legacy stream)
 *   n            rows, 1 <= n <= PHFEM_NOALLOC_MAX_ROWS (else PHFEM_EINVAL)
 *   row_ptr [n+1], col [nnz] int32, val [nnz] double   the matrix (device);
 *                every row must hold a positive diagonal entry (else
 *                PHFEM_EINVAL)
 *   rhs [n] double (device); x [n] double (device): initial guess on entry,
 *                solution on return
 *   rtol         stop when the recursive residual r (updated by the
 *                iteration, r = rhs - A x in exact arithmetic; not recomputed
 *                from x) satisfies ||r||_2 <= rtol ||rhs||_2; <= 0 -> 1e-10
 *   max_iter     iteration limit; <= 0 -> 100000 (PHFEM_ENOCONV when reached)
 *   iterations, rel_residual   host outputs, may be NULL; rel_residual is
 *                ||r||_2 / ||rhs||_2 of that recursive residual
 * Every pointer must refer to memory of the current device.  The array is
 * shared by every call on a device and keeps the last call's contents; each
 * call clears the state that must start at zero.  Calls whose GPU work
 * overlaps (different streams or host threads without ordering between them)
 * race on it.  The first call on a device looks the array's device address up
 * (cudaGetSymbolAddress) with that device current.  The call returns once the
 * solve has finished: every 32 iterations it copies the iteration state to the
 * host and waits for its stream. */
#define PHFEM_NOALLOC_MAX_ROWS 262144
PHFEM_API int phfem_csr_pcg_noalloc(void* cuda_stream, int32_t n, const int32_t* row_ptr,
                                    const int32_t* col, const double* val, const double* rhs,
                                    double* x, double rtol, int32_t max_iter, int32_t* iterations,
                                    double* rel_residual);

#ifdef __cplusplus
}
#endif
#endif /* PHFEM_H */
