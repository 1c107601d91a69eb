/*
 * fe.h -- C ABI of libfe: matrix-free element-by-element (EBE) elasticity operator
 * on 10-node tetrahedra for R load cases at once, and the conjugate-gradient
 * solvers built on it, for NVIDIA GB300 (sm_103a).
 *
 * The method is that of Yamaguchi, Fujita, Ichimura, Hori, Lalith and Nakajima,
 * "Implicit Low-Order Unstructured Finite-Element Multiple Simulation Enhanced by
 * Dense Computation using OpenACC": static linear elasticity (Sec. 2, Eq. 1a-1c)
 * discretised with second-order tetrahedra into K u = f (Eq. 2); the product
 * f = sum_i Q_i K_i Q_i^T u with element matrices recomputed on every call from
 * node coordinates and material (Eq. 3); R right-hand sides solved together with
 * the case index innermost (Sec. 3.1); a flexible CG whose preconditioner is an
 * inner block-Jacobi CG run in single precision (Algorithm 1, Sec. 2).
 *
 * Conventions shared by every entry point:
 *   - Every function returns fe_status; none throws, aborts or traps. On failure
 *     fe_last_error() returns a message (thread-local, valid until the next call
 *     on the same thread).
 *   - Pointers named *_dev are device pointers on the mesh's device, owned by the
 *     caller, contiguous, aligned to at least 16 bytes. Host pointers are read
 *     during the call only.
 *   - Multi-vectors are laid out [node][case][component] ("[N][R][3]"): the 3R
 *     values of one node are contiguous, so neighbouring threads that work on
 *     different cases of one node touch neighbouring addresses.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream). Work is
 *     stream-ordered and asynchronous unless stated otherwise.
 *   - Element geometry is straight-sided: the element map is affine, defined by
 *     the 4 corner nodes; edge nodes must lie at the midpoints of their edges.
 *   - Node order inside an element is VTK's: corners 0..3, then the midpoints of
 *     edges (0,1), (1,2), (2,0), (0,3), (1,3), (2,3).
 *   - Dirichlet conditions are homogeneous: constrained DOFs hold u = 0, and the
 *     operator applied is K_bc = P K P + (I - P), P = diag(free mask).
 */
#ifndef FE_H_
#define FE_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FE_OK = 0,
  FE_EINVAL = 1,      /* invalid argument or mesh; nothing was launched */
  FE_ENOMEM = 2,      /* device or host allocation failed */
  FE_ECUDA = 3,       /* a CUDA call failed (message has the CUDA error) */
  FE_ENOCONV = 4,     /* a solve hit its iteration cap before the tolerance */
  FE_EBREAKDOWN = 5,  /* a solve met a non-positive curvature or a NaN/Inf */
  FE_ETIMEOUT = 6     /* a bounded device-side wait gave up (reported by fe_mesh_device_status):
                         the warp-specialised EBE kernel hands tiles between its warps on
                         mbarriers, and the persistent inner-loop kernel of the solvers
                         meets at grid-wide barriers; each wait is limited to about one
                         second of SM clock, and a wait that runs out records it on the mesh
                         and the kernel finishes without waiting again, so its results are
                         not to be used */
} fe_status;

typedef enum { FE_F64 = 0, FE_F32 = 1 } fe_dtype;

typedef enum {
  FE_SOLVER_PCG64 = 0,      /* FP64 CG with 3x3 block Jacobi (the plain baseline) */
  FE_SOLVER_FCG_MIXED = 1,  /* FP64 flexible CG, FP32 inner block-Jacobi CG at level 0 (Algorithm 1) */
  FE_SOLVER_FCG_MG = 2,     /* as FCG_MIXED, with the TET4 inner loop (level 1) before level 0 */
  FE_SOLVER_FCG_AMG = 3     /* Algorithm 1 in full: inner loops at levels 2 (aggregation of the TET4
                               level), 1 and 0; needs the assembled coarse matrices */
} fe_solver;

typedef struct fe_mesh fe_mesh;   /* opaque, library-owned */

/* Solver options (Algorithm 1; inner-loop defaults from the paper's table of
 * loop settings, level 0: tolerance 0.1, 30 iterations). */
typedef struct {
  int32_t solver;        /* fe_solver */
  double tol;            /* stop case r when ||f_r - K u_r|| / ||f_r|| <= tol (1e-8) */
  int32_t max_outer;     /* cap on outer iterations (PCG64: CG iterations) */
  int32_t n_inner;       /* cap on inner steps per outer iteration (30) */
  double eps_inner;      /* inner stop: max over active cases ||e||^2/||rbar||^2 <= eps_inner (0.1) */
  int32_t use_graph;     /* 1: replay one outer iteration from a captured CUDA graph */
  int32_t literal_beta;  /* 1: the printed beta = (z,q)/rho; 0: flexible CG beta (default) */
  int32_t check_every;   /* outer iterations between host reads of the convergence flags (>= 1) */
  int32_t verbose;       /* reserved, 0 */
  int32_t n_inner1;      /* FCG_MG: cap on level-1 (TET4) inner steps per outer iteration (300) */
  double eps_inner1;     /* FCG_MG: level-1 inner stop, the same rule as eps_inner (0.05) */
  int32_t coarse_op;     /* FCG_MG level-1 operator: 0 assembled when it fits, else element by
                            element (default); 1 assembled (FE_EINVAL if it does not fit);
                            2 element by element */
  int32_t n_inner2;      /* FCG_AMG: cap on level-2 inner steps per outer iteration (3000) */
  double eps_inner2;     /* FCG_AMG: level-2 inner stop, the same rule as eps_inner (0.025) */
  double* cg_coef;       /* PCG64 only, optional (NULL: not recorded): host double
                            [cg_coef_len][R][2] receiving (alpha_k, beta_k) of CG iteration k
                            of every case (0 after the case stopped); the coefficients give
                            the Lanczos tridiagonal of M^-1 K, hence condition estimates */
  int32_t cg_coef_len;   /* iterations cg_coef holds */
  int32_t inner_kernel;  /* inner loops on the assembled levels 1 and 2 (R = 4, 8, 16 or 32):
                            1 one launch per vector pass and scalar step (default; the
                            faster on GB300, the step being bound by its vector traffic);
                            0 one persistent cooperative kernel per loop (its CTAs meet at
                            grid-wide barriers with bounded waits, see FE_ETIMEOUT) */
} fe_solve_opts;

/* Per-case results of fe_pcg_solve. */
typedef struct {
  int32_t outer_iters;   /* outer iterations (PCG64: CG iterations) this case took */
  int32_t inner_iters;   /* inner steps summed over outer iterations (0 for PCG64) */
  double relres;         /* true relative residual ||f - K u|| / ||f|| at exit (FP64 product) */
  int32_t status;        /* FE_OK, FE_ENOCONV or FE_EBREAKDOWN for this case */
  int32_t inner1_iters;  /* level-1 (TET4) inner steps summed over outer iterations (FCG_MG, FCG_AMG) */
  int32_t inner2_iters;  /* level-2 inner steps summed over outer iterations (FCG_AMG) */
  int32_t pad;
} fe_solve_stats;

/* Message of the last failure on this thread ("" if none). */
const char* fe_last_error(void);

/* Library version string. */
const char* fe_version(void);

/* Fills opts with the defaults: FCG_MIXED, tol 1e-8, max_outer 20000, n_inner 30,
 * eps_inner 0.1, use_graph 1, literal_beta 0, check_every 1, n_inner1 300,
 * eps_inner1 0.05, n_inner2 3000, eps_inner2 0.025 (the paper's table of loop settings,
 * levels 0, 1 and 2), coarse_op 0, cg_coef NULL, cg_coef_len 0, inner_kernel 1. */
void fe_solve_opts_default(fe_solve_opts* opts);

/*
 * fe_mesh_create -- validate a TET10 mesh and make its device copy.
 *   n_nodes, coords   host double [N][3], metres
 *   n_elem, conn      host int32 [E][10], 0-based node ids, VTK order
 *   young, poisson    host double [E]: Young's modulus (Pa, > 0) and Poisson ratio
 *                     (-1 < nu < 0.5) per element (isotropic C_ijkl of Eq. 1b)
 *   free_mask         host uint8 [N][3]: 1 = free DOF, 0 = fixed at zero
 *   device            CUDA device ordinal the mesh lives on
 *   stream            stream for the uploads (the call returns after they finish)
 * Checks: sizes, finite values, node ids in range and distinct within an
 * element, positive volumes, edge nodes at midpoints (relative 1e-6 of the
 * element's size), material ranges. Returns FE_EINVAL with a message naming the
 * first offending element or node. *out receives the handle (NULL on failure).
 */
fe_status fe_mesh_create(int64_t n_nodes, const double* coords, int64_t n_elem, const int32_t* conn,
                         const double* young, const double* poisson, const uint8_t* free_mask,
                         int32_t device, void* stream, fe_mesh** out);

/* Releases every device resource of the mesh (synchronises the device). NULL is a no-op. */
void fe_mesh_destroy(fe_mesh* mesh);

/*
 * fe_mesh_device_status -- synchronises `stream`, then reads and clears the mesh's
 * device status word. Returns FE_ETIMEOUT if a kernel launched on this mesh since
 * the last call gave up a bounded wait (its products are then invalid), FE_OK
 * otherwise. fe_ebe_apply does not read it on its own (that would synchronise
 * every call); fe_pcg_solve and fe_solve_many read it when they finish and then
 * return FE_ETIMEOUT.
 */
fe_status fe_mesh_device_status(const fe_mesh* mesh, void* stream);

/*
 * fe_wait_selftest -- exercises one kind of bounded device-side wait with a wait that
 * nothing ends (no counterpart in the paper; a test of the failure path without a
 * GPU fault). which = 0: the mbarrier wait of the warp-specialised EBE kernel, one
 * warp; which = 1: the grid-wide barrier of the persistent inner-loop kernel, two
 * blocks of which only one arrives. The wait gives up after `cycles` SM clock cycles
 * (1 .. 2^32; 2^21 is about a millisecond) and sets the mesh's status word, so the
 * next fe_mesh_device_status returns FE_ETIMEOUT. which = 1 synchronises `stream`.
 * FE_EINVAL for a NULL mesh or arguments out of range (nothing is launched).
 */
fe_status fe_wait_selftest(const fe_mesh* mesh, int32_t which, int64_t cycles, void* stream);

/* Node and element counts of a mesh. */
fe_status fe_mesh_info(const fe_mesh* mesh, int64_t* n_nodes, int64_t* n_elem);

/*
 * fe_mesh_set_log_young -- replace the per-element Young's moduli by exp(logE).
 * logE_dev: device double [E]. The block-Jacobi preconditioner is rebuilt on
 * the next solve. Used by gradient checks and by the adjoint workflow
 * (m_e = log E_e, Poisson ratio unchanged).
 */
fe_status fe_mesh_set_log_young(fe_mesh* mesh, const double* logE_dev, void* stream);

/*
 * fe_ebe_apply -- y = K_bc x for R cases (Eq. 3 with the multiple-vector layout
 * of Sec. 3.1).
 *   R        number of cases, 1 <= R <= 64
 *   dtype    FE_F64: double vectors, FP64 arithmetic;
 *            FE_F32: float vectors, FP32 arithmetic and FP32 accumulation
 *   x_dev    device [N][R][3] of dtype, read only
 *   y_dev    device [N][R][3] of dtype, overwritten; must not alias x_dev
 * Element matrices are never stored: each call recomputes the element geometry
 * and Lame constants from the node coordinates and (E, nu). Summation order of
 * the element contributions is not fixed (atomic accumulation), so results are
 * reproducible to rounding only.
 */
fe_status fe_ebe_apply(const fe_mesh* mesh, int32_t R, fe_dtype dtype, const void* x_dev, void* y_dev,
                       void* stream);

/*
 * fe_ebe_apply_host -- fe_ebe_apply with x and y in HOST memory: x_host is copied
 * to the device, the product runs there, and y is copied back to y_host.
 *   x_host, y_host  host [N][R][3] of dtype; page-locked memory (cudaHostAlloc,
 *                   cudaHostRegister, torch pin_memory) lets the copies run
 *                   asynchronously and overlap; pageable memory also works
 * Stream-ordered and asynchronous: the call returns once the work is queued.
 * x_host must hold the input when the call is made and must not change, and
 * y_host must not be read, until `stream` reaches the end of the call
 * (synchronise it). The copy-in does not wait for work queued earlier on
 * `stream`. The library keeps two device buffer sets and its own copy and
 * compute streams with the mesh, used by alternate calls, so that consecutive
 * calls overlap the copy-in of one, the product of the previous one and the
 * copy-out of the one before (the host<->device link and the GPU work in
 * parallel). Not safe for concurrent calls on the same mesh from several threads.
 */
fe_status fe_ebe_apply_host(fe_mesh* mesh, int32_t R, fe_dtype dtype, const void* x_host, void* y_host, void* stream);

/* EBE kernel variants (all compute fe_ebe_apply's result):
 *   FE_EBE_DIRECT  one thread per (element, case), inputs gathered from global
 *                  memory, results added with global atomics (the paper's GPU
 *                  port keeps atomics rather than element colouring, Sec. 3.2.2);
 *   FE_EBE_TILED   consecutive elements (in the library's locality order) form a
 *                  tile; the tile's node values are staged in shared memory, the
 *                  element products accumulate there with shared-memory atomics,
 *                  and each tile node gets one global atomic add per value;
 *   FE_EBE_GATHER  tiles as above, but without atomics inside the tile: every
 *                  element-case product is written to its own shared-memory slot,
 *                  then each tile node sums the slots of its incident elements
 *                  and issues one 16-byte global atomic add per 16 bytes of
 *                  values (R in {1, 2, 3, 4, 8, 16, 32});
 *   FE_EBE_GATHER_DF  FP64 products only (R in {2, 4, 8, 16, 32}): the gather
 *                  kernel with the element arithmetic and node sums in float-float
 *                  (pairs of FP32 values, about 48 significant bits) on the FP32
 *                  pipe, FP64 inputs, outputs and atomics; GB300 runs FP64
 *                  arithmetic at 1/61 of its FP32 rate;
 *   FE_EBE_GATHER_X2  FP32 products only (R in {4, 8, 16, 32}): the gather
 *                  kernel with each thread computing two cases of one element
 *                  (r and r + R/2) in paired FP32 instructions (two lanes per
 *                  multiply-add), sharing the element's geometry between them;
 *   FE_EBE_COLOUR  elements coloured so that no two of one colour share a node
 *                  (greedy, built on first use); one launch per colour, one
 *                  thread per (element, case), results added into y with plain
 *                  loads and stores instead of atomics (the scatter by element
 *                  colouring of the paper's K-computer design, Sec. 3.2.2).
 *                  Deterministic: the same inputs give bitwise the same y.
 *                  fe_ebe_set_variant ignores tile_elems; fe_ebe_get_variant
 *                  returns the number of colours there;
 *   FE_EBE_WS      FP32 products only (R in {4, 8, 16, 32}; tile_elems * R / 2 a
 *                  multiple of 32, at most 384): warp-specialised kernel, one
 *                  block per SM. Compute warps evaluate two cases of an element per
 *                  thread in paired FP32 instructions; staging warps bring in each
 *                  tile's packet (node ids and coordinates, materials, offsets) with
 *                  one bulk copy, load the tile's node values, compute the element
 *                  geometry and sum each tile node's element slots into y (one
 *                  16-byte atomic add per 4 values). Tiles are grown greedily (each
 *                  takes the element sharing most nodes with it, up to a node
 *                  budget), built per (tile_elems, R) on first use;
 *   FE_EBE_DF_LEAN FP64 products only (R in {2, 4, 8, 16, 32}): the float-float
 *                  kernel with a register-light element routine (node values and
 *                  geometry read from shared memory where they are used, outputs
 *                  stored as they are formed) and one input stage, so that two
 *                  blocks share an SM and hide each other's latency;
 *   FE_EBE_WS2     FE_EBE_WS with 256-thread blocks, two per SM (at most 4 compute
 *                  warps, so tile_elems * R / 2 in {32, 64, 96, 128}): each block's
 *                  staging and compute phases fill the other's waits. */
typedef enum {
  FE_EBE_DIRECT = 0,
  FE_EBE_TILED = 1,
  FE_EBE_GATHER = 2,
  FE_EBE_GATHER_DF = 3,
  FE_EBE_GATHER_X2 = 4,
  FE_EBE_COLOUR = 5,
  FE_EBE_WS = 6,
  FE_EBE_DF_LEAN = 7,
  FE_EBE_WS2 = 8
} fe_ebe_variant;

/*
 * fe_ebe_set_variant -- choose the kernel fe_ebe_apply (and the solvers) use for
 * (R, dtype) on this mesh. tile_elems (1..4096) applies to FE_EBE_TILED; the
 * tiling is built on first use (host work, synchronous on `stream`). Fails with
 * FE_EINVAL if the tile's shared-memory footprint exceeds the device limit.
 */
fe_status fe_ebe_set_variant(fe_mesh* mesh, int32_t R, fe_dtype dtype, int32_t variant, int32_t tile_elems,
                             void* stream);

/* Current kernel for (R, dtype): *variant (fe_ebe_variant) and *tile_elems (0 for direct). */
fe_status fe_ebe_get_variant(const fe_mesh* mesh, int32_t R, fe_dtype dtype, int32_t* variant,
                             int32_t* tile_elems);

/*
 * fe_ebe_tune -- autotuner: times the direct kernel and the tiled and gather
 * kernels over a range of tile sizes (where they fit) for (R, dtype) on this
 * mesh, using library-owned scratch vectors, and selects the fastest.
 * Synchronous. *variant receives kind * 65536 + elements per tile of the choice
 * (0 = direct); *us its time per product in microseconds.
 */
fe_status fe_ebe_tune(fe_mesh* mesh, int32_t R, fe_dtype dtype, void* stream, int32_t* variant, int32_t* us);

/*
 * fe_pcg_solve -- solve K_bc u_r = f_r for R cases at once (Algorithm 1 with the
 * inner loop at level 0 only, or plain block-Jacobi PCG).
 *   f_dev    device double [N][R][3]; constrained entries are ignored (treated as 0)
 *   u_dev    device double [N][R][3]; in: initial guess, out: solution
 *   opts     host; NULL = defaults
 *   stats    host [R], written on return
 * Synchronous: returns when u and stats are final. Each case stops on its own
 * (per-case masking): once ||f_r - K u_r||/||f_r|| <= tol, checked with an FP64
 * product, its vectors are frozen. Cases with f_r = 0 return u_r = 0 at once.
 * Returns FE_OK when every case converged, FE_ENOCONV if any hit max_outer, or
 * FE_EBREAKDOWN if any broke down; u then holds the last iterate of each case.
 * Library-owned workspace (about 12 vectors of [N][R][3], FP64 and FP32) is
 * allocated on first use per R and kept with the mesh.
 */
fe_status fe_pcg_solve(const fe_mesh* mesh, int32_t R, const double* f_dev, double* u_dev,
                       const fe_solve_opts* opts, fe_solve_stats* stats, void* stream);

/*
 * fe_solve_many -- solve K_bc u_c = f_c for n_cases load cases with at most R
 * cases in flight (the many-case workload of Sec. 5, where Green's functions of
 * hundreds of unit slips are computed in batches). The cases stream through R
 * slots of one batched solve: when a case converges (or stops), its solution is
 * stored and its slot is refilled with the next pending case between two outer
 * iterations, so one slow case does not hold back a whole batch.
 *   f_dev    device double [n_cases][N][3] (case-major), read only
 *   u_dev    device double [n_cases][N][3], out (every case starts from u = 0)
 *   R_slots  cases in flight, 1..64; 0 = choose from free device memory: the
 *            largest of 32, 16, 8, 4, 2, 1 whose solver vectors fit in 70 % of it
 *   opts     as fe_pcg_solve (NULL = defaults)
 *   stats    host [n_cases], per case
 *   R_used   host, receives the slot count used (may be NULL)
 * Synchronous. Tunes the EBE kernels for R (FP32 and FP64) and for the single-
 * case FP64 true-residual product on first use. Allocates two [N][R][3] slot
 * buffers plus the solver workspace. Returns FE_OK when every case converged,
 * else FE_ENOCONV or FE_EBREAKDOWN (per-case status in stats).
 */
fe_status fe_solve_many(const fe_mesh* mesh, int32_t n_cases, const double* f_dev, double* u_dev, int32_t R_slots,
                        const fe_solve_opts* opts, fe_solve_stats* stats, int32_t* R_used, void* stream);

/*
 * fe_block_jacobi -- the 3x3 block-Jacobi preconditioner M^-1 = diag3x3[K_bc]^-1
 * of Algorithm 1 and of the PCG baseline, built on first use from
 * the element matrices' diagonal blocks (closed form, FP64) with constrained
 * rows and columns set to the identity.
 *   binv_dev  device double [N][3][3], overwritten with the inverse blocks
 * Fails with FE_EINVAL if a free node has a singular or indefinite block.
 */
fe_status fe_block_jacobi(const fe_mesh* mesh, double* binv_dev, void* stream);

/*
 * fe_block_jacobi_noalloc -- fe_block_jacobi's result without allocating device
 * memory. The paper has no counterpart; this exists for callers that cannot
 * allocate where they need the preconditioner: latency-critical loops that must
 * not take the allocator's lock, and processes whose device memory is held by
 * another allocator's pool (a framework's caching allocator), where a fresh
 * cudaMalloc can fail mid-run.
 *   binv_dev  device double [N][3][3], overwritten with the inverse blocks
 * Scratch lives in a fixed file-scope device array (about 13.5 MiB, held on every
 * GPU that loads the library until the process exits), so the mesh may have at
 * most 131,072 nodes; larger meshes get FE_EINVAL and nothing is launched.
 * Recomputes the blocks on every call (the mesh's own copy is not touched).
 * The call synchronises `stream`: it copies an error flag back to the host and
 * returns only when the blocks are written. The first call on a device looks up
 * the array's device address (set-up, once per device) and keeps it for the life
 * of the process; make that first call before any stream capture. The kept address
 * does not survive a reset of the device's primary context (cudaDeviceReset): do
 * not call this after one. All calls share the one array: calls whose work
 * overlaps on the GPU (different streams or threads) race and must be serialised
 * by the caller.
 */
fe_status fe_block_jacobi_noalloc(const fe_mesh* mesh, double* binv_dev, void* stream);

/*
 * fe_adjoint_grad -- element sensitivities for m_e = log E_e:
 *   g_e = - sum_r (P lambda_r)_e^T K_e (P u_r)_e
 * which is dJ/dm_e when K_bc lambda_r = dJ/du_r (adjoint state) and
 * K_bc u_r = f_r. No counterpart in the paper (it is an addition of this
 * library); the element product is the same EBE kernel, reduced per element
 * instead of scattered.
 *   u_dev, lambda_dev  device double [N][R][3]
 *   g_elem_dev         device double [E], overwritten
 */
fe_status fe_adjoint_grad(const fe_mesh* mesh, int32_t R, const double* u_dev, const double* lambda_dev,
                          double* g_elem_dev, void* stream);

/*
 * Vector steps of the misfit gradient around fe_adjoint_grad (no counterpart in
 * the paper; the paper's Sec. 5 computes the Green's functions u_k of unit slips,
 * this completes a least-squares inversion workflow over them). All arrays FP64.
 *
 * fe_obs_create -- observation operator u_obs[p] = sum_j w[p][j] u[node[p][j]]
 * (for instance quadratic interpolation on the surface triangle holding each
 * observation point).
 *   n_obs, n_per   observations and nodes per observation (1..64)
 *   node, weight   host int32 / double [n_obs][n_per], node ids of the mesh (checked
 *                  on the host; FE_EINVAL names the first bad entry)
 * The operator lives on the mesh's device; release it with fe_obs_destroy.
 */
typedef struct fe_obs fe_obs;     /* opaque, library-owned */
fe_status fe_obs_create(const fe_mesh* mesh, int64_t n_obs, int32_t n_per, const int32_t* node,
                        const double* weight, fe_obs** out);
void fe_obs_destroy(fe_obs* obs);

/* u_obs_dev [n_obs][R][3] = Obs u_dev [N][R][3] (each value summed in a fixed order). */
fe_status fe_obs_apply(const fe_obs* obs, int32_t R, const double* u_dev, double* u_obs_dev, void* stream);

/* out_dev [N][R][3] = P Obs^T g_dev, g_dev [n_obs][R][3]: the adjoint right-hand side
 * of a misfit of the observations; constrained DOFs are zero. Overwrites out_dev;
 * sums in atomic order (reproducible to rounding). */
fe_status fe_obs_adjoint(const fe_mesh* mesh, const fe_obs* obs, int32_t R, const double* g_dev, double* out_dev,
                         void* stream);

/* u_dev [N][3] = sum_r a_dev[r] G_dev[:, r, :] for G_dev [N][R][3] (the displacement
 * of source amplitudes a from the Green's functions of R sources). */
fe_status fe_combine_cases(const fe_mesh* mesh, int32_t R, const double* G_dev, const double* a_dev, double* u_dev,
                           void* stream);

/* out_dev[r] = (P f_r) . lam for f_dev [N][R][3], lam_dev [N][3]: dJ/da_r for sources
 * f_r whose amplitudes a_r scale them, with lam the adjoint state. Overwrites out_dev
 * [R]; block partial sums added atomically (reproducible to rounding). */
fe_status fe_case_dots(const fe_mesh* mesh, int32_t R, const double* f_dev, const double* lam_dev, double* out_dev,
                       void* stream);

/*
 * TET4 coarse level (Sec. 2 and Algorithm 1(a): inner loop level 1).
 * The coarse mesh is the TET10 mesh without its edge nodes: same elements and
 * materials, first-order shape functions. Its nodes are the corner nodes of the
 * TET10 mesh numbered in increasing TET10 id (internal numbering of this
 * library's mesh). P1 maps coarse to fine values by linear interpolation: a
 * corner keeps its value, an edge node takes the mean of its two ends. Both
 * transfers keep Dirichlet DOFs at zero (fine DOFs after P1, coarse DOFs after
 * P1^T; a coarse node's DOF is fixed iff it is fixed on its TET10 node), and the
 * coarse operator is K1_bc = P K1 P + (I - P) with the coarse mask P, which
 * equals P1^T K_bc P1 restricted to free coarse DOFs when K is built from
 * TET10 elements whose displacement is linear (Galerkin consistency).
 * The coarse structure is built on first use (host, O(N + E)) and kept with the
 * mesh; vectors are [N4][R][3] like the fine ones.
 */

/* fe_coarse_info -- builds the coarse level if needed.
 *   n_nodes4     host, receives N4 (may be NULL)
 *   vertex_host  host int32 [N4], receives the TET10 node id of each coarse node
 *                (may be NULL)
 * Synchronous. */
fe_status fe_coarse_info(const fe_mesh* mesh, int64_t* n_nodes4, int32_t* vertex_host, void* stream);

/* fe_ebe4_apply -- y4 = K1_bc x4 for R cases, element by element (the first-order
 * EBE product of Sec. 3.2 on the coarse mesh; fixed DOFs: y = x).
 *   x4, y4   device [N4][R][3] of dtype, 16-byte aligned, not aliased; y4 overwritten
 * Asynchronous on `stream`. */
fe_status fe_ebe4_apply(const fe_mesh* mesh, int32_t R, fe_dtype dtype, const void* x4, void* y4, void* stream);

/* fe_coarse_apply -- y4 = K1_bc x4 for R cases in FP32 with K1_bc assembled in
 * 3x3 block CSR (FP64 assembly, FP32 values; built on first use and again after
 * fe_mesh_set_log_young). This is the level-1 operator of the FCG_MG solver
 * whenever the matrix (about 36 bytes per block, 15 blocks per coarse node, plus
 * a temporary FP64 copy) fits in a quarter of the free device memory; otherwise
 * the solver uses the element-by-element product. Fails with FE_EINVAL if the
 * matrix does not fit.
 *   x4, y4   device float [N4][R][3], 16-byte aligned, not aliased; y4 overwritten
 * Asynchronous on `stream` after the first call. */
fe_status fe_coarse_apply(const fe_mesh* mesh, int32_t R, const float* x4, float* y4, void* stream);

/* fe_coarse_restrict -- r4 = P (P1^T r10): r10 device [N][R][3], r4 device
 * [N4][R][3] overwritten (fixed coarse DOFs 0). Asynchronous on `stream`. */
fe_status fe_coarse_restrict(const fe_mesh* mesh, int32_t R, fe_dtype dtype, const void* r10, void* r4,
                             void* stream);

/* fe_coarse_prolong -- u10 = P (P1 u4): u4 device [N4][R][3], u10 device
 * [N][R][3] overwritten (fixed fine DOFs 0). Asynchronous on `stream`. */
fe_status fe_coarse_prolong(const fe_mesh* mesh, int32_t R, fe_dtype dtype, const void* u4, void* u10,
                            void* stream);

/* fe_coarse_block_jacobi -- the level-1 block Jacobi M1^-1 = diag3x3[K1_bc]^-1
 * (Algorithm 1(a), set-up) from the closed form of the TET4 diagonal blocks,
 * V [(lam + mu) g_a g_a^T + mu |g_a|^2 I], built on first use (FP64).
 *   binv4_dev  device double [N4][3][3], overwritten
 * Fails with FE_EINVAL if a free coarse node has a singular block. */
fe_status fe_coarse_block_jacobi(const fe_mesh* mesh, double* binv4_dev, void* stream);

/*
 * Level 2 (Sec. 2 and Algorithm 1(a): inner loop level 2), an algebraic
 * coarsening of the TET4 level: the coarse nodes are aggregated over the graph
 * of K1's block pattern in two passes in node order (a node with no aggregated
 * neighbour starts an aggregate of itself and its neighbours; each remaining
 * node joins the first-pass aggregate of its lowest-numbered neighbour that has
 * one). P2 copies an aggregate's value to its members' free DOFs, P2^T sums the
 * members' free values, and A2 = P2^T K1_bc P2 on aggregate DOFs with a free
 * member (identity on the others), assembled in FP64 and stored in FP32 3x3
 * block CSR. Built on first use with the assembled coarse matrix (values again
 * after fe_mesh_set_log_young). Vectors are [NA][R][3] FP32.
 */

/* fe_level2_info -- builds level 2 if needed; *n_agg receives NA, agg_host (host
 * int32 [N4], may be NULL) the aggregate of each coarse node. Synchronous. Fails
 * with FE_EINVAL if the coarse matrices do not fit in a quarter of free memory. */
fe_status fe_level2_info(const fe_mesh* mesh, int64_t* n_agg, int32_t* agg_host, void* stream);

/* fe_coarse_matrix_info -- builds the assembled coarse matrices if needed (as
 * fe_level2_info) and returns their block counts: *n_blocks1 of K1_bc, *n_blocks2
 * of A2 (either may be NULL). Synchronous. */
fe_status fe_coarse_matrix_info(const fe_mesh* mesh, int64_t* n_blocks1, int64_t* n_blocks2, void* stream);

/* fe_level2_apply -- y2 = A2 x2, R cases, device float [NA][R][3], not aliased. */
fe_status fe_level2_apply(const fe_mesh* mesh, int32_t R, const float* x2, float* y2, void* stream);

/* fe_level2_restrict -- r2 = P2^T r4: r4 device float [N4][R][3], r2 [NA][R][3]. */
fe_status fe_level2_restrict(const fe_mesh* mesh, int32_t R, const float* r4, float* r2, void* stream);

/* fe_level2_prolong -- u4 = P2 u2: u2 device float [NA][R][3], u4 [N4][R][3]. */
fe_status fe_level2_prolong(const fe_mesh* mesh, int32_t R, const float* u2, float* u4, void* stream);

/* fe_level2_block_jacobi -- the level-2 block Jacobi diag3x3[A2]^-1 (Algorithm 1(a),
 * set-up), device double [NA][3][3], overwritten. */
fe_status fe_level2_block_jacobi(const fe_mesh* mesh, double* binv2_dev, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* FE_H_ */
