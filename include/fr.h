/*
 * fr.h -- C ABI of the GB300 (sm_103a) library for h-adaptive flux reconstruction (FR) of the
 * compressible Euler equations on Morton-ordered linear quadtrees (2D) and octrees (3D), after
 * Wang, Witherden & Jameson, "An efficient GPU-based h-adaptation framework via linear trees for
 * the flux reconstruction method" (arXiv 2306.06744).
 *
 * Everything a call computes runs in this library's CUDA kernels on the caller's stream.
 * The library owns every device buffer of a mesh.  Host arrays passed in or out are owned by
 * the caller and are read or written before the call returns (the call synchronises its stream
 * for them).  Calls on one mesh are not thread-safe; different meshes are independent.
 *
 * Canonical layouts (identical for input and output):
 *   key   : uint64 Morton ID (Sec. 2.2, Algorithm 1): the anchor's interleaved coordinate bits at
 *           the octant's depth D, most significant level first and, inside a level, z above y
 *           above x; then dim*(Dmax-D) zero bits; then D in m_b = ceil(log2(Dmax+1)) bits.
 *           Anchors count cells of the finest level Dmax.  Sorted ascending, ancestors sort
 *           before descendants and a first child is its parent's key plus one (Sec. 3.2).
 *   box   : int32[4] = (depth, x, y, z), anchor in finest-level cells (z = 0 in 2D).
 *   u     : double[M][nv][N], nv = dim+2 conserved variables (rho, rho*u, rho*v, [rho*w], E),
 *           N = (p+1)^dim Gauss-Legendre solution points, point i = ix + n*iy + n*n*iz.
 *   faces : f = 2*axis + side (side 0 = minus face); the matching face of a neighbour is f^1.
 *   conn  : per element and face (int32 nbr, int8 ftype, int8 slot): ftype 0 conforming (slot
 *           -1); 1 = this element is the fine side of a 2:1 hanging face, nbr is the coarse
 *           element and slot its position on the coarse face (child bits along the in-face axes,
 *           lower axis least significant, Sec. 3.3); 2 = this element is the coarse side, nbr is
 *           the slot-0 fine element (slot 0).
 *
 * Errors: every int-returning call returns 0 on success or one of the negative FR_E* codes; the
 * message is available from fr_last_error(mesh) (or fr_last_error(NULL) for calls without a
 * mesh).  No call traps or aborts on bad input.
 */
#ifndef FR_GB300_H
#define FR_GB300_H
#include <stddef.h>
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

#define FR_OK 0
#define FR_EINVAL (-1)    /* bad argument, layout or configuration                        */
#define FR_ENOMEM (-2)    /* device allocation failed                                       */
#define FR_EOVERFLOW (-3) /* caller capacity too small (required size written back)        */
#define FR_ETIMEOUT (-4)  /* a bounded device wait gave up (tensor-core completion, about 1 s) */
#define FR_ECUDA (-5)     /* CUDA runtime error                                             */

typedef struct fr_mesh fr_mesh;

/* Optional device allocator (e.g. a framework's caching allocator).  alloc returns a device
   pointer usable on `stream`, or NULL on failure; free releases it in stream order.  With a NULL
   allocator the library uses cudaMallocAsync / cudaFreeAsync on the mesh's stream. */
typedef struct {
  void* (*alloc)(size_t bytes, void* stream, void* ctx);
  void (*free)(void* ptr, void* stream, void* ctx);
  void* ctx;
} fr_allocator;

/* Problem set-up (Sec. 2.1 and Sec. 5.2).  All fields are read at fr_mesh_init only. */
typedef struct {
  int32_t dim, p;          /* dim 2 or 3; polynomial degree p in 1..4                             */
  double L;                /* periodic domain [0,L]^dim                                           */
  int32_t Dbase, Dmax;     /* coarsest depth (uniform start, coarsening limit) and finest depth   */
  double gamma;            /* ratio of specific heats                                             */
  int32_t nvort;           /* number of vortices (>= 0)                                           */
  const double* vort;      /* host [nvort][4]: x centre, y centre, strength beta, core radius     */
  double uinf[3];          /* freestream velocity (the vortices move with it)                     */
  double rho_inf, p_inf;   /* freestream density and pressure                                     */
  double cfl, dt;          /* dt > 0 fixes the time step; otherwise dt = cfl*h(Dmax)/((2p+1)*smax)
                              with smax the largest |v|+c of the initial state                    */
  int32_t adapt_every;     /* fr_run adapts after every adapt_every steps (0: never)              */
  int32_t indicator;       /* 0: density gradient eta = h*max|grad rho| (refine if eta >
                              th_refine, coarsen if eta < th_coarsen); 1: analytic centre of
                              Sec. 5.2 (th_refine, th_coarsen are the radii 5 and 6 of the paper);
                              2: external flags only; 3: learned indicator set by
                              fr_set_learned_indicator, density gradient until weights are set   */
  double th_refine, th_coarsen;
  int32_t precision;       /* arithmetic of the time-step kernels (state, norms and adaptation are
                              always FP64): 0 FP64; 1 FP32 fluxes, operators, traces and common
                              fluxes with the Runge-Kutta combination in FP64; 2 as 1 with the
                              element's flux-derivative contraction on the tensor cores in TF32
                              (FP32 accumulation); 3 the same in split BF16 (bf16x3: hi*hi +
                              hi*lo + lo*hi, FP32 accumulation); 4 double-word (two-float, ~48-bit
                              significand) on the FP32 pipes.  2 and 3 are built for dim 3, p 3
                              (64-point hexahedra, Sec. 2.1's operator as 16 x 16 Kronecker blocks);
                              other dim/p return FR_EINVAL.  A tensor-core completion wait that
                              gives up is reported as FR_ETIMEOUT by the next fr_adapt/fr_run
                              adaptation                                                          */
  int32_t init_passes;     /* < 0: Dmax-Dbase passes of {closed-form state, flags, adaptation}    */
} fr_config;

typedef struct {
  double t, l2_rho;     /* time and L2 norm of the density error against the closed form (Sec. 5.2) */
  double integral[5];   /* domain integral of each conserved variable (GL quadrature x |J|)        */
  double min_rho, min_p;
  int64_t M;
} fr_norms_out;

typedef struct {
  int64_t M_old, M_new;
  int64_t n_refined, n_coarsened; /* leaves flagged and honoured                               */
  int32_t balance_passes;         /* depth passes of the 2:1 balance that split something      */
  int32_t balance_exact_depth;    /* 0, or the depth of the first balance pass run with exact
                                     sizes (large meshes; or a pass that generated more octants
                                     than an adaptation issued without synchronisation holds) */
  double ms_tree, ms_transfer, ms_conn; /* device time of the three parts (Sec. 5.2 breakdown)  */
} fr_adapt_stats;

typedef struct {
  int64_t steps;
  int64_t dof_updates; /* sum over steps of M*N*nv                                             */
  double ms;           /* device time of the steps                                             */
} fr_step_stats;

typedef struct {
  double t, dt;
  int64_t M, step;
  int32_t dim, p, nv, N;
  int64_t n_conforming, n_hanging; /* face lists of the current mesh                          */
} fr_info;

/* ---------------------------------------------------------------------------------------------
 * Mesh-level calls
 * ------------------------------------------------------------------------------------------- */

/* Builds the initial mesh: uniform at Dbase, then init_passes of {closed-form vortex state
   (Sec. 5.2) at the solution points, indicator flags, fr_adapt}; the state is the closed form on
   the final tree.  `stream` is a cudaStream_t (NULL = legacy default stream).  `alloc` may be
   NULL.  On success *out owns all device memory of the mesh.  FR_EINVAL for dim/p/Dbase/Dmax out
   of range (dim*Dmax + m_b must fit in 63 bits). */
int fr_mesh_init(const fr_config* cfg, const fr_allocator* alloc, void* stream, fr_mesh** out);

/* Releases every buffer of the mesh (stream-ordered).  NULL is ignored. */
void fr_mesh_free(fr_mesh* m);

/* nsteps explicit SSP-RK3 steps (Eq. rk3) with the fixed dt: per stage one interface kernel
   (Rusanov flux on conforming faces, mortar projection at hanging faces, Sec. 4.3) and one
   element kernel (corrected-flux divergence, Sec. 2.1, and the Runge-Kutta combination).
   stats may be NULL; when given, the call synchronises to time the steps. */
int fr_step(fr_mesh* m, int nsteps, fr_step_stats* stats);

/* nsteps steps with fr_adapt(m, NULL, ...) after every adapt_every-th step (by step count). */
int fr_run(fr_mesh* m, int nsteps, fr_step_stats* step_stats, fr_adapt_stats* adapt_stats);

/* One adaptation (Sec. 4.1 procedure, then 2:1 balance, old->new mapping, solution transfer
   Sec. 4.2, connectivity Sec. 3.3).  flags: device int8[M] in {-1,0,1} borrowed for the call, or
   NULL to evaluate the configured indicator.  Refinement at Dmax and coarsening at Dbase are
   ignored; a leaf changes at most one level before balancing.  stats may be NULL.  The whole
   adaptation is issued against device-side counts when 2^dim * M <= 2^20, and the call waits once,
   at its end, for the counts the device publishes to mapped host memory (a balance pass
   generating more than 4096 octants is then finished with exact sizes, one synchronisation per
   pass); larger meshes synchronise once per balance pass.
   FR_EINVAL if the new tree fails a consistency check; FR_ETIMEOUT from the learned indicator. */
int fr_adapt(fr_mesh* m, const int8_t* dev_flags, fr_adapt_stats* stats);

/* Indicator flags of the current state (not applied).  host flags int8[M], eta double[M] (may be
   NULL).  cap = capacity in elements; FR_EOVERFLOW if cap < M. */
int fr_flags(fr_mesh* m, int8_t* host_flags, double* host_eta, int64_t cap);

/* Right-hand side R(u) = -div F of the current state into host double[M][nv][N]. */
int fr_rhs(fr_mesh* m, double* host_R, int64_t cap);

/* Norms of the current state (deterministic FP64 reductions). */
int fr_norms(fr_mesh* m, fr_norms_out* out);

/* Copies out the sorted leaves; host_keys may be NULL to query M only. */
int fr_get_leaves(fr_mesh* m, uint64_t* host_keys, int64_t cap, int64_t* M);
int fr_get_state(fr_mesh* m, double* host_u, int64_t cap);
/* Replaces tree and state (keys must form a complete, sorted, 2:1-balanced linear tree with
   depths in [Dbase, Dmax]; FR_EINVAL otherwise, and the mesh is left as it was).  The copies,
   the validation and the connectivity take one host synchronisation. */
int fr_set_state(fr_mesh* m, const uint64_t* host_keys, int64_t M, const double* host_u);
/* Connectivity tables, host arrays of M*2*dim entries. */
int fr_get_conn(fr_mesh* m, int32_t* host_nbr, int8_t* host_ftype, int8_t* host_slot, int64_t cap);
/* Replaces the state with the closed-form vortex at time t on the current tree and sets time. */
int fr_set_exact(fr_mesh* m, double t);
int fr_set_time(fr_mesh* m, double t);
int fr_get_info(fr_mesh* m, fr_info* out);
const char* fr_last_error(const fr_mesh* m);

/* Learned adaptation indicator (an extension: the paper uses an analytic criterion, Sec. 5.2).
   A per-element MLP maps features -> 3 logits (coarsen, keep, refine): inputs x (IN = 2*3^dim+1) ->
   64 -> 64 -> 64 -> 3, GELU after each hidden layer; inputs, weights and activations in BF16,
   every dot product accumulated in FP32.  Parameters: one FP32 array of fr_mlp_param_count(IN)
   values, [W1 (64xIN, row-major) | b1 | W2 (64x64) | b2 | W3 | b3 | W4 (3x64) | b4].
   Features of an element (fr_features, BF16 [M][IN]): the state is interpolated to the 3^dim
   Gauss-Legendre points of order 3 (so one network serves every degree p); there density and
   pressure give 100*(rho_i - mean rho)/mean rho and 100*(p_i - mean p)/mean p, then
   (D - Dbase)/max(1, Dmax - Dbase).
   Labels are classes -1/0/+1 (coarsen/keep/refine), int8.  class_w = {w_coarsen, w_keep, w_refine,
   1/sum_batch w_label}: the loss is sum_b w_b CE_b * class_w[3] (weighted mean cross-entropy).
   fr_mlp_train_step performs one Adam step (beta 0.9/0.999, eps 1e-8; d_m, d_v the moment arrays,
   step counts from 0) in place on d_params; d_loss (device, may be NULL) receives the batch loss.
   fr_mlp_grad returns the gradient of that loss instead.  Device pointers throughout; 1 <= IN <= 64
   (FR_EINVAL otherwise).
   fr_mlp_forward (and the mesh's learned indicator) runs on the tensor cores: BF16 MMAs with FP32
   accumulators in tensor memory, over tiles of 128 feature rows; a completion wait that gives up
   after about a second returns FR_ETIMEOUT (from fr_adapt/fr_run when it happens inside the
   indicator).  fr_mlp_grad and fr_mlp_train_step run on the tensor cores too (batch tiles of 128
   samples, weight gradients accumulated in tensor memory, block partials summed in a fixed order:
   deterministic), with the same FR_ETIMEOUT behaviour. */
/* Bound, in SM clock cycles, of the tensor-core inference kernel's waits on its own copies and MMAs
   (fr_mlp_forward and the learned indicator); cycles <= 0 restores the default of about a second.
   A wait that reaches the bound makes the call return FR_ETIMEOUT; each block then drains what it
   issued (with the default bound), frees its tensor memory and exits, so the device stays usable.
   A bound shorter than an MMA's latency forces that path (used by the tests).  Process-wide,
   not thread-safe. */
void fr_tc_set_wait_limit(long long cycles);
int fr_mlp_param_count(int in_dim);
int fr_features(fr_mesh* m, void* d_X_bf16, int64_t cap, int32_t* in_dim);
int fr_set_learned_indicator(fr_mesh* m, const float* host_params, int64_t n);
int fr_mlp_forward(int in_dim, const float* d_params, const void* d_X_bf16, int64_t n,
                   float* d_logits, int8_t* d_flags, void* stream);
int fr_mlp_grad(int in_dim, const float* d_params, const void* d_X_bf16, const int8_t* d_y,
                int64_t B, const float* class_w, float* d_grad, float* d_loss, void* stream);
int fr_mlp_train_step(int in_dim, float* d_params, float* d_m, float* d_v, int64_t step,
                      const void* d_X_bf16, const int8_t* d_y, int64_t B, const float* class_w,
                      float lr, float* d_loss, void* stream);

/* Measurement.  With profiling on, every interface and element kernel launched by fr_step,
   fr_run and fr_rhs is bracketed by CUDA events on the mesh's stream; fr_profile_read
   synchronises, sums the event intervals and returns them with the work those launches did.
   fr_profile_enable(m, k) with k >= 1 (re)starts the counters and times every k-th stage (one
   event pair around its interface kernel and one around its element kernel; each recorded event
   costs the stream a few microseconds, so k > 1 samples with less overhead);
   fr_profile_enable(m, 0) stops recording. */
typedef struct {
  int64_t stage_launches, face_launches;
  double stage_ms, face_ms;   /* summed device time of those launches                     */
  int64_t stage_points;       /* solution points processed by the element kernel launches  */
  int64_t face_points;        /* face (mortar) points processed by the interface launches  */
  int64_t kernel_launches;    /* every kernel this library launched since enable           */
} fr_profile;
int fr_profile_enable(fr_mesh* m, int on);
int fr_profile_read(fr_mesh* m, fr_profile* out);
/* Process-wide number of kernels this library has launched (all meshes and primitives). */
int64_t fr_kernel_launches(void);

/* ---------------------------------------------------------------------------------------------
 * Tree primitives on caller-owned DEVICE arrays, stream-ordered on `stream`.  Scratch memory is
 * allocated with cudaMallocAsync on the stream and released before return.  Counts that size an
 * output are returned through host pointers (the call synchronises the stream for them).
 * ------------------------------------------------------------------------------------------- */

/* Algorithm 1 (Sec. 2.2): boxes int32[n][4] -> keys uint64[n]. */
int fr_morton_encode(int dim, int Dmax, int64_t n, const int32_t* d_boxes, uint64_t* d_keys,
                     void* stream);
/* Ascending LSD radix sort of keys in place over the dim*Dmax+m_b significant bits. */
int fr_keys_sort(int dim, int Dmax, uint64_t* d_keys, int64_t n, void* stream);

/* Allocation-free key sort.  The paper has no counterpart; this is a convenience of this library.
   Same result as fr_keys_sort, but the call allocates no device memory at all: no cudaMalloc,
   cudaMallocAsync, cudaFree or allocator callback.  It is meant for callers that cannot allocate
   at the point of the call: code whose device memory is fully reserved up front by another
   framework or a fixed budget, and loops that must not pay for an allocation or the implicit
   synchronisation an allocation can cause.
   Scratch lives in one statically sized device array inside the library (about 2.4 MB, held on
   every GPU that loads the library until the process exits), so n is limited to
   FR_NOALLOC_SORT_MAX_KEYS; larger n returns FR_EINVAL without touching the keys.
   The first call on each device looks up that array's device address (cudaGetSymbolAddress);
   make that first call before any stream capture.  That lookup is safe when several host threads
   make their first calls on a device at the same time.  All calls share the one array and every call
   writes the scratch words it later reads, so no clearing is needed between calls, but calls
   whose GPU work overlaps (for example on two streams at once) race on the scratch and must be
   serialised by the caller.  Synchronises `stream` before returning. */
#define FR_NOALLOC_SORT_MAX_KEYS (1 << 18)
int fr_keys_sort_noalloc(int dim, int Dmax, uint64_t* d_keys, int64_t n, void* stream);
/* Sort, then linearise (Sec. 3.1): drop duplicates and octants that have a descendant in the set.
   d_out may alias nothing; *n_out receives the count (FR_EOVERFLOW if > cap). */
int fr_keys_linearise(int dim, int Dmax, const uint64_t* d_keys, int64_t n, uint64_t* d_out,
                      int64_t cap, int64_t* n_out, void* stream);
/* Tree completion from scattered points (Sec. 3.1, construction algorithm; Sec. 5.1 uses a
   background at Dmin and encodes the points at Dmax): d_pts double[n][dim] in [0,L)^dim (points
   outside are clamped to the boundary cells).  Output: the coarsest complete sorted linear tree
   whose leaves are at depth >= Dmin and which holds the depth-Dmax cell of every point as a leaf.
   It is not 2:1 balanced (apply fr_tree_balance).  Each gap between consecutive seed cells is
   covered by the largest aligned octants that fit, written at scanned positions, so no
   shared-memory overflow or retry exists.  *n_out receives the leaf count (FR_EOVERFLOW if > cap). */
int fr_tree_complete(int dim, int Dmin, int Dmax, double L, const double* d_pts, int64_t n,
                     uint64_t* d_out, int64_t cap, int64_t* n_out, void* stream);
/* 2:1 balance (Sec. 3.2, strong/vertex balance, periodic) of a complete sorted linear tree: the
   coarsest balanced refinement.  Depth passes from Dmax down to 2. */
int fr_tree_balance(int dim, int Dmax, const uint64_t* d_keys, int64_t n, uint64_t* d_out,
                    int64_t cap, int64_t* n_out, void* stream);
/* Adaptation procedure (Sec. 4.1) with flags int8[n], then 2:1 balance down to depth Dbase+2. */
int fr_tree_adapt(int dim, int Dbase, int Dmax, const uint64_t* d_keys, const int8_t* d_flags,
                  int64_t n, uint64_t* d_out, int64_t cap, int64_t* n_out, void* stream);
/* Old->new mapping (Sec. 4.2): src int32[n_new], tag int8[n_new] (0 copy, 1 refined from the old
   leaf src, 2 fused from the 2^dim old leaves starting at src). */
int fr_tree_map(int dim, int Dmax, const uint64_t* d_old, int64_t n_old, const uint64_t* d_new,
                int64_t n_new, int32_t* d_src, int8_t* d_tag, void* stream);
/* Face connectivity (Sec. 3.3) of a complete sorted 2:1-balanced tree: nbr/ftype/slot [n][2dim]. */
int fr_tree_conn(int dim, int Dmax, const uint64_t* d_keys, int64_t n, int32_t* d_nbr,
                 int8_t* d_ftype, int8_t* d_slot, void* stream);

#ifdef __cplusplus
}
#endif
#endif
