/*
 * ax.h -- C ABI of libax, a GB300 (sm_103a) implementation of the
 * matrix-free Poisson element operator of high-order spectral elements
 * ("AxLocal", CEED bake-off kernel BK5) with on-the-fly geometric factors,
 * after Cao, Sun, Zhang, Li, "Towards a Higher Roofline for Matrix-Vector
 * Multiplication in Matrix-Free HOSFEM" (arXiv 2504.07042).
 *
 * Conventions used by every call
 * ------------------------------
 *  - N is the polynomial order, N1 = N+1, n3 = N1^3 nodes per element.
 *    Supported: 1 <= N <= 15.
 *  - Element-local vectors X, Y are [E][n3] arrays, node [i,j,k] of element e
 *    at offset e*n3 + i + j*N1 + k*N1^2 (i fastest; Sec. 2.2, Algorithm 1).
 *  - Vertices are [E][8][3] float64, vertex v = a + 2b + 4c at reference
 *    corner (2a-1, 2b-1, 2c-1): the Kronecker order of the trilinear map,
 *    Eq. 8 (this is NOT the counter-clockwise Exodus/Nek order).
 *  - Geometric factors are [E][7][n3] float64 in the order
 *    g00 g01 g02 g11 g12 g22 gwj, G = w_i w_j w_k |J| J^-1 J^-T and
 *    gwj = w_i w_j w_k |J| (Eq. 7).
 *  - Pointers named "device" must be device memory of the current CUDA
 *    device (or managed memory); they stay owned by the caller.  The library
 *    copies what it keeps.  "stream" is a cudaStream_t passed as void*
 *    (NULL = legacy default stream).  Every call is asynchronous on that
 *    stream unless stated otherwise.
 *  - Every call returns an ax_status; on failure, ax_last_error() gives a
 *    message.  No call aborts the process or traps the GPU.
 */
#ifndef AX_H
#define AX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ax_ctx ax_ctx;

typedef enum {
  AX_OK = 0,
  AX_EINVAL = 1,              /* bad argument (size, pointer, enum) */
  AX_ENOMEM = 2,              /* device allocation failed */
  AX_ECUDA = 3,               /* a CUDA runtime call failed */
  AX_EINVERTED = 4,           /* det J <= 0 at some GLL node */
  AX_ENOTPARALLELEPIPED = 5,  /* AX_GEOM_PARALLELEPIPED given a non-affine element */
  AX_ENOTCONV = 6,            /* iterative solve hit its iteration cap */
  AX_ETIMEOUT = 7,            /* a bounded device wait gave up */
  AX_EUNSUPPORTED = 8,        /* valid but not implemented combination */
  AX_ERANGE = 9               /* input magnitude outside the kernel's number range */
} ax_status;

/* How the geometric factors reach the kernel (Table 3 of the paper). */
typedef enum {
  AX_GEOM_STORED = 0,            /* 6 of the 7 factors per node streamed from HBM ("full access") */
  AX_GEOM_TRILINEAR = 1,         /* recomputed per node from the 8 vertices (Algorithm 2) */
  AX_GEOM_PARALLELEPIPED = 2,    /* recomputed from one constant set per element (Algorithm 3) */
  AX_GEOM_TRILINEAR_PARTIAL = 3  /* trilinear, with the per-node scalar w|J|^-1 stored (Sec. 4.2.2) */
} ax_geom_kind;

/* Number format of X, Y and of the arithmetic. */
typedef enum {
  AX_FP64 = 0,  /* X, Y float64; native FP64 arithmetic */
  AX_FP32 = 1,  /* X, Y float32; FP32 arithmetic */
  AX_TF32 = 2,  /* X, Y float32; the six contractions on tensor cores (tcgen05.mma with tensor-memory
                   accumulators) with TF32 operands and FP32 accumulation; geometry and G x in FP32
                   (error about 1-2 u, u = 2^-11, against the FP64 result) */
  AX_BF16 = 3,  /* as AX_TF32 with BF16 operands (u = 2^-8) */
  AX_FP16 = 4,  /* as AX_TF32 with FP16 operands (u = 2^-11; inputs must stay inside FP16's range,
                   which the mixed-precision solver's scaling by ||r||_inf ensures) */
  AX_F64DW = 5  /* X, Y float64; arithmetic in double-word FP32 pairs (about 47 bits) on the
                   FP32 pipe; same results as AX_FP64 to ~1e-13 relative max-norm */
} ax_precision;

/* Create a context for E elements of order N.
 *   vertices: device, [E][8][3] float64 (Eq. 8 order).  Read during the call only.
 *   kind, prec: see the enums.
 * Computes GLL tables, the per-kind geometry record (stored factors via the
 * discrete Jacobian of Sec. 3.2, vertex data, parallelepiped constants of
 * Algorithm 3, or per-node w/|J| for the partial kind) and validates the
 * mesh: AX_EINVERTED if det J <= 0 at any GLL node, AX_ENOTPARALLELEPIPED if
 * kind is PARALLELEPIPED and an element is not affine (relative 1e-12).
 * Synchronises the stream once (validity flag).  On success *out owns
 * device memory until ax_destroy(). */
ax_status ax_setup(ax_ctx **out, int64_t E, int N, const double *vertices, ax_geom_kind kind,
                   ax_precision prec, void *stream);

/* AxLocal (Algorithm 1, Poisson: lambda0 = 1, lambda1 = 0):
 *   Y[e] = A^(e) X[e] = D^T (w G) D X[e] for every element (unassembled).
 *   X, Y: device, [E][n3], float64 for AX_FP64/AX_F64DW, float32 otherwise,
 *   aligned to their element size (a 16-byte aligned X is read in 16-byte
 *   vectors where the kernel does so; any other X takes word loads and gives
 *   the same result bit for bit).
 *   Y is overwritten; X and Y must not overlap.  One kernel launch. */
ax_status ax_local(ax_ctx *c, const void *X, void *Y, void *stream);

/* Same as ax_local with host buffers (pageable or pinned): copies X to the
 * device, runs ax_local, copies Y back and synchronises the stream.  Uses
 * library-owned device buffers allocated at the first call.  The elements
 * are processed in up to 16 chunks (at least 2048 elements each) on three
 * library streams (copy in, AxLocal, copy out) ordered by events, so the
 * transfers overlap the kernels (pinned host memory lets them run
 * asynchronously); the call is ordered after prior work on `stream`.
 * Float32 X and Y (AX_FP32, AX_TF32, AX_BF16, AX_FP16) in page-locked host
 * memory the device can address are instead read and written by the
 * kernel directly over the host link (no staging buffers, one launch on
 * `stream`); X and Y must then lie wholly in such memory. */
ax_status ax_local_host(ax_ctx *c, const void *X_host, void *Y_host, void *stream);

/* ax_local_host for callers that cannot allocate device memory at call time
 * (their device-memory budget is fixed after start-up, or a cudaMalloc /
 * cudaFree would synchronise the device in the middle of their pipeline).
 * The paper has no counterpart; this is a deployment variant of
 * ax_local_host.
 *   X_host, Y_host: host buffers of [E][n3] values (float64 or float32 as for
 *   ax_local).  Copies X in, runs the same AxLocal kernel, copies Y out,
 *   synchronises the stream.
 * It calls no cudaMalloc/cudaFree: X and Y are staged through one file-scope
 * device array of 32 MiB (16 MiB per vector).  ax_setup looks up the array's
 * device address with the context's device current; that lookup loads the
 * library module holding the array, so the array is committed during
 * ax_setup on every GPU where a context is set up, and stays until the
 * process exits.  The entry point itself does no look-up, no module load and
 * no allocation.  E * (N+1)^3 * word size above 16 MiB returns AX_EINVAL
 * (use ax_local_host or ax_local instead).
 * All calls share the array and it keeps the last call's contents: calls
 * that overlap on the GPU (several host threads or streams at once) race,
 * so callers must serialise them. */
ax_status ax_local_host_static(ax_ctx *c, const void *X_host, void *Y_host, void *stream);

/* The geometric factors as the kernel of this context obtains them, written
 * to G_out: device, [E][7][n3] float64.  Stored kinds copy their table; the
 * recompute kinds run their in-kernel geometry code (Algorithm 2 or 3) and
 * write its results.  For testing the geometry step on its own. */
ax_status ax_factors(ax_ctx *c, double *G_out, void *stream);

/* Physical coordinates of every node (Eq. 8 at the GLL points):
 * XYZ_out: device, [E][3][n3] float64. */
ax_status ax_node_coords(ax_ctx *c, double *XYZ_out, void *stream);

/* Global numbering for gather-scatter: the binary global-to-local matrix Q
 * of Eq. 1, Q[e*n3 + l][global_id[e][l]] = 1.
 *   global_id: device, [E][n3] int64 in [0, n_global).
 *   dirichlet_mask: device, [n_global] uint8 (1 = homogeneous Dirichlet node,
 *   removed from the assembled system) or NULL.
 * Builds, once, a CSR of the local copies of every global node in increasing
 * local order (so every gather is a fixed-order, deterministic sum), with
 * 32-bit indices: AX_ERANGE if E*n3 or n_global exceeds 2^31 - 1.
 * Synchronises the stream.  AX_EINVAL if an id is out of range.  Frees the
 * context's solver workspaces and cached diagonal (they depend on the plan). */
ax_status gs_setup(ax_ctx *c, const int64_t *global_id, int64_t n_global, const uint8_t *dirichlet_mask,
                   void *stream);

/* Y_local <- Q Q^T Y_local in place: each local copy of a global node is
 * replaced by the sum of all its copies (Eq. 1 assembly, unmasked). */
ax_status gs_assemble(ax_ctx *c, void *Y_local, void *stream);

/* y_global = Q^T Y_local (sums of local copies; 0 on Dirichlet nodes). */
ax_status gs_gather(ax_ctx *c, const void *Y_local, void *y_global, void *stream);

/* U_local = Q u_global (copies the global value to every local copy). */
ax_status gs_scatter(ax_ctx *c, const void *u_global, void *U_local, void *stream);

/* GLL-lumped mass: Y_local = (w_i w_j w_k |J|) * F_local per node (the
 * seventh factor of Eq. 7 times F); builds right-hand sides b = Q^T (w|J| f). */
ax_status ax_mass(ax_ctx *c, const void *F_local, void *Y_local, void *stream);

/* Element diagonals: diag_local[e][l] = e_l^T A^(e) e_l (for Jacobi). */
ax_status ax_diag(ax_ctx *c, void *diag_local, void *stream);

/* Conjugate gradients on the assembled system A = Q^T blkdiag(A^(e)) Q
 * (Eq. 1) with the Dirichlet nodes of gs_setup removed, A applied with this
 * context's AxLocal kernel.
 *   b_global, x_global: device [n_global] (float64 for AX_FP64/AX_F64DW,
 *   float32 otherwise); x_global is the initial guess and receives the
 *   solution.  precond: 0 = none, 1 = Jacobi (assembled diagonal); 2 (the
 *   learned preconditioner) returns AX_EINVAL: it needs a network handle,
 *   so it has its own entry point, pcg_solve_learned(ctx, mlp, ...).
 *   Other values return AX_EUNSUPPORTED.  Stops when ||r||_2 <= rtol ||b||_2 or after maxit iterations
 *   (AX_ENOTCONV).  *iters and *relres (host) report the outcome.
 * One iteration is four kernels (direction + scatter, AxLocal, gather + p.w
 * with alpha, update + r.z, r.r with the convergence test and beta); every
 * scalar stays on the device and the grid-level sums are finished in the
 * producing kernel in a fixed order (deterministic).  Blocks of 16
 * iterations run as one CUDA graph on a private stream, ordered after and
 * before `stream` by events; the host reads the scalars once per block.
 * The work vectors, the stream and the graph are kept in the context for
 * the next call (released by gs_setup and ax_destroy); the assembled
 * Jacobi diagonal is computed at the first call and kept.  Synchronises. */
ax_status pcg_solve(ax_ctx *c, const void *b_global, void *x_global, double rtol, int maxit, int precond, int *iters,
                    double *relres, void *stream);

/* Mixed-precision solve of the same system: FP64 iterative refinement
 * around an inner Jacobi-PCG in float32 (the low-precision direction the
 * paper names as future work, Sec. 7).
 *   hi: context with AX_FP64 or AX_F64DW and gs_setup done; computes the
 *       residual r = b - A x in FP64-accurate arithmetic each outer step.
 *   lo: context of the same mesh (same E, N, vertices) with a float32
 *       precision (AX_FP32, or AX_TF32 / AX_BF16 / AX_FP16 for tensor-core
 *       contractions in the inner operator); runs
 *       the inner solve A d = r / ||r||_inf to inner_rtol (at most max_inner
 *       iterations); x += ||r||_inf d.
 *   b_global, x_global: device float64 [n_global]; x is the initial guess.
 *   Stops when ||r||_2 <= rtol ||b||_2 (AX_OK) or after max_outer outer
 *   steps (AX_ENOTCONV).  *outer_iters, *inner_iters (total), *relres: host.
 * Synchronises. */
ax_status pcg_solve_mixed(ax_ctx *hi, ax_ctx *lo, const double *b_global, double *x_global, double rtol,
                          double inner_rtol, int max_outer, int max_inner, int *outer_iters, int *inner_iters,
                          double *relres, void *stream);

/* ------------------------------------------------------------------------
 * Batches of independent meshes of uneven size and order.
 * Meshes are grouped by order N; each group runs as one AxLocal launch over
 * the union of its elements.  The batch's local vector concatenates the
 * groups' local vectors (group by increasing first appearance of N, meshes
 * in batch order inside a group); the batch's global vector concatenates the
 * meshes' global vectors in batch order (ax_batch_sizes gives the offsets).
 * ---------------------------------------------------------------------- */
typedef struct ax_batch ax_batch;

/* B meshes; mesh m: E[m] elements of order N[m], vertices[m] (device
 * [E][8][3] float64), global_id[m] (device [E][n3] int64, numbering local to
 * the mesh), n_global[m], mask[m] (device uint8 [n_global] or NULL; mask may
 * be NULL).  All meshes share kind and prec.  Also builds one per-mesh
 * context for each mesh (the per-mesh reference path of ax_batch_pcg).
 * Synchronises. */
ax_status ax_batch_setup(ax_batch **out, int B, const int64_t *E, const int *N, const double *const *vertices,
                         const int64_t *const *global_id, const int64_t *n_global, const uint8_t *const *mask,
                         ax_geom_kind kind, ax_precision prec, void *stream);

/* Sizes of the batch vectors and the per-mesh offsets (host arrays of B and
 * B+1 entries; any pointer may be NULL). */
ax_status ax_batch_sizes(const ax_batch *b, int64_t *n_local, int64_t *n_global, int64_t *local_offsets,
                         int64_t *global_offsets);

/* AxLocal of every mesh: X, Y device batch local vectors.
 * AX_FP32 batches of orders N <= 9 run as ONE persistent launch: a device
 * queue of (mesh, element tile) items over all orders, dequeued by the CTAs
 * (the paper runs one (E, N) per launch, Sec. 5.1; this goes beyond it).
 * Other batches: one launch per distinct order (ax_batch_info tells which). */
ax_status ax_batch_local(ax_batch *b, const void *X, void *Y, void *stream);

/* Autotune and keep the choice.  Persistent batches: element blocks per
 * AxLocal item for each order group ({1, 2, 4, 8}, coordinate descent) and
 * the grid (CTAs per SM: the occupancy limit or 1, 2, 4), timing the whole
 * batch's single launch; tiles[g] gets the blocks per item, grids[g] the
 * CTAs.  Other batches, per group: the tile (elements per CTA: 0 = base,
 * 1 = twice, FP32 only) and the grid (0 = one CTA per element block, else a
 * persistent grid of k * SMs CTAs).  tiles, grids: host arrays with one
 * entry per group (or NULL).  Synchronises. */
ax_status ax_batch_tune(ax_batch *b, int *tiles, int64_t *grids, void *stream);

/* Choose the persistent single launch (on = 1, the default where it exists)
 * or one launch per order group and per CG phase (on = 0).  AX_EUNSUPPORTED
 * when the batch has no persistent kernel (not AX_FP32, or an order N > 9). */
ax_status ax_batch_set_persistent(ax_batch *b, int on);

/* Launches per ax_batch_local and per CG iteration of ax_batch_pcg
 * (graph = 1) in the batch's current mode; *persistent = 1 in the
 * persistent mode.  Any pointer may be NULL. */
ax_status ax_batch_info(const ax_batch *b, int *persistent, int *local_launches, int *iteration_launches);

/* Persistent batches: bound of every dependency wait inside the single CG
 * launch, in ns (default 2e9), and a test hook: stuck_mesh >= 0 makes that
 * mesh's gather items wait for one AxLocal item more than exist, so the wait
 * runs out; ax_batch_pcg then stops and returns AX_ETIMEOUT, and the batch
 * stays usable (-1 restores the normal dependency).  The paper has no
 * counterpart.  AX_EUNSUPPORTED without a persistent kernel. */
ax_status ax_batch_set_wait(ax_batch *b, int64_t budget_ns, int stuck_mesh);

/* Independent Jacobi-PCG solves of every mesh's Dirichlet Poisson system.
 *   b_global, x_global: device batch global vectors (x: initial guess in,
 *   solutions out).  Per-mesh stop at ||r|| <= rtol ||b||.
 *   graph = 1: all meshes advance together; one CG iteration of the whole
 *   batch is captured once as a CUDA graph and launched once per iteration
 *   (per-mesh scalars, segmented reductions, converged meshes idle).  In
 *   the persistent mode the graph holds ONE kernel: a queue of AxLocal
 *   tiles (the scatter fused into their loads), gather + dot, update and
 *   direction chunks, each waiting (bounded) for its mesh's previous phase;
 *   a wait past its budget stops the solve with AX_ETIMEOUT.
 *   graph = 0: reference path, each mesh solved in turn with its own
 *   launches (pcg_solve on its per-mesh context).
 *   iters, relres: host arrays [B].  AX_ENOTCONV if a mesh hit maxit.
 * Synchronises. */
ax_status ax_batch_pcg(ax_batch *b, const void *b_global, void *x_global, double rtol, int maxit, int graph,
                       int *iters, double *relres, void *stream);

/* Message of the batch's last failed call (or of batch creation when b is NULL). */
const char *ax_batch_last_error(const ax_batch *b);

/* Release the batch (NULL accepted). */
void ax_batch_destroy(ax_batch *b);

/* ------------------------------------------------------------------------
 * Learned preconditioner (order N = 7 elements): a per-element MLP
 * 536 -> 512 (GELU) -> 512 (GELU) -> 512, BF16 GEMMs on the tcgen05 tensor
 * cores (TMA-fed, FP32 accumulation in tensor memory, fused bias/GELU
 * epilogues), FP32 master weights, Adam.  The paper has no counterpart;
 * the MLP corrects the Jacobi step of a flexible CG.  Calls that
 * synchronise return AX_ETIMEOUT if a GEMM's bounded wait gave up.
 * Element input (536 = 512 + 24): the element's local residual divided by
 * s_e = max |r_e|, and its vertex coordinates relative to vertex 0 divided by
 * h_e = |v1 - v0|; inputs are padded to 544 columns (zeros) in bf16.
 * ---------------------------------------------------------------------- */
typedef struct ax_mlp ax_mlp;

/* Create with deterministic initial weights (splitmix64 + Box-Muller from seed). */
ax_status ax_mlp_create(ax_mlp **out, uint64_t seed, void *stream);

/* Number of float32 parameters; layout W1 [512][544] (columns >= 536 zero),
 * b1 [512], W2 [512][512], b2 [512], W3 [512][512], b3 [512]. */
int64_t ax_mlp_num_params(const ax_mlp *m);

/* Copy the parameters out / in (params: host or device float32 [num_params]). */
ax_status ax_mlp_get_params(ax_mlp *m, float *params, void *stream);
ax_status ax_mlp_set_params(ax_mlp *m, const float *params, void *stream);

/* Y (device float32 [M][512]) = MLP(X) for X device bf16 [M][544]. */
ax_status ax_mlp_forward(ax_mlp *m, const void *X_bf16, float *Y, int64_t M, void *stream);

/* Loss L = 0.5 mean (MLP(X) - T)^2 over M rows (M a positive multiple of 32)
 * and its gradient w.r.t. every parameter (grads: host or device float32
 * [num_params], same layout).  For gradient checks.  Synchronises. */
ax_status ax_mlp_grad(ax_mlp *m, const void *X_bf16, const float *T, int64_t M, float *loss, float *grads,
                      void *stream);

/* Adam training (lr, beta1 0.9, beta2 0.999, eps 1e-8) on n_samples rows of
 * X (device bf16 [n][544]) and T (device float32 [n][512]): epochs passes of
 * shuffled mini-batches of `batch` rows (a multiple of 32).  loss_history:
 * host float [epochs] (last batch's loss per epoch) or NULL.  Synchronises. */
ax_status ax_mlp_train(ax_mlp *m, const void *X_bf16, const float *T, int64_t n_samples, int epochs, int batch,
                       float lr, uint64_t seed, float *loss_history, void *stream);

/* Training pairs from an iterate x_k of a solve of the context's system
 * (gs_setup done; N = 7):  r = b - A x_k (Dirichlet-masked), e = x_star - x_k,
 * d = Jacobi inverse diagonal.  For each listed element i (elements: device
 * int64 [n]): F[i] (device bf16 [544]) = element input of r, and
 * T[i] (device float32 [512]) = (h_e / s_e) (e - d r) on the element's nodes.
 * b_global, x_star, x_k: device float64 [n_global]. */
ax_status ax_mlp_pairs(ax_ctx *c, const double *b_global, const double *x_star, const double *x_k,
                       const int64_t *elements, int64_t n, void *F_bf16, float *T, void *stream);

/* Flexible CG (Polak-Ribiere beta) with the learned preconditioner
 *   z = D^-1 r + omega Q^T(c) / multiplicity,   c_e = (s_e / h_e) MLP(input of r_e),
 * on the context's Dirichlet system (float64 vectors, the context's
 * FP64-accurate AxLocal).  Safeguards: a learned step with r . z <= 0 is
 * replaced by the Jacobi step; if the residual has not halved for 200
 * iterations the solve falls back to Jacobi-PCG for the rest (*fell_back = 1).
 * Stops when ||r|| <= rtol ||b|| (AX_OK) or after maxit iterations
 * (AX_ENOTCONV).  Every scalar stays on the device (alpha, beta, the
 * safeguard and the patience test are decided by the last block of the
 * kernel that produces their sums); blocks of 16 iterations run as one CUDA
 * graph; the work vectors are kept in the context.  Synchronises. */
ax_status pcg_solve_learned(ax_ctx *c, ax_mlp *m, const double *b_global, double *x_global, double rtol, int maxit,
                            double omega, int *iters, double *relres, int *fell_back, void *stream);

/* Message of the last failed MLP call (or of creation when m is NULL). */
const char *ax_mlp_last_error(const ax_mlp *m);

/* Release the MLP (NULL accepted). */
void ax_mlp_destroy(ax_mlp *m);

/* Algorithmic cost of one ax_local call (per element): bytes moved to and
 * from HBM by the kernel's design, the paper's effective flops
 * F_ax = 12 N1^4 + 15 N1^3 (Table 2), and the arithmetic instructions the
 * kernel issues per element on its binding pipe (FP64 or FP32 lanes). */
typedef struct {
  int64_t E;
  int N;
  int kind;
  int prec;
  double bytes_per_element;
  double flops_ax_per_element;
  double pipe_ops_per_element;
  int pipe;  /* 0 = FP64 pipe, 1 = FP32 pipe, 2 = tensor pipe */
} ax_info;
ax_status ax_query(const ax_ctx *c, ax_info *info);

/* Message for the last failed call on this context (or on context creation
 * when c is NULL).  Owned by the library; valid until the next call. */
const char *ax_last_error(const ax_ctx *c);

/* Name of a status code. */
const char *ax_status_string(ax_status s);

/* Status of the context's asynchronous work: synchronises `stream`, then
 * returns AX_ETIMEOUT if a bounded wait inside one of the context's kernels
 * ran out since the last check (the tensor-core AxLocal of AX_TF32 at N = 7
 * waits on its MMAs, at most about 2 s; the output of that launch is void),
 * else AX_OK.  Clears the record. */
ax_status ax_check(ax_ctx *c, void *stream);

/* Release everything the context owns.  NULL is accepted. */
void ax_destroy(ax_ctx *c);

#ifdef __cplusplus
}
#endif
#endif /* AX_H */
