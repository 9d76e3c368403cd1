/*
 * dolinc.h — C ABI of the GB300 DOLINC stage library (libdolinc.so).
 *
 * DOLINC (arXiv 2404.08952) lifts the far-field cells a high-order finite-volume
 * reconstruction needs into "order-lifted" differentials stored in each cell, and
 * inverts them exactly at every face.  One explicit Runge-Kutta stage here is:
 *
 *   1. differentials   T^(m)_c = (1/V_c) sum_f S_{c,f} (x) [w T^(m-1)_c + (1-w) T^(m-1)_nb],
 *                      m = 1..n_diff, T^(0) = cell average            (Sec 2.3)
 *   2. inversion       far-field averages phi_{-r}..phi_{k-r-1} from the two face cells'
 *                      differentials phi^(m) = 2^m T^(m) : d^m by Eq diffDLC
 *                      (first/second order: Eqs lCoeffDLC1 .. rCoeffDLC2)  (Sec 2.3)
 *   3. reconstruction  phi_{i+1/2} = sum_j c_rj(g) phi_{i-r+j}, c_rj from Eq coeff (Sec 2.4)
 *   4. flux            upwind (linear advection), Roe (Burgers), local Lax-Friedrichs /
 *                      Rusanov (Euler)                                     (Sec 3)
 *   5. residual and    R_c = -(1/V_c) sum_f (+-)F_f, third-order TVD (SSP) Runge-Kutta
 *      update                                                              (Sec 3)
 *
 * Conventions shared by every entry point
 *   - Status codes only; no exception crosses the ABI.  dolinc_last_error() gives the
 *     calling thread's last message.
 *   - Device buffers belong to the caller.  The library never frees them.  Arguments
 *     named *_dev are device pointers on the current CUDA device; everything else is
 *     host memory.  Calls are asynchronous on the given stream, except where noted.
 *   - Cell fields are FP64, variables first: u[v * n_cells + c], in the LIBRARY's cell
 *     order (see dolinc_mesh_permutation; renumber = 0 keeps the caller's order).
 *   - Face fields are FP64 [v * n_faces + f] in the CALLER's face order and orientation.
 *   - A mesh handle may be used by one stream at a time.
 *   - Workspace: every compute entry point takes a caller-owned device buffer
 *     (ws_dev, ws_bytes) at least dolinc_workspace_size() bytes, 256-byte aligned.
 *     It is scratch: its contents between calls mean nothing, except that the
 *     first 1024 bytes hold the device status word read by dolinc_sync_status and
 *     the grid-barrier words of the batched steps.
 */
#ifndef DOLINC_H
#define DOLINC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *dolinc_stream;   /* a cudaStream_t; NULL = legacy default stream */

typedef enum {
    DOLINC_OK = 0,
    DOLINC_ERR_INVALID_ARG = 1,     /* bad pointer, size, or scheme parameter */
    DOLINC_ERR_MESH = 2,            /* mesh descriptor fails validation */
    DOLINC_ERR_UNSUPPORTED = 3,     /* valid request the library does not implement */
    DOLINC_ERR_CUDA = 4,            /* a CUDA runtime call failed (message has the CUDA error) */
    DOLINC_ERR_DEVICE_TIMEOUT = 5,  /* a bounded device-side wait gave up */
    DOLINC_ERR_NONFINITE = 6,       /* a stage produced NaN or Inf */
    DOLINC_ERR_OOM = 7              /* device or host allocation failed */
} dolinc_status;

enum { DOLINC_FLUX_UPWIND = 0, DOLINC_FLUX_BURGERS = 1, DOLINC_FLUX_RUSANOV = 2 };
enum { DOLINC_FP64 = 0, DOLINC_FP32 = 1, DOLINC_FP32_BF16 = 2 };
enum { DOLINC_LIMIT_NONE = 0, DOLINC_LIMIT_ENO3_ALL = 1, DOLINC_LIMIT_ENO3_FLAGGED = 2,
       DOLINC_LIMIT_FIRST_ORDER_FLAGGED = 3, DOLINC_LIMIT_WENO5_ALL = 4, DOLINC_LIMIT_WENO5_FLAGGED = 5 };
enum { DOLINC_RENUMBER_NONE = 0, DOLINC_RENUMBER_MORTON = 1 };

/* Mesh in owner/neighbour face form (Sec 2.1: a cell knows its neighbours only
 * through faces).  All arrays are host memory; dolinc_mesh_create copies them.
 *   nodes                [n_nodes][dim] coordinates
 *   face_node_offsets    [n_faces+1] CSR into face_nodes
 *   face_nodes           node ids, ordered so that the area vector points out of the
 *                        owner: 2D edge a->b has area vector (b_y-a_y, -(b_x-a_x));
 *                        3D polygon nodes are counter-clockwise seen from outside the
 *                        owner.  A polygon with more than 3 nodes is the union of the
 *                        triangles joining each edge to the mean of its nodes.
 *   face_owner           [n_faces] owner cell
 *   face_neighbour       [n_faces] neighbour cell, or -1 on a boundary face
 *   face_periodic_shift  [n_faces][dim] translation carrying the neighbour cell next to
 *                        the owner across a periodic face (0 elsewhere); NULL = none
 *   boundary_kind        [n_faces] 0 interior/periodic; on boundary faces (Sec 2.6)
 *                        1 zero-gradient (transmissive), 2 Dirichlet (prescribed face
 *                        value), 3 Neumann (prescribed outward normal gradient); the
 *                        values of 2 and 3 come from dolinc_set_boundary_values.
 *                        NULL = all boundary faces zero-gradient
 *   cell_face_offsets,   optional CSR cell -> faces (NULL to skip); when given, every
 *   cell_faces           face must appear in its owner's and neighbour's lists
 *   renumber             DOLINC_RENUMBER_NONE keeps the caller's cell order;
 *                        DOLINC_RENUMBER_MORTON orders cells along a Morton curve of
 *                        their centroids (better cache reuse of neighbour gathers)     */
typedef struct {
    int dim;                                   /* 2 or 3 */
    int64_t n_nodes;
    const double *nodes;
    int64_t n_cells;
    const int64_t *cell_face_offsets;
    const int64_t *cell_faces;
    int64_t n_faces;
    const int64_t *face_node_offsets;
    const int64_t *face_nodes;
    const int64_t *face_owner;
    const int64_t *face_neighbour;
    const double *face_periodic_shift;
    const int32_t *boundary_kind;
    int renumber;
} dolinc_mesh_desc;

/* Scheme of one stage.
 *   k, r        reconstruction stencil: k cells i-r .. i-r+k-1 (Eq coeff).  USR3 = (3,1),
 *               CSR4 = (4,1), USR5 = (5,2), CSR6 = (6,2), second-order upwind = (2,1).
 *               Needs differentials through order max(r, k-r-2) (Sec 2.3: r far cells
 *               upwind need order r, k-r-1 cells downwind need order k-r-2).
 *   n_diff      differential orders computed each stage (1..4), >= what (k, r) needs
 *               (and >= 2 with an ENO3 or WENO5 limiter).  Orders above the need are computed
 *               and stored but do not change the face values.
 *   flux        DOLINC_FLUX_*; nv = 1 for UPWIND and BURGERS, nv = dim+2 for RUSANOV
 *               (conserved rho, rho u.., rho E, reconstructed component-wise)
 *   precision   DOLINC_FP64: all FP64.  DOLINC_FP32: differentials, reconstruction and
 *               flux in FP32, geometry master and state update FP64.
 *               DOLINC_FP32_BF16: as FP32 with differential orders >= 2 stored in BF16.
 *   limiter     DOLINC_LIMIT_*: ENO3-DOLINC (Sec 2.4) on every face, or on faces touching
 *               a cell flagged with dolinc_set_flags / dolinc_indicator_infer; or
 *               FIRST_ORDER_FLAGGED: on faces touching a flagged cell each orientation
 *               takes its upwind cell's average (first-order Godunov fallback, not a
 *               scheme of the paper; it needs no second-order differentials); or
 *               WENO5-DOLINC (Sec 2.4: the three 3-cell DOLINC candidates with
 *               Jiang-Shu weights, linear weights reproducing the 5-cell stencil,
 *               smoothness of the candidates' quadratics on the non-uniform cells) on
 *               every face (WENO5_ALL) or on faces touching a flagged cell; ENO3 and
 *               WENO5 need n_diff >= 2
 *   gamma       ratio of specific heats (RUSANOV)
 *   adv         advection velocity (UPWIND); Burgers flux is u^2/2 (1,..,1)          */
typedef struct {
    int k, r;
    int n_diff;
    int flux;
    int nv;
    int precision;
    int limiter;
    double gamma;
    double adv[3];
} dolinc_scheme;

typedef struct dolinc_mesh dolinc_mesh;

typedef struct {
    int dim;
    int64_t n_cells, n_faces, n_boundary_faces, n_slots;
    double g_min, g_max;                       /* Eq 4 growth rates over interior faces */
    double volume;                             /* sum of cell volumes */
    double h_min;                              /* min over cells of V_c / max_f |S_f| */
} dolinc_mesh_info;

/* Validate and copy a mesh, compute its FP64 geometry (Sec 2.2 Eqs 1-4: volumes,
 * centroids, area vectors, Euclidean weights w, growth rates g = w/(1-w), centre
 * distances d), renumber, build the cell -> face slots and copy everything to the
 * current device.  Synchronous.  *out is NULL on failure. */
dolinc_status dolinc_mesh_create(const dolinc_mesh_desc *desc, dolinc_mesh **out);
void dolinc_mesh_destroy(dolinc_mesh *mesh);
dolinc_status dolinc_mesh_get_info(const dolinc_mesh *mesh, dolinc_mesh_info *info);
/* new_of_old[caller cell] = library cell (host array of n_cells). */
dolinc_status dolinc_mesh_permutation(const dolinc_mesh *mesh, int64_t *new_of_old);
/* Host copies of the library's FP64 geometry, in library cell order and caller face
 * order/orientation; any pointer may be NULL.  V [n_cells], xc [n_cells][3],
 * S [n_faces][3], w [n_faces] (weight of the caller's owner), d [n_faces][3]. */
dolinc_status dolinc_mesh_geometry(const dolinc_mesh *mesh, double *V, double *xc, double *S, double *w,
                                   double *d);

/* Bytes of workspace the compute entry points need for this scheme. */
dolinc_status dolinc_workspace_size(const dolinc_mesh *mesh, const dolinc_scheme *scheme, size_t *bytes);

/* Clears the device status word at the start of a new workspace (ws_dev, at least
 * 1024 bytes, 256-byte aligned).  Call once after allocating a workspace, before the
 * first compute call that uses it; dolinc_sync_status clears it again after reading. */
dolinc_status dolinc_workspace_init(void *ws_dev, size_t ws_bytes, dolinc_stream stream);

/* Layout of the differential buffer of dolinc_differentials.  Order m (1..order)
 * starts at element offset[m-1]; the record of cell c is `stride[m-1]` elements of
 * `elem_bytes[m-1]` bytes (8 FP64, 4 FP32, 2 BF16) at offset + c*stride; inside it
 * variable v's coefficients start at v*C_m, C_m = m+1 (2D) or (m+1)(m+2)/2 (3D).
 * Coefficient q of order m multiplies the monomial d_x^a d_y^b d_z^c (a+b+c = m) with
 * t = b+c, q = t(t+1)/2 + c (3D) or q = b (2D), so that
 *   T^(m) : d^m = sum_q coef[q] * monomial_q(d),  phi^(m) = 2^m T^(m) : d^m.
 * total_elems: size of the buffer in elements of the widest type (FP64 or FP32). */
dolinc_status dolinc_diff_layout(const dolinc_mesh *mesh, const dolinc_scheme *scheme, int order,
                                 int64_t *offset, int *stride, int *elem_bytes, int64_t *total_bytes);

/* Differentials of orders 1..order (Sec 2.3) of the FP64 cell averages u_dev, in the
 * scheme's precision, written to diff_dev (256-byte aligned, total_bytes of
 * dolinc_diff_layout; DOLINC_ERR_INVALID_ARG otherwise) with that layout. */
dolinc_status dolinc_differentials(dolinc_mesh *mesh, const dolinc_scheme *scheme, const double *u_dev,
                                   int order, void *diff_dev, void *ws_dev, size_t ws_bytes,
                                   dolinc_stream stream);

/* Left/right face states (Sec 2.3-2.4): face_L_dev[v*n_faces+f] is the reconstruction
 * with the caller's owner as upwind cell i, face_R_dev with the neighbour upwind.
 * Differentials are recomputed from u_dev.  Boundary faces return the cell value. */
dolinc_status dolinc_reconstruct_faces(dolinc_mesh *mesh, const dolinc_scheme *scheme, const double *u_dev,
                                       double *face_L_dev, double *face_R_dev, void *ws_dev, size_t ws_bytes,
                                       dolinc_stream stream);

/* Residual R_c = -(1/V_c) sum_f (+-) F_f of the FP64 cell averages u_dev. */
dolinc_status dolinc_residual(dolinc_mesh *mesh, const dolinc_scheme *scheme, const double *u_dev,
                              double *R_dev, void *ws_dev, size_t ws_bytes, dolinc_stream stream);

/* One SSP-RK3 stage (Sec 3): out = a*u0 + b*(us + dt R(us)) with
 * (a, b) = (0, 1), (3/4, 1/4), (1/3, 2/3) for stage 0, 1, 2.  out may alias us. */
dolinc_status dolinc_rk_stage(dolinc_mesh *mesh, const dolinc_scheme *scheme, double dt, int stage,
                              const double *u0_dev, const double *us_dev, double *out_dev, void *ws_dev,
                              size_t ws_bytes, dolinc_stream stream);

/* One full SSP-RK3 step of u_dev in place (three stages, each: n_diff differential
 * passes + one fused reconstruction/flux/residual/update pass).  In FP64 every stage
 * value is formed in FP64 as dolinc_rk_stage does.  Below FP64 the step runs in the
 * equivalent increment form: with d_k = dt R(u_k), u1 = u0 + D0, u2 = u0 + D1 and
 * u^{n+1} = u0 + (2/3)(D1 + d2), where D0 = d0, D1 = (D0 + d1)/4 are kept per cell in
 * the bulk precision; the stage inputs exist only as bulk-precision records and the
 * FP64 state receives one add per step. */
dolinc_status dolinc_rk_step(dolinc_mesh *mesh, const dolinc_scheme *scheme, double dt, double *u_dev,
                             void *ws_dev, size_t ws_bytes, dolinc_stream stream);

/* n_steps SSP-RK3 steps of u_dev in one call: the same results, bit for bit, as
 * n_steps calls of dolinc_rk_step.  The state stays on the device between the steps,
 * so the last stage of each step also writes the next step's bulk-precision record
 * (the first step alone converts u_dev), and under the paired schedule (diff lanes 2)
 * the last order-2 pass of a step runs with the next step's first order-1 pass.
 * Errors as dolinc_rk_step; INVALID_ARG for n_steps < 1. */
dolinc_status dolinc_rk_steps(dolinc_mesh *mesh, const dolinc_scheme *scheme, double dt, int n_steps, double *u_dev,
                              void *ws_dev, size_t ws_bytes, dolinc_stream stream);

/* One SSP-RK3 step (Sec 3), computed as dolinc_rk_step computes it, of a state held
 * in host memory: u_host (FP64 [v][c], library order) holds the step's input and
 * receives the new state.  When u_host is page-locked and mapped into the device
 * address space (cudaHostAlloc / cudaMallocHost / cudaHostRegister memory, as pinned
 * tensors are), the step's first kernel reads it in place over the host link, keeping
 * a device copy of the start state in u_dev, and the last stage writes the new state
 * to it in place: the transfers are part of the step's own kernels.  Other host
 * memory is copied to u_dev and back with cudaMemcpyAsync on the stream (which, for
 * pageable memory, returns only once the copy back has completed).
 * u_dev: caller-owned device scratch of nv * n_cells doubles, contents afterwards
 * unspecified.  With pinned memory the step is asynchronous like every call here:
 * u_host and u_dev must stay valid and untouched until the stream has completed it.
 * Errors as
 * dolinc_rk_step; DOLINC_ERR_INVALID_ARG when u_dev is not device memory or aliases
 * u_host. */
dolinc_status dolinc_rk_step_host(dolinc_mesh *mesh, const dolinc_scheme *scheme, double dt, double *u_host,
                                  double *u_dev, void *ws_dev, size_t ws_bytes, dolinc_stream stream);

/* One SSP-RK3 step, like dolinc_rk_step, without a caller workspace and without any
 * allocation: for callers that hold only the field's device pointer and cannot obtain
 * device memory themselves (for example a plugin that a host application hands its
 * state buffer to, with no allocator of its own).  The paper has no counterpart; this
 * is a deployment convenience.
 * The workspace is a fixed device array of DOLINC_NOALLOC_MAX_BYTES inside the library
 * (32 MiB, held on every GPU that loads the library until the process exits).
 * Meshes/schemes whose dolinc_workspace_size exceeds it are rejected with
 * DOLINC_ERR_INVALID_ARG and a message; nothing is allocated, ever.
 * Every call looks the array's address up on the current device (the first call on a
 * device also loads the library's device code there: make that first call before any
 * stream capture) and clears its first 1024 bytes (status and barrier words) on the
 * stream, as dolinc_workspace_init does for a caller workspace.
 * All calls on a device share the one array, which keeps the last call's contents:
 * calls that overlap on the GPU (different streams, threads or meshes at once) race
 * and must be serialised by the caller.  Device-side errors are NOT reported by this
 * entry point: neither a non-finite result nor a bounded wait of a pipelined kernel
 * that gave up (the status word lives in the array, which the caller cannot read, and
 * the next call clears it).  Callers that need those checks use dolinc_rk_step with a
 * workspace of their own and dolinc_sync_status. */
#define DOLINC_NOALLOC_MAX_BYTES ((size_t)32 << 20)
dolinc_status dolinc_rk_step_noalloc(dolinc_mesh *mesh, const dolinc_scheme *scheme, double dt, double *u_dev,
                                     dolinc_stream stream);

/* Launch-shape autotuner (no counterpart in the paper).  Times the differential and
 * stage kernels of this mesh and scheme on the given state (u_dev, FP64 [v][cell])
 * for 1, 4 and 8 lanes per cell and blocks of 64, 128, 256 threads, and for tiled
 * launches (0 lanes: one thread per cell, the block's 64/128/256 cells and the faces
 * they own staged in shared memory), and for the differential passes also the
 * persistent pipelined launch (-1 / -4 lanes: 1 / 4 lanes per cell, 128 or 256
 * threads per CTA, one CTA per resident slot, each CTA walking over tiles of cells
 * whose records and geometry arrive by bulk asynchronous copies into two
 * shared-memory buffers while the previous tile is computed; a bounded barrier wait
 * that gives up is reported as DOLINC_ERR_DEVICE_TIMEOUT by dolinc_sync_status),
 * and for the stage the face-centric pair (-2 lanes: one thread per face evaluates
 * every face once into a workspace flux array, then one thread per cell, in blocks of
 * 64/128/256, sums its signed fluxes in slot order), keeps the fastest shape in the
 * mesh handle for
 * every later call with this scheme, and appends it to the text file cache_path (one
 * line per GPU name and mesh/scheme key; may be NULL).  A key already in the file is
 * reused without timing.  Synchronous; clears the workspace status word.  Results:
 * *out (may be NULL). */
typedef struct {
    int diff_lanes, diff_block, stage_lanes, stage_block;
    int from_cache;
    double diff_ms, stage_ms;        /* best times (all differential passes / one stage) */
} dolinc_tuning;
dolinc_status dolinc_autotune(dolinc_mesh *mesh, const dolinc_scheme *scheme, const double *u_dev, void *ws_dev,
                              size_t ws_bytes, const char *cache_path, dolinc_stream stream, dolinc_tuning *out);
/* Sets the launch shape used for this mesh and scheme (lanes per cell 1, 4 or 8 with a
 * block of 32..256 threads, a multiple of 32; or lanes 0, tiled, with a block of 64,
 * 128 or 256; differential passes also lanes -1 or -4, pipelined, with 128 or 256, or
 * lanes 2: one thread per cell with the paired schedule, where a scheme computing one
 * order above what its stencil reads (n_diff = 2, stencil order 1) runs that order of
 * stage k in one launch with order 1 of stage k+1, both reading the Gauss weights once,
 * with the same results as lanes 1;
 * the stage also lanes -1, pipelined, with tiles of 64 or 128 cells, or -2, the
 * face-centric pair, with 64, 128 or 256), e.g. a shape read back from an autotuning
 * cache. */
dolinc_status dolinc_set_tuning(dolinc_mesh *mesh, const dolinc_scheme *scheme, const dolinc_tuning *tuning);

/* ---------------------------------------------------------------- troubled cells
 * The paper gives ENO3-DOLINC (Sec 2.4) but no rule for where to use it; the
 * criterion and the network below are this library's, built from the paper's ENO3
 * indicators and DOLINC differentials.  All need an Euler scheme (RUSANOV) with
 * n_diff >= 2 and recompute the differentials of u_dev in the workspace.
 *
 * Criterion: flags_dev[c] (uint8, library order) = 1 if at one of c's interior faces
 *   (i) a reconstructed state (either orientation, the scheme's stencil) has rho <= 0
 *       or p <= 0, or
 *   (ii) with c upwind, for rho or rho E, the ENO3-DOLINC three-cell indicators of
 *       Sec 2.4 satisfy |D_C| > kappa min(|D_L|, |D_R|) and |D_C| > eps (|phi_0|+|phi_1|).
 * Decisions are taken in the scheme's precision.  Defaults used by the tests and the
 * bench: kappa = 4, eps = 1e-3. */
dolinc_status dolinc_criterion(dolinc_mesh *mesh, const dolinc_scheme *scheme, const double *u_dev,
                               uint8_t *flags_dev, double kappa, double eps, void *ws_dev, size_t ws_bytes,
                               dolinc_stream stream);

/* Network inputs x24_dev [n_cells][24] (FP32): per cell its own 6 features (m = 1, 2:
 * the largest |phi^(m)| over its faces of rho, rho E and |momentum|, divided by rho,
 * |E| and sqrt(rho |E|), mapped by log(1+x)), then those of the three largest face
 * neighbours in lexicographic order (itself across a boundary face). */
dolinc_status dolinc_indicator_features(dolinc_mesh *mesh, const dolinc_scheme *scheme, const double *u_dev,
                                        float *x24_dev, void *ws_dev, size_t ws_bytes, dolinc_stream stream);

/* Indicator network 24 -> 64 -> 64 -> 64 -> 1 (ReLU; cell flagged when the logit is
 * positive).  Parameters: 9985 FP32 values W1[64][24] b1[64] W2[64][64] b2 W3[64][64]
 * b3 W4[1][64] b4[1], kept on the device (FP32 master + Adam state); the network
 * computes with their bfloat16 roundings and FP32 accumulation.  Inference runs on
 * the tensor cores (BF16 activations); training runs in FP32 on the same bfloat16
 * weights.  The handle owns its device memory (training scratch grows with the batch). */
typedef struct dolinc_mlp dolinc_mlp;
#define DOLINC_MLP_PARAMS 9985
dolinc_status dolinc_mlp_create(dolinc_mlp **out, uint64_t seed);       /* He-uniform, zero biases */
void dolinc_mlp_destroy(dolinc_mlp *mlp);
dolinc_status dolinc_mlp_get_params(const dolinc_mlp *mlp, float *host_params);   /* synchronous */
dolinc_status dolinc_mlp_set_params(dolinc_mlp *mlp, const float *host_params);   /* synchronous */
/* logits_dev [n] and/or flags_dev [n] (either may be NULL) of inputs x_dev [n][24]. */
dolinc_status dolinc_mlp_forward(dolinc_mlp *mlp, const float *x_dev, int64_t n, float *logits_dev,
                                 uint8_t *flags_dev, dolinc_stream stream);
/* Mean weighted binary cross-entropy on labels y_dev [n] (0/1) with weight pos_weight on
 * positives, into *loss_dev (device float, may be NULL), and its gradient with respect
 * to the parameters into grad_dev [9985] (may be NULL). */
dolinc_status dolinc_mlp_loss_grad(dolinc_mlp *mlp, const float *x_dev, const uint8_t *y_dev, int64_t n,
                                   float pos_weight, float *grad_dev, float *loss_dev, dolinc_stream stream);
/* One Adam step (beta 0.9 / 0.999, eps 1e-8) with learning rate lr on one batch. */
dolinc_status dolinc_mlp_train_step(dolinc_mlp *mlp, const float *x_dev, const uint8_t *y_dev, int64_t n,
                                    float lr, float pos_weight, float *loss_dev, dolinc_stream stream);
/* Features + network: flags_dev [n_cells] (and logits_dev, may be NULL).  x24_dev:
 * caller scratch of n_cells x 24 floats that receives the inputs, or NULL: the
 * network kernel then gathers each cell's 24 inputs itself, without writing them out
 * (the same flags). */
dolinc_status dolinc_indicator_infer(dolinc_mesh *mesh, const dolinc_scheme *scheme, dolinc_mlp *mlp,
                                     const double *u_dev, float *x24_dev, uint8_t *flags_dev, float *logits_dev,
                                     void *ws_dev, size_t ws_bytes, dolinc_stream stream);

/* ---------------------------------------------------------------- batches
 * Many independent meshes advanced together (no counterpart in the paper).  The
 * meshes' cells, slots and faces are concatenated into one arena: batch fields are
 * [v][total cells], mesh b occupying cells [cell_offsets[b], cell_offsets[b+1]) in its
 * own library order.  Each mesh keeps its own time step (dt_dev[b]).
 * dolinc_batch_rk_step runs each SSP-RK3 stage as ONE persistent cooperative launch over
 * all meshes: pack, differential passes and the fused reconstruction/flux/update,
 * separated by grid-wide barriers whose waits are bounded (a wait that gives up makes
 * dolinc_sync_status report DOLINC_ERR_DEVICE_TIMEOUT and leaves the stage output
 * unwritten).  With use_graph the three launches are captured once into a CUDA graph
 * (re-captured when u_dev, ws_dev, dt_dev, the scheme or the launch shape change) and
 * replayed.  Stencils of DOLINC order <= 2, no limiter.  The meshes may be destroyed
 * after dolinc_batch_create (it copies what it needs). */
typedef struct dolinc_batch dolinc_batch;
dolinc_status dolinc_batch_create(dolinc_mesh *const *meshes, int n, dolinc_batch **out);
void dolinc_batch_destroy(dolinc_batch *batch);
dolinc_status dolinc_batch_info(const dolinc_batch *batch, int64_t *n_cells, int64_t *cell_offsets /* [n+1] */);
/* Polls a grid-barrier wait makes (about 0.1 us each) before it gives up (default 2^23).
 * 0 makes every wait give up at once: a way to exercise the timeout path. */
dolinc_status dolinc_batch_set_spin_limit(dolinc_batch *batch, unsigned polls);
dolinc_status dolinc_batch_workspace_size(const dolinc_batch *batch, const dolinc_scheme *scheme, size_t *bytes);
dolinc_status dolinc_batch_rk_step(dolinc_batch *batch, const dolinc_scheme *scheme, const double *dt_dev,
                                   double *u_dev, void *ws_dev, size_t ws_bytes, int use_graph, dolinc_stream stream);
/* Times the persistent launch for blocks of 64/128/256 threads at full and half
 * occupancy on a copy of u_dev (restored afterwards) and keeps the fastest shape.
 * Synchronous. */
dolinc_status dolinc_batch_autotune(dolinc_batch *batch, const dolinc_scheme *scheme, const double *dt_dev,
                                    double *u_dev, void *ws_dev, size_t ws_bytes, dolinc_stream stream, int *block,
                                    int *grid, double *ms_per_step);

/* Cell flags for DOLINC_LIMIT_ENO3_FLAGGED / FIRST_ORDER_FLAGGED: flags_dev [n_cells] uint8 (library order),
 * non-zero = troubled.  The pointer is kept by the mesh until replaced or NULL. */
dolinc_status dolinc_set_flags(dolinc_mesh *mesh, const uint8_t *flags_dev);

/* Values of the Dirichlet and Neumann boundary faces (Sec 2.6: the boundary needs no
 * special treatment beyond the low-order one; the auxiliary cell beyond a face obeys
 * the condition).  values_host [nv][n_faces] in the caller's face order (entries of
 * other faces are not read): the face value T_f on a Dirichlet face, the outward
 * normal gradient q on a Neumann face, where T_f = T_C + q delta with delta the
 * distance from the cell centroid to the face along the outward unit normal.  The
 * first differential pass takes T_f as the face value of the Gauss gradient; higher
 * orders take the boundary cell's own differential; the face state (both
 * orientations) is T_f.  The library copies the values (synchronous); every compute
 * call with a scheme of nv variables needs values set for that nv.  Errors:
 * INVALID_ARG for nv outside 1..5, a mesh without such faces, null or non-finite
 * values.  Batches take no such meshes. */
dolinc_status dolinc_set_boundary_values(dolinc_mesh *mesh, int nv, const double *values_host);

/* Synchronises `stream`, reads and clears the device status word in ws_dev:
 * DOLINC_ERR_NONFINITE if a stage wrote NaN/Inf since the last call,
 * DOLINC_ERR_DEVICE_TIMEOUT if a bounded wait gave up, else DOLINC_OK. */
dolinc_status dolinc_sync_status(dolinc_mesh *mesh, void *ws_dev, dolinc_stream stream);

/* Per-kernel timing.  While enabled, every compute call on this mesh records CUDA
 * events around each of its kernel launches, on the call's stream.  Kernel kinds:
 * DOLINC_KERNEL_PACK (FP64 field -> order-0 record), DOLINC_KERNEL_DIFF1..DIFF4 (the
 * differential pass producing order m), DOLINC_KERNEL_STAGE (reconstruction + flux +
 * residual + update), DOLINC_KERNEL_FACES (dolinc_reconstruct_faces),
 * DOLINC_KERNEL_DIFF_PAIR (one stage's order-2 pass fused with the next stage's
 * order-1 pass, under the paired schedule of dolinc_set_tuning's diff_lanes = 2),
 * DOLINC_KERNEL_SOLVE (one linear solve of dolinc_implicit_step).
 * dolinc_profile_enable resets the counters.  dolinc_profile_read waits for the
 * recorded events and fills ms[DOLINC_KERNEL_COUNT] (summed device time) and
 * launches[DOLINC_KERNEL_COUNT]; either pointer may be NULL. */
enum { DOLINC_KERNEL_PACK = 0, DOLINC_KERNEL_DIFF1 = 1, DOLINC_KERNEL_DIFF2 = 2, DOLINC_KERNEL_DIFF3 = 3,
       DOLINC_KERNEL_DIFF4 = 4, DOLINC_KERNEL_STAGE = 5, DOLINC_KERNEL_FACES = 6, DOLINC_KERNEL_DIFF_PAIR = 7,
       DOLINC_KERNEL_SOLVE = 8, DOLINC_KERNEL_COUNT = 9 };
dolinc_status dolinc_profile_enable(dolinc_mesh *mesh, int enable);
dolinc_status dolinc_profile_read(dolinc_mesh *mesh, double *ms, int64_t *launches);

/* Skewness correction (no counterpart in the paper's method: the paper names the low
 * accuracy of its inversion on tetrahedral and hybrid grids as future work, Sec 4).
 * The Eq 3 interpolation and the DOLINC reconstruction along d give a face the value
 * of the point x*_f = x_P + (1 - w) d of the centroid line, which on a skewed mesh is
 * not the face centroid x_f.  With the correction on:
 *   - every differential pass applies, per cell, M_c^-1 to the new gradient index,
 *     M_c = (1/V_c) sum_f S_{c,f} (x) (x*_f - x_c) (the identity when every x*_f = x_f,
 *     as on geometric strips and stretched hexahedra, where the scheme is unchanged);
 *     it is folded into the mesh's weight tables, so the passes cost the same;
 *   - each face state adds (x_f - x*_f) . T^(1) of its upwind cell (not on faces of
 *     the first-order fallback).
 * Both together reproduce linear fields exactly at face centroids on meshes with
 * planar faces.  Boundary faces count as unskewed (x*_f = x_f).  A mesh option: every
 * scheme on the mesh uses it.  Synchronises the device (call between steps).  Errors:
 * UNSUPPORTED on a mesh with Dirichlet/Neumann faces, MESH if some M_c is singular
 * (the correction then stays off).  Batches take no mesh with the correction on. */
dolinc_status dolinc_mesh_set_skew_correction(dolinc_mesh *mesh, int enable);

/* ---------------------------------------------------------------- partitioned meshes
 * Halo-exchanged parts of one mesh, one part per GPU (Sec 2.6: a coupled boundary
 * exchanges only the adjacent cells' data plus their differentials).  A part holds
 * its own cells and a depth-1 layer of ghost cells (cells of other parts sharing a
 * face with an own cell).  Each differential pass reads only face neighbours and the
 * reconstruction only the two face cells' records (Secs 2.3-2.4), so before each pass
 * a part needs its ghosts' records of the order that pass reads, and before the stage
 * the ghosts' records of every order the stage reads: one exchange per order, of
 * depth 1.  A part keeps the whole mesh's library cell order and face order and
 * orientation, and copies the whole mesh's geometry, so its own cells compute exactly
 * what the whole mesh computes for them (the same operands in the same order). */

/* Space-filling-curve partition: cells in Morton order of their centroids (the
 * library order of DOLINC_RENUMBER_MORTON) cut into n_parts contiguous ranges of
 * equal size (+-1).  part_of_cell[n_cells] (host) gets each caller cell's part.
 * Host only; no GPU needed.  Errors: INVALID_ARG (null pointers, n_parts < 1 or
 * above n_cells), MESH as dolinc_mesh_create. */
dolinc_status dolinc_partition(const dolinc_mesh_desc *desc, int n_parts, int32_t *part_of_cell);

typedef struct {
    int64_t n_local;        /* own + ghost cells of the part */
    int64_t n_owned;
    int64_t n_faces;        /* faces of the own cells */
    int32_t n_peers;        /* parts this part exchanges with */
    int64_t n_send;         /* records sent per exchange (all peers) */
    int64_t n_recv;         /* records received per exchange (all peers) */
} dolinc_part_sizes;

/* The plan of part `part` of the mesh under part_of_cell (caller cell order, values
 * 0..n_parts-1; any assignment, e.g. dolinc_partition's).  Host only; no GPU needed.
 * Call with NULL arrays to get `sizes`, then with arrays of those sizes (host):
 *   local_cells [n_local]  caller cell id of each local cell, in the part's order
 *                          (the whole mesh's library order restricted to the part);
 *                          a part mesh's fields are [v * n_local + j] in this order
 *   owned       [n_local]  1 own cell, 0 ghost
 *   peers       [n_peers]  the other parts, ascending
 *   send_off, recv_off [n_peers + 1]   offsets into send_cells / recv_cells per peer
 *   send_cells  [n_send]   local indices of own cells peer q holds as ghosts
 *   recv_cells  [n_recv]   local indices of the ghosts peer q owns
 * Each list is in ascending library order, so part p's send list to q names the same
 * cells, in the same order, as q's recv list from p.  Errors: INVALID_ARG (bad part,
 * part_of_cell entry out of range, a part with no cell), MESH as dolinc_mesh_create. */
dolinc_status dolinc_part_plan(const dolinc_mesh_desc *desc, const int32_t *part_of_cell, int n_parts, int part,
                               dolinc_part_sizes *sizes, int64_t *local_cells, uint8_t *owned, int32_t *peers,
                               int64_t *send_off, int64_t *send_cells, int64_t *recv_off, int64_t *recv_cells);

/* Device mesh of part `part` (arguments as dolinc_part_plan; desc->renumber chooses
 * the library order, as for the whole mesh).  Its cells are the plan's local cells,
 * in that order (the permutation is the identity); its faces are the own cells'
 * faces; its workspace (dolinc_workspace_size) also holds the exchange buffers.
 * Destroy with dolinc_mesh_destroy.  Every other entry point accepts it; the ghosts'
 * results of those are meaningless.  Errors as dolinc_part_plan, plus OOM / CUDA. */
dolinc_status dolinc_mesh_create_part(const dolinc_mesh_desc *desc, const int32_t *part_of_cell, int n_parts,
                                      int part, dolinc_mesh **out);

dolinc_status dolinc_mesh_part_sizes(const dolinc_mesh *mesh, dolinc_part_sizes *sizes);

/* A pending halo exchange of a partitioned step.  When pending = 1 the caller moves,
 * for every peer q (in the plan's order), the record_bytes * (send_off[q+1] -
 * send_off[q]) bytes at send_dev + record_bytes * send_off[q] to peer q, and fills
 * recv_dev + record_bytes * recv_off[q] with what q sends (both device buffers inside
 * the workspace; e.g. NCCL send/recv on `stream`), then calls dolinc_part_step_continue.
 * order: the differential order being exchanged (0 = the stage's cell averages). */
typedef struct {
    int pending;
    int order;
    size_t record_bytes;
    void *send_dev;
    void *recv_dev;
} dolinc_halo;

/* One SSP-RK3 step of a part mesh, with a halo exchange before each differential
 * pass and before the stage kernel of each of the three stages (orders 0 ..
 * max(n_diff - 1, stencil order) per stage).  dolinc_part_step_begin packs u (the
 * part's FP64 state, own cells and ghosts, [v * n_local + j]; the ghosts' values are
 * not read) and stops at the first exchange with *halo filled; each
 * dolinc_part_step_continue takes the received records into the ghosts and runs to the
 * next exchange, or to the end of the step (halo->pending = 0; u then holds the own
 * cells' new state; the ghosts' entries are meaningless, and must hold finite values
 * when the step begins).  One step uses one scheme, workspace and stream from begin to
 * its end; a begin abandons a step in progress.  All launches on `stream`; the
 * exchange must be ordered on it too.  Errors: INVALID_ARG (not a part mesh, continue
 * without a step in progress, workspace), as dolinc_rk_step otherwise. */
dolinc_status dolinc_part_step_begin(dolinc_mesh *mesh, const dolinc_scheme *scheme, double dt, double *u_dev,
                                     void *ws_dev, size_t ws_bytes, dolinc_stream stream, dolinc_halo *halo);
dolinc_status dolinc_part_step_continue(dolinc_mesh *mesh, const dolinc_scheme *scheme, void *ws_dev,
                                        size_t ws_bytes, dolinc_stream stream, dolinc_halo *halo);

/* ------------------------------------------------------------ semi-implicit step
 * Sec 2.4 (Eq USR3, Eq CSR4): a DOLINC face value is  w_s phi_up + (1 - w_s) phi_down
 * + c_r,  the weights w_s, 1 - w_s of the two face cells' averages plus c_r, the part
 * that carries the inverted far-field data.  The paper notes that under an implicit
 * time integration this gives a semi-implicit scheme: the weight part is taken at the
 * new time level, c_r stays explicit.  For linear advection (flux UPWIND, nv = 1) and
 * theta in [0, 1] one step solves
 *     V (u' - u) / dt = -theta K u' - (1 - theta) K u - C(u),
 * (K x)_c = sum over the faces of c of a.S_{c,f} (w_s x_up + (1 - w_s) x_down), with
 * a.S u_c on a zero-gradient boundary face, and C(u)_c the sum of a.S_{c,f} c_r.  In
 * delta form  (V/dt + theta K) delta = V R(u),  R the explicit DOLINC residual of the
 * scheme (dolinc_residual: differentials, reconstruction, flux; at the scheme's
 * precision and with its limiter and the mesh's skewness correction), u' = u + delta.
 * The rows are scaled by their diagonal and solved by BiCGSTAB in FP64, all iterations
 * in one cooperative launch, to ||b - A delta|| <= rel_tol ||b|| on the scaled rows.
 * theta = 0 is the explicit forward Euler step.
 *
 * n_outer > 1 repeats the solve with c_r of the latest iterate at the new level
 * (deferred correction):
 *     V (u^(k+1) - u) / dt = -theta K u^(k+1) - (1 - theta) (K u + C(u)) - theta C(u^(k));
 * its fixed point is the theta scheme of the full DOLINC operator.
 *
 * dolinc_implicit_create assembles the rows on the mesh's device (the mesh must outlive
 * the solver) and waits for them.  Errors: UNSUPPORTED for another flux, nv != 1,
 * Dirichlet/Neumann faces or a part mesh; INVALID_ARG for dt <= 0 or theta outside
 * [0, 1]; OOM. */
typedef struct dolinc_implicit dolinc_implicit;
dolinc_status dolinc_implicit_create(dolinc_mesh *mesh, const dolinc_scheme *scheme, double dt, double theta,
                                     dolinc_implicit **out);
void dolinc_implicit_destroy(dolinc_implicit *solver);

/* Solver settings: relative tolerance (default 1e-10), iterations per solve (default
 * 1000), the polls a grid-barrier wait makes before it gives up (default 2^23), and
 * warm_start (default 0): the initial guess of each step's first solve is 0, the
 * previous step's first solution (1), or its linear extrapolation from the last two
 * steps, 2 x(n-1) - x(n-2) (2; the previous solution while only one is kept); the
 * outer corrections start from 0.  The call waits for the device and forgets the kept
 * solutions.  INVALID_ARG for rel_tol < 0, max_iter < 1 or warm_start outside 0..2. */
dolinc_status dolinc_implicit_set_solver(dolinc_implicit *solver, double rel_tol, int max_iter,
                                         unsigned spin_limit, int warm_start);

/* Layout of the rows the solve reads: an ELL width (4, 6 or 8, at least the mesh's
 * largest number of faces per cell; entry q of cell c at q n_cells + c, padded with the
 * cell itself at weight 0) or 0 (per face slot, the default).  Both give the same
 * rows; the per-cell sums keep their order.  Re-assembles the rows and waits for the
 * device.  INVALID_ARG for another width; OOM when the new rows do not fit, after which
 * the solver has no rows and dolinc_implicit_step / _rows return INVALID_ARG until a
 * dolinc_implicit_set_layout succeeds.  dolinc_implicit_layout returns the current
 * layout (-1 for NULL). */
dolinc_status dolinc_implicit_set_layout(dolinc_implicit *solver, int ell);
int dolinc_implicit_layout(const dolinc_implicit *solver);

/* One step on u_dev (FP64 [cell], library order, in place), n_outer >= 1 solves.  ws:
 * a workspace of the mesh and scheme (dolinc_workspace_size), used for the residual.
 * All launches on `stream`, asynchronous.  A solve that stops at max_iter or breaks
 * down still applies its last iterate; dolinc_implicit_info reports it. */
dolinc_status dolinc_implicit_step(dolinc_implicit *solver, double *u_dev, int n_outer, void *ws_dev,
                                   size_t ws_bytes, dolinc_stream stream);

/* The last step's solves: iterations summed over them, their number, whether all
 * reached rel_tol, whether one broke down (a zero BiCGSTAB denominator), and the last
 * solve's final ||b - A delta|| / ||b||; and the iterations and solves of every step
 * since the solver was created.  Waits for the last step's stream.
 * DOLINC_ERR_DEVICE_TIMEOUT if a grid-barrier wait gave up: that solve stopped in
 * every block and the step's result is not valid. */
typedef struct {
    int iterations;
    int solves;
    int converged;
    int breakdown;
    double rel_residual;
    int64_t total_iterations;
    int64_t total_solves;
} dolinc_solve_info;
dolinc_status dolinc_implicit_info(dolinc_implicit *solver, dolinc_solve_info *info);

/* Host copies of the assembled rows of V/dt + theta K, library order: row_offsets
 * [n_cells + 1] (the mesh's face slots), nbr [n_slots] the neighbour of each slot,
 * off [n_slots] its coefficient in the row (a cell can be its own neighbour across a
 * periodic face), diag [n_cells]. */
dolinc_status dolinc_implicit_rows(const dolinc_implicit *solver, int32_t *row_offsets, int32_t *nbr, double *off,
                                   double *diag);

/* Message of the calling thread's last failing call ("" if none). */
const char *dolinc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* DOLINC_H */
