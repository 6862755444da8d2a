/*
 * fem.h -- C ABI of libfem_gb300: low-order finite element integration by
 * tensor contraction on NVIDIA GB300 (sm_103a).
 *
 * Method: Knepley & Terrel, "Finite Element Integration on GPUs" (TACC
 * TR-11-01).  For every element e the library gathers the vertex
 * coordinates, forms the Jacobian J of the affine map from the reference
 * simplex, |J| = |det J| and J^{-1}, builds the geometric tensor G_e (Eq. 8,
 * times an optional per-element coefficient w_e, the piecewise-constant case
 * of Eq. 20) and contracts it with the precomputed reference tensor K
 * (Eq. 7): A_e^{ij} = G_e^{mu nu} K^{ij}_{mu nu} (Eq. 1, Eq. 6).
 *
 * Conventions shared by every entry point
 *   - Pointers named "device" are CUDA device (or managed) memory owned by the
 *     caller; the library never allocates on the integration path and never
 *     frees caller memory.  Host pointers are named "host".
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Device work is enqueued asynchronously on it; the call returns once the
 *     work is enqueued.
 *   - Host-detectable errors (null pointers, bad sizes, unsupported
 *     combinations) return a non-zero fem_status before anything is launched;
 *     fem_last_error() then gives a one-line reason (thread-local).
 *   - Device-detectable errors never trap: the element is skipped (its outputs
 *     are written as zeros) and FEM_DEVERR_* bits are OR-ed into
 *     options->dev_err when that pointer is non-NULL.
 *   - Reference simplex vertices are 0, e_1, .., e_d; J_{a mu} = x_{mu+1,a} - x_{0,a}.
 *   - Element matrices are [E][n][n] row-major.  P2 basis order: vertex
 *     functions, then edge functions over edges in lexicographic order.
 *     Vector (elasticity) DOF index = component * n_basis + basis.
 */
#ifndef FEM_GB300_H
#define FEM_GB300_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define FEM_API __attribute__((visibility("default")))
#else
#define FEM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FEM_OK = 0,
  FEM_ERR_ARG = 1,         /* invalid argument (null pointer, bad size or enum) */
  FEM_ERR_UNSUPPORTED = 2, /* valid but unsupported combination */
  FEM_ERR_WORKSPACE = 3,   /* workspace missing or too small */
  FEM_ERR_CUDA = 4         /* a CUDA runtime call failed (message in fem_last_error) */
} fem_status;

/* Weak forms (Sec. 3).  The first three take an optional per-element
 * coefficient w_e; the _W1 forms take a P1 coefficient w = sum_k w_k lambda_k
 * given by its values at the mesh vertices (Eqs. 20-23), so `coef` is
 * [n_vert] for them, and their adjoint's dcoef is the gradient of those vertex
 * values, [n_vert].  The _W1 forms have no batched path (FEM_ERR_UNSUPPORTED);
 * FEM_LAPLACE_P2_W1 also contracts on the tensor cores. */
typedef enum {
  FEM_LAPLACE_P1 = 0,    /* Eqs. 2-8 with P1 Lagrange elements */
  FEM_LAPLACE_P2 = 1,    /* same form, P2 Lagrange elements */
  FEM_ELASTIC_P1 = 2,    /* eps(v):eps(u), Eq. 10 scaled by the 1/4 of Eqs. 14 and 24, P1 vector elements */
  FEM_LAPLACE_P1_W1 = 3, /* int w grad v . grad u with w in P1 (Eqs. 20-23), P1 elements */
  FEM_LAPLACE_P2_W1 = 4, /* the same with P2 elements: K gains the coefficient's index (Eq. 21) */
  FEM_LAPLACE_P1_ISO = 5, /* the Laplacian on non-affine (quadratic-geometry) elements, Eqs. 16-19, P1 */
  FEM_LAPLACE_P2_ISO = 6, /* the same with P2 elements (fem_integrate_fwd_iso only) */
  /* Coupling blocks of a multiphysics pair (Sec. 6: coupled systems broken
   * into blocks): B_{i,(c,j)} = int_T w phi_i d psi_j / d x_c, i.e. int w q div v
   * for a scalar field q in P1 and a vector field v.  Rows i = 0..d (the P1
   * basis), columns c * nbv + j (the vector basis, component-major), so the
   * element blocks are RECTANGULAR [n_elem][d+1][d * nbv] (fem_form_shape).
   * G^{mu c} = w |J| J^{-1}_{mu c} and K^{ij}_mu = int_ref lambda_i d_mu psi_j
   * (Eq. 1 with a value and a derivative).  FP32 coordinates and output, the
   * compensated Jacobian (for the sign of det J) and the FP32 contraction;
   * forward, fem_integrate_fwd_save and the adjoint (both reductions). */
  FEM_DIV_P1P1 = 7, /* v in [P1]^d: 4 x 12 blocks on tets, 3 x 6 on triangles */
  FEM_DIV_P2P1 = 8  /* v in [P2]^d (the Taylor-Hood pair): 4 x 30 on tets, 3 x 12 on triangles */
} fem_form;

typedef enum { FEM_F32 = 0, FEM_F64 = 1 } fem_dtype;

/* Precision of the Jacobian steps (J, det J, J^{-1}, G). */
typedef enum {
  FEM_JAC_AUTO = 0,     /* COMP_F32 for FP32 coordinates and FP32 output, F64 otherwise */
  FEM_JAC_F64 = 1,      /* FP64 */
  FEM_JAC_COMP_F32 = 2, /* compensated FP32 (error-free transforms; accurate det on slivers) */
  FEM_JAC_F32 = 3       /* plain FP32, for error studies */
} fem_jac;

/* Arithmetic of the G:K contraction. */
typedef enum {
  FEM_CONTRACT_F32 = 0,   /* FP32 FMAs with K as compile-time immediates (sparse) */
  FEM_CONTRACT_BF16X3 = 1 /* tensor cores: G split into three bf16 terms, FP32 accumulate; P2 Laplacian
                             (per-element or P1 coefficient) and P1 elasticity, FP32 coordinates and
                             output, compensated Jacobian (curved P2: fem_integrate_fwd_iso) */
} fem_contract;

/* Vertex reduction of the adjoint. */
typedef enum {
  FEM_REDUCE_DETERMINISTIC = 0, /* per-element scratch + segmented sum in a fixed order */
  FEM_REDUCE_ATOMIC = 1,        /* red.global.add into dcoords (order not fixed) */
  FEM_REDUCE_DEFERRED = 2       /* element pass only: contributions stay in the workspace
                                   scratch; fem_adjoint_reduce completes dcoords */
} fem_reduce;

/* Device error bits (OR-ed into options->dev_err). */
#define FEM_DEVERR_CONN 1       /* a connectivity index is outside [0, n_vert) */
#define FEM_DEVERR_DEGENERATE 2 /* det J == 0 */

/* A simplex mesh.  conn: device int32 [n_elem][dim+1]; coords: device
 * [n_vert][dim] of coord_dtype (FP32 or FP64), row-major. */
typedef struct fem_mesh {
  int32_t dim;         /* 2 (triangles) or 3 (tetrahedra) */
  int32_t coord_dtype; /* fem_dtype */
  int64_t n_vert;
  int64_t n_elem;
  const int32_t* conn;
  const void* coords;
} fem_mesh;

/* Options; a zero-initialised struct (or NULL) selects the defaults. */
typedef struct fem_options {
  int32_t jac;           /* fem_jac */
  int32_t contract;      /* fem_contract */
  int32_t reduce;        /* fem_reduce */
  int32_t warps_per_cta; /* 0 = default; else 1..16 warps (32-element tiles) per CTA */
  int32_t ctas_per_sm;   /* 0 = one CTA per group of tiles; >0 = grid capped at this many CTAs per SM */
  int32_t reserved;      /* must be 0 */
  int32_t* dev_err;      /* optional device int32, OR-ed with FEM_DEVERR_* bits */
} fem_options;

/* Library version string (static storage). */
FEM_API const char* fem_version(void);

/* Name of a status code (static storage). */
FEM_API const char* fem_status_string(fem_status s);

/* Reason for the last non-OK status returned on the calling thread. */
FEM_API const char* fem_last_error(void);

/* Host.  Shape of a form: n = rows of A_e, n_geom = folded entries of G
 * (d(d+1)/2 for the Laplacian, d^2(d^2+1)/2 for elasticity, (d+1) d(d+1)/2
 * for the _W1 forms: slot k*d(d+1)/2 + g holds w_k G_g), den = the integer
 * scale of fem_reference_tensor.  Any output pointer may be NULL. */
FEM_API fem_status fem_form_info(int32_t form, int32_t dim, int32_t* n, int32_t* n_geom, int32_t* den);

/* Host.  Rows and columns of a form's element blocks: rows == cols == n for
 * every form but the coupling forms (d+1 rows, d * nbv columns).  Either
 * output may be NULL. */
FEM_API fem_status fem_form_shape(int32_t form, int32_t dim, int32_t* rows, int32_t* cols);

/* Host.  The reference tensor K of Eq. 7 (Eq. 14 with the symmetric gradient
 * for elasticity), folded over the symmetric G slots and scaled to exact
 * integers: K_host[g][i][j] = den * K'_g^{ij}, with A_e^{ij} = sum_g G_g K'_g^{ij}.
 * K_host: host int32 array of at least n_geom*rows*cols entries (cap =
 * entries).  For the coupling forms g = mu * d + c (G_g = w |J| J^{-1}_{mu c},
 * not folded) and K_host[g][i][c' * nbv + j] = den K^{ij}_mu when c' == c, else 0. */
FEM_API fem_status fem_reference_tensor(int32_t form, int32_t dim, int32_t* K_host, size_t cap);

/* Forward element integration, Sec. 4 / Eq. 6: A[e] = G_e : K for every element.
 *   coef : device FP32 [n_elem] per-element coefficient w_e, or NULL (w = 1);
 *          for the _W1 forms FP32 [n_vert] vertex values of the P1 coefficient
 *   A    : device [n_elem][rows][cols] of out_dtype (overwritten); rows = cols = n
 *          except for the coupling forms (fem_form_shape)
 *   FP64 output or FP64 coordinates compute the Jacobian steps in FP64.
 * Asynchronous on `stream`.  n_elem == 0 is a no-op. */
FEM_API fem_status fem_integrate_fwd(const fem_mesh* mesh, int32_t form, const float* coef, void* A,
                             int32_t out_dtype, const fem_options* options, void* stream);

/* Forward integration that also saves det J for the adjoint (reverse mode
 * keeps what the forward computed): as fem_integrate_fwd, and
 *   det : device FP32 [n_elem], overwritten: det J of each element as the
 *         Jacobian mode computed it (the compensated value by default; 0 for
 *         an element with an invalid vertex).
 * FP32 contraction only (FEM_ERR_UNSUPPORTED otherwise).  Pass det to
 * fem_integrate_bwd_saved. */
FEM_API fem_status fem_integrate_fwd_save(const fem_mesh* mesh, int32_t form, const float* coef, void* A,
                                          int32_t out_dtype, float* det, const fem_options* options, void* stream);

/* Forward integration on non-affine elements (Eqs. 16-19), forms
 * FEM_LAPLACE_P1_ISO / FEM_LAPLACE_P2_ISO, FP32 coordinates and output.  Each
 * element has quadratic geometry: its d+1 vertices and its edge-midpoint nodes
 *   mid : device FP32 [n_elem][d(d+1)/2][dim], edges in the P2 order
 *         (0,1),(0,2),(1,2) / (0,1),(0,2),(0,3),(1,2),(1,3),(2,3)
 * J^{-1} is projected onto P1 by its values at the vertices (Eq. 17) and |J|
 * is |det J| at the centroid, so G^{(k mu),(l nu)} = w |J| J^{-1}_{mu a,k}
 * J^{-1}_{nu a,l} is contracted with K^{ij}_{(k mu),(l nu)} = int_ref lambda_k
 * lambda_l d_mu phi_i d_nu phi_j (Eqs. 18-19).  The Jacobian steps run in
 * plain FP32 (options->jac FEM_JAC_AUTO or FEM_JAC_F32).  The contraction is
 * FP32 (FEM_CONTRACT_F32), or for FEM_LAPLACE_P2_ISO split-BF16 on the tensor
 * cores (FEM_CONTRACT_BF16X3: G in three BF16 terms, K exact, FP32
 * accumulation).  coef: [n_elem] or NULL; A: [n_elem][n][n] FP32.
 * Straight-sided elements (mid at the edge midpoints) give the affine
 * result. */
FEM_API fem_status fem_integrate_fwd_iso(const fem_mesh* mesh, int32_t form, const float* mid, const float* coef,
                                         float* A, const fem_options* options, void* stream);

/* Test hook for the Jacobian steps (Eqs. 5, 8): per element det J (detJ,
 * device FP64 [n_elem]; the compensated mode returns its double-float value)
 * and the Laplacian geometric tensor G^{mu nu} = w |J| sum_a Jinv_{mu a} Jinv_{nu a}
 * (G, device FP32 [n_elem][d(d+1)/2], pairs mu <= nu in row-major order).
 * Either output may be NULL.  Degenerate/invalid elements get 0. */
FEM_API fem_status fem_geometry(const fem_mesh* mesh, const float* coef, const fem_options* options,
                        double* detJ, float* G, void* stream);

/* Bytes of device workspace fem_integrate_bwd (fem_integrate_bwd_iso for the
 * non-affine forms) needs for this mesh and form (vertex->incidence CSR plus
 * per-element scratch for the deterministic reduction; 0 extra scratch for
 * FEM_REDUCE_ATOMIC). */
FEM_API fem_status fem_bwd_workspace_size(const fem_mesh* mesh, int32_t form, const fem_options* options,
                                  size_t* bytes);

/* Builds the vertex -> (element, local vertex) incidence CSR, sorted by
 * (vertex, element, local vertex), into the workspace `ws` (device, caller
 * owned, ws_bytes from fem_bwd_workspace_size).  Once per mesh connectivity;
 * it must precede fem_integrate_bwd with FEM_REDUCE_DETERMINISTIC. */
FEM_API fem_status fem_incidence_build(const fem_mesh* mesh, void* ws, size_t ws_bytes, void* stream);

/* Record layouts of a built adjoint workspace (fem_incidence_info). */
#define FEM_RECORDS_VERTEX_MAJOR 0 /* record rows grouped by vertex: the element pass writes each
                                      record to its vertex's rows (elements in spatial order) */
#define FEM_RECORDS_TILE_ORDER 1   /* records stay in tile order and the reduction gathers them
                                      (elements or vertices in no spatial order) */

/* Host query of a workspace built by fem_incidence_build (synchronizes
 * `stream`): *n_records = the records of the deterministic reduction (one per
 * distinct vertex of each 32-element tile) and *layout = the FEM_RECORDS_*
 * layout the build chose from the mesh's locality (the result bits do not
 * depend on it).  Either output may be NULL. */
FEM_API fem_status fem_incidence_info(const fem_mesh* mesh, const void* ws, size_t ws_bytes, int64_t* n_records,
                                      int32_t* layout, void* stream);

/* Adjoint of fem_integrate_fwd (FP32 coordinates): for the upstream
 * dA = dL/dA (device FP32 [n_elem][rows][cols]) computes
 *   dcoords = dL/dcoords  (device FP32 [n_vert][dim], overwritten; may be NULL)
 *   dcoef   = dL/dcoef    (device FP32 [n_elem], overwritten; may be NULL);
 *             for the _W1 forms [n_vert], the gradient of the coefficient's
 *             vertex values, summed over the elements at each vertex like
 *             dcoords (so it uses the workspace with the deterministic
 *             reduction even when dcoords is NULL)
 * The _W1 forms take the compensated Jacobian and the deterministic or atomic
 * reduction (FEM_REDUCE_DEFERRED: FEM_ERR_UNSUPPORTED); their workspace
 * (fem_bwd_workspace_size with the form) holds records of dim + 1 components.
 * through dG = dA K^T, then d|J| and d adj(J), then the vertex sums.
 * Deterministic reduction: bitwise reproducible, needs the built incidence in ws.
 * Atomic reduction: ws may be NULL.  Deferred: the element pass only (dcoords
 * must be non-NULL, is not written here; call fem_adjoint_reduce next). */
FEM_API fem_status fem_integrate_bwd(const fem_mesh* mesh, int32_t form, const float* coef,
                             const float* dA, float* dcoords, float* dcoef, void* ws,
                             size_t ws_bytes, const fem_options* options, void* stream);

/* Adjoint with det J saved by fem_integrate_fwd_save on the same mesh and
 * form (device FP32 [n_elem]): the element pass forms the edge vectors and
 * adj(J) in FP32 and takes det J from `det` instead of recomputing it, so the
 * compensated determinant is computed once per step.  With the default
 * compensated Jacobian on both sides the results are bitwise those of
 * fem_integrate_bwd; options->jac is not used.  Other arguments, the
 * reductions and the errors as fem_integrate_bwd. */
FEM_API fem_status fem_integrate_bwd_saved(const fem_mesh* mesh, int32_t form, const float* coef,
                                           const float* dA, const float* det, float* dcoords, float* dcoef,
                                           void* ws, size_t ws_bytes, const fem_options* options, void* stream);

/* Adjoint of fem_integrate_fwd_iso (Eqs. 16-19): for the upstream dA = dL/dA
 * (device FP32 [n_elem][n][n]) of the non-affine Laplacian (form
 * FEM_LAPLACE_P1_ISO or FEM_LAPLACE_P2_ISO, FP32 coordinates, the plain-FP32
 * Jacobian steps of the forward) computes
 *   dcoords = dL/dcoords (device FP32 [n_vert][dim], overwritten; may be NULL),
 *   dmid    = dL/dmid    (device FP32 [n_elem][d(d+1)/2][dim], the edge nodes'
 *             gradients element by element; may be NULL),
 *   dcoef   = dL/dcoef   (device FP32 [n_elem], per-element coefficient; may be NULL)
 * by the forward's steps in reverse: the contraction's adjoint one folded slot
 * pair at a time, then J^{-1} at the vertices (J^{-1} projected onto P1,
 * Eq. 17) and |det J| at the centroid pulled back through the quadratic
 * geometry map to the nodes.  mid, coef: as fem_integrate_fwd_iso.  The
 * reductions of dcoords as fem_integrate_bwd (the deterministic one through
 * the workspace of fem_bwd_workspace_size / fem_incidence_build with this
 * form; FEM_REDUCE_DEFERRED leaves dcoords to fem_adjoint_reduce).  Elements
 * that are degenerate (J singular at a vertex or at the centroid) or have an
 * invalid vertex contribute zeros and set the device error bits.
 * options->contract: FEM_CONTRACT_F32, or FEM_CONTRACT_BF16X3 for
 * FEM_LAPLACE_P2_ISO on tetrahedra with the deterministic or deferred
 * reduction: the contraction's adjoint (sym(dA) times K' transposed) then
 * runs on the tcgen05 tensor cores, sym(dA) split into three BF16 terms with
 * FP32 accumulation; other combinations return FEM_ERR_UNSUPPORTED. */
FEM_API fem_status fem_integrate_bwd_iso(const fem_mesh* mesh, int32_t form, const float* mid, const float* coef,
                                         const float* dA, float* dcoords, float* dmid, float* dcoef, void* ws,
                                         size_t ws_bytes, const fem_options* options, void* stream);

/* Second phase of a FEM_REDUCE_DEFERRED adjoint: dcoords[v] (device FP32
 * [n_vert][dim], overwritten) = sum over the incidence segment of v, in
 * (element, local vertex) order, of the per-element contributions the element
 * pass left in `ws`.  Same result bits as FEM_REDUCE_DETERMINISTIC. */
FEM_API fem_status fem_adjoint_reduce(const fem_mesh* mesh, const void* ws, size_t ws_bytes,
                                      float* dcoords, void* stream);

/* ------------------------------------------------------------------ batches
 * Many meshes of uneven size and mixed forms integrated by persistent kernel
 * launches (an addition beside the method; the batch notion of Sec. 4 is the
 * paper's elementBatchSize within one mesh).  Persistent CTAs pull work items
 * from a global counter: first 128-element tiles (forward A and/or the
 * adjoint's element pass), then per-mesh vertex ranges of the deterministic
 * reduction, each of which waits (bounded) for its mesh's tiles.  Modes:
 *   FEM_BATCH_SINGLE      one kernel over every mesh of every kind
 *   FEM_BATCH_GROUPED     one kind-specialised, pipelined kernel per
 *                         (dim, form) kind present, in order on `stream`
 *   FEM_BATCH_GROUPED_CONCURRENT  the same kernels, the largest group on
 *                         `stream` and the others forked onto side streams
 *                         (event fork/join, so the whole run is still
 *                         captured by a CUDA graph on `stream`)
 *   FEM_BATCH_PER_ITEM    each item through the single-mesh kernels of
 *                         fem_integrate_fwd / fem_integrate_bwd (the better
 *                         choice for a few large meshes), on `stream`
 *   FEM_BATCH_PER_ITEM_CONCURRENT  the same, the items spread over ten
 *                         streams (longest first, each to the least loaded;
 *                         event fork/join on `stream`, graph-capturable), so
 *                         small meshes run beside large ones
 *   FEM_BATCH_PHASED      per (dim, form) kind, three persistent launches over
 *                         all of the kind's meshes: the forward, the adjoint
 *                         element pass, the vertex reduction.  Each warp takes
 *                         every S-th 32-element tile of the kind's meshes
 *                         numbered one after the other, and the single-mesh
 *                         kernels' pipeline runs across mesh boundaries; the
 *                         kinds run on concurrent streams (the largest on
 *                         `stream`; event fork/join, graph-capturable)
 * Every mode gives the same result bits as the per-mesh entry points.
 * Items may also be coupling blocks (FEM_DIV_P1P1, FEM_DIV_P2P1); a batch
 * holding one runs the per-item modes only (fem_batch_set_config refuses the
 * others with FEM_ERR_UNSUPPORTED; the tuner and the default pick among the
 * per-item modes). */
#define FEM_BATCH_SINGLE 0
#define FEM_BATCH_GROUPED 1
#define FEM_BATCH_GROUPED_CONCURRENT 2
#define FEM_BATCH_PER_ITEM 3
#define FEM_BATCH_PER_ITEM_CONCURRENT 4
#define FEM_BATCH_PHASED 5

#define FEM_PHASE_FWD 1 /* forward element matrices into item.A */
#define FEM_PHASE_BWD 2 /* adjoint of item.dA into item.dcoords / item.dcoef */
#define FEM_DEVERR_TIMEOUT 4 /* a bounded wait in a batched launch gave up (that mesh's dcoords not written) */

/* One mesh of a batch (FP32 coordinates).  Pointers are device memory owned
 * by the caller and must stay valid while the batch exists; NULL disables the
 * matching output (A: no forward; dA / dcoords / dcoef: no adjoint part). */
typedef struct fem_batch_item {
  fem_mesh mesh;
  int32_t form;
  int32_t reserved; /* must be 0 */
  const float* coef; /* [n_elem] or NULL */
  float* A;          /* [n_elem][rows][cols] (fem_form_shape) */
  const float* dA;   /* [n_elem][rows][cols] */
  float* dcoords;    /* [n_vert][dim] (deterministic reduction) */
  float* dcoef;      /* [n_elem] */
} fem_batch_item;

typedef struct fem_batch fem_batch; /* opaque; host object */

/* Device workspace bytes of a batch (descriptor table, counters, the
 * per-mesh reduction records). */
FEM_API fem_status fem_batch_workspace_size(const fem_batch_item* items, int32_t n_items, size_t* bytes);

/* Creates a batch over caller-owned device workspace `ws` (256-byte aligned):
 * builds every mesh's reduction records (once) and uploads the descriptor
 * table, asynchronously on `stream`.  *out receives a host object to be
 * released with fem_batch_destroy. */
FEM_API fem_status fem_batch_create(const fem_batch_item* items, int32_t n_items, void* ws, size_t ws_bytes,
                                    fem_batch** out, void* stream);

/* Autotuner: times every mode x grid (CTAs per SM, capped per kernel at its
 * occupancy) x work-chunk size with CUDA events on `stream` (synchronizing
 * it) and keeps the fastest for later fem_batch_run calls.  The tuning
 * launches write the batch's outputs. */
FEM_API fem_status fem_batch_tune(fem_batch* batch, int32_t phases, void* stream);

/* The launch configuration in use (the tuner's choice, or the default:
 * FEM_BATCH_PHASED, or FEM_BATCH_PER_ITEM_CONCURRENT for a batch holding a
 * coupling block; full occupancy, chunk 1).  NULL outputs are skipped. */
FEM_API fem_status fem_batch_config(const fem_batch* batch, int32_t* ctas_per_sm, int32_t* chunk, int32_t* mode);

/* Sets the launch configuration: ctas_per_sm 1..32 (capped at each kernel's
 * occupancy), chunk 1..64, mode FEM_BATCH_*; FEM_ERR_ARG otherwise. */
FEM_API fem_status fem_batch_set_config(fem_batch* batch, int32_t ctas_per_sm, int32_t chunk, int32_t mode);

/* The persistent launch(es) over every mesh of the batch for `phases`
 * (FEM_PHASE_FWD | FEM_PHASE_BWD), preceded by one memset of the counters.
 * Asynchronous; graph-capturable. */
FEM_API fem_status fem_batch_run(fem_batch* batch, int32_t phases, void* stream);

/* Device error word of the last fem_batch_run (FEM_DEVERR_* bits), copied
 * synchronously to *err_host. */
FEM_API fem_status fem_batch_errors(const fem_batch* batch, int32_t* err_host, void* stream);

/* Failure injection for tests of the bounded waits (FEM_BATCH_SINGLE and the
 * grouped modes; the per-item modes have no wait).  Host only: it rewrites the
 * uploaded descriptor of `item` so that its reduction items wait for
 * n_tiles + extra_tiles counted tiles instead of n_tiles (the tiles actually
 * run are unchanged), and bounds every wait of later fem_batch_run calls at
 * spin_limit polls of about 64 ns (0 = the default, about 2^24 polls).  With
 * extra_tiles > 0 those waits give up: the run completes, the item's dcoords
 * is not written and fem_batch_errors reports FEM_DEVERR_TIMEOUT.
 * extra_tiles = 0 and spin_limit = 0 restore normal runs.  Synchronizes
 * `stream`. */
FEM_API fem_status fem_batch_inject_wait(fem_batch* batch, int32_t item, int64_t extra_tiles, uint32_t spin_limit,
                                         void* stream);

/* Releases the host object (the caller frees the workspace). */
FEM_API void fem_batch_destroy(fem_batch* batch);

/* ------------------------------------------------------------------ assembly
 * Global sparse assembly, the step after the element integration:
 * A = sum_e P_e^T A_e P_e over the vertex graph of the mesh.  The scalar P1
 * forms (FEM_LAPLACE_P1, FEM_LAPLACE_P1_W1) give CSR; FEM_ELASTIC_P1 gives BSR
 * with d x d blocks over the same pattern (node-major unknowns v*d + c; block
 * (c, c') of entry (v, w) sums A_e[(c,i),(c',j)] over the elements with
 * conn[e][i] = v, conn[e][j] = w, local unknown (c, i) being row c*(d+1) + i
 * of A_e).  The P2 forms (FEM_LAPLACE_P2, FEM_LAPLACE_P2_W1,
 * FEM_LAPLACE_P2_ISO) give CSR over the P2 unknowns: the vertices 0 .. V-1,
 * then one unknown per edge, V + k for the k-th distinct edge in increasing
 * (lower vertex, higher vertex) order (fem_assembly_unknowns returns their
 * count and each element's unknowns in the local P2 order).  Every entry is a
 * sum in a fixed order, so values are bitwise reproducible: for the scalar P1
 * forms, per 32-element tile the tile's contributions in element order, then
 * those tile sums in tile order; for the blocks and the P2 forms, all
 * contributions in element order. */

/* Device workspace bytes of the assembly maps of this mesh (depends on the
 * connectivity only; the capacity of the column array is every entry distinct). */
FEM_API fem_status fem_assembly_workspace_size(const fem_mesh* mesh, int32_t form, size_t* bytes);

/* Builds the row pattern (row_ptr [n_rows+1], col_idx [nnz], columns increasing)
 * and the assembly maps into `ws` (device, caller owned, 256-byte aligned),
 * once per connectivity, on `stream`, which it synchronizes.  *nnz receives the
 * number of nonzero entries (blocks); *n_records the number of tile records of
 * the scalar forms (the distinct entries of every 32-element tile; 0 for
 * blocks).  Either output may be NULL.  A connectivity entry outside
 * [0, n_vert) is FEM_ERR_ARG; an element that repeats a vertex, or a vertex
 * with more than 128 elements or 255 neighbours (P2: an unknown with more than
 * 255 neighbours or more than 51 incident elements on tets, 85 on triangles),
 * FEM_ERR_UNSUPPORTED.  The P2 forms' workspace also holds the vertex graph's
 * pattern, the edge numbers and the element unknowns. */
FEM_API fem_status fem_assembly_build(const fem_mesh* mesh, int32_t form, void* ws, size_t ws_bytes, int64_t* nnz,
                                      int64_t* n_records, void* stream);

/* Device pointers to the pattern inside a built workspace (row_ptr [n_rows+1],
 * col_idx [nnz], n_rows from fem_assembly_unknowns); either output may be NULL. */
FEM_API fem_status fem_assembly_pattern(const fem_mesh* mesh, int32_t form, const void* ws, size_t ws_bytes,
                                        const int32_t** row_ptr, const int32_t** col_idx);

/* The unknowns of a built assembly: *n_rows = the block rows of the matrix
 * (n_vert for the P1 forms; n_vert + the edge count for the P2 forms, read
 * from the device: this synchronizes it) and *dofs = a device pointer to each
 * element's unknowns [n_elem][nodes] in the local order of its basis (mesh->conn
 * for the P1 forms).  Either output may be NULL. */
FEM_API fem_status fem_assembly_unknowns(const fem_mesh* mesh, int32_t form, const void* ws, size_t ws_bytes,
                                         int64_t* n_rows, const int32_t** dofs);

/* Assembles the FP32 element matrices A (device [n_elem][n][n], as written by
 * fem_integrate_fwd) into values (device FP32 [nnz][b][b], b = 1 or d; overwritten),
 * asynchronously on `stream`. */
FEM_API fem_status fem_assemble(const fem_mesh* mesh, int32_t form, const float* A, const void* ws, size_t ws_bytes,
                                float* values, void* stream);

/* Bytes of the scratch array built into the library for
 * fem_integrate_bwd_noalloc (32 MiB: the deterministic adjoint of a tet mesh
 * of up to roughly 300,000 elements). */
#define FEM_NOALLOC_SCRATCH_BYTES (32u << 20)

/* The adjoint of fem_integrate_bwd (deterministic reduction) for callers that
 * cannot allocate device memory -- for example a host application that
 * reserves all GPU memory at start-up and forbids allocation later, or a
 * callback that only receives raw pointers from a framework owning the
 * allocator.  The paper has no counterpart; it is an interface convenience.
 *   Arguments, outputs and results are those of fem_integrate_bwd with
 *   FEM_REDUCE_DETERMINISTIC; the caller passes no workspace.  Instead the
 *   incidence records are rebuilt on every call inside a scratch array of
 *   FEM_NOALLOC_SCRATCH_BYTES that the library holds in device memory of every
 *   GPU that loads it, until the process exits.  Nothing is allocated.
 *   - A mesh whose workspace (fem_bwd_workspace_size) exceeds that size is
 *     rejected with FEM_ERR_UNSUPPORTED before anything is launched.
 *   - options->reduce other than FEM_REDUCE_DETERMINISTIC: FEM_ERR_UNSUPPORTED.
 *   - The first call on a device looks up the array's device address there
 *     (cudaGetSymbolAddress) and keeps it for the life of the process; make
 *     that first call before any stream capture.  cudaDeviceReset (or any
 *     reset of the device's primary context) invalidates the kept address:
 *     once this entry point has run on a device, do not reset that device.
 *   - Every refusal (bad argument, unsupported combination, a mesh too large
 *     for the array) is returned before the array is touched or anything is
 *     launched.
 *   - All calls share the one array: calls whose GPU work may overlap (other
 *     streams, other host threads on the same device) race and corrupt each
 *     other's results.  Serialize them on one stream. */
FEM_API fem_status fem_integrate_bwd_noalloc(const fem_mesh* mesh, int32_t form, const float* coef,
                                             const float* dA, float* dcoords, float* dcoef,
                                             const fem_options* options, void* stream);

/* ---- Launch-shape autotuner of the single-mesh kernels -------------------
 * The paper tunes its kernel's block shape (elements per block and elements
 * computed concurrently) by measurement on its workload (Sec. 5).  These
 * calls do the same for one mesh and form on this GPU: they time the call
 * (CUDA events on `stream`, 2 untimed and 5 timed launches per candidate) for
 * every candidate (warps_per_cta, ctas_per_sm) pair the kernel's compiled
 * shape admits, and write the fastest pair into options->warps_per_cta and
 * options->ctas_per_sm; *best_ms (may be NULL) receives its time per call.
 * The other fields of *options are the options every candidate runs with.
 * The default pair (0, 0) is always a candidate, so the result is never
 * slower than the default as measured.  Candidates: warps_per_cta in
 * {0, 1, 2, 4, 8} times ctas_per_sm in {0, 2, 4, 8, 16, 24, 32}; a kernel
 * compiled for fewer warps per CTA (one, for the compensated 3D P1
 * Laplacian) runs the largest count it admits.  The candidates run on the
 * caller's buffers: A (fem_tune_fwd) and dcoords / dcoef (fem_tune_bwd) are
 * overwritten, with the values of one call.  Synchronizes `stream`.
 * fem_tune_fwd: arguments of fem_integrate_fwd_save (det may be NULL: then
 *   fem_integrate_fwd is timed).
 * fem_tune_bwd: arguments of fem_integrate_bwd_saved (det may be NULL: then
 *   fem_integrate_bwd is timed); the workspace must be built. */
FEM_API fem_status fem_tune_fwd(const fem_mesh* mesh, int32_t form, const float* coef, void* A, int32_t out_dtype,
                                float* det, fem_options* options, float* best_ms, void* stream);
FEM_API fem_status fem_tune_bwd(const fem_mesh* mesh, int32_t form, const float* coef, const float* dA,
                                const float* det, float* dcoords, float* dcoef, void* ws, size_t ws_bytes,
                                fem_options* options, float* best_ms, void* stream);

/* ---- End-to-end step from host memory ----------------------------------
 * One mesh whose inputs and outputs live in page-locked host memory: a step
 * copies coords, conn and the upstream dA to the device, integrates A = G:K
 * (Eq. 6) saving det J, runs the deterministic adjoint taking it, and copies A
 * and dcoords back.  The elements go in slices of `chunk` elements (a multiple
 * of 32): one copy stream sends the coordinates, then each slice's
 * connectivity and dA; the forward of a slice starts when its connectivity
 * has arrived, its adjoint element pass when its dA has (on steps that reuse
 * the incidence); a second copy stream returns each slice's A once written,
 * and dcoords after the reduction.  Results are bitwise those of
 * fem_integrate_fwd_save + fem_integrate_bwd_saved on the device.
 *
 * fem_host_step_create: form FEM_LAPLACE_P1, FEM_LAPLACE_P2 or
 *   FEM_ELASTIC_P1, dim 2 or 3, n_vert/n_elem > 0, chunk > 0 (rounded up to a
 *   multiple of 32; 0 = 1 << 20).  Allocates the device arrays (coords, conn,
 *   dA, A, det, dcoords and the adjoint workspace) on the current device and
 *   two copy streams; *step owns them.  FEM_ERR_CUDA if an allocation fails.
 * fem_host_step_run: coords [n_vert][dim] FP32, conn [n_elem][dim+1] int32,
 *   dA [n_elem][n][n] FP32 (read); A [n_elem][n][n] FP32 and dcoords
 *   [n_vert][dim] FP32 (written): page-locked host memory (cudaHostAlloc or
 *   cudaHostRegister; FEM_ERR_ARG otherwise), on the step's device.  rebuild
 *   != 0 copies conn in and rebuilds the incidence from it (a new
 *   connectivity); the first run always does.  A run with rebuild == 0 keeps
 *   the connectivity and the incidence of the last building run on the
 *   device and does not read conn: per step, only coords and dA go in.
 *   Asynchronous on `stream`: the step is done, and the host
 *   buffers may be reused, when the work queued on `stream` so far is.  The
 *   next run on the same step must be queued on the same stream (it reuses the
 *   device arrays).
 * fem_host_step_destroy: waits for the step's copy streams and frees what
 *   create allocated; call it after `stream` has finished the last run. */
typedef struct fem_host_step fem_host_step; /* opaque; host object */

FEM_API fem_status fem_host_step_create(int32_t form, int32_t dim, int64_t n_vert, int64_t n_elem, int64_t chunk,
                                        fem_host_step** step);
FEM_API fem_status fem_host_step_run(fem_host_step* step, const float* coords, const int32_t* conn,
                                     const float* dA, float* A, float* dcoords, int32_t rebuild, void* stream);
FEM_API void fem_host_step_destroy(fem_host_step* step);

/* ------------------------------------------------------------------ mesh order
 * A locality numbering for unstructured meshes (an addition beside the
 * method).  The forward's coordinate gather and the adjoint's tile records
 * (elements of one 32-element tile sharing vertices) profit from elements and
 * vertices numbered along a space-filling curve; a mesh in random order loses
 * both.  Vertices are ordered by the Z-order (Morton) code of their position,
 * elements by the code of their centroid, quantised to a grid of 2^7 cells per
 * axis (tetrahedra) or 2^10 (triangles) over the mesh's bounding box; equal
 * codes keep the old order, so the result is deterministic.  An element with a
 * vertex number out of range takes code 0.
 *
 * fem_mesh_order_workspace_size: bytes of device workspace (256-byte aligned)
 *   for fem_mesh_order and fem_mesh_renumber; FP32 coordinates, dim 2 or 3.
 * fem_mesh_order: elem_perm [n_elem] and vert_perm [n_vert] (device int32,
 *   written): new position -> old number.  Synchronizes `stream` once per
 *   order to check that no grid cell holds more than 1024 vertices or
 *   elements (FEM_ERR_UNSUPPORTED otherwise: a mesh packed into few cells).
 * fem_mesh_renumber: coords_out [n_vert][dim] = coords[vert_perm] and
 *   conn_out [n_elem][dim+1] = the new numbers of conn[elem_perm] (device,
 *   written; out-of-range vertex numbers are copied unchanged); the
 *   workspace holds the inverse vertex order.  Every element keeps its
 *   vertices in their local order, so its element matrix is unchanged. */
FEM_API fem_status fem_mesh_order_workspace_size(const fem_mesh* mesh, size_t* bytes);
FEM_API fem_status fem_mesh_order(const fem_mesh* mesh, void* ws, size_t ws_bytes, int32_t* elem_perm,
                                  int32_t* vert_perm, void* stream);
FEM_API fem_status fem_mesh_renumber(const fem_mesh* mesh, const int32_t* elem_perm, const int32_t* vert_perm,
                                     void* ws, size_t ws_bytes, float* coords_out, int32_t* conn_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* FEM_GB300_H */
