// fem_internal.h -- host-side plumbing shared by the translation units of
// libfem_gb300 (launch descriptors, device queries).  Not part of the ABI.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

namespace fem {

// Everything one forward launch needs, already validated by the ABI layer.
struct FwdLaunch {
  int dim, form, jac, coord_f64, out_f64;
  const int32_t* conn;
  const void* coords;
  const float* coef;
  void* A;
  int64_t n_elem, n_vert;
  int32_t* dev_err;
  int warps, ctas_per_sm;
  cudaStream_t stream;
  float* det_out = nullptr;  // det J saved for the adjoint (fem_fwd_kernel only)
};

struct GeoLaunch {
  int dim, jac, coord_f64;
  const int32_t* conn;
  const void* coords;
  const float* coef;
  double* detJ;
  float* G;
  int64_t n_elem, n_vert;
  int32_t* dev_err;
  cudaStream_t stream;
};

// Elements per CTA tile (4 warps x 32) of the persistent and batched kernels.
constexpr int kTileElems = 128;
// Elements per record tile of the deterministic reduction: one warp's 32
// elements, so a warp forms its records without any CTA-wide barrier.
constexpr int kRecTile = 32;
// Positions of a tet tile's slot stage: the 128 slots with each record's run
// aligned for conflict-free reads (see tile_records_kernel).
constexpr int kStageCap3 = 256;

// Adjoint element pass (FP32 coordinates).
struct BwdLaunch {
  int dim, form, jac, atomic;
  const int32_t* conn;
  const float* coords;
  const float* coef;
  const float* dA;
  float* dcoef;    // may be null
  float* dcoords;  // atomic: accumulated with red.add (pre-zeroed)
  // deterministic: tile records (null when only dcoef is wanted)
  const int32_t* tile_rec;
  const uint32_t* rank;
  const uint16_t* rec_span;
  const int32_t* rec_dest;
  float* records;
  int64_t n_elem, n_vert;
  int32_t* dev_err;
  int warps, ctas_per_sm;  // warps <= 0: the default
  cudaStream_t stream;
  const float* det_in = nullptr;  // det J saved by the forward: the JAC_SAVED element pass
};

// Workspace of the deterministic adjoint (see fem_incidence.cu):
// [tile_rec T+1][rank T*32 u32][rec_span R u16][rec_dest R][rec_vertex R][voff V+1]
// [vrec R][cursor][scan partials][mode][records R*d]   with T = ceil(E/32) record
// tiles and R <= E*(d+1) records; records are stored vertex-major (record r at
// rec_dest[r]), so the records of vertex v are records[voff[v], voff[v+1]).
struct BwdWorkspace {
  int32_t* tile_rec;
  uint32_t* rank;  // per element: byte k = stage position of its local vertex k (runs in (vertex, slot) order)
  uint16_t* rec_span;  // per record: start | length << 8 of its run in the tile's slot stage
  int32_t* rec_dest;  // per record: its position in the vertex-major record array
  int32_t* rec_vertex;
  int32_t* voff;
  int32_t* vrec;
  int32_t* cursor;
  int32_t* partials;
  int32_t* mode;  // record layout chosen by the build: kRecVertexMajor or kRecTileOrder (one word)
  float* records;   // [R][ncomp]
  int64_t n_tiles;
  int ncomp;        // components of a record: d, or d + 1 for the P1-coefficient forms
  size_t bytes;
};
// Record layouts.  Vertex-major: record r is row rec_dest[r], the rows of
// vertex v are [voff[v], voff[v+1]) and the reduction reads them in place.
// Tile order (rec_dest[r] = r): the element pass writes each tile's records
// contiguously and the reduction gathers the records of vertex v through
// vrec[voff[v] .. voff[v+1]).  Both sum a vertex's records in increasing
// record order, so dcoords has the same bits either way.
constexpr int32_t kRecVertexMajor = 0;
constexpr int32_t kRecTileOrder = 1;
// ncomp: components of a record (0 = dim; dim + 1 for the P1-coefficient
// forms, whose records also carry the coefficient gradient).  Everything but
// the size of the records array is independent of it.
size_t bwd_workspace_layout(int dim, int64_t n_elem, int64_t n_vert, bool with_scratch, void* base,
                            BwdWorkspace* ws, int ncomp = 0);

cudaError_t launch_fwd_d2(const FwdLaunch& L);
cudaError_t launch_fwd_d3_lap(const FwdLaunch& L);
cudaError_t launch_fwd_d3_ela(const FwdLaunch& L);
cudaError_t launch_fwd_tc(const FwdLaunch& L);  // split-bf16 tensor-core contraction
cudaError_t launch_fwd_w1(const FwdLaunch& L);  // Laplacian with a P1 (vertex) coefficient
cudaError_t launch_fwd_iso(const FwdLaunch& L, const float* mid);  // non-affine (quadratic-geometry) elements
// The P2 non-affine forward with the tensor-core contraction (fem_tc_iso.cu).
cudaError_t launch_fwd_iso_tc(const FwdLaunch& L, const float* mid);
cudaError_t launch_geometry(const GeoLaunch& L);
// The coupling blocks int w q div v (fem_coupling.cu): forward and adjoint element pass.
cudaError_t launch_div_fwd(const FwdLaunch& L);
cudaError_t launch_div_bwd(const BwdLaunch& L);
cudaError_t launch_bwd_elem(const BwdLaunch& L);
// Adjoint element pass of the non-affine forms (LAPLACE_P1_ISO / LAPLACE_P2_ISO):
// mid [E][d(d+1)/2][d] the edge nodes, dmid the same shape (may be null).
cudaError_t launch_bwd_iso(const BwdLaunch& L, const float* mid, float* dmid);
// The same for LAPLACE_P2_ISO on tetrahedra, deterministic or deferred, with
// the contraction's adjoint on the tensor cores (fem_bwd_iso_tc.cu).
cudaError_t launch_bwd_iso_tc(const BwdLaunch& L, const float* mid, float* dmid);
cudaError_t launch_incidence_build(int dim, const int32_t* conn, int64_t n_elem, int64_t n_vert,
                                   const BwdWorkspace& ws, cudaStream_t stream);
cudaError_t launch_zero_f32(float* p, int64_t n, cudaStream_t stream);
// off[0..n_seg] and list[0..n_keys) = the CSR of the indices s with keys[s] in
// [0, n_seg), each segment sorted increasingly (keys out of range are left
// out).  cursor: n_seg + 1 ints of scratch; partials: scan_partials_count(n_seg).
cudaError_t launch_key_csr(const int32_t* keys, int64_t n_keys, int64_t n_seg, int32_t* off, int32_t* list,
                           int32_t* cursor, int32_t* partials, cudaStream_t stream);
size_t scan_partials_count(int64_t n);
// offsets[0..n] = exclusive prefix sums of cnt[0..n) (offsets[n] = total).
cudaError_t launch_exclusive_scan(const int32_t* cnt, int64_t n, int32_t* partials, int32_t* offsets,
                                  cudaStream_t stream);
// dcoords [n_vert][dim] (may be null) and, for records of dim + 1 components,
// dcoef [n_vert] (may be null) from the records of the workspace.
cudaError_t launch_vertex_reduce(int dim, const BwdWorkspace& ws, int64_t n_vert, float* dcoords,
                                 cudaStream_t stream, float* dcoef = nullptr);

// Records the reason reported by fem_last_error() for the calling thread.
void set_last_error(const char* fmt, ...);

}  // namespace fem

struct fem_mesh;
struct fem_options;

namespace fem {

// Every check of fem_integrate_bwd that needs no workspace (mesh, form,
// options, dA and the deferred-mode dcoords), with the same status and
// fem_last_error() message; 0 (FEM_OK) when the call may proceed.
int32_t bwd_preflight(const fem_mesh* mesh, int32_t form, const fem_options* options, const float* dA,
                      const float* dcoords);
// Whether fem_integrate_bwd reduces through the workspace for these outputs.
bool bwd_needs_workspace(int32_t form, bool has_dcoords, bool has_dcoef, int32_t reduce);
// Element pass of the deferred deterministic adjoint, with det J saved by the
// forward, over elements [e0, e1) of `mesh` (e0 a multiple of 32): writes the
// records of those elements' tiles into the workspace built for the whole mesh.
// Affine FP32 forms (LAPLACE_P1, LAPLACE_P2, ELASTIC_P1) without coefficient;
// the caller has validated mesh and form.  Returns a fem_status.
int32_t bwd_element_range(const fem_mesh* mesh, int32_t form, const float* dA, const float* det, void* ws,
                          size_t ws_bytes, int64_t e0, int64_t e1, cudaStream_t stream);

// Device facts of the current device (cached per device).
int device_sm_count();
size_t device_smem_optin();
// Largest warp count <= want whose per-warp stage (bytes_per_warp) fits the opt-in shared memory.
int clamp_warps(int want, size_t bytes_per_warp);
// Grid of a warp-tile pipeline kernel: one wave of resident CTAs (occupancy x SMs), or
// ctas_per_sm x SMs when given, never more CTAs than the tiles need.
unsigned pipeline_grid(const void* kernel, int warps, size_t smem, int64_t n_elem, int ctas_per_sm);
// Raises the dynamic shared memory limit of a kernel when it needs more than 48 KB.
cudaError_t ensure_smem(const void* kernel, size_t bytes);

}  // namespace fem
