// fem_api.cu -- the C ABI of libfem_gb300 (declared in include/fem.h):
// argument validation, defaults, dispatch to the kernels, status codes.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "../../include/fem.h"
#include "fem_core.cuh"
#include "fem_internal.h"

namespace {

thread_local char g_msg[512] = "";

fem_status fail(fem_status s, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
  va_end(ap);
  return s;
}

fem_status cuda_fail(cudaError_t e, const char* what) {
  return fail(FEM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

fem_status ok() {
  g_msg[0] = '\0';
  return FEM_OK;
}

const fem_options kDefaults = {0, 0, 0, 0, 0, 0, nullptr};

fem_status check_mesh(const fem_mesh* m) {
  if (!m) return fail(FEM_ERR_ARG, "mesh is NULL");
  if (m->dim != 2 && m->dim != 3) return fail(FEM_ERR_ARG, "mesh->dim must be 2 or 3 (got %d)", m->dim);
  if (m->coord_dtype != FEM_F32 && m->coord_dtype != FEM_F64)
    return fail(FEM_ERR_ARG, "mesh->coord_dtype must be FEM_F32 or FEM_F64");
  if (m->n_elem < 0 || m->n_vert < 0) return fail(FEM_ERR_ARG, "negative mesh size");
  if (m->n_elem > 0 && (!m->conn || !m->coords))
    return fail(FEM_ERR_ARG, "mesh->conn and mesh->coords must be non-NULL when n_elem > 0");
  if (m->n_vert > INT32_MAX) return fail(FEM_ERR_UNSUPPORTED, "n_vert exceeds the int32 index range");
  return FEM_OK;
}

fem_status check_options(const fem_options* o) {
  if (o->jac < FEM_JAC_AUTO || o->jac > FEM_JAC_F32) return fail(FEM_ERR_ARG, "options->jac out of range");
  if (o->contract < FEM_CONTRACT_F32 || o->contract > FEM_CONTRACT_BF16X3)
    return fail(FEM_ERR_ARG, "options->contract out of range");
  if (o->reduce < FEM_REDUCE_DETERMINISTIC || o->reduce > FEM_REDUCE_DEFERRED)
    return fail(FEM_ERR_ARG, "options->reduce out of range");
  if (o->warps_per_cta < 0 || o->warps_per_cta > 16) return fail(FEM_ERR_ARG, "options->warps_per_cta must be 0..16");
  if (o->ctas_per_sm < 0 || o->ctas_per_sm > 64) return fail(FEM_ERR_ARG, "options->ctas_per_sm must be 0..64");
  if (o->reserved != 0) return fail(FEM_ERR_ARG, "options->reserved must be 0");
  return FEM_OK;
}

bool coupling(int form) { return form == FEM_DIV_P1P1 || form == FEM_DIV_P2P1; }

int form_rows(int form, int dim) {
  if (coupling(form)) return dim + 1;
  const bool p2 = form == FEM_LAPLACE_P2 || form == FEM_LAPLACE_P2_W1 || form == FEM_LAPLACE_P2_ISO;
  const int nb = p2 ? (dim + 1) * (dim + 2) / 2 : dim + 1;
  return nb * (form == FEM_ELASTIC_P1 ? dim : 1);
}

int form_cols(int form, int dim) {
  if (!coupling(form)) return form_rows(form, dim);
  return dim * (form == FEM_DIV_P2P1 ? (dim + 1) * (dim + 2) / 2 : dim + 1);
}

bool valid_form(int form) { return form >= FEM_LAPLACE_P1 && form <= FEM_DIV_P2P1; }
bool coef_p1(int form) { return form == FEM_LAPLACE_P1_W1 || form == FEM_LAPLACE_P2_W1; }
bool non_affine(int form) { return form == FEM_LAPLACE_P1_ISO || form == FEM_LAPLACE_P2_ISO; }

int resolve_jac(int jac, bool coord_f64, bool out_f64) {
  if (jac == FEM_JAC_AUTO) return (coord_f64 || out_f64) ? fem::JAC_F64 : fem::JAC_COMP;
  if (jac == FEM_JAC_F64) return fem::JAC_F64;
  if (jac == FEM_JAC_COMP_F32) return fem::JAC_COMP;
  return fem::JAC_F32;
}

// Components of an adjoint record: the vertex gradient, plus the gradient of
// the coefficient's vertex values for the P1-coefficient forms.
int record_components(int form, int dim) { return dim + (coef_p1(form) ? 1 : 0); }

// Whether an adjoint call reduces through the workspace's records: the
// deterministic and deferred reductions of dcoords, and of dcoef when it holds
// vertex values (P1-coefficient forms).
bool bwd_uses_records(int form, bool has_dcoords, bool has_dcoef, int reduce) {
  return reduce != FEM_REDUCE_ATOMIC && (has_dcoords || (coef_p1(form) && has_dcoef));
}

// Every check of an adjoint call that needs no workspace: the mesh, the form,
// the options and the pointers.  A refused call launches nothing.
fem_status bwd_args(const fem_mesh* mesh, int32_t form, const fem_options* o, const float* dA,
                    const float* dcoords) {
  fem_status s = check_mesh(mesh);
  if (s != FEM_OK) return s;
  if (!valid_form(form)) return fail(FEM_ERR_ARG, "form out of range");
  if (non_affine(form))
    return fail(FEM_ERR_UNSUPPORTED, "the non-affine forms take their adjoint through fem_integrate_bwd_iso");
  if ((s = check_options(o)) != FEM_OK) return s;
  if (coef_p1(form) && ((o->jac != FEM_JAC_AUTO && o->jac != FEM_JAC_COMP_F32) || o->reduce == FEM_REDUCE_DEFERRED))
    return fail(FEM_ERR_UNSUPPORTED,
                "the P1-coefficient adjoint takes the compensated Jacobian and the deterministic or atomic reduction");
  if (mesh->coord_dtype != FEM_F32) return fail(FEM_ERR_UNSUPPORTED, "the adjoint takes FP32 coordinates");
  if (o->contract != FEM_CONTRACT_F32) return fail(FEM_ERR_UNSUPPORTED, "the adjoint contracts in FP32");
  if (mesh->n_elem * (mesh->dim + 1) > INT32_MAX)
    return fail(FEM_ERR_UNSUPPORTED, "n_elem * (dim + 1) exceeds the int32 slot range");
  if (o->reduce == FEM_REDUCE_DEFERRED && !dcoords)
    return fail(FEM_ERR_ARG, "FEM_REDUCE_DEFERRED needs dcoords (written by fem_adjoint_reduce)");
  if (mesh->n_elem > 0 && !dA) return fail(FEM_ERR_ARG, "dA is NULL");
  return FEM_OK;
}

// K_host[g = mu * D + c][i][c' * NBV + j] = DEN K^{ij}_mu delta_{c c'}: the
// coupling block as sum_g G_g K_g with G_{mu c} = w |J| J^{-1}_{mu c}.
template <int D, int VDEG>
void copy_div_ref(int32_t* K) {
  using T = fem::DivTraits<D, VDEG>;
  constexpr auto R = fem::make_div_ref<D, VDEG>();
  for (int mu = 0; mu < D; ++mu)
    for (int c = 0; c < D; ++c)
      for (int i = 0; i < T::NQ; ++i)
        for (int cc = 0; cc < D; ++cc)
          for (int j = 0; j < T::NBV; ++j)
            K[((mu * D + c) * T::NQ + i) * T::NCOL + cc * T::NBV + j] = cc == c ? R.v[mu][i][j] : 0;
}

template <int D, int FORM>
void copy_ref(int32_t* K) {
  using FT = fem::FormTraits<D, FORM>;
  constexpr auto R = fem::make_ref_tensor<D, FORM>();
  for (int g = 0; g < FT::NG; ++g)
    for (int i = 0; i < FT::N; ++i)
      for (int j = 0; j < FT::N; ++j) K[(g * FT::N + i) * FT::N + j] = R.v[g][i][j];
}

}  // namespace

namespace fem {
int32_t bwd_preflight(const fem_mesh* mesh, int32_t form, const fem_options* options, const float* dA,
                      const float* dcoords) {
  return bwd_args(mesh, form, options ? options : &kDefaults, dA, dcoords);
}

bool bwd_needs_workspace(int32_t form, bool has_dcoords, bool has_dcoef, int32_t reduce) {
  return bwd_uses_records(form, has_dcoords, has_dcoef, reduce);
}

int32_t bwd_element_range(const fem_mesh* mesh, int32_t form, const float* dA, const float* det, void* ws,
                          size_t ws_bytes, int64_t e0, int64_t e1, cudaStream_t stream) {
  if (e0 < 0 || e1 > mesh->n_elem || e0 > e1 || e0 % kRecTile != 0)
    return fail(FEM_ERR_ARG, "element range [%lld, %lld) must start on a tile of %d elements",
                static_cast<long long>(e0), static_cast<long long>(e1), kRecTile);
  fem::BwdWorkspace W{};
  const size_t need = fem::bwd_workspace_layout(mesh->dim, mesh->n_elem, mesh->n_vert, true, ws, &W,
                                                record_components(form, mesh->dim));
  if (!ws || ws_bytes < need) return fail(FEM_ERR_WORKSPACE, "workspace needs %zu bytes (got %zu)", need, ws_bytes);
  if (e1 == e0) return ok();
  const int64_t rows = form_rows(form, mesh->dim), cols = form_cols(form, mesh->dim);
  fem::BwdLaunch L{};
  L.dim = mesh->dim;
  L.form = form;
  L.jac = resolve_jac(FEM_JAC_AUTO, false, false);
  L.atomic = 0;
  // the element pass of elements [e0, e1) is the whole-mesh pass's restricted to
  // their tiles: per-element and per-tile arrays start at the range, the records
  // (indexed by the tile offsets) stay the whole mesh's
  L.conn = mesh->conn + e0 * (mesh->dim + 1);
  L.coords = static_cast<const float*>(mesh->coords);
  L.coef = nullptr;
  L.dA = dA + e0 * rows * cols;
  L.dcoef = nullptr;
  L.tile_rec = W.tile_rec + e0 / kRecTile;
  L.rank = W.rank + e0;
  L.rec_span = W.rec_span;
  L.rec_dest = W.rec_dest;
  L.records = W.records;
  L.dcoords = nullptr;
  L.n_elem = e1 - e0;
  L.n_vert = mesh->n_vert;
  L.dev_err = nullptr;
  L.warps = 0;
  L.ctas_per_sm = 0;
  L.stream = stream;
  L.det_in = det + e0;
  const cudaError_t e = fem::launch_bwd_elem(L);
  if (e != cudaSuccess) return cuda_fail(e, "adjoint element pass launch");
  return ok();
}

void set_last_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
  va_end(ap);
}
}  // namespace fem

extern "C" {

const char* fem_version(void) { return "fem_gb300 0.1 (sm_103a)"; }

const char* fem_status_string(fem_status s) {
  switch (s) {
    case FEM_OK: return "FEM_OK";
    case FEM_ERR_ARG: return "FEM_ERR_ARG";
    case FEM_ERR_UNSUPPORTED: return "FEM_ERR_UNSUPPORTED";
    case FEM_ERR_WORKSPACE: return "FEM_ERR_WORKSPACE";
    case FEM_ERR_CUDA: return "FEM_ERR_CUDA";
  }
  return "FEM_ERR_UNKNOWN";
}

const char* fem_last_error(void) { return g_msg; }

fem_status fem_form_info(int32_t form, int32_t dim, int32_t* n, int32_t* n_geom, int32_t* den) {
  if (!valid_form(form)) return fail(FEM_ERR_ARG, "form out of range");
  if (dim != 2 && dim != 3) return fail(FEM_ERR_ARG, "dim must be 2 or 3");
  const int np = form == FEM_ELASTIC_P1 ? dim * dim : non_affine(form) ? (dim + 1) * dim : dim;
  if (n) *n = form_rows(form, dim);
  if (n_geom) *n_geom = coupling(form) ? dim * dim : np * (np + 1) / 2 * (coef_p1(form) ? dim + 1 : 1);
  if (den)
    *den = non_affine(form) ? (dim == 2 ? 720 : 5040)
           : coef_p1(form)  ? (dim == 2 ? 120 : 720)
                            : (dim == 2 ? 24 : 120) * (form == FEM_ELASTIC_P1 ? 2 : 1);  // coupling: (d+2)!
  return ok();
}

fem_status fem_form_shape(int32_t form, int32_t dim, int32_t* rows, int32_t* cols) {
  fem_status s = fem_form_info(form, dim, nullptr, nullptr, nullptr);
  if (s != FEM_OK) return s;
  if (rows) *rows = form_rows(form, dim);
  if (cols) *cols = form_cols(form, dim);
  return ok();
}

fem_status fem_reference_tensor(int32_t form, int32_t dim, int32_t* K, size_t cap) {
  int32_t n = 0, ng = 0;
  fem_status s = fem_form_info(form, dim, &n, &ng, nullptr);
  if (s != FEM_OK) return s;
  if (!K) return fail(FEM_ERR_ARG, "K is NULL");
  const int nc = form_cols(form, dim);
  if (cap < size_t(ng) * n * nc) return fail(FEM_ERR_ARG, "K capacity %zu < %d", cap, ng * n * nc);
  if (coupling(form)) {
    if (dim == 2)
      form == FEM_DIV_P1P1 ? copy_div_ref<2, 1>(K) : copy_div_ref<2, 2>(K);
    else
      form == FEM_DIV_P1P1 ? copy_div_ref<3, 1>(K) : copy_div_ref<3, 2>(K);
    return ok();
  }
  if (dim == 2) {
    if (form == FEM_LAPLACE_P1) copy_ref<2, fem::LAPLACE_P1>(K);
    if (form == FEM_LAPLACE_P2) copy_ref<2, fem::LAPLACE_P2>(K);
    if (form == FEM_ELASTIC_P1) copy_ref<2, fem::ELASTIC_P1>(K);
    if (form == FEM_LAPLACE_P1_W1) copy_ref<2, fem::LAPLACE_P1_W1>(K);
    if (form == FEM_LAPLACE_P2_W1) copy_ref<2, fem::LAPLACE_P2_W1>(K);
    if (form == FEM_LAPLACE_P1_ISO) copy_ref<2, fem::LAPLACE_P1_ISO>(K);
    if (form == FEM_LAPLACE_P2_ISO) copy_ref<2, fem::LAPLACE_P2_ISO>(K);
  } else {
    if (form == FEM_LAPLACE_P1) copy_ref<3, fem::LAPLACE_P1>(K);
    if (form == FEM_LAPLACE_P2) copy_ref<3, fem::LAPLACE_P2>(K);
    if (form == FEM_ELASTIC_P1) copy_ref<3, fem::ELASTIC_P1>(K);
    if (form == FEM_LAPLACE_P1_W1) copy_ref<3, fem::LAPLACE_P1_W1>(K);
    if (form == FEM_LAPLACE_P2_W1) copy_ref<3, fem::LAPLACE_P2_W1>(K);
    if (form == FEM_LAPLACE_P1_ISO) copy_ref<3, fem::LAPLACE_P1_ISO>(K);
    if (form == FEM_LAPLACE_P2_ISO) copy_ref<3, fem::LAPLACE_P2_ISO>(K);
  }
  return ok();
}

static fem_status integrate_fwd(const fem_mesh* mesh, int32_t form, const float* coef, void* A, int32_t out_dtype,
                                float* det_out, const fem_options* options, void* stream) {
  fem_status s = check_mesh(mesh);
  if (s != FEM_OK) return s;
  if (!valid_form(form)) return fail(FEM_ERR_ARG, "form out of range");
  if (non_affine(form)) return fail(FEM_ERR_ARG, "non-affine forms take their edge nodes: fem_integrate_fwd_iso");
  if (out_dtype != FEM_F32 && out_dtype != FEM_F64) return fail(FEM_ERR_ARG, "out_dtype out of range");
  const fem_options* o = options ? options : &kDefaults;
  if ((s = check_options(o)) != FEM_OK) return s;
  if (mesh->n_elem == 0) return ok();
  if (!A) return fail(FEM_ERR_ARG, "A is NULL");
  const bool cf64 = mesh->coord_dtype == FEM_F64, of64 = out_dtype == FEM_F64;
  if ((cf64 || of64) && o->jac != FEM_JAC_AUTO && o->jac != FEM_JAC_F64)
    return fail(FEM_ERR_UNSUPPORTED, "FP64 coordinates or FP64 output need FEM_JAC_F64");
  const bool tc = o->contract == FEM_CONTRACT_BF16X3;
  if (coupling(form) && (cf64 || of64 || tc || (o->jac != FEM_JAC_AUTO && o->jac != FEM_JAC_COMP_F32)))
    return fail(FEM_ERR_UNSUPPORTED,
                "the coupling forms take FP32 coordinates and output, the compensated Jacobian and the FP32 "
                "contraction");
  if (tc && (form == FEM_LAPLACE_P1 || form == FEM_LAPLACE_P1_W1 || cf64 || of64 ||
             (o->jac != FEM_JAC_AUTO && o->jac != FEM_JAC_COMP_F32)))
    return fail(FEM_ERR_UNSUPPORTED,
                "the tensor-core contraction serves the P2 Laplacian (per-element or P1 coefficient) and "
                "elasticity with FP32 coordinates and output and the compensated Jacobian");
  fem::FwdLaunch L{};
  L.dim = mesh->dim;
  L.form = form;
  L.jac = resolve_jac(o->jac, cf64, of64);
  L.coord_f64 = cf64;
  L.out_f64 = of64;
  L.conn = mesh->conn;
  L.coords = mesh->coords;
  L.coef = coef;
  L.A = A;
  L.n_elem = mesh->n_elem;
  L.n_vert = mesh->n_vert;
  L.dev_err = o->dev_err;
  L.warps = o->warps_per_cta;  // 0: the kernel's default
  L.ctas_per_sm = o->ctas_per_sm;
  L.stream = static_cast<cudaStream_t>(stream);
  L.det_out = det_out;
  cudaError_t e;
  if (coupling(form))
    e = fem::launch_div_fwd(L);
  else if (tc)
    e = fem::launch_fwd_tc(L);
  else if (coef_p1(form))
    e = fem::launch_fwd_w1(L);
  else if (L.dim == 2)
    e = fem::launch_fwd_d2(L);
  else if (form == FEM_ELASTIC_P1)
    e = fem::launch_fwd_d3_ela(L);
  else
    e = fem::launch_fwd_d3_lap(L);
  if (e != cudaSuccess) return cuda_fail(e, "fem_integrate_fwd launch");
  return ok();
}

fem_status fem_integrate_fwd(const fem_mesh* mesh, int32_t form, const float* coef, void* A, int32_t out_dtype,
                             const fem_options* options, void* stream) {
  return integrate_fwd(mesh, form, coef, A, out_dtype, nullptr, options, stream);
}

fem_status fem_integrate_fwd_save(const fem_mesh* mesh, int32_t form, const float* coef, void* A,
                                  int32_t out_dtype, float* det, const fem_options* options, void* stream) {
  fem_status s = check_mesh(mesh);
  if (s != FEM_OK) return s;
  const fem_options* o = options ? options : &kDefaults;
  if (o->contract != FEM_CONTRACT_F32)
    return fail(FEM_ERR_UNSUPPORTED, "fem_integrate_fwd_save contracts in FP32");
  if (mesh->n_elem > 0 && !det) return fail(FEM_ERR_ARG, "det is NULL");
  return integrate_fwd(mesh, form, coef, A, out_dtype, det, options, stream);
}

fem_status fem_integrate_fwd_iso(const fem_mesh* mesh, int32_t form, const float* mid, const float* coef, float* A,
                                 const fem_options* options, void* stream) {
  fem_status s = check_mesh(mesh);
  if (s != FEM_OK) return s;
  if (!non_affine(form)) return fail(FEM_ERR_ARG, "form must be FEM_LAPLACE_P1_ISO or FEM_LAPLACE_P2_ISO");
  if (mesh->coord_dtype != FEM_F32) return fail(FEM_ERR_UNSUPPORTED, "non-affine elements take FP32 coordinates");
  const fem_options* o = options ? options : &kDefaults;
  if ((s = check_options(o)) != FEM_OK) return s;
  if (o->jac != FEM_JAC_AUTO && o->jac != FEM_JAC_F32)
    return fail(FEM_ERR_UNSUPPORTED, "non-affine elements compute their Jacobians in FP32");
  const bool tc = o->contract == FEM_CONTRACT_BF16X3;
  if (o->contract != FEM_CONTRACT_F32 && !(tc && form == FEM_LAPLACE_P2_ISO))
    return fail(FEM_ERR_UNSUPPORTED, "non-affine elements contract in FP32, or P2 on the tensor cores (BF16X3)");
  if (mesh->n_elem == 0) return ok();
  if (!A || !mid) return fail(FEM_ERR_ARG, "A or mid is NULL");
  fem::FwdLaunch L{};
  L.dim = mesh->dim;
  L.form = form;
  L.jac = fem::JAC_F32;
  L.conn = mesh->conn;
  L.coords = mesh->coords;
  L.coef = coef;
  L.A = A;
  L.n_elem = mesh->n_elem;
  L.n_vert = mesh->n_vert;
  L.dev_err = o->dev_err;
  L.ctas_per_sm = o->ctas_per_sm;
  L.stream = static_cast<cudaStream_t>(stream);
  cudaError_t e = tc ? fem::launch_fwd_iso_tc(L, mid) : fem::launch_fwd_iso(L, mid);
  if (e != cudaSuccess) return cuda_fail(e, "fem_integrate_fwd_iso launch");
  return ok();
}

fem_status fem_geometry(const fem_mesh* mesh, const float* coef, const fem_options* options, double* detJ,
                        float* G, void* stream) {
  fem_status s = check_mesh(mesh);
  if (s != FEM_OK) return s;
  const fem_options* o = options ? options : &kDefaults;
  if ((s = check_options(o)) != FEM_OK) return s;
  if (mesh->n_elem == 0 || (!detJ && !G)) return ok();
  const bool cf64 = mesh->coord_dtype == FEM_F64;
  if (cf64 && o->jac != FEM_JAC_AUTO && o->jac != FEM_JAC_F64)
    return fail(FEM_ERR_UNSUPPORTED, "FP64 coordinates need FEM_JAC_F64");
  fem::GeoLaunch L{};
  L.dim = mesh->dim;
  L.jac = resolve_jac(o->jac, cf64, false);
  L.coord_f64 = cf64;
  L.conn = mesh->conn;
  L.coords = mesh->coords;
  L.coef = coef;
  L.detJ = detJ;
  L.G = G;
  L.n_elem = mesh->n_elem;
  L.n_vert = mesh->n_vert;
  L.dev_err = o->dev_err;
  L.stream = static_cast<cudaStream_t>(stream);
  cudaError_t e = fem::launch_geometry(L);
  if (e != cudaSuccess) return cuda_fail(e, "fem_geometry launch");
  return ok();
}

fem_status fem_bwd_workspace_size(const fem_mesh* mesh, int32_t form, const fem_options* options,
                                  size_t* bytes) {
  fem_status s = check_mesh(mesh);
  if (s != FEM_OK) return s;
  if (!valid_form(form)) return fail(FEM_ERR_ARG, "form out of range");
  const fem_options* o = options ? options : &kDefaults;
  if ((s = check_options(o)) != FEM_OK) return s;
  if (!bytes) return fail(FEM_ERR_ARG, "bytes is NULL");
  if (mesh->n_elem * (mesh->dim + 1) > INT32_MAX)
    return fail(FEM_ERR_UNSUPPORTED, "n_elem * (dim + 1) exceeds the int32 slot range");
  *bytes = o->reduce == FEM_REDUCE_ATOMIC
               ? 0
               : fem::bwd_workspace_layout(mesh->dim, mesh->n_elem, mesh->n_vert, true, nullptr, nullptr,
                                           record_components(form, mesh->dim));
  return ok();
}

fem_status fem_incidence_build(const fem_mesh* mesh, void* ws, size_t ws_bytes, void* stream) {
  fem_status s = check_mesh(mesh);
  if (s != FEM_OK) return s;
  if (mesh->n_elem * (mesh->dim + 1) > INT32_MAX)
    return fail(FEM_ERR_UNSUPPORTED, "n_elem * (dim + 1) exceeds the int32 slot range");
  fem::BwdWorkspace W{};
  const size_t need = fem::bwd_workspace_layout(mesh->dim, mesh->n_elem, mesh->n_vert, true, ws, &W);
  if (!ws || ws_bytes < need) return fail(FEM_ERR_WORKSPACE, "workspace needs %zu bytes (got %zu)", need, ws_bytes);
  if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return fail(FEM_ERR_ARG, "workspace must be 256-byte aligned");
  cudaError_t e = fem::launch_incidence_build(mesh->dim, mesh->conn, mesh->n_elem, mesh->n_vert, W,
                                              static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "fem_incidence_build launch");
  return ok();
}

fem_status fem_incidence_info(const fem_mesh* mesh, const void* ws, size_t ws_bytes, int64_t* n_records,
                              int32_t* layout, void* stream) {
  fem_status s = check_mesh(mesh);
  if (s != FEM_OK) return s;
  fem::BwdWorkspace W{};
  const size_t need =
      fem::bwd_workspace_layout(mesh->dim, mesh->n_elem, mesh->n_vert, true, const_cast<void*>(ws), &W);
  if (!ws || ws_bytes < need) return fail(FEM_ERR_WORKSPACE, "workspace needs %zu bytes (got %zu)", need, ws_bytes);
  int32_t h[2] = {0, 0};
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(&h[0], W.tile_rec + W.n_tiles, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h[1], W.mode, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "fem_incidence_info");
  if (n_records) *n_records = h[0];
  if (layout) *layout = h[1];
  return ok();
}

static fem_status integrate_bwd(const fem_mesh* mesh, int32_t form, const float* coef, const float* dA,
                                const float* det_in, float* dcoords, float* dcoef, void* ws, size_t ws_bytes,
                                const fem_options* options, void* stream) {
  const fem_options* o = options ? options : &kDefaults;
  fem_status s = bwd_args(mesh, form, o, dA, dcoords);
  if (s != FEM_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const bool atomic = o->reduce == FEM_REDUCE_ATOMIC;
  const bool w1 = coef_p1(form);  // dcoef holds the gradient of the coefficient's vertex values
  const bool recs = bwd_uses_records(form, dcoords != nullptr, dcoef != nullptr, o->reduce);
  fem::BwdWorkspace W{};
  if (recs) {
    const size_t need = fem::bwd_workspace_layout(mesh->dim, mesh->n_elem, mesh->n_vert, true, ws, &W,
                                                  record_components(form, mesh->dim));
    if (!ws || ws_bytes < need) return fail(FEM_ERR_WORKSPACE, "workspace needs %zu bytes (got %zu)", need, ws_bytes);
    if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return fail(FEM_ERR_ARG, "workspace must be 256-byte aligned");
  }
  if (!dcoords && !dcoef) return ok();
  cudaError_t e;
  if (dcoords && atomic) {
    e = fem::launch_zero_f32(dcoords, mesh->n_vert * mesh->dim, st);
    if (e != cudaSuccess) return cuda_fail(e, "zeroing dcoords");
  }
  if (w1 && dcoef && atomic) {
    e = fem::launch_zero_f32(dcoef, mesh->n_vert, st);
    if (e != cudaSuccess) return cuda_fail(e, "zeroing dcoef");
  }
  if (mesh->n_elem > 0) {
    fem::BwdLaunch L{};
    L.dim = mesh->dim;
    L.form = form;
    L.jac = resolve_jac(o->jac, false, false);
    L.atomic = ((dcoords || (w1 && dcoef)) && atomic) ? 1 : 0;
    L.conn = mesh->conn;
    L.coords = static_cast<const float*>(mesh->coords);
    L.coef = coef;
    L.dA = dA;
    L.dcoef = dcoef;
    L.tile_rec = recs ? W.tile_rec : nullptr;
    L.rank = recs ? W.rank : nullptr;
    L.rec_span = recs ? W.rec_span : nullptr;
    L.rec_dest = recs ? W.rec_dest : nullptr;
    L.records = recs ? W.records : nullptr;
    L.dcoords = dcoords;
    L.n_elem = mesh->n_elem;
    L.n_vert = mesh->n_vert;
    L.dev_err = o->dev_err;
    L.warps = o->warps_per_cta;
    L.ctas_per_sm = o->ctas_per_sm;
    L.stream = st;
    L.det_in = det_in;
    e = coupling(form) ? fem::launch_div_bwd(L) : fem::launch_bwd_elem(L);
    if (e != cudaSuccess) return cuda_fail(e, "fem_integrate_bwd element launch");
  }
  if (recs && o->reduce == FEM_REDUCE_DETERMINISTIC) {
    e = fem::launch_vertex_reduce(mesh->dim, W, mesh->n_vert, dcoords, st, w1 ? dcoef : nullptr);
    if (e != cudaSuccess) return cuda_fail(e, "fem_integrate_bwd reduction launch");
  }
  return ok();
}

fem_status fem_integrate_bwd(const fem_mesh* mesh, int32_t form, const float* coef, const float* dA,
                             float* dcoords, float* dcoef, void* ws, size_t ws_bytes,
                             const fem_options* options, void* stream) {
  return integrate_bwd(mesh, form, coef, dA, nullptr, dcoords, dcoef, ws, ws_bytes, options, stream);
}

fem_status fem_integrate_bwd_saved(const fem_mesh* mesh, int32_t form, const float* coef, const float* dA,
                                   const float* det, float* dcoords, float* dcoef, void* ws, size_t ws_bytes,
                                   const fem_options* options, void* stream) {
  fem_status s = check_mesh(mesh);
  if (s != FEM_OK) return s;
  if (mesh->n_elem > 0 && !det) return fail(FEM_ERR_ARG, "det is NULL");
  return integrate_bwd(mesh, form, coef, dA, det, dcoords, dcoef, ws, ws_bytes, options, stream);
}

fem_status fem_integrate_bwd_iso(const fem_mesh* mesh, int32_t form, const float* mid, const float* coef,
                                 const float* dA, float* dcoords, float* dmid, float* dcoef, void* ws,
                                 size_t ws_bytes, const fem_options* options, void* stream) {
  fem_status s = check_mesh(mesh);
  if (s != FEM_OK) return s;
  if (!non_affine(form)) return fail(FEM_ERR_ARG, "form must be FEM_LAPLACE_P1_ISO or FEM_LAPLACE_P2_ISO");
  if (mesh->coord_dtype != FEM_F32) return fail(FEM_ERR_UNSUPPORTED, "non-affine elements take FP32 coordinates");
  const fem_options* o = options ? options : &kDefaults;
  if ((s = check_options(o)) != FEM_OK) return s;
  if (o->jac != FEM_JAC_AUTO && o->jac != FEM_JAC_F32)
    return fail(FEM_ERR_UNSUPPORTED, "non-affine elements compute their Jacobians in FP32");
  const bool tc = o->contract == FEM_CONTRACT_BF16X3;
  if (o->contract != FEM_CONTRACT_F32 &&
      !(tc && mesh->dim == 3 && form == FEM_LAPLACE_P2_ISO && o->reduce != FEM_REDUCE_ATOMIC))
    return fail(FEM_ERR_UNSUPPORTED,
                "the adjoint contracts in FP32, or with FEM_CONTRACT_BF16X3 for FEM_LAPLACE_P2_ISO on tetrahedra "
                "with the deterministic or deferred reduction");
  if (mesh->n_elem * (mesh->dim + 1) > INT32_MAX)
    return fail(FEM_ERR_UNSUPPORTED, "n_elem * (dim + 1) exceeds the int32 slot range");
  if (o->reduce == FEM_REDUCE_DEFERRED && !dcoords)
    return fail(FEM_ERR_ARG, "FEM_REDUCE_DEFERRED needs dcoords (written by fem_adjoint_reduce)");
  if (mesh->n_elem > 0 && (!dA || !mid)) return fail(FEM_ERR_ARG, "dA or mid is NULL");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const bool atomic = o->reduce == FEM_REDUCE_ATOMIC;
  const bool recs = dcoords && !atomic;
  fem::BwdWorkspace W{};
  if (recs) {
    const size_t need = fem::bwd_workspace_layout(mesh->dim, mesh->n_elem, mesh->n_vert, true, ws, &W);
    if (!ws || ws_bytes < need) return fail(FEM_ERR_WORKSPACE, "workspace needs %zu bytes (got %zu)", need, ws_bytes);
    if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return fail(FEM_ERR_ARG, "workspace must be 256-byte aligned");
  }
  if (!dcoords && !dmid && !dcoef) return ok();
  cudaError_t e;
  if (dcoords && atomic) {
    e = fem::launch_zero_f32(dcoords, mesh->n_vert * mesh->dim, st);
    if (e != cudaSuccess) return cuda_fail(e, "zeroing dcoords");
  }
  if (mesh->n_elem > 0) {
    fem::BwdLaunch L{};
    L.dim = mesh->dim;
    L.form = form;
    L.jac = fem::JAC_F32;
    L.atomic = atomic ? 1 : 0;
    L.conn = mesh->conn;
    L.coords = static_cast<const float*>(mesh->coords);
    L.coef = coef;
    L.dA = dA;
    L.dcoef = dcoef;
    L.tile_rec = recs ? W.tile_rec : nullptr;
    L.rank = recs ? W.rank : nullptr;
    L.rec_span = recs ? W.rec_span : nullptr;
    L.rec_dest = recs ? W.rec_dest : nullptr;
    L.records = recs ? W.records : nullptr;
    L.dcoords = dcoords;
    L.n_elem = mesh->n_elem;
    L.n_vert = mesh->n_vert;
    L.dev_err = o->dev_err;
    L.warps = 0;
    L.ctas_per_sm = o->ctas_per_sm;
    L.stream = st;
    e = tc ? fem::launch_bwd_iso_tc(L, mid, dmid) : fem::launch_bwd_iso(L, mid, dmid);
    if (e != cudaSuccess) return cuda_fail(e, "fem_integrate_bwd_iso element launch");
  }
  if (recs && o->reduce == FEM_REDUCE_DETERMINISTIC) {
    e = fem::launch_vertex_reduce(mesh->dim, W, mesh->n_vert, dcoords, st);
    if (e != cudaSuccess) return cuda_fail(e, "fem_integrate_bwd_iso reduction launch");
  }
  return ok();
}

fem_status fem_adjoint_reduce(const fem_mesh* mesh, const void* ws, size_t ws_bytes, float* dcoords,
                              void* stream) {
  fem_status s = check_mesh(mesh);
  if (s != FEM_OK) return s;
  if (!dcoords) return fail(FEM_ERR_ARG, "dcoords is NULL");
  if (mesh->n_elem * (mesh->dim + 1) > INT32_MAX)
    return fail(FEM_ERR_UNSUPPORTED, "n_elem * (dim + 1) exceeds the int32 slot range");
  fem::BwdWorkspace W{};
  const size_t need =
      fem::bwd_workspace_layout(mesh->dim, mesh->n_elem, mesh->n_vert, true, const_cast<void*>(ws), &W);
  if (!ws || ws_bytes < need) return fail(FEM_ERR_WORKSPACE, "workspace needs %zu bytes (got %zu)", need, ws_bytes);
  if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return fail(FEM_ERR_ARG, "workspace must be 256-byte aligned");
  cudaError_t e = fem::launch_vertex_reduce(mesh->dim, W, mesh->n_vert, dcoords, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "fem_adjoint_reduce launch");
  return ok();
}

}  // extern "C"
