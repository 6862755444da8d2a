// fem_host_step.cu -- end-to-end step from page-locked host memory (C ABI in
// include/fem.h): host -> device copies, the forward (Eq. 6) saving det J, the
// deterministic adjoint taking it, device -> host copies, overlapped per slice
// of elements on two copy streams beside the caller's stream.
#include <cuda_runtime.h>

#include <cstdint>
#include <new>
#include <vector>

#include "../../include/fem.h"
#include "fem_internal.h"

struct fem_host_step {
  int32_t form = 0, dim = 0, n = 0;
  int64_t n_vert = 0, n_elem = 0, chunk = 0;
  int device = 0;
  float* coords = nullptr;
  int32_t* conn = nullptr;
  float* dA = nullptr;
  float* A = nullptr;
  float* det = nullptr;
  float* dcoords = nullptr;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  bool built = false;
  cudaStream_t copy_in = nullptr, copy_out = nullptr;
  cudaEvent_t start = nullptr, reduced = nullptr, done = nullptr;
  std::vector<cudaEvent_t> conn_in, dA_in, A_written;  // per slice
};

namespace {

void release(fem_host_step* h) {
  if (h->copy_in) cudaStreamSynchronize(h->copy_in);
  if (h->copy_out) cudaStreamSynchronize(h->copy_out);
  for (auto* v : {&h->conn_in, &h->dA_in, &h->A_written})
    for (cudaEvent_t e : *v)
      if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : {h->start, h->reduced, h->done})
    if (e) cudaEventDestroy(e);
  if (h->copy_in) cudaStreamDestroy(h->copy_in);
  if (h->copy_out) cudaStreamDestroy(h->copy_out);
  for (void* p : {static_cast<void*>(h->coords), static_cast<void*>(h->conn), static_cast<void*>(h->dA),
                  static_cast<void*>(h->A), static_cast<void*>(h->det), static_cast<void*>(h->dcoords), h->ws})
    if (p) cudaFree(p);
  delete h;
}

fem_status cuda_err(cudaError_t e, const char* what) {
  fem::set_last_error("%s: %s", what, cudaGetErrorString(e));
  return FEM_ERR_CUDA;
}

fem_status arg_err(const char* msg) {
  fem::set_last_error("%s", msg);
  return FEM_ERR_ARG;
}

// Page-locked host memory: registered or allocated by CUDA, not device memory.
bool pinned_host(const void* p) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost;
}

fem_mesh device_mesh(const fem_host_step* h, int64_t e0, int64_t e1) {
  fem_mesh m{};
  m.dim = h->dim;
  m.coord_dtype = FEM_F32;
  m.n_vert = h->n_vert;
  m.n_elem = e1 - e0;
  m.conn = h->conn + e0 * (h->dim + 1);
  m.coords = h->coords;
  return m;
}

}  // namespace

extern "C" {

fem_status fem_host_step_create(int32_t form, int32_t dim, int64_t n_vert, int64_t n_elem, int64_t chunk,
                                fem_host_step** step) {
  if (!step) return arg_err("step is NULL");
  *step = nullptr;
  if (form != FEM_LAPLACE_P1 && form != FEM_LAPLACE_P2 && form != FEM_ELASTIC_P1) {
    fem::set_last_error("the host step takes FEM_LAPLACE_P1, FEM_LAPLACE_P2 or FEM_ELASTIC_P1 (got %d)", form);
    return FEM_ERR_UNSUPPORTED;
  }
  if (dim != 2 && dim != 3) return arg_err("dim must be 2 or 3");
  if (n_vert <= 0 || n_elem <= 0 || chunk < 0) return arg_err("n_vert and n_elem must be positive, chunk >= 0");
  if (n_vert > INT32_MAX || n_elem * (dim + 1) > INT32_MAX) {
    fem::set_last_error("mesh exceeds the int32 index range");
    return FEM_ERR_UNSUPPORTED;
  }
  int32_t n = 0, ng = 0, den = 0;
  fem_status s = fem_form_info(form, dim, &n, &ng, &den);
  if (s != FEM_OK) return s;
  fem_host_step* h = new (std::nothrow) fem_host_step();
  if (!h) return cuda_err(cudaErrorMemoryAllocation, "fem_host_step_create");
  h->form = form;
  h->dim = dim;
  h->n = n;
  h->n_vert = n_vert;
  h->n_elem = n_elem;
  const int64_t c = chunk > 0 ? chunk : (int64_t(1) << 20);
  h->chunk = (c + fem::kRecTile - 1) / fem::kRecTile * fem::kRecTile;
  cudaError_t e = cudaGetDevice(&h->device);
  const size_t nn = size_t(n) * n;
  if (e == cudaSuccess) e = cudaMalloc(&h->coords, sizeof(float) * n_vert * dim);
  if (e == cudaSuccess) e = cudaMalloc(&h->conn, sizeof(int32_t) * n_elem * (dim + 1));
  if (e == cudaSuccess) e = cudaMalloc(&h->dA, sizeof(float) * n_elem * nn);
  if (e == cudaSuccess) e = cudaMalloc(&h->A, sizeof(float) * n_elem * nn);
  if (e == cudaSuccess) e = cudaMalloc(&h->det, sizeof(float) * n_elem);
  if (e == cudaSuccess) e = cudaMalloc(&h->dcoords, sizeof(float) * n_vert * dim);
  if (e != cudaSuccess) {
    release(h);
    return cuda_err(e, "fem_host_step_create allocation");
  }
  const fem_mesh m = device_mesh(h, 0, n_elem);
  if ((s = fem_bwd_workspace_size(&m, form, nullptr, &h->ws_bytes)) != FEM_OK) {
    release(h);
    return s;
  }
  e = cudaMalloc(&h->ws, h->ws_bytes);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->copy_in, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->copy_out, cudaStreamNonBlocking);
  for (cudaEvent_t* ev : {&h->start, &h->reduced, &h->done})
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
  const int64_t n_slices = (n_elem + h->chunk - 1) / h->chunk;
  for (auto* v : {&h->conn_in, &h->dA_in, &h->A_written}) {
    v->assign(size_t(n_slices), nullptr);
    for (cudaEvent_t& ev : *v)
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    release(h);
    return cuda_err(e, "fem_host_step_create");
  }
  *step = h;
  fem::set_last_error("%s", "");
  return FEM_OK;
}

fem_status fem_host_step_run(fem_host_step* h, const float* coords, const int32_t* conn, const float* dA, float* A,
                             float* dcoords, int32_t rebuild, void* stream) {
  if (!h) return arg_err("step is NULL");
  if (!coords || !conn || !dA || !A || !dcoords) return arg_err("a host buffer is NULL");
  for (const void* p : {static_cast<const void*>(coords), static_cast<const void*>(conn),
                        static_cast<const void*>(dA), static_cast<const void*>(A), static_cast<const void*>(dcoords)})
    if (!pinned_host(p))
      return arg_err("host buffers must be page-locked host memory (cudaHostAlloc or cudaHostRegister)");
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_err(e, "fem_host_step_run");
  if (dev != h->device) return arg_err("the current device is not the step's device");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int d = h->dim;
  const size_t nn = size_t(h->n) * h->n;
  const int64_t E = h->n_elem, C = h->chunk;
  const int64_t n_slices = int64_t(h->conn_in.size());
  auto slice_end = [&](int64_t s) { return s + 1 < n_slices ? (s + 1) * C : E; };
  const bool build = !h->built || rebuild != 0;

  // the copies in wait for the previous step's kernels (queued on `st`)
  if ((e = cudaEventRecord(h->start, st)) != cudaSuccess) return cuda_err(e, "event record");
  if ((e = cudaStreamWaitEvent(h->copy_in, h->start, 0)) != cudaSuccess) return cuda_err(e, "stream wait");
  if ((e = cudaStreamWaitEvent(h->copy_out, h->start, 0)) != cudaSuccess) return cuda_err(e, "stream wait");
  e = cudaMemcpyAsync(h->coords, coords, sizeof(float) * h->n_vert * d, cudaMemcpyHostToDevice, h->copy_in);
  for (int64_t s = 0; s < n_slices && e == cudaSuccess; ++s) {
    const int64_t e0 = s * C, e1 = slice_end(s);
    // the connectivity goes in with the runs that build the incidence from it;
    // the other runs reuse both (conn is not read)
    if (build)
      e = cudaMemcpyAsync(h->conn + e0 * (d + 1), conn + e0 * (d + 1), sizeof(int32_t) * (e1 - e0) * (d + 1),
                          cudaMemcpyHostToDevice, h->copy_in);
    if (e == cudaSuccess) e = cudaEventRecord(h->conn_in[size_t(s)], h->copy_in);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h->dA + e0 * nn, dA + e0 * nn, sizeof(float) * (e1 - e0) * nn, cudaMemcpyHostToDevice,
                          h->copy_in);
    if (e == cudaSuccess) e = cudaEventRecord(h->dA_in[size_t(s)], h->copy_in);
  }
  if (e != cudaSuccess) return cuda_err(e, "fem_host_step_run copies in");

  const fem_mesh whole = device_mesh(h, 0, E);
  auto forward = [&](int64_t s) -> fem_status {
    const int64_t e0 = s * C, e1 = slice_end(s);
    cudaError_t ee = cudaStreamWaitEvent(st, h->conn_in[size_t(s)], 0);
    if (ee != cudaSuccess) return cuda_err(ee, "stream wait");
    const fem_mesh m = device_mesh(h, e0, e1);
    fem_status r = fem_integrate_fwd_save(&m, h->form, nullptr, h->A + e0 * nn, FEM_F32, h->det + e0, nullptr, st);
    if (r != FEM_OK) return r;
    ee = cudaEventRecord(h->A_written[size_t(s)], st);
    return ee == cudaSuccess ? FEM_OK : cuda_err(ee, "event record");
  };
  auto adjoint = [&](int64_t s) -> fem_status {
    const cudaError_t ee = cudaStreamWaitEvent(st, h->dA_in[size_t(s)], 0);
    if (ee != cudaSuccess) return cuda_err(ee, "stream wait");
    return static_cast<fem_status>(
        fem::bwd_element_range(&whole, h->form, h->dA, h->det, h->ws, h->ws_bytes, s * C, slice_end(s), st));
  };
  fem_status r = FEM_OK;
  if (!build) {
    // slice by slice in arrival order: forward on its connectivity, adjoint on its dA
    for (int64_t s = 0; s < n_slices && r == FEM_OK; ++s) {
      r = forward(s);
      if (r == FEM_OK) r = adjoint(s);
    }
  } else {
    // the incidence needs the whole connectivity: forwards, the build, then the adjoints
    for (int64_t s = 0; s < n_slices && r == FEM_OK; ++s) r = forward(s);
    if (r == FEM_OK) r = fem_incidence_build(&whole, h->ws, h->ws_bytes, st);
    if (r == FEM_OK) h->built = true;
    for (int64_t s = 0; s < n_slices && r == FEM_OK; ++s) r = adjoint(s);
  }
  if (r == FEM_OK) r = fem_adjoint_reduce(&whole, h->ws, h->ws_bytes, h->dcoords, st);
  if (r != FEM_OK) return r;

  // copies out: each slice's A once written, dcoords after the reduction
  for (int64_t s = 0; s < n_slices && e == cudaSuccess; ++s) {
    const int64_t e0 = s * C, e1 = slice_end(s);
    e = cudaStreamWaitEvent(h->copy_out, h->A_written[size_t(s)], 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(A + e0 * nn, h->A + e0 * nn, sizeof(float) * (e1 - e0) * nn, cudaMemcpyDeviceToHost,
                          h->copy_out);
  }
  if (e == cudaSuccess) e = cudaEventRecord(h->reduced, st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h->copy_out, h->reduced, 0);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dcoords, h->dcoords, sizeof(float) * h->n_vert * d, cudaMemcpyDeviceToHost, h->copy_out);
  // the caller's stream orders after every copy of this step (the copies in
  // were waited for by the last slice's adjoint)
  if (e == cudaSuccess) e = cudaEventRecord(h->done, h->copy_out);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st, h->done, 0);
  if (e != cudaSuccess) return cuda_err(e, "fem_host_step_run copies out");
  fem::set_last_error("%s", "");
  return FEM_OK;
}

void fem_host_step_destroy(fem_host_step* h) {
  if (h) release(h);
}

}  // extern "C"
