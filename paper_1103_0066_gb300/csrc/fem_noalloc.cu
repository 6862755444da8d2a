// fem_noalloc.cu -- the adjoint for callers that cannot allocate device memory.
//
// fem_integrate_bwd needs a caller-allocated workspace (the tile records and
// the vertex -> record lists of the deterministic reduction).  Some callers
// cannot provide one: a host application that reserves all device memory up
// front and forbids allocation afterwards, or a solver callback that only
// receives raw pointers from a framework owning the allocator.  This entry point
// serves them from a fixed scratch array compiled into the library instead.
//
// The array below lives in device memory of every GPU that loads this library
// and stays allocated until the process exits.  Its host-side name is only a
// stand-in for the symbol: the device address is fetched once per device with
// cudaGetSymbolAddress and handed to the kernels like any workspace pointer.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/fem.h"
#include "fem_internal.h"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[FEM_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (looked up on the
// first call made with that device current, then cached).
fem_status scratch_on_current_device(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    fem::set_last_error("cudaGetDevice: %s", cudaGetErrorString(e));
    return FEM_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    fem::set_last_error("device ordinal %d out of range", dev);
    return FEM_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      fem::set_last_error("cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
      return FEM_ERR_CUDA;
    }
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return FEM_OK;
}

}  // namespace

extern "C" {

fem_status fem_integrate_bwd_noalloc(const fem_mesh* mesh, int32_t form, const float* coef, const float* dA,
                                     float* dcoords, float* dcoef, const fem_options* options, void* stream) {
  fem_options o = options ? *options : fem_options{0, 0, 0, 0, 0, 0, nullptr};
  if (o.reduce != FEM_REDUCE_DETERMINISTIC) {
    fem::set_last_error("fem_integrate_bwd_noalloc always uses the deterministic reduction");
    return FEM_ERR_UNSUPPORTED;
  }
  // Every refusal comes before the scratch array is touched: a refused call
  // launches nothing and leaves the array as the last accepted call left it.
  fem_status s = static_cast<fem_status>(fem::bwd_preflight(mesh, form, &o, dA, dcoords));
  if (s != FEM_OK) return s;
  if (!fem::bwd_needs_workspace(form, dcoords != nullptr, dcoef != nullptr, o.reduce)) {
    // only a per-element coefficient gradient: no scratch is involved
    return fem_integrate_bwd(mesh, form, coef, dA, dcoords, dcoef, nullptr, 0, &o, stream);
  }
  size_t need = 0;
  if ((s = fem_bwd_workspace_size(mesh, form, &o, &need)) != FEM_OK) return s;
  if (need > FEM_NOALLOC_SCRATCH_BYTES) {
    fem::set_last_error(
        "mesh needs %zu bytes of scratch, more than the %u built in; use fem_integrate_bwd with a "
        "caller-allocated workspace",
        need, unsigned(FEM_NOALLOC_SCRATCH_BYTES));
    return FEM_ERR_UNSUPPORTED;
  }
  void* ws = nullptr;
  if ((s = scratch_on_current_device(&ws)) != FEM_OK) return s;
  // The incidence build rewrites (and re-zeroes) everything the reduction reads,
  // so nothing a previous call left in the array matters.
  if ((s = fem_incidence_build(mesh, ws, FEM_NOALLOC_SCRATCH_BYTES, stream)) != FEM_OK) return s;
  return fem_integrate_bwd(mesh, form, coef, dA, dcoords, dcoef, ws, FEM_NOALLOC_SCRATCH_BYTES, &o, stream);
}

}  // extern "C"
