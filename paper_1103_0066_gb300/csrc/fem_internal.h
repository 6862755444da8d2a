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

// Adjoint element pass (FP32 coordinates).
struct BwdLaunch {
  int dim, form, jac, atomic;
  const int32_t* conn;
  const float* coords;
  const float* coef;
  const float* dA;
  float* dcoef;     // may be null
  float* xbar;      // deterministic: per-element scratch [E][dim+1][dim]
  float* dcoords;   // atomic: accumulated with red.add (pre-zeroed)
  int64_t n_elem, n_vert;
  int32_t* dev_err;
  int warps, ctas_per_sm;
  cudaStream_t stream;
};

// Workspace of the adjoint: [offsets V+1][incidence E*(d+1)][cursor V][scan partials][scratch]
struct BwdWorkspace {
  int32_t* offsets;
  int32_t* incidence;
  int32_t* cursor;
  int32_t* partials;
  float* scratch;
  size_t bytes;
};
size_t bwd_workspace_layout(int dim, int64_t n_elem, int64_t n_vert, bool with_scratch, void* base,
                            BwdWorkspace* ws);

cudaError_t launch_fwd_d2(const FwdLaunch& L);
cudaError_t launch_fwd_d3_lap(const FwdLaunch& L);
cudaError_t launch_fwd_d3_ela(const FwdLaunch& L);
cudaError_t launch_geometry(const GeoLaunch& L);
cudaError_t launch_bwd_elem(const BwdLaunch& L);
cudaError_t launch_incidence_build(int dim, const int32_t* conn, int64_t n_elem, int64_t n_vert,
                                   const BwdWorkspace& ws, cudaStream_t stream);
cudaError_t launch_zero_f32(float* p, int64_t n, cudaStream_t stream);
cudaError_t launch_vertex_reduce(int dim, const BwdWorkspace& ws, int64_t n_vert, float* dcoords,
                                 cudaStream_t stream);

// Device facts of the current device (cached per device).
int device_sm_count();
size_t device_smem_optin();
// Largest warp count <= want whose per-warp stage (bytes_per_warp) fits the opt-in shared memory.
int clamp_warps(int want, size_t bytes_per_warp);
// Raises the dynamic shared memory limit of a kernel when it needs more than 48 KB.
cudaError_t ensure_smem(const void* kernel, size_t bytes);

}  // namespace fem
