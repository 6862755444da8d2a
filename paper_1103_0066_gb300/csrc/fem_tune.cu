// fem_tune.cu -- launch-shape autotuner of the single-mesh kernels (C ABI in
// include/fem.h): every candidate (warps per CTA, CTAs per SM) pair is timed
// with CUDA events on the caller's stream and the fastest is returned.
#include <cuda_runtime.h>

#include <functional>

#include "../../include/fem.h"
#include "fem_internal.h"

namespace {

constexpr int kWarps[] = {0, 1, 2, 4, 8};
constexpr int kCtas[] = {0, 2, 4, 8, 16, 24, 32};
constexpr int kUntimed = 2, kTimed = 5;

// Times `call` (one launch sequence with the given options) for every
// candidate; returns the status of the first failing candidate call if none
// ran, else FEM_OK with the fastest pair in *options.
fem_status tune(fem_options* options, float* best_ms, cudaStream_t st,
                const std::function<fem_status(const fem_options*)>& call) {
  if (!options) {
    fem::set_last_error("options is NULL");
    return FEM_ERR_ARG;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t ce = cudaEventCreate(&e0);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    fem::set_last_error("fem_tune: %s", cudaGetErrorString(ce));
    return FEM_ERR_CUDA;
  }
  fem_options best = *options;
  float best_t = -1.f;
  fem_status first_err = FEM_OK;
  for (int w : kWarps) {
    for (int c : kCtas) {
      fem_options o = *options;
      o.warps_per_cta = w;
      o.ctas_per_sm = c;
      fem_status s = FEM_OK;
      for (int i = 0; i < kUntimed && s == FEM_OK; ++i) s = call(&o);
      if (s == FEM_OK && cudaEventRecord(e0, st) != cudaSuccess) s = FEM_ERR_CUDA;
      for (int i = 0; i < kTimed && s == FEM_OK; ++i) s = call(&o);
      if (s == FEM_OK && cudaEventRecord(e1, st) != cudaSuccess) s = FEM_ERR_CUDA;
      if (s == FEM_OK && cudaEventSynchronize(e1) != cudaSuccess) s = FEM_ERR_CUDA;
      float ms = 0.f;
      if (s == FEM_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) s = FEM_ERR_CUDA;
      if (s != FEM_OK) {
        // a shape this kernel cannot launch (e.g. its stage exceeds shared
        // memory) is skipped; the default shape never fails this way
        if (first_err == FEM_OK) first_err = s;
        cudaGetLastError();
        continue;
      }
      ms /= kTimed;
      if (best_t < 0.f || ms < best_t) {
        best_t = ms;
        best = o;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (best_t < 0.f) return first_err != FEM_OK ? first_err : FEM_ERR_CUDA;
  // leave the caller's outputs with the values of one call at the chosen shape
  const fem_status s = call(&best);
  if (s != FEM_OK) return s;
  options->warps_per_cta = best.warps_per_cta;
  options->ctas_per_sm = best.ctas_per_sm;
  if (best_ms) *best_ms = best_t;
  fem::set_last_error("%s", "");
  return FEM_OK;
}

}  // namespace

extern "C" {

fem_status fem_tune_fwd(const fem_mesh* mesh, int32_t form, const float* coef, void* A, int32_t out_dtype,
                        float* det, fem_options* options, float* best_ms, void* stream) {
  return tune(options, best_ms, static_cast<cudaStream_t>(stream), [&](const fem_options* o) {
    return det ? fem_integrate_fwd_save(mesh, form, coef, A, out_dtype, det, o, stream)
               : fem_integrate_fwd(mesh, form, coef, A, out_dtype, o, stream);
  });
}

fem_status fem_tune_bwd(const fem_mesh* mesh, int32_t form, const float* coef, const float* dA, const float* det,
                        float* dcoords, float* dcoef, void* ws, size_t ws_bytes, fem_options* options,
                        float* best_ms, void* stream) {
  return tune(options, best_ms, static_cast<cudaStream_t>(stream), [&](const fem_options* o) {
    return det ? fem_integrate_bwd_saved(mesh, form, coef, dA, det, dcoords, dcoef, ws, ws_bytes, o, stream)
               : fem_integrate_bwd(mesh, form, coef, dA, dcoords, dcoef, ws, ws_bytes, o, stream);
  });
}

}  // extern "C"
