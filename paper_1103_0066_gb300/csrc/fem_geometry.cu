// fem_geometry.cu -- the Jacobian-step test hook (det J and the Laplacian G per
// element, Eqs. 5 and 8) and host-side device queries.
#include <mutex>

#include <cudaTypedefs.h>

#include "fem_core.cuh"
#include "fem_fwd.cuh"
#include "fem_internal.h"

namespace fem {

template <int D, int JAC, class CT>
__global__ void fem_geometry_kernel(const int32_t* conn, const CT* coords, const float* coef,
                                    double* detJ, float* G, int64_t n_elem, int64_t n_vert,
                                    int32_t* dev_err) {
  constexpr int NGL = D * (D + 1) / 2;
  int err = 0;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n_elem;
       e += int64_t(gridDim.x) * blockDim.x) {
    int v[D + 1];
    CT X[D + 1][D];
    double det = 0.0;
    float g[NGL];
#pragma unroll
    for (int k = 0; k < NGL; ++k) g[k] = 0.f;
    load_conn<D>(conn, e, n_elem, 0, v);
    if (!gather<D>(coords, n_vert, v, X)) {
      err |= DEVERR_CONN;
    } else {
      using GT = typename std::conditional<JAC == JAC_F64, double, float>::type;
      Jac<D, GT> j;
      if (!jacobian<D, JAC>(X, j)) {
        err |= DEVERR_DEGENERATE;
      } else {
        det = j.det_hp;
        GT s = GT(coef ? coef[e] : 1.f) / dev_abs(j.det);
        GT gg[NGL];
        geometric_tensor<D, LAPLACE_P1>(j.adj, s, gg);
#pragma unroll
        for (int k = 0; k < NGL; ++k) g[k] = float(gg[k]);
      }
    }
    if (detJ) detJ[e] = det;
    if (G) {
#pragma unroll
      for (int k = 0; k < NGL; ++k) G[e * NGL + k] = g[k];
    }
  }
  if (err && dev_err) atomicOr(dev_err, err);
}

template <int D, int JAC, class CT>
static cudaError_t launch_geo_t(const GeoLaunch& L) {
  int64_t grid = (L.n_elem + 255) / 256;
  if (grid > 65535) grid = 65535;
  fem_geometry_kernel<D, JAC, CT><<<unsigned(grid), 256, 0, L.stream>>>(
      L.conn, static_cast<const CT*>(L.coords), L.coef, L.detJ, L.G, L.n_elem, L.n_vert, L.dev_err);
  return cudaGetLastError();
}

template <int D>
static cudaError_t launch_geo_d(const GeoLaunch& L) {
  if (L.coord_f64) return launch_geo_t<D, JAC_F64, double>(L);
  switch (L.jac) {
    case JAC_F64: return launch_geo_t<D, JAC_F64, float>(L);
    case JAC_COMP: return launch_geo_t<D, JAC_COMP, float>(L);
    case JAC_F32: return launch_geo_t<D, JAC_F32, float>(L);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_geometry(const GeoLaunch& L) {
  return L.dim == 2 ? launch_geo_d<2>(L) : launch_geo_d<3>(L);
}

// ---------------------------------------------------------------- device queries

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_dev_mu;
int g_sm_count[kMaxDevices] = {0};
size_t g_smem_optin[kMaxDevices] = {0};
}  // namespace

size_t device_smem_optin() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return 48 * 1024;
  std::lock_guard<std::mutex> lk(g_dev_mu);
  if (g_smem_optin[dev] == 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess || n <= 0)
      n = 48 * 1024;
    g_smem_optin[dev] = size_t(n);
  }
  return g_smem_optin[dev];
}

int clamp_warps(int want, size_t bytes_per_warp) {
  const size_t cap = device_smem_optin();
  int w = want < 1 ? 1 : (want > 16 ? 16 : want);
  while (w > 1 && size_t(w) * bytes_per_warp > cap) --w;
  return w;
}

int device_sm_count() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return 1;
  std::lock_guard<std::mutex> lk(g_dev_mu);
  if (g_sm_count[dev] == 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
    g_sm_count[dev] = n;
  }
  return g_sm_count[dev];
}

unsigned pipeline_grid(const void* kernel, int warps, size_t smem, int64_t n_elem, int ctas_per_sm) {
  int per_sm = ctas_per_sm;
  if (per_sm <= 0) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, warps * 32, smem) != cudaSuccess ||
        per_sm <= 0) {
      cudaGetLastError();
      per_sm = 1;
    }
  }
  const int64_t ntiles = (n_elem + 31) / 32;
  int64_t grid = int64_t(per_sm) * device_sm_count();
  const int64_t need = (ntiles + warps - 1) / warps;
  if (grid > need) grid = need;
  return unsigned(grid < 1 ? 1 : grid);
}

cudaError_t ensure_smem(const void* kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
  if (e != cudaSuccess) return e;
  // prefer the largest shared-memory carveout so that several such CTAs fit on an SM
  return cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                              int(cudaSharedmemCarveoutMaxShared));
}

namespace {
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}
}  // namespace

bool encode_rows16_map(CUtensorMap* map, const void* base, int64_t rows) {
  if (!base || rows <= 0 || rows > (int64_t(1) << 32) || reinterpret_cast<uintptr_t>(base) % 16 != 0) return false;
  PFN_cuTensorMapEncodeTiled_v12000 fn = tensor_map_encoder();
  if (!fn) return false;
  const cuuint64_t dims[2] = {16, cuuint64_t(rows)};
  const cuuint64_t strides[1] = {64};  // bytes between rows
  const cuuint32_t box[2] = {16, 32};  // one warp's tile
  const cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace fem
