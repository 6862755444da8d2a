// fem_fwd.cuh -- forward element integration kernel (Knepley & Terrel, Sec. 4).
//
// Work decomposition (GB300 design, not the paper's GTX285 thread-per-entry
// mapping): a warp owns a tile of 32 consecutive elements, one element per
// lane, and walks its tiles grid-stride as a three-stage software pipeline:
//   stage 1 (tile t+2): connectivity loaded into registers (one 16-byte load per tet)
//   stage 2 (tile t+1): vertex coordinates gathered into registers (L2-resident)
//   stage 3 (tile t)  : Jacobian, geometric tensor, sparse G:K contraction with
//                       K as immediates, staging and coalesced 16-byte
//                       evict-first stores of the tile's 32 * n^2 contiguous outputs
// so the gather latency hides behind the previous tile's arithmetic.  For the
// 4x4 FP32 element matrices the stage is the 64-byte-swizzled image of the
// tile's 32 rows (16-byte chunk q of row l at q ^ ((l >> 1) & 3): bank-
// conflict-free row writes), double buffered, and one lane stores the whole
// tile with a TMA tensor store that undoes the swizzle; without a tensor map
// (unaligned A) the warp reads the stage back into coalesced 16-byte
// evict-first stores.  Other shapes use an odd row stride and the coalesced
// read-out.  Every element is integrated: the final tile is partial (no
// dropped tail; the tensor store clips rows past the end).
#pragma once
#include <cuda_runtime.h>

#include "fem_core.cuh"
#include "fem_internal.h"
#include "fem_pipe.cuh"

namespace fem {

template <class CT, class OT>
struct FwdParams {
  const int32_t* conn;
  const CT* coords;
  const float* coef;
  OT* A;
  int64_t n_elem;
  int64_t n_vert;
  int32_t* dev_err;
  int vec_conn;   // conn rows are 16-byte aligned int4 (tets)
  int vec_store;  // A is 16-byte aligned
  float* det_out = nullptr;  // [n_elem] det J saved for the adjoint, or null
};

template <int NN>
constexpr int stage_stride() {
  return NN | 1;
}
constexpr size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// CTA shape of the forward kernel.  Warps never wait for one another, so the
// CTA size only sets how finely the register file is shared out.  The 3D P1
// Laplacian in FP32 with the compensated Jacobian runs one-warp CTAs with at
// least 24 resident per SM, which holds it to 80 registers without spills
// (25 warps per SM against 20 at its natural 90 in 4-warp CTAs; 9% faster).
// The same at 96 registers made P1 elasticity and the P2 Laplacian with a P1
// coefficient 1-5% slower, so the other instantiations take up to 16 warps
// per CTA (4 by default) and the compiler's register choice.
template <int D, int FORM, int JAC, class CT, class OT>
struct FwdShape {
  static constexpr int tight_ctas() {
    if (!(D == 3 && JAC == JAC_COMP && sizeof(CT) == 4 && sizeof(OT) == 4)) return 0;
    return FORM == LAPLACE_P1 ? 24 : 0;
  }
  static constexpr bool tight = tight_ctas() > 0;
  static constexpr int threads = tight ? 32 : 512;
  static constexpr int min_ctas = tight ? tight_ctas() : 1;
  static constexpr int default_warps = tight ? 1 : 4;
};

// Shared-memory plan of one warp.
template <int D, int FORM, class CT, class OT>
struct FwdPlan {
  static constexpr int NN = FormTraits<D, FORM>::NN;
  static constexpr bool SWZ16 = (NN == 16 && sizeof(OT) == 4);  // swizzled float4 rows
  static constexpr int SST = SWZ16 ? 16 : stage_stride<NN>();
  static constexpr size_t stage_bytes = align_up(size_t(32) * SST * sizeof(OT), 128);
  static constexpr size_t per_warp = stage_bytes;
  // TMA store variant (SWZ16 only): two 2 KB stages per warp, 1024-byte aligned
  static constexpr size_t tma_per_warp = 2 * 2048;
};

template <int N, int SST, class OT>
struct StageSink {
  OT* row;
  template <int I, int J>
  __device__ __forceinline__ void put(OT v) {
    row[I * N + J] = v;
    if constexpr (I != J) row[J * N + I] = v;
  }
};

template <int N, class T>
struct RegSink {
  T a[N * N];
  template <int I, int J>
  __device__ __forceinline__ void put(T v) {
    a[I * N + J] = v;
    if constexpr (I != J) a[J * N + I] = v;
  }
};

// Connectivity of element e into registers (-1 marks "no element").
template <int D>
__device__ __forceinline__ void load_conn(const int32_t* conn, int64_t e, int64_t n_elem, int vec,
                                          int (&v)[D + 1]) {
  if (e >= n_elem) {
#pragma unroll
    for (int k = 0; k <= D; ++k) v[k] = -1;
    return;
  }
  if constexpr (D == 3) {
    if (vec) {
      int4 c = __ldcs(reinterpret_cast<const int4*>(conn) + e);
      v[0] = c.x;
      v[1] = c.y;
      v[2] = c.z;
      v[3] = c.w;
      return;
    }
  }
#pragma unroll
  for (int k = 0; k <= D; ++k) v[k] = __ldcs(conn + e * (D + 1) + k);
}

// Synchronous gather (used by the geometry hook): false when a vertex id is out of range.
template <int D, class CT>
__device__ __forceinline__ bool gather(const CT* coords, int64_t n_vert, const int (&v)[D + 1],
                                       CT (&X)[D + 1][D]) {
  bool ok = true;
#pragma unroll
  for (int k = 0; k <= D; ++k) ok &= (v[k] >= 0) & (int64_t(v[k]) < n_vert);
  if (!ok) return false;
#pragma unroll
  for (int k = 0; k <= D; ++k)
#pragma unroll
    for (int a = 0; a < D; ++a) X[k][a] = __ldg(coords + int64_t(v[k]) * D + a);
  return true;
}

// Gather flags carried from stage 2 to stage 3.
enum : int { GF_ELEM = 1, GF_OK = 2 };

// Stage 2: validates the element's vertex ids and issues the loads of its
// (d+1) x d coordinates into registers (consumed one pipeline step later).
template <int D, class CT>
__device__ __forceinline__ int gather_regs(const CT* coords, int64_t n_vert, int64_t e, int64_t n_elem,
                                           const int (&v)[D + 1], CT (&X)[D + 1][D]) {
  if (e >= n_elem) return 0;
  bool ok = true;  // n_vert <= INT32_MAX, so one unsigned compare covers v < 0
#pragma unroll
  for (int k = 0; k <= D; ++k) ok &= uint32_t(v[k]) < uint32_t(n_vert);
  if (!ok) return GF_ELEM;
#pragma unroll
  for (int k = 0; k <= D; ++k) {
    const CT* c = coords + uint32_t(v[k]) * uint64_t(D);
#pragma unroll
    for (int a = 0; a < D; ++a) X[k][a] = __ldg(c + a);
  }
  return GF_ELEM | GF_OK;
}

// A lane's element matrix and the tile's store: fill(sink) hands every unique
// entry (i <= j) to sink.put<i, j>(value); then the swizzled stage and its TMA
// tensor store (TMA), else the stage and the warp's coalesced read-out.
template <int D, int FORM, class CT, class OT, bool TMA, class Fill>
__device__ __forceinline__ void fwd_fill_store(const FwdParams<CT, OT>& p, int64_t tile, int lane, Fill&& fill,
                                               OT* st, const CUtensorMap* tmap) {
  using FT = FormTraits<D, FORM>;
  using PL = FwdPlan<D, FORM, CT, OT>;
  constexpr int NN = FT::NN;
  constexpr int SST = PL::SST;
  const int64_t e0 = tile * 32;
  const int cnt = int(p.n_elem - e0 < 32 ? p.n_elem - e0 : 32);
  OT* dst = p.A + e0 * NN;
  if constexpr (PL::SWZ16) {
    // rows as float4 chunks, chunk index XOR-swizzled with (lane >> 1) & 3
    RegSink<4, float> rs;
    fill(rs);
    const int sw = (lane >> 1) & 3;
    float* row = st + lane * 16;
    if constexpr (TMA) {
      if (lane == 0) bulk_wait_read<1>();  // the store that last read this stage (two tiles ago) is done
      __syncwarp();
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
      *reinterpret_cast<float4*>(row + 4 * (r ^ sw)) =
          make_float4(rs.a[4 * r], rs.a[4 * r + 1], rs.a[4 * r + 2], rs.a[4 * r + 3]);
    if constexpr (TMA) {
      fence_proxy_async_smem();  // the rows are visible to the tensor store
      __syncwarp();
      if (lane == 0) {
        tma_store_2d(tmap, 0, int(e0), smem_u32(st));
        bulk_commit();
      }
      return;
    }
    __syncwarp();
    // chunk c = lane + 32 r holds element (lane >> 2) + 8 r, row lane & 3
    const float* src = st + 16 * (lane >> 2) + 4 * ((lane & 3) ^ ((lane >> 3) & 3));
    if (p.vec_store) {
      float4* d4 = reinterpret_cast<float4*>(dst);
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int c = lane + 32 * r;
        if (c < 4 * cnt) __stcs(d4 + c, *reinterpret_cast<const float4*>(src + 128 * r));
      }
    } else {
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int c = lane + 32 * r;
        if (c < 4 * cnt) {
          const float4 v = *reinterpret_cast<const float4*>(src + 128 * r);
          __stcs(dst + 4 * c, v.x);
          __stcs(dst + 4 * c + 1, v.y);
          __stcs(dst + 4 * c + 2, v.z);
          __stcs(dst + 4 * c + 3, v.w);
        }
      }
    }
  } else {
    StageSink<FT::N, SST, OT> sink{st + lane * SST};
    fill(sink);
    __syncwarp();
    bool done = false;
    if constexpr (sizeof(OT) == 4 && NN % 4 == 0) {
      if (p.vec_store) {
        const int nq = cnt * (NN / 4);
        for (int q = lane; q < nq; q += 32) {
          const int idx = 4 * q;
          const int el = idx / NN;
          const OT* s = st + el * SST + (idx - el * NN);
          __stcs(reinterpret_cast<float4*>(dst) + q, make_float4(s[0], s[1], s[2], s[3]));
        }
        done = true;
      }
    }
    if (!done) {
      const int nw = cnt * NN;
      for (int idx = lane; idx < nw; idx += 32) {
        const int el = idx / NN;
        __stcs(dst + idx, st[el * SST + (idx - el * NN)]);
      }
    }
  }
  __syncwarp();
}

// Contraction of a lane's folded G with K (immediates), then the tile's store.
template <int D, int FORM, class CT, class OT, bool TMA = false>
__device__ __forceinline__ void fwd_contract_store(const FwdParams<CT, OT>& p, int64_t tile, int lane,
                                                   const OT (&Gf)[FormTraits<D, FORM>::NG], OT* st,
                                                   const CUtensorMap* tmap) {
  fwd_fill_store<D, FORM, CT, OT, TMA>(p, tile, lane, [&](auto& sink) { contract<D, FORM>(Gf, sink); }, st, tmap);
}

// The element's coefficient: one value (per-element coefficient) or the
// d+1 vertex values of a P1 coefficient (gathered like the coordinates).
template <int NW>
struct Coef {
  float v[NW];
};

template <int D, int FORM>
__device__ __forceinline__ void load_coef(const float* coef, int64_t e, int64_t n_elem, int64_t n_vert,
                                          const int (&vid)[D + 1], Coef<FormTraits<D, FORM>::NW>& w) {
  if constexpr (FormTraits<D, FORM>::W1) {
#pragma unroll
    for (int k = 0; k <= D; ++k)
      w.v[k] = (coef && e < n_elem && uint32_t(vid[k]) < uint32_t(n_vert)) ? __ldg(coef + vid[k]) : 1.f;
  } else {
    w.v[0] = (coef && e < n_elem) ? __ldg(coef + e) : 1.f;
  }
}

// Stage 3 for one tile: geometry, contraction, staging and the coalesced store
// (TMA: the tensor store of the stage through tmap).
template <int D, int FORM, int JAC, class CT, class OT, bool TMA = false>
__device__ __forceinline__ int fwd_compute_tile(const FwdParams<CT, OT>& p, int64_t tile, int lane, int flags,
                                                const Coef<FormTraits<D, FORM>::NW>& w, const CT (&X)[D + 1][D],
                                                OT* st, const CUtensorMap* tmap = nullptr) {
  using FT = FormTraits<D, FORM>;
  using PL = FwdPlan<D, FORM, CT, OT>;
  using GT = typename std::conditional<JAC == JAC_F64, double, float>::type;
  constexpr int NN = FT::NN;
  constexpr int SST = PL::SST;
  int err = 0;
  OT Gf[FT::NG];
#pragma unroll
  for (int g = 0; g < FT::NG; ++g) Gf[g] = OT(0);
  if (flags & GF_OK) {
    Jac<D, GT> jac;
    const bool nondeg = jacobian<D, JAC>(X, jac);
    err |= nondeg ? 0 : DEVERR_DEGENERATE;
    if (p.det_out) __stcs(p.det_out + tile * 32 + lane, float(jac.det));
    const float w0 = FT::W1 ? 1.f : w.v[0];  // a P1 coefficient multiplies the slots below
    GT scale;  // zero for a degenerate element: its matrix is written as zeros
    if constexpr (sizeof(GT) == 4)
      scale = nondeg ? __fdividef(w0, dev_abs(jac.det) * float(FT::DEN)) : 0.f;
    else
      scale = nondeg ? GT(w0) / (dev_abs(jac.det) * GT(FT::DEN)) : GT(0);
    GT Gt[FT::NGB];
    geometric_tensor<D, FT::BASE>(jac.adj, scale, Gt);
#pragma unroll
    for (int k = 0; k < FT::NW; ++k)
#pragma unroll
      for (int g = 0; g < FT::NGB; ++g) Gf[k * FT::NGB + g] = OT(FT::W1 ? GT(w.v[k]) * Gt[g] : Gt[g]);
  } else if (flags & GF_ELEM) {
    err |= DEVERR_CONN;
    if (p.det_out) __stcs(p.det_out + tile * 32 + lane, 0.f);
  }
  fwd_contract_store<D, FORM, CT, OT, TMA>(p, tile, lane, Gf, st, tmap);
  return err;
}

template <int D, int FORM, int JAC, class CT, class OT>
__device__ __forceinline__ int fwd_compute_tile(const FwdParams<CT, OT>& p, int64_t tile, int lane, int flags,
                                                float w, const CT (&X)[D + 1][D], OT* st) {
  static_assert(FormTraits<D, FORM>::NW == 1, "one coefficient value per element");
  return fwd_compute_tile<D, FORM, JAC, CT, OT>(p, tile, lane, flags, Coef<1>{{w}}, X, st);
}

// One pipeline step: issue the loads of tiles t + 2S (connectivity) and t + S
// (coordinates, coefficient), then compute and store tile t.  The kernel
// calls it with the register buffers swapped on alternate steps, so the
// pipeline rotates without register copies.
template <int D, int FORM, int JAC, class CT, class OT, bool TMA>
__device__ __forceinline__ void fwd_step(const FwdParams<CT, OT>& p, int64_t t, int64_t S, int lane,
                                         const int (&vnext)[D + 1], int (&vload)[D + 1],
                                         const CT (&Xcur)[D + 1][D], CT (&Xnext)[D + 1][D], int fcur,
                                         const Coef<FormTraits<D, FORM>::NW>& wcur, int& fnext,
                                         Coef<FormTraits<D, FORM>::NW>& wnext, OT* st, const CUtensorMap* tmap,
                                         int& err) {
  const int64_t en = (t + S) * 32 + lane;
  load_conn<D>(p.conn, (t + 2 * S) * 32 + lane, p.n_elem, p.vec_conn, vload);
  fnext = gather_regs<D>(p.coords, p.n_vert, en, p.n_elem, vnext, Xnext);
  load_coef<D, FORM>(p.coef, en, p.n_elem, p.n_vert, vnext, wnext);
  err |= fwd_compute_tile<D, FORM, JAC, CT, OT, TMA>(p, t, lane, fcur, wcur, Xcur, st, tmap);
}

template <int D, int FORM, int JAC, class CT, class OT, bool TMA>
__global__ void __launch_bounds__(FwdShape<D, FORM, JAC, CT, OT>::threads, FwdShape<D, FORM, JAC, CT, OT>::min_ctas)
    fem_fwd_kernel(FwdParams<CT, OT> p, const __grid_constant__ CUtensorMap tmap) {
  using PL = FwdPlan<D, FORM, CT, OT>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  // TMA: two 1024-byte-aligned stages per warp (the swizzle follows the shared address)
  unsigned char* sbase =
      TMA ? reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023))
          : smem_raw;
  OT* st = reinterpret_cast<OT*>(sbase + size_t(warp) * (TMA ? PL::tma_per_warp : PL::per_warp));
  OT* st2 = TMA ? st + 2048 / sizeof(OT) : st;
  const int64_t ntiles = (p.n_elem + 31) / 32;
  const int64_t S = int64_t(gridDim.x) * nwarps;
  int64_t t = int64_t(blockIdx.x) * nwarps + warp;
  if (t >= ntiles) return;  // warp-uniform
  int err = 0;
  int va[D + 1], vb[D + 1];
  CT Xa[D + 1][D], Xb[D + 1][D];
  int fa, fb;
  Coef<FormTraits<D, FORM>::NW> wa, wb;
  // prologue: tile t gathered, tile t + S connectivity in flight
  load_conn<D>(p.conn, t * 32 + lane, p.n_elem, p.vec_conn, va);
  fa = gather_regs<D>(p.coords, p.n_vert, t * 32 + lane, p.n_elem, va, Xa);
  load_coef<D, FORM>(p.coef, t * 32 + lane, p.n_elem, p.n_vert, va, wa);
  load_conn<D>(p.conn, (t + S) * 32 + lane, p.n_elem, p.vec_conn, va);
  for (;;) {
    fwd_step<D, FORM, JAC, CT, OT, TMA>(p, t, S, lane, va, vb, Xa, Xb, fa, wa, fb, wb, st, &tmap, err);
    if ((t += S) >= ntiles) break;
    fwd_step<D, FORM, JAC, CT, OT, TMA>(p, t, S, lane, vb, va, Xb, Xa, fb, wb, fa, wa, st2, &tmap, err);
    if ((t += S) >= ntiles) break;
  }
  if constexpr (TMA) {
    if (lane == 0) bulk_wait<0>();  // the stages outlive every tensor store that reads them
  }
  err = __reduce_or_sync(0xffffffffu, err);
  if (err && lane == 0 && p.dev_err) atomicOr(p.dev_err, err);
}

template <int D, int FORM, int JAC, class CT, class OT>
cudaError_t launch_fwd_t(const FwdLaunch& L) {
  using PL = FwdPlan<D, FORM, CT, OT>;
  FwdParams<CT, OT> p;
  p.conn = L.conn;
  p.coords = static_cast<const CT*>(L.coords);
  p.coef = L.coef;
  p.A = static_cast<OT*>(L.A);
  p.n_elem = L.n_elem;
  p.n_vert = L.n_vert;
  p.dev_err = L.dev_err;
  p.vec_conn = (D == 3) && (reinterpret_cast<uintptr_t>(L.conn) % 16 == 0);
  p.vec_store = (reinterpret_cast<uintptr_t>(L.A) % 16 == 0);
  p.det_out = L.det_out;
  CUtensorMap tmap{};
  bool tma = false;
  auto kern = fem_fwd_kernel<D, FORM, JAC, CT, OT, false>;
  if constexpr (PL::SWZ16) {
    if (encode_rows16_map(&tmap, L.A, L.n_elem)) {
      tma = true;
      kern = fem_fwd_kernel<D, FORM, JAC, CT, OT, true>;
    }
  }
  using SH = FwdShape<D, FORM, JAC, CT, OT>;
  const size_t per_warp = tma ? PL::tma_per_warp : PL::per_warp;
  const int want = L.warps > 0 ? L.warps : SH::default_warps;
  const int warps = clamp_warps(want < SH::threads / 32 ? want : SH::threads / 32, per_warp);
  const size_t smem = size_t(warps) * per_warp + (tma ? 1024 : 0);
  cudaError_t st = ensure_smem(reinterpret_cast<const void*>(kern), smem);
  if (st != cudaSuccess) return st;
  const unsigned grid = pipeline_grid(reinterpret_cast<const void*>(kern), warps, smem, L.n_elem, L.ctas_per_sm);
  kern<<<grid, warps * 32, smem, L.stream>>>(p, tmap);
  return cudaGetLastError();
}

// Dispatch one (D, FORM) over the precision combinations the ABI accepts.
template <int D, int FORM>
cudaError_t launch_fwd_form(const FwdLaunch& L) {
  if (!L.coord_f64) {
    if (!L.out_f64) {
      switch (L.jac) {
        case JAC_COMP: return launch_fwd_t<D, FORM, JAC_COMP, float, float>(L);
        case JAC_F64: return launch_fwd_t<D, FORM, JAC_F64, float, float>(L);
        case JAC_F32: return launch_fwd_t<D, FORM, JAC_F32, float, float>(L);
        default: return cudaErrorInvalidValue;
      }
    }
    return launch_fwd_t<D, FORM, JAC_F64, float, double>(L);
  }
  if (!L.out_f64) return launch_fwd_t<D, FORM, JAC_F64, double, float>(L);
  return launch_fwd_t<D, FORM, JAC_F64, double, double>(L);
}

}  // namespace fem
