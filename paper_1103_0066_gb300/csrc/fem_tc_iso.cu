// fem_tc_iso.cu -- the tensor-core contraction (fem_tc.cuh) for the P2
// Laplacian on non-affine elements (Eqs. 16-19).  G^{(k mu),(l nu)} of the
// curved element (78 folded slots on tets, 21 on triangles) is split into
// three BF16 terms; K^{ij}_{(k mu),(l nu)} * DEN is exact in BF16 (at most
// 768 = 3 * 2^8 in magnitude).  The contraction is 59% dense on tets (2538
// of 78 x 55 products), the shape the tensor cores serve.
#include <algorithm>

#include "fem_iso.cuh"
#include "fem_tc.cuh"

namespace fem {

static_assert(tc_b_exact<3, LAPLACE_P2_ISO>() && tc_b_exact<2, LAPLACE_P2_ISO>(), "K' * DEN must be exact in BF16");
__device__ const TcBImage<3, LAPLACE_P2_ISO> kTcB3iso = make_tc_b_image<3, LAPLACE_P2_ISO>();
__device__ const TcBImage<2, LAPLACE_P2_ISO> kTcB2iso = make_tc_b_image<2, LAPLACE_P2_ISO>();

struct TcKRefIso {
  template <int D, int FORM>
  __device__ __forceinline__ static const TcBImage<D, FORM>* b_image() {
    if constexpr (D == 3) {
      return &kTcB3iso;
    } else {
      return &kTcB2iso;
    }
  }
};

// G of a curved element: w |J(centroid)| J^{-1}_{mu a,k} J^{-1}_{nu a,l} / DEN over
// the folded slot pairs (Eq. 18), each entry as the FP32 kernel forms it.
struct TcGeoIso {
  template <int D, int FORM>
  __device__ __forceinline__ static int tile_g(const FwdParams<float, float>&, const float* mid, int64_t e,
                                               const float (&X)[D + 1][D], float w,
                                               float (&G)[FormTraits<D, FORM>::NG]) {
    constexpr int NE = D * (D + 1) / 2, NP = FormTraits<D, FORM>::NP;
    float ji[D + 1][D][D], scale;
    if (!iso_geometry<D, FORM>(X, mid + e * (NE * D), w, ji, scale)) return DEVERR_DEGENERATE;  // G stays 0
#pragma unroll
    for (int pp = 0; pp < NP; ++pp)
#pragma unroll
      for (int qq = pp; qq < NP; ++qq) {
        float s = 0.f;
#pragma unroll
        for (int al = 0; al < D; ++al) s = fmaf(ji[pp / D][pp % D][al], ji[qq / D][qq % D][al], s);
        G[pair_index(pp, qq, NP)] = scale * s;
      }
    return 0;
  }
};

// ------------------------------------------------------------------ curved tetrahedra: two threads per element
// The geometry of a curved tetrahedron (four vertex Jacobians and their
// inverses, 78 G entries and their bf16 split) is most of the work of its
// tensor-core contraction, and at over 200 registers a thread the kernel above
// runs two 4-warp CTAs per SM, too few warps to hide that work's latency.
// This kernel gives each element two threads, m and m + 128 of a 256-thread
// CTA.  Half h forms the Jacobians at vertices 2h and 2h + 1 (Eq. 16) and
// swaps them with its partner through shared memory; both then form the four
// inverses (Eq. 17), |J| at the centroid and the scale, and half h forms G
// entries [40h, 40h + 40) and writes their three bf16 terms into the A tile.
// Each G entry is formed by the same operations as in the kernel above, so
// the results are the same bits.  The B operand, the MMA and the accumulator
// are the same; in the epilogue warp w reads the accumulator lanes of its
// quarter (w mod 4) and stores boxes 2h and 2h + 1 of those rows.
namespace {

using IsoTP = TcPlan<3, LAPLACE_P2_ISO>;
constexpr int kPairThreads = 2 * kTileElems;
constexpr int kPairGH = 40;  // G entries per half (78 real, padded to 80)
constexpr int kPairXs = 19;  // exchange row stride in floats (odd: no bank conflicts)
static_assert(IsoTP::KT == 2 * kPairGH && IsoTP::N == 64 && IsoTP::BOXES == 4, "curved tetrahedron tile shape");
constexpr size_t kPairRegion = size_t(4) * IsoTP::BOXES * 4096 > align_up(IsoTP::a_bytes, 1024)
                                   ? size_t(4) * IsoTP::BOXES * 4096
                                   : align_up(IsoTP::a_bytes, 1024);
constexpr size_t kPairXch = size_t(2) * kTileElems * kPairXs * 4;
constexpr size_t kPairSmem = IsoTP::b_region + kPairRegion + kPairXch + 128 + 1024;

// (pp, qq) of folded G entry g: the inverse of pair_index over NP = 12.
constexpr int pair_pp(int g) {
  int pp = 0;
  while (g >= 12 - pp) {
    g -= 12 - pp;
    ++pp;
  }
  return pp;
}
constexpr int pair_qq(int g) { return pair_pp(g) + (g - pair_index(pair_pp(g), pair_pp(g), 12)); }

// Barrier 1 + q among warps q and q + 4 (the two halves of rows 32q .. 32q + 31);
// immediate ids, so that the kernel declares five barriers, not sixteen.
__device__ __forceinline__ void pair_bar(int id) {
  switch (id) {
    case 1: asm volatile("bar.sync 1, 64;\n" ::: "memory"); break;
    case 2: asm volatile("bar.sync 2, 64;\n" ::: "memory"); break;
    case 3: asm volatile("bar.sync 3, 64;\n" ::: "memory"); break;
    default: asm volatile("bar.sync 4, 64;\n" ::: "memory"); break;
  }
}

// Half H's Jacobians (vertices 2H, 2H + 1), the swap with the partner, then
// all four inverses and the scale, as iso_geometry forms them.
template <int H>
__device__ __forceinline__ bool pair_geometry(const float (&X)[4][3], const float (&M)[6][3], float w, float* mine,
                                              const float* other, int bar_id, float (&ji)[4][3][3],
                                              float& scale) {
  float nd[10][3];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int al = 0; al < 3; ++al) nd[a][al] = X[a][al] - X[0][al];
#pragma unroll
  for (int q = 0; q < 6; ++q)
#pragma unroll
    for (int al = 0; al < 3; ++al) nd[4 + q][al] = M[q][al] - X[0][al];
  float e[4][3][3];
  geo_jacobian<3, 2 * H>(nd, e[2 * H]);
  geo_jacobian<3, 2 * H + 1>(nd, e[2 * H + 1]);
#pragma unroll
  for (int k = 0; k < 2; ++k)
#pragma unroll
    for (int i = 0; i < 9; ++i) mine[9 * k + i] = e[2 * H + k][i / 3][i % 3];
  pair_bar(bar_id);
#pragma unroll
  for (int k = 0; k < 2; ++k)
#pragma unroll
    for (int i = 0; i < 9; ++i) e[2 * (1 - H) + k][i / 3][i % 3] = other[9 * k + i];
  float ec[3][3];
  bool ok = true;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
#pragma unroll
    for (int mu = 0; mu < 3; ++mu)
#pragma unroll
      for (int al = 0; al < 3; ++al) ec[mu][al] = k == 0 ? e[0][mu][al] : ec[mu][al] + e[k][mu][al];
    float adj[3][3];
    const float det = det_adj<3>(e[k], adj);
    const float r = __frcp_rn(det);
#pragma unroll
    for (int mu = 0; mu < 3; ++mu)
#pragma unroll
      for (int al = 0; al < 3; ++al) ji[k][mu][al] = adj[mu][al] * r;
    ok &= det != 0.f;
  }
  float adjc[3][3];
  float detc = det_adj<3>(ec, adjc);
  detc *= 1.f / 64.f;  // det scales by (D + 1)^D
  ok &= detc != 0.f;
  scale = w * fabsf(detc) * (1.f / float(FormTraits<3, LAPLACE_P2_ISO>::DEN));
  return ok;
}

// G entry GI of the element (zero past the 78 entries or for a flagged element).
template <int GI>
__device__ __forceinline__ float pair_g(const float (&ji)[4][3][3], float scale, bool live) {
  if constexpr (GI < FormTraits<3, LAPLACE_P2_ISO>::NG) {
    constexpr int pp = pair_pp(GI), qq = pair_qq(GI);
    float s = 0.f;
#pragma unroll
    for (int al = 0; al < 3; ++al) s = fmaf(ji[pp / 3][pp % 3][al], ji[qq / 3][qq % 3][al], s);
    return live ? scale * s : 0.f;
  } else {
    return 0.f;
  }
}

// Chunk J of half H: G entries 40H + 8J .. 40H + 8J + 7, split into three
// bf16 terms, one 16-byte chunk of each term into row m of the A tile.
template <int H, int J, int... Us>
__device__ __forceinline__ void pair_chunk(unsigned char* sa, uint32_t rowoff, const float (&ji)[4][3][3],
                                           float scale, bool live, std::integer_sequence<int, Us...>) {
  const float g[8] = {pair_g<H * kPairGH + 8 * J + Us>(ji, scale, live)...};
  uint32_t w[3][4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float x0 = g[2 * q], x1 = g[2 * q + 1];
    const __nv_bfloat162 h0 = __floats2bfloat162_rn(x0, x1);
    const float r0 = x0 - __low2float(h0), r1 = x1 - __high2float(h0);
    const __nv_bfloat162 h1 = __floats2bfloat162_rn(r0, r1);
    const float s0 = r0 - __low2float(h1), s1 = r1 - __high2float(h1);
    const __nv_bfloat162 h2 = __floats2bfloat162_rn(s0, s1);
    w[0][q] = *reinterpret_cast<const uint32_t*>(&h0);
    w[1][q] = *reinterpret_cast<const uint32_t*>(&h1);
    w[2][q] = *reinterpret_cast<const uint32_t*>(&h2);
  }
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    const int kc = t * (IsoTP::KT / 8) + H * (kPairGH / 8) + J;
    *reinterpret_cast<uint4*>(sa + uint32_t(kc) * IsoTP::A_LBO + rowoff) =
        make_uint4(w[t][0], w[t][1], w[t][2], w[t][3]);
  }
}

// Half H's G entries into row m of the A tile, eight at a time.
template <int H, int... Js>
__device__ __forceinline__ void pair_store_a(unsigned char* sa, int m, const float (&ji)[4][3][3], float scale,
                                             bool live, std::integer_sequence<int, Js...>) {
  const uint32_t rowoff = uint32_t(m / 8) * 128u + uint32_t(m % 8) * 16u;
  (pair_chunk<H, Js>(sa, rowoff, ji, scale, live, std::make_integer_sequence<int, 8>{}), ...);
}

// Boxes 2H and 2H + 1 of this warp's 32 rows: accumulator lanes -> registers
// -> swizzled stage -> two tensor stores (lane 0), left in flight.
template <int H>
__device__ __forceinline__ void pair_epilogue(uint32_t tl, unsigned char* wst, int lane, const CUtensorMap* tmap,
                                              int64_t e0, bool live) {
  float r[IsoTP::N];
  tc_load_all<IsoTP::N>(tl, r, std::make_integer_sequence<int, IsoTP::N / 16>{});
  tc_stage_rows<10, IsoTP::NT, 2 * H, 2>(r, wst + lane * 128, lane & 7, std::make_integer_sequence<int, 25>{});
  fence_proxy_async_smem();
  __syncwarp();
  if (lane == 0 && live) {
#pragma unroll
    for (int b = 0; b < 2; ++b) tma_store_2d(tmap, 32 * (2 * H + b), int(e0), smem_u32(wst + b * 4096));
    bulk_commit();
  }
}

__global__ void __launch_bounds__(kPairThreads, 2)
    fem_fwd_tc_iso_pair_kernel(FwdParams<float, float> p, const float* mid, const __grid_constant__ CUtensorMap tmap) {
  extern __shared__ __align__(128) unsigned char smem_raw_tc[];
  unsigned char* smem_raw = smem_raw_tc + ((1024u - (smem_u32(smem_raw_tc) & 1023u)) & 1023u);
  unsigned char* sb = smem_raw;                          // B operand
  unsigned char* region = smem_raw + IsoTP::b_region;    // A tile, then output stages
  float* xch = reinterpret_cast<float*>(region + kPairRegion);  // [2][128][kPairXs]
  unsigned char* tail = region + kPairRegion + kPairXch;
  uint64_t* mbar_ptr = reinterpret_cast<uint64_t*>(tail);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tail + 16);
  int* abort_flag = reinterpret_cast<int*>(tail + 32);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int h = tid >> 7, m = tid & (kTileElems - 1), wq = warp & 3;
  const uint32_t mbar = smem_u32(mbar_ptr);
  const int64_t nct = (p.n_elem + kTileElems - 1) / kTileElems;
  if (int64_t(blockIdx.x) >= nct) return;  // CTA-uniform, before any TMEM allocation

  tc_fill_b<3, LAPLACE_P2_ISO, TcKRefIso>(sb);
  if (tid == 0) {
    mbar_init(mbar);
    *abort_flag = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                 "n"(IsoTP::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  constexpr uint32_t idesc = idesc_bf16_f32<IsoTP::M, IsoTP::N>();
  int err = 0;
  uint32_t phase = 0;
  float* xmine = xch + (h * kTileElems + m) * kPairXs;
  const float* xother = xch + ((1 - h) * kTileElems + m) * kPairXs;

  int v[4];
  float Xc[4][3], Mc[6][3];
  int64_t T = blockIdx.x;
  const int vec_conn = reinterpret_cast<uintptr_t>(p.conn) % 16 == 0;
  auto load_mid = [&](int64_t e, float (&M)[6][3]) {
    if (e < p.n_elem) {
#pragma unroll
      for (int q = 0; q < 6; ++q)
#pragma unroll
        for (int al = 0; al < 3; ++al) M[q][al] = __ldcs(mid + e * 18 + q * 3 + al);
    }
  };
  load_conn<3>(p.conn, T * kTileElems + m, p.n_elem, vec_conn, v);
  int fcur = gather_regs<3>(p.coords, p.n_vert, T * kTileElems + m, p.n_elem, v, Xc);
  load_mid(T * kTileElems + m, Mc);
  float wcur = (p.coef && T * kTileElems + m < p.n_elem) ? __ldg(p.coef + T * kTileElems + m) : 1.f;
  int vn[4];
  load_conn<3>(p.conn, (T + gridDim.x) * kTileElems + m, p.n_elem, vec_conn, vn);
  for (; T < nct; T += gridDim.x) {
    const int64_t en = (T + gridDim.x) * kTileElems + m;
    int vnn[4];
    load_conn<3>(p.conn, en + int64_t(gridDim.x) * kTileElems, p.n_elem, vec_conn, vnn);
    float Xn[4][3], Mn[6][3];
    const int fnext = gather_regs<3>(p.coords, p.n_vert, en, p.n_elem, vn, Xn);
    load_mid(en, Mn);
    const float wnext = (p.coef && en < p.n_elem) ? __ldg(p.coef + en) : 1.f;
    // geometry of this pair's element (both halves take part in the swap)
    float ji[4][3][3], scale;
    const bool gok = h == 0 ? pair_geometry<0>(Xc, Mc, wcur, xmine, xother, 1 + wq, ji, scale)
                            : pair_geometry<1>(Xc, Mc, wcur, xmine, xother, 1 + wq, ji, scale);
    const bool live = (fcur & GF_OK) && gok;
    if (h == 0) {
      if (fcur & GF_OK) {
        if (!gok) err |= DEVERR_DEGENERATE;
      } else if (fcur & GF_ELEM) {
        err |= DEVERR_CONN;
      }
    }
    // the previous tile's tensor stores have read the stage (aliasing A)
    if (lane == 0) bulk_wait_read<0>();
    __syncthreads();
    if (h == 0)
      pair_store_a<0>(region, m, ji, scale, live, std::make_integer_sequence<int, kPairGH / 8>{});
    else
      pair_store_a<1>(region, m, ji, scale, live, std::make_integer_sequence<int, kPairGH / 8>{});
    fence_proxy_async_smem();  // generic-proxy writes of A -> tensor-core reads
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t sa = smem_u32(region), sbb = smem_u32(sb);
#pragma unroll
      for (int s = 0; s < IsoTP::KSTEPS; ++s) {
        const uint64_t ad = smem_desc(sa + uint32_t(2 * s) * IsoTP::A_LBO, IsoTP::A_LBO, IsoTP::A_SBO);
        const uint64_t bd =
            smem_desc(sbb + uint32_t(2 * (s % (IsoTP::KT / 16))) * IsoTP::B_LBO, IsoTP::B_LBO, IsoTP::B_SBO);
        mma_bf16(tmem, ad, bd, idesc, s > 0 ? 1u : 0u);
      }
      mma_commit(mbar);
      if (!mbar_wait(mbar, phase)) *abort_flag = 1;
    }
    __syncthreads();
    if (*abort_flag) {  // `phase` is still the pending one: teardown waits on it
      err |= DEVERR_TIMEOUT;
      break;
    }
    phase ^= 1u;
    tc_fence_after();
    const int64_t e0 = T * kTileElems + wq * 32;
    unsigned char* wst = region + size_t(wq * 4 + 2 * h) * 4096;
    if (h == 0)
      pair_epilogue<0>(tmem + (uint32_t(wq * 32) << 16), wst, lane, &tmap, e0, e0 < p.n_elem);
    else
      pair_epilogue<1>(tmem + (uint32_t(wq * 32) << 16), wst, lane, &tmap, e0, e0 < p.n_elem);
    __syncwarp();
    fcur = fnext;
    wcur = wnext;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      v[k] = vn[k];
      vn[k] = vnn[k];
#pragma unroll
      for (int a = 0; a < 3; ++a) Xc[k][a] = Xn[k][a];
    }
#pragma unroll
    for (int q = 0; q < 6; ++q)
#pragma unroll
      for (int a = 0; a < 3; ++a) Mc[q][a] = Mn[q][a];
  }
  if (lane == 0) bulk_wait<0>();  // this warp's tensor stores are complete
  if (*abort_flag && tid == 0) mbar_wait(mbar, phase);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "n"(IsoTP::TMEM_COLS)
                 : "memory");
  }
  err = __reduce_or_sync(0xffffffffu, err);
  if (err && lane == 0 && p.dev_err) atomicOr(p.dev_err, err);
}

cudaError_t launch_iso_pair(const FwdLaunch& L, const float* mid, bool* launched) {
  *launched = false;
  CUtensorMap tmap{};
  if (!encode_tc_rows_map(&tmap, L.A, L.n_elem, IsoTP::FT::NN)) return cudaSuccess;
  FwdParams<float, float> p;
  p.conn = L.conn;
  p.coords = static_cast<const float*>(L.coords);
  p.coef = L.coef;
  p.A = static_cast<float*>(L.A);
  p.n_elem = L.n_elem;
  p.n_vert = L.n_vert;
  p.dev_err = L.dev_err;
  p.vec_conn = 0;
  p.vec_store = 0;
  auto kern = fem_fwd_tc_iso_pair_kernel;
  cudaError_t st = ensure_smem(reinterpret_cast<const void*>(kern), kPairSmem);
  if (st != cudaSuccess) return st;
  // CTAs per SM from the registers and the shared memory (at most two: the
  // kernel's register bound)
  cudaFuncAttributes fa{};
  int dev = 0, regs = 0, shm = 0, rsv = 0;
  int occ = 1;
  if (cudaFuncGetAttributes(&fa, kern) == cudaSuccess && cudaGetDevice(&dev) == cudaSuccess &&
      cudaDeviceGetAttribute(&regs, cudaDevAttrMaxRegistersPerMultiprocessor, dev) == cudaSuccess &&
      cudaDeviceGetAttribute(&shm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) == cudaSuccess &&
      cudaDeviceGetAttribute(&rsv, cudaDevAttrReservedSharedMemoryPerBlock, dev) == cudaSuccess) {
    const int by_regs = regs / (((fa.numRegs + 7) / 8 * 8) * kPairThreads);
    const int by_smem = int(size_t(shm) / (kPairSmem + fa.sharedSizeBytes + size_t(rsv)));
    occ = std::max(1, std::min(std::min(by_regs, by_smem), 2));
  } else {
    cudaGetLastError();
  }
  const int per_sm = L.ctas_per_sm > 0 ? L.ctas_per_sm : occ;
  const int64_t nct = (L.n_elem + kTileElems - 1) / kTileElems;
  int64_t grid = int64_t(per_sm) * device_sm_count();
  if (grid > nct) grid = nct;
  kern<<<unsigned(grid < 1 ? 1 : grid), kPairThreads, kPairSmem, L.stream>>>(p, mid, tmap);
  *launched = true;
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_fwd_iso_tc(const FwdLaunch& L, const float* mid) {
  if (L.form != LAPLACE_P2_ISO) return cudaErrorInvalidValue;
  if (L.dim == 3) {
    if (L.n_elem > 0) {  // two threads per element, when the output takes a tensor map
      bool launched = false;
      const cudaError_t e = launch_iso_pair(L, mid, &launched);
      if (e != cudaSuccess || launched) return e;
    }
    return launch_tc_t<3, LAPLACE_P2_ISO, TcGeoIso, TcKRefIso>(L, mid);
  }
  return launch_tc_t<2, LAPLACE_P2_ISO, TcGeoIso, TcKRefIso>(L, mid);
}

}  // namespace fem
