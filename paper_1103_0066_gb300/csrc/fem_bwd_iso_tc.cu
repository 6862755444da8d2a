// fem_bwd_iso_tc.cu -- the adjoint of the curved P2 Laplacian on tetrahedra
// (Eqs. 16-19) with its contraction adjoint on the tcgen05 tensor cores.
//
// The adjoint's first step is s_g = sum_T K'[g][T] sym(dA)_T for the 78 folded
// slot pairs g of an element (2538 FMAs per element on the CUDA cores, most of
// the FP32 kernel's arithmetic): over a tile of 128 elements it is the GEMM
// S[128 x 78] = sym(dA)[128 x 55] K'^T[55 x 78].  K' * DEN is exact in BF16
// (the forward's static_assert covers the same entries), and sym(dA) is split
// into three BF16 terms (hi, mid, lo: their sum is sym(dA) to FP32's unit
// roundoff), so the three MMAs per K step reproduce the FP32 contraction up
// to the order of its additions.  A CTA of four warps, one 32-element record
// tile each:
//   1. each lane stages its element's sym(dA) as three BF16 terms into the A
//      tile (over the warps' dA slots, once every warp has read its rows);
//   2. thread 0 issues the 12 MMAs (M 128, N 80, K 192) into a TMEM
//      accumulator; meanwhile every lane forms its element's geometry;
//   3. each lane reads its s_g from TMEM, 16 at a time, and runs the FP32
//      kernel's remaining steps (fem_iso_adj.cuh): the pair terms, the
//      centroid, the pullback to the nodes, then the tile records, the
//      edge-node and the coefficient gradients.
// Every wait is bounded (FEM_DEVERR_TIMEOUT; TMEM freed after a bounded wait
// for the MMAs).
#include "fem_iso_adj.cuh"
#include "fem_tc.cuh"

namespace fem {

namespace {

using FTi = FormTraits<3, LAPLACE_P2_ISO>;
using PLi = BwdPlan<3, LAPLACE_P2_ISO>;
constexpr int kAdjKT = 64;                                    // sym(dA) entries (55), padded
constexpr int kAdjN = 80;                                     // slot pairs (78), padded
constexpr int kAdjK = 3 * kAdjKT;                             // three BF16 terms
constexpr int kAdjKSteps = kAdjK / 16;
constexpr uint32_t kAdjALBO = (kTileElems / 8) * 128, kAdjASBO = 128;
constexpr uint32_t kAdjBLBO = (kAdjN / 8) * 128, kAdjBSBO = 128;
constexpr size_t kAdjABytes = size_t(kTileElems) * kAdjK * 2;
constexpr size_t kAdjBBytes = size_t(kAdjN) * kAdjKT * 2;
constexpr int kAdjTmemCols = 128;
constexpr int kAdjWarps = kTileElems / 32;
constexpr size_t kAdjSlots = size_t(kAdjWarps) * PLi::da_slot;          // dA slots; the A tile over them
constexpr size_t kAdjMs = align_up(size_t(32) * 18 * 4, 128);           // a tile's edge nodes
constexpr size_t kAdjPerWarp = PLi::xs_bytes + 2 * kAdjMs;              // slot stage, two edge-node stages
constexpr size_t kAdjSmem = kAdjSlots + kAdjBBytes + kAdjWarps * kAdjPerWarp + 128;
static_assert(FTi::NT <= kAdjKT && FTi::NG <= kAdjN && kAdjABytes <= kAdjSlots, "curved P2 adjoint tile");

// B = K'^T in the no-swizzle K-major core-matrix layout: element (k = T, n = g).
struct alignas(16) AdjBImage {
  uint16_t v[kAdjN * kAdjKT];
};

constexpr AdjBImage make_adj_b_image() {
  const RefTensor<3, LAPLACE_P2_ISO> kt = make_ref_tensor<3, LAPLACE_P2_ISO>();
  AdjBImage im{};
  for (int n = 0; n < kAdjN; ++n)
    for (int k = 0; k < kAdjKT; ++k) {
      const int val = (n < FTi::NG && k < FTi::NT) ? kt.v[n][tri_row(k, FTi::N)][tri_col(k, FTi::N)] : 0;
      im.v[((k / 8) * (kAdjN / 8) + n / 8) * 64 + (n % 8) * 8 + k % 8] = uint16_t(bf16_of_int(val));
    }
  return im;
}

constexpr bool adj_b_exact() {
  const RefTensor<3, LAPLACE_P2_ISO> kt = make_ref_tensor<3, LAPLACE_P2_ISO>();
  for (int n = 0; n < FTi::NG; ++n)
    for (int k = 0; k < FTi::NT; ++k)
      if (bf16_of_int(kt.v[n][tri_row(k, FTi::N)][tri_col(k, FTi::N)]) > 0xFFFFu) return false;
  return true;
}
static_assert(adj_b_exact(), "K' * DEN must be exact in BF16");
__device__ const AdjBImage kAdjB = make_adj_b_image();

// Row m of the A tile: sym(dA) (zero padded to 64) as three BF16 terms, one
// 16-byte chunk (8 entries of one term) at a time.
template <int C>
__device__ __forceinline__ void adj_store_chunk(unsigned char* sa, uint32_t rowoff, const SymVals<FTi::NT>& sym) {
  float x[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) x[u] = 8 * C + u < FTi::NT ? sym.s[8 * C + u] : 0.f;
  uint32_t w[3][4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const __nv_bfloat162 h0 = __floats2bfloat162_rn(x[2 * q], x[2 * q + 1]);
    const float r0 = x[2 * q] - __low2float(h0), r1 = x[2 * q + 1] - __high2float(h0);
    const __nv_bfloat162 h1 = __floats2bfloat162_rn(r0, r1);
    const float s0 = r0 - __low2float(h1), s1 = r1 - __high2float(h1);
    const __nv_bfloat162 h2 = __floats2bfloat162_rn(s0, s1);
    w[0][q] = *reinterpret_cast<const uint32_t*>(&h0);
    w[1][q] = *reinterpret_cast<const uint32_t*>(&h1);
    w[2][q] = *reinterpret_cast<const uint32_t*>(&h2);
  }
#pragma unroll
  for (int t = 0; t < 3; ++t)
    *reinterpret_cast<uint4*>(sa + uint32_t(t * (kAdjKT / 8) + C) * kAdjALBO + rowoff) =
        make_uint4(w[t][0], w[t][1], w[t][2], w[t][3]);
}

template <int... Cs>
__device__ __forceinline__ void adj_store_row(unsigned char* sa, int m, const SymVals<FTi::NT>& sym,
                                              std::integer_sequence<int, Cs...>) {
  const uint32_t rowoff = uint32_t(m / 8) * 128u + uint32_t(m % 8) * 16u;
  (adj_store_chunk<Cs>(sa, rowoff, sym), ...);
}

// The slot-pair terms of TMEM columns 16C .. 16C + 15 (every lane loads; the
// terms apply where the element is valid).
template <int C, int... Us>
__device__ __forceinline__ void adj_chunk_terms(uint32_t tl, bool ok, const float (&ji)[4][3][3], float sc,
                                                float (&dji)[4][3][3], float& dsc, std::integer_sequence<int, Us...>) {
  float r[16];
  tmem_ld16(tl + uint32_t(16 * C), r);
  tmem_ld_wait();
  if (ok)
    (
        [&] {
          if constexpr (16 * C + Us < FTi::NG) iso_adj_apply<3, LAPLACE_P2_ISO, 16 * C + Us>(r[Us], ji, sc, dji, dsc);
        }(),
        ...);
}

template <int... Cs>
__device__ __forceinline__ void adj_all_terms(uint32_t tl, bool ok, const float (&ji)[4][3][3], float sc,
                                              float (&dji)[4][3][3], float& dsc, std::integer_sequence<int, Cs...>) {
  (adj_chunk_terms<Cs>(tl, ok, ji, sc, dji, dsc, std::make_integer_sequence<int, 16>{}), ...);
}

__global__ void __launch_bounds__(kTileElems)
    fem_bwd_iso_tc_kernel(BwdParams p, const float* __restrict__ mid, float* __restrict__ dmid) {
  constexpr int NV = 4, NE = 6, NG = n_geo(3);
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  unsigned char* sa = smem_raw;  // the A tile, over the four warps' dA slots
  float* dslot = reinterpret_cast<float*>(smem_raw + size_t(warp) * PLi::da_slot);
  unsigned char* sb = smem_raw + kAdjSlots;
  unsigned char* wx = sb + kAdjBBytes + size_t(warp) * kAdjPerWarp;
  float* xs = reinterpret_cast<float*>(wx);
  float* ms_buf[2] = {reinterpret_cast<float*>(wx + PLi::xs_bytes),
                      reinterpret_cast<float*>(wx + PLi::xs_bytes + kAdjMs)};
  unsigned char* tail = sb + kAdjBBytes + size_t(kAdjWarps) * kAdjPerWarp;
  uint64_t* mbar_ptr = reinterpret_cast<uint64_t*>(tail);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tail + 16);
  int* abort_flag = reinterpret_cast<int*>(tail + 32);
  const uint32_t mbar = smem_u32(mbar_ptr);
  const bool rec = p.tile_rec != nullptr;
  const int64_t ntiles = (p.n_elem + 31) / 32;  // record tiles (one per warp and step)
  const int64_t nct = (p.n_elem + kTileElems - 1) / kTileElems;
  if (int64_t(blockIdx.x) >= nct) return;  // CTA-uniform, before any TMEM allocation

  {  // B once per CTA; mbarrier; TMEM accumulator
    const uint4* src = reinterpret_cast<const uint4*>(kAdjB.v);
    uint4* dst = reinterpret_cast<uint4*>(sb);
    for (int i = tid; i < int(kAdjBBytes / 16); i += blockDim.x) dst[i] = __ldg(src + i);
  }
  if (tid == 0) {
    mbar_init(mbar);
    *abort_flag = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                 "n"(kAdjTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  constexpr uint32_t idesc = idesc_bf16_f32<kTileElems, kAdjN>();
  int err = 0;
  uint32_t phase = 0;

  // A step's inputs: its dA rows and edge nodes (cp.async into this warp's dA
  // slot and an edge-node stage), connectivity, coordinates and record range.
  // The next step's are issued once this step's MMAs have read the A tile (the
  // dA slots), so they arrive while this step's terms and records run.
  struct Ins {
    int v[NV];
    float X[NV][3];
    int flags;
    uint32_t rk;
    int32_t rb, rn;
  };
  auto issue = [&](int64_t TT, float* msd, Ins& in) {
    const int64_t t = TT * kAdjWarps + warp, e = t * 32 + lane;
    const int cnt = int(p.n_elem - t * 32 < 32 ? (p.n_elem - t * 32 > 0 ? p.n_elem - t * 32 : 0) : 32);
    if (TT < nct && cnt > 0) {
      copy_dA_async<3, LAPLACE_P2_ISO>(p, t, lane, dslot);
      tile_load_async(msd, mid + t * 32 * (NE * 3), cnt * (NE * 3), lane);
    }
    cp_async_commit();
    load_conn<3>(p.conn, e, p.n_elem, p.vec_conn, in.v);
    in.flags = gather_regs<3>(p.coords, p.n_vert, e, p.n_elem, in.v, in.X);
    in.rk = 0;
    in.rb = 0;
    in.rn = 0;
    if (rec && TT < nct && t < ntiles) {
      in.rk = __ldg(p.rank + e);  // ntiles * 32 entries: the tail lanes' slots too
      in.rb = __ldg(p.tile_rec + t);
      in.rn = __ldg(p.tile_rec + t + 1) - in.rb;
    }
  };
  Ins cur, nxt;
  int sb_ms = 0;  // the edge-node stage of the current step
  issue(blockIdx.x, ms_buf[0], cur);
  for (int64_t T = blockIdx.x; T < nct; T += gridDim.x) {
    const int64_t t = T * kAdjWarps + warp;  // this warp's record tile
    const int64_t e = t * 32 + lane;
    const int cnt = int(p.n_elem - t * 32 < 32 ? (p.n_elem - t * 32 > 0 ? p.n_elem - t * 32 : 0) : 32);
    float* ms = ms_buf[sb_ms];
    const int flags = cur.flags;
    const int32_t rb = cur.rb, rn = cur.rn;
    const uint32_t rk = cur.rk;
    const RecAhead ah = rec ? load_rec_ahead(p.rec_span, p.rec_dest, rb, rn, lane) : RecAhead{0u, 0};
    cp_async_wait<0>();
    __syncwarp();  // the tile's dA rows and edge nodes were copied by other lanes
    // 1. sym(dA) as three BF16 terms into row tid of the A tile
    {
      SymVals<FTi::NT> sym;
      if (e < p.n_elem) {
        stage_sym<3, LAPLACE_P2_ISO>(dslot + lane * PLi::DST, sym.s);
      } else {
#pragma unroll
        for (int T2 = 0; T2 < FTi::NT; ++T2) sym.s[T2] = 0.f;
      }
      __syncthreads();  // every warp has read its dA rows: the A tile overwrites the slots
      adj_store_row(sa, tid, sym, std::make_integer_sequence<int, kAdjKT / 8>{});
    }
    fence_proxy_async_smem();  // generic-proxy writes of A -> tensor-core reads
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t a0 = smem_u32(sa), b0 = smem_u32(sb);
#pragma unroll
      for (int s = 0; s < kAdjKSteps; ++s) {
        const uint64_t ad = smem_desc(a0 + uint32_t(2 * s) * kAdjALBO, kAdjALBO, kAdjASBO);
        const uint64_t bd = smem_desc(b0 + uint32_t(2 * (s % (kAdjKT / 16))) * kAdjBLBO, kAdjBLBO, kAdjBSBO);
        mma_bf16(tmem, ad, bd, idesc, s > 0 ? 1u : 0u);
      }
      mma_commit(mbar);
    }
    // 2. the element's geometry while the MMAs run (as the forward forms it)
    float xb[NV][3], mb[NE][3];
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
      for (int a = 0; a < 3; ++a) xb[k][a] = 0.f;
#pragma unroll
    for (int q = 0; q < NE; ++q)
#pragma unroll
      for (int a = 0; a < 3; ++a) mb[q][a] = 0.f;
    float dw = 0.f;
    bool ok = false;
    float ji[NV][3][3], adjc[3][3], detc = 0.f, w = 1.f;
    if (flags & GF_OK) {
      w = (p.coef && e < p.n_elem) ? __ldg(p.coef + e) : 1.f;
      float nd[NG][3];
#pragma unroll
      for (int a = 0; a <= 3; ++a)
#pragma unroll
        for (int al = 0; al < 3; ++al) nd[a][al] = cur.X[a][al] - cur.X[0][al];
      const float* me = ms + lane * (NE * 3);
#pragma unroll
      for (int q = 0; q < NE; ++q)
#pragma unroll
        for (int al = 0; al < 3; ++al) nd[4 + q][al] = me[q * 3 + al] - cur.X[0][al];
      float ec[3][3];
      ok = all_vertex_jinv<3>(nd, ji, ec, std::make_integer_sequence<int, NV>{});
      detc = det_adj<3>(ec, adjc) * (1.f / 64.f);
      ok &= detc != 0.f;
      if (!ok) err |= DEVERR_DEGENERATE;
    } else if (flags & GF_ELEM) {
      err |= DEVERR_CONN;
    }
    // wait for the MMAs (thread 0, bounded), then read the accumulator
    if (tid == 0 && !mbar_wait(mbar, phase)) *abort_flag = 1;
    __syncthreads();
    if (*abort_flag) {  // `phase` is still the pending one: teardown waits on it
      err |= DEVERR_TIMEOUT;
      break;
    }
    phase ^= 1u;
    tc_fence_after();
    // the MMAs have read the A tile: the next step's inputs may overwrite the dA slots
    issue(T + gridDim.x, ms_buf[sb_ms ^ 1], nxt);
    // 3. the slot-pair terms with s_g from TMEM, then the FP32 kernel's steps
    {
      const float absdet = fabsf(detc);
      const float sc = w * absdet * (1.f / float(FTi::DEN));
      float dji[NV][3][3];
#pragma unroll
      for (int k = 0; k < NV; ++k)
#pragma unroll
        for (int mu = 0; mu < 3; ++mu)
#pragma unroll
          for (int a = 0; a < 3; ++a) dji[k][mu][a] = 0.f;
      float dsc = 0.f;
      adj_all_terms(tmem + (uint32_t(warp * 32) << 16), ok, ji, sc, dji, dsc,
                    std::make_integer_sequence<int, kAdjN / 16>{});
      if (ok) {
        dw = dsc * absdet * (1.f / float(FTi::DEN));
        const float ddet = (detc > 0.f ? 1.f : -1.f) * dsc * w * (1.f / float(FTi::DEN)) * (1.f / 64.f);
        float dec[3][3];
#pragma unroll
        for (int mu = 0; mu < 3; ++mu)
#pragma unroll
          for (int al = 0; al < 3; ++al) dec[mu][al] = ddet * adjc[mu][al];
        float dnd[NG][3];
#pragma unroll
        for (int a = 0; a < NG; ++a)
#pragma unroll
          for (int al = 0; al < 3; ++al) dnd[a][al] = 0.f;
        all_vertex_pullback<3>(ji, dji, dec, dnd, std::make_integer_sequence<int, NV>{});
#pragma unroll
        for (int al = 0; al < 3; ++al) {
          float s = 0.f;
#pragma unroll
          for (int a = 1; a < NG; ++a) s += dnd[a][al];
          xb[0][al] = -s;
        }
#pragma unroll
        for (int k = 1; k <= 3; ++k)
#pragma unroll
          for (int al = 0; al < 3; ++al) xb[k][al] = dnd[k][al];
#pragma unroll
        for (int q = 0; q < NE; ++q)
#pragma unroll
          for (int al = 0; al < 3; ++al) mb[q][al] = dnd[4 + q][al];
      }
    }
    if ((flags & GF_ELEM) && p.dcoef) __stcs(p.dcoef + e, dw);
    if (rec && cnt > 0) {  // the element's vertex contributions at their stage positions (zeros when skipped)
#pragma unroll
      for (int k = 0; k < NV; ++k)
        *reinterpret_cast<float4*>(xs + ((rk >> (8 * k)) & 0xFFu) * PLi::XP) =
            make_float4(xb[k][0], xb[k][1], xb[k][2], 0.f);
      __syncwarp();  // every lane's contributions are staged
      warp_records<3, PLi::NC>(xs, p.rec_span, p.rec_dest, rb, rn, ah, p.records, lane);
    }
    if (dmid && cnt > 0) {  // the tile's edge-node gradients through the stage, stored coalesced
      __syncwarp();        // every lane has read its edge nodes
#pragma unroll
      for (int q = 0; q < NE; ++q)
#pragma unroll
        for (int al = 0; al < 3; ++al) ms[lane * (NE * 3) + q * 3 + al] = mb[q][al];
      __syncwarp();
      tile_store(dmid + t * 32 * (NE * 3), ms, cnt * (NE * 3), lane);
    }
    __syncwarp();  // the stages are rewritten next step
    cur = nxt;
    sb_ms ^= 1;
  }
  cp_async_wait<0>();
  // teardown: after an abort, give the tensor core a bounded chance to finish first
  if (*abort_flag && tid == 0) mbar_wait(mbar, phase);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "n"(kAdjTmemCols)
                 : "memory");
  }
  err = __reduce_or_sync(0xffffffffu, err);
  if (err && lane == 0 && p.dev_err) atomicOr(p.dev_err, err);
}

}  // namespace

// Deterministic (or deferred) adjoint of the curved P2 Laplacian on
// tetrahedra with its contraction on the tensor cores (host launcher).
cudaError_t launch_bwd_iso_tc(const BwdLaunch& L, const float* mid, float* dmid) {
  if (L.dim != 3 || L.form != LAPLACE_P2_ISO || L.atomic) return cudaErrorInvalidValue;
  if (L.n_elem == 0) return cudaSuccess;
  BwdParams p;
  p.conn = L.conn;
  p.coords = L.coords;
  p.coef = L.coef;
  p.dA = L.dA;
  p.tile_rec = L.tile_rec;
  p.rank = L.rank;
  p.rec_span = L.rec_span;
  p.rec_dest = L.rec_dest;
  p.records = L.records;
  p.dcoef = L.dcoef;
  p.dcoords = L.dcoords;
  p.n_elem = L.n_elem;
  p.n_vert = L.n_vert;
  p.dev_err = L.dev_err;
  p.vec_conn = reinterpret_cast<uintptr_t>(L.conn) % 16 == 0;
  p.vec_dA = reinterpret_cast<uintptr_t>(L.dA) % 16 == 0;
  auto kern = fem_bwd_iso_tc_kernel;
  cudaError_t st = ensure_smem(reinterpret_cast<const void*>(kern), kAdjSmem);
  if (st != cudaSuccess) return st;
  const int per_sm =
      L.ctas_per_sm > 0 ? L.ctas_per_sm : tc_ctas_per_sm(reinterpret_cast<const void*>(kern), kAdjSmem, kAdjTmemCols);
  const int64_t nct = (L.n_elem + kTileElems - 1) / kTileElems;
  int64_t grid = int64_t(per_sm) * device_sm_count();
  if (grid > nct) grid = nct;
  kern<<<unsigned(grid < 1 ? 1 : grid), kTileElems, kAdjSmem, L.stream>>>(p, mid, dmid);
  return cudaGetLastError();
}

}  // namespace fem
