// fem_tc.cuh -- forward integration with the G:K contraction on the 5th-generation
// tensor cores (tcgen05, TMEM accumulators) in split-BF16 arithmetic.
//
// Per CTA tile of 128 elements (one element per thread) the contraction of
// Eq. 6 is the dense product  D[e][t] = sum_k Ahat[e][k] B[k][t]  where
//   t = (i, j), i <= j, runs over the unique entries of A_e (NT of them,
//       padded to N, a multiple of 16),
//   Ahat[e] = [ g1 | g2 | g3 ]: the folded geometric tensor G_e split
//       into three bf16 terms, g1 = bf16(G), g2 = bf16(G - g1),
//       g3 = bf16(G - g1 - g2) (each rounding to bf16's 8-bit significand
//       leaves at most 2^-8 of what it rounds, so |G - g1 - g2 - g3| <=
//       2^-24 |G|, FP32's own unit roundoff), each term
//       zero-padded to KT, a multiple of 16 (K = 3 KT),
//   B[k][t] = K'[k mod KT][i][j] * DEN, small integers, exact in bf16; its
//       shared-memory image is built at compile time and copied by each CTA.
// The MMA (tcgen05.mma kind::f16, M = 128, N, K = 16 per step, FP32
// accumulation in TMEM) is issued by one thread; its completion is signalled
// on an mbarrier.  Each warp then reads its 32 rows of D with tcgen05.ld
// (lane = element) and mirrors (i, j) -> (j, i) into a 128-byte-swizzled
// shared stage, from which TMA tensor stores write 32 x 32 boxes of the
// [n_elem][N*N] output.  The stage holds as many boxes as keep the most CTAs
// resident; the last stores drain while the next tile's geometry is formed.
// (Without a tensor map, a plain stage and coalesced 16-byte stores.)  The
// warp-specialized kernel further below runs the same steps for two tiles at
// once: producers form tile i while consumers store tile i - 1.
// Operands live in shared memory in the canonical no-swizzle K-major layout:
// 8x16-byte core matrices, K-adjacent cores LBO bytes apart, M/N-adjacent cores
// SBO bytes apart.  All waits are bounded: on a timeout the kernel flags
// FEM_DEVERR_TIMEOUT, stops, waits (bounded) for the tensor core and frees TMEM.
#pragma once
#include <algorithm>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "fem_core.cuh"
#include "fem_fwd.cuh"
#include "fem_internal.h"
#include "fem_pipe.cuh"

namespace fem {

template <int D, int FORM>
struct TcPlan {
  using FT = FormTraits<D, FORM>;
  static constexpr int M = kTileElems;                   // 128 rows (elements)
  static constexpr int NT = FT::NT;                      // unique outputs
  static constexpr int N = (NT + 15) / 16 * 16;          // MMA N
  static constexpr int KT = (FT::NG + 15) / 16 * 16;     // one bf16 term of G, padded
  static constexpr int K = 3 * KT;
  static constexpr int KSTEPS = K / 16;
  static constexpr int MC = M / 8, NC = N / 8, KC = K / 8;  // core-matrix counts
  static constexpr uint32_t A_LBO = MC * 128, A_SBO = 128;  // A cores: (kc * MC + mc) * 128
  static constexpr uint32_t B_LBO = NC * 128, B_SBO = 128;  // B cores: (kc * NC + nc) * 128
  static constexpr size_t a_bytes = size_t(M) * K * 2;
  // B: K' * DEN once (KT rows); the three terms of A multiply the same B
  static constexpr size_t b_bytes = size_t(N) * KT * 2;
  static constexpr int SST = stage_stride<FT::NN>();
  // the plain epilogue's stage (without a tensor map), aliasing the A tile
  static constexpr size_t stage_bytes = align_up(size_t(4) * 32 * SST * 4, 128);
  static constexpr size_t b_region = align_up(b_bytes, 1024);  // keeps the region 1024-byte aligned
  // TMA epilogue: per warp, NN / 32 boxes (rounded up) of 32 rows x 128 bytes
  // with the 128-byte swizzle (1024-byte aligned), staged SBOX boxes at a time
  static constexpr int BOXES = (FT::NN + 31) / 32;
  static constexpr size_t region_for(int sbox) {
    return size_t(4) * sbox * 4096 > align_up(a_bytes, 1024) ? size_t(4) * sbox * 4096 : align_up(a_bytes, 1024);
  }
  static constexpr size_t smem_for(size_t region) { return b_region + region + 128 + 1024; }  // + mbarrier, TMEM slot, slack
  // CTAs that the shared memory of an SM (228 KB, 1 KB reserved per CTA)
  // holds, up to the ones the registers hold: four 128-thread CTAs at 128
  // registers a thread, two for the curved tetrahedra's geometry (over 200)
  static constexpr int reg_ctas = (FT::ISO && D == 3) ? 2 : 4;
  static constexpr int fit(int sbox) {
    return int(size_t(233472) / (smem_for(region_for(sbox)) + 1024)) < reg_ctas
               ? int(size_t(233472) / (smem_for(region_for(sbox)) + 1024))
               : reg_ctas;
  }
  // the largest stage that keeps the most CTAs resident: a smaller stage costs
  // a wait for the tensor stores inside the epilogue
  static constexpr int pick_sbox() {
    int best = BOXES;
    for (int s = BOXES - 1; s >= 1; --s)
      if (fit(s) > fit(best)) best = s;
    return best;
  }
  static constexpr int SBOX = pick_sbox();
  static constexpr int GROUPS = (BOXES + SBOX - 1) / SBOX;
  template <bool TMA>
  static constexpr size_t region_bytes = TMA ? region_for(SBOX)
                                             : (stage_bytes > a_bytes ? stage_bytes : align_up(a_bytes, 1024));
  template <bool TMA>
  static constexpr size_t smem = smem_for(region_bytes<TMA>);
  static constexpr int TMEM_COLS = N <= 32 ? 32 : (N <= 64 ? 64 : (N <= 128 ? 128 : 256));
  static_assert(N >= 16 && N <= 256 && K % 16 == 0, "MMA shape");
};

// ------------------------------------------------------------------ tcgen05 / mbarrier
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= uint64_t((saddr & 0x3FFFF) >> 4);          // bits  0-13 start address
  d |= uint64_t((lbo >> 4) & 0x3FFF) << 16;       // bits 16-29 leading (K) byte offset
  d |= uint64_t((sbo >> 4) & 0x3FFF) << 32;       // bits 32-45 stride (M/N) byte offset
  d |= uint64_t(1) << 46;                         // bits 46-48 fixed 0b001
  return d;                                       // base offset 0, no swizzle (bits 61-63 = 0)
}

template <int M, int N>
constexpr uint32_t idesc_bf16_f32() {
  return (1u << 4)                 // D format: F32
         | (1u << 7)               // A format: BF16
         | (1u << 10)              // B format: BF16
         | (0u << 15) | (0u << 16) // A, B K-major
         | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
               : "memory");
}
__device__ __forceinline__ void mbar_init(uint32_t mbar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mbar) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
// Bounded wait for the completion of the mbarrier phase with the given parity.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  for (uint32_t it = 0; it < (1u << 22); ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&r)[16]) {
  uint32_t u[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]),
        "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15])
      : "r"(taddr));
#pragma unroll
  for (int q = 0; q < 16; ++q) r[q] = __uint_as_float(u[q]);
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }

// ------------------------------------------------------------------ operand staging

// BF16 bits of an integer that BF16 holds exactly (at most 8 significant
// bits); 0x10000 for one that it does not.
constexpr uint32_t bf16_of_int(int v) {
  if (v == 0) return 0;
  const uint32_t sign = v < 0 ? 0x8000u : 0u;
  const uint32_t a = v < 0 ? uint32_t(-v) : uint32_t(v);
  int e = 31;
  while (!((a >> e) & 1u)) --e;  // leading bit
  if (e > 7 && (a & ((1u << (e - 7)) - 1u))) return 0x10000u;
  const uint32_t mant = (e >= 7 ? a >> (e - 7) : a << (7 - e)) & 0x7Fu;
  return sign | (uint32_t(e + 127) << 7) | mant;
}

// The B operand as it lies in shared memory: B[k][t] = K'_g^{ij} * DEN for
// k = term * KT + g (the same K for each of the three terms of G), (i, j) the
// t-th unique entry, zero past NG and NT; BF16 bits in the K-major core-matrix
// layout (core (k / 8, t / 8), row t % 8, column k % 8). Built at compile time.
template <int D, int FORM>
struct alignas(16) TcBImage {
  uint16_t v[TcPlan<D, FORM>::N * TcPlan<D, FORM>::KT];
};

template <int D, int FORM>
constexpr int tc_b_value(const RefTensor<D, FORM>& kt, int t, int k) {
  using TP = TcPlan<D, FORM>;
  using FT = FormTraits<D, FORM>;
  const int g = k % TP::KT;
  return (t < TP::NT && g < FT::NG) ? kt.v[g][tri_row(t, FT::N)][tri_col(t, FT::N)] : 0;
}

template <int D, int FORM>
constexpr TcBImage<D, FORM> make_tc_b_image() {
  using TP = TcPlan<D, FORM>;
  const RefTensor<D, FORM> kt = make_ref_tensor<D, FORM>();
  TcBImage<D, FORM> im{};
  for (int t = 0; t < TP::N; ++t)
    for (int k = 0; k < TP::KT; ++k)
      im.v[((k / 8) * TP::NC + t / 8) * 64 + (t % 8) * 8 + k % 8] = uint16_t(bf16_of_int(tc_b_value(kt, t, k)));
  return im;
}

// Whether every entry of K' * DEN is exact in BF16 (the split of G carries all
// of the rounding).
template <int D, int FORM>
constexpr bool tc_b_exact() {
  const RefTensor<D, FORM> kt = make_ref_tensor<D, FORM>();
  for (int t = 0; t < TcPlan<D, FORM>::N; ++t)
    for (int k = 0; k < TcPlan<D, FORM>::KT; ++k)
      if (bf16_of_int(tc_b_value(kt, t, k)) > 0xFFFFu) return false;
  return true;
}

// B into shared memory, once per CTA: a copy of KRef::b_image<D, FORM>() in
// 16-byte loads.
template <int D, int FORM, class KRef>
__device__ void tc_fill_b(unsigned char* sb) {
  using TP = TcPlan<D, FORM>;
  static_assert(TP::b_bytes % 16 == 0 && sizeof(TcBImage<D, FORM>) == TP::b_bytes, "B image");
  const uint4* src = reinterpret_cast<const uint4*>(KRef::template b_image<D, FORM>()->v);
  uint4* dst = reinterpret_cast<uint4*>(sb);
  for (int i = threadIdx.x; i < int(TP::b_bytes / 16); i += blockDim.x) dst[i] = __ldg(src + i);
}

// Row m of the A tile: the three bf16 terms of G (zero padded) in the core layout.
// A 16-byte chunk covers 8 consecutive k of one term (KT is a multiple of 16).
template <int D, int FORM>
__device__ __forceinline__ void tc_store_a_row(unsigned char* sa, int m, const float (&G)[FormTraits<D, FORM>::NG]) {
  using TP = TcPlan<D, FORM>;
  using FT = FormTraits<D, FORM>;
  constexpr int KW = TP::KT / 2;  // packed bf16 pairs per term
  uint32_t w[3][KW];
#pragma unroll
  for (int q = 0; q < KW; ++q) {
    // two G entries at once: h = bf16x2(x), r = x - h exactly, then the same on r
    const float x0 = 2 * q < FT::NG ? G[2 * q] : 0.f, x1 = 2 * q + 1 < FT::NG ? G[2 * q + 1] : 0.f;
    const __nv_bfloat162 h0 = __floats2bfloat162_rn(x0, x1);
    const float r0 = x0 - __low2float(h0), r1 = x1 - __high2float(h0);
    const __nv_bfloat162 h1 = __floats2bfloat162_rn(r0, r1);
    const float s0 = r0 - __low2float(h1), s1 = r1 - __high2float(h1);
    const __nv_bfloat162 h2 = __floats2bfloat162_rn(s0, s1);
    w[0][q] = *reinterpret_cast<const uint32_t*>(&h0);
    w[1][q] = *reinterpret_cast<const uint32_t*>(&h1);
    w[2][q] = *reinterpret_cast<const uint32_t*>(&h2);
  }
  const uint32_t rowoff = uint32_t(m / 8) * 128u + uint32_t(m % 8) * 16u;
#pragma unroll
  for (int kc = 0; kc < TP::KC; ++kc) {
    const int term = (kc * 8) / TP::KT, q0 = ((kc * 8) % TP::KT) / 2;
    *reinterpret_cast<uint4*>(sa + uint32_t(kc) * TP::A_LBO + rowoff) =
        make_uint4(w[term][q0], w[term][q0 + 1], w[term][q0 + 2], w[term][q0 + 3]);
  }
}

// Writes the 16 accumulator columns of chunk C (unique entries t = 16C + q) to
// both (i, j) and (j, i) of the element's stage row; indices are compile-time.
template <int N, int NT, int C, int... Qs>
__device__ __forceinline__ void tc_mirror_chunk(const float (&r)[16], float* row, std::integer_sequence<int, Qs...>) {
  (
      [&] {
        constexpr int t = C * 16 + Qs;
        if constexpr (t < NT) {
          constexpr int i = tri_row(t, N), j = tri_col(t, N);
          row[i * N + j] = r[Qs];
          if constexpr (i != j) row[j * N + i] = r[Qs];
        }
      }(),
      ...);
}

template <int D, int FORM, int C>
__device__ __forceinline__ void tc_epilogue_chunks(uint32_t tl, float* row) {
  using TP = TcPlan<D, FORM>;
  if constexpr (C < TP::N / 16) {
    float r[16];
    tmem_ld16(tl + uint32_t(C * 16), r);
    tmem_ld_wait();
    tc_mirror_chunk<FormTraits<D, FORM>::N, TP::NT, C>(r, row, std::make_integer_sequence<int, 16>{});
    tc_epilogue_chunks<D, FORM, C + 1>(tl, row);
  }
}

// The N accumulator columns of this thread's TMEM lane (unique entries t of
// the element matrix, t < NT), loaded 16 at a time.
template <int N, int... Cs>
__device__ __forceinline__ void tc_load_all(uint32_t tl, float (&r)[N], std::integer_sequence<int, Cs...>) {
  (
      [&] {
        float c[16];
        tmem_ld16(tl + uint32_t(Cs * 16), c);
#pragma unroll
        for (int q = 0; q < 16; ++q) r[Cs * 16 + q] = c[q];
      }(),
      ...);
  tmem_ld_wait();
}

// Unique-entry index of A[i][j] (symmetric: the (min, max) entry); entries
// past the matrix (the padding of its last chunk) read entry 0.
constexpr int tc_tri_index(int k, int n) {
  return k >= n * n ? 0 : ((k / n) <= (k % n) ? pair_index(k / n, k % n, n) : pair_index(k % n, k / n, n));
}

// This thread's element row-major matrix as 16-byte chunks into its row of the
// swizzled stage: chunk c lies in box c / 8 at 16-byte slot (c % 8) ^ sw of
// the thread's 128-byte row (compile-time gather from the registers).
// Only boxes B0 .. B0 + NB - 1 are written, box B0 first in the stage.
template <int N, int NT, int B0, int NB, int... Cs>
__device__ __forceinline__ void tc_stage_rows(const float (&r)[((NT + 15) / 16) * 16], unsigned char* row, int sw,
                                              std::integer_sequence<int, Cs...>) {
  (([&] {
     if constexpr (Cs / 8 >= B0 && Cs / 8 < B0 + NB) {
       *reinterpret_cast<float4*>(row + (Cs / 8 - B0) * 4096 + 16 * ((Cs % 8) ^ sw)) =
           make_float4(r[tc_tri_index(4 * Cs, N)], r[tc_tri_index(4 * Cs + 1, N)], r[tc_tri_index(4 * Cs + 2, N)],
                       r[tc_tri_index(4 * Cs + 3, N)]);
     }
   }()),
   ...);
}

// A warp's 32 element matrices (rows e0 .. e0 + 31 of the [n_elem][N*N] array)
// out through its stage, SBOX boxes per group; lane 0 issues the tensor
// stores and, between groups, waits until they have read the stage. The last
// group's stores are left in flight.
template <class TP, int N, int NT, int... Gs>
__device__ __forceinline__ void tc_store_groups(const float (&r)[((NT + 15) / 16) * 16], unsigned char* wst, int lane,
                                                const CUtensorMap* tmap, int64_t e0, bool live,
                                                std::integer_sequence<int, Gs...>) {
  (([&] {
     constexpr int B0 = Gs * TP::SBOX;
     constexpr int NB = TP::BOXES - B0 < TP::SBOX ? TP::BOXES - B0 : TP::SBOX;
     if constexpr (Gs > 0) {
       if (lane == 0) bulk_wait_read<0>();
       __syncwarp();
     }
     tc_stage_rows<N, NT, B0, NB>(r, wst + lane * 128, lane & 7, std::make_integer_sequence<int, (N * N + 3) / 4>{});
     fence_proxy_async_smem();
     __syncwarp();
     if (lane == 0 && live) {
#pragma unroll
       for (int b = 0; b < NB; ++b) tma_store_2d(tmap, 32 * (B0 + b), int(e0), smem_u32(wst + b * 4096));
       bulk_commit();
     }
   }()),
   ...);
}

// Geo::tile_g<D, FORM>(p, mid, e, X, w, G) forms element e's folded G (zero on
// return for an element it flags) and returns its device-error bits.
template <int D, int FORM, class Geo, class KRef, bool TMA>
__global__ void __launch_bounds__(kTileElems)
    fem_fwd_tc_kernel(FwdParams<float, float> p, const float* mid, const __grid_constant__ CUtensorMap tmap) {
  using TP = TcPlan<D, FORM>;
  using FT = FormTraits<D, FORM>;
  constexpr int N = FT::N, NN = FT::NN, SST = TP::SST;
  extern __shared__ __align__(128) unsigned char smem_raw_tc[];
  // 1024-byte aligned base: the swizzled TMA stage follows the shared address
  unsigned char* smem_raw = smem_raw_tc + ((1024u - (smem_u32(smem_raw_tc) & 1023u)) & 1023u);
  unsigned char* sb = smem_raw;                                      // B operand
  unsigned char* region = smem_raw + TP::b_region;                   // A tile, then output stages
  uint64_t* mbar_ptr = reinterpret_cast<uint64_t*>(region + TP::template region_bytes<TMA>);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(region + TP::template region_bytes<TMA> + 16);
  int* abort_flag = reinterpret_cast<int*>(region + TP::template region_bytes<TMA> + 32);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t mbar = smem_u32(mbar_ptr);
  const int64_t nct = (p.n_elem + kTileElems - 1) / kTileElems;
  if (int64_t(blockIdx.x) >= nct) return;  // CTA-uniform, before any TMEM allocation

  // set-up: B operand, mbarrier, TMEM accumulator
  tc_fill_b<D, FORM, KRef>(sb);
  if (tid == 0) {
    mbar_init(mbar);
    *abort_flag = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                 "n"(TP::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  constexpr uint32_t idesc = idesc_bf16_f32<TP::M, TP::N>();
  int err = 0;
  uint32_t phase = 0;

  int v[D + 1];
  float Xc[D + 1][D];
  int64_t T = blockIdx.x;
  const int vec_conn = (D == 3) && (reinterpret_cast<uintptr_t>(p.conn) % 16 == 0);
  load_conn<D>(p.conn, T * kTileElems + tid, p.n_elem, vec_conn, v);
  int fcur = gather_regs<D>(p.coords, p.n_vert, T * kTileElems + tid, p.n_elem, v, Xc);
  float wcur = (p.coef && T * kTileElems + tid < p.n_elem) ? __ldg(p.coef + T * kTileElems + tid) : 1.f;
  int vn[D + 1];  // the next tile's connectivity, loaded a tile before its gather
  load_conn<D>(p.conn, (T + gridDim.x) * kTileElems + tid, p.n_elem, vec_conn, vn);
  for (; T < nct; T += gridDim.x) {
    // prefetch: connectivity two tiles ahead, the next tile's coordinates
    // (its connectivity arrived during the previous tile)
    const int64_t en = (T + gridDim.x) * kTileElems + tid;
    int vnn[D + 1];
    load_conn<D>(p.conn, en + int64_t(gridDim.x) * kTileElems, p.n_elem, vec_conn, vnn);
    float Xn[D + 1][D];
    const int fnext = gather_regs<D>(p.coords, p.n_vert, en, p.n_elem, vn, Xn);
    const float wnext = (p.coef && en < p.n_elem) ? __ldg(p.coef + en) : 1.f;
    // geometric tensor of this thread's element -> bf16 split into the A tile
    float G[FT::NG];
#pragma unroll
    for (int g = 0; g < FT::NG; ++g) G[g] = 0.f;
    if (fcur & GF_OK) {
      err |= Geo::template tile_g<D, FORM>(p, mid, T * kTileElems + tid, Xc, wcur, G);
    } else if (fcur & GF_ELEM) {
      err |= DEVERR_CONN;
    }
    if constexpr (TMA) {
      // the previous tile's tensor stores drained while G was formed; every
      // warp's stage has been read before any thread overwrites it with A
      if (lane == 0) bulk_wait_read<0>();
      __syncthreads();
    }
    tc_store_a_row<D, FORM>(region, tid, G);
    fence_proxy_async_smem();  // generic-proxy writes of A -> tensor-core reads
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t sa = smem_u32(region), sbb = smem_u32(sb);
#pragma unroll
      for (int s = 0; s < TP::KSTEPS; ++s) {
        const uint64_t ad = smem_desc(sa + uint32_t(2 * s) * TP::A_LBO, TP::A_LBO, TP::A_SBO);
        const uint64_t bd = smem_desc(sbb + uint32_t(2 * (s % (TP::KT / 16))) * TP::B_LBO, TP::B_LBO, TP::B_SBO);
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
    const int64_t e0 = T * kTileElems + warp * 32;
    if constexpr (TMA) {
      // epilogue: this thread's TMEM lane -> registers -> its row's 16-byte
      // chunks in the 128-byte-swizzled stage (chunk c of box b at c ^ (row & 7):
      // conflict-free) -> one TMA tensor store per box, rows and columns past
      // the array clipped
      unsigned char* wst = region + size_t(warp) * TP::SBOX * 4096;
      float r[TP::N];
      tc_load_all<TP::N>(tmem + (uint32_t(warp * 32) << 16), r, std::make_integer_sequence<int, TP::N / 16>{});
      tc_store_groups<TP, N, TP::NT>(r, wst, lane, &tmap, e0, e0 < p.n_elem,
                                     std::make_integer_sequence<int, TP::GROUPS>{});
      __syncwarp();
    } else {
    // epilogue: this warp's 32 rows of D -> mirrored stage -> coalesced stores
    float* st = reinterpret_cast<float*>(region) + warp * 32 * SST;
    float* row = st + lane * SST;
    tc_epilogue_chunks<D, FORM, 0>(tmem + (uint32_t(warp * 32) << 16), row);
    __syncwarp();
    if (e0 < p.n_elem) {
      const int cnt = int(p.n_elem - e0 < 32 ? p.n_elem - e0 : 32);
      float* dst = p.A + e0 * NN;
      if (p.vec_store && NN % 4 == 0) {
        const int nq = cnt * (NN / 4);
        for (int q = lane; q < nq; q += 32) {
          const int idx = 4 * q;
          const int el = idx / NN;
          const float* s = st + el * SST + (idx - el * NN);
          __stcs(reinterpret_cast<float4*>(dst) + q, make_float4(s[0], s[1], s[2], s[3]));
        }
      } else {
        const int nw = cnt * NN;
        for (int idx = lane; idx < nw; idx += 32) {
          const int el = idx / NN;
          __stcs(dst + idx, st[el * SST + (idx - el * NN)]);
        }
      }
    }
    }
    if constexpr (!TMA) {
      tc_fence_before();
      __syncthreads();  // the stage (aliasing the A tile) is reused by the next tile
      tc_fence_after();
    }
    fcur = fnext;
    wcur = wnext;
#pragma unroll
    for (int k = 0; k <= D; ++k) {
      vn[k] = vnn[k];
#pragma unroll
      for (int a = 0; a < D; ++a) Xc[k][a] = Xn[k][a];
    }
  }
  if constexpr (TMA) {
    if (lane == 0) bulk_wait<0>();  // this warp's tensor stores are complete
  }
  // teardown: after an abort, give the tensor core a bounded chance to finish first
  if (*abort_flag && tid == 0) mbar_wait(mbar, phase);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "n"(TP::TMEM_COLS)
                 : "memory");
  }
  err = __reduce_or_sync(0xffffffffu, err);
  if (err && lane == 0 && p.dev_err) atomicOr(p.dev_err, err);
}

// ------------------------------------------------------------------ warp-specialized pipeline
// The kernel above takes each tile through geometry, split, MMA and epilogue
// in turn.  This one overlaps them: a CTA of 8 warps where warps 0-3
// (producers, one element per thread) form G, split it and write A tile i
// into one of two A buffers while warps 4-7 (consumers) read the accumulator
// of tile i - 1 from the other of two TMEM buffers and store it.  Thread 0
// issues each tile's MMAs once its A rows are written and the consumers have
// released that TMEM buffer.  mbarriers (all waits bounded):
//   full[b]  -- the MMAs of the tile in buffer b completed (tcgen05.commit):
//               the consumers may read D[b], the producers may rewrite A[b];
//   empty[b] -- the four consumer warps read D[b] (one arrival each): the next
//               MMAs into D[b] may start.
// Use k of buffer b (tile i = 2k + b) waits on phase parity k & 1, so no
// barrier ever runs more than one phase ahead of a waiter.  A timeout flags
// FEM_DEVERR_TIMEOUT; the producers stop together at their next barrier, the
// consumers at their next wait, and the teardown waits (bounded) for the last
// MMAs before freeing TMEM.
// Whether launches with a tensor map take the warp-specialized pipeline.
constexpr bool kTcPipelined = true;

template <int D, int FORM>
struct TcWsPlan {
  using TP = TcPlan<D, FORM>;
  static constexpr int BOXES = TP::BOXES;
  static constexpr size_t a_region = align_up(TP::a_bytes, 1024);
  static constexpr size_t smem_for(int sbox) {
    return TP::b_region + 2 * a_region + size_t(4) * sbox * 4096 + 128 + 1024;
  }
  static constexpr size_t kMaxSmem = 232448;  // opt-in shared memory of one CTA
  static constexpr int pick_sbox() {
    int s = BOXES;
    while (s > 1 && smem_for(s) > kMaxSmem) --s;
    return s;
  }
  static constexpr int SBOX = pick_sbox();
  static constexpr int GROUPS = (BOXES + SBOX - 1) / SBOX;
  static constexpr size_t stage_region = size_t(4) * SBOX * 4096;
  static constexpr size_t smem = smem_for(SBOX);
  static constexpr int TMEM_COLS = 2 * TP::N <= 32 ? 32 : (2 * TP::N <= 64 ? 64 : (2 * TP::N <= 128 ? 128 : 256));
  static constexpr bool fits = smem <= kMaxSmem && 2 * TP::N <= 256;
  // Whether the launcher takes this kernel.  Not for the curved elements:
  // their G costs four inverse Jacobians per element (214 registers), and
  // four producer warps per SM then bound the tile rate (measured 2.07 ms
  // against 1.99 ms for two 4-warp CTAs of the kernel above on the warped
  // 128^3 cube; elasticity 1.54 -> 1.14 ms, the P1-coefficient P2
  // Laplacian 1.46 -> 1.36 ms).
  static constexpr bool preferred = fits && !FormTraits<D, FORM>::ISO;
};

__device__ __forceinline__ void mbar_init_count(uint32_t mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(mbar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(mbar) : "memory");
}
// Barrier 1 of the CTA, among its first 128 threads (the producer warps).
__device__ __forceinline__ void producer_sync() { asm volatile("bar.sync 1, 128;\n" ::: "memory"); }

template <int D, int FORM, class Geo, class KRef>
__global__ void __launch_bounds__(2 * kTileElems, 1)
    fem_fwd_tc_ws_kernel(FwdParams<float, float> p, const float* mid, const __grid_constant__ CUtensorMap tmap) {
  using TP = TcPlan<D, FORM>;
  using WP = TcWsPlan<D, FORM>;
  using FT = FormTraits<D, FORM>;
  extern __shared__ __align__(128) unsigned char smem_raw_ws[];
  unsigned char* base = smem_raw_ws + ((1024u - (smem_u32(smem_raw_ws) & 1023u)) & 1023u);
  unsigned char* sb = base;                                            // B operand
  unsigned char* sa0 = base + TP::b_region;                            // A buffers 0, 1
  unsigned char* stages = base + TP::b_region + 2 * WP::a_region;     // consumer warps' output stages
  uint64_t* bars = reinterpret_cast<uint64_t*>(stages + WP::stage_region);  // full[2], empty[2]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 4);
  int* pabort = reinterpret_cast<int*>(bars + 5);  // written by thread 0 only, read after a producer barrier
  int* cabort = pabort + 1;                        // a consumer warp timed out
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t nct = (p.n_elem + kTileElems - 1) / kTileElems;
  if (int64_t(blockIdx.x) >= nct) return;  // CTA-uniform, before any barrier or TMEM allocation
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + 2);

  tc_fill_b<D, FORM, KRef>(sb);
  if (tid == 0) {
    mbar_init_count(full0, 1);
    mbar_init_count(full0 + 8, 1);
    mbar_init_count(empty0, 4);
    mbar_init_count(empty0 + 8, 4);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    *pabort = 0;
    *cabort = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                 "n"(WP::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  int err = 0;
  int issued = 0;  // thread 0: tiles whose MMAs it committed

  if (warp < 4) {
    // ---- producers: geometry, split, A tile, MMA issue (thread 0)
    constexpr uint32_t idesc = idesc_bf16_f32<TP::M, TP::N>();
    int v[D + 1];
    float Xc[D + 1][D];
    int64_t T = blockIdx.x;
    const int vec_conn = (D == 3) && (reinterpret_cast<uintptr_t>(p.conn) % 16 == 0);
    load_conn<D>(p.conn, T * kTileElems + tid, p.n_elem, vec_conn, v);
    int fcur = gather_regs<D>(p.coords, p.n_vert, T * kTileElems + tid, p.n_elem, v, Xc);
    float wcur = (p.coef && T * kTileElems + tid < p.n_elem) ? __ldg(p.coef + T * kTileElems + tid) : 1.f;
    int vn[D + 1];
    load_conn<D>(p.conn, (T + gridDim.x) * kTileElems + tid, p.n_elem, vec_conn, vn);
    for (int i = 0; T < nct; ++i, T += gridDim.x) {
      const int b = i & 1;
      const int64_t en = (T + gridDim.x) * kTileElems + tid;
      int vnn[D + 1];
      load_conn<D>(p.conn, en + int64_t(gridDim.x) * kTileElems, p.n_elem, vec_conn, vnn);
      float Xn[D + 1][D];
      const int fnext = gather_regs<D>(p.coords, p.n_vert, en, p.n_elem, vn, Xn);
      const float wnext = (p.coef && en < p.n_elem) ? __ldg(p.coef + en) : 1.f;
      float G[FT::NG];
#pragma unroll
      for (int g = 0; g < FT::NG; ++g) G[g] = 0.f;
      if (fcur & GF_OK) {
        err |= Geo::template tile_g<D, FORM>(p, mid, T * kTileElems + tid, Xc, wcur, G);
      } else if (fcur & GF_ELEM) {
        err |= DEVERR_CONN;
      }
      // A[b] was last read by the MMAs of tile i - 2 (phase (i >> 1) - 1 of full[b])
      if (i >= 2 && tid == 0 && !mbar_wait(full0 + 8 * b, uint32_t((i >> 1) - 1) & 1u)) *pabort = 1;
      producer_sync();
      if (*pabort) {
        err |= DEVERR_TIMEOUT;
        break;
      }
      tc_store_a_row<D, FORM>(sa0 + size_t(b) * WP::a_region, tid, G);
      fence_proxy_async_smem();  // generic-proxy writes of A -> tensor-core reads
      tc_fence_before();
      producer_sync();
      if (tid == 0) {
        // D[b] was last read by the consumers of tile i - 2
        if (i >= 2 && !mbar_wait(empty0 + 8 * b, uint32_t((i >> 1) - 1) & 1u)) {
          *pabort = 1;  // seen by every producer after their next barrier
        } else {
          tc_fence_after();
          const uint32_t sa = smem_u32(sa0 + size_t(b) * WP::a_region), sbb = smem_u32(sb);
#pragma unroll
          for (int s = 0; s < TP::KSTEPS; ++s) {
            const uint64_t ad = smem_desc(sa + uint32_t(2 * s) * TP::A_LBO, TP::A_LBO, TP::A_SBO);
            const uint64_t bd = smem_desc(sbb + uint32_t(2 * (s % (TP::KT / 16))) * TP::B_LBO, TP::B_LBO, TP::B_SBO);
            mma_bf16(tmem + uint32_t(b * TP::N), ad, bd, idesc, s > 0 ? 1u : 0u);
          }
          mma_commit(full0 + 8 * b);
          ++issued;
        }
      }
      fcur = fnext;
      wcur = wnext;
#pragma unroll
      for (int k = 0; k <= D; ++k) {
        vn[k] = vnn[k];
#pragma unroll
        for (int a = 0; a < D; ++a) Xc[k][a] = Xn[k][a];
      }
    }
  } else {
    // ---- consumers: TMEM lanes 32 cw .. 32 cw + 31 of D[b] -> swizzled stage -> TMA stores
    const int cw = warp - 4;
    unsigned char* wst = stages + size_t(cw) * WP::SBOX * 4096;
    int64_t T = blockIdx.x;
    for (int i = 0; T < nct; ++i, T += gridDim.x) {
      const int b = i & 1;
      int ok = 1;
      if (lane == 0) ok = mbar_wait(full0 + 8 * b, uint32_t(i >> 1) & 1u) ? 1 : 0;
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) {
        if (lane == 0) *cabort = 1;
        err |= DEVERR_TIMEOUT;
        break;
      }
      tc_fence_after();
      float r[TP::N];
      tc_load_all<TP::N>(tmem + (uint32_t(cw * 32) << 16) + uint32_t(b * TP::N), r,
                         std::make_integer_sequence<int, TP::N / 16>{});
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(empty0 + 8 * b);  // this warp has read its lanes of D[b]
      const int64_t e0 = T * kTileElems + cw * 32;
      if (lane == 0) bulk_wait_read<0>();  // the previous tile's tensor stores have read the stage
      __syncwarp();
      tc_store_groups<WP, FT::N, TP::NT>(r, wst, lane, &tmap, e0, e0 < p.n_elem,
                                         std::make_integer_sequence<int, WP::GROUPS>{});
      __syncwarp();
    }
    if (lane == 0) bulk_wait<0>();  // this warp's tensor stores are complete
  }

  // teardown: after a timeout, give the tensor core a bounded chance to finish the
  // last committed MMAs before TMEM is freed
  tc_fence_before();
  __syncthreads();
  if (tid == 0 && (*pabort || *cabort) && issued > 0)
    mbar_wait(full0 + 8 * ((issued - 1) & 1), uint32_t((issued - 1) >> 1) & 1u);
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "n"(WP::TMEM_COLS)
                 : "memory");
  }
  err = __reduce_or_sync(0xffffffffu, err);
  if (err && lane == 0 && p.dev_err) atomicOr(p.dev_err, err);
}

// G of an affine element with the compensated Jacobian (Eq. 8 / Eq. 15).
struct TcGeoAffine {
  template <int D, int FORM>
  __device__ __forceinline__ static int tile_g(const FwdParams<float, float>&, const float*, int64_t,
                                               const float (&X)[D + 1][D], float w,
                                               float (&G)[FormTraits<D, FORM>::NG]) {
    using FT = FormTraits<D, FORM>;
    Jac<D, float> jac;
    const bool nondeg = jacobian<D, JAC_COMP>(X, jac);
    const float scale = nondeg ? __fdividef(w, dev_abs(jac.det) * float(FT::DEN)) : 0.f;
    geometric_tensor<D, FORM>(jac.adj, scale, G);
    return nondeg ? 0 : DEVERR_DEGENERATE;
  }
};

// Host: tensor map of a row-major [rows][cols] FP32 array (cols * 4 bytes a
// multiple of 16) in boxes of 32 columns x 32 rows with the 128-byte swizzle;
// false when it cannot be described (fem_tc.cu).
bool encode_tc_rows_map(CUtensorMap* map, const void* base, int64_t rows, int cols);

// CTAs of 128 threads that fit on an SM by registers (allocated per warp in
// units of 8 per thread), shared memory (with the per-block reservation),
// threads and TMEM columns (512 per SM: a CTA beyond them would wait in
// tcgen05.alloc until another finished).  The occupancy API reports one for
// these kernels where two fit and run side by side (measured 1.5x faster).
inline int tc_ctas_per_sm(const void* kern, size_t smem, int tmem_cols) {
  cudaFuncAttributes fa{};
  int dev = 0, regs = 0, shm = 0, rsv = 0, thr = 0, blk = 0;
  if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&regs, cudaDevAttrMaxRegistersPerMultiprocessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&shm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&rsv, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&thr, cudaDevAttrMaxThreadsPerMultiProcessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&blk, cudaDevAttrMaxBlocksPerMultiprocessor, dev) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  const int warps = kTileElems / 32;
  const int regs_per_warp = (fa.numRegs + 7) / 8 * 8 * 32;
  const int by_regs = regs_per_warp > 0 ? regs / regs_per_warp / warps : blk;
  const int by_smem = int(size_t(shm) / (smem + fa.sharedSizeBytes + size_t(rsv)));
  const int by_thr = thr / kTileElems;
  const int by_tmem = 512 / tmem_cols;  // TMEM columns of an SM
  const int n = std::min(std::min(std::min(by_regs, by_smem), std::min(by_thr, blk)), by_tmem);
  return n < 1 ? 1 : n;
}

template <int D, int FORM, class Geo, class KRef>
cudaError_t launch_tc_t(const FwdLaunch& L, const float* mid) {
  using TP = TcPlan<D, FORM>;
  FwdParams<float, float> p;
  p.conn = L.conn;
  p.coords = static_cast<const float*>(L.coords);
  p.coef = L.coef;
  p.A = static_cast<float*>(L.A);
  p.n_elem = L.n_elem;
  p.n_vert = L.n_vert;
  p.dev_err = L.dev_err;
  p.vec_conn = 0;
  p.vec_store = reinterpret_cast<uintptr_t>(L.A) % 16 == 0;
  CUtensorMap tmap{};
  const bool tma = encode_tc_rows_map(&tmap, L.A, L.n_elem, TcPlan<D, FORM>::FT::NN);
  if constexpr (kTcPipelined && TcWsPlan<D, FORM>::preferred) {
    if (tma) {  // the warp-specialized pipeline: one CTA of 8 warps per SM
      using WP = TcWsPlan<D, FORM>;
      auto wk = fem_fwd_tc_ws_kernel<D, FORM, Geo, KRef>;
      cudaError_t st = ensure_smem(reinterpret_cast<const void*>(wk), WP::smem);
      if (st != cudaSuccess) return st;
      const int64_t nct = (L.n_elem + kTileElems - 1) / kTileElems;
      int64_t grid = int64_t(L.ctas_per_sm > 0 ? L.ctas_per_sm : 1) * device_sm_count();
      if (grid > nct) grid = nct;
      wk<<<unsigned(grid < 1 ? 1 : grid), 2 * kTileElems, WP::smem, L.stream>>>(p, mid, tmap);
      return cudaGetLastError();
    }
  }
  auto kern = tma ? fem_fwd_tc_kernel<D, FORM, Geo, KRef, true> : fem_fwd_tc_kernel<D, FORM, Geo, KRef, false>;
  const size_t smem = tma ? TP::template smem<true> : TP::template smem<false>;
  cudaError_t st = ensure_smem(reinterpret_cast<const void*>(kern), smem);
  if (st != cudaSuccess) return st;
  const int per_sm =
      L.ctas_per_sm > 0 ? L.ctas_per_sm : tc_ctas_per_sm(reinterpret_cast<const void*>(kern), smem, TP::TMEM_COLS);
  const unsigned grid = pipeline_grid(reinterpret_cast<const void*>(kern), 4, smem, L.n_elem, per_sm);
  kern<<<grid, kTileElems, smem, L.stream>>>(p, mid, tmap);
  return cudaGetLastError();
}

}  // namespace fem
