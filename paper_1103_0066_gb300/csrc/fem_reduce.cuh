// fem_reduce.cuh -- the sum of one vertex's adjoint records (the second phase
// of the deterministic reduction), shared by the single-mesh and multi-mesh
// reduction kernels so that both add in the same order.
//
// dcoords[v] = the sum of the records of v in increasing record order (and,
// for the P1-coefficient forms, whose records carry NC = D + 1 components,
// dcoef[v] = the sum of their last component).
// Vertex-major layout: they are rows [voff[v], voff[v+1]), read in blocks of
// 8 predicated loads, all in flight before the block's additions (a vertex
// has a handful of records: one block, one round trip).  Tile-order layout:
// they are rows vrec[voff[v] .. voff[v+1]) -- the same order, so the same
// bits -- read as four indices, then four records, per step.
#pragma once

#include <cstdint>

namespace fem {

template <int D, int NC>
__device__ __forceinline__ void reduce_store(const float (&acc)[NC], int64_t v, float* __restrict__ dcoords,
                                             float* __restrict__ dcoef) {
  if (dcoords)
#pragma unroll
    for (int a = 0; a < D; ++a) dcoords[v * D + a] = acc[a];
  if constexpr (NC > D) {
    if (dcoef) dcoef[v] = acc[D];
  }
}

template <int D, int NC>
__device__ __forceinline__ void reduce_vertex_direct(const int32_t* __restrict__ voff,
                                                     const float* __restrict__ records, int64_t v,
                                                     float* __restrict__ dcoords, float* __restrict__ dcoef) {
  const int32_t b = __ldg(voff + v), e = __ldg(voff + v + 1);
  float acc[NC];
#pragma unroll
  for (int a = 0; a < NC; ++a) acc[a] = 0.f;
  for (int32_t k0 = b; k0 < e; k0 += 8) {
    float r[8][NC];
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int a = 0; a < NC; ++a) r[u][a] = k0 + u < e ? __ldg(records + int64_t(k0 + u) * NC + a) : 0.f;
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (k0 + u < e)
#pragma unroll
        for (int a = 0; a < NC; ++a) acc[a] += r[u][a];
  }
  reduce_store<D, NC>(acc, v, dcoords, dcoef);
}

template <int D, int NC>
__device__ __forceinline__ void reduce_vertex_gather(const int32_t* __restrict__ voff,
                                                     const int32_t* __restrict__ vrec,
                                                     const float* __restrict__ records, int64_t v,
                                                     float* __restrict__ dcoords, float* __restrict__ dcoef) {
  const int32_t b = __ldg(voff + v), e = __ldg(voff + v + 1);
  float acc[NC];
#pragma unroll
  for (int a = 0; a < NC; ++a) acc[a] = 0.f;
  for (int32_t k0 = b; k0 < e; k0 += 4) {
    int32_t row[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) row[u] = k0 + u < e ? __ldg(vrec + k0 + u) : 0;
    float r[4][NC];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int a = 0; a < NC; ++a) r[u][a] = k0 + u < e ? __ldg(records + int64_t(row[u]) * NC + a) : 0.f;
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (k0 + u < e)
#pragma unroll
        for (int a = 0; a < NC; ++a) acc[a] += r[u][a];
  }
  reduce_store<D, NC>(acc, v, dcoords, dcoef);
}

}  // namespace fem
