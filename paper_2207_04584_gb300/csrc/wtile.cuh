// Dense weight tiles of a plan (built on the first grid call of a kernel
// that reads them): one per 32-candidate sub-chunk, the image the cell-major
// tensor-core kernel's A builders assemble in shared memory (Eq. 1's weights
// w of one block's 128 cells x 32 candidates, scaled by 2^15): the FP16 high
// halves, K-major with the 64-byte swizzle of tile_off, then the FP16 low
// halves (w * 2^15 - hi) in the same layout; 16 KB.  Cells a candidate does
// not reach hold zeros.
#pragma once

#include <cuda_fp16.h>

#include "hegrid_internal.cuh"

namespace hg {

constexpr uint32_t kWTileHalfBytes = (uint32_t)HG_BLOCK_CELLS * 64u;  // 128 rows x 64 bytes
constexpr uint32_t kWTileBytes = 2u * kWTileHalfBytes;               // hi, then lo

// Writes the entries [e0, e1) of one sub-chunk into `tile` (shared memory,
// 16-byte aligned, zero where no entry lands), by the kThreads threads of
// the CTA (thread t).  Entries are read four at a time (one 8-byte load of
// offsets, one 16-byte load of weights: the arrays' bases are 16-byte
// aligned and reach at least 3 entries past the last one), quads that
// straddle e0 or e1 masked, and a thread loads up to four quads before it
// stores any, so one round trip to memory brings most of a sub-chunk.
template <int kThreads>
__device__ __forceinline__ void wtile_scatter(uint8_t* tile, const uint16_t* ent_ck,
                                              const float* ent_w, int64_t e0, int64_t e1,
                                              int t) {
  auto put = [&](uint32_t off, float w) {
    const float ws = w * kTcWeightScale;
    const __half hw = __float2half_rn(ws);
    const __half lw = __float2half_rn(ws - __half2float(hw));
    *reinterpret_cast<__half*>(tile + off) = hw;
    *reinterpret_cast<__half*>(tile + kWTileHalfBytes + off) = lw;
  };
  auto put_quad = [&](int64_t q, uint2 ck, float4 w) {
    const int64_t e = 4 * q;
    if (e >= e0 && e < e1) put(ck.x & 0xffffu, w.x);
    if (e + 1 >= e0 && e + 1 < e1) put(ck.x >> 16, w.y);
    if (e + 2 >= e0 && e + 2 < e1) put(ck.y & 0xffffu, w.z);
    if (e + 3 >= e0 && e + 3 < e1) put(ck.y >> 16, w.w);
  };
  const int64_t q1 = (e1 + 3) >> 2;
  int64_t q = (e0 >> 2) + t;
  for (; q + 3 * kThreads < q1; q += 4 * kThreads) {
    uint2 ck[4];
    float4 w[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      ck[u] = *reinterpret_cast<const uint2*>(ent_ck + 4 * (q + u * kThreads));
      w[u] = *reinterpret_cast<const float4*>(ent_w + 4 * (q + u * kThreads));
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) put_quad(q + u * kThreads, ck[u], w[u]);
  }
  for (; q < q1; q += kThreads)
    put_quad(q, *reinterpret_cast<const uint2*>(ent_ck + 4 * q),
             *reinterpret_cast<const float4*>(ent_w + 4 * q));
}

// Copies `tile` to global memory at dst (16-byte aligned) in coalesced
// 16-byte stores and leaves it zero for the next sub-chunk.
template <int kThreads>
__device__ __forceinline__ void wtile_flush(uint8_t* tile, uint8_t* dst, int t) {
  uint4* s = reinterpret_cast<uint4*>(tile);
  uint4* d = reinterpret_cast<uint4*>(dst);
#pragma unroll
  for (int i = t; i < (int)(kWTileBytes / 16); i += kThreads) {
    d[i] = s[i];
    s[i] = make_uint4(0u, 0u, 0u, 0u);
  }
}

// Zeroes `tile` (before the first sub-chunk).
template <int kThreads>
__device__ __forceinline__ void wtile_zero(uint8_t* tile, int t) {
  uint4* s = reinterpret_cast<uint4*>(tile);
#pragma unroll
  for (int i = t; i < (int)(kWTileBytes / 16); i += kThreads) s[i] = make_uint4(0u, 0u, 0u, 0u);
}

}  // namespace hg
