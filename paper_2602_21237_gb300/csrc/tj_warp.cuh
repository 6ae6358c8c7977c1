// Warp-level ranking shared by the onesweep passes (tj_radix.cu) and the
// fused partition-resident join (tj_fused.cu): stable ranks of a warp's rows
// by a small digit, found with one ballot per digit bit (rank_items) or with a
// per-warp table of lane masks for the low 7 bits and one ballot per higher
// bit (rank_items_or).
#pragma once

#include <stdint.h>

namespace tj {

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm volatile("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Stable ranks of a warp's rows by digit.  Row i*32 + lane of the warp holds
// digit dr[i] (low 16 bits); rows at or beyond nv are padding.  Lanes with the
// same digit are found by one ballot per digit bit; the group's highest lane
// adds the group size to the warp's 16-bit counter of that digit (two per
// word; items in order, so ranks follow row order), and the rank (returned
// base + lanes of the group below this one) goes to the high 16 bits of dr[i].
template <int NB, int ITEMS>
__device__ __forceinline__ void rank_items(uint32_t (&dr)[ITEMS], int nv, uint32_t* wh) {
  const int lane = threadIdx.x & 31;
  const uint32_t ltm = lanemask_lt();
  constexpr int kHalf = ITEMS % 4 == 0 ? 4 : (ITEMS % 3 == 0 ? 3 : (ITEMS % 2 == 0 ? 2 : 1));
#pragma unroll
  for (int i0 = 0; i0 < ITEMS; i0 += kHalf) {
    uint32_t peers[kHalf];
#pragma unroll
    for (int h = 0; h < kHalf; ++h) {
      const bool ok = (i0 + h) * 32 + lane < nv;
      const uint32_t v = __ballot_sync(0xFFFFFFFFu, ok);
      peers[h] = ok ? v : ~v;
    }
#pragma unroll
    for (int b = 0; b < NB; ++b) {
#pragma unroll
      for (int h = 0; h < kHalf; ++h) {
        const int32_t m = (int32_t)(dr[i0 + h] << (31 - b)) >> 31;  // bit b: -1, else 0
        const uint32_t x = __ballot_sync(0xFFFFFFFFu, m != 0);
        peers[h] &= ~(x ^ (uint32_t)m);  // lanes whose bit b equals this lane's
      }
    }
#pragma unroll
    for (int h = 0; h < kHalf; ++h) {
      const int i = i0 + h;
      const bool ok = i * 32 + lane < nv;
      const int leader = 31 - __clz(peers[h]);
      const uint32_t d = dr[i] & 0xFFFFu;
      const uint32_t sh = (d & 1u) * 16u;
      uint32_t base = 0u;
      if (ok && leader == lane)
        base = (atomicAdd(&wh[d >> 1], (uint32_t)__popc(peers[h]) << sh) >> sh) & 0xFFFFu;
      base = __shfl_sync(0xFFFFFFFFu, base, leader);
      dr[i] |= (base + __popc(peers[h] & ltm)) << 16;
    }
  }
}

// Stable ranks as rank_items, with the lanes of each digit found through a
// per-warp table of lane masks in shared memory (wm[min(bins, 128)], zero on
// entry and on exit): every lane ORs its bit into the word of its digit's low
// 7 bits, the warp reads the words back, one ballot per higher digit bit (NH
// of them) drops the lanes that differ above, and each group's highest lane
// clears the word.  One shared atomic and NH ballots per row instead of one
// ballot per digit bit; the tables of all warps must fit the slot-index array.
template <int NH, int ITEMS>
__device__ __forceinline__ void rank_items_or(uint32_t (&dr)[ITEMS], int nv, uint32_t* wh,
                                              uint32_t* wm) {
  const int lane = threadIdx.x & 31;
  const uint32_t ltm = lanemask_lt();
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    if (i * 32 >= nv) break;  // the warp's remaining items are padding
    const bool ok = i * 32 + lane < nv;
    const uint32_t d = dr[i] & 0xFFFFu;
    const uint32_t w = d & 127u;
    if (ok) atomicOr(&wm[w], 1u << lane);
    __syncwarp();
    uint32_t peers = ok ? wm[w] : (1u << lane);
#pragma unroll
    for (int b = 7; b < 7 + NH; ++b) {
      const int32_t m = (int32_t)(d << (31 - b)) >> 31;  // bit b: -1, else 0
      const uint32_t x = __ballot_sync(0xFFFFFFFFu, m != 0);
      peers &= ~(x ^ (uint32_t)m);
    }
    __syncwarp();
    const int leader = 31 - __clz(peers);
    const uint32_t sh = (d & 1u) * 16u;
    uint32_t base = 0u;
    if (ok && leader == lane) {
      wm[w] = 0u;
      base = (atomicAdd(&wh[d >> 1], (uint32_t)__popc(peers) << sh) >> sh) & 0xFFFFu;
    }
    __syncwarp();
    base = __shfl_sync(0xFFFFFFFFu, base, leader);
    dr[i] |= (base + __popc(peers & ltm)) << 16;
  }
}

}  // namespace tj
