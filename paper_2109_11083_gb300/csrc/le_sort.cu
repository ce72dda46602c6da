// Stable LSD radix sort of (cell key, slot) pairs: the "resort" step that
// re-bins particles into cells at every list build.  8-bit digits, three
// kernels per pass: per-tile digit counts, one exclusive scan over the
// digit-major count table, and a stable scatter in which each tile ranks its
// keys chunk by chunk (warp match on the digit, then a per-digit prefix over
// the warps of the block).  Stability keeps the previous order of particles
// inside a cell, so the list order and every floating-point sum that follows
// it are deterministic.
#include <cuda_runtime.h>

#include "le_launch.h"

namespace le {

namespace {

constexpr int kWarps = kSortThreads / 32;

__global__ void __launch_bounds__(kSortThreads) k_rs_hist(const uint32_t *__restrict__ key, int n,
                                                          int shift, int nblocks,
                                                          uint32_t *__restrict__ hist) {
  __shared__ uint32_t cnt[kSortBuckets];
  for (int b = threadIdx.x; b < kSortBuckets; b += blockDim.x) cnt[b] = 0;
  __syncthreads();
  const int base = blockIdx.x * kSortTile;
#pragma unroll 4
  for (int k = 0; k < kSortItems; ++k) {
    const int i = base + k * kSortThreads + threadIdx.x;
    if (i < n) atomicAdd(&cnt[(key[i] >> shift) & (kSortBuckets - 1)], 1u);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < kSortBuckets; b += blockDim.x)
    hist[(size_t)b * nblocks + blockIdx.x] = cnt[b];
}

// Exclusive scan of m counts by one block of 1024 threads.
__global__ void __launch_bounds__(1024) k_rs_scan(uint32_t *__restrict__ hist, int m) {
  __shared__ uint32_t part[1024];
  const int t = threadIdx.x;
  const int per = (m + 1023) / 1024;
  const int lo = t * per;
  const int hi = min(lo + per, m);
  uint32_t s = 0;
  for (int i = lo; i < hi; ++i) s += hist[i];
  part[t] = s;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    uint32_t v = t >= o ? part[t - o] : 0u;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  uint32_t run = part[t] - s;
  for (int i = lo; i < hi; ++i) {
    const uint32_t c = hist[i];
    hist[i] = run;
    run += c;
  }
}

__global__ void __launch_bounds__(kSortThreads) k_rs_scatter(
    const uint32_t *__restrict__ kin, const uint32_t *__restrict__ vin, uint32_t *__restrict__ kout,
    uint32_t *__restrict__ vout, int n, int shift, int nblocks, const uint32_t *__restrict__ hist) {
  __shared__ uint32_t base[kSortBuckets];          // global start of each digit for this tile
  __shared__ uint32_t wcnt[kWarps][kSortBuckets];  // per-warp counts -> per-warp offsets
  __shared__ uint32_t total[kSortBuckets];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  for (int b = t; b < kSortBuckets; b += blockDim.x) {
    base[b] = hist[(size_t)b * nblocks + blockIdx.x];
    for (int w = 0; w < kWarps; ++w) wcnt[w][b] = 0;
  }
  __syncthreads();
  const int tile = blockIdx.x * kSortTile;
  for (int c = 0; c < kSortItems; ++c) {
    const int i = tile + c * kSortThreads + t;
    const bool valid = i < n;
    const uint32_t k = valid ? kin[i] : 0u;
    const uint32_t v = valid ? vin[i] : 0u;
    // invalid lanes get a digit outside the bucket range so they never match
    const uint32_t dig = valid ? ((k >> shift) & (kSortBuckets - 1)) : (uint32_t)kSortBuckets + lane;
    const uint32_t peers = __match_any_sync(0xffffffffu, dig);
    const uint32_t before = __popc(peers & ((1u << lane) - 1u));
    const int leader = __ffs(peers) - 1;
    if (valid && lane == leader) wcnt[warp][dig] = __popc(peers);
    __syncthreads();
    for (int b = t; b < kSortBuckets; b += blockDim.x) {
      uint32_t run = 0;
      for (int w = 0; w < kWarps; ++w) {
        const uint32_t x = wcnt[w][b];
        wcnt[w][b] = run;
        run += x;
      }
      total[b] = run;
    }
    __syncthreads();
    if (valid) {
      const uint32_t pos = base[dig] + wcnt[warp][dig] + before;
      if (pos < (uint32_t)n) {  // always true for a consistent count table
        kout[pos] = k;
        vout[pos] = v;
      }
    }
    __syncthreads();
    for (int b = t; b < kSortBuckets; b += blockDim.x) {
      base[b] += total[b];
      for (int w = 0; w < kWarps; ++w) wcnt[w][b] = 0;
    }
    __syncthreads();
  }
}

}  // namespace

void radix_sort_pairs(uint32_t *key[2], uint32_t *val[2], uint32_t *hist, int n, int passes,
                      int blocks, cudaStream_t st) {
  for (int p = 0; p < passes; ++p) {
    const int shift = p * kSortRadixBits;
    const int in = p & 1, out = in ^ 1;
    k_rs_hist<<<blocks, kSortThreads, 0, st>>>(key[in], n, shift, blocks, hist);
    k_rs_scan<<<1, 1024, 0, st>>>(hist, kSortBuckets * blocks);
    k_rs_scatter<<<blocks, kSortThreads, 0, st>>>(key[in], val[in], key[out], val[out], n, shift,
                                                  blocks, hist);
  }
}

}  // namespace le
