// Stable LSD radix sort of (cell key, slot) pairs: the "resort" step that
// re-bins particles into cells at every list build.  Digits of up to 9 bits
// (two passes for the 18-bit cell index of a 60^3 grid), three kernels per
// pass: per-tile digit counts, a multi-block exclusive scan over the
// digit-major count table, and a stable scatter in which each tile ranks its
// keys chunk by chunk (warp match on the digit, then a per-digit prefix over
// the warps of the block).  Stability keeps the previous order of particles
// inside a cell, so the list order and every floating-point sum that follows
// it are deterministic.
#include <cuda_runtime.h>

#include <algorithm>

#include "le_launch.h"

namespace le {

namespace {

constexpr int kWarps = kSortThreads / 32;
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanChunk = kScanThreads * kScanItems;

// Keys per thread of each of the nblocks tiles (1 to kSortItems): a small
// sort runs more, shorter tiles in parallel (see sort_blocks_for).
__device__ __forceinline__ int sort_tile_items(int n, int nblocks) {
  const int per = nblocks * kSortThreads;
  return (n + per - 1) / per;
}

__device__ __forceinline__ void rs_hist_body(const uint32_t *__restrict__ key, int n, int shift,
                                             int bits, int nblocks, uint32_t *__restrict__ hist,
                                             int bx) {
  __shared__ uint32_t cnt[kSortBuckets];
  const int nb = 1 << bits;
  const uint32_t mask = (uint32_t)nb - 1u;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) cnt[b] = 0;
  __syncthreads();
  const int items = sort_tile_items(n, nblocks);
  const int base = bx * kSortThreads * items;
#pragma unroll 4
  for (int k = 0; k < items; ++k) {
    const int i = base + k * kSortThreads + threadIdx.x;
    if (i < n) atomicAdd(&cnt[(key[i] >> shift) & mask], 1u);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < nb; b += blockDim.x) hist[(size_t)b * nblocks + bx] = cnt[b];
}
__global__ void __launch_bounds__(kSortThreads) k_rs_hist(const uint32_t *__restrict__ key, int n,
                                                          int shift, int bits, int nblocks,
                                                          uint32_t *__restrict__ hist) {
  rs_hist_body(key, n, shift, bits, nblocks, hist, (int)blockIdx.x);
}

// Block-wide inclusive scan of one value per thread (1024 threads).
__device__ __forceinline__ uint32_t block_incl_scan(uint32_t v, uint32_t *warp_tot) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += y;
  }
  if (lane == 31) warp_tot[warp] = v;
  __syncthreads();
  if (warp == 0) {
    uint32_t t = warp_tot[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    warp_tot[lane] = t;
  }
  __syncthreads();
  return v + (warp > 0 ? warp_tot[warp - 1] : 0u);
}

// Pass 1 of the scan: the sum of each chunk of kScanChunk counts.
__device__ __forceinline__ void scan_sums_body(const uint32_t *__restrict__ a, int m,
                                               uint32_t *__restrict__ part, int bx) {
  __shared__ uint32_t wt[32];
  const int base = bx * kScanChunk + threadIdx.x * kScanItems;
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k)
    if (base + k < m) s += a[base + k];
  const uint32_t incl = block_incl_scan(s, wt);
  if (threadIdx.x == kScanThreads - 1) part[bx] = incl;
}
__global__ void __launch_bounds__(kScanThreads) k_scan_sums(const uint32_t *__restrict__ a, int m,
                                                            uint32_t *__restrict__ part) {
  scan_sums_body(a, m, part, (int)blockIdx.x);
}

// Pass 2: exclusive scan of the chunk sums (one block, up to 4 per thread).
__device__ __forceinline__ void scan_top_body(uint32_t *__restrict__ part, int np, int bx) {
  __shared__ uint32_t wt[32];
  const int base = threadIdx.x * 4;
  uint32_t v[4], s = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    v[k] = base + k < np ? part[base + k] : 0u;
    s += v[k];
  }
  uint32_t run = block_incl_scan(s, wt) - s;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (base + k < np) part[base + k] = run;
    run += v[k];
  }
}
__global__ void __launch_bounds__(kScanThreads) k_scan_top(uint32_t *__restrict__ part, int np) {
  scan_top_body(part, np, (int)blockIdx.x);
}

// Pass 3: exclusive scan inside each chunk, offset by the chunk's start
// (part == nullptr: a table of one chunk, scanned by this pass alone).
__device__ __forceinline__ void scan_apply_body(uint32_t *__restrict__ a, int m,
                                                const uint32_t *__restrict__ part, int bx) {
  __shared__ uint32_t wt[32];
  const int base = bx * kScanChunk + threadIdx.x * kScanItems;
  uint32_t v[kScanItems], s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = base + k < m ? a[base + k] : 0u;
    s += v[k];
  }
  uint32_t run = block_incl_scan(s, wt) - s + (part ? part[bx] : 0u);
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < m) a[base + k] = run;
    run += v[k];
  }
}
__global__ void __launch_bounds__(kScanThreads) k_scan_apply(
    uint32_t *__restrict__ a, int m, const uint32_t *__restrict__ part) {
  scan_apply_body(a, m, part, (int)blockIdx.x);
}

// A table of up to kScanSeqChunks chunks scanned by one block, chunk after
// chunk with the running total carried: one launch instead of three for a
// small sort.
constexpr int kScanSeqChunks = 8;
__device__ __forceinline__ void scan_seq_body(uint32_t *__restrict__ a, int m) {
  __shared__ uint32_t wt[32];
  __shared__ uint32_t carry;
  if (threadIdx.x == 0) carry = 0u;
  __syncthreads();
  for (int c = 0; c * kScanChunk < m; ++c) {
    const int base = c * kScanChunk + threadIdx.x * kScanItems;
    uint32_t v[kScanItems], s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      v[k] = base + k < m ? a[base + k] : 0u;
      s += v[k];
    }
    const uint32_t incl = block_incl_scan(s, wt);
    uint32_t run = incl - s + carry;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      if (base + k < m) a[base + k] = run;
      run += v[k];
    }
    __syncthreads();  // every thread has read carry and the warp totals
    if (threadIdx.x == kScanThreads - 1) carry += incl;
    __syncthreads();
  }
}
__global__ void __launch_bounds__(kScanThreads) k_scan_seq(uint32_t *__restrict__ a, int m) {
  scan_seq_body(a, m);
}

__device__ __forceinline__ void rs_scatter_body(const uint32_t *__restrict__ kin,
                                                const uint32_t *__restrict__ vin,
                                                uint32_t *__restrict__ kout,
                                                uint32_t *__restrict__ vout, int n, int shift,
                                                int bits, int nblocks,
                                                const uint32_t *__restrict__ hist, int bx) {
  __shared__ uint32_t base[kSortBuckets];          // global start of each digit for this tile
  __shared__ uint32_t wcnt[kWarps][kSortBuckets];  // per-warp counts -> per-warp offsets
  __shared__ uint32_t total[kSortBuckets];
  const int nb = 1 << bits;
  const uint32_t mask = (uint32_t)nb - 1u;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  for (int b = t; b < nb; b += blockDim.x) {
    base[b] = hist[(size_t)b * nblocks + bx];
    for (int w = 0; w < kWarps; ++w) wcnt[w][b] = 0;
  }
  __syncthreads();
  const int items = sort_tile_items(n, nblocks);
  const int tile = bx * kSortThreads * items;
  for (int c = 0; c < items; ++c) {
    const int i = tile + c * kSortThreads + t;
    const bool valid = i < n;
    const uint32_t k = valid ? kin[i] : 0u;
    const uint32_t v = valid ? vin[i] : 0u;
    // invalid lanes get a digit outside the bucket range so they never match
    const uint32_t dig = valid ? ((k >> shift) & mask) : (uint32_t)kSortBuckets + lane;
    const uint32_t peers = __match_any_sync(0xffffffffu, dig);
    const uint32_t before = __popc(peers & ((1u << lane) - 1u));
    const int leader = __ffs(peers) - 1;
    if (valid && lane == leader) wcnt[warp][dig] = __popc(peers);
    __syncthreads();
    for (int b = t; b < nb; b += blockDim.x) {
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
    for (int b = t; b < nb; b += blockDim.x) {
      base[b] += total[b];
      for (int w = 0; w < kWarps; ++w) wcnt[w][b] = 0;
    }
    __syncthreads();
  }
}
__global__ void __launch_bounds__(kSortThreads) k_rs_scatter(
    const uint32_t *__restrict__ kin, const uint32_t *__restrict__ vin, uint32_t *__restrict__ kout,
    uint32_t *__restrict__ vout, int n, int shift, int bits, int nblocks,
    const uint32_t *__restrict__ hist) {
  rs_scatter_body(kin, vin, kout, vout, n, shift, bits, nblocks, hist, (int)blockIdx.x);
}


// ------------------------------------------------------------ batched sort
// The same pass kernels for every member of a batch group in one launch.
// Each block finds its member in the kind's table of members that rebuild
// this step (act: one kind's slice, batch_active); blocks past them, and
// those of members with no pass p, exit.
template <class R>
__global__ void __launch_bounds__(kSortThreads) kb_rs_hist(const MemberDev<R> *__restrict__ mem,
                                                           const int *__restrict__ act, int M, int p) {
  int m, bx;
  if (!batch_active(act, M, (int)blockIdx.x, m, bx)) return;
  const MemberDev<R> &q = mem[m];
  if (p >= q.sort_passes) return;
  int shift, w;
  sort_pass_digit(q.g.sort_bits, q.sort_passes, p, shift, w);
  rs_hist_body(q.w.key[p & 1], q.g.n, shift, w, q.sort_blocks, q.w.hist, bx);
}

template <class R>
__global__ void __launch_bounds__(kScanThreads) kb_scan_sums(const MemberDev<R> *__restrict__ mem,
                                                             const int *__restrict__ act, int M, int p) {
  int m, bx;
  if (!batch_active(act, M, (int)blockIdx.x, m, bx)) return;
  const MemberDev<R> &q = mem[m];
  int shift, w;
  sort_pass_digit(q.g.sort_bits, q.sort_passes, p, shift, w);
  const int mm = (1 << w) * q.sort_blocks;
  if (mm <= kScanSeqChunks * kScanChunk) return;  // a small table: scan_apply's first block
  scan_sums_body(q.w.hist, mm, q.sort_part, bx);
}

template <class R>
__global__ void __launch_bounds__(kScanThreads) kb_scan_top(const MemberDev<R> *__restrict__ mem,
                                                            const int *__restrict__ act, int M, int p) {
  int m, bx;
  if (!batch_active(act, M, (int)blockIdx.x, m, bx)) return;
  const MemberDev<R> &q = mem[m];
  if (p >= q.sort_passes) return;
  int shift, w;
  sort_pass_digit(q.g.sort_bits, q.sort_passes, p, shift, w);
  const int mm = (1 << w) * q.sort_blocks;
  if (mm <= kScanSeqChunks * kScanChunk) return;
  scan_top_body(q.sort_part, (mm + kScanChunk - 1) / kScanChunk, 0);
}

template <class R>
__global__ void __launch_bounds__(kScanThreads) kb_scan_apply(const MemberDev<R> *__restrict__ mem,
                                                              const int *__restrict__ act, int M, int p) {
  int m, bx;
  if (!batch_active(act, M, (int)blockIdx.x, m, bx)) return;
  const MemberDev<R> &q = mem[m];
  int shift, w;
  sort_pass_digit(q.g.sort_bits, q.sort_passes, p, shift, w);
  const int mm = (1 << w) * q.sort_blocks;
  if (mm <= kScanSeqChunks * kScanChunk) {
    if (bx == 0) scan_seq_body(q.w.hist, mm);  // the member's whole table
    return;
  }
  scan_apply_body(q.w.hist, mm, q.sort_part, bx);
}

template <class R>
__global__ void __launch_bounds__(kSortThreads) kb_rs_scatter(const MemberDev<R> *__restrict__ mem,
                                                              const int *__restrict__ act, int M, int p) {
  int m, bx;
  if (!batch_active(act, M, (int)blockIdx.x, m, bx)) return;
  const MemberDev<R> &q = mem[m];
  if (p >= q.sort_passes) return;
  int shift, w;
  sort_pass_digit(q.g.sort_bits, q.sort_passes, p, shift, w);
  const int in = p & 1, out = in ^ 1;
  rs_scatter_body(q.w.key[in], q.w.val[in], q.w.key[out], q.w.val[out], q.g.n, shift, w,
                  q.sort_blocks, q.w.hist, bx);
}

template <class R>
void batch_sort_passes(const BatchGrid &bg, cudaStream_t st) {
  const MemberDev<R> *mem = static_cast<const MemberDev<R> *>(bg.mem);
  const int M = bg.M, S = batch_act_stride(bg.M);
  const int *act_sort = bg.act + kBSort * S, *act_one = bg.act + kBOne * S;
  for (int p = 0; p < bg.passes; ++p) {
    const int *act_scan = bg.act + (kBScan0 + p) * S;
    const int nscan = bg.blocks[kBScan0 + p];
    if (nscan == 0) continue;
    kb_rs_hist<R><<<bg.blocks[kBSort], kSortThreads, 0, st>>>(mem, act_sort, M, p);
    if (bg.scan_large[p]) {
      kb_scan_sums<R><<<nscan, kScanThreads, 0, st>>>(mem, act_scan, M, p);
      kb_scan_top<R><<<M, kScanThreads, 0, st>>>(mem, act_one, M, p);
    }
    kb_scan_apply<R><<<nscan, kScanThreads, 0, st>>>(mem, act_scan, M, p);
    kb_rs_scatter<R><<<bg.blocks[kBSort], kSortThreads, 0, st>>>(mem, act_sort, M, p);
  }
}

}  // namespace

int sort_passes_for(int bits) { return (bits + kSortMaxDigitBits - 1) / kSortMaxDigitBits; }

// Tiles of kSortThreads x items keys: items = kSortItems for a large sort,
// fewer (down to one) when that would leave fewer than ~2 tiles per SM of a
// GB300, so that a small system's passes spread over the GPU instead of
// running a few long tiles.  Any tiling gives the same stable order.
int sort_blocks_for(int64_t n) {
  const int64_t per = kSortThreads, spread = 304;
  const int64_t items = std::min<int64_t>(kSortItems, std::max<int64_t>(1, (n + per * spread - 1) / (per * spread)));
  return (int)((n + per * items - 1) / (per * items));
}

size_t sort_scan_parts(int blocks) {
  return ((size_t)kSortBuckets * blocks + kScanChunk - 1) / kScanChunk;
}

int sort_scan_blocks(int bits, int blocks, int p) {
  const int passes = sort_passes_for(bits);
  if (p >= passes) return 0;
  int shift, w;
  sort_pass_digit(bits, passes, p, shift, w);
  const int m = (1 << w) * blocks;
  return (m + kScanChunk - 1) / kScanChunk;
}

bool sort_scan_large(int bits, int blocks, int p) {
  const int passes = sort_passes_for(bits);
  if (p >= passes) return false;
  int shift, w;
  sort_pass_digit(bits, passes, p, shift, w);
  return (1 << w) * blocks > kScanSeqChunks * kScanChunk;
}

void radix_sort_pairs(uint32_t *key[2], uint32_t *val[2], uint32_t *hist, uint32_t *part, int n,
                      int bits, int blocks, cudaStream_t st) {
  const int passes = sort_passes_for(bits);
  for (int p = 0; p < passes; ++p) {
    int shift, w;
    sort_pass_digit(bits, passes, p, shift, w);
    const int in = p & 1, out = in ^ 1;
    const int m = (1 << w) * blocks;
    const int np = (m + kScanChunk - 1) / kScanChunk;
    k_rs_hist<<<blocks, kSortThreads, 0, st>>>(key[in], n, shift, w, blocks, hist);
    if (np > kScanSeqChunks) {
      k_scan_sums<<<np, kScanThreads, 0, st>>>(hist, m, part);
      k_scan_top<<<1, kScanThreads, 0, st>>>(part, np);
      k_scan_apply<<<np, kScanThreads, 0, st>>>(hist, m, part);
    } else {
      k_scan_seq<<<1, kScanThreads, 0, st>>>(hist, m);  // a small table: one block
    }
    k_rs_scatter<<<blocks, kSortThreads, 0, st>>>(key[in], val[in], key[out], val[out], n, shift,
                                                  w, blocks, hist);
  }
}

void launch_batch_sort(const BatchGrid &bg, cudaStream_t st) {
  if (bg.prec == 1) batch_sort_passes<float>(bg, st);
  else batch_sort_passes<double>(bg, st);
}

}  // namespace le

// ---------------------------------------------------------------- C entry
// The resort step on its own: a stable sort of cell keys, returning the
// permutation (see le_sort_cell_keys in le.h).
#include <vector>

#include "../../include/le.h"

extern "C" LE_API le_status le_sort_cell_keys(int64_t n, const uint32_t *keys, int bits,
                                              uint32_t *order, uint32_t *sorted_keys,
                                              void *cuda_stream) {
  using namespace le;
  if (n < 1 || n > kMaxParticles || !keys || !order || bits < 1 || bits > 32)
    return LE_ERR_INVALID_ARG;
  if (bits < 32)
    for (int64_t i = 0; i < n; ++i)
      if (keys[i] >> bits) return LE_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int blocks = sort_blocks_for(n);
  const size_t nb = sizeof(uint32_t) * (size_t)n;
  uint32_t *buf = nullptr;  // key[0], key[1], val[0], val[1], hist, part
  const size_t hist = (size_t)kSortBuckets * blocks, part = sort_scan_parts(blocks);
  const size_t words = 4 * (size_t)n + hist + part;
  if (cudaMalloc(&buf, words * sizeof(uint32_t)) != cudaSuccess) {
    cudaGetLastError();
    return LE_ERR_OOM;
  }
  uint32_t *key[2] = {buf, buf + n}, *val[2] = {buf + 2 * n, buf + 3 * n};
  std::vector<uint32_t> iota((size_t)n);
  for (int64_t i = 0; i < n; ++i) iota[(size_t)i] = (uint32_t)i;
  cudaError_t e = cudaMemcpyAsync(key[0], keys, nb, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(val[0], iota.data(), nb, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    radix_sort_pairs(key, val, buf + 4 * n, buf + 4 * n + hist, (int)n, bits, blocks, st);
    e = cudaGetLastError();
  }
  const int res = sort_passes_for(bits) & 1;
  if (e == cudaSuccess) e = cudaMemcpyAsync(order, val[res], nb, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && sorted_keys)
    e = cudaMemcpyAsync(sorted_keys, key[res], nb, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(buf);
  return e == cudaSuccess ? LE_OK : LE_ERR_CUDA;
}
