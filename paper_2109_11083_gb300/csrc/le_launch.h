// Host-side launchers of the LE kernels (implemented in le_kernels.cu and
// le_sort.cu) and the device-side description of one system.
#pragma once

#include <algorithm>
#include <cmath>

#include "le_common.cuh"

namespace le {

constexpr int kDriftThreads = 256;
// Largest block sizes of the pair and list kernels (static shared arrays and
// launch bounds); the sizes a system launches with are SysDev::force_threads
// and SysDev::list_threads, which the autotuner may lower.
constexpr int kForceThreads = 256;
constexpr int kListMaxThreads = 256;
constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;   // keys per thread and sort tile
constexpr int kSortMaxDigitBits = 9;
constexpr int kSortBuckets = 1 << kSortMaxDigitBits;

struct SysDev {
  Geom g;
  Dyn *dyn = nullptr;
  Bufs<float> f32[2];
  Bufs<double> f64[2];
  Work w;
  int prec = 0;         // 0: FP64, 1: FP32
  int force_threads = 256;  // pair-kernel block (multiple of 32, <= kForceThreads)
  int list_threads = 128;   // list-build block (multiple of 32, <= kListMaxThreads)
  int sort_passes = 1;  // radix passes; the sorted keys end in buffer (sort_passes & 1)
  int sort_blocks = 1;
  uint32_t *sort_part = nullptr;  // chunk sums of the count-table scan
  double *stage = nullptr;   // [6n] host<->device staging (caller order)
  double *partials = nullptr;// [observe blocks][16]
};

inline int blocks_for(int n, int threads) { return (n + threads - 1) / threads; }

// FP32 fixed-point position units of a system with cells lc[] already chosen:
// 2^-S with S the largest shift (at most 27) whose int32 range holds every
// displacement from a build-cell centre that the rebuild trigger allows --
// half a cell, the peculiar drift (skin / 2) and the streaming along x of
// a particle at the top or bottom face until the trigger's shear term fires
// (|shear| tau rc < skin, so at most skin Lz / (2 rc)) -- and every list
// separation (< rc + 2 skin), with a factor 2 to spare.
inline void set_fixed_point(Geom &g) {
  double lmax = std::max(g.lc[0], std::max(g.lc[1], g.lc[2]));
  double pmax = 0.5 * lmax + g.skin + (g.shear_rate != 0.0 ? g.skin * g.L[2] / (2.0 * g.rc) : 0.0);
  pmax = std::max(pmax, g.rl + 2.0 * g.skin);
  pmax = std::max(pmax, g.fene_R0 + g.skin);
  int S = 27;
  while (S > 8 && 2.0 * pmax * std::ldexp(1.0, S) >= 2147483647.0) --S;
  g.qshift = S;
  for (int a = 0; a < 3; ++a) g.qL[a] = (int)std::llrint(std::ldexp(g.lc[a], S));
  g.qmax = (float)(2147483647.0 / 2.0 * std::ldexp(1.0, -S));
}

void launch_drift(const SysDev &s, cudaStream_t st);
// use_cond: set the graph's conditional handle h (0 when launched outside a graph)
void launch_decide(const SysDev &s, cudaGraphConditionalHandle h, int use_cond, cudaStream_t st);
// Rebuild pipeline.  from_import: positions come from the import staging
// (launch_import already binned them); otherwise the current state is re-based.
void launch_rebuild(const SysDev &s, bool from_import, cudaStream_t st);
// Re-creates the slot tables, the neighbour list and the bond entries of the
// current set from its stored build record (checkpoint restore, rollback).
void launch_relist(const SysDev &s, cudaStream_t st);
// mode 0: a normal step (forces, thermostat, second half kick, samples);
// mode 1: initial forces only (velocity unchanged, no samples);
// mode 2: mode 0 followed by the next step's kick and drift of each particle
//         (FP32 without DPD only: can_fuse_drift), forces not stored.
void launch_force(const SysDev &s, int mode, cudaStream_t st);
// failure-detection self-test: out[0] = 1 once a wait on a barrier that
// nothing completes has given up (the pair kernel's bounded wait)
void launch_wait_probe(int *out, cudaStream_t st);
// whether launch_force may run mode 2 for this system
bool can_fuse_drift(const SysDev &s);
void launch_fold(const SysDev &s, cudaStream_t st);
// reads stage[0:3n] pos, [3n:6n] vel; particles [i0, i1) (i1 < 0: to n)
void launch_import(const SysDev &s, cudaStream_t st, int i0 = 0, int i1 = -1);
void launch_export(const SysDev &s, cudaStream_t st);     // writes stage: pos, vel; and fc into partial-free area
// positions and velocities of caller ids [g0, g1) into the staging buffer
void launch_export_ids(const SysDev &s, cudaStream_t st, int g0, int g1);
void launch_export_forces(const SysDev &s, cudaStream_t st);  // writes stage[0:3n] = Fc
int observe_blocks(const SysDev &s);
void launch_observe(const SysDev &s, cudaStream_t st);    // partials[b][0:9] stress sums, [9] epot
void launch_tables(const SysDev &s, cudaStream_t st);  // slot tables from dyn->s and dyn->f_build

int sort_passes_for(int bits);
// tiles (blocks) of one radix pass over n keys
int sort_blocks_for(int64_t n);
size_t sort_scan_parts(int blocks);
void radix_sort_pairs(uint32_t *key[2], uint32_t *val[2], uint32_t *hist, uint32_t *part, int n,
                      int bits, int blocks, cudaStream_t st);
// Digit of radix pass p for keys of `bits` bits sorted in `passes` passes.
__host__ __device__ inline void sort_pass_digit(int bits, int passes, int p, int &shift, int &width) {
  const int wmax = (bits + passes - 1) / passes;
  shift = p * wmax;
  width = bits - shift < wmax ? bits - shift : wmax;
}
// Blocks of the count-table scan of pass p (0 when the sort has no pass p).
int sort_scan_blocks(int bits, int blocks, int p);
// Whether the count table of pass p is scanned by the three-kernel scan
// (chunk sums, top level, apply) rather than in one block.
bool sort_scan_large(int bits, int blocks, int p);

// ------------------------------------------------------------ batched steps
// A batch of independent systems advances with ONE launch per kernel kind:
// every block finds its system in a per-kind prefix table of block counts
// and runs that system's own kernel body on its own data, so each member's
// trajectory is bit-identical to stepping it alone.  The rebuild kernels run
// every step with grids sized for every member; after the step decision a
// one-block kernel lists, per kind, the members that rebuild and the prefix
// of their block counts, so the first blocks of each rebuild launch are
// exactly the rebuilding members' blocks and the rest exit after two loads.
// Members of one launch share precision, bonds, thermostat kind and launch
// shapes (a group).
constexpr int kMaxSortPasses = 4;
constexpr int kActThreads = 256;  // block of kb_activate (members scanned per chunk)
enum BatchKind : int {
  kB256 = 0,   // blocks_for(n, 256): drift, bin, permute (with the ranges), bonds, vcopy
  kBForce,     // blocks_for(n, force_threads)
  kBList,      // blocks_for(n, list_threads)
  kBSort,      // sort tiles
  kBOne,       // one block per member: decide, scan top, finish
  kBScan0,     // count-table scan blocks of pass p: kBScan0 + p
  kBKinds = kBScan0 + kMaxSortPasses
};
template <class R> struct MemberDev {
  Geom g;
  Dyn *d;
  Bufs<R> s0, s1;
  Work w;
  uint32_t *sort_part;
  int sort_passes, sort_blocks;
};
struct BatchGrid {
  const void *mem = nullptr;  // MemberDev<R>[M] in device memory
  const int *off = nullptr;   // [kBKinds][M + 1] block prefix per kind, device memory
  int *act = nullptr;         // [kBKinds][batch_act_stride(M)] rebuilding members, device memory
  int M = 0;
  int blocks[kBKinds] = {};   // grid size per kind
  int prec = 1, bonds = 0, dpd = 0;
  int force_threads = 256, list_threads = 128, nbins = 1, passes = 1;
  // pass p has a member whose count table needs the three-kernel scan
  // (sort_scan_large); without one, the chunk-sum and top-level launches of
  // that pass are left out (every table is scanned in one block)
  bool scan_large[kMaxSortPasses] = {};
};
// One step of every member of the group (drift, decide, gated rebuild,
// force).  drift = false skips the drift launch (the previous step's force
// launch ran it); fuse = true runs the next step's drift inside this step's
// force launch (mode 2: only where batch_can_fuse_drift).
void launch_batch_step(const BatchGrid &bg, cudaStream_t st, bool drift = true, bool fuse = false);
inline bool batch_can_fuse_drift(const BatchGrid &bg) { return bg.prec == 1 && !bg.dpd; }
void launch_batch_sort(const BatchGrid &bg, cudaStream_t st);  // gated radix sort, all passes

__device__ __forceinline__ int batch_member(const int *off, int M, int bid) {
  int lo = 0, hi = M - 1;  // the last member whose first block is <= bid
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= bid) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Rebuild table of one kind: act[0] = A, the members that rebuild this step
// (and have blocks of that kind); act[1 + a] = the a-th of them (in member
// order); act[1 + M + a] = its first block, act[1 + M + A] = their total.
__host__ __device__ constexpr int batch_act_stride(int M) { return 2 * M + 2; }
// Member m and its own block index of block bid of a rebuild launch; false
// for a block past the rebuilding members' blocks.
__device__ __forceinline__ bool batch_active(const int *act, int M, int bid, int &m, int &bx) {
  const int na = act[0];
  const int *aoff = act + 1 + M;
  if (bid >= aoff[na]) return false;  // also every block when na = 0 (aoff[0] = 0)
  const int a = batch_member(aoff, na, bid);
  m = act[1 + a];
  bx = bid - aoff[a];
  return true;
}

}  // namespace le
