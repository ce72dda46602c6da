// Shared device-side definitions of the Lees-Edwards (LE) shear-flow MD
// library: the per-system geometry, the device-resident dynamic record, the
// particle buffer sets, the neighbour-slot encoding and the Philox4x64-10
// counter-based generator.
//
// Representation (see le_kernels.cu for the kernels that use it):
//   Particles are kept sorted by the cell they occupied at the last list
//   build (their "build cell").  Each particle stores its displacement p from
//   the reference point of its build cell, X_ref(c) = (c + 1/2) * l_cell.
//   Between builds p is NOT wrapped: a particle that crosses the top face keeps
//   its continuous (unwrapped) coordinate and velocity.  The LE wrap of Eq. 4
//   (x -= dX, z -= Lz) and the velocity jump (vx -= shear_rate*Lz) are applied
//   at every list build and at every export, when the representation is
//   re-based on new cells.  The friction of Eq. 5 acts on v - v_s(z) with z
//   the same unwrapped coordinate, which is the wrapped peculiar velocity
//   exactly (both v and v_s shift by shear_rate*Lz across the face).
//
//   In FP32 mode the pair loop reads a second, derived copy of p: q, the
//   displacement in int32 fixed point of 2^-S (S = Geom::qshift, 27 for the
//   usual cells), rounded from the double-float p = hi + lo.  A pair's
//   separation in those units, q_i - q_j + off(slot) with integer cell
//   edges and cross-face shift, is exact integer arithmetic; its one rounding
//   is the conversion to float.  FP32 storage of p itself (24 bits) would
//   round every position and every difference.
//
//   A neighbour-list entry is (j | slot << 24): slot names the image of j as
//   seen from i's build cell, as bit fields: an x-cell offset k in [-3,4]
//   (3 bits), y and z cell offsets in [-1,1] (2 bits each) and whether the
//   pair straddles the top/bottom face (1 bit).  The separation is
//   d = p_i - p_j + off(slot) with
//       off = (k*lx + cross*dcz*s(t), dcy*ly, dcz*lz),
//   s(t) = f_b + (dX(t) - dX(t_b)), f_b = dX(t_b) mod lx: the image offset of
//   Eq. 4 enters only through s(t), so the pair loop has no minimum-image
//   arithmetic and no FP64; the pair kernel decodes the offset from the bit
//   fields with a few ALU operations instead of a table lookup.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace le {

// A list or bond entry packs the neighbour's sorted index (high 24 bits) and
// its 8-bit slot code (low byte): the slot's bit fields then sit inside a
// float mantissa, so the pair loop decodes each with one logic operation.
constexpr int kIndexBits = 24;
constexpr int kSlotBits = 8;
constexpr int kNumSlots = 256;   // 8-bit slot codes (90 of them are used)
// end marker of a particle's bond entries (slot 255 is never a valid code)
constexpr uint32_t kNoBond = 0xFFFFFFFFu;
constexpr int kMaxBonds = 8;
constexpr int kMaxBins = 1024;
constexpr int64_t kMaxParticles = int64_t(1) << kIndexBits;

// Fixed-point scale of the per-step sample accumulators: integer atomics
// make the sums independent of the order in which blocks finish.
constexpr double kFix = 1073741824.0;          // 2^30
constexpr double kInvFix = 1.0 / 1073741824.0;
// per-particle vx contributions to the z-profile: 2^20 fixed point in int32
constexpr double kFixP = 1048576.0;
constexpr double kInvFixP = 1.0 / 1048576.0;

enum ErrBits : int {
  kErrBond = 1,       // a FENE bond reached R0
  kErrNonfinite = 2,  // a force or velocity is NaN/Inf
  kErrCapacity = 4,   // neighbour list overflow
  kErrSlot = 8,       // a bonded pair outside the 90-slot window
  kErrTimeout = 16,   // a bounded wait on a bulk copy gave up
  kErrRange = 32,     // a sampled profile value outside its fixed-point range
  kErrInput = 64,     // a non-finite coordinate or velocity given to the import
};
// Range of the per-particle profile values held as 2^-20 fixed point in the
// per-step integer sums: |vx| and m vy^2 beyond these are reported, not summed.
constexpr float kProfVxMax = 1000.f;
constexpr float kProfVy2Max = 2000.f;

__host__ __device__ inline int slot_code(int k, int dcy, int dcz, int cross) {
  return (k + 3) | ((dcy + 1) << 3) | ((dcz + 1) << 5) | (cross << 7);
}

__host__ __device__ inline uint32_t make_entry(int j, int slot) {
  return ((uint32_t)j << kSlotBits) | (uint32_t)slot;
}
__host__ __device__ inline int entry_index(uint32_t e) { return (int)(e >> kSlotBits); }
__host__ __device__ inline int entry_slot(uint32_t e) { return (int)(e & 0xFFu); }

__host__ __device__ inline void slot_decode(int s, int &k, int &dcy, int &dcz, int &cross) {
  k = (s & 7) - 3;
  dcy = ((s >> 3) & 3) - 1;
  dcz = ((s >> 5) & 3) - 1;
  cross = (s >> 7) & 1;
}

// Kernel constants in one precision, computed on the host so that no kernel
// evaluates FP64 divisions or square roots per thread (FP64 runs at 1/64 of
// the FP32 rate on this part).
template <class R> struct KConst {
  R half_dt_m;    // dt / (2m)
  R dt;
  R rc2;          // rc^2
  R sig2;         // sigma^2
  R eps24;        // 24 eps
  R amp;          // sqrt(24 xi kT m / dt): random-force amplitude (Eq. 5/7 pattern)
  R xim;          // xi m
  R shear;        // shear rate
  R half_Lz;
  R Lz;
  R shear_Lz;     // shear rate * Lz (velocity jump)
  R R02;          // FENE R0^2
  R fene_k;
  R ang_k;        // bending constant of Eq. 12 (0: none)
  R dpd_xi;       // DPD friction xi (Eq. 6)
  R dpd_amp;      // sqrt(24 kT xi / dt): DPD random-force amplitude (Eq. 7)
  R inv_rc;       // 1 / rc (the DPD weight of Eq. 8)
  R mass;
  R bins_per_Lz;  // nbins / Lz
};

// Constant per-system parameters, passed to every kernel by value.
struct Geom {
  double L[3];
  double shear_rate, dt, mass, kT, xi;
  double rc, skin, rl;            // rl = list radius (rc + skin)
  double eps, sigma, fene_k, fene_R0;
  double force_cap;               // > 0: LJ pair force magnitude limit (FP64 kernels)
  double lc[3];                   // cell edge
  double inv_L[3], inv_lcd[3];    // 1 / box edge, 1 / cell edge (FP64; floor_div corrects)
  double inv_volume, inv_dof;     // 1 / V and 1 / (3n - 3) (1 for one particle): sample folds
  int nc[3];                      // cells per dimension
  int ncell;
  int n, npad;                    // particles, n rounded up to 32
  int maxnb;                      // neighbour slots per particle
  int maxb;                       // bond slots per particle (0: no bonds)
  int thermostat, lj_shift, nbins, sample_every;
  int sort_bits;                  // bits of the largest cell index
  uint64_t seed, system;
  float rl2_build;                // (rl (1 + 1e-5))^2: list radius with a rounding margin
  float inv_lc[3];                // 1 / cell edge
  float half_lc_f[3];             // half cell edge with a rounding margin (list pruning)
  float lc_hi[3], lc_lo[3];       // cell edge as an unevaluated float sum
  // FP32 fixed-point positions q (units of 2^-qshift): cell edges in those
  // units and the largest |p| component the units can hold with the pair
  // separations (beyond it the step reports LE_ERR_RANGE)
  int qshift;
  int qL[3];
  float qmax;
  KConst<float> cf;
  KConst<double> cd;
};

template <class R> __device__ __forceinline__ const KConst<R> &kc(const Geom &g);
template <> __device__ __forceinline__ const KConst<float> &kc<float>(const Geom &g) { return g.cf; }
template <> __device__ __forceinline__ const KConst<double> &kc<double>(const Geom &g) { return g.cd; }

// Device-resident dynamic record of one system (one per handle).
struct Dyn {
  long long step;        // current integer step n
  long long build_step;  // step of the last list build
  double dX;             // dX(step)
  double dX_build;       // dX(build_step)
  double f_build;        // dX(build_step) - m_build * lx, in [0, lx)
  double s;              // continuous cross-face shift of this step
  float s_f;             // s rounded to float
  int s_q;               // s in FP32 fixed-point position units (2^-qshift)
  float f_hi, f_lo;      // f_build as an unevaluated float sum (FP32 re-basing)
  int m_build;
  int win_lo[2], win_hi[2];  // x-cell window of rows across the top/bottom face, [dcz=-1, dcz=+1]
  int cur;               // buffer set holding the current state
  int qpar;              // 1: the current fixed-point copy is q2 (FP32)
  int qflip;             // set by a fused pair+drift launch: swap q and q2 at the next decision
  unsigned maxdisp2;     // float bits of the largest squared peculiar displacement since the build
  int rebuild;           // 1 if this step rebuilt the lists
  int err;               // ErrBits
  int list_max;          // largest neighbour count at a build
  int force_rebuild;     // set by the host to force the next step to rebuild
  int pending;           // per-step accumulators hold an unfolded sample
  long long nrebuild, nimage;
  long long list_entries;        // neighbour entries written by the last build
  long long acc_sxz, acc_ke;     // per-step fixed-point sums (see kFix)
  double sum_sxz, sum_tpec;      // running sums over samples
  long long nsamples;
  double off[kNumSlots][4];      // slot offsets of this step
  double off_build[kNumSlots][4];// slot offsets at the last build (s = f_build)
};

struct alignas(32) D4 {
  double x, y, z, w;
};

template <class R> struct Vec;
template <> struct Vec<float> { using T = float4; };
template <> struct Vec<double> { using T = D4; };

// One complete copy of the per-particle state, in cell-sorted order.
template <class R> struct Bufs {
  typename Vec<R>::T *p;   // displacement from the build-cell reference; w = z of that reference
  float4 *plo;             // FP32 mode: low parts of p (x,y,z); unused in FP64 mode
  typename Vec<R>::T *v;   // velocity (unwrapped representation)
  typename Vec<R>::T *ft;  // total force of Eq. 5 (for the next half kick)
  typename Vec<R>::T *fc;  // conservative force (LJ + FENE)
  float4 *pb;              // p at the last build (x,y,z); w = build cell id (int bits)
  int *gid;                // caller's particle id
  int4 *q;                 // FP32 mode: p in fixed point (x,y,z); w = bits of p.w (float)
  int4 *q2;                // FP32 mode: second fixed-point copy (Dyn::qpar names the current one)
};

// Shared (not double-buffered) work arrays of one system.
struct Work {
  uint32_t *nbr;           // [npad/32][maxnb][32] neighbour entries
  int *ncount;             // [n]
  int *cell_start;         // [ncell + 1]
  uint32_t *bond_e;        // [n][maxb] bond entries of sorted slots (kNoBond: none)
  int *bond_gid;           // [n][maxb] bond partners by particle id (-1: none)
  int *rank;               // [n] sorted slot of each particle id
  void *tmp_p;             // [n] re-based displacement (Vec<R>), pre-sort order
  float4 *tmp_lo;          // [n] FP32 mode: its low parts
  double *Xs;              // [3n] FP64 build positions, sorted order (bonded systems)
  void *vnew;              // [n] DPD: kicked velocities (Vec<R>), copied back after the pair kernel
  uint32_t *key[2], *val[2];  // radix-sort ping-pong buffers
  uint32_t *hist;          // radix-sort digit counts
  long long *acc_prof;     // [3*nbins] per-step fixed-point vx sums, counts, m vy^2 sums
  double *sum_prof;        // [2*nbins] running vx sums, then m vy^2 sums
  long long *cnt_prof;     // [nbins] running counts
};

template <class R>
__device__ __forceinline__ Bufs<R> pick(int cur, const Bufs<R> &a, const Bufs<R> &b) {
  Bufs<R> r;
  r.p = cur ? b.p : a.p;
  r.plo = cur ? b.plo : a.plo;
  r.v = cur ? b.v : a.v;
  r.ft = cur ? b.ft : a.ft;
  r.fc = cur ? b.fc : a.fc;
  r.pb = cur ? b.pb : a.pb;
  r.gid = cur ? b.gid : a.gid;
  r.q = cur ? b.q : a.q;
  r.q2 = cur ? b.q2 : a.q2;
  return r;
}

// The buffer set with q naming the fixed-point copy of the current positions
// and q2 the other one (a pair kernel fused with the next drift reads q and
// writes the drifted copy to q2; the next step decision swaps them).
template <class R>
__device__ __forceinline__ Bufs<R> with_cur_q(Bufs<R> b, int qpar) {
  if (qpar) {
    int4 *t = b.q;
    b.q = b.q2;
    b.q2 = t;
  }
  return b;
}

// Image offset of Eq. 4 at integer step n, in [0, Lx).
__device__ __forceinline__ double image_offset(const Geom &g, long long n) {
  double t = (double)n * g.dt;
  double d = fmod(g.shear_rate * g.L[2] * t, g.L[0]);
  if (d < 0.0) d += g.L[0];
  return d;
}

// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of the
// multiply-xor bijection; the two key words advance by the Weyl constants
// (golden ratio and sqrt(3) - 1, scaled to 2^64) between rounds.
__device__ __forceinline__ void philox4x64_10(uint64_t c[4], uint64_t k0, uint64_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B97F4A7C15ull;
      k1 += 0xBB67AE8584CAA73Bull;
    }
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    uint64_t hi0 = __umul64hi(M0, c[0]), lo0 = M0 * c[0];
    uint64_t hi1 = __umul64hi(M1, c[2]), lo1 = M1 * c[2];
    uint64_t n0 = hi1 ^ c[1] ^ k0;
    uint64_t n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
  }
}

// Three uniforms on [-1/2, 1/2) for particle `gid` at step `n`, key
// (seed, system), counter (n, gid, 0, 0).  FP64: the top 53 bits of each word;
// FP32: the top 24 bits (both conversions are exact).
template <class R>
__device__ __forceinline__ void uniform3(const Geom &g, long long n, int gid, R u[3]) {
  uint64_t c[4] = {(uint64_t)n, (uint64_t)(uint32_t)gid, 0ull, 0ull};
  philox4x64_10(c, g.seed, g.system);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    if constexpr (sizeof(R) == 8)
      u[k] = (double)(c[k] >> 11) * 0x1.0p-53 - 0.5;
    else
      u[k] = (float)(uint32_t)(c[k] >> 40) * 0x1.0p-24f - 0.5f;
  }
}

// DPD pair noise theta_ij (Eq. 7): shared by the two members of a pair,
// counter (step, min id, max id, 1) -- the 1 keeps it apart from the
// Langevin stream -- first output word mapped like uniform3.
template <class R>
__device__ __forceinline__ R pair_uniform(const Geom &g, long long n, int a, int b) {
  const uint32_t lo = (uint32_t)min(a, b), hi = (uint32_t)max(a, b);
  uint64_t c[4] = {(uint64_t)n, (uint64_t)lo, (uint64_t)hi, 1ull};
  philox4x64_10(c, g.seed, g.system);
  if constexpr (sizeof(R) == 8)
    return (double)(c[0] >> 11) * 0x1.0p-53 - 0.5;
  else
    return (float)(uint32_t)(c[0] >> 40) * 0x1.0p-24f - 0.5f;
}

}  // namespace le
