// CUDA kernels of the Lees-Edwards shear-flow MD step (sm_103a).
//
// One step n -> n+1 (velocity Verlet, the order of every implementation in
// this repository):
//   k_drift   v += dt/2m Ftot(n); r += dt v; max displacement since the build
//   k_decide  dX(n+1) from the integer step (Eq. 4); rebuild trigger
//             2*max|dr| + |shift of the sheared images since the build| >= skin;
//             per-step slot-offset table; folds the previous step's samples
//   [if rebuild: k_rb_bin -> radix sort -> k_rb_permute (and cell ranges) ->
//                k_rb_list -> k_rb_bonds -> k_rb_finish]
//   k_force   LJ (Eq. 9/10) over the Verlet list + FENE (Eq. 11) under the LE
//             minimum image; Ftot = Fc - xi m (v - v_s e_x) + random (Eq. 5);
//             v += dt/2m Ftot; Eq. 15 xz stress, peculiar temperature and the
//             vx(z) profile as fixed-point integer sums.
// Inside a multi-step graph (FP32 without DPD) k_force of step n also runs the
// k_drift of step n+1 for its own particle (mode 2): neighbours are read only
// through the fixed-point copy q, so the drifted copy goes to a second array
// q2, and k_decide swaps the two.  Same arithmetic, same results.
#include <cuda_runtime.h>

#include "le_common.cuh"
#include "le_launch.h"

namespace le {

namespace {

template <class R> using V4 = typename Vec<R>::T;

__device__ __forceinline__ float4 load4(const float4 *p) { return __ldg(p); }
__device__ __forceinline__ D4 load4(const D4 *p) { return *p; }

template <class R> __device__ __forceinline__ V4<R> make4(R x, R y, R z, R w) {
  V4<R> v;
  v.x = x;
  v.y = y;
  v.z = z;
  v.w = w;
  return v;
}

// Rounded operations that the compiler may not contract into FMAs: the DPD
// pair arithmetic and the thermostat's streaming velocity are written
// with them so that every kernel that inlines them (a system's own step, a
// batch launch) computes the same bits.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

// hi + lo += a with the rounding error of the sum kept in lo (TwoSum followed
// by a renormalisation): ~48 significant bits for the displacement.
__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float a) {
  float s = __fadd_rn(hi, a);
  float bb = __fsub_rn(s, hi);
  float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(a, bb));
  lo = __fadd_rn(lo, e);
  hi = __fadd_rn(s, lo);
  lo = __fsub_rn(lo, __fsub_rn(hi, s));
}

// FP32 fixed-point copy of a displacement hi + lo: each part scaled by 2^S
// (exact) and rounded to an integer, so the copy is p rounded to 2^-S within
// one unit; w carries the bits of hi.w (the build cell's reference z).
__device__ __forceinline__ int4 quantize(const Geom &g, const float4 &hi, const float4 &lo) {
  const float sc = __int_as_float((127 + g.qshift) << 23);  // 2^S
  int4 q;
  q.x = __float2int_rn(hi.x * sc) + __float2int_rn(lo.x * sc);
  q.y = __float2int_rn(hi.y * sc) + __float2int_rn(lo.y * sc);
  q.z = __float2int_rn(hi.z * sc) + __float2int_rn(lo.z * sc);
  q.w = __float_as_int(hi.w);
  return q;
}

__device__ __forceinline__ void cell_coords(const Geom &g, int c, int &cx, int &cy, int &cz) {
  cx = c % g.nc[0];
  int r = c / g.nc[0];
  cy = r % g.nc[1];
  cz = r / g.nc[1];
}

// FP64 position of a sorted slot: build-cell reference + displacement.
template <class R>
__device__ __forceinline__ void absolute_position(const Geom &g, const Bufs<R> &b, int i,
                                                  double x[3]) {
  const float4 q = b.pb[i];
  int cx, cy, cz;
  cell_coords(g, __float_as_int(q.w), cx, cy, cz);
  const V4<R> p = b.p[i];
  x[0] = ((double)cx + 0.5) * g.lc[0] + (double)p.x;
  x[1] = ((double)cy + 0.5) * g.lc[1] + (double)p.y;
  x[2] = ((double)cz + 0.5) * g.lc[2] + (double)p.z;
  if constexpr (sizeof(R) == 4) {
    const float4 lo = b.plo[i];
    x[0] += (double)lo.x;
    x[1] += (double)lo.y;
    x[2] += (double)lo.z;
  }
}

// floor(x / L) from a multiplication by 1/L, corrected so that the
// remainder x - k L lies in [0, L): FP64 division is a long instruction
// sequence on this GPU, a multiply and an FMA are not.
__device__ __forceinline__ double floor_div(double x, double L, double invL) {
  double k = floor(x * invL);
  const double r = fma(-k, L, x);
  if (r < 0.0) k -= 1.0;
  else if (r >= L) k += 1.0;
  return k;
}

// LE wrap of Eq. 4 at image offset dX: through the top face z -= Lz,
// x -= dX, vx -= shear_rate*Lz; through the bottom face the mirror image;
// x and y periodic.  Returns the z image index that was removed.
__device__ __forceinline__ int le_wrap(const Geom &g, double dX, double x[3], double &vx) {
  const double Lx = g.L[0], Ly = g.L[1], Lz = g.L[2];
  int nz = 0;
  if (x[2] >= Lz) {
    x[2] -= Lz;
    x[0] -= dX;
    vx -= g.shear_rate * Lz;
    nz = 1;
  } else if (x[2] < 0.0) {
    double zz = x[2] + Lz;
    if (zz < Lz) {
      x[2] = zz;
      x[0] += dX;
      vx += g.shear_rate * Lz;
      nz = -1;
    } else {
      x[2] = 0.0;  // within rounding of the bottom face: no image change
    }
  }
  x[0] -= Lx * floor_div(x[0], Lx, g.inv_L[0]);
  if (x[0] >= Lx) x[0] -= Lx;
  x[1] -= Ly * floor_div(x[1], Ly, g.inv_L[1]);
  if (x[1] >= Ly) x[1] -= Ly;
  return nz;
}

__device__ __forceinline__ int cell_of(const Geom &g, const double x[3]) {
  int c[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int k = (int)floor_div(x[a], g.lc[a], g.inv_lcd[a]);
    c[a] = k < 0 ? 0 : (k >= g.nc[a] ? g.nc[a] - 1 : k);
  }
  return c[0] + g.nc[0] * (c[1] + g.nc[1] * c[2]);
}

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block index of a kernel body: the hardware register for a system's own
// launch, a stored value for a batched launch (member-relative index).
struct HwBlock {
  __device__ __forceinline__ int operator()() const { return (int)blockIdx.x; }
};
struct VBlock {
  int b;
  __device__ __forceinline__ int operator()() const { return b; }
};

// ------------------------------------------------------------------ k_drift
// First half kick of particle i with the total force f, drift, and (FP32) the
// fixed-point copy of the new position written to qout[i].  Returns the
// squared peculiar displacement since the build: the streaming
// shear*tau*(z_b - Lz/2) along x (z_b = build-time z = reference + build
// displacement) is shared by neighbours and does not use up the skin.
template <class R>
__device__ __forceinline__ float kick_drift(const Geom &g, Dyn *__restrict__ d, const Bufs<R> &b,
                                            int4 *qout, int i, V4<R> v, const V4<R> &f,
                                            float shear_tau) {
  const R half = kc<R>(g).half_dt_m;
  const R dt = kc<R>(g).dt;
  // explicit fma (and explicitly rounded products below) wherever a product
  // meets a sum: every kernel that inlines this code (a system's own step, a
  // batch launch, fused with the pair kernel or not) then rounds alike, and
  // their results stay bit-identical
  v.x = fma(half, f.x, v.x);
  v.y = fma(half, f.y, v.y);
  v.z = fma(half, f.z, v.z);
  V4<R> p = b.p[i];
  if constexpr (sizeof(R) == 4) {
    float4 lo = b.plo[i];
    two_sum_acc(p.x, lo.x, dt * v.x);
    two_sum_acc(p.y, lo.y, dt * v.y);
    two_sum_acc(p.z, lo.z, dt * v.z);
    b.plo[i] = lo;
    // a displacement beyond the fixed-point range is reported (LE_ERR_RANGE)
    if (!(fmaxf(fabsf(p.x), fmaxf(fabsf(p.y), fabsf(p.z))) < g.qmax))
      atomicOr(&d->err, (int)kErrRange);
    qout[i] = quantize(g, p, lo);
  } else {
    p.x = fma(dt, v.x, p.x);
    p.y = fma(dt, v.y, p.y);
    p.z = fma(dt, v.z, p.z);
  }
  b.v[i] = v;
  b.p[i] = p;
  const float4 q = b.pb[i];
  const float zb = (float)p.w + q.z;
  const float dx = fmaf(-shear_tau, zb - (float)kc<R>(g).half_Lz, (float)p.x - q.x);
  const float dy = (float)p.y - q.y, dz = (float)p.z - q.z;
  return fmaf(dz, dz, fmaf(dy, dy, dx * dx));
}

// Largest value of v over the block, folded into d->maxdisp2 (one atomic per
// block; all threads of the block call it).
template <int NWARPS>
__device__ __forceinline__ void block_max_disp(Dyn *__restrict__ d, float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  __shared__ float sm[NWARPS];
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    float m = sm[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, sm[w]);
    if (m > 0.f) atomicMax(&d->maxdisp2, __float_as_uint(m));
  }
}

// time since the build at the step a drift from the current step produces
__device__ __forceinline__ float drift_shear_tau(const Geom &g, const Dyn *__restrict__ d) {
  return g.cf.shear * (float)(d->step + 1 - d->build_step) * g.cf.dt;
}

template <class R>
__device__ __forceinline__ void drift_body(const Geom g, Dyn *__restrict__ d, Bufs<R> s0,
                                           Bufs<R> s1, int bx) {
  const Bufs<R> b = with_cur_q(pick(d->cur, s0, s1), d->qpar);
  const int i = bx * blockDim.x + threadIdx.x;
  const float shear_tau = drift_shear_tau(g, d);
  float disp2 = 0.f;
  if (i < g.n) disp2 = kick_drift<R>(g, d, b, b.q, i, b.v[i], b.ft[i], shear_tau);
  block_max_disp<kDriftThreads / 32>(d, disp2);
}
template <class R>
__global__ void __launch_bounds__(kDriftThreads) k_drift(const __grid_constant__ Geom g,
                                                         Dyn *__restrict__ d, Bufs<R> s0, Bufs<R> s1) {
  drift_body<R>(g, d, s0, s1, (int)blockIdx.x);
}

// x-cell window of the neighbour rows across the top/bottom face for a build
// with f_b = dX(t_b) mod lx: every cell whose image lies within rl of the
// shifted row (3 or 4 cells; index 0 for dcz = -1, 1 for dcz = +1).
// x-cell window of a neighbour row across the top/bottom face (z offset dcz)
// for a build with f_b = dX(t_b) mod lx: candidate j in x cell k has d_x
// within one cell edge of off(k) = k lx + dcz f_b, and d_x must reach
// (-rl, rl): 3 or 4 cells.
__device__ __forceinline__ void cross_window(const Geom &g, double fb, Dyn *d) {
  const double lx = g.lc[0];
  const double margin = 1e-5 * g.rl + 1e-9;
  for (int side = 0; side < 2; ++side) {
    const int dcz = side ? 1 : -1;
    const double lower = -g.rl - margin;
    const double upper = g.rl + margin;
    // k lx + dcz fb + lx > lower  and  k lx + dcz fb - lx < upper
    int kmin = (int)floor((lower - lx - dcz * fb) / lx) + 1;
    int kmax = (int)ceil((upper + lx - dcz * fb) / lx) - 1;
    d->win_lo[side] = max(kmin, -3);
    d->win_hi[side] = min(kmax, 4);
  }
}

// ------------------------------------------------------------------ k_decide
// One block.  Folds the previous step's fixed-point samples into the running
// sums, advances the step, evaluates the rebuild trigger and fills the slot
// offset table.
__device__ __forceinline__ void decide_body(const Geom g, Dyn *__restrict__ d, Work w,
                                            cudaGraphConditionalHandle h, int use_cond, int bx) {
  __shared__ double s_sh;
  __shared__ int need_sh;
  const int t = threadIdx.x;
  const int pending = d->pending;
  if (pending) {
    for (int b = t; b < g.nbins; b += blockDim.x) {
      w.sum_prof[b] += (double)w.acc_prof[b] * kInvFixP;
      w.sum_prof[g.nbins + b] += (double)w.acc_prof[2 * g.nbins + b] * kInvFixP;
      w.cnt_prof[b] += w.acc_prof[g.nbins + b];
      w.acc_prof[b] = 0;
      w.acc_prof[g.nbins + b] = 0;
      w.acc_prof[2 * g.nbins + b] = 0;
    }
  }
  __syncthreads();
  if (t == 0) {
    // every field this thread reads, loaded together before the first store
    const int qflip = d->qflip, qpar = d->qpar;
    const long long acc_sxz = d->acc_sxz, acc_ke = d->acc_ke;
    const long long n1 = d->step + 1;
    const unsigned maxdisp2 = d->maxdisp2;
    const double dX_build = d->dX_build, f_build = d->f_build;
    const long long build_step = d->build_step;
    const int force_rebuild = d->force_rebuild;
    // a pair kernel fused with the drift wrote the new positions to q2
    if (qflip) {
      d->qpar = qpar ^ 1;
      d->qflip = 0;
    }
    if (pending) {
      // 1 / V and 1 / (3n - 3) come with the geometry (no FP64 division here)
      d->sum_sxz += -(double)acc_sxz * kInvFix * g.inv_volume;
      d->sum_tpec += (double)acc_ke * kInvFix * g.inv_dof;
      d->nsamples += 1;
      d->acc_sxz = 0;
      d->acc_ke = 0;
      d->pending = 0;
    }
    const double dX1 = image_offset(g, n1);
    const float maxd = sqrtf(__uint_as_float(maxdisp2));
    d->maxdisp2 = 0u;
    // continuous change of the image offset since the build (dX is reduced
    // modulo Lx; the shear sign tells which way it wrapped)
    double ds = dX1 - dX_build;
    if (g.shear_rate > 0.0 && ds < -0.5 * g.L[0]) ds += g.L[0];
    if (g.shear_rate < 0.0 && ds > 0.5 * g.L[0]) ds -= g.L[0];
    const double margin = 1e-6 * g.rl;
    const bool disp_need = 2.0 * (double)maxd * (1.0 + 1e-6) + margin >= g.skin;
    // maxd is the largest PECULIAR displacement w since the build (streaming
    // along the profile of Eq. 1 removed).  A pair's separation changes by
    // w_i - w_j + shear*tau*dz_build e_x; pairs across the face included,
    // since the drift of the image offset cancels their streaming
    // difference.  A pair that can reach rc has |dz_build| < rc + 2 maxd.
    const double tau = (double)(n1 - build_step) * g.dt;
    const double shear_term = fabs(g.shear_rate) * tau * (g.rc + 2.0 * (double)maxd);
    const bool need = force_rebuild || disp_need ||
                      (2.0 * (double)maxd * (1.0 + 1e-6) + shear_term + margin >= g.skin);
    double s;
    if (need) {
      int m = (int)floor(dX1 * g.inv_lcd[0]);  // corrected to [0, lx) below
      double f = dX1 - (double)m * g.lc[0];
      if (f >= g.lc[0]) { f -= g.lc[0]; m += 1; }
      if (f < 0.0) { f += g.lc[0]; m -= 1; }
      d->m_build = m;
      d->f_build = f;
      d->f_hi = (float)f;
      d->f_lo = (float)(f - (double)d->f_hi);
      d->dX_build = dX1;
      d->build_step = n1;
      d->list_entries = 0;
      cross_window(g, f, d);
      d->nrebuild += 1;
      if (!disp_need && !force_rebuild) d->nimage += 1;
      s = f;
    } else {
      s = f_build + ds;
    }
    d->s = s;
    d->s_f = (float)s;
    d->s_q = (int)llrint(ldexp(s, g.qshift));
    d->dX = dX1;
    d->step = n1;
    d->rebuild = need ? 1 : 0;
    d->force_rebuild = 0;
    s_sh = s;
    need_sh = need ? 1 : 0;
    if (use_cond) cudaGraphSetConditional(h, need ? 1u : 0u);
  }
  __syncthreads();
  const double s = s_sh;
  for (int e = t; e < kNumSlots; e += blockDim.x) {
    int k, dcy, dcz, cross;
    slot_decode(e, k, dcy, dcz, cross);
    const double ox = (double)k * g.lc[0] + (cross ? (double)dcz * s : 0.0);
    const double oy = (double)dcy * g.lc[1];
    const double oz = (double)dcz * g.lc[2];
    d->off[e][0] = ox;
    d->off[e][1] = oy;
    d->off[e][2] = oz;
    d->off[e][3] = 0.0;
    if (need_sh) {
      d->off_build[e][0] = ox;
      d->off_build[e][1] = oy;
      d->off_build[e][2] = oz;
      d->off_build[e][3] = 0.0;
    }
  }
}
__global__ void __launch_bounds__(128) k_decide(const __grid_constant__ Geom g, Dyn *__restrict__ d,
                                                Work w, cudaGraphConditionalHandle h, int use_cond) {
  decide_body(g, d, w, h, use_cond, (int)blockIdx.x);
}

// Folds pending samples outside the step graph (end of a le_step call).
__global__ void k_fold(Geom g, Dyn *__restrict__ d, Work w) {
  const int t = threadIdx.x;
  const int pending = d->pending;
  if (pending) {
    for (int b = t; b < g.nbins; b += blockDim.x) {
      w.sum_prof[b] += (double)w.acc_prof[b] * kInvFixP;
      w.sum_prof[g.nbins + b] += (double)w.acc_prof[2 * g.nbins + b] * kInvFixP;
      w.cnt_prof[b] += w.acc_prof[g.nbins + b];
      w.acc_prof[b] = 0;
      w.acc_prof[g.nbins + b] = 0;
      w.acc_prof[2 * g.nbins + b] = 0;
    }
  }
  __syncthreads();
  if (t == 0 && pending) {
    // the same arithmetic as the fold in k_decide
    d->sum_sxz += -(double)d->acc_sxz * kInvFix * g.inv_volume;
    d->sum_tpec += (double)d->acc_ke * kInvFix * g.inv_dof;
    d->nsamples += 1;
    d->acc_sxz = 0;
    d->acc_ke = 0;
    d->pending = 0;
  }
}

// ------------------------------------------------------------------ k_force
// Bulk-copy (TMA, cp.async.bulk) helpers for streaming a warp's neighbour-list
// rows into shared memory.  Waits are bounded: after kWaitNs nanoseconds of
// the global timer (or kWaitLimit polls, whichever comes first) the kernel
// records kErrTimeout instead of spinning on.
constexpr int kRowsPerChunk = 16;                  // 16 rows x 128 B = 2 KB per stage
constexpr int kForceWarps = kForceThreads / 32;
// neighbour gathers in flight per thread in the pair loop, and the FP32
// kernel's resident blocks per SM the register budget is sized for
#ifndef LE_FORCE_UNROLL
#define LE_FORCE_UNROLL 8
#endif
#ifndef LE_FORCE_MINB32
#define LE_FORCE_MINB32 4
#endif
constexpr int kForceUnroll = LE_FORCE_UNROLL;
// candidate loads in flight per thread in the list build, and its resident
// blocks of the largest shape per SM
#ifndef LE_LIST_UNROLL
#define LE_LIST_UNROLL 6
#endif
#ifndef LE_LIST_MINB
#define LE_LIST_MINB 4
#endif
constexpr int kListUnroll = LE_LIST_UNROLL;
constexpr uint32_t kWaitLimit = 1u << 22;
constexpr unsigned long long kWaitNs = 1000000000ull;  // one second

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void bulk_rows(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes) : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// true once the phase of the given parity has completed; false after about
// kWaitNs (the timer is read only once the first poll has failed)
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  unsigned long long t0 = 0;
  for (uint32_t it = 0; it < kWaitLimit; ++it) {
    uint32_t ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok) : "r"(smem_addr(bar)), "r"(parity) : "memory");
    if (ok) return true;
    const unsigned long long now = global_ns();
    if (it == 0) t0 = now;
    else if (now - t0 > kWaitNs) return false;
  }
  return false;
}

// Image offset of a slot (bit fields, see le_common.cuh) from the cell edges
// and the cross-face shift s of this step: a handful of ALU operations.
template <class R> struct SlotGeo {
  R lx, ly, lz, s;
};
template <class R>
__device__ __forceinline__ void slot_offset(uint32_t e, const SlotGeo<R> &G, R &ox, R &oy, R &oz) {
  const int slot = entry_slot(e);
  const int k = (slot & 7) - 3;
  const int dcy = ((slot >> 3) & 3) - 1;
  const int dcz = ((slot >> 5) & 3) - 1;
  const int cz = (slot & 128) ? dcz : 0;
  ox = R(k) * G.lx + R(cz) * G.s;
  oy = R(dcy) * G.ly;
  oz = R(dcz) * G.lz;
}

// Separation d = p_i - (p_j + image offset of the slot).
template <class R>
__device__ __forceinline__ void slot_sep(uint32_t e, const SlotGeo<R> &G, const V4<R> &pi,
                                         const V4<R> &pj, R &dx, R &dy, R &dz) {
  R ox, oy, oz;
  slot_offset<R>(e, G, ox, oy, oz);
  dx = (pi.x - pj.x) + ox;
  dy = (pi.y - pj.y) + oy;
  dz = (pi.z - pj.z) + oz;
}

// A per-particle sample value in 2^-30 fixed point (the scale is a power of
// two, so only the final rounding to an integer is inexact).
__device__ __forceinline__ long long to_fix(float x) { return __float2ll_rn(x * 1073741824.0f); }
__device__ __forceinline__ long long to_fix(double x) { return llrint(x * kFix); }

template <class R> __device__ __forceinline__ R recip(R x) { return R(1) / x; }
// FP32 pair loop: hardware reciprocal (rcp.approx, within 1 ulp), covered by
// the per-pair evaluation rounding allowed in the FP32 error bound
template <> __device__ __forceinline__ float recip<float>(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

template <class R>
__device__ __forceinline__ void lj_pair(const V4<R> &pi, const V4<R> &pj, uint32_t e,
                                        const SlotGeo<R> &G, R rc2, R c12, R c6, R cap,
                                        R &fx, R &fy, R &fz, R &vir) {
  R dx, dy, dz;
  slot_sep<R>(e, G, pi, pj, dx, dy, dz);
  const R r2 = dx * dx + dy * dy + dz * dz;
  // branch-free: nearly every row has some lane inside rc, so the warp would
  // execute the body anyway; lanes outside get a zero factor (r2 > 0 for
  // every list entry, so the reciprocal is finite either way)
  const R ir2 = recip<R>(r2);
  const R ir6 = ir2 * ir2 * ir2;
  // 24 eps (2 (sigma/r)^12 - (sigma/r)^6) / r^2 = ir2 ir6 (c12 ir6 - c6)
  R fr = r2 < rc2 ? ir2 * ir6 * fma(c12, ir6, -c6) : R(0);
  // push-off: |F| = |fr| r limited to cap (FP64 kernels only)
  if (cap > R(0)) {
    const R lim = cap / sqrt(r2);
    fr = fr > lim ? lim : (fr < -lim ? -lim : fr);
  }
  const R tx = fr * dx;
  fx += tx;
  fy += fr * dy;
  fz += fr * dz;
  vir += tx * dz;
}

// FP32 separations from the fixed-point copies q (units 2^-S): for a list
// entry e of particle o, d' = 2^S (p_o - p_j + off(slot)) =
//   q_o - q_j + (k lx, dcy ly, dcz lz) + cross dcz s   (all in units),
// exact in wrapping 32-bit integer arithmetic (|d'| < 2^31 for every list
// entry), then rounded once to float.  The slot fields' biases (k + 3,
// dcy + 1, dcz + 1) are folded into per-particle constants.
struct SlotQ {
  uint32_t X0, Y0, Z0;       // q_o minus (3 lx, ly, lz) in units
  uint32_t LX, LY, LZ, Sq;   // cell edges and the cross-face shift s(t) in units
  float inv;                 // 2^-S
};
__device__ __forceinline__ SlotQ slot_q(const Geom &g, int s_q, const int4 &qo) {
  SlotQ G;
  G.LX = (uint32_t)g.qL[0];
  G.LY = (uint32_t)g.qL[1];
  G.LZ = (uint32_t)g.qL[2];
  G.Sq = (uint32_t)s_q;
  G.X0 = (uint32_t)qo.x - 3u * G.LX;
  G.Y0 = (uint32_t)qo.y - G.LY;
  G.Z0 = (uint32_t)qo.z - G.LZ;
  G.inv = __int_as_float((127 - g.qshift) << 23);
  return G;
}
// d' (float, units of 2^-S) of entry e against the neighbour's copy qj
__device__ __forceinline__ void q_sep(uint32_t e, const SlotQ &G, const int4 &qj, float &dx,
                                      float &dy, float &dz) {
  const uint32_t k = e & 7u, dy1 = (e >> 3) & 3u, dz1 = (e >> 5) & 3u;
  const uint32_t cross = 0u - ((e >> 7) & 1u);          // all ones across the face
  const uint32_t czs = (dz1 * G.Sq - G.Sq) & cross;      // cross dcz s
  dx = __int2float_rn((int)(k * G.LX + G.X0 - (uint32_t)qj.x + czs));
  dy = __int2float_rn((int)(dy1 * G.LY + G.Y0 - (uint32_t)qj.y));
  dz = __int2float_rn((int)(dz1 * G.LZ + G.Z0 - (uint32_t)qj.z));
}
// the same separation in length units (the scaling by 2^-S is exact)
__device__ __forceinline__ void q_sep_real(uint32_t e, const SlotQ &G, const int4 &qj, float &dx,
                                           float &dy, float &dz) {
  q_sep(e, G, qj, dx, dy, dz);
  dx = __fmul_rn(dx, G.inv);
  dy = __fmul_rn(dy, G.inv);
  dz = __fmul_rn(dz, G.inv);
}

// Two FP32 LJ pairs at once with the paired FP32 instructions of this
// architecture (fma/mul/add.rn.f32x2): lane x of every float2 is pair a,
// lane y pair b; the sums of the two lanes are kept apart and added once
// after the list loop.  cut.y = 0 drops pair b (an odd pair left over).
__device__ __forceinline__ void lj_pair2_q(const SlotQ &G, const int4 &qa, const int4 &qb,
                                           uint32_t ea, uint32_t eb, float2 cut, float2 s2S,
                                           float2 c12, float2 mc6, float2 &fx, float2 &fy,
                                           float2 &fz, float2 &vir) {
  float ax, ay, az, bx, by, bz;
  q_sep(ea, G, qa, ax, ay, az);
  q_sep(eb, G, qb, bx, by, bz);
  const float2 dx = make_float2(ax, bx), dy = make_float2(ay, by), dz = make_float2(az, bz);
  const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
  const float2 ir2 = __fmul2_rn(make_float2(recip<float>(r2.x), recip<float>(r2.y)), s2S);
  const float2 ir6 = __fmul2_rn(__fmul2_rn(ir2, ir2), ir2);
  float2 fr = __fmul2_rn(__fmul2_rn(ir2, ir6), __ffma2_rn(c12, ir6, mc6));
  fr.x = r2.x < cut.x ? fr.x : 0.f;
  fr.y = r2.y < cut.y ? fr.y : 0.f;
  const float2 tx = __fmul2_rn(fr, dx);
  fx = __fadd2_rn(fx, tx);
  fy = __ffma2_rn(fr, dy, fy);
  fz = __ffma2_rn(fr, dz, fz);
  vir = __ffma2_rn(tx, dz, vir);
}

// DPD (Eqs. 6-8, read as the fluctuation-dissipation form): the dissipative
// and random pair forces for r < rc, added to t (the thermostat part of the
// total force, not the conservative force).  v_ij is taken against the image
// of j the slot names: across the face that image moves at cz shear_rate Lz
// (cz = dcz for a pair across the face, else 0), the time derivative of the
// slot offset cz s(t).  Each thread evaluates its own side of a pair; the
// shared theta_ij and the exact antisymmetry of d make F_ji = -F_ij.

template <class R>
__device__ __forceinline__ void dpd_pair(const Geom &g, const V4<R> &pi, const V4<R> &vi, int gi,
                                         const Bufs<R> &b, uint32_t e, const SlotGeo<R> &G,
                                         const SlotQ &GQ, long long n1, R rc2, R &tx, R &ty,
                                         R &tz) {
  const int j = entry_index(e);
  R dx, dy, dz;
  if constexpr (sizeof(R) == 4) {
    q_sep_real(e, GQ, __ldg(b.q + j), dx, dy, dz);
  } else {
    const V4<R> pj = load4(b.p + j);
    slot_sep<R>(e, G, pi, pj, dx, dy, dz);
  }
  const R r2 = fma_rn(dz, dz, fma_rn(dy, dy, mul_rn(dx, dx)));
  if (!(r2 < rc2)) return;
  const KConst<R> &K = kc<R>(g);
  const V4<R> vj = load4(b.v + j);
  const int dcz = ((entry_slot(e) >> 5) & 3) - 1;
  const R cz = (e & 0x80u) ? R(dcz) : R(0);
  const R vx = add_rn(sub_rn(vi.x, vj.x), mul_rn(cz, K.shear_Lz));
  const R vy = sub_rn(vi.y, vj.y), vz = sub_rn(vi.z, vj.z);
  const R r = sqrt(r2);
  const R ir = R(1) / r;
  const R w = sub_rn(R(1), mul_rn(r, K.inv_rc));
  const R ev = mul_rn(fma_rn(dz, vz, fma_rn(dy, vy, mul_rn(dx, vx))), ir);
  const R theta = pair_uniform<R>(g, n1, gi, b.gid[j]);
  const R f = mul_rn(mul_rn(fma_rn(mul_rn(-K.dpd_xi, w), ev, mul_rn(K.dpd_amp, theta)), w), ir);
  tx = fma_rn(f, dx, tx);
  ty = fma_rn(f, dy, ty);
  tz = fma_rn(f, dz, tz);
}

// DPD: the kicked half-step velocities, held back while k_force still read
// the old ones of the neighbours, become the particles' velocities.
template <class R>
__device__ __forceinline__ void vcopy_body(const Geom g, Dyn *__restrict__ d, Bufs<R> s0,
                                           Bufs<R> s1, Work w, int bx) {
  const int i = bx * blockDim.x + threadIdx.x;
  if (i >= g.n) return;
  const Bufs<R> &b = d->cur ? s1 : s0;
  b.v[i] = reinterpret_cast<const V4<R> *>(w.vnew)[i];
}
template <class R>
__global__ void __launch_bounds__(256) k_vcopy(const __grid_constant__ Geom g, Dyn *__restrict__ d,
                                               Bufs<R> s0, Bufs<R> s1, Work w) {
  vcopy_body<R>(g, d, s0, s1, w, (int)blockIdx.x);
}

// One thread per particle; each warp streams its 32 particles' list rows
// (column-major: row k holds entry k of all 32 lanes, 128 B) through a
// two-stage shared-memory ring filled by bulk copies, and gathers neighbour
// positions four at a time.
template <class R, bool BONDS, bool DPD, class BX>
__device__ __forceinline__ void force_body(const Geom &g, Dyn *__restrict__ d, Bufs<R> s0,
                                           Bufs<R> s1, Work w, int mode, BX bx) {
  __shared__ long long s_red[2][kForceWarps];
  __shared__ __align__(128) uint32_t s_rows[kForceWarps][2][kRowsPerChunk][32];
  __shared__ __align__(8) uint64_t s_bar[kForceWarps][2];
  extern __shared__ long long s_prof[];  // [3 * nbins]: vx sums, counts, m vy^2 sums
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int cur = d->cur;
  const long long n1 = d->step;
  // cell edges and cross-face shift (the FP64 pair path; the FP32 one works
  // on the fixed-point copies)
  SlotGeo<R> G;
  G.lx = R(g.lc[0]);
  G.ly = R(g.lc[1]);
  G.lz = R(g.lc[2]);
  G.s = R(d->s);
  const bool sample = mode != 1 && g.sample_every > 0 && (n1 % g.sample_every) == 0;
  // mode 2 (the next step's kick and drift) exists only in FP32 without DPD
  constexpr bool kCanFuse = sizeof(R) == 4 && !DPD;
  const bool fused = kCanFuse && mode == 2;
  if (sample)
    for (int b = t; b < 3 * g.nbins; b += blockDim.x) s_prof[b] = 0;
  if (lane == 0) {
    mbar_init(&s_bar[warp][0], 1);
    mbar_init(&s_bar[warp][1], 1);
  }
  mbar_init_fence();
  __syncthreads();

  const Bufs<R> b = with_cur_q(pick(cur, s0, s1), d->qpar);
  const KConst<R> &K = kc<R>(g);
  const int i = bx() * blockDim.x + t;
  const bool active = i < g.n;
  const int cnt = active ? min(w.ncount[i], g.maxnb) : 0;
  int kmax = cnt;
#pragma unroll
  for (int o = 16; o; o >>= 1) kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
  const int nchunks = (kmax + kRowsPerChunk - 1) / kRowsPerChunk;
  const uint32_t *wrows = w.nbr + (size_t)(i >> 5) * (size_t)g.maxnb * 32u;
  auto issue = [&](int c) {
    const int r0 = c * kRowsPerChunk;
    const int rows = min(kRowsPerChunk, kmax - r0);
    bulk_rows(&s_rows[warp][c & 1][0][0], wrows + (size_t)r0 * 32u, (uint32_t)rows * 128u,
              &s_bar[warp][c & 1]);
  };
  if (lane == 0)
    for (int c = 0; c < min(2, nchunks); ++c) issue(c);

  const R rc2 = K.rc2;
  // c6 = 24 eps sigma^6, c12 = 48 eps sigma^12
  const R sig6 = K.sig2 * K.sig2 * K.sig2;
  const R c6 = K.eps24 * sig6, c12 = R(2) * c6 * sig6;
  const R cap = sizeof(R) == 8 ? R(g.force_cap) : R(0);
  R fx = R(0), fy = R(0), fz = R(0), vir = R(0);
  R tdx = R(0), tdy = R(0), tdz = R(0);  // DPD pair forces
  V4<R> pi = make4<R>(R(0), R(0), R(0), R(0));
  // FP32: the fixed-point copy (pair separations) and p rebuilt from it
  int4 qi = make_int4(0, 0, 0, 0);
  SlotQ GQ{};
  if constexpr (sizeof(R) == 4) {
    if (active) qi = b.q[i];
    GQ = slot_q(g, d->s_q, qi);
    pi = make4<R>(__int2float_rn(qi.x) * GQ.inv, __int2float_rn(qi.y) * GQ.inv,
                  __int2float_rn(qi.z) * GQ.inv, __int_as_float(qi.w));
  } else {
    if (active) pi = b.p[i];
  }
  // FP32 LJ constants for separations in units of 2^-S, and the two-lane
  // partial sums of the paired pair loop
  const float s2S = __int_as_float((127 + 2 * g.qshift) << 23);   // 2^2S
  const float rc2q = (float)K.rc2 * s2S;
  const float2 cut2 = make_float2(rc2q, rc2q), s2S2 = make_float2(s2S, s2S);
  const float2 c12_2 = make_float2((float)c12, (float)c12), mc6_2 = make_float2(-(float)c6, -(float)c6);
  float2 fx2 = make_float2(0.f, 0.f), fy2 = fx2, fz2 = fx2, vir2 = fx2;
  V4<R> vi = make4<R>(R(0), R(0), R(0), R(0));
  int gi = 0;
  if (DPD && active) {
    vi = b.v[i];
    gi = b.gid[i];
  }
  bool ok = true;
  int waited = 0;  // chunks whose barrier has been passed
  for (int c = 0; c < nchunks; ++c) {
    const int st = c & 1;
    if (!mbar_wait(&s_bar[warp][st], (uint32_t)(c >> 1) & 1u)) {
      ok = false;
      break;
    }
    waited = c + 1;
    const uint32_t(*rows)[32] = s_rows[warp][st];
    const int rn = min(kRowsPerChunk, cnt - c * kRowsPerChunk);
    int r = 0;
    // all gathers of a group are issued before the first is used; the
    // pairs are still summed in list order (same result for any group size)
    // (FP64 and DPD keep four: their larger register state would spill)
    constexpr int U = (sizeof(R) == 4 && !DPD) ? kForceUnroll : 4;
    if constexpr (sizeof(R) == 4) {
      for (; r + U <= rn; r += U) {
        uint32_t e[U];
        int4 q[U];
#pragma unroll
        for (int u = 0; u < U; ++u) e[u] = rows[r + u][lane];
#pragma unroll
        for (int u = 0; u < U; ++u) q[u] = __ldg(b.q + entry_index(e[u]));
#pragma unroll
        for (int u = 0; u < U; u += 2)
          lj_pair2_q(GQ, q[u], q[u + 1], e[u], e[u + 1], cut2, s2S2, c12_2, mc6_2, fx2, fy2,
                     fz2, vir2);
        if constexpr (DPD) {
#pragma unroll
          for (int u = 0; u < U; ++u)
            dpd_pair<R>(g, pi, vi, gi, b, e[u], G, GQ, n1, rc2, tdx, tdy, tdz);
        }
      }
      for (; r < rn; r += 2) {
        // the last pair of an odd count goes with a dropped copy of itself
        const bool two = r + 1 < rn;
        const uint32_t ea = rows[r][lane], eb = two ? rows[r + 1][lane] : ea;
        const int4 qa = __ldg(b.q + entry_index(ea));
        const int4 qb = two ? __ldg(b.q + entry_index(eb)) : qa;
        lj_pair2_q(GQ, qa, qb, ea, eb, make_float2(rc2q, two ? rc2q : 0.f), s2S2, c12_2,
                   mc6_2, fx2, fy2, fz2, vir2);
        if constexpr (DPD) {
          dpd_pair<R>(g, pi, vi, gi, b, ea, G, GQ, n1, rc2, tdx, tdy, tdz);
          if (two) dpd_pair<R>(g, pi, vi, gi, b, eb, G, GQ, n1, rc2, tdx, tdy, tdz);
        }
      }
    } else {
      for (; r + U <= rn; r += U) {
        uint32_t e[U];
        V4<R> q[U];
#pragma unroll
        for (int u = 0; u < U; ++u) e[u] = rows[r + u][lane];
#pragma unroll
        for (int u = 0; u < U; ++u) q[u] = load4(b.p + entry_index(e[u]));
#pragma unroll
        for (int u = 0; u < U; ++u)
          lj_pair<R>(pi, q[u], e[u], G, rc2, c12, c6, cap, fx, fy, fz, vir);
        if constexpr (DPD) {
#pragma unroll
          for (int u = 0; u < U; ++u)
            dpd_pair<R>(g, pi, vi, gi, b, e[u], G, GQ, n1, rc2, tdx, tdy, tdz);
        }
      }
      for (; r < rn; ++r) {
        const uint32_t e = rows[r][lane];
        const V4<R> q = load4(b.p + entry_index(e));
        lj_pair<R>(pi, q, e, G, rc2, c12, c6, cap, fx, fy, fz, vir);
        if constexpr (DPD) dpd_pair<R>(g, pi, vi, gi, b, e, G, GQ, n1, rc2, tdx, tdy, tdz);
      }
    }
    __syncwarp();
    if (lane == 0 && c + 2 < nchunks) {
      fence_async_smem();  // the rows just read are overwritten by the async proxy
      issue(c + 2);
    }
  }
  if (!ok) {
    atomicOr(&d->err, (int)kErrTimeout);
    // let copies still in flight land before the block's shared memory is released
    for (int c = waited; c < min(waited + 2, nchunks); ++c)
      mbar_wait(&s_bar[warp][c & 1], (uint32_t)(c >> 1) & 1u);
  }

  if constexpr (sizeof(R) == 4) {
    // the two lanes' pair sums, taken in units of 2^S (force) and 2^2S (virial)
    fx = (fx2.x + fx2.y) * GQ.inv;
    fy = (fy2.x + fy2.y) * GQ.inv;
    fz = (fz2.x + fz2.y) * GQ.inv;
    vir = (vir2.x + vir2.y) * (GQ.inv * GQ.inv);
  }
  // separation of o (at po; fixed-point copy qo) from the image of the
  // particle that bond entry e names, in length units
  auto bond_sep = [&](const V4<R> &po, const int4 &qo, uint32_t e, R &dx, R &dy, R &dz) {
    const int j = entry_index(e);
    if constexpr (sizeof(R) == 4) {
      q_sep_real(e, slot_q(g, d->s_q, qo), __ldg(b.q + j), dx, dy, dz);
    } else {
      const V4<R> pj = load4(b.p + j);
      R ox, oy, oz;
      slot_offset<R>(e, G, ox, oy, oz);
      dx = (po.x - pj.x) + ox;
      dy = (po.y - pj.y) + oy;
      dz = (po.z - pj.z) + oz;
    }
  };
  R sxz = R(0), ke = R(0);
  float disp2 = 0.f;  // mode 2: squared peculiar displacement after the drift
  int bin = -1;
  R vxw = R(0), vy2 = R(0);
  if (active) {
    if constexpr (BONDS) {
      const R R02 = K.R02, kf = K.fene_k;
      for (int q = 0; q < g.maxb; ++q) {
        const uint32_t e = w.bond_e[(size_t)i * g.maxb + q];
        if (e == kNoBond) break;
        R dx, dy, dz;
        bond_sep(pi, qi, e, dx, dy, dz);
        const R x = R(1) - (dx * dx + dy * dy + dz * dz) / R02;
        if (!(x > R(0))) {
          atomicOr(&d->err, (int)kErrBond);
          continue;
        }
        const R fr = -kf / x;
        const R tx = fr * dx;
        fx += tx;
        fy += fr * dy;
        fz += fr * dz;
        vir += tx * dz;
      }
      if (K.ang_k != R(0)) {
        // Eq. 12, read as k_a (1 + cos theta): every angle this particle is
        // part of -- as the middle bead of two of its bonds, or as an end of
        // two bonds of a neighbour -- gathered here, so no other thread writes
        // this force.  Separations use each bond's own slot (the neighbour's
        // for its bonds), so angles across the sheared face need no extra
        // image arithmetic.
        const R ka = K.ang_k;
        // force on the end bead at a = r_end - r_mid, the other end at c
        auto end_force = [&](R ax, R ay, R az, R cx, R cy, R cz, R &gx, R &gy, R &gz) {
          const R ia = R(1) / sqrt(ax * ax + ay * ay + az * az);
          const R ic = R(1) / sqrt(cx * cx + cy * cy + cz * cz);
          ax *= ia;
          ay *= ia;
          az *= ia;
          cx *= ic;
          cy *= ic;
          cz *= ic;
          const R ct = ax * cx + ay * cy + az * cz;
          gx = -ka * (cx - ct * ax) * ia;
          gy = -ka * (cy - ct * ay) * ia;
          gz = -ka * (cz - ct * az) * ia;
        };
        for (int u = 0; u < g.maxb; ++u) {
          const uint32_t eu = w.bond_e[(size_t)i * g.maxb + u];
          if (eu == kNoBond) break;
          R ux, uy, uz;  // r_i - r_j for the bonded neighbour j
          bond_sep(pi, qi, eu, ux, uy, uz);
          for (int v = u + 1; v < g.maxb; ++v) {
            const uint32_t ev = w.bond_e[(size_t)i * g.maxb + v];
            if (ev == kNoBond) break;
            R vx, vy, vz;
            bond_sep(pi, qi, ev, vx, vy, vz);
            // i in the middle: the ends sit at -u and -v from i
            R ax, ay, az, cx, cy, cz;
            end_force(-ux, -uy, -uz, -vx, -vy, -vz, ax, ay, az);
            end_force(-vx, -vy, -vz, -ux, -uy, -uz, cx, cy, cz);
            fx -= ax + cx;
            fy -= ay + cy;
            fz -= az + cz;
          }
          // i at an end: the angles in the middle of j, with j's other bonds
          const int j = entry_index(eu);
          V4<R> pj = make4<R>(R(0), R(0), R(0), R(0));
          int4 qj = make_int4(0, 0, 0, 0);
          if constexpr (sizeof(R) == 4) qj = __ldg(b.q + j);
          else pj = load4(b.p + j);
          for (int q = 0; q < g.maxb; ++q) {
            const uint32_t ek = w.bond_e[(size_t)j * g.maxb + q];
            if (ek == kNoBond) break;
            if (entry_index(ek) == i) continue;  // the bond back to i
            R kx, ky, kz;  // r_j - r_k
            bond_sep(pj, qj, ek, kx, ky, kz);
            R ax, ay, az;
            end_force(ux, uy, uz, -kx, -ky, -kz, ax, ay, az);
            fx += ax;
            fy += ay;
            fz += az;
            // the angle's virial a (x) F_end, once per angle (vir is halved)
            vir += R(2) * ux * az;
          }
        }
      }
    }
    // Eq. 5: friction on the peculiar velocity plus the random force
    const V4<R> v = b.v[i];
    const R zu = pi.z + pi.w;  // unwrapped z (reference + displacement)
    // an explicitly rounded product: vs is subtracted below, and no kernel
    // that inlines this may fuse it into an FMA
    const R vs = mul_rn(K.shear, zu - K.half_Lz);
    R ftx = fx + tdx, fty = fy + tdy, ftz = fz + tdz;
    if (g.thermostat == 1 || g.thermostat == 2) {
      // 1: friction on the peculiar velocity (Eq. 5); 2: on the absolute
      // velocity (the comparison variant of Sec. 2.2), same noise.  Between
      // builds a particle that crossed the top/bottom face is kept unwrapped,
      // velocity jump not yet applied: v - v_s is the same either way, but the
      // absolute friction must see the wrapped lab velocity v - nz shear Lz.
      R u[3];
      uniform3<R>(g, n1, b.gid[i], u);
      const R amp = K.amp;
      const R xm = K.xim;
      const R vf = g.thermostat == 1
                       ? vs
                       : (zu >= K.Lz ? K.shear_Lz : (zu < R(0) ? -K.shear_Lz : R(0)));
      ftx += fma(amp, u[0], -xm * (v.x - vf));
      fty += fma(amp, u[1], -xm * v.y);
      ftz += fma(amp, u[2], -xm * v.z);
    }
    V4<R> nv = v;
    if (mode != 1) {
      const R half = K.half_dt_m;
      nv.x = fma(half, ftx, v.x);
      nv.y = fma(half, fty, v.y);
      nv.z = fma(half, ftz, v.z);
    }
    // fused with the next drift (mode 2), the total force goes straight into
    // the next half kick and neither force is stored
    if (!fused) {
      b.fc[i] = make4<R>(fx, fy, fz, R(0));
      b.ft[i] = make4<R>(ftx, fty, ftz, R(0));
    }
    // DPD reads the other particles' half-step velocities: the kicked ones go
    // to a scratch array, copied back once every thread has read
    if constexpr (DPD) reinterpret_cast<V4<R> *>(w.vnew)[i] = nv;
    else if (!fused) b.v[i] = nv;
    if (!isfinite(ftx + fty + ftz) || !isfinite(nv.x + nv.y + nv.z))
      atomicOr(&d->err, (int)kErrNonfinite);
    if (sample) {
      const R m = K.mass;
      const R vpx = nv.x - vs;
      // explicit fma (the same rounding in every instantiation)
      sxz = fma(m * vpx, nv.z, R(0.5) * vir);
      ke = m * fma(nv.z, nv.z, fma(nv.y, nv.y, vpx * vpx));
      R zw = zu, vw = nv.x;
      const R Lz = K.Lz;
      if (zw >= Lz) {
        zw -= Lz;
        vw -= K.shear_Lz;
      } else if (zw < R(0)) {
        zw += Lz;
        vw += K.shear_Lz;
      }
      // same operation order as the bins of the oracle: z / Lz * nbins
      int bb = (int)floor(zw / Lz * R(g.nbins));
      bin = bb < 0 ? 0 : (bb >= g.nbins ? g.nbins - 1 : bb);
      vxw = vw;
      vy2 = m * nv.y * nv.y;  // T_y profile (Sec. 3.1)
    }
    // mode 2: the next step's first half kick and drift (FP32 without DPD,
    // where neighbours are read only through the fixed-point copy q; the
    // drifted copy goes to q2)
    if constexpr (kCanFuse) {
      if (fused)
        disp2 = kick_drift<R>(g, d, b, b.q2, i, nv, make4<R>(ftx, fty, ftz, R(0)),
                              drift_shear_tau(g, d));
    }
  }
  if constexpr (kCanFuse) {
    if (fused) {
      block_max_disp<kForceWarps>(d, disp2);
      if (t == 0 && bx() == 0) d->qflip = 1;
    }
  }
  if (!sample) return;
  // each particle's contribution in 2^-30 fixed point, then integer sums:
  // the same totals for any grouping of particles into warps, blocks or
  // batches (launch shapes change no sample)
  const long long a = warp_sum(to_fix(sxz));
  const long long c = warp_sum(to_fix(ke));
  if (lane == 0) {
    s_red[0][warp] = a;
    s_red[1][warp] = c;
  }
  {
    // lanes of a warp mostly share a z bin: one shared atomic per distinct
    // bin and warp (integer sums, so the order of addition does not matter)
    // a value beyond the fixed-point range is reported as an error (the step
    // is rolled back), and clamped only so that the integer sums stay defined
    const float vxf = (float)vxw, vyf = (float)vy2;
    if (bin >= 0 && !(fabsf(vxf) <= kProfVxMax && vyf <= kProfVy2Max))
      atomicOr(&d->err, (int)kErrRange);
    const float vc = fminf(fmaxf(vxf, -kProfVxMax), kProfVxMax);
    const int q = bin >= 0 ? __float2int_rn(vc * (float)kFixP) : 0;
    const float yc = fminf(fmaxf(vyf, 0.f), kProfVy2Max);
    const int qy = bin >= 0 ? __float2int_rn(yc * (float)kFixP) : 0;
    unsigned todo = __ballot_sync(0xffffffffu, bin >= 0);
    while (todo) {
      const int leader = __ffs(todo) - 1;
      const int b0 = __shfl_sync(0xffffffffu, bin, leader);
      const unsigned grp = __ballot_sync(0xffffffffu, bin == b0);
      // split the 2^20 fixed-point values so 32 of them cannot overflow int32
      const int hi = __reduce_add_sync(0xffffffffu, bin == b0 ? (q >> 10) : 0);
      const int lo = __reduce_add_sync(0xffffffffu, bin == b0 ? (q & 1023) : 0);
      const int yhi = __reduce_add_sync(0xffffffffu, bin == b0 ? (qy >> 10) : 0);
      const int ylo = __reduce_add_sync(0xffffffffu, bin == b0 ? (qy & 1023) : 0);
      if (lane == leader) {
        atomicAdd((unsigned long long *)&s_prof[b0],
                  (unsigned long long)((long long)hi * 1024 + (long long)lo));
        atomicAdd((unsigned long long *)&s_prof[g.nbins + b0], (unsigned long long)__popc(grp));
        atomicAdd((unsigned long long *)&s_prof[2 * g.nbins + b0],
                  (unsigned long long)((long long)yhi * 1024 + (long long)ylo));
      }
      todo &= ~grp;
    }
  }
  __syncthreads();
  if (t == 0) {
    long long A = 0, B = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      A += s_red[0][k];
      B += s_red[1][k];
    }
    atomicAdd((unsigned long long *)&d->acc_sxz, (unsigned long long)A);
    atomicAdd((unsigned long long *)&d->acc_ke, (unsigned long long)B);
    if (bx() == 0) d->pending = 1;
  }
  for (int q = t; q < g.nbins; q += blockDim.x) {
    const long long cn = s_prof[g.nbins + q];
    if (cn) {
      atomicAdd((unsigned long long *)&w.acc_prof[q], (unsigned long long)s_prof[q]);
      atomicAdd((unsigned long long *)&w.acc_prof[g.nbins + q], (unsigned long long)cn);
      atomicAdd((unsigned long long *)&w.acc_prof[2 * g.nbins + q],
                (unsigned long long)s_prof[2 * g.nbins + q]);
    }
  }
}
template <class R, bool BONDS, bool DPD>
__global__ void __launch_bounds__(kForceThreads, (DPD || sizeof(R) == 8) ? 2 : LE_FORCE_MINB32) k_force(
    const __grid_constant__ Geom g, Dyn *__restrict__ d, Bufs<R> s0, Bufs<R> s1, Work w, int mode) {
  force_body<R, BONDS, DPD>(g, d, s0, s1, w, mode, HwBlock{});
}

// --------------------------------------------------------------- rebuild: bin
// Re-basing without FP64 (FP32 mode): a displacement is the unevaluated sum
// hi + lo of two floats; moving it to another cell subtracts an integer
// number of cell edges, each edge itself split into hi + lo.
__device__ __forceinline__ void df_add(float &hi, float &lo, float bh, float bl) {
  const float s = __fadd_rn(hi, bh);
  const float bb = __fsub_rn(s, hi);
  float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(bh, bb));
  e = __fadd_rn(e, __fadd_rn(lo, bl));
  hi = __fadd_rn(s, e);
  lo = __fsub_rn(e, __fsub_rn(hi, s));
}
// (hi, lo) -= k * (eh + el) for a small integer k (the product is split exactly)
__device__ __forceinline__ void df_sub_edges(float &hi, float &lo, int k, float eh, float el) {
  if (k == 0) return;
  const float fk = (float)(-k);
  const float t = __fmul_rn(fk, eh);
  const float te = __fmaf_rn(fk, eh, -t);
  df_add(hi, lo, t, __fmaf_rn(fk, el, te));
}

template <class R> struct Disp;   // a displacement being re-based
template <> struct Disp<float> {
  float h[3], l[3];
  __device__ void sub_edges(const Geom &g, int a, int k) { df_sub_edges(h[a], l[a], k, g.lc_hi[a], g.lc_lo[a]); }
  __device__ void sub_x(float fh, float fl) { df_add(h[0], l[0], -fh, -fl); }
  __device__ float approx(int a) const { return h[a]; }
};
template <> struct Disp<double> {
  double h[3];
  __device__ void sub_edges(const Geom &g, int a, int k) { h[a] -= (double)k * g.lc[a]; }
  __device__ float approx(int a) const { return (float)h[a]; }
};

__device__ __forceinline__ int wrap_index(int c, int n) {
  c %= n;
  return c < 0 ? c + n : c;
}

// Re-bases the current state on the cells the particles occupy now: the
// unwrapped cell index, the LE wrap through the top/bottom face (z image
// removed, x -= dX as m_b cells + f_b, vx -= shear_rate*Lz), periodic x/y.
// Writes the new displacement (pre-sort order) and the sort keys/values.
template <class R>
__device__ __forceinline__ void rb_bin_body(const Geom g, Dyn *__restrict__ d, Bufs<R> s0,
                                            Bufs<R> s1, Work w, int bx) {
  const Bufs<R> b = pick(d->cur, s0, s1);
  const int i = bx * blockDim.x + threadIdx.x;
  if (i >= g.n) return;
  const float4 q = b.pb[i];
  int c0, c1, c2;
  cell_coords(g, __float_as_int(q.w), c0, c1, c2);
  const V4<R> p = b.p[i];
  Disp<R> u;
  u.h[0] = p.x;
  u.h[1] = p.y;
  u.h[2] = p.z;
  if constexpr (sizeof(R) == 4) {
    const float4 lo = b.plo[i];
    u.l[0] = lo.x;
    u.l[1] = lo.y;
    u.l[2] = lo.z;
  }
  const int dz = (int)floorf(0.5f + u.approx(2) * g.inv_lc[2]);
  u.sub_edges(g, 2, dz);
  int cz = c2 + dz, wz = 0;
  if (cz >= g.nc[2]) { cz -= g.nc[2]; wz = 1; }
  else if (cz < 0) { cz += g.nc[2]; wz = -1; }
  cz = min(max(cz, 0), g.nc[2] - 1);
  int cx = c0;
  if (wz != 0) {
    // x -= wz * dX with dX = m_b lx + f_b
    if constexpr (sizeof(R) == 4) {
      if (wz > 0) u.sub_x(d->f_hi, d->f_lo);
      else u.sub_x(-d->f_hi, -d->f_lo);
    } else {
      u.h[0] -= (double)wz * d->f_build;
    }
    cx -= wz * d->m_build;
    V4<R> v = b.v[i];
    v.x -= R(wz) * kc<R>(g).shear_Lz;
    b.v[i] = v;
  }
  const int dx = (int)floorf(0.5f + u.approx(0) * g.inv_lc[0]);
  u.sub_edges(g, 0, dx);
  cx = wrap_index(cx + dx, g.nc[0]);
  const int dy = (int)floorf(0.5f + u.approx(1) * g.inv_lc[1]);
  u.sub_edges(g, 1, dy);
  const int cy = wrap_index(c1 + dy, g.nc[1]);
  w.key[0][i] = (uint32_t)(cx + g.nc[0] * (cy + g.nc[1] * cz));
  w.val[0][i] = (uint32_t)i;
  V4<R> *tp = reinterpret_cast<V4<R> *>(w.tmp_p);
  tp[i] = make4<R>(u.h[0], u.h[1], u.h[2], R(0));
  if constexpr (sizeof(R) == 4) w.tmp_lo[i] = make_float4(u.l[0], u.l[1], u.l[2], 0.f);
}
template <class R>
__global__ void __launch_bounds__(256) k_rb_bin(const __grid_constant__ Geom g, Dyn *__restrict__ d,
                                                Bufs<R> s0, Bufs<R> s1, Work w) {
  rb_bin_body<R>(g, d, s0, s1, w, (int)blockIdx.x);
}

// Initial load: caller-order FP64 positions/velocities (staging) wrapped as
// images at the current offset, binned, displacement from the cell reference.
template <class R>
__global__ void __launch_bounds__(256) k_import(Geom g, Dyn *__restrict__ d, Bufs<R> s0,
                                                Bufs<R> s1, Work w, const double *__restrict__ stage,
                                                int i0, int i1) {
  const Bufs<R> b = pick(d->cur, s0, s1);
  const int i = i0 + (int)(blockIdx.x * blockDim.x + threadIdx.x);
  if (i >= i1) return;
  double x[3] = {stage[3 * (size_t)i], stage[3 * (size_t)i + 1], stage[3 * (size_t)i + 2]};
  double vx = stage[3 * (size_t)g.n + 3 * (size_t)i];
  double vy = stage[3 * (size_t)g.n + 3 * (size_t)i + 1];
  double vz = stage[3 * (size_t)g.n + 3 * (size_t)i + 2];
  // a non-finite input is reported (the call fails) and replaced by zero
  if (!(isfinite(x[0]) && isfinite(x[1]) && isfinite(x[2]) && isfinite(vx) && isfinite(vy) &&
        isfinite(vz))) {
    atomicOr(&d->err, (int)kErrInput);
    x[0] = x[1] = x[2] = vx = vy = vz = 0.0;
  }
  // any number of images away: remove whole boxes along z first
  const double nzf = floor_div(x[2], g.L[2], g.inv_L[2]);
  if (nzf != 0.0) {
    x[2] -= nzf * g.L[2];
    x[0] -= nzf * d->dX;
    vx -= nzf * g.shear_rate * g.L[2];
  }
  le_wrap(g, d->dX, x, vx);
  const int c = cell_of(g, x);
  int cx, cy, cz;
  cell_coords(g, c, cx, cy, cz);
  const double r[3] = {((double)cx + 0.5) * g.lc[0], ((double)cy + 0.5) * g.lc[1],
                       ((double)cz + 0.5) * g.lc[2]};
  V4<R> *tp = reinterpret_cast<V4<R> *>(w.tmp_p);
  if constexpr (sizeof(R) == 4) {
    float h[3], l[3];
    for (int a = 0; a < 3; ++a) {
      const double dd = x[a] - r[a];
      h[a] = (float)dd;
      l[a] = (float)(dd - (double)h[a]);
    }
    tp[i] = make_float4(h[0], h[1], h[2], 0.f);
    w.tmp_lo[i] = make_float4(l[0], l[1], l[2], 0.f);
  } else {
    tp[i] = make4<double>(x[0] - r[0], x[1] - r[1], x[2] - r[2], 0.0);
  }
  w.key[0][i] = (uint32_t)c;
  w.val[0][i] = (uint32_t)i;
  b.v[i] = make4<R>(R(vx), R(vy), R(vz), R(0));
  b.ft[i] = make4<R>(R(0), R(0), R(0), R(0));
  b.fc[i] = make4<R>(R(0), R(0), R(0), R(0));
  b.gid[i] = i;
}

// ----------------------------------------------------------- rebuild: ranges
// cell_start[c] = first sorted slot of cell c (every entry written once).
// Run inside the permute kernel after a sort; k_rb_ranges alone on restore.
__device__ __forceinline__ void rb_ranges_body(const Geom g, const uint32_t *__restrict__ skey,
                                               int *__restrict__ cell_start, int bx) {
  const int k = bx * blockDim.x + threadIdx.x;
  if (k >= g.n) return;
  const int c = min((int)skey[k], g.ncell - 1);
  const int prev = k == 0 ? -1 : min((int)skey[k - 1], g.ncell - 1);
  for (int cc = prev + 1; cc <= c; ++cc) cell_start[cc] = k;
  if (k == g.n - 1)
    for (int cc = c + 1; cc <= g.ncell; ++cc) cell_start[cc] = g.n;
}
__global__ void __launch_bounds__(256) k_rb_ranges(const __grid_constant__ Geom g,
                                                   const uint32_t *__restrict__ skey,
                                                   int *__restrict__ cell_start) {
  rb_ranges_body(g, skey, cell_start, (int)blockIdx.x);
}

// ---------------------------------------------------------- rebuild: permute
// Gathers the re-based state into cell order, and writes the cell ranges of
// the same sorted slots (both read only the sorted keys).  Forces are not
// moved: the pair kernel of the same step overwrites them before anything
// reads them.
template <class R>
__device__ __forceinline__ void rb_permute_body(const Geom g, Dyn *__restrict__ d, Bufs<R> s0,
                                                Bufs<R> s1, Work w,
                                                const uint32_t *__restrict__ skey,
                                                const uint32_t *__restrict__ sval, int bx) {
  rb_ranges_body(g, skey, w.cell_start, bx);
  const int cur = d->cur;
  const Bufs<R> src = pick(cur, s0, s1);
  const Bufs<R> dst = with_cur_q(pick(1 - cur, s0, s1), d->qpar);
  const int k = bx * blockDim.x + threadIdx.x;
  if (k >= g.n) return;
  const int o = min((int)sval[k], g.n - 1);
  const int c = min((int)skey[k], g.ncell - 1);
  const int cz = c / (g.nc[0] * g.nc[1]);
  const V4<R> h = reinterpret_cast<const V4<R> *>(w.tmp_p)[o];
  const R zref = (R(cz) + R(0.5)) * R(g.lc[2]);
  dst.p[k] = make4<R>(h.x, h.y, h.z, zref);
  if constexpr (sizeof(R) == 4) {
    const float4 lo = w.tmp_lo[o];
    dst.plo[k] = lo;
    dst.q[k] = quantize(g, make4<float>(h.x, h.y, h.z, zref), lo);
  }
  dst.pb[k] = make_float4((float)h.x, (float)h.y, (float)h.z, __int_as_float(c));
  dst.v[k] = src.v[o];
  const int gid = src.gid[o];
  dst.gid[k] = gid;
  w.rank[gid] = k;  // the sorted slot of each particle id (exports, bonds)
  if (g.maxb > 0) {
    int cx, cy, czz;
    cell_coords(g, c, cx, cy, czz);
    double x0 = ((double)cx + 0.5) * g.lc[0] + (double)h.x;
    double x1 = ((double)cy + 0.5) * g.lc[1] + (double)h.y;
    double x2 = ((double)czz + 0.5) * g.lc[2] + (double)h.z;
    if constexpr (sizeof(R) == 4) {
      const float4 lo = w.tmp_lo[o];
      x0 += (double)lo.x;
      x1 += (double)lo.y;
      x2 += (double)lo.z;
    }
    w.Xs[3 * (size_t)k] = x0;
    w.Xs[3 * (size_t)k + 1] = x1;
    w.Xs[3 * (size_t)k + 2] = x2;
  }
}
template <class R>
__global__ void __launch_bounds__(256) k_rb_permute(const __grid_constant__ Geom g,
                                                    Dyn *__restrict__ d, Bufs<R> s0, Bufs<R> s1,
                                                    Work w, const uint32_t *__restrict__ skey,
                                                    const uint32_t *__restrict__ sval) {
  rb_permute_body<R>(g, d, s0, s1, w, skey, sval, (int)blockIdx.x);
}

// Restore path (checkpoint or rollback): sort keys, build-time FP64
// positions and ranks from the stored build record of the current set.
template <class R>
__global__ void k_relist_prep(Geom g, Dyn *__restrict__ d, Bufs<R> s0, Bufs<R> s1, Work w) {
  const Bufs<R> b = with_cur_q(pick(d->cur, s0, s1), d->qpar);
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= g.n) return;
  const float4 q = b.pb[k];
  const int c = __float_as_int(q.w);
  int cx, cy, cz;
  cell_coords(g, c, cx, cy, cz);
  w.key[0][k] = (uint32_t)c;
  w.Xs[3 * (size_t)k] = ((double)cx + 0.5) * g.lc[0] + (double)q.x;
  w.Xs[3 * (size_t)k + 1] = ((double)cy + 0.5) * g.lc[1] + (double)q.y;
  w.Xs[3 * (size_t)k + 2] = ((double)cz + 0.5) * g.lc[2] + (double)q.z;
  w.rank[b.gid[k]] = k;
  // the fixed-point copy of a restored state
  if constexpr (sizeof(R) == 4) b.q[k] = quantize(g, b.p[k], b.plo[k]);
}

// Slot-offset tables from d->s (this step) and d->f_build (last build).
__global__ void k_tables(Geom g, Dyn *__restrict__ d) {
  const double s = d->s, fb = d->f_build;
  if (threadIdx.x == 0) {
    d->list_entries = 0;
    cross_window(g, fb, d);
    d->f_hi = (float)fb;
    d->f_lo = (float)(fb - (double)d->f_hi);
  }
  for (int e = threadIdx.x; e < kNumSlots; e += blockDim.x) {
    int k, dcy, dcz, cross;
    slot_decode(e, k, dcy, dcz, cross);
    d->off[e][0] = (double)k * g.lc[0] + (cross ? (double)dcz * s : 0.0);
    d->off_build[e][0] = (double)k * g.lc[0] + (cross ? (double)dcz * fb : 0.0);
    d->off[e][1] = d->off_build[e][1] = (double)dcy * g.lc[1];
    d->off[e][2] = d->off_build[e][2] = (double)dcz * g.lc[2];
    d->off[e][3] = d->off_build[e][3] = 0.0;
  }
}

// ------------------------------------------------------------- rebuild: list
// The list builds' arithmetic, rounded explicitly so that both forms below
// (and every kernel that inlines them) take the same decisions: the distance
// along one axis from a point at a to a cell box of half edge h around 0,
// and the squared distance of a candidate q from the point (ax, ay, az).
__device__ __forceinline__ float box_gap(float a, float h) {
  return fmaxf(__fsub_rn(fabsf(a), h), 0.f);
}
__device__ __forceinline__ float list_dist2(float ax, float ay, float az, const float4 &q) {
  const float dx = __fsub_rn(ax, q.x), dy = __fsub_rn(ay, q.y), dz = __fsub_rn(az, q.z);
  return __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
}

// LE-aware Verlet list from the build positions.  Neighbour cells of cell
// (cx,cy,cz): for a y/z neighbour row inside the box, the x cells cx-1..cx+1;
// for a row across the top/bottom face, the x window shifted by the image
// offset: 3 or 4 cells covering every cell within rl of the shifted row
// (f_build/lx decides whether the window reaches a 4th cell).  Rows and
// cells whose box lies farther than rl from the particle are skipped.
template <class R, class BX>
__device__ __forceinline__ void rb_list_body(const Geom g, Dyn *__restrict__ d, Bufs<R> s0,
                                             Bufs<R> s1, Work w, int target_cur, BX bx) {
  __shared__ float s_offx[kNumSlots];
  for (int e = threadIdx.x; e < kNumSlots; e += blockDim.x) s_offx[e] = (float)d->off_build[e][0];
  __syncthreads();
  const int tgt = target_cur ? d->cur : 1 - d->cur;
  const Bufs<R> b = pick(tgt, s0, s1);
  const int i = bx() * blockDim.x + threadIdx.x;
  int cnt = 0;
  if (i < g.n) {
    const float4 qi = b.pb[i];
    int cx, cy, cz;
    cell_coords(g, __float_as_int(qi.w), cx, cy, cz);
    const float rl2 = g.rl2_build;
    const float hx = g.half_lc_f[0], hy = g.half_lc_f[1], hz = g.half_lc_f[2];
    const float ly = (float)g.lc[1], lz = (float)g.lc[2];
    const int mb = d->m_build;
    uint32_t *out = w.nbr + (size_t)(i >> 5) * (size_t)g.maxnb * 32u + (i & 31);
    const int cap = g.maxnb - 1;
    for (int dcz = -1; dcz <= 1; ++dcz) {
      const float az = __fmaf_rn((float)dcz, lz, qi.z);
      const float gz = box_gap(az, hz);
      if (__fmul_rn(gz, gz) >= rl2) continue;
      int czj = cz - dcz, cross = 0;
      if (czj < 0) { czj += g.nc[2]; cross = 1; }
      else if (czj >= g.nc[2]) { czj -= g.nc[2]; cross = 1; }
      int kmin = -1, kmax = 1;
      if (cross) {
        kmin = d->win_lo[dcz > 0 ? 1 : 0];
        kmax = d->win_hi[dcz > 0 ? 1 : 0];
      }
      for (int dcy = -1; dcy <= 1; ++dcy) {
        const float ay = __fmaf_rn((float)dcy, ly, qi.y);
        const float gy = box_gap(ay, hy);
        const float gyz = __fmaf_rn(gy, gy, __fmul_rn(gz, gz));
        if (gyz >= rl2) continue;
        const int cyj = wrap_index(cy - dcy, g.nc[1]);
        const int rowbase = g.nc[0] * (cyj + g.nc[1] * czj);
        for (int k = kmin; k <= kmax; ++k) {
          const int slot = slot_code(k, dcy, dcz, cross);
          const float ax = __fadd_rn(qi.x, s_offx[slot]);
          const float gx = box_gap(ax, hx);
          if (__fmaf_rn(gx, gx, gyz) >= rl2) continue;
          const int cxj = wrap_index(cx - k + (cross ? dcz * mb : 0), g.nc[0]);
          const int cj = rowbase + cxj;
          // clamped so that a corrupt range can never leave the particle arrays
          const int j0 = min(max(w.cell_start[cj], 0), g.n);
          const int j1 = min(max(w.cell_start[cj + 1], j0), g.n);
          // the particle itself is a candidate only in its own cell's slot
          const int self_j = slot == slot_code(0, 0, 0, 0) ? i : -1;
          const uint32_t tag = (uint32_t)slot;
          int j = j0;
          auto emit = [&](int jj, const float4 &q) {
            if (list_dist2(ax, ay, az, q) < rl2 && jj != self_j) {
              // past the capacity the last row is overwritten (the overflow is
              // reported and the list regrown)
              out[min(cnt, cap) * 32] = ((uint32_t)jj << kSlotBits) | tag;
              ++cnt;
            }
          };
          // kListUnroll candidates per pass: their loads are in flight together
          for (; j + kListUnroll <= j1; j += kListUnroll) {
            float4 q[kListUnroll];
#pragma unroll
            for (int u = 0; u < kListUnroll; ++u) q[u] = __ldg(b.pb + j + u);
#pragma unroll
            for (int u = 0; u < kListUnroll; ++u) emit(j + u, q[u]);
          }
          for (; j < j1; ++j) emit(j, __ldg(b.pb + j));
        }
      }
    }
    w.ncount[i] = cnt;
    atomicMax(&d->list_max, cnt);
    if (cnt > g.maxnb) atomicOr(&d->err, (int)kErrCapacity);
  }
  // total list entries (for the mean list length), one atomic per block
  __shared__ unsigned long long s_tot[kListMaxThreads / 32];
  const unsigned long long c = warp_sum((unsigned long long)cnt);
  if ((threadIdx.x & 31) == 0) s_tot[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += s_tot[k];
    atomicAdd((unsigned long long *)&d->list_entries, t);
  }
}
template <class R>
__global__ void __launch_bounds__(kListMaxThreads, LE_LIST_MINB) k_rb_list(
    const __grid_constant__ Geom g, Dyn *__restrict__ d, Bufs<R> s0, Bufs<R> s1, Work w,
    int target_cur) {
  rb_list_body<R>(g, d, s0, s1, w, target_cur, HwBlock{});
}

// The same list for systems too small to fill the GPU with one thread per
// particle (kSmallListTests): one warp per particle and one lane per neighbour
// cell, taken in rb_list_body's order (dcz, then dcy, then the x window k),
// 32 cells per round (one round unless a face window is unusually wide).
// Each lane counts the candidates of its cell that it keeps, the counts are
// prefix-summed across the warp, and each lane writes its entries from its
// offset: the same entries in the same order as rb_list_body, with every
// cell's loads and tests in parallel instead of one cell after another.
constexpr int kListWppWarps = 8;  // particles per block
template <class R>
__global__ void __launch_bounds__(32 * kListWppWarps) k_rb_list_wpp(
    const __grid_constant__ Geom g, Dyn *__restrict__ d, Bufs<R> s0, Bufs<R> s1, Work w,
    int target_cur) {
  __shared__ float s_offx[kNumSlots];
  __shared__ int s_cnt[kListWppWarps];
  for (int e = threadIdx.x; e < kNumSlots; e += blockDim.x) s_offx[e] = (float)d->off_build[e][0];
  __syncthreads();
  const int tgt = target_cur ? d->cur : 1 - d->cur;
  const Bufs<R> b = pick(tgt, s0, s1);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i = blockIdx.x * kListWppWarps + warp;
  int total = 0;
  if (i < g.n) {  // the same for the whole warp
    const float4 qi = b.pb[i];
    int cx, cy, cz;
    cell_coords(g, __float_as_int(qi.w), cx, cy, cz);
    const float rl2 = g.rl2_build;
    const float hx = g.half_lc_f[0], hy = g.half_lc_f[1], hz = g.half_lc_f[2];
    const float ly = (float)g.lc[1], lz = (float)g.lc[2];
    const int mb = d->m_build;
    uint32_t *out = w.nbr + (size_t)(i >> 5) * (size_t)g.maxnb * 32u + (i & 31);
    const int cap = g.maxnb - 1;
    // the three z rows: target row, face crossing, x window
    int czj[3], cross[3], kmin[3], width[3];
#pragma unroll
    for (int z = 0; z < 3; ++z) {
      const int dcz = z - 1;
      int c = cz - dcz, cr = 0;
      if (c < 0) { c += g.nc[2]; cr = 1; }
      else if (c >= g.nc[2]) { c -= g.nc[2]; cr = 1; }
      czj[z] = c;
      cross[z] = cr;
      kmin[z] = cr ? d->win_lo[dcz > 0 ? 1 : 0] : -1;
      width[z] = (cr ? d->win_hi[dcz > 0 ? 1 : 0] : 1) - kmin[z] + 1;
    }
    const int ncells = 3 * (width[0] + width[1] + width[2]);
    for (int r0 = 0; r0 < ncells; r0 += 32) {
      // this lane's cell (t < ncells): row z, dcy, window slot k
      const int t = r0 + lane;
      int z = 0, rem = t;
      if (rem >= 3 * width[0]) {
        rem -= 3 * width[0];
        z = 1;
        if (rem >= 3 * width[1]) {
          rem -= 3 * width[1];
          z = 2;
        }
      }
      const int wz = z == 0 ? width[0] : z == 1 ? width[1] : width[2];
      const int dcz = z - 1, dcy = rem / wz - 1, k = (z == 0 ? kmin[0] : z == 1 ? kmin[1] : kmin[2]) + rem % wz;
      const int crz = z == 0 ? cross[0] : z == 1 ? cross[1] : cross[2];
      const int cjz = z == 0 ? czj[0] : z == 1 ? czj[1] : czj[2];
      // pruned exactly as rb_list_body prunes rows and cells
      const float az = __fmaf_rn((float)dcz, lz, qi.z);
      const float gz = box_gap(az, hz);
      const float ay = __fmaf_rn((float)dcy, ly, qi.y);
      const float gy = box_gap(ay, hy);
      const float gyz = __fmaf_rn(gy, gy, __fmul_rn(gz, gz));
      const int slot = slot_code(k, dcy, dcz, crz);
      const float ax = __fadd_rn(qi.x, s_offx[t < ncells ? slot : 0]);
      const float gx = box_gap(ax, hx);
      const bool scan = t < ncells && __fmul_rn(gz, gz) < rl2 && gyz < rl2 &&
                        __fmaf_rn(gx, gx, gyz) < rl2;
      int j0 = 0, j1 = 0;
      if (scan) {
        const int cyj = wrap_index(cy - dcy, g.nc[1]);
        const int cj = g.nc[0] * (cyj + g.nc[1] * cjz) +
                       wrap_index(cx - k + (crz ? dcz * mb : 0), g.nc[0]);
        // clamped so that a corrupt range can never leave the particle arrays
        j0 = min(max(w.cell_start[cj], 0), g.n);
        j1 = min(max(w.cell_start[cj + 1], j0), g.n);
      }
      // the particle itself is a candidate only in its own cell's slot
      const int self_j = slot == slot_code(0, 0, 0, 0) ? i : -1;
      // pass 1 counts the kept candidates, pass 2 writes them from the offset
      auto sweep = [&](bool write, int m) {
        int c = 0;
        for (int j = j0; j < j1; j += 4) {
          float4 q[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) q[u] = __ldg(b.pb + min(j + u, j1 - 1));
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int jj = j + u;
            if (jj < j1 && list_dist2(ax, ay, az, q[u]) < rl2 && jj != self_j) {
              if (write) out[min(m + c, cap) * 32] = ((uint32_t)jj << kSlotBits) | (uint32_t)slot;
              ++c;
            }
          }
        }
        return c;
      };
      const int c = sweep(false, 0);
      int incl = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      if (c > 0) sweep(true, total + incl - c);
      total += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (lane == 0) {
      w.ncount[i] = total;
      if (total > g.maxnb) atomicOr(&d->err, (int)kErrCapacity);
    }
  }
  // largest and total list length, one atomic each per block
  if (lane == 0) s_cnt[warp] = total;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    int mx = 0;
    for (int k = 0; k < kListWppWarps; ++k) {
      t += (unsigned long long)s_cnt[k];
      mx = max(mx, s_cnt[k]);
    }
    atomicMax(&d->list_max, mx);
    atomicAdd((unsigned long long *)&d->list_entries, t);
  }
}

// ------------------------------------------------------------ rebuild: bonds
// Slot of every bond: its LE minimum image at the build (FP64), expressed as
// build-cell offset + image, then matched to the 90-slot table.
template <class R>
__device__ __forceinline__ void rb_bonds_body(const Geom g, Dyn *__restrict__ d, Bufs<R> s0,
                                              Bufs<R> s1, Work w, int target_cur, int bx) {
  const int tgt = target_cur ? d->cur : 1 - d->cur;
  const Bufs<R> b = pick(tgt, s0, s1);
  const int k = bx * blockDim.x + threadIdx.x;
  if (k >= g.n) return;
  const int gid = b.gid[k];
  const double dXb = d->dX_build;
  const double fb = d->f_build;
  int ck[3];
  cell_coords(g, __float_as_int(b.pb[k].w), ck[0], ck[1], ck[2]);
  for (int q = 0; q < g.maxb; ++q) {
    const int h = w.bond_gid[(size_t)gid * g.maxb + q];
    uint32_t entry = kNoBond;
    if (h >= 0 && h < g.n) {
      const int j = min(max(w.rank[h], 0), g.n - 1);
      const double *xi = w.Xs + 3 * (size_t)k;
      const double *xj = w.Xs + 3 * (size_t)j;
      double dd[3] = {xi[0] - xj[0], xi[1] - xj[1], xi[2] - xj[2]};
      double nz = 0.0;
      if (dd[2] > 0.5 * g.L[2]) { dd[2] -= g.L[2]; dd[0] -= dXb; nz = 1.0; }
      else if (dd[2] < -0.5 * g.L[2]) { dd[2] += g.L[2]; dd[0] += dXb; nz = -1.0; }
      // quotients by multiplication with the stored inverses: each is within
      // rounding of an integer or of zero, far from a rint tie
      dd[0] -= g.L[0] * rint(dd[0] * g.inv_L[0]);
      dd[1] -= g.L[1] * rint(dd[1] * g.inv_L[1]);
      int cj[3];
      cell_coords(g, __float_as_int(b.pb[j].w), cj[0], cj[1], cj[2]);
      // off = X_ref(i) - X_ref(j) - image shift, shift = (x_i - x_j) - d
      double off[3];
      for (int a = 0; a < 3; ++a) {
        const double shift = (xi[a] - xj[a]) - dd[a];
        off[a] = (double)(ck[a] - cj[a]) * g.lc[a] - shift;
      }
      const int dcz = (int)rint(off[2] * g.inv_lcd[2]);
      const int dcy = (int)rint(off[1] * g.inv_lcd[1]);
      const int cross = nz != 0.0 ? 1 : 0;
      const int kk = (int)rint((off[0] - (cross ? (double)dcz * fb : 0.0)) * g.inv_lcd[0]);
      if (dcz < -1 || dcz > 1 || dcy < -1 || dcy > 1 || kk < -3 || kk > 4 ||
          (cross && dcz == 0)) {
        atomicOr(&d->err, (int)kErrSlot);
      } else {
        entry = make_entry(j, slot_code(kk, dcy, dcz, cross));
      }
    }
    w.bond_e[(size_t)k * g.maxb + q] = entry;
  }
}
template <class R>
__global__ void __launch_bounds__(256) k_rb_bonds(const __grid_constant__ Geom g,
                                                  Dyn *__restrict__ d, Bufs<R> s0, Bufs<R> s1,
                                                  Work w, int target_cur) {
  rb_bonds_body<R>(g, d, s0, s1, w, target_cur, (int)blockIdx.x);
}

__device__ __forceinline__ void rb_finish_body(Dyn *__restrict__ d, int bx) { d->cur = 1 - d->cur; }
__global__ void k_rb_finish(Dyn *__restrict__ d) {
  rb_finish_body(d, (int)blockIdx.x);
}

// ------------------------------------------------------------------ exports
template <class R>
__global__ void __launch_bounds__(256) k_export(Geom g, Dyn *__restrict__ d, Bufs<R> s0,
                                                Bufs<R> s1, double *__restrict__ stage) {
  const Bufs<R> b = pick(d->cur, s0, s1);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.n) return;
  double x[3];
  absolute_position<R>(g, b, i, x);
  const V4<R> v = b.v[i];
  double vx = (double)v.x;
  le_wrap(g, d->dX, x, vx);
  const size_t o = 3 * (size_t)b.gid[i];
  stage[o] = x[0];
  stage[o + 1] = x[1];
  stage[o + 2] = x[2];
  const size_t q = 3 * (size_t)g.n + o;
  stage[q] = vx;
  stage[q + 1] = (double)v.y;
  stage[q + 2] = (double)v.z;
}

// The same output for caller ids [g0, g1), read through the rank table:
// consecutive threads write consecutive ids, so a piece of the output is
// complete (and can be copied to the host) as soon as its launch is.
template <class R>
__global__ void __launch_bounds__(256) k_export_ids(Geom g, Dyn *__restrict__ d, Bufs<R> s0,
                                                    Bufs<R> s1, const int *__restrict__ rank,
                                                    double *__restrict__ stage, int g0, int g1) {
  const Bufs<R> b = pick(d->cur, s0, s1);
  const int id = g0 + (int)(blockIdx.x * blockDim.x + threadIdx.x);
  if (id >= g1) return;
  const int i = min(max(rank[id], 0), g.n - 1);
  double x[3];
  absolute_position<R>(g, b, i, x);
  const V4<R> v = b.v[i];
  double vx = (double)v.x;
  le_wrap(g, d->dX, x, vx);
  const size_t o = 3 * (size_t)id;
  stage[o] = x[0];
  stage[o + 1] = x[1];
  stage[o + 2] = x[2];
  const size_t q = 3 * (size_t)g.n + o;
  stage[q] = vx;
  stage[q + 1] = (double)v.y;
  stage[q + 2] = (double)v.z;
}

template <class R>
__global__ void __launch_bounds__(256) k_export_forces(Geom g, Dyn *__restrict__ d, Bufs<R> s0,
                                                       Bufs<R> s1, double *__restrict__ stage) {
  const Bufs<R> b = pick(d->cur, s0, s1);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.n) return;
  const V4<R> f = b.fc[i];
  const size_t o = 3 * (size_t)b.gid[i];
  stage[o] = (double)f.x;
  stage[o + 1] = (double)f.y;
  stage[o + 2] = (double)f.z;
}

// Instantaneous Eq. 15 tensor and potential energy: per-block FP64 partials
// [b][0..8] = sum m u(x)u + 1/2 sum_j d(x)F (row-major), [b][9] = energy.
template <class R, bool BONDS>
__global__ void __launch_bounds__(128) k_observe(Geom g, Dyn *__restrict__ d, Bufs<R> s0,
                                                 Bufs<R> s1, Work w, double *__restrict__ part) {
  __shared__ double s_off[kNumSlots][3];
  __shared__ double s_acc[10][128];
  const int t = threadIdx.x;
  for (int e = t; e < kNumSlots; e += blockDim.x) {
    s_off[e][0] = d->off[e][0];
    s_off[e][1] = d->off[e][1];
    s_off[e][2] = d->off[e][2];
  }
  __syncthreads();
  const Bufs<R> b = pick(d->cur, s0, s1);
  const int i = blockIdx.x * blockDim.x + t;
  double acc[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  if (i < g.n) {
    double xi[3];
    absolute_position<R>(g, b, i, xi);
    int ci[3];
    cell_coords(g, __float_as_int(b.pb[i].w), ci[0], ci[1], ci[2]);
    const double rc2 = g.rc * g.rc;
    double eshift = 0.0;
    if (g.lj_shift) {
      const double c2 = g.sigma * g.sigma / rc2, c6 = c2 * c2 * c2;
      eshift = 4.0 * g.eps * (c6 * c6 - c6);
    }
    auto pair = [&](int j, int slot, bool bond) {
      double xj[3];
      absolute_position<R>(g, b, j, xj);
      int cj[3];
      cell_coords(g, __float_as_int(b.pb[j].w), cj[0], cj[1], cj[2]);
      double dd[3];
      for (int a = 0; a < 3; ++a) {
        // reference-relative displacements, as in the pair kernel, in FP64
        const double pi_a = xi[a] - ((double)ci[a] + 0.5) * g.lc[a];
        const double pj_a = xj[a] - ((double)cj[a] + 0.5) * g.lc[a];
        dd[a] = (pi_a - pj_a) + s_off[slot][a];
      }
      const double r2 = dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2];
      double fr = 0.0, e = 0.0;
      if (!bond) {
        if (!(r2 < rc2)) return;
        const double s2 = g.sigma * g.sigma / r2, s6 = s2 * s2 * s2;
        fr = 24.0 * g.eps * (2.0 * s6 * s6 - s6) / r2;
        e = 4.0 * g.eps * (s6 * s6 - s6) - eshift;
      } else {
        const double R02 = g.fene_R0 * g.fene_R0, x = 1.0 - r2 / R02;
        if (!(x > 0.0)) return;
        fr = -g.fene_k / x;
        e = -0.5 * g.fene_k * R02 * log(x);
      }
      for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c) acc[3 * a + c] += 0.5 * dd[a] * fr * dd[c];
      acc[9] += 0.5 * e;
    };
    const int cnt = min(w.ncount[i], g.maxnb);
    const uint32_t *nl = w.nbr + (size_t)(i >> 5) * (size_t)g.maxnb * 32u + (i & 31);
    for (int k = 0; k < cnt; ++k) {
      const uint32_t e = nl[(size_t)k * 32u];
      pair(entry_index(e), entry_slot(e), false);
    }
    if constexpr (BONDS) {
      for (int q = 0; q < g.maxb; ++q) {
        const uint32_t e = w.bond_e[(size_t)i * g.maxb + q];
        if (e == kNoBond) break;
        pair(entry_index(e), entry_slot(e), true);
      }
      if (g.cd.ang_k != 0.0) {
        // Eq. 12 (k_a (1 + cos theta)): the energy once per angle at its
        // middle bead, the virial a (x) F_end at each end bead
        const double ka = g.cd.ang_k;
        auto sepd = [&](int o, uint32_t e, double dd[3]) {
          double xo[3], xq[3];
          int co[3], cq[3];
          const int q = entry_index(e);
          absolute_position<R>(g, b, o, xo);
          absolute_position<R>(g, b, q, xq);
          cell_coords(g, __float_as_int(b.pb[o].w), co[0], co[1], co[2]);
          cell_coords(g, __float_as_int(b.pb[q].w), cq[0], cq[1], cq[2]);
          const int slot = entry_slot(e);
          for (int a = 0; a < 3; ++a)
            dd[a] = ((xo[a] - ((double)co[a] + 0.5) * g.lc[a]) -
                     (xq[a] - ((double)cq[a] + 0.5) * g.lc[a])) + s_off[slot][a];
        };
        auto cosang = [](const double a[3], const double c[3], double ah[3], double ch[3],
                         double &la) {
          la = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
          const double lc = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
          for (int k = 0; k < 3; ++k) {
            ah[k] = a[k] / la;
            ch[k] = c[k] / lc;
          }
          return ah[0] * ch[0] + ah[1] * ch[1] + ah[2] * ch[2];
        };
        for (int u = 0; u < g.maxb; ++u) {
          const uint32_t eu = w.bond_e[(size_t)i * g.maxb + u];
          if (eu == kNoBond) break;
          double du[3];
          sepd(i, eu, du);
          for (int v = u + 1; v < g.maxb; ++v) {
            const uint32_t ev = w.bond_e[(size_t)i * g.maxb + v];
            if (ev == kNoBond) break;
            double dv[3], a[3], c[3], ah[3], ch[3], la;
            sepd(i, ev, dv);
            for (int k = 0; k < 3; ++k) {
              a[k] = -du[k];
              c[k] = -dv[k];
            }
            acc[9] += ka * (1.0 + cosang(a, c, ah, ch, la));
          }
          const int j = entry_index(eu);
          for (int q = 0; q < g.maxb; ++q) {
            const uint32_t ek = w.bond_e[(size_t)j * g.maxb + q];
            if (ek == kNoBond) break;
            if (entry_index(ek) == i) continue;
            double dk[3], c[3], ah[3], ch[3], la;
            sepd(j, ek, dk);
            for (int k = 0; k < 3; ++k) c[k] = -dk[k];
            const double ct = cosang(du, c, ah, ch, la);
            for (int a = 0; a < 3; ++a)
              for (int cc = 0; cc < 3; ++cc)
                acc[3 * a + cc] += du[a] * (-ka * (ch[cc] - ct * ah[cc]) / la);
          }
        }
      }
    }
    const V4<R> v = b.v[i];
    const double zu = (double)b.p[i].z + (double)b.p[i].w;
    const double u[3] = {(double)v.x - g.shear_rate * (zu - 0.5 * g.L[2]), (double)v.y,
                         (double)v.z};
    for (int a = 0; a < 3; ++a)
      for (int c = 0; c < 3; ++c) acc[3 * a + c] += g.mass * u[a] * u[c];
  }
  for (int q = 0; q < 10; ++q) s_acc[q][t] = acc[q];
  __syncthreads();
  if (t < 10) {
    double s = 0.0;
    for (int k = 0; k < blockDim.x; ++k) s += s_acc[t][k];
    part[(size_t)blockIdx.x * 16 + t] = s;
  }
}


// ------------------------------------------------------------ batched steps
// One launch per kernel kind for a whole batch group: each block locates its
// member in the kind's block prefix table and runs that member's own kernel
// body.  The rebuild kinds look up the same in the kind's table of rebuilding
// members (kb_activate), so their blocks past those members' exit at once.
#define LE_MEMBER(KIND)                                            \
  const int *off_ = off + (KIND) * (M + 1);                        \
  const int m_ = batch_member(off_, M, (int)blockIdx.x);           \
  const MemberDev<R> &q = mem[m_];                                 \
  const int bx_ = (int)blockIdx.x - off_[m_]
#define LE_ACTIVE(KIND)                                                                    \
  int m_, bx_;                                                                             \
  if (!batch_active(act + (KIND) * batch_act_stride(M), M, (int)blockIdx.x, m_, bx_)) return; \
  const MemberDev<R> &q = mem[m_]

template <class R>
__global__ void __launch_bounds__(kDriftThreads) kb_drift(const MemberDev<R> *__restrict__ mem,
                                                          const int *__restrict__ off, int M) {
  LE_MEMBER(kB256);
  drift_body<R>(q.g, q.d, q.s0, q.s1, bx_);
}

template <class R>
__global__ void __launch_bounds__(128) kb_decide(const MemberDev<R> *__restrict__ mem) {
  const MemberDev<R> &q = mem[blockIdx.x];
  decide_body(q.g, q.d, q.w, cudaGraphConditionalHandle(0), 0, 0);
}

// The rebuild tables of every kind (batch_act_stride) from the decisions
// kb_decide has just written: per kind, a block-wide scan over the members
// (in chunks of the block) of "rebuilds and has blocks of this kind" and of
// the block counts of those that do.
template <class R>
__global__ void __launch_bounds__(kActThreads) kb_activate(const MemberDev<R> *__restrict__ mem,
                                                           const int *__restrict__ off, int M,
                                                           int *__restrict__ act) {
  __shared__ int s_a[kBKinds][kActThreads / 32], s_b[kBKinds][kActThreads / 32];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nw = kActThreads / 32;
  int ca[kBKinds], cb[kBKinds];  // members and blocks listed so far (the same in every thread)
#pragma unroll
  for (int k = 0; k < kBKinds; ++k) ca[k] = cb[k] = 0;
  for (int m0 = 0; m0 < M; m0 += kActThreads) {
    const int m = m0 + t;
    const bool reb = m < M && mem[m].d->rebuild != 0;
    int nb[kBKinds], ia[kBKinds], ib[kBKinds];
#pragma unroll
    for (int k = 0; k < kBKinds; ++k) {
      const int *o = off + k * (M + 1);
      nb[k] = reb ? o[m + 1] - o[m] : 0;
      ia[k] = nb[k] > 0 ? 1 : 0;
      ib[k] = nb[k];
    }
    // inclusive scans within the warp, then across the warps' totals
#pragma unroll
    for (int sh = 1; sh < 32; sh <<= 1) {
#pragma unroll
      for (int k = 0; k < kBKinds; ++k) {
        const int xa = __shfl_up_sync(0xffffffffu, ia[k], sh);
        const int xb = __shfl_up_sync(0xffffffffu, ib[k], sh);
        if (lane >= sh) {
          ia[k] += xa;
          ib[k] += xb;
        }
      }
    }
    if (lane == 31) {
#pragma unroll
      for (int k = 0; k < kBKinds; ++k) {
        s_a[k][warp] = ia[k];
        s_b[k][warp] = ib[k];
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kBKinds; ++k) {
      int pa = 0, pb = 0, ta = 0, tb = 0;
      for (int w2 = 0; w2 < nw; ++w2) {
        const int xa = s_a[k][w2], xb = s_b[k][w2];
        if (w2 < warp) {
          pa += xa;
          pb += xb;
        }
        ta += xa;
        tb += xb;
      }
      if (nb[k] > 0) {
        int *a = act + k * batch_act_stride(M);
        const int pos = ca[k] + pa + ia[k] - 1;
        a[1 + pos] = m;
        a[1 + M + pos] = cb[k] + pb + ib[k] - nb[k];
      }
      ca[k] += ta;
      cb[k] += tb;
    }
    __syncthreads();  // the warp totals of the next chunk
  }
  if (t == 0) {
#pragma unroll
    for (int k = 0; k < kBKinds; ++k) {
      int *a = act + k * batch_act_stride(M);
      a[0] = ca[k];
      a[1 + M + ca[k]] = cb[k];
    }
  }
}

template <class R>
__global__ void __launch_bounds__(256) kb_rb_bin(const MemberDev<R> *__restrict__ mem,
                                                 const int *__restrict__ act, int M) {
  LE_ACTIVE(kB256);
  rb_bin_body<R>(q.g, q.d, q.s0, q.s1, q.w, bx_);
}

template <class R>
__global__ void __launch_bounds__(256) kb_rb_permute(const MemberDev<R> *__restrict__ mem,
                                                     const int *__restrict__ act, int M) {
  LE_ACTIVE(kB256);
  const int fin = q.sort_passes & 1;
  rb_permute_body<R>(q.g, q.d, q.s0, q.s1, q.w, q.w.key[fin], q.w.val[fin], bx_);
}

template <class R>
__global__ void __launch_bounds__(kListMaxThreads, 3) kb_rb_list(
    const MemberDev<R> *__restrict__ mem, const int *__restrict__ act, int M) {
  LE_ACTIVE(kBList);
  rb_list_body<R>(q.g, q.d, q.s0, q.s1, q.w, 0, VBlock{bx_});
}

template <class R>
__global__ void __launch_bounds__(256) kb_rb_bonds(const MemberDev<R> *__restrict__ mem,
                                                   const int *__restrict__ act, int M) {
  LE_ACTIVE(kB256);
  if (q.g.maxb == 0) return;
  rb_bonds_body<R>(q.g, q.d, q.s0, q.s1, q.w, 0, bx_);
}

template <class R>
__global__ void kb_rb_finish(const MemberDev<R> *__restrict__ mem, const int *__restrict__ act,
                             int M) {
  LE_ACTIVE(kBOne);
  (void)bx_;
  rb_finish_body(q.d, 0);
}

template <class R, bool BONDS, bool DPD>
__global__ void __launch_bounds__(kForceThreads, sizeof(R) == 8 ? 1 : DPD ? 2 : LE_FORCE_MINB32)
    kb_force(const MemberDev<R> *__restrict__ mem, const int *__restrict__ off, int M, int mode) {
  LE_MEMBER(kBForce);
  force_body<R, BONDS, DPD>(q.g, q.d, q.s0, q.s1, q.w, mode, VBlock{bx_});
}

template <class R>
__global__ void __launch_bounds__(256) kb_vcopy(const MemberDev<R> *__restrict__ mem,
                                                const int *__restrict__ off, int M) {
  LE_MEMBER(kB256);
  vcopy_body<R>(q.g, q.d, q.s0, q.s1, q.w, bx_);
}
#undef LE_MEMBER
#undef LE_ACTIVE

template <class R>
void batch_step(const BatchGrid &bg, cudaStream_t st, bool drift, int mode) {
  const MemberDev<R> *mem = static_cast<const MemberDev<R> *>(bg.mem);
  const int M = bg.M;
  const int *off = bg.off;
  const int *act = bg.act;
  const int n256 = bg.blocks[kB256];
  if (drift) kb_drift<R><<<n256, kDriftThreads, 0, st>>>(mem, off, M);
  kb_decide<R><<<M, 128, 0, st>>>(mem);
  kb_activate<R><<<1, kActThreads, 0, st>>>(mem, off, M, bg.act);
  kb_rb_bin<R><<<n256, 256, 0, st>>>(mem, act, M);
  launch_batch_sort(bg, st);
  kb_rb_permute<R><<<n256, 256, 0, st>>>(mem, act, M);
  kb_rb_list<R><<<bg.blocks[kBList], bg.list_threads, 0, st>>>(mem, act, M);
  if (bg.bonds) kb_rb_bonds<R><<<n256, 256, 0, st>>>(mem, act, M);
  kb_rb_finish<R><<<M, 1, 0, st>>>(mem, act, M);
  const size_t smem = sizeof(long long) * 3 * (size_t)bg.nbins;
  const int nf = bg.blocks[kBForce];
  if (bg.dpd) {
    if (bg.bonds) kb_force<R, true, true><<<nf, bg.force_threads, smem, st>>>(mem, off, M, 0);
    else kb_force<R, false, true><<<nf, bg.force_threads, smem, st>>>(mem, off, M, 0);
    kb_vcopy<R><<<n256, 256, 0, st>>>(mem, off, M);
  } else if (bg.bonds) {
    kb_force<R, true, false><<<nf, bg.force_threads, smem, st>>>(mem, off, M, mode);
  } else {
    kb_force<R, false, false><<<nf, bg.force_threads, smem, st>>>(mem, off, M, mode);
  }
}

// Failure-detection self-test: one warp waits on an mbarrier that nothing
// arrives on, through the same bounded wait as the pair kernel, and records
// whether the wait gave up (1) or, impossibly, completed (0).
__global__ void k_wait_probe(int *out) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  mbar_init_fence();
  __syncthreads();
  const bool ok = mbar_wait(&bar, 0u);
  if (threadIdx.x == 0) out[0] = ok ? 0 : 1;
}

}  // namespace

void launch_wait_probe(int *out, cudaStream_t st) { k_wait_probe<<<1, 32, 0, st>>>(out); }

// ------------------------------------------------------------------ launchers
#define LE_DISPATCH(s, FN)            \
  do {                                \
    if ((s).prec == 1) {              \
      FN(float, (s).f32[0], (s).f32[1]);  \
    } else {                          \
      FN(double, (s).f64[0], (s).f64[1]); \
    }                                 \
  } while (0)

void launch_drift(const SysDev &s, cudaStream_t st) {
  const int nb = blocks_for(s.g.n, kDriftThreads);
#define FN(R, A, B) k_drift<R><<<nb, kDriftThreads, 0, st>>>(s.g, s.dyn, A, B)
  LE_DISPATCH(s, FN);
#undef FN
}

void launch_decide(const SysDev &s, cudaGraphConditionalHandle h, int use_cond, cudaStream_t st) {
  k_decide<<<1, 128, 0, st>>>(s.g, s.dyn, s.w, h, use_cond);
}

void launch_fold(const SysDev &s, cudaStream_t st) { k_fold<<<1, 256, 0, st>>>(s.g, s.dyn, s.w); }

bool can_fuse_drift(const SysDev &s) { return s.prec == 1 && s.g.thermostat != 3; }

void launch_force(const SysDev &s, int mode, cudaStream_t st) {
  const int nb = blocks_for(s.g.n, s.force_threads);
  const size_t smem = sizeof(long long) * 3 * (size_t)s.g.nbins;
  const bool bonds = s.g.maxb > 0;
  const bool dpd = s.g.thermostat == 3;
#define K3(R, BO, DP, A, B) \
  k_force<R, BO, DP><<<nb, s.force_threads, smem, st>>>(s.g, s.dyn, A, B, s.w, mode)
#define FN(R, A, B)                   \
  do {                                \
    if (dpd) {                        \
      if (bonds)                      \
        K3(R, true, true, A, B);      \
      else                            \
        K3(R, false, true, A, B);     \
      k_vcopy<R><<<blocks_for(s.g.n, 256), 256, 0, st>>>(s.g, s.dyn, A, B, s.w); \
    } else if (bonds) {               \
      K3(R, true, false, A, B);       \
    } else {                          \
      K3(R, false, false, A, B);      \
    }                                 \
  } while (0)
  LE_DISPATCH(s, FN);
#undef FN
#undef K3
}

// The list build in the form the system's size calls for.  A warp per
// particle does about twice the candidate tests' instructions of a thread
// per particle but waits on memory once per particle instead of once per
// cell; it pays while the candidate tests, n x particles per cell, stay
// under kSmallListTests (measured on GB300: a 4,000-particle LJ box at 19
// per cell 12% faster, a 20,000-bead melt at 2.5 per cell 6% faster, a
// 32,000-particle LJ box 10% slower).  The same entries in the same order
// either way.
constexpr double kSmallListTests = 131072.0;
template <class R>
static void launch_list(const SysDev &s, Bufs<R> A, Bufs<R> B, int target_cur, cudaStream_t st) {
  const double tests = (double)s.g.n * (double)s.g.n / (double)s.g.ncell;
  if (tests <= kSmallListTests)
    k_rb_list_wpp<R><<<blocks_for(s.g.n, kListWppWarps), 32 * kListWppWarps, 0, st>>>(
        s.g, s.dyn, A, B, s.w, target_cur);
  else
    k_rb_list<R><<<blocks_for(s.g.n, s.list_threads), s.list_threads, 0, st>>>(
        s.g, s.dyn, A, B, s.w, target_cur);
}

static void rebuild_tail(const SysDev &s, cudaStream_t st) {
  const int n = s.g.n;
  radix_sort_pairs(const_cast<uint32_t **>(s.w.key), const_cast<uint32_t **>(s.w.val), s.w.hist,
                   s.sort_part, n, s.g.sort_bits, s.sort_blocks, st);
  const uint32_t *skey = s.w.key[s.sort_passes & 1];
  const uint32_t *sval = s.w.val[s.sort_passes & 1];
  const int nb = blocks_for(n, 256);
#define FN(R, A, B) k_rb_permute<R><<<nb, 256, 0, st>>>(s.g, s.dyn, A, B, s.w, skey, sval)
  LE_DISPATCH(s, FN);
#undef FN
#define FN(R, A, B) launch_list<R>(s, A, B, 0, st)
  LE_DISPATCH(s, FN);
#undef FN
  if (s.g.maxb > 0) {
#define FN(R, A, B) k_rb_bonds<R><<<nb, 256, 0, st>>>(s.g, s.dyn, A, B, s.w, 0)
    LE_DISPATCH(s, FN);
#undef FN
  }
  k_rb_finish<<<1, 1, 0, st>>>(s.dyn);
}

void launch_rebuild(const SysDev &s, bool from_import, cudaStream_t st) {
  const int nb = blocks_for(s.g.n, 256);
  if (!from_import) {
#define FN(R, A, B) k_rb_bin<R><<<nb, 256, 0, st>>>(s.g, s.dyn, A, B, s.w)
    LE_DISPATCH(s, FN);
#undef FN
  }
  rebuild_tail(s, st);
}

void launch_tables(const SysDev &s, cudaStream_t st) { k_tables<<<1, 128, 0, st>>>(s.g, s.dyn); }

void launch_relist(const SysDev &s, cudaStream_t st) {
  const int n = s.g.n;
  const int nb = blocks_for(n, 256);
  launch_tables(s, st);
#define FN(R, A, B) k_relist_prep<R><<<nb, 256, 0, st>>>(s.g, s.dyn, A, B, s.w)
  LE_DISPATCH(s, FN);
#undef FN
  k_rb_ranges<<<nb, 256, 0, st>>>(s.g, s.w.key[0], s.w.cell_start);
#define FN(R, A, B) launch_list<R>(s, A, B, 1, st)
  LE_DISPATCH(s, FN);
#undef FN
  if (s.g.maxb > 0) {
#define FN(R, A, B) k_rb_bonds<R><<<nb, 256, 0, st>>>(s.g, s.dyn, A, B, s.w, 1)
    LE_DISPATCH(s, FN);
#undef FN
  }
}

void launch_import(const SysDev &s, cudaStream_t st, int i0, int i1) {
  if (i1 < 0) i1 = s.g.n;
  if (i1 <= i0) return;
  const int nb = blocks_for(i1 - i0, 256);
#define FN(R, A, B) k_import<R><<<nb, 256, 0, st>>>(s.g, s.dyn, A, B, s.w, s.stage, i0, i1)
  LE_DISPATCH(s, FN);
#undef FN
}

void launch_export(const SysDev &s, cudaStream_t st) {
  const int nb = blocks_for(s.g.n, 256);
#define FN(R, A, B) k_export<R><<<nb, 256, 0, st>>>(s.g, s.dyn, A, B, s.stage)
  LE_DISPATCH(s, FN);
#undef FN
}

void launch_export_ids(const SysDev &s, cudaStream_t st, int g0, int g1) {
  if (g1 <= g0) return;
  const int nb = blocks_for(g1 - g0, 256);
#define FN(R, A, B) k_export_ids<R><<<nb, 256, 0, st>>>(s.g, s.dyn, A, B, s.w.rank, s.stage, g0, g1)
  LE_DISPATCH(s, FN);
#undef FN
}

void launch_export_forces(const SysDev &s, cudaStream_t st) {
  const int nb = blocks_for(s.g.n, 256);
#define FN(R, A, B) k_export_forces<R><<<nb, 256, 0, st>>>(s.g, s.dyn, A, B, s.stage)
  LE_DISPATCH(s, FN);
#undef FN
}

int observe_blocks(const SysDev &s) { return blocks_for(s.g.n, 128); }

void launch_observe(const SysDev &s, cudaStream_t st) {
  const int nb = observe_blocks(s);
  const bool bonds = s.g.maxb > 0;
#define FN(R, A, B)                                                              \
  do {                                                                           \
    if (bonds)                                                                   \
      k_observe<R, true><<<nb, 128, 0, st>>>(s.g, s.dyn, A, B, s.w, s.partials);  \
    else                                                                         \
      k_observe<R, false><<<nb, 128, 0, st>>>(s.g, s.dyn, A, B, s.w, s.partials); \
  } while (0)
  LE_DISPATCH(s, FN);
#undef FN
}

void launch_batch_step(const BatchGrid &bg, cudaStream_t st, bool drift, bool fuse) {
  const bool can = batch_can_fuse_drift(bg);
  const int mode = fuse && can ? 2 : 0;
  if (bg.prec == 1) batch_step<float>(bg, st, drift || !can, mode);
  else batch_step<double>(bg, st, true, 0);
}

}  // namespace le
