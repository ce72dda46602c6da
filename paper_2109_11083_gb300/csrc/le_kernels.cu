// CUDA kernels of the Lees-Edwards shear-flow MD step (sm_103a).
//
// One step n -> n+1 (velocity Verlet, the order of every implementation in
// this repository):
//   k_drift   v += dt/2m Ftot(n); r += dt v; max displacement since the build
//   k_decide  dX(n+1) from the integer step (Eq. 4); rebuild trigger
//             2*max|dr| + |shift of the sheared images since the build| >= skin;
//             per-step slot-offset table; folds the previous step's samples
//   [if rebuild: k_rb_bin -> radix sort -> k_rb_permute -> k_rb_ranges ->
//                k_rb_list -> k_rb_bonds -> k_rb_finish]
//   k_force   LJ (Eq. 9/10) over the Verlet list + FENE (Eq. 11) under the LE
//             minimum image; Ftot = Fc - xi m (v - v_s e_x) + random (Eq. 5);
//             v += dt/2m Ftot; Eq. 15 xz stress, peculiar temperature and the
//             vx(z) profile as fixed-point integer sums.
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
  x[0] -= Lx * floor(x[0] / Lx);
  if (x[0] >= Lx) x[0] -= Lx;
  x[1] -= Ly * floor(x[1] / Ly);
  if (x[1] >= Ly) x[1] -= Ly;
  return nz;
}

__device__ __forceinline__ int cell_of(const Geom &g, const double x[3]) {
  int c[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    int k = (int)(x[a] / g.lc[a]);
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

// ------------------------------------------------------------------ k_drift
template <class R>
__global__ void __launch_bounds__(kDriftThreads) k_drift(Geom g, Dyn *__restrict__ d,
                                                         Bufs<R> s0, Bufs<R> s1) {
  const Bufs<R> b = pick(d->cur, s0, s1);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  float disp2 = 0.f;
  if (i < g.n) {
    const R half = R(0.5 * g.dt / g.mass);
    const R dt = R(g.dt);
    V4<R> v = b.v[i];
    const V4<R> f = b.ft[i];
    v.x += half * f.x;
    v.y += half * f.y;
    v.z += half * f.z;
    V4<R> p = b.p[i];
    if constexpr (sizeof(R) == 4) {
      float4 lo = b.plo[i];
      two_sum_acc(p.x, lo.x, dt * v.x);
      two_sum_acc(p.y, lo.y, dt * v.y);
      two_sum_acc(p.z, lo.z, dt * v.z);
      b.plo[i] = lo;
    } else {
      p.x += dt * v.x;
      p.y += dt * v.y;
      p.z += dt * v.z;
    }
    b.v[i] = v;
    b.p[i] = p;
    const float4 q = b.pb[i];
    const float dx = (float)p.x - q.x, dy = (float)p.y - q.y, dz = (float)p.z - q.z;
    disp2 = dx * dx + dy * dy + dz * dz;
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) disp2 = fmaxf(disp2, __shfl_xor_sync(0xffffffffu, disp2, o));
  __shared__ float sm[kDriftThreads / 32];
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = disp2;
  __syncthreads();
  if (threadIdx.x == 0) {
    float m = sm[0];
    for (int w = 1; w < kDriftThreads / 32; ++w) m = fmaxf(m, sm[w]);
    if (m > 0.f) atomicMax(&d->maxdisp2, __float_as_uint(m));
  }
}

// ------------------------------------------------------------------ k_decide
// One block.  Folds the previous step's fixed-point samples into the running
// sums, advances the step, evaluates the rebuild trigger and fills the slot
// offset table.
__global__ void __launch_bounds__(128) k_decide(Geom g, Dyn *__restrict__ d, Work w,
                                                cudaGraphConditionalHandle h) {
  __shared__ double s_sh;
  __shared__ int need_sh;
  const int t = threadIdx.x;
  const int pending = d->pending;
  if (pending) {
    for (int b = t; b < g.nbins; b += blockDim.x) {
      w.sum_prof[b] += (double)w.acc_prof[b] * kInvFixP;
      w.cnt_prof[b] += w.acc_prof[g.nbins + b];
      w.acc_prof[b] = 0;
      w.acc_prof[g.nbins + b] = 0;
    }
  }
  __syncthreads();
  if (t == 0) {
    if (pending) {
      const double V = g.L[0] * g.L[1] * g.L[2];
      d->sum_sxz += -(double)d->acc_sxz * kInvFix / V;
      d->sum_tpec += (double)d->acc_ke * kInvFix / (g.n > 1 ? 3.0 * g.n - 3.0 : 1.0);
      d->nsamples += 1;
      d->acc_sxz = 0;
      d->acc_ke = 0;
      d->pending = 0;
    }
    const long long n1 = d->step + 1;
    const double dX1 = image_offset(g, n1);
    const float maxd = sqrtf(__uint_as_float(d->maxdisp2));
    d->maxdisp2 = 0u;
    // continuous change of the image offset since the build (dX is reduced
    // modulo Lx; the shear sign tells which way it wrapped)
    double ds = dX1 - d->dX_build;
    if (g.shear_rate > 0.0 && ds < -0.5 * g.L[0]) ds += g.L[0];
    if (g.shear_rate < 0.0 && ds > 0.5 * g.L[0]) ds -= g.L[0];
    const double margin = 1e-6 * g.rl;
    const bool disp_need = 2.0 * (double)maxd * (1.0 + 1e-6) + margin >= g.skin;
    const bool need = d->force_rebuild || disp_need ||
                      (2.0 * (double)maxd * (1.0 + 1e-6) + fabs(ds) + margin >= g.skin);
    double s;
    if (need) {
      int m = (int)floor(dX1 / g.lc[0]);
      double f = dX1 - (double)m * g.lc[0];
      if (f >= g.lc[0]) { f -= g.lc[0]; m += 1; }
      if (f < 0.0) { f += g.lc[0]; m -= 1; }
      d->m_build = m;
      d->f_build = f;
      d->dX_build = dX1;
      d->build_step = n1;
      d->list_entries = 0;
      d->nrebuild += 1;
      if (!disp_need && !d->force_rebuild) d->nimage += 1;
      s = f;
    } else {
      s = d->f_build + ds;
    }
    d->s = s;
    d->dX = dX1;
    d->step = n1;
    d->rebuild = need ? 1 : 0;
    d->force_rebuild = 0;
    s_sh = s;
    need_sh = need ? 1 : 0;
    cudaGraphSetConditional(h, need ? 1u : 0u);
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

// Folds pending samples outside the step graph (end of a le_step call).
__global__ void k_fold(Geom g, Dyn *__restrict__ d, Work w) {
  const int t = threadIdx.x;
  const int pending = d->pending;
  if (pending) {
    for (int b = t; b < g.nbins; b += blockDim.x) {
      w.sum_prof[b] += (double)w.acc_prof[b] * kInvFixP;
      w.cnt_prof[b] += w.acc_prof[g.nbins + b];
      w.acc_prof[b] = 0;
      w.acc_prof[g.nbins + b] = 0;
    }
  }
  __syncthreads();
  if (t == 0 && pending) {
    const double V = g.L[0] * g.L[1] * g.L[2];
    d->sum_sxz += -(double)d->acc_sxz * kInvFix / V;
    d->sum_tpec += (double)d->acc_ke * kInvFix / (g.n > 1 ? 3.0 * g.n - 3.0 : 1.0);
    d->nsamples += 1;
    d->acc_sxz = 0;
    d->acc_ke = 0;
    d->pending = 0;
  }
}

// ------------------------------------------------------------------ k_force
template <class R, bool BONDS>
__global__ void __launch_bounds__(kForceThreads) k_force(Geom g, Dyn *__restrict__ d,
                                                         Bufs<R> s0, Bufs<R> s1, Work w,
                                                         int mode) {
  __shared__ V4<R> s_off[kNumSlots];
  __shared__ double s_red[2][kForceThreads / 32];
  extern __shared__ long long s_prof[];  // [2 * nbins]
  const int t = threadIdx.x;
  for (int e = t; e < kNumSlots; e += blockDim.x)
    s_off[e] = make4<R>(R(d->off[e][0]), R(d->off[e][1]), R(d->off[e][2]), R(0));
  const int cur = d->cur;
  const long long n1 = d->step;
  const bool sample = mode == 0 && g.sample_every > 0 && (n1 % g.sample_every) == 0;
  if (sample)
    for (int b = t; b < 2 * g.nbins; b += blockDim.x) s_prof[b] = 0;
  __syncthreads();

  const Bufs<R> b = pick(cur, s0, s1);
  const int i = blockIdx.x * blockDim.x + t;
  R sxz = R(0), ke = R(0);
  int bin = -1;
  R vxw = R(0);
  if (i < g.n) {
    const V4<R> pi = b.p[i];
    const int cnt = min(w.ncount[i], g.maxnb);
    const uint32_t *nl = w.nbr + (size_t)(i >> 5) * (size_t)g.maxnb * 32u + (i & 31);
    const R rc2 = R(g.rc * g.rc), sig2 = R(g.sigma * g.sigma), eps24 = R(24.0 * g.eps);
    R fx = R(0), fy = R(0), fz = R(0), vir = R(0);
    for (int k = 0; k < cnt; ++k) {
      const uint32_t e = __ldg(nl + (size_t)k * 32u);
      const int j = (int)(e & kIndexMask);
      const V4<R> pj = load4(b.p + j);
      const V4<R> o = s_off[e >> kIndexBits];
      const R dx = (pi.x - pj.x) + o.x;
      const R dy = (pi.y - pj.y) + o.y;
      const R dz = (pi.z - pj.z) + o.z;
      const R r2 = dx * dx + dy * dy + dz * dz;
      if (r2 < rc2) {
        const R ir2 = R(1) / r2;
        const R s2 = sig2 * ir2;
        const R s6 = s2 * s2 * s2;
        const R fr = eps24 * ir2 * s6 * (R(2) * s6 - R(1));
        const R tx = fr * dx;
        fx += tx;
        fy += fr * dy;
        fz += fr * dz;
        vir += tx * dz;
      }
    }
    if constexpr (BONDS) {
      const R R02 = R(g.fene_R0 * g.fene_R0), kf = R(g.fene_k);
      for (int q = 0; q < g.maxb; ++q) {
        const uint32_t e = w.bond_e[(size_t)i * g.maxb + q];
        if (e == kNoBond) break;
        const int j = (int)(e & kIndexMask);
        const V4<R> pj = load4(b.p + j);
        const V4<R> o = s_off[e >> kIndexBits];
        const R dx = (pi.x - pj.x) + o.x;
        const R dy = (pi.y - pj.y) + o.y;
        const R dz = (pi.z - pj.z) + o.z;
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
    }
    // Eq. 5: friction on the peculiar velocity plus the random force
    const V4<R> v = b.v[i];
    const R zu = pi.z + pi.w;  // unwrapped z (reference + displacement)
    const R vs = R(g.shear_rate) * (zu - R(0.5 * g.L[2]));
    R ftx = fx, fty = fy, ftz = fz;
    if (g.thermostat == 1) {
      R u[3];
      uniform3<R>(g, n1, b.gid[i], u);
      const R amp = R(sqrt(24.0 * g.xi * g.kT * g.mass / g.dt));
      const R xm = R(g.xi * g.mass);
      ftx += -xm * (v.x - vs) + amp * u[0];
      fty += -xm * v.y + amp * u[1];
      ftz += -xm * v.z + amp * u[2];
    }
    V4<R> nv = v;
    if (mode == 0) {
      const R half = R(0.5 * g.dt / g.mass);
      nv.x = v.x + half * ftx;
      nv.y = v.y + half * fty;
      nv.z = v.z + half * ftz;
    }
    b.fc[i] = make4<R>(fx, fy, fz, R(0));
    b.ft[i] = make4<R>(ftx, fty, ftz, R(0));
    b.v[i] = nv;
    if (!isfinite(ftx + fty + ftz) || !isfinite(nv.x + nv.y + nv.z))
      atomicOr(&d->err, (int)kErrNonfinite);
    if (sample) {
      const R m = R(g.mass);
      const R vpx = nv.x - vs;
      sxz = m * vpx * nv.z + R(0.5) * vir;
      ke = m * (vpx * vpx + nv.y * nv.y + nv.z * nv.z);
      R zw = zu, vw = nv.x;
      const R Lz = R(g.L[2]);
      if (zw >= Lz) {
        zw -= Lz;
        vw -= R(g.shear_rate * g.L[2]);
      } else if (zw < R(0)) {
        zw += Lz;
        vw += R(g.shear_rate * g.L[2]);
      }
      int bb = (int)floor((double)zw * (double)g.nbins / g.L[2]);
      bin = bb < 0 ? 0 : (bb >= g.nbins ? g.nbins - 1 : bb);
      vxw = vw;
    }
  }
  if (!sample) return;
  // deterministic block sums -> fixed-point integer atomics
  double a = (double)warp_sum(sxz);
  double c = (double)warp_sum(ke);
  if ((t & 31) == 0) {
    s_red[0][t >> 5] = a;
    s_red[1][t >> 5] = c;
  }
  if (bin >= 0) {
    atomicAdd((unsigned long long *)&s_prof[bin], (unsigned long long)(long long)__float2int_rn((float)vxw * (float)kFixP));
    atomicAdd((unsigned long long *)&s_prof[g.nbins + bin], 1ull);
  }
  __syncthreads();
  if (t == 0) {
    double A = 0.0, B = 0.0;
    for (int k = 0; k < kForceThreads / 32; ++k) {
      A += s_red[0][k];
      B += s_red[1][k];
    }
    atomicAdd((unsigned long long *)&d->acc_sxz, (unsigned long long)llrint(A * kFix));
    atomicAdd((unsigned long long *)&d->acc_ke, (unsigned long long)llrint(B * kFix));
    if (blockIdx.x == 0) d->pending = 1;
  }
  for (int q = t; q < g.nbins; q += blockDim.x) {
    const long long cnt = s_prof[g.nbins + q];
    if (cnt) {
      atomicAdd((unsigned long long *)&w.acc_prof[q], (unsigned long long)s_prof[q]);
      atomicAdd((unsigned long long *)&w.acc_prof[g.nbins + q], (unsigned long long)cnt);
    }
  }
}

// --------------------------------------------------------------- rebuild: bin
// Re-bases the current state: FP64 absolute position, LE wrap with the
// velocity jump at the current offset, new cell.  Writes X (pre-sort order)
// and the sort keys/values.
template <class R>
__global__ void __launch_bounds__(256) k_rb_bin(Geom g, Dyn *__restrict__ d, Bufs<R> s0,
                                                Bufs<R> s1, Work w) {
  const Bufs<R> b = pick(d->cur, s0, s1);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.n) return;
  double x[3];
  absolute_position<R>(g, b, i, x);
  V4<R> v = b.v[i];
  double vx = (double)v.x;
  if (le_wrap(g, d->dX, x, vx) != 0) {
    v.x = R(vx);
    b.v[i] = v;
  }
  w.X[3 * (size_t)i + 0] = x[0];
  w.X[3 * (size_t)i + 1] = x[1];
  w.X[3 * (size_t)i + 2] = x[2];
  w.key[0][i] = (uint32_t)cell_of(g, x);
  w.val[0][i] = (uint32_t)i;
}

// Initial load: caller-order FP64 positions/velocities (staging) wrapped as
// images at the current offset, into the current buffer set at row i.
template <class R>
__global__ void __launch_bounds__(256) k_import(Geom g, Dyn *__restrict__ d, Bufs<R> s0,
                                                Bufs<R> s1, Work w, const double *__restrict__ stage) {
  const Bufs<R> b = pick(d->cur, s0, s1);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.n) return;
  double x[3] = {stage[3 * (size_t)i], stage[3 * (size_t)i + 1], stage[3 * (size_t)i + 2]};
  double vx = stage[3 * (size_t)g.n + 3 * (size_t)i];
  const double vy = stage[3 * (size_t)g.n + 3 * (size_t)i + 1];
  const double vz = stage[3 * (size_t)g.n + 3 * (size_t)i + 2];
  // any number of images away: remove whole boxes along z first
  const double nzf = floor(x[2] / g.L[2]);
  if (nzf != 0.0) {
    x[2] -= nzf * g.L[2];
    x[0] -= nzf * d->dX;
    vx -= nzf * g.shear_rate * g.L[2];
  }
  le_wrap(g, d->dX, x, vx);
  w.X[3 * (size_t)i + 0] = x[0];
  w.X[3 * (size_t)i + 1] = x[1];
  w.X[3 * (size_t)i + 2] = x[2];
  w.key[0][i] = (uint32_t)cell_of(g, x);
  w.val[0][i] = (uint32_t)i;
  b.v[i] = make4<R>(R(vx), R(vy), R(vz), R(0));
  b.ft[i] = make4<R>(R(0), R(0), R(0), R(0));
  b.fc[i] = make4<R>(R(0), R(0), R(0), R(0));
  b.gid[i] = i;
}

// ---------------------------------------------------------- rebuild: permute
template <class R>
__global__ void __launch_bounds__(256) k_rb_permute(Geom g, Dyn *__restrict__ d, Bufs<R> s0,
                                                    Bufs<R> s1, Work w,
                                                    const uint32_t *__restrict__ skey,
                                                    const uint32_t *__restrict__ sval) {
  const int cur = d->cur;
  const Bufs<R> src = pick(cur, s0, s1);
  const Bufs<R> dst = pick(1 - cur, s0, s1);
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= g.n) return;
  const int o = min((int)sval[k], g.n - 1);
  const int c = min((int)skey[k], g.ncell - 1);
  int cx, cy, cz;
  cell_coords(g, c, cx, cy, cz);
  const double X0 = w.X[3 * (size_t)o], X1 = w.X[3 * (size_t)o + 1], X2 = w.X[3 * (size_t)o + 2];
  const double r0 = ((double)cx + 0.5) * g.lc[0];
  const double r1 = ((double)cy + 0.5) * g.lc[1];
  const double r2 = ((double)cz + 0.5) * g.lc[2];
  const double p0 = X0 - r0, p1 = X1 - r1, p2 = X2 - r2;
  if constexpr (sizeof(R) == 4) {
    const float h0 = (float)p0, h1 = (float)p1, h2 = (float)p2;
    dst.p[k] = make_float4(h0, h1, h2, (float)r2);
    dst.plo[k] = make_float4((float)(p0 - (double)h0), (float)(p1 - (double)h1),
                             (float)(p2 - (double)h2), 0.f);
    dst.pb[k] = make_float4(h0, h1, h2, __int_as_float(c));
  } else {
    dst.p[k] = make4<double>(p0, p1, p2, r2);
    dst.pb[k] = make_float4((float)p0, (float)p1, (float)p2, __int_as_float(c));
  }
  dst.v[k] = src.v[o];
  dst.ft[k] = src.ft[o];
  dst.fc[k] = src.fc[o];
  const int gid = src.gid[o];
  dst.gid[k] = gid;
  w.rank[gid] = k;
  w.Xs[3 * (size_t)k] = X0;
  w.Xs[3 * (size_t)k + 1] = X1;
  w.Xs[3 * (size_t)k + 2] = X2;
}

// ----------------------------------------------------------- rebuild: ranges
// cell_start[c] = first sorted slot of cell c (every entry written once).
__global__ void __launch_bounds__(256) k_rb_ranges(Geom g, const uint32_t *__restrict__ skey,
                                                   int *__restrict__ cell_start) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= g.n) return;
  const int c = min((int)skey[k], g.ncell - 1);
  const int prev = k == 0 ? -1 : min((int)skey[k - 1], g.ncell - 1);
  for (int cc = prev + 1; cc <= c; ++cc) cell_start[cc] = k;
  if (k == g.n - 1)
    for (int cc = c + 1; cc <= g.ncell; ++cc) cell_start[cc] = g.n;
}

// Restore path (checkpoint or rollback): sort keys, build-time FP64
// positions and ranks from the stored build record of the current set.
template <class R>
__global__ void k_relist_prep(Geom g, Dyn *__restrict__ d, Bufs<R> s0, Bufs<R> s1, Work w) {
  const Bufs<R> b = pick(d->cur, s0, s1);
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
}

// Slot-offset tables from d->s (this step) and d->f_build (last build).
__global__ void k_tables(Geom g, Dyn *__restrict__ d) {
  const double s = d->s, fb = d->f_build;
  if (threadIdx.x == 0) d->list_entries = 0;
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
// LE-aware Verlet list from the build positions.  Neighbour cells of cell
// (cx,cy,cz): for a y/z neighbour row inside the box, the x cells cx-1..cx+1;
// for a row across the top/bottom face, the x window shifted by the image
// offset: 3 or 4 cells covering every cell within rl of the shifted row
// (f_build/lx decides whether the window reaches a 4th cell).
template <class R>
__global__ void __launch_bounds__(kListThreads) k_rb_list(Geom g, Dyn *__restrict__ d, Bufs<R> s0,
                                                         Bufs<R> s1, Work w, int target_cur) {
  __shared__ float4 s_off[kNumSlots];
  for (int e = threadIdx.x; e < kNumSlots; e += blockDim.x)
    s_off[e] = make_float4((float)d->off_build[e][0], (float)d->off_build[e][1],
                           (float)d->off_build[e][2], 0.f);
  __syncthreads();
  const int tgt = target_cur ? d->cur : 1 - d->cur;
  const Bufs<R> b = pick(tgt, s0, s1);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  int cnt = 0;
  if (i < g.n) {
  const float4 qi = b.pb[i];
  int cx, cy, cz;
  cell_coords(g, __float_as_int(qi.w), cx, cy, cz);
  const float rl = (float)(g.rl * (1.0 + 1e-5));
  const float rl2 = rl * rl;
  const double phi = d->f_build / g.lc[0];
  const double rho = g.rl / g.lc[0] * (1.0 + 1e-5) + 1e-9;
  const int mb = d->m_build;
  uint32_t *out = w.nbr + (size_t)(i >> 5) * (size_t)g.maxnb * 32u + (i & 31);
  for (int dcz = -1; dcz <= 1; ++dcz) {
    int czj = cz - dcz, cross = 0;
    if (czj < 0) { czj += g.nc[2]; cross = 1; }
    else if (czj >= g.nc[2]) { czj -= g.nc[2]; cross = 1; }
    int kmin = -1, kmax = 1;
    if (cross) {
      if (dcz > 0) {
        kmin = phi > 1.0 - rho ? -2 : -1;
        kmax = phi < rho ? 1 : 0;
      } else {
        kmin = phi < rho ? -1 : 0;
        kmax = phi > 1.0 - rho ? 2 : 1;
      }
    }
    for (int dcy = -1; dcy <= 1; ++dcy) {
      int cyj = cy - dcy;
      cyj = ((cyj % g.nc[1]) + g.nc[1]) % g.nc[1];
      const int rowbase = g.nc[0] * (cyj + g.nc[1] * czj);
      for (int k = kmin; k <= kmax; ++k) {
        int cxj = cx - k + (cross ? dcz * mb : 0);
        cxj = ((cxj % g.nc[0]) + g.nc[0]) % g.nc[0];
        const int slot = slot_code(k, dcy, dcz, cross);
        const float4 o = s_off[slot];
        const int cj = rowbase + cxj;
        // clamped so that a corrupt range can never leave the particle arrays
        const int j0 = min(max(w.cell_start[cj], 0), g.n);
        const int j1 = min(max(w.cell_start[cj + 1], j0), g.n);
        const bool self_slot = (slot == slot_code(0, 0, 0, 0));
        for (int j = j0; j < j1; ++j) {
          if (self_slot && j == i) continue;
          const float4 qj = b.pb[j];
          const float dx = (qi.x - qj.x) + o.x;
          const float dy = (qi.y - qj.y) + o.y;
          const float dz = (qi.z - qj.z) + o.z;
          if (dx * dx + dy * dy + dz * dz < rl2) {
            if (cnt < g.maxnb) out[(size_t)cnt * 32u] = (uint32_t)j | ((uint32_t)slot << kIndexBits);
            ++cnt;
          }
        }
      }
    }
  }
  w.ncount[i] = cnt;
  atomicMax(&d->list_max, cnt);
  if (cnt > g.maxnb) atomicOr(&d->err, (int)kErrCapacity);
  }
  // total list entries (for the mean list length), one atomic per block
  __shared__ unsigned long long s_tot[kListThreads / 32];
  const unsigned long long c = warp_sum((unsigned long long)cnt);
  if ((threadIdx.x & 31) == 0) s_tot[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int k = 0; k < kListThreads / 32; ++k) t += s_tot[k];
    atomicAdd((unsigned long long *)&d->list_entries, t);
  }
}

// ------------------------------------------------------------ rebuild: bonds
// Slot of every bond: its LE minimum image at the build (FP64), expressed as
// build-cell offset + image, then matched to the 90-slot table.
template <class R>
__global__ void __launch_bounds__(256) k_rb_bonds(Geom g, Dyn *__restrict__ d, Bufs<R> s0,
                                                  Bufs<R> s1, Work w, int target_cur) {
  const int tgt = target_cur ? d->cur : 1 - d->cur;
  const Bufs<R> b = pick(tgt, s0, s1);
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
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
      dd[0] -= g.L[0] * rint(dd[0] / g.L[0]);
      dd[1] -= g.L[1] * rint(dd[1] / g.L[1]);
      int cj[3];
      cell_coords(g, __float_as_int(b.pb[j].w), cj[0], cj[1], cj[2]);
      // off = X_ref(i) - X_ref(j) - image shift, shift = (x_i - x_j) - d
      double off[3];
      for (int a = 0; a < 3; ++a) {
        const double shift = (xi[a] - xj[a]) - dd[a];
        off[a] = (double)(ck[a] - cj[a]) * g.lc[a] - shift;
      }
      const int dcz = (int)rint(off[2] / g.lc[2]);
      const int dcy = (int)rint(off[1] / g.lc[1]);
      const int cross = nz != 0.0 ? 1 : 0;
      const int kk = (int)rint((off[0] - (cross ? (double)dcz * fb : 0.0)) / g.lc[0]);
      if (dcz < -1 || dcz > 1 || dcy < -1 || dcy > 1 || kk < -2 || kk > 2 ||
          (cross && dcz == 0)) {
        atomicOr(&d->err, (int)kErrSlot);
      } else {
        entry = (uint32_t)j | ((uint32_t)slot_code(kk, dcy, dcz, cross) << kIndexBits);
      }
    }
    w.bond_e[(size_t)k * g.maxb + q] = entry;
  }
}

__global__ void k_rb_finish(Dyn *__restrict__ d) { d->cur = 1 - d->cur; }

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
      pair((int)(e & kIndexMask), (int)(e >> kIndexBits), false);
    }
    if constexpr (BONDS) {
      for (int q = 0; q < g.maxb; ++q) {
        const uint32_t e = w.bond_e[(size_t)i * g.maxb + q];
        if (e == kNoBond) break;
        pair((int)(e & kIndexMask), (int)(e >> kIndexBits), true);
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

}  // namespace

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

void launch_decide(const SysDev &s, cudaGraphConditionalHandle h, cudaStream_t st) {
  k_decide<<<1, 128, 0, st>>>(s.g, s.dyn, s.w, h);
}

void launch_fold(const SysDev &s, cudaStream_t st) { k_fold<<<1, 256, 0, st>>>(s.g, s.dyn, s.w); }

void launch_force(const SysDev &s, int mode, cudaStream_t st) {
  const int nb = blocks_for(s.g.n, kForceThreads);
  const size_t smem = sizeof(long long) * 2 * (size_t)s.g.nbins;
  const bool bonds = s.g.maxb > 0;
#define FN(R, A, B)                                                                  \
  do {                                                                               \
    if (bonds)                                                                       \
      k_force<R, true><<<nb, kForceThreads, smem, st>>>(s.g, s.dyn, A, B, s.w, mode);  \
    else                                                                             \
      k_force<R, false><<<nb, kForceThreads, smem, st>>>(s.g, s.dyn, A, B, s.w, mode); \
  } while (0)
  LE_DISPATCH(s, FN);
#undef FN
}

static void rebuild_tail(const SysDev &s, cudaStream_t st) {
  const int n = s.g.n;
  radix_sort_pairs(const_cast<uint32_t **>(s.w.key), const_cast<uint32_t **>(s.w.val), s.w.hist, n,
                   s.sort_passes, s.sort_blocks, st);
  const uint32_t *skey = s.w.key[s.sort_passes & 1];
  const uint32_t *sval = s.w.val[s.sort_passes & 1];
  const int nb = blocks_for(n, 256);
#define FN(R, A, B) k_rb_permute<R><<<nb, 256, 0, st>>>(s.g, s.dyn, A, B, s.w, skey, sval)
  LE_DISPATCH(s, FN);
#undef FN
  k_rb_ranges<<<nb, 256, 0, st>>>(s.g, skey, s.w.cell_start);
  const int nl = blocks_for(n, kListThreads);
#define FN(R, A, B) k_rb_list<R><<<nl, kListThreads, 0, st>>>(s.g, s.dyn, A, B, s.w, 0)
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
  const int nl = blocks_for(n, kListThreads);
#define FN(R, A, B) k_rb_list<R><<<nl, kListThreads, 0, st>>>(s.g, s.dyn, A, B, s.w, 1)
  LE_DISPATCH(s, FN);
#undef FN
  if (s.g.maxb > 0) {
#define FN(R, A, B) k_rb_bonds<R><<<nb, 256, 0, st>>>(s.g, s.dyn, A, B, s.w, 1)
    LE_DISPATCH(s, FN);
#undef FN
  }
}

void launch_import(const SysDev &s, cudaStream_t st) {
  const int nb = blocks_for(s.g.n, 256);
#define FN(R, A, B) k_import<R><<<nb, 256, 0, st>>>(s.g, s.dyn, A, B, s.w, s.stage)
  LE_DISPATCH(s, FN);
#undef FN
}

void launch_export(const SysDev &s, cudaStream_t st) {
  const int nb = blocks_for(s.g.n, 256);
#define FN(R, A, B) k_export<R><<<nb, 256, 0, st>>>(s.g, s.dyn, A, B, s.stage)
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

}  // namespace le
