// le_forces_noalloc: conservative forces of a set of positions under the
// sheared images, computed without allocating any device memory.
//
// Who needs it: some callers cannot call cudaMalloc at the point where they
// want forces -- a control loop that must not allocate (or risk an
// out-of-memory failure from fragmentation) once it is running, or a host
// program whose device memory is entirely owned by another pool or framework.
// For them this entry point runs the same kernels as a handle's initial force
// evaluation (wrap and bin, radix sort, LE-aware Verlet list, pair forces),
// with every buffer carved out of one file-scope static device array.
//
// The static array lives on every device that loads this library until the
// process exits.  Its device address is looked up, with the device current,
// by the first call made in each CUDA context (a device's primary context,
// or a new one after the old one was reset or destroyed: the module, and with
// it the array, may then sit at another address); make the first call on a
// device before any stream capture begins.  Every call shares the array and
// leaves its contents behind; what must start at zero is cleared by each
// call.  A call returns only after its device work has finished, and calls
// from different host threads are serialised by a lock, so within one
// process calls never overlap on the GPU; work from elsewhere that overlapped
// a call on the same array would race with it.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/le.h"
#include "le_launch.h"

using namespace le;

namespace {

constexpr int64_t kNoAllocMaxParticles = 16384;
constexpr size_t kNoAllocBytes = size_t(32) << 20;  // 32 MiB
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_lock;
// the address of the array in the context it was looked up in
struct ScratchAddr {
  unsigned long long ctx_id = 0;
  unsigned char *addr = nullptr;
};
ScratchAddr g_scratch_addr[kMaxDevices];

using CtxGetCurrentFn = CUresult (*)(CUcontext *);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long *);

// Identity of the current CUDA context (unique for the life of the process),
// through the driver entry points, so the library needs no link to libcuda.
cudaError_t current_context_id(unsigned long long *id) {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  if (!get_current || !get_id) {
    void *a = nullptr, *b = nullptr;
    cudaDriverEntryPointQueryResult qa, qb;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000,
                                                     cudaEnableDefault, &qa);
    if (e == cudaSuccess)
      e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb);
    if (e != cudaSuccess) return e;
    if (qa != cudaDriverEntryPointSuccess || qb != cudaDriverEntryPointSuccess || !a || !b)
      return cudaErrorNotSupported;
    get_current = reinterpret_cast<CtxGetCurrentFn>(a);
    get_id = reinterpret_cast<CtxGetIdFn>(b);
  }
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return cudaErrorDeviceUninitialized;
  if (get_id(ctx, id) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
  return cudaSuccess;
}

// Device address of the static array in the current context, looked up again
// whenever the context differs from the one of the cached address.
cudaError_t scratch_address(unsigned char **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  unsigned long long id = 0;
  e = current_context_id(&id);
  if (e == cudaErrorDeviceUninitialized) {
    // no context is current yet: the runtime creates the device's primary
    // context on this first symbol lookup
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e == cudaSuccess) e = current_context_id(&id);
  }
  if (e != cudaSuccess) return e;
  ScratchAddr &c = g_scratch_addr[dev];
  if (!c.addr || c.ctx_id != id) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    c.addr = static_cast<unsigned char *>(p);
    c.ctx_id = id;
  }
  *out = c.addr;
  return cudaSuccess;
}

// Bump allocator over the static array (256-byte aligned pieces).
struct Carver {
  unsigned char *base;
  size_t used = 0;
  template <class T> T *take(size_t count) {
    used = (used + 255) & ~size_t(255);
    T *p = reinterpret_cast<T *>(base + used);
    used += std::max<size_t>(count * sizeof(T), 256);
    return p;
  }
};

}  // namespace

namespace {

// Geometry and per-precision constants of a force-only evaluation (no
// thermostat, no bonds, no samples).
le_status setup_geom(Geom &g, const double box[3], double shear_rate, double rc, double skin,
                     const le_params *p, int64_t n) {
  std::memset(&g, 0, sizeof g);
  const double rl = rc + skin;
  for (int a = 0; a < 3; ++a) {
    if (!(box[a] > 0.0) || !std::isfinite(box[a])) return LE_ERR_INVALID_ARG;
    if (!(rl < 0.5 * box[a])) return LE_ERR_BOX_TOO_SMALL;
    g.L[a] = box[a];
  }
  g.shear_rate = shear_rate;
  g.dt = p->dt;
  g.mass = p->mass;
  g.kT = p->kT;
  g.xi = 0.0;
  g.rc = rc;
  g.skin = skin;
  g.rl = rl;
  g.eps = p->eps;
  g.sigma = p->sigma;
  g.fene_k = p->fene_k;
  g.fene_R0 = p->fene_R0;
  g.thermostat = LE_THERMO_NONE;
  g.lj_shift = p->lj_shift;
  g.nbins = 1;
  g.sample_every = 0;
  g.seed = p->seed;
  g.system = p->system_id;
  const double rlb = rl * (1.0 + 1e-5);
  g.rl2_build = (float)(rlb * rlb);
  KConst<double> &c = g.cd;
  c.half_dt_m = 0.5 * p->dt / p->mass;
  c.dt = p->dt;
  c.rc2 = rc * rc;
  c.sig2 = p->sigma * p->sigma;
  c.eps24 = 24.0 * p->eps;
  c.amp = 0.0;
  c.xim = 0.0;
  c.shear = shear_rate;
  c.half_Lz = 0.5 * box[2];
  c.Lz = box[2];
  c.shear_Lz = shear_rate * box[2];
  c.R02 = p->fene_R0 * p->fene_R0;
  c.fene_k = p->fene_k;
  c.ang_k = 0.0;  // no bonds here
  c.dpd_xi = 0.0;  // no DPD here
  c.dpd_amp = 0.0;
  c.inv_rc = 0.0;
  c.mass = p->mass;
  c.bins_per_Lz = 1.0 / box[2];
  KConst<float> &f = g.cf;
  f.half_dt_m = (float)c.half_dt_m;
  f.dt = (float)c.dt;
  f.rc2 = (float)c.rc2;
  f.sig2 = (float)c.sig2;
  f.eps24 = (float)c.eps24;
  f.amp = 0.f;
  f.xim = 0.f;
  f.shear = (float)c.shear;
  f.half_Lz = (float)c.half_Lz;
  f.Lz = (float)c.Lz;
  f.shear_Lz = (float)c.shear_Lz;
  f.R02 = (float)c.R02;
  f.fene_k = (float)c.fene_k;
  f.ang_k = 0.f;
  f.dpd_xi = 0.f;
  f.dpd_amp = 0.f;
  f.inv_rc = 0.f;
  f.mass = (float)c.mass;
  f.bins_per_Lz = (float)c.bins_per_Lz;
  // cell grid of edge >= rc + skin
  g.ncell = 1;
  for (int a = 0; a < 3; ++a) {
    g.nc[a] = std::max(1, (int)std::floor(g.L[a] / rl));
    g.lc[a] = g.L[a] / g.nc[a];
    if ((double)g.ncell * g.nc[a] > 1e8) return LE_ERR_INVALID_ARG;
    g.ncell *= g.nc[a];
    g.inv_lc[a] = (float)(1.0 / g.lc[a]);
    g.inv_lcd[a] = 1.0 / g.lc[a];
    g.inv_L[a] = 1.0 / g.L[a];
    g.half_lc_f[a] = (float)(0.5 * g.lc[a] * (1.0 + 1e-6) + 1e-6);
    g.lc_hi[a] = (float)g.lc[a];
    g.lc_lo[a] = (float)(g.lc[a] - (double)g.lc_hi[a]);
  }
  int bits = 1;
  while ((1ll << bits) < (long long)g.ncell) ++bits;
  g.sort_bits = bits;
  set_fixed_point(g);
  g.n = (int)n;
  g.inv_volume = 1.0 / (g.L[0] * g.L[1] * g.L[2]);
  g.inv_dof = 1.0 / (n > 1 ? 3.0 * (double)n - 3.0 : 1.0);
  g.npad = (int)((n + 31) / 32 * 32);
  g.maxb = 0;
  const double V = g.L[0] * g.L[1] * g.L[2];
  const double mean_nb = 4.18879020478639 * rl * rl * rl * (double)n / V;
  g.maxnb = (int)std::ceil(mean_nb * 1.6) + 32;
  return LE_OK;
}

template <class R> void carve_set(Carver &cv, Bufs<R> &b, int64_t n, bool lo) {
  b.p = cv.take<typename Vec<R>::T>(n);
  b.plo = lo ? cv.take<float4>(n) : nullptr;
  b.v = cv.take<typename Vec<R>::T>(n);
  b.ft = cv.take<typename Vec<R>::T>(n);
  b.fc = cv.take<typename Vec<R>::T>(n);
  b.pb = cv.take<float4>(n);
  b.gid = cv.take<int>(n);
  b.q = lo ? cv.take<int4>(n) : nullptr;
  b.q2 = nullptr;  // no fused drift here
}

// Lays every buffer of a one-shot force evaluation out in the static array.
size_t carve(SysDev &s, unsigned char *base, int64_t n) {
  Carver cv{base};
  const Geom &g = s.g;
  s.dyn = cv.take<Dyn>(1);
  if (s.prec == 1) {
    carve_set(cv, s.f32[0], n, true);
    carve_set(cv, s.f32[1], n, true);
  } else {
    carve_set(cv, s.f64[0], n, false);
    carve_set(cv, s.f64[1], n, false);
  }
  Work &w = s.w;
  w.nbr = cv.take<uint32_t>((size_t)g.npad * (size_t)g.maxnb);
  w.ncount = cv.take<int>(n);
  w.cell_start = cv.take<int>((size_t)g.ncell + 1);
  w.bond_e = cv.take<uint32_t>(n);
  w.bond_gid = cv.take<int>(n);
  w.rank = cv.take<int>(n);
  w.tmp_p = s.prec == 1 ? (void *)cv.take<float4>(n) : (void *)cv.take<D4>(n);
  w.tmp_lo = s.prec == 1 ? cv.take<float4>(n) : nullptr;
  w.Xs = cv.take<double>(3 * (size_t)n);
  for (int k = 0; k < 2; ++k) {
    w.key[k] = cv.take<uint32_t>(n);
    w.val[k] = cv.take<uint32_t>(n);
  }
  s.sort_blocks = sort_blocks_for(n);
  s.sort_passes = sort_passes_for(g.sort_bits);
  w.hist = cv.take<uint32_t>((size_t)kSortBuckets * s.sort_blocks);
  s.sort_part = cv.take<uint32_t>(sort_scan_parts(s.sort_blocks));
  w.acc_prof = cv.take<long long>(3);
  w.sum_prof = cv.take<double>(2);
  w.cnt_prof = cv.take<long long>(1);
  w.vnew = nullptr;
  s.stage = cv.take<double>(6 * (size_t)n);
  s.partials = cv.take<double>(16);
  return cv.used;
}

}  // namespace

extern "C" LE_API le_status le_forces_noalloc(const double box[3], double shear_rate, double rc,
                                              double skin, const le_params *p, int64_t step,
                                              int64_t n, const double *pos, double *forces,
                                              void *cuda_stream) {
  if (!box || !p || !pos || !forces) return LE_ERR_INVALID_ARG;
  if (n < 1 || n > kNoAllocMaxParticles || step < 0) return LE_ERR_INVALID_ARG;
  if (!(rc > 0.0) || !(skin >= 0.0) || !(p->dt > 0.0) || !(p->mass > 0.0) ||
      !std::isfinite(shear_rate))
    return LE_ERR_INVALID_ARG;
  if (p->precision != LE_FP64 && p->precision != LE_FP32) return LE_ERR_INVALID_ARG;
  for (int64_t q = 0; q < 3 * n; ++q)
    if (!std::isfinite(pos[q])) return LE_ERR_INVALID_ARG;

  std::lock_guard<std::mutex> guard(g_lock);
  unsigned char *base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return LE_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  SysDev s;
  s.prec = p->precision;
  le_status rs = setup_geom(s.g, box, shear_rate, rc, skin, p, n);
  if (rs != LE_OK) return rs;

  // the image offset of Eq. 4 at this step, as a handle computes it
  const double t = (double)step * p->dt;
  double dX = std::fmod(shear_rate * box[2] * t, box[0]);
  if (dX < 0.0) dX += box[0];
  const double lx = s.g.lc[0];
  int m = (int)std::floor(dX / lx);
  double f = dX - (double)m * lx;
  if (f >= lx) { f -= lx; m += 1; }
  if (f < 0.0) { f += lx; m -= 1; }

  for (int attempt = 0; attempt < 3; ++attempt) {
    if (carve(s, base, n) > kNoAllocBytes) return LE_ERR_INVALID_ARG;  // too large for the array
    Dyn d;
    std::memset(&d, 0, sizeof d);
    d.step = step;
    d.build_step = step;
    d.dX = dX;
    d.dX_build = dX;
    d.m_build = m;
    d.f_build = f;
    d.s = f;
    d.s_f = (float)f;
    d.s_q = (int)std::llrint(std::ldexp(f, s.g.qshift));
    d.cur = 0;
    cudaError_t e = cudaMemcpyAsync(s.dyn, &d, sizeof d, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(s.w.acc_prof, 0, 3 * sizeof(long long), st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(s.stage, pos, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(s.stage + 3 * n, 0, sizeof(double) * 3 * n, st);
    if (e != cudaSuccess) return LE_ERR_CUDA;
    launch_tables(s, st);
    launch_import(s, st);
    launch_rebuild(s, true, st);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&d, s.dyn, sizeof d, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return LE_ERR_CUDA;
    if (d.list_max > s.g.maxnb) {  // denser than estimated: a longer list, if it fits
      s.g.maxnb = (int)std::ceil(d.list_max * 1.25) + 16;
      continue;
    }
    launch_force(s, 1, st);
    launch_export_forces(s, st);
    e = cudaGetLastError();
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(forces, s.stage, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&d, s.dyn, sizeof d, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return LE_ERR_CUDA;
    if (d.err & kErrNonfinite) return LE_ERR_NONFINITE;
    if (d.err & kErrTimeout) return LE_ERR_TIMEOUT;
    if (d.err) return LE_ERR_CAPACITY;
    return LE_OK;
  }
  return LE_ERR_CAPACITY;
}
