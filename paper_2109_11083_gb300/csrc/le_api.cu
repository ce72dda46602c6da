// C ABI of the Lees-Edwards shear-flow MD library (declared in include/le.h).
//
// A handle owns one system's device memory, two private capture streams and
// the instantiated step graphs.  One step is captured as
//   k_drift -> k_decide -> IF(rebuild){bin, radix sort, permute, ranges,
//   Verlet list, bonds, finish} -> k_force,
// where k_decide sets the conditional handle on the device, so the rebuild
// decision of the skin/image-shift trigger never needs a host round trip.
// le_step launches a 16-step graph repeatedly and a 1-step graph for the rest.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <map>
#include <tuple>
#include <vector>

#include "../../include/le.h"
#include "le_launch.h"

using namespace le;

namespace {
constexpr int kChunk = 16;
constexpr uint64_t kStateMagic = 0x4c45534d53544154ull;  // "LESMSTAT"
constexpr int kStateVersion = 5;
constexpr int kUpChunks = 4;
}  // namespace

struct le_sim {
  double box[3] = {0, 0, 0};
  double shear_rate = 0, rc = 0, skin = 0;
  le_params prm{};
  cudaStream_t stream = nullptr;     // where the work runs
  bool own_stream = false;
  cudaStream_t cap_main = nullptr, cap_side = nullptr;  // private capture streams
  // le_set_particles: host -> device copies in kUpChunks pieces on up_stream,
  // each piece imported on the main stream as soon as it has landed
  cudaStream_t up_stream = nullptr;
  cudaEvent_t up_ev[kUpChunks] = {};
  cudaEvent_t up_go = nullptr;
  SysDev s;
  bool has_particles = false;
  int64_t n = 0;
  std::vector<int32_t> bonds;        // nb x 2
  std::vector<void *> allocs;
  double *h_stage = nullptr;         // pinned host staging, 6n doubles
  long long *h_scalar = nullptr;     // pinned host scratch
  Dyn *h_dyn = nullptr;              // pinned mirror of the device record
  cudaGraphExec_t exec_chunk = nullptr, exec_one = nullptr;
  // graphs of r = 2 .. kChunk-1 steps, captured when a call first ends with
  // r steps after its whole chunks (the drift fused into the pair kernel
  // across all r steps, as in a chunk)
  cudaGraphExec_t exec_rem[kChunk] = {};
  bool eager = false;                // launch kernels directly (no graphs)
  bool dry_run = false;              // allocate() only counts bytes
  size_t device_bytes = 0;           // device memory of the particle buffers
  // layout of the current device allocation (reused when a later
  // le_set_particles needs the same one): n, list slots, bond slots, cells
  long long alloc_key[4] = {-1, -1, -1, -1};
  // rollback snapshot of the current buffer set and the dynamic record
  std::vector<void *> snap;
  std::string err;
};

namespace {

le_status fail(le_sim *s, le_status st, const std::string &msg) {
  if (s) s->err = msg;
  return st;
}

#define CK(call)                                                                        \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) {                                                            \
      return fail(s, e_ == cudaErrorMemoryAllocation ? LE_ERR_OOM : LE_ERR_CUDA,        \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                  \
    }                                                                                   \
  } while (0)

#define CKS(expr)                 \
  do {                            \
    le_status st_ = (expr);       \
    if (st_ != LE_OK) return st_; \
  } while (0)

template <class T> le_status dalloc(le_sim *s, T **p, size_t count) {
  void *q = nullptr;
  size_t bytes = std::max<size_t>(count * sizeof(T), 256);
  s->device_bytes += bytes;
  if (s->dry_run) {  // counting only (admission by memory budget)
    *p = nullptr;
    return LE_OK;
  }
  CK(cudaMalloc(&q, bytes));
  s->allocs.push_back(q);
  *p = static_cast<T *>(q);
  return LE_OK;
}

// Every captured step graph of s (they hold the buffer addresses and the list
// capacity of the capture).
void destroy_graphs(le_sim *s) {
  if (s->exec_chunk) cudaGraphExecDestroy(s->exec_chunk);
  if (s->exec_one) cudaGraphExecDestroy(s->exec_one);
  s->exec_chunk = s->exec_one = nullptr;
  for (cudaGraphExec_t &g : s->exec_rem) {
    if (g) cudaGraphExecDestroy(g);
    g = nullptr;
  }
}

void free_device(le_sim *s) {
  for (long long &k : s->alloc_key) k = -1;
  destroy_graphs(s);
  for (void *p : s->allocs) cudaFree(p);
  s->allocs.clear();
  for (void *p : s->snap) cudaFree(p);
  s->snap.clear();
  if (s->h_stage) cudaFreeHost(s->h_stage);
  s->h_stage = nullptr;
  s->has_particles = false;
}

size_t vec_bytes(int prec) { return prec == 1 ? sizeof(float4) : sizeof(D4); }

// True for page-locked (or device-visible) host memory, which the copy
// engines read and write directly; pageable memory goes through the pinned
// staging buffer.
bool is_pinned(const void *p) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeManaged;
}

// Host -> device copy of n doubles from the caller's array into dst.
le_status upload(le_sim *s, double *dst, const double *src, size_t n, double *stage_part,
                 cudaStream_t st) {
  if (is_pinned(src)) {
    CK(cudaMemcpyAsync(dst, src, sizeof(double) * n, cudaMemcpyHostToDevice, st));
  } else {
    std::memcpy(stage_part, src, sizeof(double) * n);
    CK(cudaMemcpyAsync(dst, stage_part, sizeof(double) * n, cudaMemcpyHostToDevice, st));
  }
  return LE_OK;
}

// First particle of upload piece c of n (pieces of whole particles).
int64_t up_piece(int64_t n, int c) { return n * c / kUpChunks; }

// The caller's positions and velocities into the staging buffer, in
// kUpChunks pieces on up_stream (after the main stream's earlier work), each
// piece's end recorded in up_ev[c] for the import (initialise) to wait on.
le_status upload_particles(le_sim *s, const double *pos, const double *vel) {
  const int64_t n = s->n;
  CK(cudaEventRecord(s->up_go, s->stream));
  CK(cudaStreamWaitEvent(s->up_stream, s->up_go, 0));
  for (int c = 0; c < kUpChunks; ++c) {
    const int64_t a = up_piece(n, c), b = up_piece(n, c + 1);
    if (b > a) {
      CKS(upload(s, s->s.stage + 3 * a, pos + 3 * a, 3 * (size_t)(b - a), s->h_stage + 3 * a,
                 s->up_stream));
      CKS(upload(s, s->s.stage + 3 * n + 3 * a, vel + 3 * a, 3 * (size_t)(b - a),
                 s->h_stage + 3 * n + 3 * a, s->up_stream));
    }
    CK(cudaEventRecord(s->up_ev[c], s->up_stream));
  }
  return LE_OK;
}

// Device -> host copy of n doubles into the caller's array (after a sync
// for pageable destinations, through the pinned staging buffer).
le_status download(le_sim *s, double *dst, const double *src, size_t n, double *stage_part) {
  if (is_pinned(dst)) {
    CK(cudaMemcpyAsync(dst, src, sizeof(double) * n, cudaMemcpyDeviceToHost, s->stream));
  } else {
    CK(cudaMemcpyAsync(stage_part, src, sizeof(double) * n, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    std::memcpy(dst, stage_part, sizeof(double) * n);
  }
  return LE_OK;
}

// Pointers of one buffer set as raw bytes, in a fixed order (for snapshots
// and checkpoints): p, plo, v, ft, fc, pb, gid.
void set_fields(le_sim *s, int which, void *ptr[7], size_t bytes[7]) {
  const size_t n = (size_t)s->n;
  const size_t vb = vec_bytes(s->s.prec);
  if (s->s.prec == 1) {
    const Bufs<float> &b = s->s.f32[which];
    ptr[0] = b.p; ptr[1] = b.plo; ptr[2] = b.v; ptr[3] = b.ft; ptr[4] = b.fc; ptr[5] = b.pb; ptr[6] = b.gid;
  } else {
    const Bufs<double> &b = s->s.f64[which];
    ptr[0] = b.p; ptr[1] = b.plo; ptr[2] = b.v; ptr[3] = b.ft; ptr[4] = b.fc; ptr[5] = b.pb; ptr[6] = b.gid;
  }
  bytes[0] = n * vb;
  bytes[1] = s->s.prec == 1 ? n * sizeof(float4) : 0;
  bytes[2] = bytes[3] = bytes[4] = n * vb;
  bytes[5] = n * sizeof(float4);
  bytes[6] = n * sizeof(int);
}

le_status sync(le_sim *s) {
  CK(cudaStreamSynchronize(s->stream));
  return LE_OK;
}

le_status read_dyn(le_sim *s) {
  CK(cudaMemcpyAsync(s->h_dyn, s->s.dyn, sizeof(Dyn), cudaMemcpyDeviceToHost, s->stream));
  return sync(s);
}

le_status status_from_err(le_sim *s, int err) {
  if (err & kErrInput) return fail(s, LE_ERR_INVALID_ARG, "non-finite input");
  if (err & kErrBond) return fail(s, LE_ERR_BOND_BROKEN, "a FENE bond reached R0 (Eq. 11)");
  if (err & kErrNonfinite) return fail(s, LE_ERR_NONFINITE, "a force or velocity became non-finite");
  if (err & kErrCapacity) return fail(s, LE_ERR_CAPACITY, "neighbour list capacity exceeded");
  if (err & kErrSlot) return fail(s, LE_ERR_BOND_BROKEN, "a bond spans more than one cell");
  if (err & kErrTimeout) return fail(s, LE_ERR_TIMEOUT, "a bounded wait on a bulk copy gave up");
  if (err & kErrRange)
    return fail(s, LE_ERR_RANGE, "a sampled |vx| above 1000 or m vy^2 above 2000 (profile range)");
  return LE_OK;
}

// ------------------------------------------------------------- allocation
le_status allocate(le_sim *s, int64_t n, int maxnb) {
  const long long key[4] = {n, maxnb, s->s.g.maxb, s->s.g.ncell};
  if (!s->dry_run && !s->allocs.empty() && std::equal(key, key + 4, s->alloc_key)) {
    // the same layout: keep every buffer (and the step graphs, whose kernel
    // arguments are these buffers and the unchanged geometry)
    s->has_particles = false;
    return LE_OK;
  }
  free_device(s);
  std::copy(key, key + 4, s->alloc_key);
  s->device_bytes = 0;
  Geom &g = s->s.g;
  const int prec = s->s.prec;
  g.n = (int)n;
  g.inv_volume = 1.0 / (g.L[0] * g.L[1] * g.L[2]);
  g.inv_dof = 1.0 / (n > 1 ? 3.0 * (double)n - 3.0 : 1.0);
  g.npad = (int)((n + 31) / 32 * 32);
  g.maxnb = maxnb;
  const size_t vb = vec_bytes(prec);
  for (int k = 0; k < 2; ++k) {
    void *p, *plo, *v, *ft, *fc;
    float4 *pb;
    int *gid;
    int4 *q = nullptr, *q2 = nullptr;
    CKS(dalloc(s, (char **)&p, n * vb));
    plo = nullptr;
    if (prec == 1) CKS(dalloc(s, (char **)&plo, n * sizeof(float4)));
    if (prec == 1) CKS(dalloc(s, &q, n));
    if (prec == 1) CKS(dalloc(s, &q2, n));
    CKS(dalloc(s, (char **)&v, n * vb));
    CKS(dalloc(s, (char **)&ft, n * vb));
    CKS(dalloc(s, (char **)&fc, n * vb));
    CKS(dalloc(s, &pb, n));
    CKS(dalloc(s, &gid, n));
    if (prec == 1) {
      s->s.f32[k] = Bufs<float>{(float4 *)p, (float4 *)plo, (float4 *)v, (float4 *)ft, (float4 *)fc, pb, gid, q, q2};
    } else {
      s->s.f64[k] = Bufs<double>{(D4 *)p, (float4 *)plo, (D4 *)v, (D4 *)ft, (D4 *)fc, pb, gid, nullptr, nullptr};
    }
  }
  Work &w = s->s.w;
  CKS(dalloc(s, &w.nbr, (size_t)g.npad * (size_t)maxnb));
  CKS(dalloc(s, &w.ncount, n));
  CKS(dalloc(s, &w.cell_start, (size_t)g.ncell + 1));
  const int mb = std::max(g.maxb, 1);
  CKS(dalloc(s, &w.bond_e, (size_t)n * mb));
  CKS(dalloc(s, &w.bond_gid, (size_t)n * mb));
  CKS(dalloc(s, &w.rank, n));
  CKS(dalloc(s, (char **)&w.tmp_p, (size_t)n * vb));
  if (prec == 1) CKS(dalloc(s, &w.tmp_lo, n));
  CKS(dalloc(s, &w.Xs, 3 * (size_t)n));
  w.vnew = nullptr;
  if (g.thermostat == LE_THERMO_DPD) CKS(dalloc(s, (char **)&w.vnew, (size_t)n * vb));
  for (int k = 0; k < 2; ++k) {
    CKS(dalloc(s, &w.key[k], n));
    CKS(dalloc(s, &w.val[k], n));
  }
  s->s.sort_blocks = sort_blocks_for(n);
  CKS(dalloc(s, &w.hist, (size_t)kSortBuckets * s->s.sort_blocks));
  CKS(dalloc(s, &s->s.sort_part, sort_scan_parts(s->s.sort_blocks)));
  CKS(dalloc(s, &w.acc_prof, 3 * (size_t)g.nbins));
  CKS(dalloc(s, &w.sum_prof, 2 * (size_t)g.nbins));
  CKS(dalloc(s, &w.cnt_prof, (size_t)g.nbins));
  CKS(dalloc(s, &s->s.dyn, 1));
  CKS(dalloc(s, &s->s.stage, 6 * (size_t)n));
  CKS(dalloc(s, &s->s.partials, (size_t)observe_blocks(s->s) * 16));
  if (!s->dry_run) CK(cudaMallocHost(&s->h_stage, sizeof(double) * 6 * (size_t)n));
  s->n = n;
  return LE_OK;
}

// Cell grid: edge >= rc + skin (and >= R0 when bonds exist, so that a bond
// never spans more than one cell in a direction).
void choose_cells(le_sim *s) {
  Geom &g = s->s.g;
  double edge = g.rl;
  if (!s->bonds.empty()) edge = std::max(edge, g.fene_R0);
  g.ncell = 1;
  for (int a = 0; a < 3; ++a) {
    g.nc[a] = std::max(1, (int)std::floor(g.L[a] / edge));
    g.lc[a] = g.L[a] / g.nc[a];
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
  s->s.sort_passes = sort_passes_for(g.sort_bits);
  set_fixed_point(g);
}

// Per-system parameters and per-precision kernel constants.
void fill_geom(le_sim *s, const double box[3], double shear_rate, double rc, double skin,
               const le_params *p) {
  const double rl = rc + skin;
  Geom &g = s->s.g;
  std::memset(&g, 0, sizeof g);
  for (int a = 0; a < 3; ++a) g.L[a] = box[a];
  g.shear_rate = shear_rate;
  g.dt = p->dt;
  g.mass = p->mass;
  g.kT = p->kT;
  g.xi = p->xi;
  g.rc = rc;
  g.skin = skin;
  g.rl = rl;
  g.eps = p->eps;
  g.sigma = p->sigma;
  g.fene_k = p->fene_k;
  g.fene_R0 = p->fene_R0;
  g.thermostat = p->thermostat;
  g.lj_shift = p->lj_shift;
  g.nbins = p->profile_bins;
  g.sample_every = p->sample_every;
  g.seed = p->seed;
  g.system = p->system_id;
  {
    const double rlb = rl * (1.0 + 1e-5);
    g.rl2_build = (float)(rlb * rlb);
    KConst<double> &c = g.cd;
    c.half_dt_m = 0.5 * p->dt / p->mass;
    c.dt = p->dt;
    c.rc2 = rc * rc;
    c.sig2 = p->sigma * p->sigma;
    c.eps24 = 24.0 * p->eps;
    c.amp = std::sqrt(24.0 * p->xi * p->kT * p->mass / p->dt);
    c.xim = p->xi * p->mass;
    c.shear = shear_rate;
    c.half_Lz = 0.5 * box[2];
    c.Lz = box[2];
    c.shear_Lz = shear_rate * box[2];
    c.R02 = p->fene_R0 * p->fene_R0;
    c.fene_k = p->fene_k;
    c.ang_k = p->angle_k;
    g.force_cap = p->force_cap;
    c.dpd_xi = p->xi;
    c.dpd_amp = std::sqrt(24.0 * p->kT * p->xi / p->dt);
    c.inv_rc = 1.0 / rc;
    c.mass = p->mass;
    c.bins_per_Lz = p->profile_bins / box[2];
    KConst<float> &f = g.cf;
    f.half_dt_m = (float)c.half_dt_m;
    f.dt = (float)c.dt;
    f.rc2 = (float)c.rc2;
    f.sig2 = (float)c.sig2;
    f.eps24 = (float)c.eps24;
    f.amp = (float)c.amp;
    f.xim = (float)c.xim;
    f.shear = (float)c.shear;
    f.half_Lz = (float)c.half_Lz;
    f.Lz = (float)c.Lz;
    f.shear_Lz = (float)c.shear_Lz;
    f.R02 = (float)c.R02;
    f.fene_k = (float)c.fene_k;
    f.ang_k = (float)c.ang_k;
    f.dpd_xi = (float)c.dpd_xi;
    f.dpd_amp = (float)c.dpd_amp;
    f.inv_rc = (float)c.inv_rc;
    f.mass = (float)c.mass;
    f.bins_per_Lz = (float)c.bins_per_Lz;
  }
  s->s.prec = p->precision;
}

// ------------------------------------------------------------- graph capture
// Records `steps` steps of system s on stream st, which must already be
// capturing into `graph`: drift, decide (sets the IF condition), IF(rebuild),
// force.  Where the system allows it, the force launch of every step but the
// last also runs the next step's drift (mode 2), so only the first step has a
// drift launch of its own.
cudaError_t record_steps(le_sim *s, cudaStream_t st, cudaGraph_t graph, int steps,
                         std::vector<cudaEvent_t> *ev) {
  cudaError_t ce = cudaSuccess;
  const bool fuse = can_fuse_drift(s->s);
  for (int k = 0; k < steps && ce == cudaSuccess; ++k) {
    cudaGraphConditionalHandle handle;
    ce = cudaGraphConditionalHandleCreate(&handle, graph, 0, 0);
    if (ce != cudaSuccess) break;
    if (ev) cudaEventRecordWithFlags((*ev)[4 * k + 0], st, cudaEventRecordExternal);
    if (k == 0 || !fuse) launch_drift(s->s, st);
    if (ev) cudaEventRecordWithFlags((*ev)[4 * k + 1], st, cudaEventRecordExternal);
    launch_decide(s->s, handle, 1, st);
    const cudaGraphNode_t *deps = nullptr;
    size_t ndeps = 0;
    cudaStreamCaptureStatus cs;
    ce = cudaStreamGetCaptureInfo(st, &cs, nullptr, nullptr, &deps, nullptr, &ndeps);
    if (ce != cudaSuccess) break;
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = handle;
    cp.conditional.type = cudaGraphCondTypeIf;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    ce = cudaGraphAddNode(&node, graph, deps, nullptr, ndeps, &cp);
    if (ce != cudaSuccess) break;
    ce = cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1,
                                             cudaStreamSetCaptureDependencies);
    if (ce != cudaSuccess) break;
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    ce = cudaStreamBeginCaptureToGraph(s->cap_side, body, nullptr, nullptr, 0,
                                       cudaStreamCaptureModeThreadLocal);
    if (ce != cudaSuccess) break;
    launch_rebuild(s->s, false, s->cap_side);
    ce = cudaStreamEndCapture(s->cap_side, &body);
    if (ce != cudaSuccess) break;
    if (ev) cudaEventRecordWithFlags((*ev)[4 * k + 2], st, cudaEventRecordExternal);
    launch_force(s->s, fuse && k + 1 < steps ? 2 : 0, st);
    if (ev) cudaEventRecordWithFlags((*ev)[4 * k + 3], st, cudaEventRecordExternal);
  }
  return ce;
}

le_status capture(le_sim *s, int steps, std::vector<cudaEvent_t> *ev, cudaGraphExec_t *out) {
  cudaGraph_t graph = nullptr;
  CK(cudaGraphCreate(&graph, 0));
  CK(cudaStreamBeginCaptureToGraph(s->cap_main, graph, nullptr, nullptr, 0,
                                   cudaStreamCaptureModeThreadLocal));
  cudaError_t ce = record_steps(s, s->cap_main, graph, steps, ev);
  cudaGraph_t captured = nullptr;
  cudaError_t ee = cudaStreamEndCapture(s->cap_main, &captured);
  if (ce == cudaSuccess) ce = ee;
  if (ce == cudaSuccess) ce = cudaGetLastError();
  if (ce == cudaSuccess) ce = cudaGraphInstantiate(out, graph, 0);
  cudaGraphDestroy(graph);
  if (ce != cudaSuccess)
    return fail(s, LE_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
  return LE_OK;
}

le_status ensure_graphs(le_sim *s) {
  if (!s->exec_one) CKS(capture(s, 1, nullptr, &s->exec_one));
  if (!s->exec_chunk) CKS(capture(s, kChunk, nullptr, &s->exec_chunk));
  return LE_OK;
}

// ------------------------------------------------------------- snapshots
le_status take_snapshot(le_sim *s) {
  void *ptr[7];
  size_t bytes[7];
  set_fields(s, s->h_dyn->cur, ptr, bytes);
  if (s->snap.empty()) {
    for (int f = 0; f < 7; ++f) {
      void *q = nullptr;
      CK(cudaMalloc(&q, std::max<size_t>(bytes[f], 256)));
      s->snap.push_back(q);
    }
    for (int f = 0; f < 4; ++f) {  // dyn, sum_prof, cnt_prof, acc_prof
      void *q = nullptr;
      CK(cudaMalloc(&q, std::max<size_t>(sizeof(Dyn) + 24 * (size_t)s->s.g.nbins, 256)));
      s->snap.push_back(q);
    }
  }
  for (int f = 0; f < 7; ++f)
    if (bytes[f]) CK(cudaMemcpyAsync(s->snap[f], ptr[f], bytes[f], cudaMemcpyDeviceToDevice, s->stream));
  const size_t nb = (size_t)s->s.g.nbins;
  CK(cudaMemcpyAsync(s->snap[7], s->s.dyn, sizeof(Dyn), cudaMemcpyDeviceToDevice, s->stream));
  CK(cudaMemcpyAsync(s->snap[8], s->s.w.sum_prof, 16 * nb, cudaMemcpyDeviceToDevice, s->stream));
  CK(cudaMemcpyAsync(s->snap[9], s->s.w.cnt_prof, 8 * nb, cudaMemcpyDeviceToDevice, s->stream));
  CK(cudaMemcpyAsync(s->snap[10], s->s.w.acc_prof, 24 * nb, cudaMemcpyDeviceToDevice, s->stream));
  return LE_OK;
}

le_status restore_snapshot(le_sim *s, int cur) {
  void *ptr[7];
  size_t bytes[7];
  set_fields(s, cur, ptr, bytes);
  for (int f = 0; f < 7; ++f)
    if (bytes[f]) CK(cudaMemcpyAsync(ptr[f], s->snap[f], bytes[f], cudaMemcpyDeviceToDevice, s->stream));
  const size_t nb = (size_t)s->s.g.nbins;
  CK(cudaMemcpyAsync(s->s.dyn, s->snap[7], sizeof(Dyn), cudaMemcpyDeviceToDevice, s->stream));
  CK(cudaMemcpyAsync(s->s.w.sum_prof, s->snap[8], 16 * nb, cudaMemcpyDeviceToDevice, s->stream));
  CK(cudaMemcpyAsync(s->s.w.cnt_prof, s->snap[9], 8 * nb, cudaMemcpyDeviceToDevice, s->stream));
  CK(cudaMemcpyAsync(s->s.w.acc_prof, s->snap[10], 24 * nb, cudaMemcpyDeviceToDevice, s->stream));
  // the snapshot's cur names the set it was taken from
  int c = cur;
  CK(cudaMemcpyAsync(&s->s.dyn->cur, &c, sizeof(int), cudaMemcpyHostToDevice, s->stream));
  launch_relist(s->s, s->stream);
  CK(cudaGetLastError());
  return sync(s);
}

// Initial list build + forces for the particles staged in s->s.stage.
le_status initialise(le_sim *s) {
  Dyn d{};
  d.step = 0;
  d.build_step = 0;
  d.cur = 0;
  CK(cudaMemcpyAsync(s->s.dyn, &d, sizeof(Dyn), cudaMemcpyHostToDevice, s->stream));
  CK(cudaMemsetAsync(s->s.w.acc_prof, 0, 24 * (size_t)s->s.g.nbins, s->stream));
  CK(cudaMemsetAsync(s->s.w.sum_prof, 0, 16 * (size_t)s->s.g.nbins, s->stream));
  CK(cudaMemsetAsync(s->s.w.cnt_prof, 0, 8 * (size_t)s->s.g.nbins, s->stream));
  launch_tables(s->s, s->stream);
  // each piece is imported once its copy has landed (the copies of the later
  // pieces overlap the import of the earlier ones)
  for (int c = 0; c < kUpChunks; ++c) {
    CK(cudaStreamWaitEvent(s->stream, s->up_ev[c], 0));
    launch_import(s->s, s->stream, (int)up_piece(s->n, c), (int)up_piece(s->n, c + 1));
  }
  launch_rebuild(s->s, true, s->stream);
  CK(cudaGetLastError());
  CKS(read_dyn(s));
  if (s->h_dyn->list_max > s->s.g.maxnb) {
    // grow the list and build it again from the stored build record
    const int need = (int)std::ceil(s->h_dyn->list_max * 1.5) + 16;
    return fail(s, LE_ERR_CAPACITY, "grow:" + std::to_string(need));
  }
  launch_force(s->s, 1, s->stream);
  CK(cudaGetLastError());
  CKS(read_dyn(s));
  return status_from_err(s, s->h_dyn->err);
}

}  // namespace

// =================================================================== C ABI
extern "C" {

LE_API void le_default_params(le_params *p) {
  if (!p) return;
  std::memset(p, 0, sizeof *p);
  p->eps = p->sigma = p->mass = p->kT = p->xi = 1.0;
  p->dt = 0.005;
  p->lj_shift = 1;
  p->thermostat = LE_THERMO_PECULIAR;
  p->fene_k = 30.0;
  p->fene_R0 = 1.5;
  p->precision = LE_FP64;
  p->seed = 0;
  p->system_id = 0;
  p->sample_every = 1;
  p->profile_bins = 20;
}

LE_API le_status le_wait_selftest(void *cuda_stream, double *waited_ms) {
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int *flag = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t ce = cudaMalloc(&flag, sizeof(int));
  if (ce == cudaSuccess) ce = cudaMemsetAsync(flag, 0, sizeof(int), st);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e0);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
  if (ce == cudaSuccess) ce = cudaEventRecord(e0, st);
  if (ce == cudaSuccess) {
    launch_wait_probe(flag, st);
    ce = cudaGetLastError();
  }
  if (ce == cudaSuccess) ce = cudaEventRecord(e1, st);
  if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
  int gave_up = 0;
  if (ce == cudaSuccess) ce = cudaMemcpy(&gave_up, flag, sizeof(int), cudaMemcpyDeviceToHost);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (flag) cudaFree(flag);
  if (ce != cudaSuccess) return LE_ERR_CUDA;
  if (waited_ms) *waited_ms = (double)ms;
  return gave_up ? LE_ERR_TIMEOUT : LE_OK;
}

LE_API const char *le_status_string(le_status st) {
  switch (st) {
    case LE_OK: return "ok";
    case LE_ERR_INVALID_ARG: return "invalid argument";
    case LE_ERR_CUDA: return "CUDA error";
    case LE_ERR_OOM: return "out of device memory";
    case LE_ERR_BOX_TOO_SMALL: return "box too small for rc + skin";
    case LE_ERR_BOND_BROKEN: return "FENE bond broken";
    case LE_ERR_NONFINITE: return "non-finite force or velocity";
    case LE_ERR_CAPACITY: return "neighbour list capacity exceeded";
    case LE_ERR_TIMEOUT: return "device wait timed out";
    case LE_ERR_STATE: return "call out of order";
    case LE_ERR_RANGE: return "sampled value outside the profile range";
  }
  return "unknown status";
}

LE_API const char *le_last_error(const le_sim *s) { return s ? s->err.c_str() : "null handle"; }

LE_API le_status le_create(const double box[3], double shear_rate, double rc, double skin,
                           const le_params *p, void *cuda_stream, le_sim **out) {
  le_sim *s = nullptr;
  if (!out || !box || !p) return LE_ERR_INVALID_ARG;
  *out = nullptr;
  for (int a = 0; a < 3; ++a)
    if (!(box[a] > 0.0) || !std::isfinite(box[a])) return LE_ERR_INVALID_ARG;
  if (!(rc > 0.0) || !(skin >= 0.0) || !(p->dt > 0.0) || !(p->mass > 0.0) || !std::isfinite(shear_rate))
    return LE_ERR_INVALID_ARG;
  if (p->profile_bins < 1 || p->profile_bins > kMaxBins) return LE_ERR_INVALID_ARG;
  if (p->precision != LE_FP64 && p->precision != LE_FP32) return LE_ERR_INVALID_ARG;
  if (p->thermostat < LE_THERMO_NONE || p->thermostat > LE_THERMO_DPD) return LE_ERR_INVALID_ARG;
  if (!(p->force_cap >= 0.0) || (p->force_cap > 0.0 && p->precision != LE_FP64))
    return LE_ERR_INVALID_ARG;
  const double rl = rc + skin;
  for (int a = 0; a < 3; ++a)
    if (!(rl < 0.5 * box[a])) return LE_ERR_BOX_TOO_SMALL;
  s = new (std::nothrow) le_sim;
  if (!s) return LE_ERR_OOM;
  std::memcpy(s->box, box, sizeof s->box);
  s->shear_rate = shear_rate;
  s->rc = rc;
  s->skin = skin;
  s->prm = *p;
  fill_geom(s, box, shear_rate, rc, skin, p);
  s->s.prec = p->precision;
  cudaError_t e;
  if (cuda_stream) {
    s->stream = (cudaStream_t)cuda_stream;
  } else {
    e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) { delete s; return LE_ERR_CUDA; }
    s->own_stream = true;
  }
  e = cudaStreamCreateWithFlags(&s->cap_main, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->cap_side, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->up_stream, cudaStreamNonBlocking);
  for (int c = 0; c < kUpChunks && e == cudaSuccess; ++c)
    e = cudaEventCreateWithFlags(&s->up_ev[c], cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->up_go, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMallocHost(&s->h_scalar, 64);
  if (e == cudaSuccess) e = cudaMallocHost(&s->h_dyn, sizeof(Dyn));
  if (e != cudaSuccess) {
    le_destroy(s);
    return LE_ERR_CUDA;
  }
  *out = s;
  return LE_OK;
}

LE_API le_status le_set_eager(le_sim *s, int eager) {
  if (!s) return LE_ERR_INVALID_ARG;
  s->eager = eager != 0;
  return LE_OK;
}

LE_API le_status le_destroy(le_sim *s) {
  if (!s) return LE_ERR_INVALID_ARG;
  if (s->stream) cudaStreamSynchronize(s->stream);
  free_device(s);
  if (s->h_scalar) cudaFreeHost(s->h_scalar);
  if (s->h_dyn) cudaFreeHost(s->h_dyn);
  if (s->cap_main) cudaStreamDestroy(s->cap_main);
  if (s->cap_side) cudaStreamDestroy(s->cap_side);
  if (s->up_stream) {
    cudaStreamSynchronize(s->up_stream);
    cudaStreamDestroy(s->up_stream);
  }
  for (cudaEvent_t ev : s->up_ev)
    if (ev) cudaEventDestroy(ev);
  if (s->up_go) cudaEventDestroy(s->up_go);
  if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
  delete s;
  return LE_OK;
}

LE_API le_status le_set_bonds(le_sim *s, int64_t nb, const int32_t *pairs) {
  if (!s || nb < 0 || (nb > 0 && !pairs)) return fail(s, LE_ERR_INVALID_ARG, "bad bond arguments");
  for (int64_t b = 0; b < nb; ++b) {
    const int32_t i = pairs[2 * b], j = pairs[2 * b + 1];
    if (i < 0 || j < 0 || i == j) return fail(s, LE_ERR_INVALID_ARG, "bad bond pair");
    if (s->has_particles && (i >= s->n || j >= s->n))
      return fail(s, LE_ERR_INVALID_ARG, "bond id out of range");
  }
  s->bonds.assign(pairs, pairs + 2 * nb);
  if (!s->has_particles) return LE_OK;
  // re-initialise from the current state
  std::vector<double> pos(3 * s->n), vel(3 * s->n);
  CKS(le_positions(s, pos.data(), vel.data()));
  return le_set_particles(s, s->n, pos.data(), vel.data());
}

LE_API le_status le_set_particles(le_sim *s, int64_t n, const double *pos, const double *vel) {
  if (!s) return LE_ERR_INVALID_ARG;
  if (n < 1 || n > kMaxParticles || !pos || !vel)
    return fail(s, LE_ERR_INVALID_ARG, "n out of range or null arrays");
  // non-finite coordinates or velocities are found by the import kernel
  // bond table by particle id (host work only when there are bonds)
  std::vector<int> deg;
  int maxb = 0;
  if (!s->bonds.empty()) {
    deg.assign(n, 0);
    for (size_t b = 0; b < s->bonds.size() / 2; ++b) {
      const int i = s->bonds[2 * b], j = s->bonds[2 * b + 1];
      if (i >= n || j >= n) return fail(s, LE_ERR_INVALID_ARG, "bond id out of range");
      ++deg[i];
      ++deg[j];
    }
    for (int64_t i = 0; i < n; ++i) maxb = std::max(maxb, deg[i]);
  }
  if (maxb > kMaxBonds) return fail(s, LE_ERR_INVALID_ARG, "more than 8 bonds on a particle");
  Geom &g = s->s.g;
  g.maxb = maxb;
  choose_cells(s);
  const double V = g.L[0] * g.L[1] * g.L[2];
  const double mean_nb = 4.18879020478639 * g.rl * g.rl * g.rl * (double)n / V;
  int maxnb = (int)std::ceil(mean_nb * 1.6) + 32;
  maxnb = std::min<long long>(maxnb, n) < 8 ? 8 : maxnb;
  for (int attempt = 0; attempt < 4; ++attempt) {
    CKS(allocate(s, n, maxnb));
    if (maxb > 0) {
      std::vector<int> bg((size_t)n * maxb, -1);
      std::fill(deg.begin(), deg.end(), 0);
      for (size_t b = 0; b < s->bonds.size() / 2; ++b) {
        const int i = s->bonds[2 * b], j = s->bonds[2 * b + 1];
        bg[(size_t)i * maxb + deg[i]++] = j;
        bg[(size_t)j * maxb + deg[j]++] = i;
      }
      CK(cudaMemcpyAsync(s->s.w.bond_gid, bg.data(), sizeof(int) * bg.size(),
                         cudaMemcpyHostToDevice, s->stream));
      // the pageable copy has left bg by the time it returns
    } else {
      // no bonds: the one slot per particle holds -1 (every byte 0xFF)
      CK(cudaMemsetAsync(s->s.w.bond_gid, 0xFF, sizeof(int) * (size_t)n, s->stream));
    }
    CKS(upload_particles(s, pos, vel));
    le_status st = initialise(s);
    if (st == LE_ERR_CAPACITY && s->err.rfind("grow:", 0) == 0) {
      maxnb = std::stoi(s->err.substr(5));
      continue;
    }
    if (st != LE_OK) return st;
    s->has_particles = true;
    return LE_OK;
  }
  return fail(s, LE_ERR_CAPACITY, "neighbour list could not be sized");
}

// One step without graphs: the host reads the rebuild decision back.  The
// same launches as a graph of the call's steps: `drift` is false where the
// previous step's force launch ran this step's drift, `fuse` (mode 2) hands
// the next step's drift to this force launch.
static le_status eager_step(le_sim *s, cudaEvent_t *ev, bool drift, bool fuse) {
  if (ev) CK(cudaEventRecord(ev[0], s->stream));
  if (drift) launch_drift(s->s, s->stream);
  if (ev) CK(cudaEventRecord(ev[1], s->stream));
  launch_decide(s->s, 0, 0, s->stream);
  CK(cudaMemcpyAsync(s->h_scalar, &s->s.dyn->rebuild, sizeof(int), cudaMemcpyDeviceToHost,
                     s->stream));
  CKS(sync(s));
  if (*(int *)s->h_scalar) launch_rebuild(s->s, false, s->stream);
  if (ev) CK(cudaEventRecord(ev[2], s->stream));
  launch_force(s->s, fuse ? 2 : 0, s->stream);
  if (ev) CK(cudaEventRecord(ev[3], s->stream));
  CK(cudaGetLastError());
  return LE_OK;
}

// eager_step k of a call of n steps, fused as a graph of n steps would be
static le_status eager_step_of(le_sim *s, cudaEvent_t *ev, int64_t k, int64_t n) {
  const bool f = can_fuse_drift(s->s);
  return eager_step(s, ev, k == 0 || !f, f && k + 1 < n);
}

static le_status step_once(le_sim *s, int64_t nsteps) {
  if (s->eager) {
    for (int64_t k = 0; k < nsteps; ++k) CKS(eager_step_of(s, nullptr, k, nsteps));
    launch_fold(s->s, s->stream);
    CK(cudaGetLastError());
    return read_dyn(s);
  }
  CKS(ensure_graphs(s));
  int64_t left = nsteps;
  while (left >= kChunk) {
    CK(cudaGraphLaunch(s->exec_chunk, s->stream));
    left -= kChunk;
  }
  if (left > 0) {
    // the remaining steps as one graph (captured on first use)
    cudaGraphExec_t &g = left == 1 ? s->exec_one : s->exec_rem[left];
    if (!g) CKS(capture(s, (int)left, nullptr, &g));
    CK(cudaGraphLaunch(g, s->stream));
  }
  launch_fold(s->s, s->stream);
  CK(cudaGetLastError());
  return read_dyn(s);
}

// A longer neighbour list (the graphs captured the old one and are dropped),
// rebuilt from the current build record.
static le_status grow_list(le_sim *s, int maxnb) {
  uint32_t *old = s->s.w.nbr;
  for (size_t k = 0; k < s->allocs.size(); ++k)
    if (s->allocs[k] == old) {
      s->allocs.erase(s->allocs.begin() + (long)k);
      break;
    }
  CK(cudaStreamSynchronize(s->stream));
  CK(cudaFree(old));
  s->s.w.nbr = nullptr;
  CKS(dalloc(s, &s->s.w.nbr, (size_t)s->s.g.npad * (size_t)maxnb));
  s->s.g.maxnb = maxnb;
  destroy_graphs(s);
  launch_relist(s->s, s->stream);
  CK(cudaGetLastError());
  return sync(s);
}

LE_API le_status le_step(le_sim *s, int64_t nsteps) {
  if (!s) return LE_ERR_INVALID_ARG;
  if (!s->has_particles) return fail(s, LE_ERR_STATE, "le_set_particles has not been called");
  if (nsteps < 0) return fail(s, LE_ERR_INVALID_ARG, "negative step count");
  if (nsteps == 0) return LE_OK;
  for (int attempt = 0; attempt < 4; ++attempt) {
    CKS(read_dyn(s));
    const int cur0 = s->h_dyn->cur;
    CKS(take_snapshot(s));
    CKS(step_once(s, nsteps));
    const int err = s->h_dyn->err;
    if (!err) return LE_OK;
    le_status st = status_from_err(s, err);
    const std::string msg = s->err;
    const int seen = s->h_dyn->list_max;
    CKS(restore_snapshot(s, cur0));
    if (st != LE_ERR_CAPACITY)
      return fail(s, st, msg + " (state rolled back to the start of the call)");
    // the list overflowed: roll back, lengthen it and run the call again
    CKS(grow_list(s, (int)std::ceil(std::max(seen, s->s.g.maxnb) * 1.3) + 16));
  }
  return fail(s, LE_ERR_CAPACITY, "neighbour list capacity could not be grown enough");
}

LE_API le_status le_step_profiled(le_sim *s, int64_t nsteps, double *force_ms, double *integrate_ms,
                                  double *total_ms) {
  if (!s) return LE_ERR_INVALID_ARG;
  if (!s->has_particles) return fail(s, LE_ERR_STATE, "le_set_particles has not been called");
  if (nsteps < 1 || nsteps > 100000) return fail(s, LE_ERR_INVALID_ARG, "nsteps out of range");
  std::vector<cudaEvent_t> ev(4 * nsteps);
  for (auto &e : ev) CK(cudaEventCreate(&e));
  cudaEvent_t t0, t1;
  CK(cudaEventCreate(&t0));
  CK(cudaEventCreate(&t1));
  cudaGraphExec_t exec = nullptr;
  le_status st = LE_OK;
  if (s->eager) {
    CK(cudaEventRecord(t0, s->stream));
    for (int64_t k = 0; k < nsteps && st == LE_OK; ++k) st = eager_step_of(s, &ev[4 * k], k, nsteps);
    CK(cudaEventRecord(t1, s->stream));
    launch_fold(s->s, s->stream);
    if (st == LE_OK) st = read_dyn(s);
  } else {
    st = capture(s, (int)nsteps, &ev, &exec);
    if (st == LE_OK) {
      CK(cudaEventRecord(t0, s->stream));
      CK(cudaGraphLaunch(exec, s->stream));
      CK(cudaEventRecord(t1, s->stream));
      launch_fold(s->s, s->stream);
      st = read_dyn(s);
    }
  }
  if (st == LE_OK) {
    double fsum = 0, isum = 0;
    for (int64_t k = 0; k < nsteps; ++k) {
      float a = 0, b = 0;
      CK(cudaEventElapsedTime(&a, ev[4 * k + 0], ev[4 * k + 1]));
      CK(cudaEventElapsedTime(&b, ev[4 * k + 2], ev[4 * k + 3]));
      isum += a;
      fsum += b;
    }
    float tt = 0;
    CK(cudaEventElapsedTime(&tt, t0, t1));
    if (force_ms) *force_ms = fsum;
    if (integrate_ms) *integrate_ms = isum;
    if (total_ms) *total_ms = tt;
    st = status_from_err(s, s->h_dyn->err);
  }
  if (exec) cudaGraphExecDestroy(exec);
  for (auto &e : ev) cudaEventDestroy(e);
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  return st;
}

LE_API le_status le_forces(le_sim *s, double *out) {
  if (!s || !out) return fail(s, LE_ERR_INVALID_ARG, "null argument");
  if (!s->has_particles) return fail(s, LE_ERR_STATE, "no particles");
  launch_export_forces(s->s, s->stream);
  CK(cudaGetLastError());
  CKS(download(s, out, s->s.stage, 3 * (size_t)s->n, s->h_stage));
  return sync(s);
}

LE_API le_status le_positions(le_sim *s, double *pos, double *vel) {
  if (!s) return LE_ERR_INVALID_ARG;
  if (!s->has_particles) return fail(s, LE_ERR_STATE, "no particles");
  const int64_t n = s->n;
  if ((!pos || is_pinned(pos)) && (!vel || is_pinned(vel))) {
    // pinned destinations: the output in kUpChunks pieces of caller ids, each
    // copied back on up_stream while the next piece is exported
    for (int c = 0; c < kUpChunks; ++c) {
      const int64_t a = up_piece(n, c), b = up_piece(n, c + 1);
      launch_export_ids(s->s, s->stream, (int)a, (int)b);
      CK(cudaGetLastError());
      CK(cudaEventRecord(s->up_ev[c], s->stream));
      CK(cudaStreamWaitEvent(s->up_stream, s->up_ev[c], 0));
      if (b > a && pos)
        CK(cudaMemcpyAsync(pos + 3 * a, s->s.stage + 3 * a, sizeof(double) * 3 * (size_t)(b - a),
                           cudaMemcpyDeviceToHost, s->up_stream));
      if (b > a && vel)
        CK(cudaMemcpyAsync(vel + 3 * a, s->s.stage + 3 * n + 3 * a,
                           sizeof(double) * 3 * (size_t)(b - a), cudaMemcpyDeviceToHost,
                           s->up_stream));
    }
    CK(cudaStreamSynchronize(s->up_stream));
    return sync(s);
  }
  launch_export(s->s, s->stream);
  CK(cudaGetLastError());
  if (pos) CKS(download(s, pos, s->s.stage, 3 * (size_t)n, s->h_stage));
  if (vel) CKS(download(s, vel, s->s.stage + 3 * n, 3 * (size_t)n, s->h_stage + 3 * n));
  return sync(s);
}

LE_API le_status le_stress(le_sim *s, double out9[9], double *xz_avg, int64_t *nsamples) {
  if (!s) return LE_ERR_INVALID_ARG;
  if (!s->has_particles) return fail(s, LE_ERR_STATE, "no particles");
  if (out9) {
    const int nb = observe_blocks(s->s);
    launch_observe(s->s, s->stream);
    CK(cudaGetLastError());
    std::vector<double> part((size_t)nb * 16);
    CK(cudaMemcpyAsync(part.data(), s->s.partials, sizeof(double) * part.size(),
                       cudaMemcpyDeviceToHost, s->stream));
    CKS(sync(s));
    double acc[9] = {0};
    for (int b = 0; b < nb; ++b)
      for (int q = 0; q < 9; ++q) acc[q] += part[(size_t)b * 16 + q];
    const Geom &g = s->s.g;
    const double V = g.L[0] * g.L[1] * g.L[2];
    for (int q = 0; q < 9; ++q) out9[q] = -acc[q] / V;
  }
  CKS(read_dyn(s));
  if (xz_avg) *xz_avg = s->h_dyn->nsamples ? s->h_dyn->sum_sxz / (double)s->h_dyn->nsamples : 0.0;
  if (nsamples) *nsamples = s->h_dyn->nsamples;
  return LE_OK;
}

LE_API le_status le_temperature(le_sim *s, double *tpec_avg) {
  if (!s || !tpec_avg) return LE_ERR_INVALID_ARG;
  if (!s->has_particles) return fail(s, LE_ERR_STATE, "no particles");
  CKS(read_dyn(s));
  *tpec_avg = s->h_dyn->nsamples ? s->h_dyn->sum_tpec / (double)s->h_dyn->nsamples : 0.0;
  return LE_OK;
}

LE_API le_status le_velocity_profile(le_sim *s, int nbins, double *vx_mean, int64_t *counts) {
  if (!s) return LE_ERR_INVALID_ARG;
  if (!s->has_particles) return fail(s, LE_ERR_STATE, "no particles");
  if (nbins != s->s.g.nbins) return fail(s, LE_ERR_INVALID_ARG, "nbins differs from profile_bins");
  std::vector<double> sum(nbins);
  std::vector<long long> cnt(nbins);
  CK(cudaMemcpyAsync(sum.data(), s->s.w.sum_prof, 8 * (size_t)nbins, cudaMemcpyDeviceToHost, s->stream));
  CK(cudaMemcpyAsync(cnt.data(), s->s.w.cnt_prof, 8 * (size_t)nbins, cudaMemcpyDeviceToHost, s->stream));
  CKS(sync(s));
  for (int b = 0; b < nbins; ++b) {
    if (vx_mean) vx_mean[b] = cnt[b] ? sum[b] / (double)cnt[b] : NAN;
    if (counts) counts[b] = cnt[b];
  }
  return LE_OK;
}

LE_API le_status le_profiles(le_sim *s, int nbins, double *vx_mean, double *t_y, double *density,
                             int64_t *counts) {
  if (!s) return LE_ERR_INVALID_ARG;
  if (!s->has_particles) return fail(s, LE_ERR_STATE, "no particles");
  if (nbins != s->s.g.nbins) return fail(s, LE_ERR_INVALID_ARG, "nbins differs from profile_bins");
  std::vector<double> sum(2 * (size_t)nbins);
  std::vector<long long> cnt(nbins);
  CK(cudaMemcpyAsync(sum.data(), s->s.w.sum_prof, 16 * (size_t)nbins, cudaMemcpyDeviceToHost, s->stream));
  CK(cudaMemcpyAsync(cnt.data(), s->s.w.cnt_prof, 8 * (size_t)nbins, cudaMemcpyDeviceToHost, s->stream));
  CKS(read_dyn(s));
  const Geom &g = s->s.g;
  const double vbin = g.L[0] * g.L[1] * g.L[2] / nbins;
  const long long ns = s->h_dyn->nsamples;
  for (int b = 0; b < nbins; ++b) {
    if (vx_mean) vx_mean[b] = cnt[b] ? sum[b] / (double)cnt[b] : NAN;
    if (t_y) t_y[b] = cnt[b] ? sum[nbins + b] / (double)cnt[b] : NAN;
    if (density) density[b] = ns ? (double)cnt[b] / ((double)ns * vbin) : NAN;
    if (counts) counts[b] = cnt[b];
  }
  return LE_OK;
}

LE_API le_status le_reset_samples(le_sim *s) {
  if (!s) return LE_ERR_INVALID_ARG;
  if (!s->has_particles) return fail(s, LE_ERR_STATE, "no particles");
  CKS(read_dyn(s));
  Dyn d = *s->h_dyn;
  d.sum_sxz = d.sum_tpec = 0.0;
  d.nsamples = 0;
  d.acc_sxz = d.acc_ke = 0;
  d.pending = 0;
  CK(cudaMemcpyAsync(s->s.dyn, &d, sizeof(Dyn), cudaMemcpyHostToDevice, s->stream));
  const size_t nb = (size_t)s->s.g.nbins;
  CK(cudaMemsetAsync(s->s.w.acc_prof, 0, 24 * nb, s->stream));
  CK(cudaMemsetAsync(s->s.w.sum_prof, 0, 16 * nb, s->stream));
  CK(cudaMemsetAsync(s->s.w.cnt_prof, 0, 8 * nb, s->stream));
  return sync(s);
}

LE_API le_status le_get_counters(le_sim *s, le_counters *out) {
  if (!s || !out) return LE_ERR_INVALID_ARG;
  std::memset(out, 0, sizeof *out);
  if (!s->has_particles) return LE_OK;
  CKS(read_dyn(s));
  out->step = s->h_dyn->step;
  out->particles = s->n;
  out->rebuilds = s->h_dyn->nrebuild;
  out->image_rebuilds = s->h_dyn->nimage;
  out->list_capacity = s->s.g.maxnb;
  out->list_max = s->h_dyn->list_max;
  for (int a = 0; a < 3; ++a) out->cells[a] = s->s.g.nc[a];
  out->dX = s->h_dyn->dX;
  out->list_mean = (double)s->h_dyn->list_entries / (double)s->n;
  out->force_threads = s->s.force_threads;
  out->list_threads = s->s.list_threads;
  return LE_OK;
}

static void drop_graphs(le_sim *s) { destroy_graphs(s); }

LE_API le_status le_set_launch(le_sim *s, int force_threads, int list_threads) {
  if (!s) return LE_ERR_INVALID_ARG;
  auto ok = [](int t, int mx) { return t >= 32 && t <= mx && t % 32 == 0; };
  if (!ok(force_threads, kForceThreads) || !ok(list_threads, kListMaxThreads))
    return fail(s, LE_ERR_INVALID_ARG, "launch shape: multiples of 32 up to 256 threads");
  s->s.force_threads = force_threads;
  s->s.list_threads = list_threads;
  drop_graphs(s);
  return LE_OK;
}

// The autotuner: every candidate shape runs the system's own step graph from
// the same snapshot (one chunk to warm, then the timed chunks), and the state
// is restored after each trial, so tuning leaves no trace but the choice.
LE_API le_status le_tune(le_sim *s, int steps_per_trial, int *best_force, int *best_list,
                         double *ms_per_step) {
  if (!s) return LE_ERR_INVALID_ARG;
  if (!s->has_particles) return fail(s, LE_ERR_STATE, "le_set_particles has not been called");
  if (steps_per_trial < 1) return fail(s, LE_ERR_INVALID_ARG, "steps_per_trial < 1");
  const int chunks = std::max(1, steps_per_trial / kChunk);
  CKS(read_dyn(s));
  const int cur0 = s->h_dyn->cur;
  CKS(take_snapshot(s));
  const int forces[2] = {128, 256}, lists[3] = {64, 128, 256};
  int bf = s->s.force_threads, bl = s->s.list_threads;
  double best = 0.0;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  le_status st = LE_OK;
  // two sweeps over the shapes, each shape scored by its faster trial
  double tmin[2][3] = {{0, 0, 0}, {0, 0, 0}};
  for (int rep = 0; rep < 2 && st == LE_OK; ++rep)
  for (int a = 0; a < 2 && st == LE_OK; ++a)
    for (int c = 0; c < 3 && st == LE_OK; ++c) {
      s->s.force_threads = forces[a];
      s->s.list_threads = lists[c];
      drop_graphs(s);
      st = ensure_graphs(s);
      if (st != LE_OK) break;
      CK(cudaGraphLaunch(s->exec_chunk, s->stream));
      CK(cudaEventRecord(e0, s->stream));
      for (int k = 0; k < chunks; ++k) CK(cudaGraphLaunch(s->exec_chunk, s->stream));
      CK(cudaEventRecord(e1, s->stream));
      CKS(read_dyn(s));
      const int err = s->h_dyn->err;
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      CKS(restore_snapshot(s, cur0));
      if (err) {
        st = status_from_err(s, err);
        break;
      }
      const double per = (double)ms / (double)(chunks * kChunk);
      if (tmin[a][c] == 0.0 || per < tmin[a][c]) tmin[a][c] = per;
    }
  for (int a = 0; a < 2; ++a)
    for (int c = 0; c < 3; ++c)
      if (tmin[a][c] > 0.0 && (best == 0.0 || tmin[a][c] < best)) {
        best = tmin[a][c];
        bf = forces[a];
        bl = lists[c];
      }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  s->s.force_threads = bf;
  s->s.list_threads = bl;
  drop_graphs(s);
  if (st != LE_OK) return st;
  if (!s->eager) CKS(ensure_graphs(s));
  if (best_force) *best_force = bf;
  if (best_list) *best_list = bl;
  if (ms_per_step) *ms_per_step = best;
  return LE_OK;
}

namespace {
struct StateHeader {
  uint64_t magic;
  int32_t version, prec;
  int64_t n;
  int32_t maxb, nbins;
  int32_t ncell, pad;
};
}  // namespace

LE_API le_status le_get_state(le_sim *s, void *buf, size_t *bytes) {
  if (!s || !bytes) return LE_ERR_INVALID_ARG;
  if (!s->has_particles) return fail(s, LE_ERR_STATE, "no particles");
  CKS(read_dyn(s));
  void *ptr[7];
  size_t fb[7];
  set_fields(s, s->h_dyn->cur, ptr, fb);
  const size_t nb = (size_t)s->s.g.nbins;
  size_t total = sizeof(StateHeader) + sizeof(Dyn) + 16 * nb + 8 * nb + 24 * nb;
  for (int f = 0; f < 7; ++f) total += fb[f];
  if (!buf) {
    *bytes = total;
    return LE_OK;
  }
  if (*bytes < total) return fail(s, LE_ERR_INVALID_ARG, "state buffer too small");
  char *o = static_cast<char *>(buf);
  StateHeader h{kStateMagic, kStateVersion, s->s.prec, s->n, s->s.g.maxb, (int32_t)nb, s->s.g.ncell, 0};
  std::memcpy(o, &h, sizeof h);
  o += sizeof h;
  std::memcpy(o, s->h_dyn, sizeof(Dyn));
  o += sizeof(Dyn);
  for (int f = 0; f < 7; ++f) {
    if (fb[f]) CK(cudaMemcpyAsync(o, ptr[f], fb[f], cudaMemcpyDeviceToHost, s->stream));
    o += fb[f];
  }
  CK(cudaMemcpyAsync(o, s->s.w.sum_prof, 16 * nb, cudaMemcpyDeviceToHost, s->stream));
  o += 16 * nb;
  CK(cudaMemcpyAsync(o, s->s.w.cnt_prof, 8 * nb, cudaMemcpyDeviceToHost, s->stream));
  o += 8 * nb;
  CK(cudaMemcpyAsync(o, s->s.w.acc_prof, 24 * nb, cudaMemcpyDeviceToHost, s->stream));
  *bytes = total;
  return sync(s);
}

LE_API le_status le_set_state(le_sim *s, const void *buf, size_t bytes) {
  if (!s || !buf) return LE_ERR_INVALID_ARG;
  if (!s->has_particles) return fail(s, LE_ERR_STATE, "load particles of the same size first");
  StateHeader h;
  if (bytes < sizeof h) return fail(s, LE_ERR_INVALID_ARG, "state blob too small");
  std::memcpy(&h, buf, sizeof h);
  const size_t nb = (size_t)s->s.g.nbins;
  if (h.magic != kStateMagic || h.version != kStateVersion || h.prec != s->s.prec || h.n != s->n ||
      h.maxb != s->s.g.maxb || (size_t)h.nbins != nb || h.ncell != s->s.g.ncell)
    return fail(s, LE_ERR_INVALID_ARG, "state blob does not match this handle");
  void *ptr[7];
  size_t fb[7];
  set_fields(s, 0, ptr, fb);
  size_t total = sizeof(StateHeader) + sizeof(Dyn) + 48 * nb;
  for (int f = 0; f < 7; ++f) total += fb[f];
  if (bytes < total) return fail(s, LE_ERR_INVALID_ARG, "state blob truncated");
  const char *o = static_cast<const char *>(buf) + sizeof h;
  Dyn d;
  std::memcpy(&d, o, sizeof d);
  o += sizeof d;
  d.cur = 0;
  d.err = 0;
  d.maxdisp2 = 0;
  CK(cudaMemcpy(s->s.dyn, &d, sizeof d, cudaMemcpyHostToDevice));
  for (int f = 0; f < 7; ++f) {
    if (fb[f]) CK(cudaMemcpy(ptr[f], o, fb[f], cudaMemcpyHostToDevice));
    o += fb[f];
  }
  CK(cudaMemcpy(s->s.w.sum_prof, o, 16 * nb, cudaMemcpyHostToDevice));
  o += 16 * nb;
  CK(cudaMemcpy(s->s.w.cnt_prof, o, 8 * nb, cudaMemcpyHostToDevice));
  o += 8 * nb;
  CK(cudaMemcpy(s->s.w.acc_prof, o, 24 * nb, cudaMemcpyHostToDevice));
  launch_relist(s->s, s->stream);
  CK(cudaGetLastError());
  CKS(read_dyn(s));
  return status_from_err(s, s->h_dyn->err);
}

}  // extern "C"

// =================================================================== batches
// Many independent boxes advanced by one graph launch: each member's steps
// are recorded on its own capture stream, forked from and joined back into
// one batch capture, so the graph holds one branch per member and the device
// runs the members' kernels concurrently.  The kernels are the members' own,
// so every member's trajectory is bit-identical to stepping it alone.
// Device tables of one batch group (members sharing precision, bonds,
// thermostat kind): the member records and the per-kind block prefixes.
struct BatchGroup {
  le::BatchGrid grid;
  void *d_mem = nullptr;
  int *d_off = nullptr;
  int *d_act = nullptr;  // rebuild tables, rewritten on the device every step
};

struct le_batch {
  size_t budget = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaStream_t cap = nullptr;
  std::vector<le_sim *> members;
  cudaGraphExec_t exec_chunk = nullptr, exec_one = nullptr;
  std::vector<BatchGroup> groups;
  std::string err;
};

namespace {

le_status bfail(le_batch *b, le_status st, const std::string &msg) {
  if (b) b->err = msg;
  return st;
}

void batch_drop_graphs(le_batch *b) {
  if (b->exec_chunk) cudaGraphExecDestroy(b->exec_chunk);
  if (b->exec_one) cudaGraphExecDestroy(b->exec_one);
  b->exec_chunk = b->exec_one = nullptr;
  // the tables hold member pointers, shapes and capacities: rebuilt with the graphs
  for (BatchGroup &gr : b->groups) {
    if (gr.d_mem) cudaFree(gr.d_mem);
    if (gr.d_off) cudaFree(gr.d_off);
    if (gr.d_act) cudaFree(gr.d_act);
  }
  b->groups.clear();
}

// Sort tiles of a batch member: always the full 16 keys per thread.  A batch
// fills the GPU with many members, so the smaller tiles a system sorted on
// its own gets (sort_blocks_for) would only add tiles and count-table
// entries.  Fewer tiles than the member's own never outgrow its tables.
int batch_sort_blocks(int64_t n) {
  const int64_t tile = (int64_t)kSortThreads * kSortItems;
  return (int)((n + tile - 1) / tile);
}

template <class R>
void fill_members(const std::vector<le_sim *> &sims, std::vector<MemberDev<R>> &out) {
  out.resize(sims.size());
  for (size_t k = 0; k < sims.size(); ++k) {
    const SysDev &sd = sims[k]->s;
    MemberDev<R> &m = out[k];
    m.g = sd.g;
    m.d = sd.dyn;
    if constexpr (sizeof(R) == 4) {
      m.s0 = sd.f32[0];
      m.s1 = sd.f32[1];
    } else {
      m.s0 = sd.f64[0];
      m.s1 = sd.f64[1];
    }
    m.w = sd.w;
    m.sort_part = sd.sort_part;
    m.sort_passes = sd.sort_passes;
    m.sort_blocks = batch_sort_blocks(sd.g.n);
  }
}

// Groups the members and uploads each group's tables.  All members of a
// group launch with the first member's shapes (shapes change no result).
le_status batch_build_groups(le_batch *b) {
  std::map<std::tuple<int, int, int>, std::vector<le_sim *>> bykey;
  for (le_sim *s : b->members)
    bykey[std::make_tuple(s->s.prec, s->s.g.maxb > 0 ? 1 : 0,
                          s->s.g.thermostat == LE_THERMO_DPD ? 1 : 0)]
        .push_back(s);
  for (auto &kv : bykey) {
    const std::vector<le_sim *> &sims = kv.second;
    BatchGroup gr;
    BatchGrid &bg = gr.grid;
    bg.M = (int)sims.size();
    bg.prec = std::get<0>(kv.first);
    bg.bonds = std::get<1>(kv.first);
    bg.dpd = std::get<2>(kv.first);
    bg.force_threads = sims[0]->s.force_threads;
    bg.list_threads = sims[0]->s.list_threads;
    bg.nbins = 1;
    bg.passes = 1;
    const int M1 = bg.M + 1;
    std::vector<int> off((size_t)kBKinds * M1, 0);
    for (int k = 0; k < bg.M; ++k) {
      const SysDev &sd = sims[k]->s;
      bg.nbins = std::max(bg.nbins, sd.g.nbins);
      bg.passes = std::max(bg.passes, sd.sort_passes);
      int cnt[kBKinds];
      cnt[kB256] = blocks_for(sd.g.n, 256);
      cnt[kBForce] = blocks_for(sd.g.n, bg.force_threads);
      cnt[kBList] = blocks_for(sd.g.n, bg.list_threads);
      cnt[kBSort] = batch_sort_blocks(sd.g.n);
      cnt[kBOne] = 1;
      for (int p = 0; p < kMaxSortPasses; ++p) {
        cnt[kBScan0 + p] = sort_scan_blocks(sd.g.sort_bits, batch_sort_blocks(sd.g.n), p);
        if (sort_scan_large(sd.g.sort_bits, batch_sort_blocks(sd.g.n), p)) bg.scan_large[p] = true;
      }
      for (int kind = 0; kind < kBKinds; ++kind)
        off[(size_t)kind * M1 + k + 1] = off[(size_t)kind * M1 + k] + cnt[kind];
    }
    for (int kind = 0; kind < kBKinds; ++kind) bg.blocks[kind] = off[(size_t)kind * M1 + bg.M];
    size_t mem_bytes = 0;
    std::vector<MemberDev<float>> mf;
    std::vector<MemberDev<double>> md;
    const void *host_mem = nullptr;
    if (bg.prec == 1) {
      fill_members(sims, mf);
      host_mem = mf.data();
      mem_bytes = mf.size() * sizeof(MemberDev<float>);
    } else {
      fill_members(sims, md);
      host_mem = md.data();
      mem_bytes = md.size() * sizeof(MemberDev<double>);
    }
    const size_t act_bytes = (size_t)kBKinds * batch_act_stride(bg.M) * sizeof(int);
    cudaError_t ce = cudaMalloc(&gr.d_mem, mem_bytes);
    if (ce == cudaSuccess) ce = cudaMalloc(&gr.d_off, off.size() * sizeof(int));
    if (ce == cudaSuccess) ce = cudaMalloc(&gr.d_act, act_bytes);
    if (ce == cudaSuccess) ce = cudaMemset(gr.d_act, 0, act_bytes);  // no member listed
    if (ce == cudaSuccess) ce = cudaMemcpy(gr.d_mem, host_mem, mem_bytes, cudaMemcpyHostToDevice);
    if (ce == cudaSuccess)
      ce = cudaMemcpy(gr.d_off, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice);
    bg.mem = gr.d_mem;
    bg.off = gr.d_off;
    bg.act = gr.d_act;
    b->groups.push_back(gr);
    if (ce != cudaSuccess) return bfail(b, LE_ERR_CUDA, std::string("batch tables: ") + cudaGetErrorString(ce));
  }
  return LE_OK;
}

le_status batch_capture(le_batch *b, int steps, cudaGraphExec_t *out) {
  if (b->groups.empty()) {
    le_status st = batch_build_groups(b);
    if (st != LE_OK) return st;
  }
  cudaError_t ce = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
  if (ce != cudaSuccess) return bfail(b, LE_ERR_CUDA, cudaGetErrorString(ce));
  // as for one system: where a group allows it, each force launch but the
  // last also runs the next step's drift
  for (int k = 0; k < steps; ++k)
    for (const BatchGroup &gr : b->groups)
      launch_batch_step(gr.grid, b->cap, k == 0, k + 1 < steps);
  cudaGraph_t captured = nullptr;
  cudaError_t ee = cudaStreamEndCapture(b->cap, &captured);
  if (ce == cudaSuccess) ce = ee;
  if (ce == cudaSuccess) ce = cudaGetLastError();
  if (ce == cudaSuccess) ce = cudaGraphInstantiate(out, captured, 0);
  if (captured) cudaGraphDestroy(captured);
  if (ce != cudaSuccess)
    return bfail(b, LE_ERR_CUDA, std::string("batch graph capture: ") + cudaGetErrorString(ce));
  return LE_OK;
}

le_status batch_run(le_batch *b, int64_t nsteps) {
  if (!b->exec_one) {
    le_status st = batch_capture(b, 1, &b->exec_one);
    if (st != LE_OK) return st;
  }
  if (!b->exec_chunk) {
    le_status st = batch_capture(b, kChunk, &b->exec_chunk);
    if (st != LE_OK) return st;
  }
  int64_t left = nsteps;
  cudaError_t ce = cudaSuccess;
  while (ce == cudaSuccess && left >= kChunk) {
    ce = cudaGraphLaunch(b->exec_chunk, b->stream);
    left -= kChunk;
  }
  while (ce == cudaSuccess && left > 0) {
    ce = cudaGraphLaunch(b->exec_one, b->stream);
    --left;
  }
  for (le_sim *s : b->members) launch_fold(s->s, b->stream);
  if (ce == cudaSuccess) ce = cudaGetLastError();
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(b->stream);
  if (ce != cudaSuccess) return bfail(b, LE_ERR_CUDA, cudaGetErrorString(ce));
  return LE_OK;
}

}  // namespace

extern "C" {

LE_API le_status le_estimate_device_bytes(const double box[3], double shear_rate, double rc,
                                          double skin, const le_params *p, int64_t n,
                                          int64_t nbonds, size_t *bytes) {
  if (!box || !p || !bytes || n < 1 || n > kMaxParticles || nbonds < 0) return LE_ERR_INVALID_ARG;
  for (int a = 0; a < 3; ++a)
    if (!(box[a] > 0.0) || !((rc + skin) < 0.5 * box[a])) return LE_ERR_INVALID_ARG;
  le_sim *s = new (std::nothrow) le_sim;
  if (!s) return LE_ERR_OOM;
  fill_geom(s, box, shear_rate, rc, skin, p);
  if (nbonds > 0) s->bonds.assign(2, 0);  // only "bonds exist" matters for the cell edge
  Geom &g = s->s.g;
  g.maxb = nbonds > 0 ? 2 : 0;
  choose_cells(s);
  const double V = g.L[0] * g.L[1] * g.L[2];
  const double mean_nb = 4.18879020478639 * g.rl * g.rl * g.rl * (double)n / V;
  const int maxnb = (int)std::ceil(mean_nb * 1.6) + 32;
  s->dry_run = true;
  le_status st = allocate(s, n, maxnb);
  // the rollback snapshot holds one more buffer set
  const size_t vb = vec_bytes(s->s.prec);
  const size_t snap = (size_t)n * (4 * vb + (s->s.prec == 1 ? 16 : 0) + 16 + 4) + sizeof(Dyn);
  *bytes = s->device_bytes + snap;
  s->dry_run = false;
  delete s;
  return st;
}

LE_API le_status le_batch_create(size_t budget_bytes, void *cuda_stream, le_batch **out) {
  if (!out) return LE_ERR_INVALID_ARG;
  *out = nullptr;
  le_batch *b = new (std::nothrow) le_batch;
  if (!b) return LE_ERR_OOM;
  b->budget = budget_bytes;
  cudaError_t e = cudaSuccess;
  if (cuda_stream) {
    b->stream = (cudaStream_t)cuda_stream;
  } else {
    e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    b->own_stream = true;
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    le_batch_destroy(b);
    return LE_ERR_CUDA;
  }
  *out = b;
  return LE_OK;
}

LE_API le_status le_batch_add(le_batch *b, le_sim *s) {
  if (!b || !s) return LE_ERR_INVALID_ARG;
  if (!s->has_particles) return bfail(b, LE_ERR_STATE, "a member needs its particles first");
  size_t used = 0;
  for (le_sim *m : b->members) {
    if (m == s) return bfail(b, LE_ERR_INVALID_ARG, "already a member");
    used += m->device_bytes;
  }
  if (b->budget && used + s->device_bytes > b->budget)
    return bfail(b, LE_ERR_OOM, "the batch memory budget is full");
  b->members.push_back(s);
  batch_drop_graphs(b);
  return LE_OK;
}

LE_API le_status le_batch_remove(le_batch *b, le_sim *s) {
  if (!b || !s) return LE_ERR_INVALID_ARG;
  for (size_t k = 0; k < b->members.size(); ++k)
    if (b->members[k] == s) {
      b->members.erase(b->members.begin() + (long)k);
      batch_drop_graphs(b);
      return LE_OK;
    }
  return bfail(b, LE_ERR_INVALID_ARG, "not a member");
}

LE_API le_status le_batch_step(le_batch *b, int64_t nsteps) {
  if (!b || nsteps < 0) return LE_ERR_INVALID_ARG;
  if (nsteps == 0 || b->members.empty()) return LE_OK;
  for (int attempt = 0; attempt < 4; ++attempt) {
    std::vector<int> cur0(b->members.size());
    for (size_t k = 0; k < b->members.size(); ++k) {
      le_sim *s = b->members[k];
      le_status st = read_dyn(s);
      if (st == LE_OK) st = take_snapshot(s);
      if (st == LE_OK) st = sync(s);
      if (st != LE_OK) return bfail(b, st, s->err);
      cur0[k] = s->h_dyn->cur;
    }
    le_status st = batch_run(b, nsteps);
    if (st != LE_OK) return st;
    bool failed = false, grow = false;
    le_status first = LE_OK;
    std::string msg;
    for (le_sim *s : b->members) {
      st = read_dyn(s);
      if (st != LE_OK) return bfail(b, st, s->err);
      if (s->h_dyn->err) {
        failed = true;
        le_status e = status_from_err(s, s->h_dyn->err);
        if (e == LE_ERR_CAPACITY) grow = true;
        else if (first == LE_OK) {
          first = e;
          msg = s->err;
        }
      }
    }
    if (!failed) return LE_OK;
    // roll every member back to the start of the call
    std::vector<int> seen(b->members.size());
    for (size_t k = 0; k < b->members.size(); ++k) seen[k] = b->members[k]->h_dyn->list_max;
    for (size_t k = 0; k < b->members.size(); ++k) {
      st = restore_snapshot(b->members[k], cur0[k]);
      if (st != LE_OK) return bfail(b, st, b->members[k]->err);
    }
    if (first != LE_OK) return bfail(b, first, msg + " (all members rolled back)");
    if (!grow) break;
    for (size_t k = 0; k < b->members.size(); ++k) {
      le_sim *s = b->members[k];
      if (seen[k] > s->s.g.maxnb) {
        st = grow_list(s, (int)std::ceil(seen[k] * 1.3) + 16);
        if (st != LE_OK) return bfail(b, st, s->err);
      }
    }
    batch_drop_graphs(b);
  }
  return bfail(b, LE_ERR_CAPACITY, "neighbour list capacity could not be grown enough");
}

LE_API le_status le_batch_tune(le_batch *b, int steps_per_trial, int *best_force, int *best_list,
                               double *ms_per_step) {
  if (!b || steps_per_trial < 1) return LE_ERR_INVALID_ARG;
  if (b->members.empty()) return LE_OK;
  const int chunks = std::max(1, steps_per_trial / kChunk);
  std::vector<int> cur0(b->members.size());
  for (size_t k = 0; k < b->members.size(); ++k) {
    le_sim *s = b->members[k];
    le_status st = read_dyn(s);
    if (st == LE_OK) st = take_snapshot(s);
    if (st == LE_OK) st = sync(s);
    if (st != LE_OK) return bfail(b, st, s->err);
    cur0[k] = s->h_dyn->cur;
  }
  auto restore_all = [&]() -> le_status {
    for (size_t k = 0; k < b->members.size(); ++k) {
      le_status st = restore_snapshot(b->members[k], cur0[k]);
      if (st != LE_OK) return bfail(b, st, b->members[k]->err);
    }
    return LE_OK;
  };
  auto apply = [&](int f, int l) {
    for (le_sim *s : b->members) {
      s->s.force_threads = f;
      s->s.list_threads = l;
      drop_graphs(s);
    }
    batch_drop_graphs(b);
  };
  const int forces[2] = {128, 256}, lists[3] = {64, 128, 256};
  int bf = b->members[0]->s.force_threads, bl = b->members[0]->s.list_threads;
  double best = 0.0;
  for (int a = 0; a < 2; ++a)
    for (int c = 0; c < 3; ++c) {
      apply(forces[a], lists[c]);
      le_status st = batch_run(b, kChunk);  // captures and warms
      std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
      if (st == LE_OK) st = batch_run(b, (int64_t)chunks * kChunk);
      const double secs =
          std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      bool failed = st != LE_OK;
      for (le_sim *s : b->members) {
        if (read_dyn(s) != LE_OK || s->h_dyn->err) failed = true;
      }
      le_status rs = restore_all();
      if (rs != LE_OK) return rs;
      if (failed) {
        apply(bf, bl);
        return bfail(b, LE_ERR_CAPACITY, "a tuning trial failed (all members rolled back)");
      }
      const double per = secs * 1e3 / (double)(chunks * kChunk);
      if (best == 0.0 || per < best) {
        best = per;
        bf = forces[a];
        bl = lists[c];
      }
    }
  apply(bf, bl);
  // the step graphs of the chosen shape, so the next step does not pay for them
  le_status st = batch_capture(b, 1, &b->exec_one);
  if (st == LE_OK) st = batch_capture(b, kChunk, &b->exec_chunk);
  if (st != LE_OK) return st;
  if (best_force) *best_force = bf;
  if (best_list) *best_list = bl;
  if (ms_per_step) *ms_per_step = best;
  return LE_OK;
}

LE_API le_status le_batch_destroy(le_batch *b) {
  if (!b) return LE_ERR_INVALID_ARG;
  if (b->stream) cudaStreamSynchronize(b->stream);
  batch_drop_graphs(b);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
  return LE_OK;
}

LE_API const char *le_batch_last_error(const le_batch *b) { return b ? b->err.c_str() : "null batch"; }

}  // extern "C"
