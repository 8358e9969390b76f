// C ABI (include/rhif.h): factorization driver, application, PCG.
//
// The factorization runs level by level (Sec. 3.1 / 3.2).  The host plans a
// level (plan.cpp), uploads its index tables in one copy, launches the batched
// kernels of the level on the caller's stream, then reads back the skeleton
// ranks and pivot orders (the only data-dependent sizes) to plan the next
// level.  The root front A_L (Eq. 3.3) is level L of the same machinery.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdlib>
#include <cmath>
#include <cstdio>
#include <climits>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/rhif.h"
#include "host_pool.h"
#include "kernels.h"
#include "plan.h"
#include "tables.h"

namespace rhif {

thread_local std::string g_detail;

void set_error_detail(const std::string& msg) { g_detail = msg; }

static int fail(int code, const std::string& msg) {
  g_detail = msg;
  return code;
}

#define CK(call)                                                                        \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) {                                                            \
      return fail(e_ == cudaErrorMemoryAllocation ? RHIF_ERR_OOM : RHIF_ERR_CUDA,       \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                  \
    }                                                                                   \
  } while (0)

// Device allocation, stream-ordered; every pointer is released by the handle.
struct DevMem {
  std::vector<void*> ptrs;
  cudaStream_t s = nullptr;
  size_t bytes = 0;
  int get(void** p, size_t n) {
    *p = nullptr;
    if (n == 0) n = 16;
    cudaError_t e = cudaMallocAsync(p, n, s);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(RHIF_ERR_OOM, "device allocation of " + std::to_string(n) + " bytes failed");
    }
    ptrs.push_back(*p);
    bytes += n;
    return RHIF_OK;
  }
  void release(void* p) {
    for (auto& q : ptrs)
      if (q == p) {
        cudaFreeAsync(q, s);
        q = nullptr;
      }
  }
  void release_all() {
    for (void* p : ptrs)
      if (p) cudaFreeAsync(p, s);
    ptrs.clear();
  }
};

// Packs host vectors into one staging buffer and uploads it in one copy.
// Host tables bound for one device buffer: `add` records a vector and returns
// its 16-byte-aligned offset; `upload` packs them into pinned staging memory
// and queues one host-to-device copy.  The staging buffer belongs to the
// calling thread and is reused by later uploads once the copy that last read
// it has completed (an event recorded behind it), so repeated
// factorizations neither allocate pinned memory nor copy from pageable memory.
struct Packer {
  std::vector<std::pair<const void*, size_t>> part;
  std::vector<size_t> off;
  size_t total = 0;
  template <typename V>
  size_t add(const std::vector<V>& v) {
    const size_t o = (total + 15) & ~size_t(15);
    part.emplace_back(v.data(), v.size() * sizeof(V));
    off.push_back(o);
    total = o + v.size() * sizeof(V);
    return o;
  }
  int upload(void* dst, cudaStream_t s) const;
};

struct Staging {
  char* p = nullptr;
  size_t cap = 0;
  cudaEvent_t done = nullptr;
  int device = -1;
};
static thread_local Staging t_stage;

int Packer::upload(void* dst, cudaStream_t s) const {
  if (!total) return 0;
  Staging& st = t_stage;
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (st.done) CK(cudaEventSynchronize(st.done));   // the previous copy out of the buffer
  if (st.done && st.device != dev) {
    CK(cudaEventDestroy(st.done));
    st.done = nullptr;
  }
  if (!st.done) {
    CK(cudaEventCreateWithFlags(&st.done, cudaEventDisableTiming));
    st.device = dev;
  }
  if (st.cap < total) {
    if (st.p) CK(cudaFreeHost(st.p));
    st.p = nullptr;
    st.cap = 0;
    const size_t cap = std::max(total + total / 2, size_t(1) << 20);
    CK(cudaHostAlloc((void**)&st.p, cap, cudaHostAllocPortable));
    st.cap = cap;
  }
  // large tables (the level-0 DOF list is 4 bytes per DOF) are copied into
  // the staging buffer in 256 KB chunks by the planner's host threads
  constexpr size_t kChunk = size_t(256) << 10;
  std::vector<std::pair<size_t, size_t>> big;   // (part, chunk)
  for (size_t i = 0; i < part.size(); ++i) {
    if (part[i].second >= 2 * kChunk) {
      for (size_t c = 0; c * kChunk < part[i].second; ++c) big.emplace_back(i, c);
    } else if (part[i].second) {
      std::memcpy(st.p + off[i], part[i].first, part[i].second);
    }
  }
  if (!big.empty())
    HostPool::get().parallel_for((int64_t)big.size(), 1, [&](int64_t b0, int64_t b1) {
      for (int64_t b = b0; b < b1; ++b) {
        const size_t i = big[b].first, o = big[b].second * kChunk;
        const size_t len = std::min(kChunk, part[i].second - o);
        std::memcpy(st.p + off[i] + o, (const char*)part[i].first + o, len);
      }
    });
  CK(cudaMemcpyAsync(dst, st.p, total, cudaMemcpyHostToDevice, s));
  CK(cudaEventRecord(st.done, s));
  return 0;
}


// ---------------------------------------------------------------------------
// kernel instrumentation: launch counters per category, optional CUDA-event timing
// ---------------------------------------------------------------------------
enum Cat {
  kCatStencil, kCatLeafElim, kCatExpandGids, kCatExtendAdd, kCatPartialChol, kCatPrecondDiag, kCatPrecondScale,
  kCatSkel, kCatApplyCellUp, kCatApplyCellDown, kCatApplyGroupUp, kCatApplyGroupDown, kCatSpmv,
  kCatVector, kCatAssemble, kCatGrad, kCatApplyLeafUp, kCatApplyLeafDown, kCatBandInverse,
  kCatLeafCond, kCatLeafFp64, kNumCat
};
static const char* kCatName[kNumCat] = {
    "stencil_from_csr", "leaf_elim", "expand_gids", "extend_add", "partial_chol", "precond_diag",
    "precond_scale", "skel", "apply_cell_up", "apply_cell_down", "apply_group_up",
    "apply_group_down", "spmv", "pcg_vector", "assemble_fd", "grad_logcoef", "apply_leaf_up",
    "apply_leaf_down", "band_inverse", "leaf_cond", "leaf_fp64"};
struct KStat {
  int64_t launches = 0;
  double ms = 0, flops = 0, bytes = 0;
};
static KStat g_kstat[kNumCat];
static bool g_timing = false;
static std::mutex g_kmu;
struct Pending {
  int cat;
  cudaEvent_t a, b;
};
static std::vector<Pending> g_pending;
static std::vector<cudaEvent_t> g_event_pool;

static cudaEvent_t pooled_event() {
  if (!g_event_pool.empty()) {
    cudaEvent_t e = g_event_pool.back();
    g_event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// While this thread captures a CUDA graph, launches are counted here instead
// (nothing runs during a capture; the graph's replays are credited instead).
static thread_local KStat* t_capture_stats = nullptr;

// Counts (and, with timing on, brackets with events) the launches issued while alive.
struct Launch {
  int cat;
  cudaStream_t s;
  cudaEvent_t a = nullptr, b = nullptr;
  Launch(int cat_, cudaStream_t s_, double flops, double bytes, int count = 1) : cat(cat_), s(s_) {
    if (t_capture_stats) {
      t_capture_stats[cat].launches += count;
      t_capture_stats[cat].flops += flops;
      t_capture_stats[cat].bytes += bytes;
      return;
    }
    std::lock_guard<std::mutex> lk(g_kmu);
    g_kstat[cat].launches += count;
    g_kstat[cat].flops += flops;
    g_kstat[cat].bytes += bytes;
    if (g_timing) {
      a = pooled_event();
      b = pooled_event();
      cudaEventRecord(a, s);
    }
  }
  ~Launch() {
    if (a) {
      cudaEventRecord(b, s);
      std::lock_guard<std::mutex> lk(g_kmu);
      g_pending.push_back({cat, a, b});
    }
  }
};

// Fronts at least this large, at levels with at most this many cells, are
// eliminated by many CTAs per front.
constexpr int kBigFront = 384;
constexpr int kBigFrontCells = 304;
constexpr int kNumSMsHint = 152;   // CTAs wanted per cluster launch (one per SM)

static void add_launches(int cat, int64_t n) {
  if (t_capture_stats) {
    t_capture_stats[cat].launches += n;
    return;
  }
  std::lock_guard<std::mutex> lk(g_kmu);
  g_kstat[cat].launches += n;
}

static void add_work(int cat, double flops, double bytes) {
  if (t_capture_stats) {
    t_capture_stats[cat].flops += flops;
    t_capture_stats[cat].bytes += bytes;
    return;
  }
  std::lock_guard<std::mutex> lk(g_kmu);
  g_kstat[cat].flops += flops;
  g_kstat[cat].bytes += bytes;
}

struct PhaseStore {
  PhaseDev dev{};
  std::vector<int> h_rank, h_perm;
};

// The level-0 plan of a single problem depends on the grid, the leaf size
// and the options only (the leaves and the level-0 separators are fixed by
// the geometry, Sec. 3.1): the last one built is kept with a device copy of
// its tables and shared, read-only, by later factorizations of the same kind.
struct Plan0 {
  LevelPlan plan;
  void* tables = nullptr;   // upload_level's layout of the plan's tables
  ~Plan0() {
    if (tables) cudaFree(tables);
  }
};

struct LevelStore {
  LevelPlan own;                       // this factorization's plan of the level
  std::shared_ptr<const Plan0> p0;     // or the shared level-0 plan
  const LevelPlan& plan() const { return p0 ? p0->plan : own; }
  LevelDev dev{};
  std::vector<PhaseStore> phases;
  void* tables = nullptr;
  // algorithmic work of one sweep direction of the application, per right-hand side
  double cell_flops = 0, cell_bytes = 0;
  std::vector<double> grp_flops, grp_bytes;   // per phase
  bool big_apply = false;   // eliminated with the many-CTA schedule: many-CTA cell sweeps
};

}  // namespace rhif

struct rhif_handle {
  rhif::Geometry G;
  rhif::GeoDev gd{};
  int precision = RHIF_FP64;
  bool precondition = true, edge_skel = false;
  bool precond_diag = false;   // diagonal local preconditioner in place of block Cholesky
  double leaf_fp64 = 0.0;      // FP32 factors: FP64 re-elimination of leaves above this condition (0 = never)
  int fp64_leaves = -1;        // leaves re-eliminated in FP64 (read back on request)
  int big_front = 0, big_frame = 0;   // many-CTA thresholds (see rhif_opts)
  int skel_cluster = 0;
  bool skel_warp = true;   // small units: one warp each
  bool tensor_cores = true;   // FP32 Schur complements of large fronts on tcgen05
  double tol = 0.0;
  std::vector<rhif::LevelStore> levels;   // 0..L
  double* diag = nullptr;
  double* off = nullptr;
  int* status = nullptr;
  rhif::DevMem mem;
  // reusable work space
  double* ubuf = nullptr;
  int64_t ubuf_elems = 0;
  int64_t ub_len = 0;   // scratch column: max over levels of sum nB, then the interior part
  int64_t ui_len = 0;   // max DOF-list length of the levels with big_apply
  int64_t ui_base = 0;  // offset of the interior part in the scratch column
  std::vector<int64_t> xoff_host;   // per-cell offsets of the L^{-1} scratch (upload source)
  double* work = nullptr;
  int64_t work_elems = 0;
  double* mv_work = nullptr;   // work space of y = F x (rhif_apply with RHIF_MATVEC)
  int64_t mv_elems = 0;
  int mv_iters = 0;            // CG iterations of the last y = F x
  double flops = 0.0, apply_bytes = 0.0, factor_ms = 0.0;
  int units = 0;
  // Merged batch (rhif_factor_batch): the problems' grids and first DOFs in
  // the concatenated numbering, their stencil views on the device, and per
  // level the bases of the problems' parts in the merged plan (empty for a
  // single problem).
  std::vector<rhif::Geometry> pG;
  std::vector<int64_t> pbase;
  rhif::BatchGeo* bgeo = nullptr;
  std::vector<std::vector<rhif::PartBase>> part_bases;
  std::vector<std::vector<int>> part_prob;
  rhif::VecSeg vseg{};   // PCG vector blocks of the batch (tables on the device, built on first use)
  // One F^{-1} application (the sweeps of apply_impl) as a CUDA graph, captured
  // for one (output, leading dimension, nrhs, scratch) and replayed by PCG;
  // the launch counts of one application are credited at every replay.
  cudaGraphExec_t apply_graph = nullptr;
  cudaStream_t capture_stream = nullptr;
  double* ag_y = nullptr;
  double* ag_ubuf = nullptr;
  int64_t ag_ldy = 0;
  int ag_nrhs = 0;
  int64_t ag_launches[rhif::kNumCat] = {};
  double ag_flops[rhif::kNumCat] = {}, ag_bytes[rhif::kNumCat] = {};
  // The iterations of rhif_pcg as one CUDA graph (iteration 1, then a
  // conditional WHILE node over the others), for one (solution, work
  // buffers, scratch, nrhs, rtol, maxit); the launch counts of the part
  // before the loop and of one loop body, credited per run.
  cudaGraphExec_t pcg_graph = nullptr;
  const void* pg_u = nullptr;
  const void* pg_work = nullptr;
  const void* pg_ubuf = nullptr;
  int64_t pg_ldu = 0;
  int pg_nrhs = 0, pg_maxit = 0;
  double pg_rtol = 0.0;
  rhif::KStat pg_pre[rhif::kNumCat] = {}, pg_body[rhif::kNumCat] = {};
};

namespace rhif {

static GeoDev geo_dev(const Geometry& G) {
  GeoDev g{};
  g.d = G.d;
  g.leaf = G.leaf;
  for (int a = 0; a < 3; ++a) {
    g.ns[a] = G.ns[a];
    g.stride[a] = G.stride[a];
  }
  g.N = G.N;
  return g;
}

template <typename T>
static int configure_once() {
  static int done = 0;
  static int rc = 0;
  if (!done) {
    rc = configure_factor_kernels<T>();
    if (rc == 0) rc = configure_apply_kernels<T>();
    if (rc == 0) rc = configure_tc_kernels();
    // keep freed factor memory in this process's stream-ordered pool between factorizations
    int dev = 0;
    cudaMemPool_t pool;
    if (rc == 0 && cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t thr = ~0ull;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    done = 1;
  }
  return rc;
}

// Upload the index tables of a level and fill the device views.
// Offsets of a plan's tables in one device buffer (upload_level's layout).
struct TableLayout {
  size_t bucket, code, cstart, nI, nB, goff, boff, foff, froff, frld, bw, boff2, zoff, soff, sg,
      sp, gt, gs, gsz, gco, gc, gp, eao, eac, eamo, eam, cprob;
  struct PhOff {
    size_t pg, po, gp, ug, un, umo, uro, upo, gu;
  };
  std::vector<PhOff> po;
};

static TableLayout table_layout(const LevelPlan& P, Packer& pk) {
  TableLayout t;
  t.bucket = pk.add(P.bucket);
  t.code = pk.add(P.cell_code);
  t.cstart = pk.add(P.cell_start);
  t.nI = pk.add(P.nI);
  t.nB = pk.add(P.nB);
  t.goff = pk.add(P.gid_off);
  t.boff = pk.add(P.b_off);
  t.foff = pk.add(P.front_off);
  t.froff = pk.add(P.frame_off);
  t.frld = pk.add(P.frame_ld);
  t.bw = pk.add(P.band_w);
  t.boff2 = pk.add(P.band_off);
  t.zoff = pk.add(P.z_off);
  t.soff = pk.add(P.seg_off);
  t.sg = pk.add(P.seg_group);
  t.sp = pk.add(P.seg_pos);
  t.gt = pk.add(P.group_t);
  t.gs = pk.add(P.group_start);
  t.gsz = pk.add(P.group_size);
  t.gco = pk.add(P.group_cell_off);
  t.gc = pk.add(P.group_cell);
  t.gp = pk.add(P.group_pos);
  t.eao = pk.add(P.ea_off);
  t.eac = pk.add(P.ea_child);
  t.eamo = pk.add(P.ea_map_off);
  t.eam = pk.add(P.ea_map);
  t.cprob = pk.add(P.cell_prob);
  t.po.resize(P.phases.size());
  for (size_t i = 0; i < P.phases.size(); ++i) {
    const PhasePlan& ph = P.phases[i];
    const UnitTable& U = ph.units;
    t.po[i] = {pk.add(ph.pre_group), pk.add(ph.pre_off), pk.add(ph.group_pre), pk.add(U.group),
               pk.add(U.nrow), pk.add(U.m_off), pk.add(U.rec_off), pk.add(U.perm_off),
               pk.add(ph.group_unit)};
  }
  return t;
}

static int upload_level(rhif_handle* H, LevelStore& S, size_t elem) {
  const LevelPlan& P = S.plan();
  Packer pk;
  const TableLayout t = table_layout(P, pk);
  void* d = nullptr;
  int rc = RHIF_OK;
  if (S.p0) {   // the shared level-0 tables, already on the device
    d = S.p0->tables;
  } else {
    if ((rc = H->mem.get(&d, pk.total))) return rc;
    S.tables = d;
    if ((rc = pk.upload(d, H->mem.s))) return rc;
  }
  char* b = (char*)d;
  LevelDev& L = S.dev;
  L.level = P.level;
  L.ncell = P.ncell();
  L.ngroup = P.ngroup();
  L.width = P.width;
  L.code_base = P.code_base;
  L.max_nI = P.max_nI;
  L.max_nB = P.max_nB;
  L.max_n = P.max_n;
  L.max_group = P.max_group;
  L.max_w = P.max_w;
  L.bucket = (const int32_t*)(b + t.bucket);
  L.cell_code = (const int64_t*)(b + t.code);
  L.cell_start = (const int32_t*)(b + t.cstart);
  L.nI = (const int*)(b + t.nI);
  L.nB = (const int*)(b + t.nB);
  L.gid_off = (const int64_t*)(b + t.goff);
  L.b_off = (const int64_t*)(b + t.boff);
  L.front_off = (const int64_t*)(b + t.foff);
  L.frame_off = (const int64_t*)(b + t.froff);
  L.frame_ld = (const int*)(b + t.frld);
  L.band_w = (const int*)(b + t.bw);
  L.band_off = (const int64_t*)(b + t.boff2);
  L.z_off = (const int64_t*)(b + t.zoff);
  L.seg_off = (const int*)(b + t.soff);
  L.seg_group = (const int*)(b + t.sg);
  L.seg_pos = (const int*)(b + t.sp);
  L.group_t = (const int*)(b + t.gt);
  L.group_start = (const int32_t*)(b + t.gs);
  L.group_size = (const int*)(b + t.gsz);
  L.group_cell_off = (const int*)(b + t.gco);
  L.group_cell = (const int*)(b + t.gc);
  L.group_pos = (const int*)(b + t.gp);
  L.ea_off = (const int*)(b + t.eao);
  L.ea_child = (const int*)(b + t.eac);
  L.ea_map_off = (const int64_t*)(b + t.eamo);
  L.ea_map = (const int*)(b + t.eam);
  L.status = H->status;
  L.cell_prob = P.cell_prob.empty() ? nullptr : (const int*)(b + t.cprob);
  L.bgeo = P.cell_prob.empty() ? nullptr : H->bgeo;
  if ((rc = H->mem.get((void**)&L.gids, P.gid_off.back() * sizeof(int32_t)))) return rc;
  if (P.level == 0) {
    if ((rc = H->mem.get(&L.frame_base, P.frame_total * elem))) return rc;
    if ((rc = H->mem.get(&L.band, P.band_total * elem))) return rc;
    if ((rc = H->mem.get((void**)&L.cpl_i, P.b_off.back() * sizeof(int)))) return rc;
    if ((rc = H->mem.get(&L.cpl_a, P.b_off.back() * elem))) return rc;
    L.front = nullptr;
  } else {
    if ((rc = H->mem.get(&L.front, P.front_total * elem))) return rc;
    L.frame_base = L.front;
  }
  S.phases.resize(P.phases.size());
  for (size_t i = 0; i < P.phases.size(); ++i) {
    const PhasePlan& ph = P.phases[i];
    const UnitTable& U = ph.units;
    PhaseDev& D = S.phases[i].dev;
    D.unit_type = ph.unit_type;
    D.pre_min_type = ph.pre_min_type;
    D.npre = (int)ph.pre_group.size();
    D.diag_only = H->precond_diag ? 1 : 0;
    D.pre_group = (const int*)(b + t.po[i].pg);
    D.pre_off = (const int64_t*)(b + t.po[i].po);
    D.group_pre = (const int*)(b + t.po[i].gp);
    D.nunit = (int)U.group.size();
    D.max_n = U.max_n;
    D.u_group = (const int*)(b + t.po[i].ug);
    D.u_nrow = (const int*)(b + t.po[i].un);
    D.u_m_off = (const int64_t*)(b + t.po[i].umo);
    D.u_rec_off = (const int64_t*)(b + t.po[i].uro);
    D.u_perm_off = (const int64_t*)(b + t.po[i].upo);
    D.group_unit = (const int*)(b + t.po[i].gu);
    if ((rc = H->mem.get(&D.Lbuf, ph.pre_total * elem))) return rc;
    if ((rc = H->mem.get(&D.rec, U.rec_total * elem))) return rc;
    if ((rc = H->mem.get((void**)&D.perm, U.perm_total * sizeof(int)))) return rc;
    if ((rc = H->mem.get((void**)&D.rank, U.group.size() * sizeof(int)))) return rc;
    D.Mbuf = nullptr;
  }
  return RHIF_OK;
}

static int status_message(const int* st, const char* where);

static int check_status(rhif_handle* H, const char* where) {
  int st[4] = {0, 0, 0, 0};
  CK(cudaMemcpyAsync(st, H->status, sizeof(st), cudaMemcpyDeviceToHost, H->mem.s));
  CK(cudaStreamSynchronize(H->mem.s));
  CK(cudaGetLastError());
  return status_message(st, where);
}

// Pinned host memory of the calling thread for the small per-phase readbacks
// (status words, ranks, pivot orders), grown as needed; the caller
// synchronizes the stream before reading it and before the next use.
static thread_local int* t_rb = nullptr;
static thread_local size_t t_rb_cap = 0;

static int readback_buffer(size_t ints, int** out) {
  if (t_rb_cap < ints) {
    if (t_rb) CK(cudaFreeHost(t_rb));
    t_rb = nullptr;
    t_rb_cap = 0;
    const size_t cap = std::max(ints + ints / 2, size_t(1) << 16);
    CK(cudaHostAlloc((void**)&t_rb, cap * sizeof(int), cudaHostAllocPortable));
    t_rb_cap = cap;
  }
  *out = t_rb;
  return RHIF_OK;
}

static int status_message(const int* st, const char* where) {
  if (st[0] == 0) return RHIF_OK;
  static const char* kinds[] = {"?", "cell", "group", "unit", "root", "argument"};
  char buf[256];
  const int kind = (st[2] >= 0 && st[2] <= 5) ? st[2] : 0;
  std::snprintf(buf, sizeof(buf), "%s: %s at level %d, %s %d", where,
                st[0] == RHIF_ERR_NOT_SPD ? "non-positive pivot (not SPD)" : "invalid input",
                st[1], kinds[kind], st[3]);
  return fail(st[0], buf);
}

static double cell_flops(double nI, double nB) {
  return nI * nI * nI / 3.0 + nI * nI * nB + nI * nB * nB;
}

// Skeletonization of one phase: one CTA per unit while every unit's ID matrix
// fits in shared memory, else one thread-block cluster per unit.  The cluster
// size is the smallest power of two whose row slices fit in shared memory,
// raised until the launch has at least one CTA per SM, capped at 16 and at
// what the device can schedule.
template <typename T>
static int skeletonize(rhif_handle* H, const LevelPlan& P, const PhasePlan& ph, const LevelDev& L,
                       const PhaseDev& D, uint8_t* alive, cudaStream_t s) {
  const int64_t nunit = (int64_t)ph.units.group.size();
  if (!nunit) return RHIF_OK;
  const size_t elem = sizeof(T);
  const size_t budget = 216 * 1024;
  const bool fits1 = skel_smem_bytes<T>(ph.units.max_n) + ph.units.max_m * elem <= 200 * 1024;
  if (H->skel_cluster == 0 && H->skel_warp &&
      launch_skel_warp<T>(L, D, alive, H->tol, H->status, ph.units.max_m, s)) {
    CK(cudaGetLastError());
    return RHIF_OK;
  }
  if (H->skel_cluster < 0 || (H->skel_cluster == 0 && fits1)) {
    launch_skel<T>(L, D, alive, H->tol, H->status, ph.units.max_m, s);
    CK(cudaGetLastError());
    return RHIF_OK;
  }
  auto fixed = [&](int C) { return skel_cluster_fixed_bytes<T>(ph.units.max_n, C); };
  auto max_slice = [&](int C) {
    int64_t m = 0;
    for (int64_t u = 0; u < nunit; ++u) {
      const int64_t n = P.group_size[ph.units.group[u]];
      const int64_t sr = (ph.units.nrow[u] + C - 1) / C;
      m = std::max(m, sr * n);
    }
    return m;
  };
  int C = H->skel_cluster;
  if (C == 0) {
    int cfit = 16;
    for (int c = 2; c <= 16; c *= 2)
      if (fixed(c) + max_slice(c) * elem <= budget) {
        cfit = c;
        break;
      }
    int cfill = 1;
    while (cfill < 16 && nunit * cfill < kNumSMsHint) cfill *= 2;
    C = std::max(cfit, cfill);
  }
  for (;;) {
    const size_t fx = fixed(C);
    if (fx <= budget) {
      const int64_t ms = max_slice(C);
      const int64_t cap = fx + ms * elem <= budget ? ms : (int64_t)((budget - fx) / elem);
      const size_t smem = fx + (size_t)cap * elem;
      if (C == 1 || skel_cluster_schedulable<T>(C, smem) > 0) {
        CK(launch_skel_cluster<T>(L, D, alive, H->tol, H->status, C, cap, smem, s));
        return RHIF_OK;
      }
    }
    if (C == 1) {   // no room for the cluster tables: one CTA per unit, M in global memory
      launch_skel<T>(L, D, alive, H->tol, H->status, ph.units.max_m, s);
      CK(cudaGetLastError());
      return RHIF_OK;
    }
    C /= 2;
  }
}

// Plan of level `lvl` (Sec. 3.1 grouping).  A single problem: its level plan
// from the previous one and the survivor flags.  A merged batch: the plan of
// every problem that still has this level (its own previous plan and its
// slice of the flags), concatenated by merge_plans; `pprev` holds the
// problems' own plans of the previous level and receives those of this one.
static LevelPlan plan_level(rhif_handle* H, int lvl, const std::vector<uint8_t>& keep,
                            std::vector<LevelPlan>& pprev) {
  if (H->pG.empty())
    return build_level(H->G, lvl, keep, lvl ? &H->levels[lvl - 1].plan() : nullptr, H->precondition,
                       H->edge_skel);
  const int np = (int)H->pG.size();
  std::vector<LevelPlan> cur(np);
  std::vector<const LevelPlan*> parts;
  std::vector<int> prob, prev_cell, prev_part;
  std::vector<int64_t> base;
  int j = 0;   // part of problem p in the previous level
  for (int p = 0; p < np; ++p) {
    if (lvl > H->pG[p].L) continue;
    int pc = 0, pj = -1;
    if (lvl) {
      const std::vector<int>& pr = H->part_prob[lvl - 1];
      while (j < (int)pr.size() && pr[j] < p) ++j;
      pj = j;
      pc = H->part_bases[lvl - 1][j].cell;
    }
    parts.push_back(&cur[p]);
    prob.push_back(p);
    prev_cell.push_back(pc);
    prev_part.push_back(pj);
    base.push_back(H->pbase[p]);
  }
  // the problems' plans are independent: one per planner-pool thread (each
  // build_level then runs its own loops on its thread; the pool's threads
  // keep their planner storage between factorizations)
  HostPool::get().parallel_for((int64_t)prob.size(), 1, [&](int64_t q0, int64_t q1) {
    std::vector<uint8_t> kp;
    for (int64_t q = q0; q < q1; ++q) {
      const int p = prob[q];
      const LevelPlan* pp = nullptr;
      kp.clear();
      if (lvl) {
        const PartBase& B = H->part_bases[lvl - 1][prev_part[q]];
        pp = &pprev[p];
        kp.assign(keep.begin() + B.bucket, keep.begin() + B.bucket + pp->bucket.size());
      }
      cur[p] = build_level(H->pG[p], lvl, kp, pp, H->precondition, H->edge_skel);
    }
  });
  LevelPlan M;
  if ((int)H->part_bases.size() <= lvl) {
    H->part_bases.resize(lvl + 1);
    H->part_prob.resize(lvl + 1);
  }
  merge_plans(H->G.d, parts, prob, base, prev_cell, M, H->part_bases[lvl]);
  H->part_prob[lvl] = prob;
  pprev.swap(cur);
  return M;
}

// Level-0 plan of a single problem: the shared one when the last one built
// matches (device, grid, leaf size, local preconditioner, edge
// skeletonization), else a new one, uploaded once (synchronously, so that
// other streams may use it) and published for later factorizations.
struct Plan0Key {
  int device, d, ns[3], leaf, precondition, edge;
  bool operator==(const Plan0Key& o) const {
    return device == o.device && d == o.d && ns[0] == o.ns[0] && ns[1] == o.ns[1] &&
           ns[2] == o.ns[2] && leaf == o.leaf && precondition == o.precondition && edge == o.edge;
  }
};
static std::mutex g_p0_mu;
static Plan0Key g_p0_key{};
static std::shared_ptr<const Plan0>* g_p0 = new std::shared_ptr<const Plan0>();   // never destroyed

static int plan0_get(rhif_handle* H, LevelStore& S) {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  const Geometry& G = H->G;
  const Plan0Key key{dev, G.d, {G.ns[0], G.ns[1], G.ns[2]}, G.leaf,
                     H->precondition, H->edge_skel ? 1 : 0};
  {
    std::lock_guard<std::mutex> lk(g_p0_mu);
    if (*g_p0 && g_p0_key == key) {
      S.p0 = *g_p0;
      return RHIF_OK;
    }
  }
  auto e = std::make_shared<Plan0>();
  static const std::vector<uint8_t> none;
  e->plan = build_level(G, 0, none, nullptr, H->precondition, H->edge_skel);
  Packer pk;
  table_layout(e->plan, pk);
  CK(cudaMalloc(&e->tables, std::max<size_t>(pk.total, 16)));
  int rc = pk.upload(e->tables, H->mem.s);
  if (rc) return rc;
  CK(cudaStreamSynchronize(H->mem.s));
  {
    std::lock_guard<std::mutex> lk(g_p0_mu);
    *g_p0 = e;
    g_p0_key = key;
  }
  S.p0 = e;
  return RHIF_OK;
}

template <typename T>
static int factor_impl(rhif_handle* H, const rhif_csr* A) {
  const Geometry& G = H->G;
  cudaStream_t s = H->mem.s;
  const size_t elem = sizeof(T);
  int rc = configure_once<T>();
  if (rc) return fail(RHIF_ERR_CUDA, "cannot configure kernel shared memory");
  double* offb = nullptr;
  uint8_t* alive_d = nullptr;
  if ((rc = H->mem.get((void**)&H->diag, G.N * sizeof(double)))) return rc;
  if ((rc = H->mem.get((void**)&H->off, G.d * G.N * sizeof(double)))) return rc;
  if ((rc = H->mem.get((void**)&offb, G.d * G.N * sizeof(double)))) return rc;
  if ((rc = H->mem.get((void**)&H->status, 8 * sizeof(int)))) return rc;
  if ((rc = H->mem.get((void**)&alive_d, G.N))) return rc;
  CK(cudaMemsetAsync(H->off, 0, G.d * G.N * sizeof(double), s));
  CK(cudaMemsetAsync(offb, 0, G.d * G.N * sizeof(double), s));
  CK(cudaMemsetAsync(H->status, 0, 8 * sizeof(int), s));
  CK(cudaMemsetAsync(alive_d, 1, G.N, s));
  if (H->pG.empty()) {
    Launch t(kCatStencil, s, 0.0, double(A->nnz) * 12 + G.N * (8.0 + 24.0 * G.d), 2);
    launch_stencil_from_csr(H->gd, A->rowptr, A->col, A->val, A->nnz, H->diag, H->off, offb,
                            H->status, s);
  } else {   // merged batch: each problem's stencil in its own block of diag / off
    std::vector<BatchGeo> bg(H->pG.size());
    for (size_t p = 0; p < H->pG.size(); ++p) {
      const Geometry& Gp = H->pG[p];
      const int64_t b = H->pbase[p];
      bg[p] = BatchGeo{geo_dev(Gp), b, H->diag + b, H->off + G.d * b};
      Launch t(kCatStencil, s, 0.0, double(A[p].nnz) * 12 + Gp.N * (8.0 + 24.0 * G.d), 2);
      launch_stencil_from_csr(bg[p].G, A[p].rowptr, A[p].col, A[p].val, A[p].nnz, H->diag + b,
                              H->off + G.d * b, offb + G.d * b, H->status, s);
    }
    if ((rc = H->mem.get((void**)&H->bgeo, bg.size() * sizeof(BatchGeo)))) return rc;
    CK(cudaMemcpyAsync(H->bgeo, bg.data(), bg.size() * sizeof(BatchGeo), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));   // bg is a host local
  }

  // per position of the current level's bucket: the DOF survives into the
  // next level (only separator-group positions are read by the planner)
  static thread_local std::vector<uint8_t> keep;   // storage reused by later factorizations
  keep.clear();
  H->levels.resize(G.L + 1);
  const bool trace = std::getenv("RHIF_TRACE") != nullptr;
  using clk = std::chrono::steady_clock;
  auto ms_since = [](clk::time_point t) {
    return std::chrono::duration<double, std::milli>(clk::now() - t).count();
  };
  // The plan of level 0 depends on the grid only: it is built and its tables
  // queued for upload while the GPU converts the CSR matrix, before the
  // pattern check waits for that conversion.
  double t_plan = 0.0, t_up = 0.0;
  std::vector<LevelPlan> pprev;   // merged batch: the problems' own plans of the last level
  {
    auto t0 = clk::now();
    if (H->pG.empty()) {
      if ((rc = plan0_get(H, H->levels[0]))) return rc;
    } else {
      H->levels[0].own = plan_level(H, 0, keep, pprev);
    }
    t_plan = ms_since(t0);
    auto t1 = clk::now();
    if ((rc = upload_level(H, H->levels[0], elem))) return rc;
    t_up = ms_since(t1);
  }
  if ((rc = check_status(H, "CSR pattern check"))) return rc;
  H->mem.release(offb);

  for (int lvl = 0; lvl <= G.L; ++lvl) {
    LevelStore& S = H->levels[lvl];
    if (lvl) {
      auto t0 = clk::now();
      S.own = plan_level(H, lvl, keep, pprev);
      t_plan = ms_since(t0);
      auto t1 = clk::now();
      if ((rc = upload_level(H, S, elem))) return rc;
      t_up = ms_since(t1);
    }
    keep.assign(S.plan().bucket.size(), 1);
    auto t2 = clk::now();
    const LevelPlan& P = S.plan();
    H->ub_len = std::max<int64_t>(H->ub_len, P.b_off.back());
    {
      Launch t(kCatExpandGids, s, 0.0, 8.0 * P.gid_off.back());
      launch_expand_gids(S.dev, s);
    }
    double lvl_flops = 0.0;
    if (lvl == 0) {
      for (int c = 0; c < P.ncell(); ++c) {
        const double nI = P.nI[c], nB = P.nB[c], w = P.band_w[c];
        // banded Cholesky + L^{-1} A_IB (columns start at their coupled row) + Z^T Z
        lvl_flops += nI * w * w + nB * nI * w + nI * nB * nB;
        H->apply_bytes += 2.0 * elem * (nI * (w + 1) + nB);
      }
      if (leaf_elim_needs_z(H->gd, S.dev, elem)) {
        void* Zb = nullptr;
        if ((rc = H->mem.get(&Zb, P.z_total * elem))) return rc;
        S.dev.zbuf = Zb;
      }
      {
        Launch t(kCatLeafElim, s, lvl_flops, 0.0);
        launch_leaf_elim<T>(H->gd, S.dev, H->diag, H->off, H->status, s);
      }
      // precision pattern: leaves of an FP32 factor whose Jacobi-scaled
      // condition estimate exceeds the threshold are eliminated again in FP64
      // (their band, couplings and frame rounded to FP32) before any later
      // step reads them
      if (sizeof(T) == 4 && H->leaf_fp64 > 0.0 && P.max_nB <= 64) {
        int* list = nullptr;   // the flagged leaves; their count is status word 4
        if ((rc = H->mem.get((void**)&list, P.ncell() * sizeof(int)))) return rc;
        {
          Launch t(kCatLeafCond, s, 0.0, 0.0);
          launch_leaf_cond(H->gd, S.dev, H->diag, H->off, H->leaf_fp64, list, H->status + 4, s);
        }
        {
          Launch t(kCatLeafFp64, s, 0.0, 0.0);
          launch_leaf_fp64_redo(H->gd, S.dev, H->diag, H->off, H->status, list, H->status + 4, s);
        }
        H->mem.release(list);
      }
    } else {
      for (int c = 0; c < P.ncell(); ++c) {
        const double nI = P.nI[c], nB = P.nB[c];
        lvl_flops += cell_flops(nI, nB);
        H->apply_bytes += 2.0 * elem * (nI * (nI + 1) / 2 + nI * nB);
      }
      {
        Launch t(kCatExtendAdd, s, 0.0, double(P.front_total) * elem, 0);
        int slots = 0;
        for (int c = 0; c < P.ncell(); ++c) slots = std::max(slots, P.ea_off[c + 1] - P.ea_off[c]);
        add_launches(kCatExtendAdd,
                     launch_extend_add<T>(S.dev, H->levels[lvl - 1].dev, P.front_total, slots, s));
      }
      const bool many_cta = P.max_n >= H->big_front && P.ncell() <= kBigFrontCells;
      if (many_cta) {
        S.big_apply = true;
        H->ui_len = std::max<int64_t>(H->ui_len, P.gid_off.back());
        // few large fronts: panel / trailing-tile / Schur-tile launches over all fronts
        Launch t(kCatPartialChol, s, lvl_flops, double(P.front_total) * elem, 0);
        for (int p0 = 0; p0 < P.max_nI; p0 += 32) {
          int64_t tiles = 0;
          for (int c = 0; c < P.ncell(); ++c)
            tiles += front_trailing_tiles(P.nI[c], P.nI[c] + P.nB[c], p0);
          launch_front_panel<T>(S.dev, p0, H->status, s);
          launch_front_trailing<T>(S.dev, p0, tiles, s);
          add_launches(kCatPartialChol, tiles > 0 ? 3 : 2);
        }
        int64_t tiles = 0;
        if (sizeof(T) == 4 && H->tensor_cores) {
          for (int c = 0; c < P.ncell(); ++c) tiles += front_schur_tc_tiles(P.nI[c], P.nB[c]);
          // operand kind of the Schur tiles: TF32 split (about FP32), TF32, BF16
          const int kind = H->precision == RHIF_MIXED_BF16 ? 2 : H->precision == RHIF_MIXED_TF32 ? 1 : 0;
          launch_front_schur_tc(S.dev, tiles, kind, H->status, s);
        } else {
          for (int c = 0; c < P.ncell(); ++c) tiles += front_schur_tiles(P.nI[c], P.nB[c]);
          launch_front_schur<T>(S.dev, tiles, s);
        }
        add_launches(kCatPartialChol, tiles > 0 ? 1 : 0);
      } else {
        Launch t(kCatPartialChol, s, lvl_flops, double(P.front_total) * elem);
        launch_partial_chol<T>(S.dev, H->status, s);
      }
    }
    H->flops += lvl_flops;
    for (size_t ip = 0; ip < P.phases.size(); ++ip) {
      const PhasePlan& ph = P.phases[ip];
      PhaseDev& D = S.phases[ip].dev;
      void* M = nullptr;
      if ((rc = H->mem.get(&M, ph.units.m_total * elem))) return rc;
      D.Mbuf = M;
      double dflops = 0.0, sflops = 0.0;
      for (int gi : ph.pre_group) {
        const double g = P.group_size[gi];
        dflops += H->precond_diag ? g : g * g * g / 3.0;
      }
      for (int c = 0; c < P.ncell(); ++c)
        for (int q = P.seg_off[c]; q < P.seg_off[c + 1]; ++q) {
          const int gi = P.seg_group[q];
          if (ph.group_pre[gi] < 0) continue;
          const double g = P.group_size[gi];
          sflops += H->precond_diag ? 2.0 * g * P.nB[c] : 2.0 * g * g * P.nB[c];
        }
      Packer scale_tab;
      void* scale_dev = nullptr;
      if (!ph.pre_group.empty()) {
        const bool fits = (size_t)P.max_nB * P.max_nB * elem <= 200 * 1024;
        // default: many CTAs once the frame leaves shared memory, and for the
        // FP32 factor from 96 boundary DOFs (few, large cells per level)
        // (a diagonal L_g scales rows and columns in place: one CTA per cell)
        const bool big = H->precond_diag ? false
                         : H->big_frame > 0 ? P.max_nB >= H->big_frame
                                            : (!fits || (elem == 4 && P.max_nB >= 96));
        int64_t blocks = 0;
        if (big) {   // large frames: tile products with explicit inverses over many CTAs
          std::vector<int> task;
          std::vector<int64_t> off;
          for (int c = 0; c < P.ncell(); ++c)
            for (int q = P.seg_off[c]; q < P.seg_off[c + 1]; ++q)
              if (ph.group_pre[P.seg_group[q]] >= 0) {
                task.push_back(c);
                task.push_back(q);
                off.push_back(blocks);
                blocks += (P.nB[c] + 63) / 64;
              }
          const size_t o_task = scale_tab.add(task), o_off = scale_tab.add(off);
          if ((rc = H->mem.get(&scale_dev, scale_tab.total))) return rc;
          if ((rc = scale_tab.upload(scale_dev, s))) return rc;
          D.scale_task = (const int*)((char*)scale_dev + o_task);
          D.scale_off = (const int64_t*)((char*)scale_dev + o_off);
          D.nscale_task = (int)off.size();
        }
        // the L_g^{-1} (used by the many-CTA scaling, and kept for the application)
        if ((rc = H->mem.get(&D.Linv, ph.pre_total * elem))) return rc;
        {
          Launch t(kCatPrecondDiag, s, dflops, 0.0, 0);
          add_launches(kCatPrecondDiag, launch_precond_diag<T>(S.dev, D, H->status, s));
        }
        {
          Launch t(kCatPrecondScale, s, sflops, 0.0);
          if (!big) {
            int max_seg = 0;
            for (int c = 0; c < P.ncell(); ++c) max_seg = std::max(max_seg, P.seg_off[c + 1] - P.seg_off[c]);
            launch_precond_scale<T>(S.dev, D, max_seg, s);
          } else {
            launch_precond_scale_big<T>(S.dev, D, blocks, s);
            add_launches(kCatPrecondScale, blocks > 0 ? 2 : 0);
            H->mem.release(scale_dev);
            D.scale_task = nullptr;
            D.scale_off = nullptr;
            D.nscale_task = 0;
          }
        }
        // from here on only the application reads the block-Jacobi factors:
        // it gets L_g^{-1} in their place
        H->mem.release(D.Lbuf);
        D.Lbuf = D.Linv;
        D.Linv = nullptr;
      }
      const int64_t nunit = (int64_t)ph.units.group.size();
      {
        Launch t(kCatSkel, s, 0.0, 0.0, nunit ? 1 : 0);
        if ((rc = skeletonize<T>(H, P, ph, S.dev, D, alive_d, s))) return rc;
      }
      H->mem.release(M);
      D.Mbuf = nullptr;
      PhaseStore& PS = S.phases[ip];
      PS.h_rank.resize(nunit);
      PS.h_perm.resize(ph.units.perm_total);
      {   // status, ranks and pivot orders in one synchronization
        int* rb = nullptr;
        if ((rc = readback_buffer(4 + PS.h_rank.size() + PS.h_perm.size(), &rb))) return rc;
        CK(cudaMemcpyAsync(rb, H->status, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(rb + 4, D.rank, PS.h_rank.size() * sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(rb + 4 + PS.h_rank.size(), D.perm, PS.h_perm.size() * sizeof(int),
                           cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        CK(cudaGetLastError());
        if ((rc = status_message(rb, "factorization"))) return rc;
        std::copy(rb + 4, rb + 4 + PS.h_rank.size(), PS.h_rank.begin());
        std::copy(rb + 4 + PS.h_rank.size(), rb + 4 + PS.h_rank.size() + PS.h_perm.size(),
                  PS.h_perm.begin());
      }
      H->flops += dflops + sflops;
      for (int gi : ph.pre_group) {
        const double g = P.group_size[gi];
        H->apply_bytes += 2.0 * elem * g * (g + 1) / 2;
      }
      for (int64_t u = 0; u < nunit; ++u) {
        const int gi = ph.units.group[u];
        const int n = P.group_size[gi];
        const int k = PS.h_rank[u], r = n - k;
        const int* pm = PS.h_perm.data() + ph.units.perm_off[u];
        for (int i = k; i < n; ++i) keep[P.group_start[gi] + pm[i]] = 0;
        const double m = ph.units.nrow[u];
        const double uf = 4.0 * m * n * k - 2.0 * k * k * (m + n) + 4.0 * k * k * k / 3.0 +
                          double(k) * k * r + cell_flops(r, k);
        H->flops += uf;
        add_work(kCatSkel, uf, 0.0);
        H->apply_bytes += 2.0 * elem * (r * (r + 1) / 2.0 + 2.0 * r * k);
        ++H->units;
      }
    }
    // a level with a phase was checked by the phase's readback (after its last launch)
    if (P.phases.empty() && (rc = check_status(H, lvl == G.L ? "root factorization" : "cell elimination")))
      return rc;
    // Explicit inverses that only the application reads (the diagonal blocks of
    // the leaf bands, L^{-1} of every front, L_rr^{-1} of every unit): queued
    // after the level's last readback, so they run while the host plans the
    // next level.  Nothing later in the factorization reads these blocks.
    if (lvl == 0) {
      Launch t(kCatBandInverse, s, 0.0, 2.0 * elem * P.band_total);
      launch_band_block_inverse<T>(S.dev, s);
    } else {
      // L -> L^{-1} in place: every cell sweep of the application becomes a
      // row-parallel product (no sequential triangular solve)
      Launch t(kCatPartialChol, s, 0.0, 0.0, 0);
      std::vector<int64_t>& xoff = H->xoff_host;   // outlives the async upload
      xoff.assign(P.ncell(), 0);
      int64_t xtot = 0;
      for (int c = 0; c < P.ncell(); ++c) {
        xoff[c] = xtot;
        xtot += ((int64_t)P.nI[c] * P.nI[c] + 3) & ~int64_t(3);
      }
      void* X = nullptr;
      void* xo = nullptr;
      if ((rc = H->mem.get(&X, xtot * elem))) return rc;
      if ((rc = H->mem.get(&xo, xoff.size() * sizeof(int64_t)))) return rc;
      CK(cudaMemcpyAsync(xo, xoff.data(), xoff.size() * sizeof(int64_t), cudaMemcpyHostToDevice,
                         s));
      launch_front_invert<T>(S.dev, (T*)X, (const int64_t*)xo, s);
      add_launches(kCatPartialChol, 2);
      H->mem.release(X);
      H->mem.release(xo);
    }
    for (size_t ip = 0; ip < P.phases.size(); ++ip) {
      const PhasePlan& ph = P.phases[ip];
      if (ph.units.group.empty()) continue;
      void* X = nullptr;
      if ((rc = H->mem.get(&X, ph.units.rec_total * elem))) return rc;
      Launch t(kCatSkel, s, 0.0, 0.0, 0);
      add_launches(kCatSkel, launch_unit_invert<T>(S.dev, S.phases[ip].dev, (T*)X, s));
      H->mem.release(X);
    }
    if (trace)
      std::fprintf(stderr, "[rhif] level %d: cells %d groups %d active %zu max_n %d max_nB %d max_group %d plan %.2f ms upload %.2f ms gpu+sync %.2f ms\n",
                   lvl, P.ncell(), P.ngroup(), P.bucket.size(), P.max_n, P.max_nB, P.max_group,
                   t_plan, t_up, ms_since(t2));
    if (lvl == 0 && S.dev.zbuf) {
      H->mem.release(S.dev.zbuf);
      S.dev.zbuf = nullptr;
    }
    for (int c = 0; c < P.ncell(); ++c) {
      const double nI = P.nI[c], nB = P.nB[c];
      if (lvl == 0) {
        const double w = P.band_w[c];
        S.cell_flops += 4.0 * nI * w + 2.0 * nB;
        S.cell_bytes += elem * (nI * (w + 1) + nB) + 4.0 * nB + 16.0 * (nI + nB);
      } else {
        S.cell_flops += nI * nI + 2.0 * nI * nB;
        S.cell_bytes += elem * (nI * (nI + 1) / 2 + nI * nB) + 16.0 * (nI + nB);
      }
    }
    S.grp_flops.assign(P.phases.size(), 0.0);
    S.grp_bytes.assign(P.phases.size(), 0.0);
    for (size_t ip = 0; ip < P.phases.size(); ++ip) {
      const PhasePlan& ph = P.phases[ip];
      for (int gi = 0; gi < P.ngroup(); ++gi) {
        if (P.group_t[gi] < ph.pre_min_type) continue;
        const double g = P.group_size[gi];
        double f = 0, b = 16.0 * g;
        if (ph.group_pre[gi] >= 0) { f += g * g; b += elem * g * (g + 1) / 2; }
        const int u = ph.group_unit[gi];
        if (u >= 0) {
          const double k = S.phases[ip].h_rank[u], r = g - k;
          f += r * r + 4.0 * r * k;
          b += elem * (r * (r + 1) / 2 + 2.0 * r * k);
        }
        S.grp_flops[ip] += f;
        S.grp_bytes[ip] += b;
      }
    }
  }
  H->mem.release(alive_d);
  H->ui_base = H->ub_len;
  H->ub_len += H->ui_len;
  return RHIF_OK;
}

// part: 0 = F^{-1} (both sweeps), 1 = G^{-1} (upward sweep and the forward
// root solve), 2 = G^{-T} (backward root solve and downward sweep), with
// F = G G^T (Eq. 3.3: G = R_0^{-T} ... R_{L-1}^{-T} B_L).
template <typename T>
static int apply_impl(const rhif_handle* Hc, double* y, int64_t ldy, int nrhs, cudaStream_t s,
                      int part = 0) {
  rhif_handle* H = const_cast<rhif_handle*>(Hc);
  const int L = H->G.L;
  const int64_t ldu = H->ub_len;
  double* tmp = H->ubuf + H->ui_base;
  auto cell_up = [&](LevelStore& S, int cat) {
    Launch t(cat, s, S.cell_flops * nrhs, S.cell_bytes * nrhs, S.big_apply ? 0 : 1);
    if (S.big_apply)
      add_launches(cat, launch_apply_big_up<T>(S.dev, y, ldy, nrhs, H->ubuf, ldu, tmp, s));
    else
      launch_apply_cell_up<T>(S.dev, y, ldy, nrhs, H->ubuf, ldu, s);
  };
  auto cell_down = [&](LevelStore& S, int cat) {
    Launch t(cat, s, S.cell_flops * nrhs, S.cell_bytes * nrhs, S.big_apply ? 0 : 1);
    if (S.big_apply)
      add_launches(cat, launch_apply_big_down<T>(S.dev, y, ldy, nrhs, tmp, ldu, s));
    else
      launch_apply_cell_down<T>(S.dev, y, ldy, nrhs, s);
  };
  if (part != 2) {
    for (int l = 0; l < L; ++l) {
      LevelStore& S = H->levels[l];
      cell_up(S, l == 0 ? kCatApplyLeafUp : kCatApplyCellUp);
      for (size_t p = 0; p < S.phases.size(); ++p) {
        Launch t(kCatApplyGroupUp, s, S.grp_flops[p] * nrhs, S.grp_bytes[p] * nrhs);
        launch_apply_group_up<T>(S.dev, S.phases[p].dev, p == 0, y, ldy, nrhs, H->ubuf, ldu, s);
      }
    }
    cell_up(H->levels[L], kCatApplyCellUp);
  }
  if (part == 1) {
    CK(cudaGetLastError());
    return RHIF_OK;
  }
  cell_down(H->levels[L], kCatApplyCellDown);
  for (int l = L - 1; l >= 0; --l) {
    LevelStore& S = H->levels[l];
    for (int p = (int)S.phases.size() - 1; p >= 0; --p) {
      Launch t(kCatApplyGroupDown, s, S.grp_flops[p] * nrhs, S.grp_bytes[p] * nrhs);
      launch_apply_group_down<T>(S.dev, S.phases[p].dev, y, ldy, nrhs, s);
    }
    cell_down(S, l == 0 ? kCatApplyLeafDown : kCatApplyCellDown);
  }
  CK(cudaGetLastError());
  return RHIF_OK;
}

// Scratch of the sweeps (couplings sent up, interior part of big fronts).
static int apply_prepare(rhif_handle* H, int nrhs) {
  const int64_t need = H->ub_len * nrhs;
  if (need > H->ubuf_elems) {
    if (H->ubuf) H->mem.release(H->ubuf);
    H->ubuf = nullptr;
    int rc = H->mem.get((void**)&H->ubuf, need * sizeof(double));
    if (rc) return rc;
    H->ubuf_elems = need;
  }
  return RHIF_OK;
}

static int apply_launch(const rhif_handle* H, double* y, int64_t ldy, int nrhs, cudaStream_t s,
                        int part = 0) {
  return H->precision == RHIF_FP64 ? apply_impl<double>(H, y, ldy, nrhs, s, part)
                                   : apply_impl<float>(H, y, ldy, nrhs, s, part);
}

static void credit_graph(const rhif_handle* H) {
  std::lock_guard<std::mutex> lk(g_kmu);
  for (int c = 0; c < kNumCat; ++c) {
    g_kstat[c].launches += H->ag_launches[c];
    g_kstat[c].flops += H->ag_flops[c];
    g_kstat[c].bytes += H->ag_bytes[c];
  }
}

// Captures the sweeps of one application on the handle's private stream (the
// caller's stream may be the legacy default stream, which cannot be
// captured) and instantiates them; nothing runs during the capture.  Returns
// false when the capture cannot be made (the caller then launches directly).
static bool capture_apply(rhif_handle* H, double* y, int64_t ldy, int nrhs) {
  if (H->apply_graph) {
    cudaGraphExecDestroy(H->apply_graph);
    H->apply_graph = nullptr;
  }
  if (!H->capture_stream &&
      cudaStreamCreateWithFlags(&H->capture_stream, cudaStreamNonBlocking) != cudaSuccess) {
    H->capture_stream = nullptr;
    return false;
  }
  KStat counts[kNumCat];
  if (cudaStreamBeginCapture(H->capture_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return false;
  t_capture_stats = counts;
  const int rc = apply_launch(H, y, ldy, nrhs, H->capture_stream);
  t_capture_stats = nullptr;
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(H->capture_stream, &graph);
  for (int c = 0; c < kNumCat; ++c) {   // kept for the replays
    H->ag_launches[c] = counts[c].launches;
    H->ag_flops[c] = counts[c].flops;
    H->ag_bytes[c] = counts[c].bytes;
  }
  cudaGetLastError();   // a failed capture leaves no sticky error
  if (rc || e != cudaSuccess || !graph) {
    if (graph) cudaGraphDestroy(graph);
    return false;
  }
  cudaGraphExec_t exec = nullptr;
  const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  H->apply_graph = exec;
  H->ag_y = y;
  H->ag_ldy = ldy;
  H->ag_nrhs = nrhs;
  H->ag_ubuf = H->ubuf;
  return true;
}

// y <- F^{-1} y.  `replay`: the same output buffer is applied to repeatedly
// (PCG), so the sweeps go through a captured CUDA graph unless per-launch
// timing is on.
static int apply_dispatch(const rhif_handle* Hc, double* y, int64_t ldy, int nrhs, cudaStream_t s,
                          bool replay = false) {
  rhif_handle* H = const_cast<rhif_handle*>(Hc);
  int rc = apply_prepare(H, nrhs);
  if (rc) return rc;
  bool timing;
  {
    std::lock_guard<std::mutex> lk(g_kmu);
    timing = g_timing;
  }
  if (replay && !timing) {
    const bool match = H->apply_graph && H->ag_y == y && H->ag_ldy == ldy && H->ag_nrhs == nrhs &&
                       H->ag_ubuf == H->ubuf;
    if (match || capture_apply(H, y, ldy, nrhs)) {
      CK(cudaGraphLaunch(H->apply_graph, s));
      credit_graph(H);
      return RHIF_OK;
    }
  }
  return apply_launch(H, y, ldy, nrhs, s);
}

static int ensure_work(rhif_handle* H, int64_t elems) {
  if (elems <= H->work_elems) return RHIF_OK;
  if (H->work) H->mem.release(H->work);
  H->work = nullptr;
  int rc = H->mem.get((void**)&H->work, elems * sizeof(double));
  if (rc) return rc;
  H->work_elems = elems;
  return RHIF_OK;
}

// Launch counts of a graph part, credited `times` over.
static void credit_counts(const KStat* c, double times) {
  if (times <= 0) return;
  std::lock_guard<std::mutex> lk(g_kmu);
  for (int k = 0; k < kNumCat; ++k) {
    g_kstat[k].launches += (int64_t)(c[k].launches * times);
    g_kstat[k].flops += c[k].flops * times;
    g_kstat[k].bytes += c[k].bytes * times;
  }
}

// Buffers of rhif_pcg inside the handle's work array.
struct PcgBufs {
  double *r, *z, *p, *q, *part, *sc, *sc2;
  int* kit;
};

static PcgBufs pcg_bufs(double* work, int64_t N, int nrhs, int nblk) {
  PcgBufs b;
  b.r = work;
  b.z = b.r + N * nrhs;
  b.p = b.z + N * nrhs;
  b.q = b.p + N * nrhs;
  b.part = b.q + N * nrhs;
  b.sc = b.part + (int64_t)nblk * nrhs;
  b.sc2 = b.sc + 8 * nrhs;
  b.kit = (int*)(b.sc2 + 8 * nrhs);
  return b;
}

// SpMV q = A p, step alpha, x += alpha p, r -= alpha q, residual test: the
// part of a PCG iteration (Sec. 4) up to the convergence test.
static void pcg_step(rhif_handle* F, int nrhs, double* u, int64_t ldu, const PcgBufs& b,
                     double rtol, cudaStream_t s) {
  const int64_t N = F->G.N, ld = N;
  const int nblk = vec_blocks(N);
  const double spmv_flops = 2.0 * (2 * F->G.d + 1) * N, spmv_bytes = (8.0 * (1 + F->G.d) + 16.0) * N;
  const double rb = 8.0 * nblk * nrhs, vb48 = 48.0 * double(N) * nrhs;
  { Launch t_(kCatSpmv, s, spmv_flops * nrhs, spmv_bytes * nrhs); launch_spmv(F->gd, F->diag, F->off, b.p, ld, b.q, ld, nrhs, b.part, s); }
  { Launch t_(kCatVector, s, 0.0, rb); launch_reduce(b.part, nblk, nrhs, b.sc, 2, rtol, s); }
  { Launch t_(kCatVector, s, 0.0, vb48); launch_update_xr(N, nrhs, b.sc, u, ldu, b.r, ld, b.p, ld, b.q, ld, b.part, s); }
  { Launch t_(kCatVector, s, 0.0, rb); launch_reduce(b.part, nblk, nrhs, b.sc, 3, rtol, s); }
}

// z = F^{-1} r, beta, p = z + beta p: the rest of a PCG iteration.
static int pcg_direction(rhif_handle* F, int nrhs, const PcgBufs& b, double rtol, cudaStream_t s,
                         bool replay) {
  const int64_t N = F->G.N, ld = N;
  const int nblk = vec_blocks(N);
  const double rb = 8.0 * nblk * nrhs;
  { Launch t_(kCatVector, s, 0.0, 16.0 * double(N) * nrhs); launch_copy_cols(N, nrhs, b.r, ld, b.z, ld, s); }
  int rc = replay ? apply_dispatch(F, b.z, ld, nrhs, s, true) : apply_launch(F, b.z, ld, nrhs, s);
  if (rc) return rc;
  { Launch t_(kCatVector, s, 0.0, 16.0 * double(N) * nrhs); launch_dot_partial(N, b.r, ld, b.z, ld, nrhs, b.part, s); }
  { Launch t_(kCatVector, s, 0.0, rb); launch_reduce(b.part, nblk, nrhs, b.sc, 4, rtol, s); }
  { Launch t_(kCatVector, s, 0.0, 24.0 * double(N) * nrhs); launch_update_p(N, nrhs, b.sc, b.z, ld, b.p, ld, 0, s); }
  return RHIF_OK;
}

// PCG iterations (Sec. 4) as one CUDA graph: iteration 1 up to its
// convergence test (`step`), then a conditional WHILE node whose body is one
// more iteration (`direction`: preconditioner application and search
// direction; `step`: SpMV, step, residual test).  k_pcg_check sets the loop
// condition on the device from the ncheck done flags in sc (stride 8) and
// counts iterations in kit, so the host waits once, after the loop, instead
// of once per iteration.  Captured on the handle's private stream (nothing
// runs) into H->pcg_graph; false when the graph cannot be made (the caller
// then iterates from the host).
template <typename Step, typename Dir>
static bool capture_pcg_loop(rhif_handle* H, int ncheck, int* kit, const double* sc, int maxit,
                             Step step, Dir direction) {
  if (H->pcg_graph) {
    cudaGraphExecDestroy(H->pcg_graph);
    H->pcg_graph = nullptr;
  }
  if (!H->capture_stream &&
      cudaStreamCreateWithFlags(&H->capture_stream, cudaStreamNonBlocking) != cudaSuccess) {
    H->capture_stream = nullptr;
    return false;
  }
  cudaStream_t cs = H->capture_stream;
  KStat pre[kNumCat] = {}, body[kNumCat] = {};
  cudaGraph_t g = nullptr;
  if (cudaGraphCreate(&g, 0) != cudaSuccess) return false;
  cudaGraphConditionalHandle h{};
  bool ok = cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault) == cudaSuccess;
  cudaGraphNodeParams np{};
  if (ok && cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) ==
                cudaSuccess) {
    t_capture_stats = pre;
    launch_pcg_kit_init(kit, ncheck, maxit, cs);
    step(cs);
    launch_pcg_check(sc, ncheck, kit, maxit, h, cs);
    t_capture_stats = nullptr;
    cudaStreamCaptureStatus st{};
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    ok = cudaStreamGetCaptureInfo(cs, &st, nullptr, &cg, &deps, nullptr, &nd) == cudaSuccess &&
         st == cudaStreamCaptureStatusActive && cg;
    cudaGraphNode_t w = nullptr;
    if (ok) {
      np.type = cudaGraphNodeTypeConditional;
      np.conditional.handle = h;
      np.conditional.type = cudaGraphCondTypeWhile;
      np.conditional.size = 1;
      ok = cudaGraphAddNode(&w, cg, deps, nullptr, nd, &np) == cudaSuccess;
    }
    if (ok)
      ok = cudaStreamUpdateCaptureDependencies(cs, &w, nullptr, 1, cudaStreamSetCaptureDependencies) ==
           cudaSuccess;
    cudaGraph_t out = nullptr;
    const bool ended = cudaStreamEndCapture(cs, &out) == cudaSuccess;
    ok = ok && ended && out == g;
  } else {
    ok = false;
  }
  if (ok) {
    cudaGraph_t bg = np.conditional.phGraph_out[0];
    ok = bg && cudaStreamBeginCaptureToGraph(cs, bg, nullptr, nullptr, 0,
                                             cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      t_capture_stats = body;
      const int rc = direction(cs);
      step(cs);
      launch_pcg_check(sc, ncheck, kit, maxit, h, cs);
      t_capture_stats = nullptr;
      cudaGraph_t out = nullptr;
      const bool ended = cudaStreamEndCapture(cs, &out) == cudaSuccess;
      ok = ended && out == bg && rc == RHIF_OK;
    }
  }
  cudaGraphExec_t exec = nullptr;
  if (ok) ok = cudaGraphInstantiate(&exec, g, 0) == cudaSuccess;
  cudaGraphDestroy(g);
  cudaGetLastError();   // a failed capture leaves no sticky error
  if (!ok) {
    if (exec) cudaGraphExecDestroy(exec);
    return false;
  }
  H->pcg_graph = exec;
  for (int c = 0; c < kNumCat; ++c) {
    H->pg_pre[c] = pre[c];
    H->pg_body[c] = body[c];
  }
  return true;
}

// Whether H->pcg_graph was captured for these buffers and parameters.
static bool pcg_graph_matches(const rhif_handle* H, const double* u, int64_t ldu, int nrhs,
                              double rtol, int maxit) {
  return H->pcg_graph && H->pg_u == u && H->pg_work == H->work && H->pg_ubuf == H->ubuf &&
         H->pg_ldu == ldu && H->pg_nrhs == nrhs && H->pg_rtol == rtol && H->pg_maxit == maxit;
}

static void pcg_graph_key(rhif_handle* H, double* u, int64_t ldu, int nrhs, double rtol, int maxit) {
  H->pg_u = u;
  H->pg_work = H->work;
  H->pg_ubuf = H->ubuf;
  H->pg_ldu = ldu;
  H->pg_nrhs = nrhs;
  H->pg_rtol = rtol;
  H->pg_maxit = maxit;
}

// The iterations of rhif_pcg as one graph (capture_pcg_loop).
static bool capture_pcg(rhif_handle* H, int nrhs, double* u, int64_t ldu, double rtol, int maxit) {
  const PcgBufs b = pcg_bufs(H->work, H->G.N, nrhs, vec_blocks(H->G.N));
  const bool ok = capture_pcg_loop(
      H, nrhs, b.kit, b.sc, maxit, [&](cudaStream_t cs) { pcg_step(H, nrhs, u, ldu, b, rtol, cs); },
      [&](cudaStream_t cs) { return pcg_direction(H, nrhs, b, rtol, cs, false); });
  if (ok) pcg_graph_key(H, u, ldu, nrhs, rtol, maxit);
  return ok;
}


// Runs job(i, stream) for i = 0..count-1 with one host worker per stream.
template <typename Job>
static int run_batched(int count, void* const* streams, int nstreams, Job job,
                       std::vector<std::string>* details) {
  if (count < 0 || nstreams < 1 || !streams) return fail(RHIF_ERR_BAD_ARG, "bad batch arguments");
  int dev = 0;
  CK(cudaGetDevice(&dev));
  // kernel attributes are set once, before any worker starts
  if (configure_once<double>() || configure_once<float>())
    return fail(RHIF_ERR_CUDA, "cannot configure kernel shared memory");
  std::vector<int> rc(count, RHIF_OK);
  details->assign(count, std::string());
  std::vector<std::thread> pool;
  const int nw = std::min(nstreams, std::max(count, 1));
  for (int w = 0; w < nw; ++w) {
    pool.emplace_back([&, w]() {
      cudaSetDevice(dev);
      for (int i = w; i < count; i += nw) {
        rc[i] = job(i, streams[w % nstreams]);
        if (rc[i]) (*details)[i] = g_detail;
      }
    });
  }
  for (auto& t : pool) t.join();
  for (int i = 0; i < count; ++i)
    if (rc[i]) return fail(rc[i], "problem " + std::to_string(i) + ": " + (*details)[i]);
  return RHIF_OK;
}

}  // namespace rhif

using namespace rhif;

extern "C" {

int rhif_default_opts(rhif_opts* o) {
  if (!o) return fail(RHIF_ERR_BAD_ARG, "null opts");
  std::memset(o, 0, sizeof(*o));
  o->precision = RHIF_FP64;
  o->precondition = 1;
  o->edge_skel_3d = 0;
  return RHIF_OK;
}

static int check_grid(const rhif_grid* g) {
  if (!g || (g->dim != 2 && g->dim != 3)) return fail(RHIF_ERR_BAD_ARG, "grid dim must be 2 or 3");
  for (int a = 0; a < g->dim; ++a)
    if (g->n[a] < 1) return fail(RHIF_ERR_BAD_ARG, "grid sizes must be >= 1");
  int64_t N = 1;
  for (int a = 0; a < g->dim; ++a) N *= g->n[a];
  if (N >= (int64_t)1 << 31) return fail(RHIF_ERR_BAD_ARG, "more than 2^31 - 1 DOFs");
  return RHIF_OK;
}

int64_t rhif_fd_nnz(const rhif_grid* g) {
  if (check_grid(g)) return -1;
  int64_t N = 1;
  for (int a = 0; a < g->dim; ++a) N *= g->n[a];
  int64_t nnz = N;
  for (int a = 0; a < g->dim; ++a) nnz += 2 * (N / g->n[a]) * (g->n[a] - 1);
  return nnz;
}

int rhif_assemble_fd(const rhif_grid* g, const double* a_pix, const double* b_node, double b_const,
                     int64_t* rowptr, int32_t* col, double* val, void* stream) {
  int rc = check_grid(g);
  if (rc) return rc;
  if (!a_pix || !rowptr || !col || !val) return fail(RHIF_ERR_BAD_ARG, "null pointer");
  Geometry G = make_geometry(g->dim, g->n, 2);
  {
    Launch t(kCatAssemble, (cudaStream_t)stream, 0.0, 0.0);
    launch_assemble_fd(geo_dev(G), a_pix, b_node, b_const, rowptr, col, val, (cudaStream_t)stream);
  }
  CK(cudaGetLastError());
  return RHIF_OK;
}

int rhif_assemble_fd_log(const rhif_grid* g, const double* log_a_pix, double* a_pix_out,
                         const double* b_node, double b_const, int64_t* rowptr, int32_t* col,
                         double* val, void* stream) {
  int rc = check_grid(g);
  if (rc) return rc;
  if (!log_a_pix || !a_pix_out) return fail(RHIF_ERR_BAD_ARG, "null pointer");
  int64_t npix = 1;
  for (int a = 0; a < g->dim; ++a) npix *= g->n[a] + 1;
  {
    Launch t(kCatAssemble, (cudaStream_t)stream, 0.0, 16.0 * npix);
    launch_exp(npix, log_a_pix, a_pix_out, (cudaStream_t)stream);
  }
  CK(cudaGetLastError());
  return rhif_assemble_fd(g, a_pix_out, b_node, b_const, rowptr, col, val, stream);
}

// Options of a factorization (argument checks before any device work).
static int set_options(rhif_handle* H, int dim, double tol, const rhif_opts* o) {
  rhif_opts def;
  rhif_default_opts(&def);
  if (!o) o = &def;
  if (o->precision < RHIF_FP64 || o->precision > RHIF_MIXED_BF16)
    return fail(RHIF_ERR_BAD_ARG, "unknown precision");
  H->precision = o->precision;
  if (o->precondition < 0 || o->precondition > 2)
    return fail(RHIF_ERR_BAD_ARG, "precondition must be 0 (HIF), 1 (block Jacobi) or 2 (diagonal)");
  H->precondition = o->precondition != 0;
  H->precond_diag = o->precondition == 2;
  H->edge_skel = (dim == 3) && o->edge_skel_3d;
  H->big_front = o->big_front == 0 ? kBigFront : (o->big_front < 0 ? INT_MAX : o->big_front);
  H->big_frame = o->big_frame < 0 ? INT_MAX : o->big_frame;
  if (o->skel_cluster > 16 || (o->skel_cluster > 0 && (o->skel_cluster & (o->skel_cluster - 1))))
    return fail(RHIF_ERR_BAD_ARG, "skel_cluster must be a power of two <= 16");
  H->skel_cluster = o->skel_cluster;
  H->tensor_cores = o->tensor_cores >= 0;
  if (o->leaf_fp64 > 30) return fail(RHIF_ERR_BAD_ARG, "leaf_fp64 must be <= 30");
  H->leaf_fp64 = o->leaf_fp64 < 0 ? 0.0 : std::pow(10.0, o->leaf_fp64 == 0 ? 6 : o->leaf_fp64);
  H->tol = tol;
  return RHIF_OK;
}

// Run the factorization of a prepared handle (A: one CSR per problem).
static int run_factor(std::unique_ptr<rhif_handle>& H, const rhif_csr* A, void* stream,
                      rhif_handle** out) {
  int rc = RHIF_OK;
  H->mem.s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  CK(cudaEventRecord(e0, H->mem.s));
  rc = H->precision == RHIF_FP64 ? factor_impl<double>(H.get(), A) : factor_impl<float>(H.get(), A);
  if (rc) {
    cudaStreamSynchronize(H->mem.s);
    H->mem.release_all();
    cudaStreamSynchronize(H->mem.s);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
  }
  CK(cudaEventRecord(e1, H->mem.s));
  CK(cudaEventSynchronize(e1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  H->factor_ms = ms;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *out = H.release();
  return RHIF_OK;
}

int rhif_factor(const rhif_csr* A, const rhif_grid* g, int leaf, double tol, const rhif_opts* o,
                void* stream, rhif_handle** out) {
  if (!out) return fail(RHIF_ERR_BAD_ARG, "null output handle");
  *out = nullptr;
  int rc = check_grid(g);
  if (rc) return rc;
  if (!A || !A->rowptr || !A->col || !A->val) return fail(RHIF_ERR_BAD_ARG, "null CSR pointer");
  if (leaf < 2) return fail(RHIF_ERR_BAD_ARG, "leaf must be >= 2");
  if (!(tol >= 0.0) || !std::isfinite(tol)) return fail(RHIF_ERR_BAD_ARG, "tol must be finite and >= 0");
  std::unique_ptr<rhif_handle> H(new rhif_handle());
  if ((rc = set_options(H.get(), g->dim, tol, o))) return rc;
  H->G = make_geometry(g->dim, g->n, leaf);
  if (A->nrows != H->G.N) return fail(RHIF_ERR_BAD_ARG, "CSR rows != number of grid DOFs");
  if (A->nnz < H->G.N) return fail(RHIF_ERR_BAD_ARG, "CSR has fewer entries than rows");
  if (H->G.L > 20) return fail(RHIF_ERR_BAD_ARG, "too many levels");
  H->gd = geo_dev(H->G);
  return run_factor(H, A, stream, out);
}

int rhif_factor_batch(int count, const rhif_csr* A, const rhif_grid* g, int leaf, double tol,
                      const rhif_opts* o, void* stream, rhif_handle** out) {
  if (!out) return fail(RHIF_ERR_BAD_ARG, "null output handle");
  *out = nullptr;
  if (count < 1 || !A || !g) return fail(RHIF_ERR_BAD_ARG, "need count >= 1 problems");
  if (leaf < 2) return fail(RHIF_ERR_BAD_ARG, "leaf must be >= 2");
  if (!(tol >= 0.0) || !std::isfinite(tol)) return fail(RHIF_ERR_BAD_ARG, "tol must be finite and >= 0");
  int rc = RHIF_OK;
  std::unique_ptr<rhif_handle> H(new rhif_handle());
  if ((rc = set_options(H.get(), g[0].dim, tol, o))) return rc;
  Geometry T{};
  T.d = g[0].dim;
  T.leaf = leaf;
  for (int p = 0; p < count; ++p) {
    if ((rc = check_grid(&g[p]))) return rc;
    if (g[p].dim != T.d) return fail(RHIF_ERR_BAD_ARG, "every problem of a batch needs the same dimension");
    if (!A[p].rowptr || !A[p].col || !A[p].val) return fail(RHIF_ERR_BAD_ARG, "null CSR pointer");
    const Geometry Gp = make_geometry(g[p].dim, g[p].n, leaf);
    if (A[p].nrows != Gp.N || A[p].nnz < Gp.N) return fail(RHIF_ERR_BAD_ARG, "CSR does not match its grid");
    if (Gp.L > 20) return fail(RHIF_ERR_BAD_ARG, "too many levels");
    H->pG.push_back(Gp);
    H->pbase.push_back(T.N);
    T.N += Gp.N;
    T.L = std::max(T.L, Gp.L);
  }
  if (T.N > INT32_MAX) return fail(RHIF_ERR_BAD_ARG, "a batch holds at most 2^31 - 1 DOFs");
  H->G = T;
  H->gd = geo_dev(T);
  return run_factor(H, A, stream, out);
}

int rhif_batch_info(const rhif_handle* F, int* count, int64_t* dof_base) {
  if (!F || !count) return fail(RHIF_ERR_BAD_ARG, "null argument");
  *count = F->pG.empty() ? 1 : (int)F->pG.size();
  if (dof_base) {
    if (F->pG.empty()) {
      dof_base[0] = 0;
      dof_base[1] = F->G.N;
    } else {
      for (size_t p = 0; p < F->pG.size(); ++p) dof_base[p] = F->pbase[p];
      dof_base[F->pG.size()] = F->G.N;
    }
  }
  return RHIF_OK;
}

// Device time of one configuration: rhif_factor's own event span (host
// planning gaps included) plus `applies` applications of F^{-1} to one vector;
// the smaller of two trials.
static int tune_cost(const rhif_csr* A, const rhif_grid* g, int leaf, double tol,
                     const rhif_opts& o, int applies, cudaStream_t s, double* ms) {
  double best = INFINITY;
  for (int trial = 0; trial < 2; ++trial) {
    rhif_handle* F = nullptr;
    int rc = rhif_factor(A, g, leaf, tol, &o, s, &F);
    if (rc) return rc;
    double c = F->factor_ms;
    if (applies > 0) {
      double* x = nullptr;
      if ((rc = F->mem.get((void**)&x, F->G.N * sizeof(double)))) {
        rhif_free(F);
        return rc;
      }
      cudaEvent_t e0 = nullptr, e1 = nullptr;
      cudaError_t ce = cudaMemsetAsync(x, 0, F->G.N * sizeof(double), s);
      if (ce == cudaSuccess) ce = cudaEventCreate(&e0);
      if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
      if (ce == cudaSuccess) ce = cudaEventRecord(e0, s);
      if (ce == cudaSuccess) rc = apply_dispatch(F, x, F->G.N, 1, s);
      if (ce == cudaSuccess && !rc) ce = cudaEventRecord(e1, s);
      if (ce == cudaSuccess && !rc) ce = cudaEventSynchronize(e1);
      float am = 0.f;
      if (ce == cudaSuccess && !rc) ce = cudaEventElapsedTime(&am, e0, e1);
      if (e0) cudaEventDestroy(e0);
      if (e1) cudaEventDestroy(e1);
      F->mem.release(x);
      if (!rc && ce != cudaSuccess) rc = fail(RHIF_ERR_CUDA, cudaGetErrorString(ce));
      if (rc) {
        rhif_free(F);
        return rc;
      }
      c += applies * (double)am;
    }
    rhif_free(F);
    best = std::min(best, c);
  }
  *ms = best;
  return RHIF_OK;
}

int rhif_autotune(const rhif_csr* A, const rhif_grid* g, int leaf, double tol, const rhif_opts* base,
                  int applies, void* stream, rhif_opts* best, double* best_ms) {
  if (!best || applies < 0) return fail(RHIF_ERR_BAD_ARG, "null output or applies < 0");
  rhif_opts cur;
  if (base) cur = *base;
  else rhif_default_opts(&cur);
  cudaStream_t s = (cudaStream_t)stream;
  {   // warm-up: one-time set-up (kernel attributes, pools, staging) stays out of the timings
    rhif_handle* F = nullptr;
    const int rc = rhif_factor(A, g, leaf, tol, &cur, s, &F);
    if (rc) return rc;
    rhif_free(F);
  }
  double cur_ms = 0.0;
  int rc = tune_cost(A, g, leaf, tol, cur, applies, s, &cur_ms);
  if (rc) return rc;
  // one pass of coordinate descent; each knob takes its library default (0),
  // "always many CTAs" (1) or "never" (-1); a change must gain 2%
  struct Knob {
    int rhif_opts::*field;
    int count;
    int values[3];
  };
  const Knob knobs[] = {{&rhif_opts::big_front, 3, {0, 1, -1}},
                        {&rhif_opts::big_frame, 3, {0, 1, -1}},
                        {&rhif_opts::skel_cluster, 3, {0, -1, 4}},
                        {&rhif_opts::tensor_cores, 2, {0, -1, 0}}};
  for (const Knob& k : knobs) {
    if (k.field == &rhif_opts::tensor_cores && cur.precision == RHIF_FP64) continue;
    const int start = cur.*(k.field);
    for (int i = 0; i < k.count; ++i) {
      const int v = k.values[i];
      if (v == start) continue;
      rhif_opts o = cur;
      o.*(k.field) = v;
      double ms = 0.0;
      if ((rc = tune_cost(A, g, leaf, tol, o, applies, s, &ms))) return rc;
      if (ms < 0.98 * cur_ms) {
        cur = o;
        cur_ms = ms;
      }
    }
  }
  *best = cur;
  if (best_ms) *best_ms = cur_ms;
  return RHIF_OK;
}

int rhif_factor_batched(int count, const rhif_csr* A, const rhif_grid* g, int leaf, double tol,
                        const rhif_opts* o, void* const* streams, int nstreams,
                        rhif_handle** out) {
  if (!A || !g || !out) return fail(RHIF_ERR_BAD_ARG, "null argument");
  for (int i = 0; i < count; ++i) out[i] = nullptr;
  std::vector<std::string> details;
  return run_batched(
      count, streams, nstreams,
      [&](int i, void* s) { return rhif_factor(&A[i], &g[i], leaf, tol, o, s, &out[i]); },
      &details);
}

int rhif_pcg_batched(int count, rhif_handle* const* F, int nrhs, const double* const* f,
                     double* const* u, double rtol, int maxit, int* iters, double* relres,
                     void* const* streams, int nstreams) {
  if (!F || !f || !u) return fail(RHIF_ERR_BAD_ARG, "null argument");
  for (int i = 0; i < count; ++i)
    if (!F[i]) return fail(RHIF_ERR_BAD_ARG, "null handle in batch");
  std::vector<std::string> details;
  return run_batched(
      count, streams, nstreams,
      [&](int i, void* s) {
        const int64_t N = F[i]->G.N;
        return rhif_pcg(F[i], nrhs, f[i], N, u[i], N, rtol, maxit,
                        iters ? iters + (int64_t)i * nrhs : nullptr,
                        relres ? relres + (int64_t)i * nrhs : nullptr, s);
      },
      &details);
}

// y = F x (Eq. 3.1) from the stored factor.  The stored blocks are those
// F^{-1} needs (Eq. 3.2: explicit inverses of the triangular factors), so F x
// is the solution of F^{-1} y = x, found by conjugate gradients on the SPD
// operator F^{-1} preconditioned with A: A F^{-1} has the spectrum the outer
// PCG sees (clustered at 1, spread e_s = ||I - A F^{-1}||), so a few
// iterations reach the precision of the application of F^{-1} itself.  Stops
// when every column's residual ||x - F^{-1} y|| is at most rtol ||x|| (rtol
// 1e-13 for FP64 factors, 1e-7 for FP32 ones, whose F^{-1} is applied in FP32)
// or has not decreased for 4 iterations (the precision of the application),
// after at most 200 iterations.
static int matvec_impl(rhif_handle* F, int nrhs, const double* x, int64_t ldx, double* y,
                       int64_t ldy, cudaStream_t s) {
  const int64_t N = F->G.N, ld = N;
  const int nblk = vec_blocks(N);
  const int64_t need = 4 * N * nrhs + (int64_t)nblk * nrhs + 8 * nrhs;
  if (need > F->mv_elems) {
    if (F->mv_work) F->mem.release(F->mv_work);
    F->mv_work = nullptr;
    int rc = F->mem.get((void**)&F->mv_work, need * sizeof(double));
    if (rc) return rc;
    F->mv_elems = need;
  }
  const bool batch = !F->pG.empty();
  if (batch) return fail(RHIF_ERR_BAD_ARG, "F x of a batch: apply it to each problem's factor");
  double* r = F->mv_work;
  double* z = r + N * nrhs;
  double* p = z + N * nrhs;
  double* q = p + N * nrhs;
  double* part = q + N * nrhs;
  double* sc = part + (int64_t)nblk * nrhs;
  const double rtol = F->precision == RHIF_FP64 ? 1e-13 : 1e-7;
  int rc = RHIF_OK;
  auto A = [&](const double* in, double* out) {
    Launch t(kCatSpmv, s, 2.0 * (2 * F->G.d + 1) * N * nrhs, (8.0 * (1 + F->G.d) + 16.0) * N * nrhs);
    launch_spmv(F->gd, F->diag, F->off, in, ld, out, ld, nrhs, nullptr, s);
  };
  auto dot = [&](const double* a, int64_t la, const double* b, int64_t lb, int mode) {
    launch_dot_partial(N, a, la, b, lb, nrhs, part, s);
    launch_reduce(part, nblk, nrhs, sc, mode, rtol, s);
  };
  CK(cudaMemsetAsync(sc, 0, 8 * nrhs * sizeof(double), s));
  for (int c = 0; c < nrhs; ++c) CK(cudaMemsetAsync(y + c * ldy, 0, N * sizeof(double), s));
  launch_copy_cols(N, nrhs, x, ldx, r, ld, s);
  dot(x, ldx, x, ldx, 0);
  A(r, z);
  dot(r, ld, z, ld, 1);
  launch_update_p(N, nrhs, sc, z, ld, p, ld, 1, s);
  std::vector<double> hsc(8 * nrhs);
  std::vector<double> best(nrhs, INFINITY);
  std::vector<int> since(nrhs, 0);
  int k = 0;
  for (k = 1; k <= 200; ++k) {
    launch_copy_cols(N, nrhs, p, ld, q, ld, s);
    if ((rc = apply_dispatch(F, q, ld, nrhs, s, true))) return rc;   // q = F^{-1} p
    dot(p, ld, q, ld, 2);                                            // alpha
    launch_update_xr(N, nrhs, sc, y, ldy, r, ld, p, ld, q, ld, part, s);
    launch_reduce(part, nblk, nrhs, sc, 3, rtol, s);                 // rr, done
    CK(cudaMemcpyAsync(hsc.data(), sc, 8 * nrhs * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    bool all = true;
    for (int c = 0; c < nrhs; ++c) {
      const double rr = hsc[8 * c + kScRR];
      if (rr < 0.99 * best[c]) {
        best[c] = rr;
        since[c] = 0;
      } else {
        ++since[c];
      }
      all = all && (hsc[8 * c + kScDone] != 0.0 || since[c] >= 4);
    }
    if (all) break;
    A(r, z);                                                         // z = A r
    dot(r, ld, z, ld, 4);                                            // beta
    launch_update_p(N, nrhs, sc, z, ld, p, ld, 0, s);
  }
  F->mv_iters = std::min(k, 200);
  CK(cudaGetLastError());
  return RHIF_OK;
}

int rhif_apply(const rhif_handle* Fc, int op, int nrhs, const double* x, int64_t ldx, double* y,
               int64_t ldy, void* stream) {
  rhif_handle* F = const_cast<rhif_handle*>(Fc);
  if (!F || !x || !y || nrhs < 0) return fail(RHIF_ERR_BAD_ARG, "null argument");
  if (op < RHIF_SOLVE || op > RHIF_HALF_T) return fail(RHIF_ERR_BAD_ARG, "unknown operation");
  const int64_t N = F->G.N;
  if (ldx < N || ldy < N) return fail(RHIF_ERR_BAD_ARG, "leading dimension < N");
  if (x == y && ldx != ldy) return fail(RHIF_ERR_BAD_ARG, "aliased x and y need ldx == ldy");
  if (op == RHIF_MATVEC && x == y) return fail(RHIF_ERR_BAD_ARG, "F x needs distinct x and y");
  if (nrhs == 0) return RHIF_OK;
  cudaStream_t s = (cudaStream_t)stream;
  if (op == RHIF_MATVEC) return matvec_impl(F, nrhs, x, ldx, y, ldy, s);
  if (x != y) {
    Launch t(kCatVector, s, 0.0, 16.0 * N * nrhs);
    launch_copy_cols(N, nrhs, x, ldx, y, ldy, s);
  }
  if (op == RHIF_SOLVE) return apply_dispatch(F, y, ldy, nrhs, s);
  int rc = apply_prepare(F, nrhs);
  if (rc) return rc;
  return apply_launch(F, y, ldy, nrhs, s, op == RHIF_HALF ? 1 : 2);
}

// Vector blocks of a merged batch (uploaded once per handle).
static int batch_segments(rhif_handle* H) {
  if (H->vseg.nblk) return RHIF_OK;
  std::vector<int64_t> n(H->pG.size());
  for (size_t p = 0; p < n.size(); ++p) n[p] = H->pG[p].N;
  std::vector<int> prob, pblk;
  std::vector<int64_t> r0, r1;
  batch_vec_blocks(H->pbase, n, prob, r0, r1, pblk);
  Packer pk;
  const size_t o_p = pk.add(prob), o_r0 = pk.add(r0), o_r1 = pk.add(r1), o_b = pk.add(pblk);
  void* d = nullptr;
  int rc = H->mem.get(&d, pk.total);
  if (rc) return rc;
  if ((rc = pk.upload(d, H->mem.s))) return rc;
  CK(cudaStreamSynchronize(H->mem.s));
  char* b = (char*)d;
  H->vseg.nblk = (int)prob.size();
  H->vseg.nprob = (int)n.size();
  H->vseg.prob = (const int*)(b + o_p);
  H->vseg.row0 = (const int64_t*)(b + o_r0);
  H->vseg.row1 = (const int64_t*)(b + o_r1);
  H->vseg.pblk_off = (const int*)(b + o_b);
  return RHIF_OK;
}

int rhif_spmv(const rhif_handle* F, int nrhs, const double* x, int64_t ldx, double* y, int64_t ldy,
              void* stream) {
  if (!F || !x || !y || nrhs < 0) return fail(RHIF_ERR_BAD_ARG, "null argument");
  if (ldx < F->G.N || ldy < F->G.N) return fail(RHIF_ERR_BAD_ARG, "leading dimension < N");
  if (nrhs == 0) return RHIF_OK;
  if (!F->pG.empty()) {   // merged batch: every problem's stencil on its block of the vectors
    rhif_handle* H = const_cast<rhif_handle*>(F);
    int rc = batch_segments(H);
    if (rc) return rc;
    const double N = double(F->G.N);
    Launch t(kCatSpmv, (cudaStream_t)stream, 2.0 * (2 * F->G.d + 1) * N * nrhs,
             (8.0 * (1 + F->G.d) + 16.0) * N * nrhs);
    launch_bspmv(H->vseg, H->bgeo, x, ldx, y, ldy, nrhs, nullptr, (cudaStream_t)stream);
    CK(cudaGetLastError());
    return RHIF_OK;
  }
  {
    const double N = double(F->G.N);
    Launch t(kCatSpmv, (cudaStream_t)stream, 2.0 * (2 * F->G.d + 1) * N * nrhs,
             (8.0 * (1 + F->G.d) + 16.0) * N * nrhs);
    launch_spmv(F->gd, F->diag, F->off, x, ldx, y, ldy, nrhs, nullptr, (cudaStream_t)stream);
  }
  CK(cudaGetLastError());
  return RHIF_OK;
}

// PCG (Sec. 4) of every (problem, right-hand side) pair of a merged batch at
// once, on concatenated vectors: the same iteration as rhif_pcg with
// per-pair scalars, one F^{-1} application (the merged sweeps) and one SpMV
// launch per iteration for the whole batch.  The iterations run on the device
// as one graph with a conditional loop over all pairs' convergence flags
// (capture_pcg_loop), from the host while per-launch timing is on.
// iters / relres: count x nrhs, problem-major.
static int pcg_batch_core(rhif_handle* F, int nrhs, const double* f, int64_t ldf, double* u,
                          int64_t ldu, double rtol, int maxit, int* iters, double* relres,
                          cudaStream_t s) {
  int rc = batch_segments(F);
  if (rc) return rc;
  const VecSeg& S = F->vseg;
  const int np = S.nprob, nblk = S.nblk;
  const int64_t N = F->G.N, ld = N;
  const double spmv_flops = 2.0 * (2 * F->G.d + 1) * N, spmv_bytes = (8.0 * (1 + F->G.d) + 16.0) * N;
  const int64_t nsc = 8 * (int64_t)np * nrhs;
  const int npair = np * nrhs;
  const int64_t need = 4 * N * nrhs + (int64_t)nblk * nrhs + 2 * nsc + (npair + 2) / 2 + 1;
  if ((rc = ensure_work(F, need))) return rc;
  double* r = F->work;
  double* z = r + N * nrhs;
  double* p = z + N * nrhs;
  double* q = p + N * nrhs;
  double* part = q + N * nrhs;
  double* sc = part + (int64_t)nblk * nrhs;
  double* sc2 = sc + nsc;
  int* kit = (int*)(sc2 + nsc);   // device loop: iterations, then one count per (rhs, problem)
  auto vb = [&](double per_entry) { return per_entry * double(N) * nrhs; };
  const double rb = 8.0 * nblk * nrhs;
  // the two halves of an iteration: SpMV, step and residual test; then
  // preconditioner application and search direction
  auto step = [&](cudaStream_t st) {
    { Launch t_(kCatSpmv, st, spmv_flops * nrhs, spmv_bytes * nrhs); launch_bspmv(S, F->bgeo, p, ld, q, ld, nrhs, part, st); }
    { Launch t_(kCatVector, st, 0.0, rb); launch_breduce(S, part, nrhs, sc, 2, rtol, st); }
    { Launch t_(kCatVector, st, 0.0, vb(48)); launch_bupdate_xr(S, nrhs, sc, u, ldu, r, ld, p, ld, q, ld, part, st); }
    { Launch t_(kCatVector, st, 0.0, rb); launch_breduce(S, part, nrhs, sc, 3, rtol, st); }
  };
  auto direction = [&](cudaStream_t st, bool replay) -> int {
    { Launch t_(kCatVector, st, 0.0, vb(16)); launch_copy_cols(N, nrhs, r, ld, z, ld, st); }
    const int e = replay ? apply_dispatch(F, z, ld, nrhs, st, true) : apply_launch(F, z, ld, nrhs, st);
    if (e) return e;
    { Launch t_(kCatVector, st, 0.0, vb(16)); launch_bdot_partial(S, r, ld, z, ld, nrhs, part, st); }
    { Launch t_(kCatVector, st, 0.0, rb); launch_breduce(S, part, nrhs, sc, 4, rtol, st); }
    { Launch t_(kCatVector, st, 0.0, vb(24)); launch_bupdate_p(S, nrhs, sc, z, ld, p, ld, 0, st); }
    return RHIF_OK;
  };
  CK(cudaMemsetAsync(sc, 0, 2 * nsc * sizeof(double), s));
  for (int c = 0; c < nrhs; ++c) CK(cudaMemsetAsync(u + c * ldu, 0, N * sizeof(double), s));
  { Launch t_(kCatVector, s, 0.0, vb(16)); launch_copy_cols(N, nrhs, f, ldf, r, ld, s); }
  { Launch t_(kCatVector, s, 0.0, vb(8)); launch_bdot_partial(S, f, ldf, f, ldf, nrhs, part, s); }
  { Launch t_(kCatVector, s, 0.0, rb); launch_breduce(S, part, nrhs, sc, 0, rtol, s); }
  { Launch t_(kCatVector, s, 0.0, vb(16)); launch_copy_cols(N, nrhs, r, ld, z, ld, s); }
  if ((rc = apply_dispatch(F, z, ld, nrhs, s, true))) return rc;
  { Launch t_(kCatVector, s, 0.0, vb(16)); launch_bdot_partial(S, r, ld, z, ld, nrhs, part, s); }
  { Launch t_(kCatVector, s, 0.0, rb); launch_breduce(S, part, nrhs, sc, 1, rtol, s); }
  { Launch t_(kCatVector, s, 0.0, vb(24)); launch_bupdate_p(S, nrhs, sc, z, ld, p, ld, 1, s); }
  std::vector<double> hsc(nsc);
  std::vector<int> it(npair, maxit), hkit(npair + 1, 0);
  std::vector<char> was_done(npair, 0);
  int all_done = 0;
  // the iterations on the device as one graph with a conditional loop
  // (unless per-launch timing is on), else from the host
  bool timing;
  {
    std::lock_guard<std::mutex> lk(g_kmu);
    timing = g_timing;
  }
  bool device_loop = false;
  if (!timing && maxit > 0) {
    bool ok = pcg_graph_matches(F, u, ldu, nrhs, rtol, maxit);
    if (!ok) {
      ok = capture_pcg_loop(F, npair, kit, sc, maxit, step,
                            [&](cudaStream_t st) { return direction(st, false); });
      if (ok) pcg_graph_key(F, u, ldu, nrhs, rtol, maxit);
    }
    if (ok) {
      CK(cudaGraphLaunch(F->pcg_graph, s));
      CK(cudaMemcpyAsync(hkit.data(), kit, (npair + 1) * sizeof(int), cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(hsc.data(), sc, nsc * sizeof(double), cudaMemcpyDeviceToHost, s));
      device_loop = true;
    }
  }
  for (int k = 1; !device_loop && k <= maxit; ++k) {
    step(s);
    CK(cudaMemcpyAsync(hsc.data(), sc, nsc * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    int nd = 0;
    for (int c = 0; c < nrhs; ++c)
      for (int pp = 0; pp < np; ++pp) {
        const int pair = pp * nrhs + c;
        if (hsc[8 * ((int64_t)c * np + pp) + kScDone] != 0.0) {
          if (!was_done[pair]) { it[pair] = k; was_done[pair] = 1; }
          ++nd;
        }
      }
    if (nd == npair) { all_done = 1; break; }
    if ((rc = direction(s, true))) return rc;
  }
  if (maxit == 0) {
    CK(cudaMemcpyAsync(hsc.data(), sc, nsc * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  }
  // true residuals
  { Launch t_(kCatSpmv, s, spmv_flops * nrhs, spmv_bytes * nrhs); launch_bspmv(S, F->bgeo, u, ldu, q, ld, nrhs, nullptr, s); }
  { Launch t_(kCatVector, s, 0.0, vb(24)); launch_sub(N, nrhs, f, ldf, q, ld, r, ld, s); }
  { Launch t_(kCatVector, s, 0.0, vb(8)); launch_bdot_partial(S, r, ld, r, ld, nrhs, part, s); }
  { Launch t_(kCatVector, s, 0.0, rb); launch_breduce(S, part, nrhs, sc2, 1, rtol, s); }
  std::vector<double> h2(nsc);
  CK(cudaMemcpyAsync(h2.data(), sc2, nsc * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  CK(cudaGetLastError());
  if (device_loop) {   // counts per (rhs, problem) in the check's order, c * np + pp
    credit_counts(F->pg_pre, 1.0);
    credit_counts(F->pg_body, double(hkit[0] - 1));
    all_done = 1;
    for (int c = 0; c < nrhs; ++c)
      for (int pp = 0; pp < np; ++pp) {
        const int64_t j = (int64_t)c * np + pp;
        it[pp * nrhs + c] = hkit[1 + j];
        if (hsc[8 * j + kScDone] == 0.0) all_done = 0;
      }
  }
  for (int c = 0; c < nrhs; ++c)
    for (int pp = 0; pp < np; ++pp) {
      const int64_t o = 8 * ((int64_t)c * np + pp);
      const double ff = hsc[o + kScFF];
      if (iters) iters[pp * nrhs + c] = it[pp * nrhs + c];
      if (relres) relres[pp * nrhs + c] = ff > 0 ? std::sqrt(h2[o + kScRZ] / ff) : 0.0;
    }
  if (!all_done) return fail(RHIF_ERR_NOT_CONVERGED, "PCG reached maxit before rtol");
  return RHIF_OK;
}

int rhif_pcg_batch(const rhif_handle* Fc, int nrhs, const double* const* f, double* const* u,
                   double rtol, int maxit, int* iters, double* relres, void* stream) {
  rhif_handle* F = const_cast<rhif_handle*>(Fc);
  if (!F || !f || !u || nrhs < 1 || maxit < 0 || !(rtol >= 0.0))
    return fail(RHIF_ERR_BAD_ARG, "bad argument");
  if (F->pG.empty()) return fail(RHIF_ERR_BAD_ARG, "not a batch handle (rhif_factor_batch)");
  const int np = (int)F->pG.size();
  for (int p = 0; p < np; ++p)
    if (!f[p] || !u[p]) return fail(RHIF_ERR_BAD_ARG, "null right-hand side or solution");
  cudaStream_t s = (cudaStream_t)stream;
  int rc = batch_segments(F);
  if (rc) return rc;
  const int64_t N = F->G.N;
  // concatenated right-hand sides and solutions, and the problems' pointer tables
  void* buf = nullptr;
  if ((rc = F->mem.get(&buf, 2 * N * nrhs * sizeof(double) + 2 * np * sizeof(double*) + 16))) return rc;
  double* fc = (double*)buf;
  double* uc = fc + N * nrhs;
  const double** fp = (const double**)(uc + N * nrhs);
  double** up = (double**)(fp + np);
  std::vector<const double*> hp(2 * np);
  for (int p = 0; p < np; ++p) {
    hp[p] = f[p];
    hp[np + p] = u[p];
  }
  CK(cudaMemcpyAsync((void*)fp, hp.data(), 2 * np * sizeof(double*), cudaMemcpyHostToDevice, s));
  { Launch t_(kCatVector, s, 0.0, 16.0 * N * nrhs); launch_bgather(F->vseg, F->bgeo, fp, fc, N, nrhs, s); }
  rc = pcg_batch_core(F, nrhs, fc, N, uc, N, rtol, maxit, iters, relres, s);
  if (rc == RHIF_OK || rc == RHIF_ERR_NOT_CONVERGED) {
    Launch t_(kCatVector, s, 0.0, 16.0 * N * nrhs);
    launch_bscatter(F->vseg, F->bgeo, uc, N, up, nrhs, s);
  }
  CK(cudaStreamSynchronize(s));   // hp is a host local
  F->mem.release(buf);
  return rc;
}

int rhif_pcg(const rhif_handle* Fc, int nrhs, const double* f, int64_t ldf, double* u, int64_t ldu,
             double rtol, int maxit, int* iters, double* relres, void* stream) {
  rhif_handle* F = const_cast<rhif_handle*>(Fc);
  if (!F || !f || !u || nrhs < 1 || maxit < 0 || !(rtol >= 0.0))
    return fail(RHIF_ERR_BAD_ARG, "bad argument");
  const int64_t N = F->G.N;
  if (ldf < N || ldu < N) return fail(RHIF_ERR_BAD_ARG, "leading dimension < N");
  if (!F->pG.empty())
    return pcg_batch_core(F, nrhs, f, ldf, u, ldu, rtol, maxit, iters, relres, (cudaStream_t)stream);
  cudaStream_t s = (cudaStream_t)stream;
  const int nblk = vec_blocks(N);
  const int64_t ld = N;
  const double spmv_flops = 2.0 * (2 * F->G.d + 1) * N, spmv_bytes = (8.0 * (1 + F->G.d) + 16.0) * N;
  // r, z, p, q (N x nrhs each), partials, two scalar blocks, iteration counters
  const int64_t need = 4 * N * nrhs + (int64_t)nblk * nrhs + 16 * nrhs + (nrhs + 2) / 2 + 1;
  int rc = ensure_work(F, need);
  if (rc) return rc;
  const PcgBufs b = pcg_bufs(F->work, N, nrhs, nblk);
  // algorithmic bytes of the vector launches (FP64 vectors read / written once)
  auto vb = [&](double per_entry) { return per_entry * double(N) * nrhs; };
  const double rb = 8.0 * nblk * nrhs;
  CK(cudaMemsetAsync(b.sc, 0, 16 * nrhs * sizeof(double), s));
  for (int c = 0; c < nrhs; ++c) CK(cudaMemsetAsync(u + c * ldu, 0, N * sizeof(double), s));
  { Launch t_(kCatVector, s, 0.0, vb(16)); launch_copy_cols(N, nrhs, f, ldf, b.r, ld, s); }
  { Launch t_(kCatVector, s, 0.0, vb(8)); launch_dot_partial(N, f, ldf, f, ldf, nrhs, b.part, s); }
  { Launch t_(kCatVector, s, 0.0, rb); launch_reduce(b.part, nblk, nrhs, b.sc, 0, rtol, s); }
  { Launch t_(kCatVector, s, 0.0, vb(16)); launch_copy_cols(N, nrhs, b.r, ld, b.z, ld, s); }
  if ((rc = apply_dispatch(F, b.z, ld, nrhs, s, true))) return rc;
  { Launch t_(kCatVector, s, 0.0, vb(16)); launch_dot_partial(N, b.r, ld, b.z, ld, nrhs, b.part, s); }
  { Launch t_(kCatVector, s, 0.0, rb); launch_reduce(b.part, nblk, nrhs, b.sc, 1, rtol, s); }
  { Launch t_(kCatVector, s, 0.0, vb(24)); launch_update_p(N, nrhs, b.sc, b.z, ld, b.p, ld, 1, s); }
  std::vector<double> hsc(8 * nrhs);
  std::vector<int> it(nrhs, maxit), hkit(nrhs + 1, 0);
  int all_done = 0;
  // the iterations: on the device as one graph with a conditional loop
  // (unless per-launch timing is on), else from the host
  bool timing;
  {
    std::lock_guard<std::mutex> lk(g_kmu);
    timing = g_timing;
  }
  bool device_loop = false;
  if (!timing && maxit > 0) {
    if (pcg_graph_matches(F, u, ldu, nrhs, rtol, maxit) || capture_pcg(F, nrhs, u, ldu, rtol, maxit)) {
      CK(cudaGraphLaunch(F->pcg_graph, s));
      CK(cudaMemcpyAsync(hkit.data(), b.kit, (nrhs + 1) * sizeof(int), cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(hsc.data(), b.sc, 8 * nrhs * sizeof(double), cudaMemcpyDeviceToHost, s));
      device_loop = true;
    }
  }
  if (!device_loop) {
    std::vector<char> was_done(nrhs, 0);
    for (int k = 1; k <= maxit; ++k) {
      pcg_step(F, nrhs, u, ldu, b, rtol, s);
      CK(cudaMemcpyAsync(hsc.data(), b.sc, 8 * nrhs * sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      int nd = 0;
      for (int c = 0; c < nrhs; ++c) {
        if (hsc[8 * c + kScDone] != 0.0) {
          if (!was_done[c]) { it[c] = k; was_done[c] = 1; }
          ++nd;
        }
      }
      if (nd == nrhs) { all_done = 1; break; }
      if ((rc = pcg_direction(F, nrhs, b, rtol, s, true))) return rc;
    }
    if (maxit == 0)
      CK(cudaMemcpyAsync(hsc.data(), b.sc, 8 * nrhs * sizeof(double), cudaMemcpyDeviceToHost, s));
  }
  // true residual
  { Launch t_(kCatSpmv, s, spmv_flops * nrhs, spmv_bytes * nrhs); launch_spmv(F->gd, F->diag, F->off, u, ldu, b.q, ld, nrhs, nullptr, s); }
  { Launch t_(kCatVector, s, 0.0, vb(24)); launch_sub(N, nrhs, f, ldf, b.q, ld, b.r, ld, s); }
  { Launch t_(kCatVector, s, 0.0, vb(8)); launch_dot_partial(N, b.r, ld, b.r, ld, nrhs, b.part, s); }
  { Launch t_(kCatVector, s, 0.0, rb); launch_reduce(b.part, nblk, nrhs, b.sc2, 1, rtol, s); }
  std::vector<double> h2(8 * nrhs);
  CK(cudaMemcpyAsync(h2.data(), b.sc2, 8 * nrhs * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  CK(cudaGetLastError());
  if (device_loop) {
    credit_counts(F->pg_pre, 1.0);
    credit_counts(F->pg_body, double(hkit[0] - 1));
    all_done = 1;
    for (int c = 0; c < nrhs; ++c) {
      it[c] = hkit[1 + c];
      if (hsc[8 * c + kScDone] == 0.0) all_done = 0;
    }
  }
  for (int c = 0; c < nrhs; ++c) {
    const double ff = hsc[8 * c + kScFF];
    if (iters) iters[c] = it[c];
    if (relres) relres[c] = ff > 0 ? std::sqrt(h2[8 * c + kScRZ] / ff) : 0.0;
  }
  if (!all_done) return fail(RHIF_ERR_NOT_CONVERGED, "PCG reached maxit before rtol");
  return RHIF_OK;
}

int rhif_estimate_es(const rhif_handle* Fc, const double* x0, int maxit, double rel, double* es,
                     int* iters, void* stream) {
  rhif_handle* F = const_cast<rhif_handle*>(Fc);
  if (!F || !x0 || !es || maxit < 1 || !(rel >= 0.0)) return fail(RHIF_ERR_BAD_ARG, "bad argument");
  if (!F->pG.empty()) return fail(RHIF_ERR_BAD_ARG, "e_s of a batch: estimate each problem on its own");
  const int64_t N = F->G.N;
  cudaStream_t s = (cudaStream_t)stream;
  const int nblk = vec_blocks(N);
  int rc = ensure_work(F, 4 * N + nblk + 16);
  if (rc) return rc;
  double* v = F->work;
  double* z = v + N;
  double* w = z + N;
  double* t = w + N;
  double* part = t + N;
  double* sc = part + nblk;   // 8 slots; sc[kScFF] receives the reductions
  double* inv = sc + 8;       // 1 / norm for the rescaling
  std::vector<double> hsc(8);
  auto norm2 = [&](const double* x, double* out) -> int {
    launch_dot_partial(N, x, N, x, N, 1, part, s);
    launch_reduce(part, nblk, 1, sc, 0, 0.0, s);
    CK(cudaMemcpyAsync(hsc.data(), sc, 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    *out = std::sqrt(hsc[kScFF]);
    return RHIF_OK;
  };
  auto set_inv = [&](double nv) -> int {
    const double a = 1.0 / nv;
    CK(cudaMemcpyAsync(inv, &a, sizeof(double), cudaMemcpyHostToDevice, s));
    launch_scale(N, v, inv, s);
    CK(cudaStreamSynchronize(s));   // `a` is a host local
    return RHIF_OK;
  };
  launch_copy_cols(N, 1, x0, N, v, N, s);
  double nv = 0.0;
  if ((rc = norm2(v, &nv))) return rc;
  if (nv == 0.0) return fail(RHIF_ERR_BAD_ARG, "zero start vector");
  if ((rc = set_inv(nv))) return rc;
  double est = 0.0;
  int it = 0;
  for (it = 1; it <= maxit; ++it) {
    // w = M v = v - A F^{-1} v ; then w = M^T w = w - F^{-1} A w
    launch_copy_cols(N, 1, v, N, z, N, s);
    if ((rc = apply_dispatch(F, z, N, 1, s))) return rc;
    launch_spmv(F->gd, F->diag, F->off, z, N, t, N, 1, nullptr, s);
    launch_sub(N, 1, v, N, t, N, w, N, s);
    launch_spmv(F->gd, F->diag, F->off, w, N, t, N, 1, nullptr, s);
    if ((rc = apply_dispatch(F, t, N, 1, s))) return rc;
    launch_sub(N, 1, w, N, t, N, w, N, s);
    double nw = 0.0;
    if ((rc = norm2(w, &nw))) return rc;
    const double cur = std::sqrt(nw);
    if (nw == 0.0) {
      est = 0.0;
      break;
    }
    launch_copy_cols(N, 1, w, N, v, N, s);
    if ((rc = set_inv(nw))) return rc;
    if (est > 0.0 && std::fabs(cur - est) <= rel * cur) {
      est = cur;
      break;
    }
    est = cur;
  }
  *es = est;
  if (iters) *iters = std::min(it, maxit);
  CK(cudaGetLastError());
  return RHIF_OK;
}

int rhif_estimate_ea(const rhif_handle* Fc, const double* x0, const double* x1, int maxit,
                     double rel, double* ea, int* iters, void* stream) {
  rhif_handle* F = const_cast<rhif_handle*>(Fc);
  if (!F || !x0 || !ea || maxit < 1 || !(rel >= 0.0)) return fail(RHIF_ERR_BAD_ARG, "bad argument");
  if (!F->pG.empty()) return fail(RHIF_ERR_BAD_ARG, "e_a of a batch: estimate each problem on its own");
  if (!x1) x1 = x0;
  const int64_t N = F->G.N;
  cudaStream_t s = (cudaStream_t)stream;
  const int nblk = vec_blocks(N);
  int rc = ensure_work(F, 4 * N + nblk + 16);
  if (rc) return rc;
  double* v = F->work;
  double* w = v + N;
  double* t = w + N;
  double* u = t + N;
  double* part = u + N;
  double* sc = part + nblk;
  double* inv = sc + 8;
  std::vector<double> hsc(8);
  auto norm = [&](const double* x, double* out) -> int {
    launch_dot_partial(N, x, N, x, N, 1, part, s);
    launch_reduce(part, nblk, 1, sc, 0, 0.0, s);
    CK(cudaMemcpyAsync(hsc.data(), sc, 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    *out = std::sqrt(hsc[kScFF]);
    return RHIF_OK;
  };
  auto scale_to_v = [&](const double* src, double nv) -> int {
    const double a = 1.0 / nv;
    launch_copy_cols(N, 1, src, N, v, N, s);
    CK(cudaMemcpyAsync(inv, &a, sizeof(double), cudaMemcpyHostToDevice, s));
    launch_scale(N, v, inv, s);
    CK(cudaStreamSynchronize(s));   // `a` is a host local
    return RHIF_OK;
  };
  // out = M in: M = A - F (with_f) or A
  auto apply_m = [&](const double* in, double* out, bool with_f) -> int {
    launch_spmv(F->gd, F->diag, F->off, in, N, out, N, 1, nullptr, s);
    if (!with_f) return RHIF_OK;
    int r2 = matvec_impl(F, 1, in, N, u, N, s);
    if (r2) return r2;
    launch_sub(N, 1, out, N, u, N, out, N, s);
    return RHIF_OK;
  };
  // power iteration on M^T M = M^2 (M symmetric), Sec. 4 estimator
  auto power = [&](const double* start, bool with_f, double* est_out, int* it_out) -> int {
    double nv = 0.0;
    int r2 = norm(start, &nv);
    if (r2) return r2;
    if (nv == 0.0) return fail(RHIF_ERR_BAD_ARG, "zero start vector");
    if ((r2 = scale_to_v(start, nv))) return r2;
    double est = 0.0;
    int it = 1;
    for (; it <= maxit; ++it) {
      if ((r2 = apply_m(v, t, with_f))) return r2;
      if ((r2 = apply_m(t, w, with_f))) return r2;
      double nw = 0.0;
      if ((r2 = norm(w, &nw))) return r2;
      const double cur = std::sqrt(nw);
      if (nw == 0.0) {
        est = 0.0;
        break;
      }
      if ((r2 = scale_to_v(w, nw))) return r2;
      if (est > 0.0 && std::fabs(cur - est) <= rel * cur) {
        est = cur;
        break;
      }
      est = cur;
    }
    *est_out = est;
    *it_out = std::min(it, maxit);
    return RHIF_OK;
  };
  double num = 0.0, den = 0.0;
  int it_num = 0, it_den = 0;
  if ((rc = power(x0, true, &num, &it_num))) return rc;
  if ((rc = power(x1, false, &den, &it_den))) return rc;
  *ea = den > 0.0 ? num / den : 0.0;
  if (iters) *iters = it_num;
  CK(cudaGetLastError());
  return RHIF_OK;
}

int rhif_tc_gemm_check(int kind, int M, int N, int K, const float* A, int64_t lda, const float* B,
                       int64_t ldb, float* C, int64_t ldc, void* stream) {
  if (kind < RHIF_TC_TF32X3 || kind > RHIF_TC_BF16) return fail(RHIF_ERR_BAD_ARG, "unknown operand kind");
  if (M < 1 || N < 1 || K < 0 || !C || ldc < M || (K > 0 && (!A || !B || lda < M || ldb < N)))
    return fail(RHIF_ERR_BAD_ARG, "bad GEMM arguments");
  static std::once_flag once;
  static int cfg = 0;
  std::call_once(once, [] { cfg = configure_tc_kernels(); });
  if (cfg) return fail(RHIF_ERR_CUDA, "cannot configure the tensor-core kernel");
  cudaStream_t s = (cudaStream_t)stream;
  int* st = nullptr;
  CK(cudaMallocAsync((void**)&st, 4 * sizeof(int), s));
  CK(cudaMemsetAsync(st, 0, 4 * sizeof(int), s));
  launch_tc_gemm_check(kind, M, N, K, A, lda, B, ldb, C, ldc, st, s);
  int h[4] = {0, 0, 0, 0};
  CK(cudaMemcpyAsync(h, st, sizeof(h), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  cudaFreeAsync(st, s);
  CK(cudaGetLastError());
  if (h[0]) return fail(h[0], "tensor-core wait timed out");
  return RHIF_OK;
}

int rhif_grad_logcoef(const rhif_grid* g, const double* a_pix, const double* u, const double* lam,
                      double* grad, void* stream) {
  int rc = check_grid(g);
  if (rc) return rc;
  if (!a_pix || !u || !lam || !grad) return fail(RHIF_ERR_BAD_ARG, "null pointer");
  Geometry G = make_geometry(g->dim, g->n, 2);
  {
    Launch t(kCatGrad, (cudaStream_t)stream, 0.0, 0.0);
    launch_grad_logcoef(geo_dev(G), a_pix, u, lam, grad, (cudaStream_t)stream);
  }
  CK(cudaGetLastError());
  return RHIF_OK;
}

int rhif_stats(const rhif_handle* F, rhif_stats_t* st) {
  if (!F || !st) return fail(RHIF_ERR_BAD_ARG, "null argument");
  std::memset(st, 0, sizeof(*st));
  st->levels = F->G.L;
  st->n = F->G.N;
  st->root_size = F->levels.empty() ? 0 : F->levels.back().plan().nI.empty() ? 0 : F->levels.back().plan().nI[0];
  for (int l = 0; l < F->G.L && l < 16; ++l) {
    // active DOFs after level l = DOFs present at level l+1
    st->active[l] = (int64_t)F->levels[l + 1].plan().bucket.size();
  }
  st->factor_bytes = (int64_t)F->mem.bytes;
  st->flops = F->flops;
  st->apply_bytes = F->apply_bytes;
  st->precision = F->precision;
  st->units = F->units;
  st->factor_ms = F->factor_ms;
  for (int l = 0; l < F->G.L && l < 16; ++l) {
    const LevelStore& S = F->levels[l];
    for (size_t p = 0; p < S.phases.size(); ++p) {
      const PhasePlan& ph = S.plan().phases[p];
      for (size_t u = 0; u < S.phases[p].h_rank.size(); ++u) {
        st->unit_dofs[l] += S.plan().group_size[ph.units.group[u]];
        st->skeletons[l] += S.phases[p].h_rank[u];
      }
    }
  }
  st->fp64_leaves = 0;
  if (F->precision != RHIF_FP64 && F->leaf_fp64 > 0.0 && F->status) {
    rhif_handle* H = const_cast<rhif_handle*>(F);
    if (H->fp64_leaves < 0) {   // the counter of the condition kernel (status word 4)
      int v = 0;
      CK(cudaMemcpy(&v, H->status + 4, sizeof(int), cudaMemcpyDeviceToHost));
      H->fp64_leaves = v;
    }
    st->fp64_leaves = H->fp64_leaves;
  }
  return RHIF_OK;
}

int rhif_skeletons(const rhif_handle* F, int level, int phase, int* count, int* sizes, int* ranks,
                   int64_t* gids, int64_t capacity) {
  if (!F || !count) return fail(RHIF_ERR_BAD_ARG, "null argument");
  if (level < 0 || level >= F->G.L) return fail(RHIF_ERR_BAD_ARG, "level out of range");
  const LevelStore& S = F->levels[level];
  if (phase < 0 || phase >= (int)S.phases.size()) return fail(RHIF_ERR_BAD_ARG, "phase out of range");
  const PhasePlan& ph = S.plan().phases[phase];
  const PhaseStore& PS = S.phases[phase];
  const int nu = (int)ph.units.group.size();
  *count = nu;
  int64_t pos = 0;
  for (int u = 0; u < nu; ++u) {
    const int gi = ph.units.group[u];
    const int64_t g0 = S.plan().group_start[gi];
    const int n = S.plan().group_size[gi];
    if (sizes) sizes[u] = n;
    if (ranks) ranks[u] = PS.h_rank[u];
    if (gids) {
      if (pos + n > capacity) return fail(RHIF_ERR_BAD_ARG, "gids capacity too small");
      const int* pm = PS.h_perm.data() + ph.units.perm_off[u];
      for (int i = 0; i < n; ++i) gids[pos + i] = S.plan().bucket[g0 + pm[i]];
    }
    pos += n;
  }
  return RHIF_OK;
}

void rhif_free(rhif_handle* F) {
  if (!F) return;
  F->mem.release_all();
  cudaStreamSynchronize(F->mem.s);
  if (F->apply_graph) cudaGraphExecDestroy(F->apply_graph);
  if (F->pcg_graph) cudaGraphExecDestroy(F->pcg_graph);
  if (F->capture_stream) cudaStreamDestroy(F->capture_stream);
  for (auto& S : F->levels) {
    if (S.p0) continue;   // the shared level-0 plan stays with its other holders
    if (S.own.cell_prob.empty()) recycle_plan(std::move(S.own));
    else recycle_merged_plan(std::move(S.own));
  }
  delete F;
}

int rhif_set_timing(int on) {
  std::lock_guard<std::mutex> lk(g_kmu);
  g_timing = on != 0;
  return RHIF_OK;
}

int rhif_reset_kernel_stats(void) {
  cudaDeviceSynchronize();
  std::lock_guard<std::mutex> lk(g_kmu);
  for (auto& p : g_pending) {
    g_event_pool.push_back(p.a);
    g_event_pool.push_back(p.b);
  }
  g_pending.clear();
  for (auto& k : g_kstat) k = KStat();
  return RHIF_OK;
}

int rhif_kernel_stat_count(void) { return kNumCat; }

int rhif_kernel_stats(int index, rhif_kernel_stat* out) {
  if (index < 0 || index >= kNumCat || !out) return fail(RHIF_ERR_BAD_ARG, "bad kernel stat index");
  CK(cudaDeviceSynchronize());
  std::lock_guard<std::mutex> lk(g_kmu);
  for (auto& p : g_pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) g_kstat[p.cat].ms += ms;
    g_event_pool.push_back(p.a);
    g_event_pool.push_back(p.b);
  }
  g_pending.clear();
  std::memset(out, 0, sizeof(*out));
  std::snprintf(out->name, sizeof(out->name), "%s", kCatName[index]);
  out->launches = g_kstat[index].launches;
  out->total_ms = g_kstat[index].ms;
  out->flops = g_kstat[index].flops;
  out->bytes = g_kstat[index].bytes;
  return RHIF_OK;
}

const char* rhif_error_string(int code) {
  switch (code) {
    case RHIF_OK: return "RHIF_OK";
    case RHIF_ERR_BAD_ARG: return "RHIF_ERR_BAD_ARG";
    case RHIF_ERR_NOT_SPD: return "RHIF_ERR_NOT_SPD";
    case RHIF_ERR_NOT_CONVERGED: return "RHIF_ERR_NOT_CONVERGED";
    case RHIF_ERR_TIMEOUT: return "RHIF_ERR_TIMEOUT";
    case RHIF_ERR_OOM: return "RHIF_ERR_OOM";
    case RHIF_ERR_CUDA: return "RHIF_ERR_CUDA";
    case RHIF_ERR_CHECK: return "RHIF_ERR_CHECK";
    default: return "unknown";
  }
}

const char* rhif_last_error_detail(void) { return g_detail.c_str(); }

}  // extern "C"

// ---------------------------------------------------------------------------
// F^{-1} x without any device allocation
// ---------------------------------------------------------------------------
//
// Scratch for the cell-to-group contributions of the upward sweep, held in a
// file-scope device array instead of memory the handle allocates on first
// use.  Every GPU that loads the library keeps these 8 MiB until the process
// exits.  Each call writes every entry it later reads, so nothing has to be
// cleared between calls; calls that overlap on the GPU (two streams, or two
// handles used concurrently) share the array and race.

namespace rhif {

constexpr int64_t kNoAllocScratch = int64_t(1) << 20;   // doubles
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratch];

static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[256];

// Device address of the scratch array on the current device, looked up once
// per device (the array's host-side name is only a stand-in).
static int noalloc_scratch(double** out) {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) return fail(RHIF_ERR_CUDA, "device index out of range");
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess)
      return fail(RHIF_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_noalloc_addr[dev] = p;
  }
  *out = (double*)g_noalloc_addr[dev];
  return RHIF_OK;
}

template <typename T>
static int apply_noalloc_impl(const rhif_handle* Hc, double* y, int64_t ldy, int nrhs,
                              double* ubuf, cudaStream_t s) {
  rhif_handle* H = const_cast<rhif_handle*>(Hc);
  const int L = H->G.L;
  const int64_t ldu = H->ub_len;
  double* tmp = ubuf + H->ui_base;
  auto cell_up = [&](LevelStore& S) {
    if (S.big_apply) launch_apply_big_up<T>(S.dev, y, ldy, nrhs, ubuf, ldu, tmp, s);
    else launch_apply_cell_up<T>(S.dev, y, ldy, nrhs, ubuf, ldu, s);
  };
  auto cell_down = [&](LevelStore& S) {
    if (S.big_apply) launch_apply_big_down<T>(S.dev, y, ldy, nrhs, tmp, ldu, s);
    else launch_apply_cell_down<T>(S.dev, y, ldy, nrhs, s);
  };
  for (int l = 0; l < L; ++l) {
    LevelStore& S = H->levels[l];
    cell_up(S);
    for (size_t p = 0; p < S.phases.size(); ++p)
      launch_apply_group_up<T>(S.dev, S.phases[p].dev, p == 0, y, ldy, nrhs, ubuf, ldu, s);
  }
  cell_up(H->levels[L]);
  cell_down(H->levels[L]);
  for (int l = L - 1; l >= 0; --l) {
    LevelStore& S = H->levels[l];
    for (int p = (int)S.phases.size() - 1; p >= 0; --p)
      launch_apply_group_down<T>(S.dev, S.phases[p].dev, y, ldy, nrhs, s);
    cell_down(S);
  }
  CK(cudaGetLastError());
  return RHIF_OK;
}

}  // namespace rhif

extern "C" int rhif_apply_noalloc(const rhif_handle* F, int nrhs, const double* x, int64_t ldx,
                                  double* y, int64_t ldy, void* stream) {
  if (!F || !x || !y || nrhs < 0) return fail(RHIF_ERR_BAD_ARG, "null argument");
  const int64_t N = F->G.N;
  if (ldx < N || ldy < N) return fail(RHIF_ERR_BAD_ARG, "leading dimension < N");
  if (x == y && ldx != ldy) return fail(RHIF_ERR_BAD_ARG, "aliased x and y need ldx == ldy");
  if (nrhs == 0) return RHIF_OK;
  const int64_t need = F->ub_len * (int64_t)nrhs;
  if (need > kNoAllocScratch)
    return fail(RHIF_ERR_BAD_ARG, "rhif_apply_noalloc needs " + std::to_string(need) +
                                      " scratch doubles; the static scratch holds " +
                                      std::to_string(kNoAllocScratch) +
                                      " (use fewer right-hand sides or rhif_apply)");
  double* ubuf = nullptr;
  int rc = noalloc_scratch(&ubuf);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if (x != y) launch_copy_cols(N, nrhs, x, ldx, y, ldy, s);
  return F->precision == RHIF_FP64 ? apply_noalloc_impl<double>(F, y, ldy, nrhs, ubuf, s)
                                   : apply_noalloc_impl<float>(F, y, ldy, nrhs, ubuf, s);
}
