// Application of F^{-1} (Eq. 3.2) and the FP64 vector kernels of PCG.
//
// F^{-1} x = R_0 ... R_{L-1} A_L^{-1} R_{L-1}^T ... R_0^T x with
// R_l = E_l C_l K_l.  Per level the upward sweep applies E_l^T per cell
// (y = L^{-1} x_I, x_B -= W y with W = A_BI L^{-T}), then C_l^T and K_l^T per
// separator group; the downward sweep applies K_l, C_l per group and E_l per
// cell (x_I = L^{-T}(x_I - W^T x_B)).  The cell contributions to a shared
// boundary DOF are written per cell and summed by the owning group in cell
// order, so the result does not depend on scheduling.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"
#include "tables.h"
#include "../../include/rhif.h"

namespace rhif {

constexpr int kApplyThreads = 256;
constexpr int kGroupThreads = 128;
constexpr int kLeafWarps = 4;                 // at most this many leaf cells per CTA (one warp each)
constexpr int kGroupWarps = 4;                // small groups per CTA (one warp each)
constexpr size_t kStageBudget = 160 * 1024;   // shared memory for staged factor blocks

// Timeout of a bulk copy: record it, give the copy a second bounded chance to
// land (the shared memory must not be released while it is in flight), and
// tell the caller to skip the work.
__device__ inline bool staged_ok(uint64_t* bar, int* status, int level, int kind, int index) {
  if (mbar_wait(bar, 0)) return true;
  report(status, RHIF_ERR_TIMEOUT, level, kind, index);
  mbar_wait(bar, 0);
  return false;
}

// ---------------------------------------------------------------------------
// level 0: banded leaf factors, one warp per cell
// ---------------------------------------------------------------------------

// Forms for w <= 15 (all 2D leaves up to leaf 16).  The factor stores, in
// the in-block slots of every diagonal w x w block of the band, the explicit
// inverse X of that block (k_band_block_inverse); the slots coupling a block
// to the next one keep L.  A block solve is then the coupling update of the
// lane's row followed by one row (column) of X times the block's right-hand
// sides: independent shuffles and FMAs, no dependent chain inside the block.
constexpr int kBandRegW = kBandInvW;

template <typename T>
__device__ inline void warp_band_fwd_inv(const T* band, int n, int w, T* y) {
  const int lane = threadIdx.x & 31;
  const int w1 = w + 1;
  for (int s0 = 0; s0 < n; s0 += w) {
    const int B = min(w, n - s0);
    const int i = s0 + lane;
    const bool act = lane < B;
    T cp[kBandRegW + 1], yp[kBandRegW + 1], xr[kBandRegW];
#pragma unroll
    for (int d = 1; d <= kBandRegW; ++d) {
      const int j = i - d;
      const bool ok = act && d <= w && d > lane && j >= 0;
      cp[d] = ok ? band[j * w1 + d] : T(0);
      yp[d] = ok ? y[j] : T(0);
    }
#pragma unroll
    for (int c = 0; c < kBandRegW; ++c)   // row `lane` of X
      xr[c] = (act && c <= lane) ? band[(s0 + c) * w1 + (lane - c)] : T(0);
    T acc = act ? y[i] : T(0);
#pragma unroll
    for (int d = 1; d <= kBandRegW; ++d) acc -= cp[d] * yp[d];
    T out = T(0);
#pragma unroll
    for (int c = 0; c < kBandRegW; ++c) {
      const T rc = __shfl_sync(0xffffffffu, acc, c);
      out += xr[c] * rc;
    }
    if (act) y[i] = out;
    __syncwarp();
  }
}

template <typename T>
__device__ inline void warp_band_bwd_inv(const T* band, int n, int w, T* y) {
  const int lane = threadIdx.x & 31;
  const int w1 = w + 1;
  const int nblk = (n + w - 1) / w;
  for (int bi = nblk - 1; bi >= 0; --bi) {
    const int s0 = bi * w;
    const int B = min(w, n - s0);
    const int i = s0 + lane;
    const bool act = lane < B;
    T cp[kBandRegW + 1], yn[kBandRegW + 1], xc[kBandRegW];
#pragma unroll
    for (int d = 1; d <= kBandRegW; ++d) {
      const int j = i + d;
      const bool ok = act && d <= w && d >= B - lane && j < n;
      cp[d] = ok ? band[i * w1 + d] : T(0);
      yn[d] = ok ? y[j] : T(0);
    }
#pragma unroll
    for (int c = 0; c < kBandRegW; ++c)   // column `lane` of X
      xc[c] = (act && c >= lane && c < B) ? band[(s0 + lane) * w1 + (c - lane)] : T(0);
    T acc = act ? y[i] : T(0);
#pragma unroll
    for (int d = 1; d <= kBandRegW; ++d) acc -= cp[d] * yn[d];
    T out = T(0);
#pragma unroll
    for (int c = 0; c < kBandRegW; ++c) {
      const T rc = __shfl_sync(0xffffffffu, acc, c);
      out += xc[c] * rc;
    }
    if (act) y[i] = out;
    __syncwarp();
  }
}

template <typename T>
__device__ inline void band_fwd(const T* band, int n, int w, T* y) {
  if (w >= 1 && w <= kBandRegW) warp_band_fwd_inv(band, n, w, y);
  else if (w >= 1 && w <= 31) warp_band_fwd_blk(band, n, w, y);
  else warp_band_fwd(band, n, w, y);
}

template <typename T>
__device__ inline void band_bwd(const T* band, int n, int w, T* y) {
  if (w >= 1 && w <= kBandRegW) warp_band_bwd_inv(band, n, w, y);
  else if (w >= 1 && w <= 31) warp_band_bwd_blk(band, n, w, y);
  else warp_band_bwd(band, n, w, y);
}

// dst[i] = T(xr[g[i]]) for i < n, one warp: indices of a 256-entry chunk
// first, then the gathered values, so each chunk costs two load latencies.
template <typename T>
__device__ inline void warp_gather(const double* xr, const int32_t* g, int n, T* dst) {
  const int lane = threadIdx.x & 31;
  for (int i0 = 0; i0 < n; i0 += 256) {
    int idx[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int i = i0 + 32 * u + lane;
      idx[u] = i < n ? g[i] : -1;
    }
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = idx[u] >= 0 ? xr[idx[u]] : 0.0;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int i = i0 + 32 * u + lane;
      if (i < n) dst[i] = T(v[u]);
    }
  }
}

// per-warp shared memory of the leaf kernels: [mbarrier | band | y | z]
template <typename T>
__host__ __device__ inline size_t leaf_band_bytes(int max_nI, int max_w) {
  return round16((size_t)max_nI * (max_w + 1) * sizeof(T));
}

// Bands of half bandwidth <= kBandRegW are read in place (global memory,
// prefetched into L2 as the warp starts): the per-warp shared memory then
// holds only the vectors, so every leaf of a level is resident at once.
// Wider (3D) bands are staged in shared memory by one bulk copy.
template <typename T>
static bool leaf_staged(const LevelDev& Lv) {
  return Lv.max_w > kBandRegW;
}

template <typename T>
static size_t leaf_warp_smem(const LevelDev& Lv, bool staged) {
  return 16 + (staged ? leaf_band_bytes<T>(Lv.max_nI, Lv.max_w) : 0) +
         round16((2 * (Lv.max_nI + 1) + Lv.max_nB) * sizeof(T));
}

template <typename T>
static int leaf_warps_per_cta(const LevelDev& Lv, bool staged) {
  const size_t per = leaf_warp_smem<T>(Lv, staged);
  int w = (int)(kStageBudget / per);
  return w < 1 ? 1 : (w > kLeafWarps ? kLeafWarps : w);
}

// The band of leaf c in place, its cache lines prefetched into L2.
template <typename T>
__device__ inline const T* leaf_inplace(const LevelDev& Lv, int c) {
  const int lane = threadIdx.x & 31;
  const T* band = (const T*)Lv.band + Lv.band_off[c];
  const size_t bytes = (size_t)Lv.nI[c] * (Lv.band_w[c] + 1) * sizeof(T);
  const char* p = (const char*)band;
  for (size_t off = (size_t)lane * 128; off < bytes; off += 32 * 128)
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p + off));
  return band;
}

// Starts the bulk copy of this warp's leaf band; returns the band in shared memory.
template <typename T>
__device__ inline T* leaf_stage(const LevelDev& Lv, int c, unsigned char* base, uint64_t** bar_out) {
  const int lane = threadIdx.x & 31;
  uint64_t* bar = (uint64_t*)base;
  T* sb = (T*)(base + 16);
  if (lane == 0) {
    const uint32_t bytes = round16((size_t)Lv.nI[c] * (Lv.band_w[c] + 1) * sizeof(T));
    mbar_init(bar, 1);
    mbar_expect_tx(bar, bytes);
    if (bytes) bulk_g2s(sb, (const T*)Lv.band + Lv.band_off[c], bytes, bar);
  }
  __syncwarp();
  *bar_out = bar;
  return sb;
}

// E_0^T per leaf: y = L^{-1} x_I ; x_B -= A_BI L^{-T} y (sent to the owning groups) ; x_I = y
template <typename T, bool STAGE>
__global__ void __launch_bounds__(32 * kLeafWarps)
k_apply_leaf_up(LevelDev Lv, double* x, int64_t ldx, int nrhs, double* ubuf, int64_t ldu,
                int per_warp_bytes) {
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char smraw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = blockIdx.x * (blockDim.x >> 5) + warp;
  if (c >= Lv.ncell) return;
  unsigned char* base = smraw + (size_t)warp * per_warp_bytes;
  uint64_t* bar = nullptr;
  const T* band = STAGE ? leaf_stage<T>(Lv, c, base, &bar) : leaf_inplace<T>(Lv, c);
  T* y = (T*)(base + 16 + (STAGE ? leaf_band_bytes<T>(Lv.max_nI, Lv.max_w) : 0));
  T* z = y + Lv.max_nI + 1;
  const int nI = Lv.nI[c], nB = Lv.nB[c], w = Lv.band_w[c];
  const int32_t* gI = Lv.gids + Lv.gid_off[c];
  const int* ci = Lv.cpl_i + Lv.b_off[c];
  const T* ca = (const T*)Lv.cpl_a + Lv.b_off[c];
  pdl_wait();   // the vectors come from the previous kernel of the sweep
  for (int r = blockIdx.y; r < nrhs; r += gridDim.y) {   // right-hand sides over grid.y
    double* xr = x + r * ldx;
    warp_gather(xr, gI, nI, y);
    if (STAGE && r == (int)blockIdx.y && !staged_ok(bar, Lv.status, 0, kKindCell, c)) return;
    __syncwarp();
    band_fwd(band, nI, w, y);
    for (int i = lane; i < nI; i += 32) {
      xr[gI[i]] = double(y[i]);
      z[i] = y[i];
    }
    __syncwarp();
    band_bwd(band, nI, w, z);
    double* u = ubuf + r * ldu + Lv.b_off[c];
    for (int b = lane; b < nB; b += 32) u[b] = ci[b] >= 0 ? double(ca[b] * z[ci[b]]) : 0.0;
    __syncwarp();
  }
}

// E_0 per leaf: x_I = L^{-T}(x_I - L^{-1} A_BI^T x_B)
template <typename T, bool STAGE>
__global__ void __launch_bounds__(32 * kLeafWarps)
k_apply_leaf_down(LevelDev Lv, double* x, int64_t ldx, int nrhs, int per_warp_bytes) {
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char smraw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = blockIdx.x * (blockDim.x >> 5) + warp;
  if (c >= Lv.ncell) return;
  unsigned char* base = smraw + (size_t)warp * per_warp_bytes;
  uint64_t* bar = nullptr;
  const T* band = STAGE ? leaf_stage<T>(Lv, c, base, &bar) : leaf_inplace<T>(Lv, c);
  T* t = (T*)(base + 16 + (STAGE ? leaf_band_bytes<T>(Lv.max_nI, Lv.max_w) : 0));
  T* v = t + Lv.max_nI + 1;
  const int nI = Lv.nI[c], nB = Lv.nB[c], w = Lv.band_w[c];
  const int32_t* gI = Lv.gids + Lv.gid_off[c];
  const int32_t* gB = gI + nI;
  const int* ci = Lv.cpl_i + Lv.b_off[c];
  const T* ca = (const T*)Lv.cpl_a + Lv.b_off[c];
  T* xb = v + Lv.max_nI + 1;   // boundary values
  pdl_wait();   // the vectors come from the previous kernel of the sweep
  for (int r = blockIdx.y; r < nrhs; r += gridDim.y) {   // right-hand sides over grid.y
    double* xr = x + r * ldx;
    for (int i = lane; i < nI; i += 32) v[i] = T(0);
    warp_gather(xr, gI, nI, t);
#pragma unroll 2
    for (int b = lane; b < nB; b += 32) xb[b] = ci[b] >= 0 ? ca[b] * T(xr[gB[b]]) : T(0);
    __syncwarp();
    if (lane == 0)   // A_BI^T x_B in a fixed order (several boundary DOFs may face one interior DOF)
      for (int b = 0; b < nB; ++b)
        if (ci[b] >= 0) v[ci[b]] += xb[b];
    if (STAGE && r == (int)blockIdx.y && !staged_ok(bar, Lv.status, 0, kKindCell, c)) return;
    __syncwarp();
    band_fwd(band, nI, w, v);
    for (int i = lane; i < nI; i += 32) t[i] -= v[i];
    __syncwarp();
    band_bwd(band, nI, w, t);
    for (int i = lane; i < nI; i += 32) xr[gI[i]] = double(t[i]);
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// level 0, many right-hand sides: one warp per (leaf, 32 right-hand sides),
// lane = right-hand side.  The band (inverted diagonal blocks, w <= 15) is
// staged once in shared memory and read as broadcasts; each lane solves its
// own vector with the operations of warp_band_{fwd,bwd}_inv in the same
// order.  The vectors sit in shared memory with a row of 33 per DOF
// (v[i * 33 + r]): gathers and scatters run one right-hand side at a time with
// the lanes over DOFs (coalesced along the leaf's rows), the solves one lane
// per right-hand side (conflict-free).
// ---------------------------------------------------------------------------

constexpr int kMrLd = 33;

// Solves with the half bandwidth W a compile-time constant: the rows of the
// previous (next) block that couple into the current one stay in registers,
// so a block reads only its band entries (broadcasts) from shared memory.
template <typename T, int W>
__device__ inline void lane_band_fwd_w(const T* band, int n, T* v) {
  const int lane = threadIdx.x & 31;
  constexpr int w1 = W + 1;
  T prev[W];   // outputs of the previous block, row s0 - W + q in prev[q]
#pragma unroll
  for (int q = 0; q < W; ++q) prev[q] = T(0);
  for (int s0 = 0; s0 < n; s0 += W) {
    const int B = min(W, n - s0);
    T acc[W];
#pragma unroll
    for (int r = 0; r < W; ++r) {
      const int i = s0 + r;
      T a = r < B ? v[i * kMrLd + lane] : T(0);
#pragma unroll
      for (int d = 1; d <= kBandRegW; ++d) {   // the one-vector kernel's order: d ascending
        if (d > W || d <= r) continue;
        const int j = i - d;
        const bool ok = j >= 0 && r < B;
        const T cp = ok ? band[j * w1 + d] : T(0);
        a -= cp * (ok ? prev[W + r - d] : T(0));
      }
      acc[r] = a;
    }
#pragma unroll
    for (int r = 0; r < W; ++r) {
      T out = T(0);
#pragma unroll
      for (int c = 0; c < kBandRegW; ++c) {
        if (c >= W) continue;
        const T xr = (c <= r && r < B && c < B) ? band[(s0 + c) * w1 + (r - c)] : T(0);
        out += xr * (c < B ? acc[c] : T(0));
      }
      if (r < B) v[(s0 + r) * kMrLd + lane] = out;
      prev[r] = out;
    }
  }
}

template <typename T, int W>
__device__ inline void lane_band_bwd_w(const T* band, int n, T* v) {
  const int lane = threadIdx.x & 31;
  constexpr int w1 = W + 1;
  const int nblk = (n + W - 1) / W;
  T next[W];   // outputs of the next block, row s0 + B + q in next[q]
#pragma unroll
  for (int q = 0; q < W; ++q) next[q] = T(0);
  for (int bi = nblk - 1; bi >= 0; --bi) {
    const int s0 = bi * W;
    const int B = min(W, n - s0);
    T acc[W];
#pragma unroll
    for (int r = 0; r < W; ++r) {
      const int i = s0 + r;
      T a = r < B ? v[i * kMrLd + lane] : T(0);
      // couplings to the next block (only a full block has one: the last
      // block is the only partial one)
      if (B == W) {
#pragma unroll
        for (int d = 1; d <= kBandRegW; ++d) {
          if (d > W || r + d - W < 0) continue;
          const int j = i + d;
          const bool ok = j < n;
          const T cp = ok ? band[i * w1 + d] : T(0);
          a -= cp * (ok ? next[r + d - W] : T(0));
        }
      }
      acc[r] = a;
    }
#pragma unroll
    for (int r = 0; r < W; ++r) {
      T out = T(0);
#pragma unroll
      for (int c = 0; c < kBandRegW; ++c) {
        if (c >= W) continue;
        const T xc = (c >= r && c < B && r < B) ? band[(s0 + r) * w1 + (c - r)] : T(0);
        out += xc * (c < B ? acc[c] : T(0));
      }
      if (r < B) v[(s0 + r) * kMrLd + lane] = out;
      acc[r] = out;
    }
#pragma unroll
    for (int r = 0; r < W; ++r) next[r] = acc[r];
  }
}

template <typename T>
__device__ inline void lane_band_fwd_inv(const T* band, int n, int w, T* v) {
  switch (w) {
#define RHIF_W(k) case k: lane_band_fwd_w<T, k>(band, n, v); break;
    RHIF_W(1) RHIF_W(2) RHIF_W(3) RHIF_W(4) RHIF_W(5) RHIF_W(6) RHIF_W(7) RHIF_W(8)
    RHIF_W(9) RHIF_W(10) RHIF_W(11) RHIF_W(12) RHIF_W(13) RHIF_W(14) RHIF_W(15)
#undef RHIF_W
    default: break;
  }
}

template <typename T>
__device__ inline void lane_band_bwd_inv(const T* band, int n, int w, T* v) {
  switch (w) {
#define RHIF_W(k) case k: lane_band_bwd_w<T, k>(band, n, v); break;
    RHIF_W(1) RHIF_W(2) RHIF_W(3) RHIF_W(4) RHIF_W(5) RHIF_W(6) RHIF_W(7) RHIF_W(8)
    RHIF_W(9) RHIF_W(10) RHIF_W(11) RHIF_W(12) RHIF_W(13) RHIF_W(14) RHIF_W(15)
#undef RHIF_W
    default: break;
  }
}

// Per-warp shared memory of the many-right-hand-side leaf kernels: the band,
// two vectors of max_nI rows and one of max_nB rows, kMrLd entries a row.
template <typename T>
__host__ __device__ inline size_t leaf_mr_bytes(int max_nI, int max_nB, int max_w) {
  return round16((size_t)max_nI * (max_w + 1) * sizeof(T)) +
         2 * round16((size_t)max_nI * kMrLd * sizeof(T)) + round16((size_t)max_nB * kMrLd * sizeof(T));
}

// v[i * kMrLd + r] = T(x[g[i] + (r0 + r) ldx]) for i < n, r < 32 (0 for r >= R,
// or where ci[i] < 0 when ci is given): lanes along i, eight right-hand sides'
// loads in flight before their stores.
template <typename T>
__device__ inline void mr_gather(const double* x, int64_t ldx, int r0, int R, const int32_t* g,
                                 int n, T* v, const int* ci = nullptr) {
  const int lane = threadIdx.x & 31;
  for (int i = lane; i < n; i += 32) {
    const bool use = !ci || ci[i] >= 0;
    const int64_t gi = g[i];
    for (int rb = 0; rb < 32; rb += 8) {
      double t[8];
#pragma unroll
      for (int q = 0; q < 8; ++q)
        t[q] = (use && rb + q < R) ? x[gi + (int64_t)(r0 + rb + q) * ldx] : 0.0;
#pragma unroll
      for (int q = 0; q < 8; ++q) v[i * kMrLd + rb + q] = T(t[q]);
    }
  }
  __syncwarp();
}

// x[g[i] + (r0 + r) ldx] = double(v[i * kMrLd + r]) for i < n, r < R.
template <typename T>
__device__ inline void mr_scatter(double* x, int64_t ldx, int r0, int R, const int32_t* g, int n,
                                  const T* v) {
  const int lane = threadIdx.x & 31;
  __syncwarp();
  for (int i = lane; i < n; i += 32) {
    const int64_t gi = g[i];
    for (int r = 0; r < R; ++r) x[gi + (int64_t)(r0 + r) * ldx] = double(v[i * kMrLd + r]);
  }
}

template <typename T>
__device__ inline const T* leaf_mr_stage(const LevelDev& Lv, int c, unsigned char* base) {
  const int lane = threadIdx.x & 31;
  T* sb = (T*)base;
  const T* g = (const T*)Lv.band + Lv.band_off[c];
  const int cnt = Lv.nI[c] * (Lv.band_w[c] + 1);
  for (int i = lane; i < cnt; i += 32) sb[i] = g[i];
  __syncwarp();
  return sb;
}

// E_0^T per leaf for right-hand sides r0 + lane, r0 = 32 blockIdx.y, 32 (blockIdx.y +
// gridDim.y), ...: as k_apply_leaf_up.
template <typename T>
__global__ void __launch_bounds__(128)
k_apply_leaf_up_mr(LevelDev Lv, double* x, int64_t ldx, int nrhs, double* ubuf, int64_t ldu,
                   int per_warp_bytes) {
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char smraw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = blockIdx.x * (blockDim.x >> 5) + warp;
  if (c >= Lv.ncell) return;
  unsigned char* base = smraw + (size_t)warp * per_warp_bytes;
  const T* band = leaf_mr_stage<T>(Lv, c, base);
  T* y = (T*)(base + round16((size_t)Lv.max_nI * (Lv.max_w + 1) * sizeof(T)));
  T* z = y + (round16((size_t)Lv.max_nI * kMrLd * sizeof(T)) / sizeof(T));
  const int nI = Lv.nI[c], nB = Lv.nB[c], w = Lv.band_w[c];
  const int32_t* gI = Lv.gids + Lv.gid_off[c];
  const int* ci = Lv.cpl_i + Lv.b_off[c];
  const T* ca = (const T*)Lv.cpl_a + Lv.b_off[c];
  pdl_wait();   // the vectors come from the previous kernel of the sweep
  for (int r0 = blockIdx.y * 32; r0 < nrhs; r0 += gridDim.y * 32) {
    const int R = min(32, nrhs - r0);
    mr_gather<T>(x, ldx, r0, R, gI, nI, y);
    lane_band_fwd_inv(band, nI, w, y);
    for (int i = 0; i < nI; ++i) z[i * kMrLd + lane] = y[i * kMrLd + lane];
    __syncwarp();
    mr_scatter<T>(x, ldx, r0, R, gI, nI, y);
    lane_band_bwd_inv(band, nI, w, z);
    __syncwarp();
    for (int r = 0; r < R; ++r) {
      double* u = ubuf + (int64_t)(r0 + r) * ldu + Lv.b_off[c];
      for (int b = lane; b < nB; b += 32)
        u[b] = ci[b] >= 0 ? double(ca[b] * z[ci[b] * kMrLd + r]) : 0.0;
    }
    __syncwarp();
  }
}

// E_0 per leaf for right-hand sides r0 + lane (as above): as k_apply_leaf_down.
template <typename T>
__global__ void __launch_bounds__(128)
k_apply_leaf_down_mr(LevelDev Lv, double* x, int64_t ldx, int nrhs, int per_warp_bytes) {
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char smraw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = blockIdx.x * (blockDim.x >> 5) + warp;
  if (c >= Lv.ncell) return;
  unsigned char* base = smraw + (size_t)warp * per_warp_bytes;
  const T* band = leaf_mr_stage<T>(Lv, c, base);
  T* t = (T*)(base + round16((size_t)Lv.max_nI * (Lv.max_w + 1) * sizeof(T)));
  T* v = t + (round16((size_t)Lv.max_nI * kMrLd * sizeof(T)) / sizeof(T));
  T* xb = v + (round16((size_t)Lv.max_nI * kMrLd * sizeof(T)) / sizeof(T));
  const int nI = Lv.nI[c], nB = Lv.nB[c], w = Lv.band_w[c];
  const int32_t* gI = Lv.gids + Lv.gid_off[c];
  const int32_t* gB = gI + nI;
  const int* ci = Lv.cpl_i + Lv.b_off[c];
  const T* ca = (const T*)Lv.cpl_a + Lv.b_off[c];
  pdl_wait();   // the vectors come from the previous kernel of the sweep
  for (int r0 = blockIdx.y * 32; r0 < nrhs; r0 += gridDim.y * 32) {
    const int R = min(32, nrhs - r0);
    mr_gather<T>(x, ldx, r0, R, gI, nI, t);
    mr_gather<T>(x, ldx, r0, R, gB, nB, xb, ci);   // coupled boundary values only
    for (int b = lane; b < nB; b += 32)
      if (ci[b] >= 0)
        for (int r = 0; r < 32; ++r) xb[b * kMrLd + r] *= ca[b];
    for (int i = 0; i < nI; ++i) v[i * kMrLd + lane] = T(0);
    __syncwarp();
    for (int b = 0; b < nB; ++b)   // A_BI^T x_B in boundary order, as the one-vector kernel
      if (ci[b] >= 0) v[ci[b] * kMrLd + lane] += xb[b * kMrLd + lane];
    lane_band_fwd_inv(band, nI, w, v);
    for (int i = 0; i < nI; ++i) t[i * kMrLd + lane] -= v[i * kMrLd + lane];
    lane_band_bwd_inv(band, nI, w, t);
    __syncwarp();
    mr_scatter<T>(x, ldx, r0, R, gI, nI, t);
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// dense fronts (levels >= 1 and the root)
// ---------------------------------------------------------------------------

// Starts the bulk copy of the first nI columns of the front (n x nI, contiguous).
template <typename T>
__device__ inline const T* front_stage(const T* F, int n, int nI, T* dst, uint64_t* bar) {
  if (threadIdx.x == 0) {
    const uint32_t bytes = round16((size_t)n * nI * sizeof(T));
    mbar_init(bar, 1);
    mbar_expect_tx(bar, bytes);
    if (bytes) bulk_g2s(dst, F, bytes, bar);
  }
  return dst;
}

// RC right-hand sides per pass (1, or 8 when there are many): each element of
// the front read from shared memory serves RC products; every right-hand side
// keeps the summation order of the one-vector pass.
template <typename T, int RC>
__global__ void __launch_bounds__(kApplyThreads)
k_apply_cell_up(LevelDev Lv, double* x, int64_t ldx, int nrhs, double* ubuf, int64_t ldu,
                int stage) {
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ __align__(8) uint64_t bar;
  const int ld = Lv.max_nI + 1;
  T* x_in = (T*)smraw;
  T* y = x_in + RC * ld;
  const int c = blockIdx.x;
  const int nI = Lv.nI[c], nB = Lv.nB[c], n = nI + nB;
  const T* F = (const T*)Lv.front + Lv.front_off[c];
  if (stage) F = front_stage(F, n, nI, (T*)(smraw + round16(2 * RC * ld * sizeof(T))), &bar);
  const int32_t* gI = Lv.gids + Lv.gid_off[c];
  __syncthreads();
  pdl_wait();   // the vectors come from the previous kernel of the sweep
  for (int r0 = blockIdx.y * RC; r0 < nrhs; r0 += gridDim.y * RC) {   // chunks over grid.y
    const int rc = min(RC, nrhs - r0);
    for (int idx = threadIdx.x; idx < rc * nI; idx += blockDim.x) {
      const int q = idx / nI, i = idx % nI;
      x_in[q * ld + i] = T(x[(int64_t)(r0 + q) * ldx + gI[i]]);
    }
    if (stage && r0 == (int)blockIdx.y * RC &&
        !staged_ok(&bar, Lv.status, Lv.level, kKindCell, c))
      return;
    __syncthreads();
    // y = L^{-1} x_I: the front's L block holds L^{-1} (one row per thread)
    for (int i = threadIdx.x; i < nI; i += blockDim.x) {
      T sq[RC];
#pragma unroll
      for (int q = 0; q < RC; ++q) sq[q] = T(0);
      for (int k = 0; k <= i; ++k) {
        const T f = F[i + (int64_t)k * n];
#pragma unroll
        for (int q = 0; q < RC; ++q)
          if (q < rc) sq[q] += f * x_in[q * ld + k];
      }
#pragma unroll
      for (int q = 0; q < RC; ++q)
        if (q < rc) y[q * ld + i] = sq[q];
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < rc * nI; idx += blockDim.x) {
      const int q = idx / nI, i = idx % nI;
      x[(int64_t)(r0 + q) * ldx + gI[i]] = double(y[q * ld + i]);
    }
    for (int b = threadIdx.x; b < nB; b += blockDim.x) {
      T sq[RC];
#pragma unroll
      for (int q = 0; q < RC; ++q) sq[q] = T(0);
      for (int k = 0; k < nI; ++k) {
        const T f = F[(nI + b) + (int64_t)k * n];
#pragma unroll
        for (int q = 0; q < RC; ++q)
          if (q < rc) sq[q] += f * y[q * ld + k];
      }
#pragma unroll
      for (int q = 0; q < RC; ++q)
        if (q < rc) ubuf[(int64_t)(r0 + q) * ldu + Lv.b_off[c] + b] = double(sq[q]);
    }
    __syncthreads();
  }
}

template <typename T, int RC>
__global__ void __launch_bounds__(kApplyThreads)
k_apply_cell_down(LevelDev Lv, double* x, int64_t ldx, int nrhs, int stage) {
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ __align__(8) uint64_t bar;
  const int ldi = Lv.max_nI, ldb = Lv.max_nB + 1;
  T* t = (T*)smraw;
  T* xb = t + RC * ldi;
  T* xo = xb + RC * ldb;
  const int c = blockIdx.x;
  const int nI = Lv.nI[c], nB = Lv.nB[c], n = nI + nB;
  const T* F = (const T*)Lv.front + Lv.front_off[c];
  if (stage)
    F = front_stage(F, n, nI,
                    (T*)(smraw + round16(RC * (2 * Lv.max_nI + Lv.max_nB + 1) * sizeof(T))), &bar);
  const int32_t* gI = Lv.gids + Lv.gid_off[c];
  const int32_t* gB = gI + nI;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  __syncthreads();
  pdl_wait();   // the vectors come from the previous kernel of the sweep
  for (int r0 = blockIdx.y * RC; r0 < nrhs; r0 += gridDim.y * RC) {   // chunks over grid.y
    const int rc = min(RC, nrhs - r0);
    for (int idx = threadIdx.x; idx < rc * nB; idx += blockDim.x) {
      const int q = idx / nB, b = idx % nB;
      xb[q * ldb + b] = T(x[(int64_t)(r0 + q) * ldx + gB[b]]);
    }
    if (stage && r0 == (int)blockIdx.y * RC &&
        !staged_ok(&bar, Lv.status, Lv.level, kKindCell, c))
      return;
    __syncthreads();
    for (int k = warp; k < nI; k += nwarps) {
      T sq[RC];
#pragma unroll
      for (int q = 0; q < RC; ++q) sq[q] = T(0);
      for (int b = lane; b < nB; b += 32) {
        const T f = F[(nI + b) + (int64_t)k * n];
#pragma unroll
        for (int q = 0; q < RC; ++q)
          if (q < rc) sq[q] += f * xb[q * ldb + b];
      }
#pragma unroll
      for (int q = 0; q < RC; ++q) {
        if (q >= rc) break;
        const T sr = warp_sum(sq[q]);
        if (lane == 0) t[q * ldi + k] = T(x[(int64_t)(r0 + q) * ldx + gI[k]]) - sr;
      }
    }
    __syncthreads();
    // x_I = L^{-T} t: the front's L block holds L^{-1}; one row per warp
    for (int i = warp; i < nI; i += nwarps) {
      T sq[RC];
#pragma unroll
      for (int q = 0; q < RC; ++q) sq[q] = T(0);
      for (int k = i + lane; k < nI; k += 32) {
        const T f = F[k + (int64_t)i * n];
#pragma unroll
        for (int q = 0; q < RC; ++q)
          if (q < rc) sq[q] += f * t[q * ldi + k];
      }
#pragma unroll
      for (int q = 0; q < RC; ++q) {
        if (q >= rc) break;
        const T sr = warp_sum(sq[q]);
        if (lane == 0) xo[q * ldi + i] = sr;
      }
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < rc * nI; idx += blockDim.x) {
      const int q = idx / nI, i = idx % nI;
      x[(int64_t)(r0 + q) * ldx + gI[i]] = double(xo[q * ldi + i]);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// cells of levels with large fronts, whose L block holds L^{-1} (explicit
// inverse taken at factorization): each sweep is two launches of row-parallel
// products over many CTAs, with y / t kept in a scratch column `tmp` at the
// cell's DOF-list offset.  Right-hand sides go in chunks of `rc` (<= 4), the
// chunk's input vector staged in shared memory.
//   up:   y = L^{-1} x_I ;  x_I = y, u_B = W y       (W = rows nI..n of the front)
//   down: t = x_I - W^T x_B ;  x_I = L^{-T} t
// ---------------------------------------------------------------------------

constexpr int kBigRows = 128;   // rows per CTA (one per thread) in up1 / up2
constexpr int kBigWarps = 8;    // rows per CTA (one per warp) in down1 / down2

template <typename T>
__global__ void __launch_bounds__(kBigRows)
k_apply_big_up1(LevelDev Lv, const double* x, int64_t ldx, int nrhs, int rc, double* tmp,
                int64_t ldt) {
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char smraw[];
  T* xs = (T*)smraw;   // [kend][rc]
  const int c = blockIdx.y;
  const int nI = Lv.nI[c];
  const int r0 = blockIdx.x * kBigRows;
  if (r0 >= nI) return;
  const int n = nI + Lv.nB[c];
  const int i = r0 + threadIdx.x;
  const int kend = min(nI, r0 + kBigRows);
  const T* F = (const T*)Lv.front + Lv.front_off[c];
  const int32_t* gI = Lv.gids + Lv.gid_off[c];
  double* tc = tmp + Lv.gid_off[c];
  pdl_wait();   // the vectors come from the previous kernel of the sweep
  for (int q0 = 0; q0 < nrhs; q0 += rc) {
    const int nr = min(rc, nrhs - q0);
    __syncthreads();
    for (int idx = threadIdx.x; idx < kend * nr; idx += blockDim.x) {
      const int k = idx / nr, rr = idx % nr;
      xs[k * rc + rr] = T(x[(int64_t)(q0 + rr) * ldx + gI[k]]);
    }
    __syncthreads();
    T acc[4] = {T(0), T(0), T(0), T(0)};
    const int kl = i < nI ? min(i + 1, kend) : 0;
#pragma unroll 4
    for (int k = 0; k < kl; ++k) {
      const T l = F[i + (int64_t)k * n];
#pragma unroll
      for (int rr = 0; rr < 4; ++rr)
        if (rr < nr) acc[rr] += l * xs[k * rc + rr];
    }
    if (i < nI)
      for (int rr = 0; rr < nr; ++rr) tc[(int64_t)(q0 + rr) * ldt + i] = double(acc[rr]);
  }
}

template <typename T>
__global__ void __launch_bounds__(kBigRows)
k_apply_big_up2(LevelDev Lv, double* x, int64_t ldx, int nrhs, int rc, double* ubuf, int64_t ldu,
                const double* tmp, int64_t ldt) {
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char smraw[];
  T* ys = (T*)smraw;   // [nI][rc]
  const int c = blockIdx.y;
  const int nI = Lv.nI[c], nB = Lv.nB[c], n = nI + nB;
  const int r0 = blockIdx.x * kBigRows;
  if (r0 >= max(nI, nB)) return;
  const int row = r0 + threadIdx.x;
  const T* F = (const T*)Lv.front + Lv.front_off[c];
  const int32_t* gI = Lv.gids + Lv.gid_off[c];
  const double* tc = tmp + Lv.gid_off[c];
  pdl_wait();   // the vectors come from the previous kernel of the sweep
  for (int q0 = 0; q0 < nrhs; q0 += rc) {
    const int nr = min(rc, nrhs - q0);
    if (row < nI)
      for (int rr = 0; rr < nr; ++rr)
        x[(int64_t)(q0 + rr) * ldx + gI[row]] = tc[(int64_t)(q0 + rr) * ldt + row];
    if (r0 >= nB) continue;
    __syncthreads();
    for (int idx = threadIdx.x; idx < nI * nr; idx += blockDim.x) {
      const int k = idx / nr, rr = idx % nr;
      ys[k * rc + rr] = T(tc[(int64_t)(q0 + rr) * ldt + k]);
    }
    __syncthreads();
    if (row < nB) {
      T acc[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll 4
      for (int k = 0; k < nI; ++k) {
        const T w = F[(nI + row) + (int64_t)k * n];
#pragma unroll
        for (int rr = 0; rr < 4; ++rr)
          if (rr < nr) acc[rr] += w * ys[k * rc + rr];
      }
      for (int rr = 0; rr < nr; ++rr)
        ubuf[(int64_t)(q0 + rr) * ldu + Lv.b_off[c] + row] = double(acc[rr]);
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(32 * kBigWarps)
k_apply_big_down1(LevelDev Lv, const double* x, int64_t ldx, int nrhs, int rc, double* tmp,
                  int64_t ldt) {
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char smraw[];
  T* xb = (T*)smraw;   // [nB][rc]
  const int c = blockIdx.y;
  const int nI = Lv.nI[c], nB = Lv.nB[c], n = nI + nB;
  const int r0 = blockIdx.x * kBigWarps;
  if (r0 >= nI) return;
  const int lane = threadIdx.x & 31, i = r0 + (threadIdx.x >> 5);
  const T* F = (const T*)Lv.front + Lv.front_off[c];
  const int32_t* gI = Lv.gids + Lv.gid_off[c];
  const int32_t* gB = gI + nI;
  double* tc = tmp + Lv.gid_off[c];
  pdl_wait();   // the vectors come from the previous kernel of the sweep
  for (int q0 = 0; q0 < nrhs; q0 += rc) {
    const int nr = min(rc, nrhs - q0);
    __syncthreads();
    for (int idx = threadIdx.x; idx < nB * nr; idx += blockDim.x) {
      const int b = idx / nr, rr = idx % nr;
      xb[b * rc + rr] = T(x[(int64_t)(q0 + rr) * ldx + gB[b]]);
    }
    __syncthreads();
    if (i >= nI) continue;
    T acc[4] = {T(0), T(0), T(0), T(0)};
    for (int b = lane; b < nB; b += 32) {
      const T w = F[(nI + b) + (int64_t)i * n];
#pragma unroll
      for (int rr = 0; rr < 4; ++rr)
        if (rr < nr) acc[rr] += w * xb[b * rc + rr];
    }
#pragma unroll
    for (int rr = 0; rr < 4; ++rr) acc[rr] = warp_sum(acc[rr]);
    if (lane < nr) {
      T a = acc[0];
#pragma unroll
      for (int rr = 1; rr < 4; ++rr)
        if (lane == rr) a = acc[rr];
      tc[(int64_t)(q0 + lane) * ldt + i] = x[(int64_t)(q0 + lane) * ldx + gI[i]] - double(a);
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(32 * kBigWarps)
k_apply_big_down2(LevelDev Lv, double* x, int64_t ldx, int nrhs, int rc, const double* tmp,
                  int64_t ldt) {
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char smraw[];
  T* ts = (T*)smraw;   // [nI][rc]
  const int c = blockIdx.y;
  const int nI = Lv.nI[c], n = nI + Lv.nB[c];
  const int r0 = blockIdx.x * kBigWarps;
  if (r0 >= nI) return;
  const int lane = threadIdx.x & 31, i = r0 + (threadIdx.x >> 5);
  const T* F = (const T*)Lv.front + Lv.front_off[c];
  const int32_t* gI = Lv.gids + Lv.gid_off[c];
  const double* tc = tmp + Lv.gid_off[c];
  pdl_wait();   // the vectors come from the previous kernel of the sweep
  for (int q0 = 0; q0 < nrhs; q0 += rc) {
    const int nr = min(rc, nrhs - q0);
    __syncthreads();
    for (int idx = threadIdx.x; idx < (nI - r0) * nr; idx += blockDim.x) {
      const int k = r0 + idx / nr, rr = idx % nr;
      ts[(k - r0) * rc + rr] = T(tc[(int64_t)(q0 + rr) * ldt + k]);
    }
    __syncthreads();
    if (i >= nI) continue;
    T acc[4] = {T(0), T(0), T(0), T(0)};
    for (int k = i + lane; k < nI; k += 32) {
      const T l = F[k + (int64_t)i * n];
#pragma unroll
      for (int rr = 0; rr < 4; ++rr)
        if (rr < nr) acc[rr] += l * ts[(k - r0) * rc + rr];
    }
#pragma unroll
    for (int rr = 0; rr < 4; ++rr) acc[rr] = warp_sum(acc[rr]);
    if (lane < nr) {
      T a = acc[0];
#pragma unroll
      for (int rr = 1; rr < 4; ++rr)
        if (lane == rr) a = acc[rr];
      x[(int64_t)(q0 + lane) * ldx + gI[i]] = double(a);
    }
  }
}

// ---------------------------------------------------------------------------
// separator groups: C_l and K_l
// ---------------------------------------------------------------------------

// Layout of a group's staged blocks: [L_g | unit front | T], each padded to 16 bytes.
template <typename T>
__host__ __device__ inline size_t group_block_bytes(int n) {
  const size_t nn = (size_t)n * n;
  return 2 * round16(nn * sizeof(T)) + round16(nn / 4 * sizeof(T) + 16);
}

// Starts the bulk copies of the group's blocks (issued by `leader`).
template <typename T>
__device__ inline void group_stage(const PhaseDev& Ph, int pi, int u, int n, unsigned char* dst,
                                   uint64_t* bar, bool leader, const T** Lg, const T** Fu,
                                   const T** Tm) {
  const size_t nn = (size_t)n * n;
  T* sL = (T*)dst;
  T* sF = (T*)(dst + round16(nn * sizeof(T)));
  T* sT = (T*)(dst + 2 * round16(nn * sizeof(T)));
  *Lg = pi >= 0 ? sL : nullptr;
  *Fu = u >= 0 ? sF : nullptr;
  *Tm = u >= 0 ? sT : nullptr;
  if (!leader) return;
  uint32_t total = 0;
  const uint32_t bL = round16(nn * sizeof(T));
  uint32_t bT = 0;
  if (pi >= 0) total += bL;
  if (u >= 0) {
    const int k = Ph.rank[u];
    bT = round16((size_t)k * (n - k) * sizeof(T));
    total += bL + bT;
  }
  mbar_init(bar, 1);
  mbar_expect_tx(bar, total);
  if (pi >= 0) bulk_g2s(sL, (const T*)Ph.Lbuf + Ph.pre_off[pi], bL, bar);
  if (u >= 0) {
    const T* src = (const T*)Ph.rec + Ph.u_rec_off[u];
    bulk_g2s(sF, src, bL, bar);
    if (bT) bulk_g2s(sT, src + pad4e((int64_t)nn), bT, bar);
  }
}

// out = X in and out = X^T in for a lower-triangular n x n X (ld), in and
// out in shared memory (distinct).  The factor stores the inverses of the
// block-Jacobi factors L_g and of the units' L_rr, so every step of the group
// application is a product.
template <typename T>
__device__ inline void cta_trmv_lower(const T* X, int64_t ld, int n, const T* in, T* out) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    T s = T(0);
    for (int j = 0; j <= i; ++j) s += X[i + (int64_t)j * ld] * in[j];
    out[i] = s;
  }
}

template <typename T>
__device__ inline void cta_trmv_lower_t(const T* X, int64_t ld, int n, const T* in, T* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (int i = warp; i < n; i += nwarps) {
    T s = T(0);
    for (int j = i + lane; j < n; j += 32) s += X[j + (int64_t)i * ld] * in[j];
    s = warp_sum(s);
    if (lane == 0) out[i] = s;
  }
}

// K_l^T of one unit on its group's values xg (Fu holds L_rr^{-1} and W):
// x_rd -= T^T x_sk ; y = L_rr^{-1} x_rd ; x_sk -= W y ; x_rd = y
template <typename T>
__device__ void unit_up(const PhaseDev& Ph, int u, int n, T* xg, T* tmp, const T* Fu, const T* Tm) {
  const int k = Ph.rank[u], r = n - k;
  const int* perm = Ph.perm + Ph.u_perm_off[u];
  for (int a = threadIdx.x; a < r; a += blockDim.x) {
    T s = xg[perm[k + a]];
    for (int q = 0; q < k; ++q) s -= Tm[q + (int64_t)a * k] * xg[perm[q]];
    tmp[a] = s;
  }
  __syncthreads();
  for (int a = threadIdx.x; a < r; a += blockDim.x) {   // y into the redundant slots
    T s = T(0);
    for (int c = 0; c <= a; ++c) s += Fu[a + (int64_t)c * n] * tmp[c];
    xg[perm[k + a]] = s;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < k; q += blockDim.x) {
    T s = xg[perm[q]];
    for (int a = 0; a < r; ++a) s -= Fu[(r + q) + (int64_t)a * n] * xg[perm[k + a]];
    xg[perm[q]] = s;
  }
  __syncthreads();
}

// K_l of one unit: x_rd = L_rr^{-T} (x_rd - W^T x_sk) ; x_sk -= T x_rd
template <typename T>
__device__ void unit_down(const PhaseDev& Ph, int u, int n, T* xg, T* tmp, const T* Fu, const T* Tm) {
  const int k = Ph.rank[u], r = n - k;
  const int* perm = Ph.perm + Ph.u_perm_off[u];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (int a = warp; a < r; a += nwarps) {
    T s = T(0);
    for (int q = lane; q < k; q += 32) s += Fu[(r + q) + (int64_t)a * n] * xg[perm[q]];
    s = warp_sum(s);
    if (lane == 0) tmp[a] = xg[perm[k + a]] - s;
  }
  __syncthreads();
  for (int a = warp; a < r; a += nwarps) {   // y = L_rr^{-T} tmp into the redundant slots
    T s = T(0);
    for (int c = a + lane; c < r; c += 32) s += Fu[c + (int64_t)a * n] * tmp[c];
    s = warp_sum(s);
    if (lane == 0) xg[perm[k + a]] = s;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < k; q += blockDim.x) {
    T s = xg[perm[q]];
    for (int a = 0; a < r; ++a) s -= Tm[q + (int64_t)a * k] * xg[perm[k + a]];
    xg[perm[q]] = s;
  }
  __syncthreads();
}

// Points Lg / Fu / Tm at the group's blocks in global memory.
template <typename T>
__device__ inline void group_global(const PhaseDev& Ph, int pi, int u, int n, const T** Lg,
                                    const T** Fu, const T** Tm) {
  *Lg = pi >= 0 ? (const T*)Ph.Lbuf + Ph.pre_off[pi] : nullptr;
  *Fu = u >= 0 ? (const T*)Ph.rec + Ph.u_rec_off[u] : nullptr;
  *Tm = u >= 0 ? *Fu + pad4e((int64_t)n * n) : nullptr;
}

template <typename T>
__global__ void __launch_bounds__(kGroupThreads)
k_apply_group_up(LevelDev Lv, PhaseDev Ph, int gather, double* x, int64_t ldx, int nrhs,
                 const double* ubuf, int64_t ldu, int stage) {
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ __align__(8) uint64_t bar;
  T* xg = (T*)smraw;
  T* tmp = xg + Lv.max_group;
  const int g = blockIdx.x;
  if (Lv.group_t[g] < Ph.pre_min_type) return;
  const int n = Lv.group_size[g];
  const int32_t* gid = Lv.bucket + Lv.group_start[g];
  const int pi = Ph.group_pre[g], u = Ph.group_unit[g];
  const T *Lg, *Fu, *Tm;
  if (stage)
    group_stage(Ph, pi, u, n, smraw + round16(2 * (Lv.max_group + 1) * sizeof(T)), &bar,
                threadIdx.x == 0, &Lg, &Fu, &Tm);
  else
    group_global(Ph, pi, u, n, &Lg, &Fu, &Tm);
  __syncthreads();
  pdl_wait();   // the vectors come from the previous kernel of the sweep
  for (int r = blockIdx.y; r < nrhs; r += gridDim.y) {   // right-hand sides over grid.y
    double* xr = x + r * ldx;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      double v = xr[gid[i]];
      if (gather) {
        for (int k = Lv.group_cell_off[g]; k < Lv.group_cell_off[g + 1]; ++k)
          v -= ubuf[r * ldu + Lv.b_off[Lv.group_cell[k]] + Lv.group_pos[k] + i];
      }
      xg[i] = T(v);
    }
    if (stage && r == (int)blockIdx.y && !staged_ok(&bar, Lv.status, Lv.level, kKindGroup, g)) return;
    __syncthreads();
    if (Lg) {   // C^T: x_g = L_g^{-1} x_g
      cta_trmv_lower(Lg, n, n, xg, tmp);
      __syncthreads();
      for (int i = threadIdx.x; i < n; i += blockDim.x) xg[i] = tmp[i];
      __syncthreads();
    }
    if (Fu) unit_up(Ph, u, n, xg, tmp, Fu, Tm);
    for (int i = threadIdx.x; i < n; i += blockDim.x) xr[gid[i]] = double(xg[i]);
    __syncthreads();
  }
}

template <typename T>
__global__ void __launch_bounds__(kGroupThreads)
k_apply_group_down(LevelDev Lv, PhaseDev Ph, double* x, int64_t ldx, int nrhs, int stage) {
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ __align__(8) uint64_t bar;
  T* xg = (T*)smraw;
  T* tmp = xg + Lv.max_group;
  const int g = blockIdx.x;
  if (Lv.group_t[g] < Ph.pre_min_type) return;
  const int n = Lv.group_size[g];
  const int32_t* gid = Lv.bucket + Lv.group_start[g];
  const int pi = Ph.group_pre[g], u = Ph.group_unit[g];
  const T *Lg, *Fu, *Tm;
  if (stage)
    group_stage(Ph, pi, u, n, smraw + round16(2 * (Lv.max_group + 1) * sizeof(T)), &bar,
                threadIdx.x == 0, &Lg, &Fu, &Tm);
  else
    group_global(Ph, pi, u, n, &Lg, &Fu, &Tm);
  __syncthreads();
  pdl_wait();   // the vectors come from the previous kernel of the sweep
  for (int r = blockIdx.y; r < nrhs; r += gridDim.y) {   // right-hand sides over grid.y
    double* xr = x + r * ldx;
    for (int i = threadIdx.x; i < n; i += blockDim.x) xg[i] = T(xr[gid[i]]);
    if (stage && r == (int)blockIdx.y && !staged_ok(&bar, Lv.status, Lv.level, kKindGroup, g)) return;
    __syncthreads();
    if (Fu) unit_down(Ph, u, n, xg, tmp, Fu, Tm);
    if (Lg) {   // C: x_g = L_g^{-T} x_g
      cta_trmv_lower_t(Lg, n, n, xg, tmp);
      __syncthreads();
      for (int i = threadIdx.x; i < n; i += blockDim.x) xg[i] = tmp[i];
      __syncthreads();
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) xr[gid[i]] = double(xg[i]);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// separator groups of at most 32 DOFs: one warp per group, values in registers
// ---------------------------------------------------------------------------

template <typename T>
static size_t group_warp_smem(int max_group) {
  return 16 + group_block_bytes<T>(max_group) + round16(max_group * sizeof(int));
}

template <typename T>
__global__ void __launch_bounds__(32 * kGroupWarps)
k_apply_group_up_warp(LevelDev Lv, PhaseDev Ph, int gather, double* x, int64_t ldx, int nrhs,
                      const double* ubuf, int64_t ldu, int per_warp_bytes) {
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char smraw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = blockIdx.x * kGroupWarps + warp;
  if (g >= Lv.ngroup || Lv.group_t[g] < Ph.pre_min_type) return;
  const int n = Lv.group_size[g];
  const int32_t* gid = Lv.bucket + Lv.group_start[g];
  const int pi = Ph.group_pre[g], u = Ph.group_unit[g];
  unsigned char* base = smraw + (size_t)warp * per_warp_bytes;
  uint64_t* bar = (uint64_t*)base;
  int* invp = (int*)(base + 16 + group_block_bytes<T>(Lv.max_group));
  const T *Lg, *Fu, *Tm;
  group_stage(Ph, pi, u, n, base + 16, bar, lane == 0, &Lg, &Fu, &Tm);
  const bool staged = pi >= 0 || u >= 0;
  const int k = u >= 0 ? Ph.rank[u] : 0;
  const int r = n - k;
  const int* perm = u >= 0 ? Ph.perm + Ph.u_perm_off[u] : nullptr;
  if (u >= 0 && lane < n) invp[perm[lane]] = lane;
  __syncwarp();
  const int p_sk = (u >= 0 && lane < k) ? perm[lane] : 0;
  const int p_rd = (u >= 0 && lane < r) ? perm[k + lane] : 0;
  const int my_idx = (u >= 0 && lane < n) ? invp[lane] : 0;
  pdl_wait();   // the vectors come from the previous kernel of the sweep
  for (int rr = blockIdx.y; rr < nrhs; rr += gridDim.y) {   // right-hand sides over grid.y
    double* xr = x + rr * ldx;
    T xv = T(0);
    if (lane < n) {
      double v = xr[gid[lane]];
      if (gather)
        for (int q = Lv.group_cell_off[g]; q < Lv.group_cell_off[g + 1]; ++q)
          v -= ubuf[rr * ldu + Lv.b_off[Lv.group_cell[q]] + Lv.group_pos[q] + lane];
      xv = T(v);
    }
    if (staged && rr == (int)blockIdx.y && !staged_ok(bar, Lv.status, Lv.level, kKindGroup, g)) return;
    if (Lg) {   // C^T: x_g = L_g^{-1} x_g (the factor keeps L_g^{-1})
      T y = T(0);
      for (int c = 0; c < n; ++c) {
        const T v = __shfl_sync(0xffffffffu, xv, c);
        if (c <= lane && lane < n) y += Lg[lane + c * n] * v;
      }
      xv = y;
    }
    if (u >= 0) {   // K^T: x_rd -= T^T x_sk ; y = L^{-1} x_rd ; x_sk -= W y ; x_rd = y
      T xs = __shfl_sync(0xffffffffu, xv, p_sk);
      T xd = __shfl_sync(0xffffffffu, xv, p_rd);
      for (int q = 0; q < k; ++q) {
        const T v = __shfl_sync(0xffffffffu, xs, q);
        if (lane < r) xd -= Tm[q + lane * k] * v;
      }
      {   // y = L_rr^{-1} x_rd
        T y = T(0);
        for (int c = 0; c < r; ++c) {
          const T v = __shfl_sync(0xffffffffu, xd, c);
          if (c <= lane && lane < r) y += Fu[lane + c * n] * v;
        }
        xd = y;
      }
      for (int a = 0; a < r; ++a) {
        const T v = __shfl_sync(0xffffffffu, xd, a);
        if (lane < k) xs -= Fu[(r + lane) + a * n] * v;
      }
      const T from_sk = __shfl_sync(0xffffffffu, xs, my_idx < k ? my_idx : 0);
      const T from_rd = __shfl_sync(0xffffffffu, xd, my_idx >= k ? my_idx - k : 0);
      xv = my_idx < k ? from_sk : from_rd;
    }
    if (lane < n) xr[gid[lane]] = double(xv);
  }
}

template <typename T>
__global__ void __launch_bounds__(32 * kGroupWarps)
k_apply_group_down_warp(LevelDev Lv, PhaseDev Ph, double* x, int64_t ldx, int nrhs,
                        int per_warp_bytes) {
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char smraw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = blockIdx.x * kGroupWarps + warp;
  if (g >= Lv.ngroup || Lv.group_t[g] < Ph.pre_min_type) return;
  const int n = Lv.group_size[g];
  const int32_t* gid = Lv.bucket + Lv.group_start[g];
  const int pi = Ph.group_pre[g], u = Ph.group_unit[g];
  unsigned char* base = smraw + (size_t)warp * per_warp_bytes;
  uint64_t* bar = (uint64_t*)base;
  int* invp = (int*)(base + 16 + group_block_bytes<T>(Lv.max_group));
  const T *Lg, *Fu, *Tm;
  group_stage(Ph, pi, u, n, base + 16, bar, lane == 0, &Lg, &Fu, &Tm);
  const bool staged = pi >= 0 || u >= 0;
  const int k = u >= 0 ? Ph.rank[u] : 0;
  const int r = n - k;
  const int* perm = u >= 0 ? Ph.perm + Ph.u_perm_off[u] : nullptr;
  if (u >= 0 && lane < n) invp[perm[lane]] = lane;
  __syncwarp();
  const int p_sk = (u >= 0 && lane < k) ? perm[lane] : 0;
  const int p_rd = (u >= 0 && lane < r) ? perm[k + lane] : 0;
  const int my_idx = (u >= 0 && lane < n) ? invp[lane] : 0;
  pdl_wait();   // the vectors come from the previous kernel of the sweep
  for (int rr = blockIdx.y; rr < nrhs; rr += gridDim.y) {   // right-hand sides over grid.y
    double* xr = x + rr * ldx;
    T xv = lane < n ? T(xr[gid[lane]]) : T(0);
    if (staged && rr == (int)blockIdx.y && !staged_ok(bar, Lv.status, Lv.level, kKindGroup, g)) return;
    if (u >= 0) {   // K: x_rd = L^{-T}(x_rd - W^T x_sk) ; x_sk -= T x_rd
      T xs = __shfl_sync(0xffffffffu, xv, p_sk);
      T xd = __shfl_sync(0xffffffffu, xv, p_rd);
      for (int q = 0; q < k; ++q) {
        const T v = __shfl_sync(0xffffffffu, xs, q);
        if (lane < r) xd -= Fu[(r + q) + lane * n] * v;
      }
      {   // x_rd = L_rr^{-T} x_rd
        T y = T(0);
        for (int c = 0; c < r; ++c) {
          const T v = __shfl_sync(0xffffffffu, xd, c);
          if (c >= lane && lane < r) y += Fu[c + lane * n] * v;
        }
        xd = y;
      }
      for (int a = 0; a < r; ++a) {
        const T v = __shfl_sync(0xffffffffu, xd, a);
        if (lane < k) xs -= Tm[lane + a * k] * v;
      }
      const T from_sk = __shfl_sync(0xffffffffu, xs, my_idx < k ? my_idx : 0);
      const T from_rd = __shfl_sync(0xffffffffu, xd, my_idx >= k ? my_idx - k : 0);
      xv = my_idx < k ? from_sk : from_rd;
    }
    if (Lg) {   // C: x_g = L_g^{-T} x_g
      T y = T(0);
      for (int c = 0; c < n; ++c) {
        const T v = __shfl_sync(0xffffffffu, xv, c);
        if (c >= lane && lane < n) y += Lg[c + lane * n] * v;
      }
      xv = y;
    }
    if (lane < n) xr[gid[lane]] = double(xv);
  }
}

// ---------------------------------------------------------------------------
// separator groups with many right-hand sides: one warp per group and one lane
// per right-hand side (32 a pass); the group's values are lane-strided in
// shared memory, the factor blocks staged beside them and read as broadcasts.
// Every lane does the one-vector warp kernels' products in their order, as
// scalar loops, in place (the unit steps need no second vector).
// ---------------------------------------------------------------------------

// Per-warp bytes: barrier, staged blocks, the unit's permutation, the values.
template <typename T>
__host__ __device__ inline size_t group_mr_bytes(int max_group) {
  return 16 + group_block_bytes<T>(max_group) + round16(max_group * sizeof(int)) +
         round16((size_t)max_group * kMrLd * sizeof(T));
}

// v[i kMrLd + lane] = T(x[gid[i] + (r0 + lane) ldx] - the cells' updates
// ubuf[(r0 + lane) ldu + b_off[cell] + pos + i] in the group's cell order)
// for lanes < R (0 above), eight entries' loads in flight.
template <typename T>
__device__ inline void group_mr_gather(const LevelDev& Lv, int g, int n, const int32_t* gid,
                                       const double* x, int64_t ldx, const double* ubuf,
                                       int64_t ldu, int r0, int R, T* v) {
  const int lane = threadIdx.x & 31;
  const bool on = lane < R;
  const double* xr = x + (int64_t)(r0 + (on ? lane : 0)) * ldx;
  const double* ur = ubuf ? ubuf + (int64_t)(r0 + (on ? lane : 0)) * ldu : nullptr;
  const int k0 = Lv.group_cell_off[g], k1 = Lv.group_cell_off[g + 1];
  for (int i0 = 0; i0 < n; i0 += 8) {
    double t[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) t[q] = (on && i0 + q < n) ? xr[gid[i0 + q]] : 0.0;
    if (ur)
      for (int k = k0; k < k1; ++k) {
        const double* u = ur + Lv.b_off[Lv.group_cell[k]] + Lv.group_pos[k] + i0;
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if (on && i0 + q < n) t[q] -= u[q];
      }
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (i0 + q < n) v[(i0 + q) * kMrLd + lane] = T(t[q]);
  }
  __syncwarp();
}

template <typename T>
__device__ inline void group_mr_scatter(double* x, int64_t ldx, const int32_t* gid, int n, int r0,
                                        int R, const T* v) {
  const int lane = threadIdx.x & 31;
  __syncwarp();
  if (lane >= R) return;
  double* xr = x + (int64_t)(r0 + lane) * ldx;
  for (int i = 0; i < n; ++i) xr[gid[i]] = double(v[i * kMrLd + lane]);
}

// Shared setup of the two sweeps: stage the group's blocks, copy the unit's
// permutation, return the warp's value rows (nullptr: group not in this phase).
template <typename T>
__device__ inline T* group_mr_setup(const LevelDev& Lv, const PhaseDev& Ph, int g, int per_warp_bytes,
                                    const T** Lg, const T** Fu, const T** Tm, int** perm,
                                    uint64_t** bar) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n = Lv.group_size[g];
  const int pi = Ph.group_pre[g], u = Ph.group_unit[g];
  unsigned char* base = smraw + (size_t)warp * per_warp_bytes;
  *bar = (uint64_t*)base;
  *perm = (int*)(base + 16 + group_block_bytes<T>(Lv.max_group));
  group_stage(Ph, pi, u, n, base + 16, *bar, lane == 0, Lg, Fu, Tm);
  if (u >= 0)
    for (int i = lane; i < n; i += 32) (*perm)[i] = Ph.perm[Ph.u_perm_off[u] + i];
  return (T*)((unsigned char*)*perm + round16(Lv.max_group * sizeof(int)));
}

// C_l^T then K_l^T of group blockIdx.x * warps + warp for right-hand sides
// r0 + lane, r0 = 32 blockIdx.y, 32 (blockIdx.y + gridDim.y), ...: as
// k_apply_group_up_warp.
template <typename T>
__global__ void __launch_bounds__(32 * kGroupWarps)
k_apply_group_up_mr(LevelDev Lv, PhaseDev Ph, int gather, double* x, int64_t ldx, int nrhs,
                    const double* ubuf, int64_t ldu, int per_warp_bytes) {
  pdl_trigger();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = blockIdx.x * (blockDim.x >> 5) + warp;
  if (g >= Lv.ngroup || Lv.group_t[g] < Ph.pre_min_type) return;
  const int n = Lv.group_size[g];
  const int32_t* gid = Lv.bucket + Lv.group_start[g];
  const int pi = Ph.group_pre[g], u = Ph.group_unit[g];
  const T *Lg, *Fu, *Tm;
  int* perm;
  uint64_t* bar;
  T* v = group_mr_setup<T>(Lv, Ph, g, per_warp_bytes, &Lg, &Fu, &Tm, &perm, &bar);
  T* xv = v + lane;   // xv[i * kMrLd]: entry i of this lane's right-hand side
  pdl_wait();   // the vectors come from the previous kernel of the sweep
  for (int r0 = blockIdx.y * 32; r0 < nrhs; r0 += gridDim.y * 32) {
    const int R = min(32, nrhs - r0);
    group_mr_gather<T>(Lv, g, n, gid, x, ldx, gather ? ubuf : nullptr, ldu, r0, R, v);
    if ((pi >= 0 || u >= 0) && r0 == (int)blockIdx.y * 32 &&
        !staged_ok(bar, Lv.status, Lv.level, kKindGroup, g))
      return;
    if (Lg)             // C^T: x_g = L_g^{-1} x_g, rows from the last (in place)
      for (int i = n - 1; i >= 0; --i) {
        T s = T(0);
        for (int c = 0; c <= i; ++c) s += Lg[i + c * n] * xv[c * kMrLd];
        xv[i * kMrLd] = s;
      }
    if (u >= 0) {   // K^T: x_rd -= T^T x_sk ; x_rd = L_rr^{-1} x_rd ; x_sk -= W x_rd
      const int k = Ph.rank[u], r = n - k;
      for (int a = 0; a < r; ++a) {
        T s = xv[perm[k + a] * kMrLd];
        for (int q = 0; q < k; ++q) s -= Tm[q + a * k] * xv[perm[q] * kMrLd];
        xv[perm[k + a] * kMrLd] = s;
      }
      for (int a = r - 1; a >= 0; --a) {
        T s = T(0);
        for (int c = 0; c <= a; ++c) s += Fu[a + c * n] * xv[perm[k + c] * kMrLd];
        xv[perm[k + a] * kMrLd] = s;
      }
      for (int q = 0; q < k; ++q) {
        T s = xv[perm[q] * kMrLd];
        for (int a = 0; a < r; ++a) s -= Fu[(r + q) + a * n] * xv[perm[k + a] * kMrLd];
        xv[perm[q] * kMrLd] = s;
      }
    }
    group_mr_scatter<T>(x, ldx, gid, n, r0, R, v);
  }
}

// K_l then C_l: as k_apply_group_down_warp.
template <typename T>
__global__ void __launch_bounds__(32 * kGroupWarps)
k_apply_group_down_mr(LevelDev Lv, PhaseDev Ph, double* x, int64_t ldx, int nrhs, int per_warp_bytes) {
  pdl_trigger();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = blockIdx.x * (blockDim.x >> 5) + warp;
  if (g >= Lv.ngroup || Lv.group_t[g] < Ph.pre_min_type) return;
  const int n = Lv.group_size[g];
  const int32_t* gid = Lv.bucket + Lv.group_start[g];
  const int pi = Ph.group_pre[g], u = Ph.group_unit[g];
  const T *Lg, *Fu, *Tm;
  int* perm;
  uint64_t* bar;
  T* v = group_mr_setup<T>(Lv, Ph, g, per_warp_bytes, &Lg, &Fu, &Tm, &perm, &bar);
  T* xv = v + lane;
  pdl_wait();   // the vectors come from the previous kernel of the sweep
  for (int r0 = blockIdx.y * 32; r0 < nrhs; r0 += gridDim.y * 32) {
    const int R = min(32, nrhs - r0);
    group_mr_gather<T>(Lv, g, n, gid, x, ldx, nullptr, 0, r0, R, v);
    if ((pi >= 0 || u >= 0) && r0 == (int)blockIdx.y * 32 &&
        !staged_ok(bar, Lv.status, Lv.level, kKindGroup, g))
      return;
    if (u >= 0) {   // K: x_rd = L_rr^{-T}(x_rd - W^T x_sk) ; x_sk -= T x_rd
      const int k = Ph.rank[u], r = n - k;
      for (int a = 0; a < r; ++a) {
        T s = xv[perm[k + a] * kMrLd];
        for (int q = 0; q < k; ++q) s -= Fu[(r + q) + a * n] * xv[perm[q] * kMrLd];
        xv[perm[k + a] * kMrLd] = s;
      }
      for (int a = 0; a < r; ++a) {   // rows from the first (in place)
        T s = T(0);
        for (int c = a; c < r; ++c) s += Fu[c + a * n] * xv[perm[k + c] * kMrLd];
        xv[perm[k + a] * kMrLd] = s;
      }
      for (int q = 0; q < k; ++q) {
        T s = xv[perm[q] * kMrLd];
        for (int a = 0; a < r; ++a) s -= Tm[q + a * k] * xv[perm[k + a] * kMrLd];
        xv[perm[q] * kMrLd] = s;
      }
    }
    if (Lg)   // C: x_g = L_g^{-T} x_g
      for (int i = 0; i < n; ++i) {
        T s = T(0);
        for (int c = i; c < n; ++c) s += Lg[c + i * n] * xv[c * kMrLd];
        xv[i * kMrLd] = s;
      }
    group_mr_scatter<T>(x, ldx, gid, n, r0, R, v);
  }
}

// Lane-per-right-hand-side group kernels: from 8 right-hand sides, where a
// warp's blocks and values fit the shared-memory budget.
template <typename T>
static int group_mr_warps(const LevelDev& Lv, int nrhs) {
  if (nrhs < 8) return 0;
  const size_t per = group_mr_bytes<T>(Lv.max_group);
  if (per > kStageBudget) return 0;
  return (int)std::min<size_t>(kGroupWarps, (200 * 1024) / per);
}

// grid.y of the lane-per-right-hand-side kernels: one 32-wide chunk of
// right-hand sides each, looping beyond 65535 chunks.
static inline unsigned mr_chunks(int nrhs) {
  return (unsigned)std::min(std::max((nrhs + 31) / 32, 1), 65535);
}

// Lane-per-right-hand-side leaf kernels: from 8 right-hand sides, for leaf
// levels whose bands all hold inverted diagonal blocks (w <= 15: 2D) and fit
// the shared-memory budget.
template <typename T>
static bool leaf_lanes_per_rhs(const LevelDev& Lv, int nrhs) {
  return nrhs >= 8 && Lv.max_w >= 1 && Lv.max_w <= kBandRegW &&
         leaf_mr_bytes<T>(Lv.max_nI, Lv.max_nB, Lv.max_w) <= kStageBudget;
}

// Right-hand sides over grid.y: the per-RHS work of the sweeps is
// independent.  A launch gets as many CTAs per vector as keep it at about
// 2432 CTAs (152 SMs x 16); the remaining right-hand sides loop inside each
// CTA, which then reads its factor blocks once (staged in shared memory, or
// from L1) for all of them instead of once per right-hand side.
static inline unsigned rhs_grid(int nrhs, int64_t gridx) {
  const int64_t target = 152 * 16;
  int64_t gy = (target + std::max<int64_t>(gridx, 1) - 1) / std::max<int64_t>(gridx, 1);
  gy = std::min<int64_t>(std::max<int64_t>(gy, 1), std::max(nrhs, 1));
  return (unsigned)std::min<int64_t>(gy, 65535);
}

template <typename T>
void launch_apply_cell_up(const LevelDev& Lv, double* x, int64_t ldx, int nrhs, double* ubuf,
                          int64_t ldu, cudaStream_t s) {
  if (!Lv.ncell) return;
  if (Lv.level == 0) {
    if (leaf_lanes_per_rhs<T>(Lv, nrhs)) {   // many right-hand sides: lane = right-hand side
      const size_t per = leaf_mr_bytes<T>(Lv.max_nI, Lv.max_nB, Lv.max_w);
      const int wpc = (int)std::max<size_t>(1, std::min<size_t>(4, kStageBudget / per));
      const dim3 grid((Lv.ncell + wpc - 1) / wpc, mr_chunks(nrhs));
      launch_pdl(k_apply_leaf_up_mr<T>, grid, 32 * wpc, wpc * per, s, Lv, x, ldx, nrhs, ubuf, ldu, (int)per);
      return;
    }
    const bool multi = nrhs > (int)rhs_grid(nrhs, Lv.ncell / kLeafWarps + 1);
    const bool staged = leaf_staged<T>(Lv) || multi;
    const int wpc = leaf_warps_per_cta<T>(Lv, staged);
    const size_t per = leaf_warp_smem<T>(Lv, staged);
    const unsigned grid = (Lv.ncell + wpc - 1) / wpc;
    const unsigned gy = rhs_grid(nrhs, grid);
    if (staged)
      launch_pdl(k_apply_leaf_up<T, true>, dim3(grid, gy), 32 * wpc, wpc * per, s, Lv, x, ldx, nrhs, ubuf, ldu, (int)per);
    else
      launch_pdl(k_apply_leaf_up<T, false>, dim3(grid, gy), 32 * wpc, wpc * per, s, Lv, x, ldx, nrhs, ubuf, ldu, (int)per);
    return;
  }
  const int rcn = nrhs >= 8 ? 8 : 1;   // right-hand sides per pass
  const size_t base = round16(2 * rcn * (Lv.max_nI + 1) * sizeof(T));
  const size_t blk = round16((size_t)Lv.max_n * Lv.max_nI * sizeof(T));
  const int stage = blk <= kStageBudget && base + blk <= 200 * 1024;
  const dim3 grid(Lv.ncell, rhs_grid((nrhs + rcn - 1) / rcn, Lv.ncell));
  if (rcn == 8)
    launch_pdl(k_apply_cell_up<T, 8>, grid, kApplyThreads, base + (stage ? blk : 0), s, Lv, x, ldx, nrhs,
                                                                                ubuf, ldu, stage);
  else
    launch_pdl(k_apply_cell_up<T, 1>, grid, kApplyThreads, base + (stage ? blk : 0), s, Lv, x, ldx, nrhs,
                                                                                ubuf, ldu, stage);
}

template <typename T>
void launch_apply_cell_down(const LevelDev& Lv, double* x, int64_t ldx, int nrhs, cudaStream_t s) {
  if (!Lv.ncell) return;
  if (Lv.level == 0) {
    if (leaf_lanes_per_rhs<T>(Lv, nrhs)) {   // many right-hand sides: lane = right-hand side
      const size_t per = leaf_mr_bytes<T>(Lv.max_nI, Lv.max_nB, Lv.max_w);
      const int wpc = (int)std::max<size_t>(1, std::min<size_t>(4, kStageBudget / per));
      const dim3 grid((Lv.ncell + wpc - 1) / wpc, mr_chunks(nrhs));
      launch_pdl(k_apply_leaf_down_mr<T>, grid, 32 * wpc, wpc * per, s, Lv, x, ldx, nrhs, (int)per);
      return;
    }
    const bool multi = nrhs > (int)rhs_grid(nrhs, Lv.ncell / kLeafWarps + 1);
    const bool staged = leaf_staged<T>(Lv) || multi;
    const int wpc = leaf_warps_per_cta<T>(Lv, staged);
    const size_t per = leaf_warp_smem<T>(Lv, staged);
    const unsigned grid = (Lv.ncell + wpc - 1) / wpc;
    const unsigned gy = rhs_grid(nrhs, grid);
    if (staged)
      launch_pdl(k_apply_leaf_down<T, true>, dim3(grid, gy), 32 * wpc, wpc * per, s, Lv, x, ldx, nrhs, (int)per);
    else
      launch_pdl(k_apply_leaf_down<T, false>, dim3(grid, gy), 32 * wpc, wpc * per, s, Lv, x, ldx, nrhs, (int)per);
    return;
  }
  const int rcn = nrhs >= 8 ? 8 : 1;   // right-hand sides per pass
  const size_t base = round16(rcn * (2 * Lv.max_nI + Lv.max_nB + 1) * sizeof(T));
  const size_t blk = round16((size_t)Lv.max_n * Lv.max_nI * sizeof(T));
  const int stage = blk <= kStageBudget && base + blk <= 200 * 1024;
  const dim3 grid(Lv.ncell, rhs_grid((nrhs + rcn - 1) / rcn, Lv.ncell));
  if (rcn == 8)
    launch_pdl(k_apply_cell_down<T, 8>, grid, kApplyThreads, base + (stage ? blk : 0), s, Lv, x, ldx, nrhs,
                                                                                  stage);
  else
    launch_pdl(k_apply_cell_down<T, 1>, grid, kApplyThreads, base + (stage ? blk : 0), s, Lv, x, ldx, nrhs,
                                                                                  stage);
}

// right-hand sides per chunk so that a chunk of an rows-long vector fits in
// the shared-memory budget
template <typename T>
static int big_rhs_chunk(int rows) {
  const size_t per = (size_t)(rows > 0 ? rows : 1) * sizeof(T);
  return (int)std::max<size_t>(1, std::min<size_t>(4, kStageBudget / per));
}

template <typename T>
int launch_apply_big_up(const LevelDev& Lv, double* x, int64_t ldx, int nrhs, double* ubuf,
                        int64_t ldu, double* tmp, cudaStream_t s) {
  if (!Lv.ncell || !Lv.max_nI) return 0;
  const int rc = big_rhs_chunk<T>(Lv.max_nI);
  const size_t sm = (size_t)Lv.max_nI * rc * sizeof(T);
  launch_pdl(k_apply_big_up1<T>, dim3((Lv.max_nI + kBigRows - 1) / kBigRows, Lv.ncell), kBigRows, sm, s,
      Lv, x, ldx, nrhs, rc, tmp, ldu);
  const int rows = std::max(Lv.max_nI, Lv.max_nB);
  launch_pdl(k_apply_big_up2<T>, dim3((rows + kBigRows - 1) / kBigRows, Lv.ncell), kBigRows, sm, s,
      Lv, x, ldx, nrhs, rc, ubuf, ldu, tmp, ldu);
  return 2;
}

template <typename T>
int launch_apply_big_down(const LevelDev& Lv, double* x, int64_t ldx, int nrhs, double* tmp,
                          int64_t ldt, cudaStream_t s) {
  if (!Lv.ncell || !Lv.max_nI) return 0;
  const unsigned gx = (Lv.max_nI + kBigWarps - 1) / kBigWarps;
  const int rcb = big_rhs_chunk<T>(Lv.max_nB);
  launch_pdl(k_apply_big_down1<T>, dim3(gx, Lv.ncell), 32 * kBigWarps,
             (size_t)std::max(Lv.max_nB, 1) * rcb * sizeof(T), s, Lv, x, ldx, nrhs, rcb, tmp, ldt);
  const int rci = big_rhs_chunk<T>(Lv.max_nI);
  launch_pdl(k_apply_big_down2<T>, dim3(gx, Lv.ncell), 32 * kBigWarps,
             (size_t)Lv.max_nI * rci * sizeof(T), s, Lv, x, ldx, nrhs, rci, tmp, ldt);
  return 2;
}

template <typename T>
void launch_apply_group_up(const LevelDev& Lv, const PhaseDev& Ph, int gather, double* x,
                           int64_t ldx, int nrhs, const double* ubuf, int64_t ldu, cudaStream_t s) {
  if (!Lv.ngroup) return;
  if (const int wpc = group_mr_warps<T>(Lv, nrhs)) {
    const size_t per = group_mr_bytes<T>(Lv.max_group);
    const unsigned grid = (Lv.ngroup + wpc - 1) / wpc;
    launch_pdl(k_apply_group_up_mr<T>, dim3(grid, mr_chunks(nrhs)), 32 * wpc, wpc * per, s,
        Lv, Ph, gather, x, ldx, nrhs, ubuf, ldu, (int)per);
    return;
  }
  if (Lv.max_group <= 32) {
    const size_t per = group_warp_smem<T>(Lv.max_group);
    const unsigned grid = (Lv.ngroup + kGroupWarps - 1) / kGroupWarps;
    launch_pdl(k_apply_group_up_warp<T>, dim3(grid, rhs_grid(nrhs, grid)), 32 * kGroupWarps, kGroupWarps * per, s,
        Lv, Ph, gather, x, ldx, nrhs, ubuf, ldu, (int)per);
    return;
  }
  const size_t base = round16(2 * (Lv.max_group + 1) * sizeof(T));
  const size_t blk = group_block_bytes<T>(Lv.max_group);
  const int stage = blk <= kStageBudget;
  launch_pdl(k_apply_group_up<T>, dim3(Lv.ngroup, rhs_grid(nrhs, Lv.ngroup)), kGroupThreads, base + (stage ? blk : 0), s,
      Lv, Ph, gather, x, ldx, nrhs, ubuf, ldu, stage);
}

template <typename T>
void launch_apply_group_down(const LevelDev& Lv, const PhaseDev& Ph, double* x, int64_t ldx,
                             int nrhs, cudaStream_t s) {
  if (!Lv.ngroup) return;
  if (const int wpc = group_mr_warps<T>(Lv, nrhs)) {
    const size_t per = group_mr_bytes<T>(Lv.max_group);
    const unsigned grid = (Lv.ngroup + wpc - 1) / wpc;
    launch_pdl(k_apply_group_down_mr<T>, dim3(grid, mr_chunks(nrhs)), 32 * wpc, wpc * per, s,
        Lv, Ph, x, ldx, nrhs, (int)per);
    return;
  }
  if (Lv.max_group <= 32) {
    const size_t per = group_warp_smem<T>(Lv.max_group);
    const unsigned grid = (Lv.ngroup + kGroupWarps - 1) / kGroupWarps;
    launch_pdl(k_apply_group_down_warp<T>, dim3(grid, rhs_grid(nrhs, grid)), 32 * kGroupWarps, kGroupWarps * per, s,
        Lv, Ph, x, ldx, nrhs, (int)per);
    return;
  }
  const size_t base = round16(2 * (Lv.max_group + 1) * sizeof(T));
  const size_t blk = group_block_bytes<T>(Lv.max_group);
  const int stage = blk <= kStageBudget;
  launch_pdl(k_apply_group_down<T>, dim3(Lv.ngroup, rhs_grid(nrhs, Lv.ngroup)), kGroupThreads, base + (stage ? blk : 0), s,
      Lv, Ph, x, ldx, nrhs, stage);
}

template <typename T>
int configure_apply_kernels() {
  const int big = 200 * 1024;
  cudaError_t e = cudaSuccess;
  e = cudaFuncSetAttribute(k_apply_cell_up<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_apply_cell_up<T, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_apply_cell_down<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_apply_cell_down<T, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_apply_group_up<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_apply_group_down<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_apply_leaf_up<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_apply_leaf_down<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_apply_leaf_up_mr<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_apply_leaf_down_mr<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_apply_group_up_warp<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_apply_group_up_mr<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_apply_group_down_mr<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_apply_group_down_warp<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_apply_big_up1<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_apply_big_up2<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_apply_big_down1<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_apply_big_down2<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  return e == cudaSuccess ? 0 : -1;
}

#define RHIF_APPLY_INST(T)                                                                         \
  template void launch_apply_cell_up<T>(const LevelDev&, double*, int64_t, int, double*, int64_t,  \
                                        cudaStream_t);                                             \
  template void launch_apply_cell_down<T>(const LevelDev&, double*, int64_t, int, cudaStream_t);   \
  template void launch_apply_group_up<T>(const LevelDev&, const PhaseDev&, int, double*, int64_t,  \
                                         int, const double*, int64_t, cudaStream_t);               \
  template void launch_apply_group_down<T>(const LevelDev&, const PhaseDev&, double*, int64_t, int, \
                                           cudaStream_t);                                          \
  template int launch_apply_big_up<T>(const LevelDev&, double*, int64_t, int, double*, int64_t,   \
                                      double*, cudaStream_t);                                      \
  template int launch_apply_big_down<T>(const LevelDev&, double*, int64_t, int, double*, int64_t,  \
                                        cudaStream_t);                                             \
  template int configure_apply_kernels<T>();

RHIF_APPLY_INST(double)
RHIF_APPLY_INST(float)

// ---------------------------------------------------------------------------
// FP64 stencil SpMV and PCG vector kernels
// ---------------------------------------------------------------------------

constexpr int kVecThreads = 256;

__device__ inline double block_sum(double v) {
  __shared__ double part[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) part[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (warp == 0) {
    s = lane < (int)(blockDim.x >> 5) ? part[lane] : 0.0;
    s = warp_sum(s);
  }
  return s;   // valid in thread 0
}

// y = A x (+ partial sums of x.y per block when partial != nullptr)
__global__ void k_spmv(GeoDev G, const double* diag, const double* off, const double* x,
                       int64_t ldx, double* y, int64_t ldy, double* partial) {
  const int r = blockIdx.y;
  const double* xr = x + r * ldx;
  double* yr = y + r * ldy;
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < G.N;
       i += (int64_t)gridDim.x * blockDim.x) {
    double s = diag[i] * xr[i];
    int64_t rem = i;
    for (int a = 0; a < G.d; ++a) {
      const int xa = (int)(rem % G.ns[a]);
      rem /= G.ns[a];
      const int64_t st = G.stride[a];
      if (xa + 1 < G.ns[a]) s += off[a * G.N + i] * xr[i + st];
      if (xa >= 1) s += off[a * G.N + i - st] * xr[i - st];
    }
    yr[i] = s;
    acc += s * xr[i];
  }
  if (partial) {
    const double t = block_sum(acc);
    if (threadIdx.x == 0) partial[blockIdx.x + (int64_t)gridDim.x * r] = t;
  }
}

// partial sums of a.b per block
__global__ void k_dot_partial(int64_t N, const double* a, int64_t lda, const double* b, int64_t ldb,
                              double* partial) {
  const int r = blockIdx.y;
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x)
    acc += a[i + r * lda] * b[i + r * ldb];
  const double t = block_sum(acc);
  if (threadIdx.x == 0) partial[blockIdx.x + (int64_t)gridDim.x * r] = t;
}

// PCG scalar slots per right-hand side (doubles): see enum in kernels.h
// mode 0: ff ; 1: rz (init) ; 2: pq -> alpha ; 3: rr -> done ; 4: rz_new -> beta
__global__ void k_reduce(const double* partial, int nblk, double* sc, int mode, double rtol) {
  const int r = blockIdx.x;
  double acc = 0.0;
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) acc += partial[i + (int64_t)nblk * r];
  const double s = block_sum(acc);
  if (threadIdx.x != 0) return;
  double* S = sc + 8 * r;
  switch (mode) {
    case 0: S[kScFF] = s; break;
    case 1: S[kScRZ] = s; break;
    case 2:
      S[kScPQ] = s;
      S[kScAlpha] = (S[kScDone] != 0.0 || s == 0.0) ? 0.0 : S[kScRZ] / s;
      break;
    case 3:
      S[kScRR] = s;
      if (S[kScDone] == 0.0 && sqrt(s) <= rtol * sqrt(S[kScFF])) S[kScDone] = 1.0;
      break;
    case 4:
      S[kScBeta] = (S[kScDone] != 0.0 || S[kScRZ] == 0.0) ? 0.0 : s / S[kScRZ];
      S[kScRZ] = s;
      break;
  }
}

// Device-side PCG loop (the iterations as a conditional WHILE node of a CUDA
// graph).  kit[0]: iterations done; kit[1 + c]: first iteration at which
// right-hand side c met the tolerance (maxit until then).  After each
// iteration's residual reduction the check records newly converged
// right-hand sides and sets the loop condition: go on while some right-hand
// side has not converged and fewer than maxit iterations ran, so the loop
// always ends.
__global__ void k_pcg_kit_init(int* kit, int nrhs, int maxit) {
  for (int c = threadIdx.x; c <= nrhs; c += blockDim.x) kit[c] = c == 0 ? 0 : maxit;
}

__global__ void k_pcg_check(const double* sc, int nrhs, int* kit, int maxit,
                            cudaGraphConditionalHandle h) {
  __shared__ int live;
  if (threadIdx.x == 0) live = 0;
  __syncthreads();
  const int k = kit[0] + 1;
  int mine = 0;
  for (int c = threadIdx.x; c < nrhs; c += blockDim.x) {
    if (sc[8 * c + kScDone] != 0.0) {
      if (kit[1 + c] > k) kit[1 + c] = k;
    } else {
      mine = 1;
    }
  }
  if (mine) atomicOr(&live, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    kit[0] = k;
    cudaGraphSetConditional(h, (live && k < maxit) ? 1u : 0u);
  }
}

void launch_pcg_kit_init(int* kit, int nrhs, int maxit, cudaStream_t s) {
  k_pcg_kit_init<<<1, 256, 0, s>>>(kit, nrhs, maxit);
}

void launch_pcg_check(const double* sc, int nrhs, int* kit, int maxit,
                      cudaGraphConditionalHandle h, cudaStream_t s) {
  k_pcg_check<<<1, 256, 0, s>>>(sc, nrhs, kit, maxit, h);
}

// x += alpha p ; r -= alpha q ; partial r.r
__global__ void k_update_xr(int64_t N, const double* sc, double* x, int64_t ldx, double* rv,
                            int64_t ldr, const double* p, int64_t ldp, const double* q,
                            int64_t ldq, double* partial) {
  const int r = blockIdx.y;
  const double* S = sc + 8 * r;
  const double alpha = S[kScAlpha];
  const bool live = S[kScDone] == 0.0;
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    double ri = rv[i + r * ldr];
    if (live) {
      x[i + r * ldx] += alpha * p[i + r * ldp];
      ri -= alpha * q[i + r * ldq];
      rv[i + r * ldr] = ri;
    }
    acc += ri * ri;
  }
  const double t = block_sum(acc);
  if (threadIdx.x == 0) partial[blockIdx.x + (int64_t)gridDim.x * r] = t;
}

// p = z (first iteration; p is not read: it holds whatever the scratch held)
// or p = z + beta p
__global__ void k_update_p(int64_t N, const double* sc, const double* z, int64_t ldz, double* p,
                           int64_t ldp, int first) {
  const int r = blockIdx.y;
  const double* S = sc + 8 * r;
  if (!first && S[kScDone] != 0.0) return;
  const double beta = first ? 0.0 : S[kScBeta];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i + r * ldp] = first ? z[i + r * ldz] : z[i + r * ldz] + beta * p[i + r * ldp];
}

// y = a - b (true residual)
__global__ void k_sub(int64_t N, const double* a, int64_t lda, const double* b, int64_t ldb,
                      double* y, int64_t ldy) {
  const int r = blockIdx.y;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i + r * ldy] = a[i + r * lda] - b[i + r * ldb];
}

__global__ void k_copy_cols(int64_t N, const double* a, int64_t lda, double* y, int64_t ldy) {
  const int r = blockIdx.y;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i + r * ldy] = a[i + r * lda];
}

// x <- alpha x (alpha read from the device: sc[0])
__global__ void k_scale(int64_t N, double* x, const double* alpha) {
  const double a = *alpha;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] *= a;
}

int vec_blocks(int64_t N) {
  int64_t b = (N + kVecThreads - 1) / kVecThreads;
  if (b > 1216) b = 1216;   // 8 blocks per SM on 152 SMs
  return (int)(b < 1 ? 1 : b);
}

void launch_spmv(const GeoDev& G, const double* diag, const double* off, const double* x,
                 int64_t ldx, double* y, int64_t ldy, int nrhs, double* partial, cudaStream_t s) {
  dim3 grid(vec_blocks(G.N), nrhs);
  k_spmv<<<grid, kVecThreads, 0, s>>>(G, diag, off, x, ldx, y, ldy, partial);
}
void launch_dot_partial(int64_t N, const double* a, int64_t lda, const double* b, int64_t ldb,
                        int nrhs, double* partial, cudaStream_t s) {
  dim3 grid(vec_blocks(N), nrhs);
  k_dot_partial<<<grid, kVecThreads, 0, s>>>(N, a, lda, b, ldb, partial);
}
void launch_reduce(const double* partial, int nblk, int nrhs, double* sc, int mode, double rtol,
                   cudaStream_t s) {
  k_reduce<<<nrhs, 256, 0, s>>>(partial, nblk, sc, mode, rtol);
}
void launch_update_xr(int64_t N, int nrhs, const double* sc, double* x, int64_t ldx, double* r,
                      int64_t ldr, const double* p, int64_t ldp, const double* q, int64_t ldq,
                      double* partial, cudaStream_t s) {
  dim3 grid(vec_blocks(N), nrhs);
  k_update_xr<<<grid, kVecThreads, 0, s>>>(N, sc, x, ldx, r, ldr, p, ldp, q, ldq, partial);
}
void launch_update_p(int64_t N, int nrhs, const double* sc, const double* z, int64_t ldz, double* p,
                     int64_t ldp, int first, cudaStream_t s) {
  dim3 grid(vec_blocks(N), nrhs);
  k_update_p<<<grid, kVecThreads, 0, s>>>(N, sc, z, ldz, p, ldp, first);
}
void launch_sub(int64_t N, int nrhs, const double* a, int64_t lda, const double* b, int64_t ldb,
                double* y, int64_t ldy, cudaStream_t s) {
  dim3 grid(vec_blocks(N), nrhs);
  k_sub<<<grid, kVecThreads, 0, s>>>(N, a, lda, b, ldb, y, ldy);
}
void launch_scale(int64_t N, double* x, const double* alpha, cudaStream_t s) {
  k_scale<<<vec_blocks(N), kVecThreads, 0, s>>>(N, x, alpha);
}
void launch_copy_cols(int64_t N, int nrhs, const double* a, int64_t lda, double* y, int64_t ldy,
                      cudaStream_t s) {
  dim3 grid(vec_blocks(N), nrhs);
  k_copy_cols<<<grid, kVecThreads, 0, s>>>(N, a, lda, y, ldy);
}

// ---------------------------------------------------------------------------
// finite-difference assembly (Eq. 1.1, Secs. 3.1/3.2) and the log-coefficient gradient
// ---------------------------------------------------------------------------

__device__ inline int64_t nb_sum(int c, int n) {   // sum_{v=0}^{c-1} ([v>0] + [v<n-1])
  return (int64_t)max(c - 1, 0) + (int64_t)min(c, n - 1);
}
__device__ inline int nb_one(int v, int n) { return (v > 0) + (v < n - 1); }

// mean of the per-pixel coefficient over the pixels touching the grid edge that
// starts at node coordinates x (1-based, boundary nodes allowed) along axis ax
__device__ double edge_weight(const GeoDev& G, const double* a_pix, const int x[3], int ax) {
  double s = 0.0;
  int cnt = 0;
  const int nx = G.ns[0] + 1, ny = G.ns[1] + 1;
  for (int m = 0; m < (1 << (G.d - 1)); ++m) {
    int p[3] = {0, 0, 0};
    int bit = 0;
    for (int a = 0; a < G.d; ++a) {
      if (a == ax) p[a] = x[a];
      else { p[a] = x[a] - 1 + ((m >> bit) & 1); ++bit; }
    }
    s += a_pix[p[0] + (int64_t)nx * (p[1] + (int64_t)ny * p[2])];
    ++cnt;
  }
  return s * (1.0 / cnt);   // cnt = 2^(d-1): the same value as s / cnt, without a divide
}

// One thread per row.  I: index type of the row arithmetic (32-bit while the
// entry count fits: GB300 has no fast 64-bit divide, and its FP64 divide is
// slow too, so the 1/h^2 factor is applied as the exact integer (n + 1)^2).
template <typename I>
__global__ void k_assemble_fd(GeoDev G, const double* a_pix, const double* b_node, double b_const,
                              int64_t* rowptr, int32_t* col, double* val) {
  const int64_t i64 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i64 >= G.N) return;
  const I i = (I)i64;
  int x[3] = {0, 0, 0};   // 0-based
  I rem = i;
  for (int a = 0; a < G.d; ++a) {
    x[a] = (int)(rem % (I)G.ns[a]);
    rem /= (I)G.ns[a];
  }
  // entries before row i, counted slab by slab from the last axis
  I before = 0;
  {
    I inner = 1;   // rows in one slab of the lower axes
    for (int a = 0; a < G.d; ++a) inner *= (I)G.ns[a];
    for (int a = G.d - 1; a >= 0; --a) {
      inner /= (I)G.ns[a];
      // rows with coordinate a in [0, x[a]) and equal higher coordinates: box [0,n_0)x..x[0,x[a])x{x_{a+1}}..
      const I cnt = inner * (I)x[a];
      I nbs = cnt;   // diagonal entries
      for (int b = 0; b < G.d; ++b) {
        I sb;
        if (b < a) sb = (I)nb_sum(G.ns[b], G.ns[b]) * (cnt / (I)G.ns[b]);
        else if (b == a) sb = (I)nb_sum(x[a], G.ns[a]) * inner;
        else sb = (I)nb_one(x[b], G.ns[b]) * cnt;
        nbs += sb;
      }
      before += nbs;
    }
  }
  rowptr[i64] = (int64_t)before;
  if (i64 == G.N - 1) {
    int64_t own = 1;
    for (int a = 0; a < G.d; ++a) own += nb_one(x[a], G.ns[a]);
    rowptr[G.N] = (int64_t)before + own;
  }
  int x1[3] = {1, 1, 1};
  for (int a = 0; a < G.d; ++a) x1[a] = x[a] + 1;
  double diag = b_node ? b_node[i64] : b_const;
  double offv[3][2];
  for (int a = 0; a < G.d; ++a) {
    const double q = (double)(G.ns[a] + 1);   // 1/h^2 = (n + 1)^2, exact
    const double ih2 = q * q;
    int xl[3] = {x1[0], x1[1], x1[2]};
    xl[a] = x1[a] - 1;
    const double wl = edge_weight(G, a_pix, xl, a) * ih2;   // edge from x-1 to x
    const double wr = edge_weight(G, a_pix, x1, a) * ih2;   // edge from x to x+1
    diag += wl + wr;
    offv[a][0] = -wl;
    offv[a][1] = -wr;
  }
  int64_t k = (int64_t)before;
  for (int a = G.d - 1; a >= 0; --a)
    if (x[a] >= 1) { col[k] = (int32_t)(i64 - G.stride[a]); val[k] = offv[a][0]; ++k; }
  col[k] = (int32_t)i64; val[k] = diag; ++k;
  for (int a = 0; a < G.d; ++a)
    if (x[a] + 1 < G.ns[a]) { col[k] = (int32_t)(i64 + G.stride[a]); val[k] = offv[a][1]; ++k; }
}

__global__ void k_exp(int64_t n, const double* x, double* y) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = exp(x[i]);
}

void launch_exp(int64_t n, const double* x, double* y, cudaStream_t s) {
  if (n > 0) k_exp<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, x, y);
}

void launch_assemble_fd(const GeoDev& G, const double* a_pix, const double* b_node, double b_const,
                        int64_t* rowptr, int32_t* col, double* val, cudaStream_t s) {
  if (!G.N) return;
  const unsigned grid = (unsigned)((G.N + 255) / 256);
  if (G.N * (2 * G.d + 1) < (int64_t(1) << 31))   // every entry offset fits 32 bits
    k_assemble_fd<int32_t><<<grid, 256, 0, s>>>(G, a_pix, b_node, b_const, rowptr, col, val);
  else
    k_assemble_fd<int64_t><<<grid, 256, 0, s>>>(G, a_pix, b_node, b_const, rowptr, col, val);
}

// one thread per pixel: -a_p / 2^(d-1) * sum over the 2^(d-1)*d grid edges of
// pixel p of (lam_i - lam_j)(u_i - u_j)/h^2, u = lam = 0 on boundary nodes
__global__ void k_grad_logcoef(GeoDev G, const double* a_pix, const double* u, const double* lam,
                               double* grad, int64_t npix) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= npix) return;
  int pc[3] = {0, 0, 0};
  int64_t rem = p;
  for (int a = 0; a < G.d; ++a) {
    pc[a] = (int)(rem % (G.ns[a] + 1));
    rem /= (G.ns[a] + 1);
  }
  auto node = [&](const int c[3], const double* v) -> double {
    int64_t id = 0, mul = 1;
    for (int a = 0; a < G.d; ++a) {
      if (c[a] < 1 || c[a] > G.ns[a]) return 0.0;
      id += (int64_t)(c[a] - 1) * mul;
      mul *= G.ns[a];
    }
    return v[id];
  };
  double acc = 0.0;
  for (int ax = 0; ax < G.d; ++ax) {
    const double q = (double)(G.ns[ax] + 1);   // 1/h^2 = (n + 1)^2, exact (as the assembly)
    const double ih2 = q * q;
    for (int m = 0; m < (1 << (G.d - 1)); ++m) {
      int c0[3] = {0, 0, 0};
      int bit = 0;
      for (int a = 0; a < G.d; ++a) {
        if (a == ax) c0[a] = pc[a];
        else { c0[a] = pc[a] + ((m >> bit) & 1); ++bit; }
      }
      int c1[3] = {c0[0], c0[1], c0[2]};
      c1[ax] += 1;
      acc += (node(c1, u) - node(c0, u)) * (node(c1, lam) - node(c0, lam)) * ih2;
    }
  }
  grad[p] = -a_pix[p] * acc * (1.0 / double(1 << (G.d - 1)));   // exact: a power of two
}

void launch_grad_logcoef(const GeoDev& G, const double* a_pix, const double* u, const double* lam,
                         double* grad, cudaStream_t s) {
  int64_t npix = 1;
  for (int a = 0; a < G.d; ++a) npix *= (G.ns[a] + 1);
  k_grad_logcoef<<<(unsigned)((npix + 255) / 256), 256, 0, s>>>(G, a_pix, u, lam, grad, npix);
}

}  // namespace rhif
