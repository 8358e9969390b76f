// Factorization kernels (Sec. 2 primitives batched over one level of Sec. 3).
//
// One CTA per independent object of a level: a cell (elimination,
// Sec. 2.1), a separator group (block Jacobi preconditioning, Sec. 2.3) or a
// skeletonization unit (interpolative decomposition + zeroing + elimination of
// the redundant DOFs, Sec. 2.2).  Cells commute (Sec. 2.1), preconditioning
// blocks commute (Sec. 2.3) and all IDs of a level are taken before any
// zeroing (the parallel order of Sec. 2.2), so each kernel is one launch over
// all objects of the level.  Every cross-cell sum is a gather in a fixed cell
// order (no atomics), so results are bitwise reproducible.
#include <cooperative_groups.h>

#include "common.cuh"
#include "kernels.h"
#include "tables.h"
#include "../../include/rhif.h"

namespace rhif {

// ---------------------------------------------------------------------------
// CSR -> stencil form (diagonal + coupling to the +1 neighbour along each axis)
// ---------------------------------------------------------------------------

__global__ void k_stencil_from_csr(GeoDev G, const int64_t* rowptr, const int32_t* col,
                                   const double* val, int64_t nnz, double* diag, double* off,
                                   double* offb, int* status) {
  pdl_trigger();
  pdl_wait();   // what the previous kernel of the stream wrote
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= G.N) return;
  const int64_t b = rowptr[i], e = rowptr[i + 1];
  if (b < 0 || e < b || e > nnz) {
    report(status, RHIF_ERR_BAD_ARG, -1, kKindArg, (int)i);
    return;
  }
  int x[3] = {0, 0, 0};
  int64_t rem = i;
  for (int a = 0; a < G.d; ++a) {
    x[a] = (int)(rem % G.ns[a]);
    rem /= G.ns[a];
  }
  double dg = 0.0;
  for (int64_t k = b; k < e; ++k) {
    const int64_t j = col[k];
    const double v = val[k];
    if (j == i) {
      dg += v;
      continue;
    }
    const int64_t delta = j - i;
    bool ok = false;
    for (int a = 0; a < G.d && !ok; ++a) {
      if (delta == G.stride[a] && x[a] + 1 < G.ns[a]) {
        off[a * G.N + i] = v;
        ok = true;
      } else if (delta == -G.stride[a] && x[a] >= 1) {
        offb[a * G.N + j] = v;
        ok = true;
      }
    }
    if (!ok) report(status, RHIF_ERR_BAD_ARG, -1, kKindArg, (int)i);
  }
  diag[i] = dg;
}

__global__ void k_stencil_check(int64_t n, const double* off, const double* offb, int* status) {
  pdl_trigger();
  pdl_wait();   // what the previous kernel of the stream wrote
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n && off[i] != offb[i]) report(status, RHIF_ERR_BAD_ARG, -1, kKindArg, (int)(i % 2147483647));
}

// ---------------------------------------------------------------------------
// front-order DOF lists: interior, then the segments of the closure
// ---------------------------------------------------------------------------

__global__ void k_expand_gids(LevelDev Lv) {
  pdl_trigger();
  pdl_wait();   // what the previous kernel of the stream wrote
  const int c = blockIdx.x;
  const int nI = Lv.nI[c];
  int32_t* out = Lv.gids + Lv.gid_off[c];
  const int32_t* I = Lv.bucket + Lv.cell_start[c];
  for (int p = threadIdx.x; p < nI; p += blockDim.x) out[p] = I[p];
  for (int s = Lv.seg_off[c]; s < Lv.seg_off[c + 1]; ++s) {
    const int g = Lv.seg_group[s];
    const int32_t* src = Lv.bucket + Lv.group_start[g];
    int32_t* dst = out + nI + Lv.seg_pos[s];
    for (int o = threadIdx.x; o < Lv.group_size[g]; o += blockDim.x) dst[o] = src[o];
  }
}

// ---------------------------------------------------------------------------
// level 0: banded elimination of every leaf interior straight from the stencil
// ---------------------------------------------------------------------------

// Merged batches: point the kernel's grid and stencil at cell c's problem;
// returns the first DOF of that problem in the concatenated numbering (0 for
// a single problem, whose grid and stencil are the kernel's arguments).
__device__ inline int64_t bind_cell_geo(const LevelDev& Lv, int c, GeoDev& G, const double*& diag,
                                        const double*& off) {
  if (!Lv.cell_prob) return 0;
  const BatchGeo& b = Lv.bgeo[Lv.cell_prob[c]];
  G = b.G;
  diag = b.diag;
  off = b.off;
  return b.base;
}

__device__ inline void coords1(const GeoDev& G, int64_t gid, int x[3]) {
  int64_t rem = gid;
  x[0] = x[1] = x[2] = 1;
  for (int a = 0; a < G.d; ++a) {
    x[a] = (int)(rem % G.ns[a]) + 1;
    rem /= G.ns[a];
  }
}

template <typename T>
__device__ inline T* frame_of(const LevelDev& Lv, int c, int* ld) {
  *ld = Lv.frame_ld[c];
  return (T*)Lv.frame_base + Lv.frame_off[c];
}

// Shared memory: band (nI x (w+1)) + position table + SYRK workspace + a
// panel of Z columns (at least 16, at most nB).
constexpr size_t kLeafSmemBudget = 200 * 1024;

template <typename T>
__host__ __device__ size_t leaf_fixed_smem(int max_nI, int max_w, int leaf, int d) {
  int tab = 1;
  for (int a = 0; a < d; ++a) tab *= leaf + 1;
  size_t band = (size_t)max_nI * (max_w + 1) * sizeof(T);
  band = (band + 15) & ~size_t(15);
  size_t t = ((size_t)tab * sizeof(int) + 15) & ~size_t(15);
  return band + t + 2 * kKC * (kTile + 1) * sizeof(T);
}

template <typename T>
__host__ __device__ int leaf_panel_cols(int max_nI, int max_nB, int max_w, int leaf, int d) {
  const size_t fixed = leaf_fixed_smem<T>(max_nI, max_w, leaf, d);
  if (max_nI == 0) return 16;
  size_t room = kLeafSmemBudget > fixed ? kLeafSmemBudget - fixed : 0;
  int cols = (int)(room / ((size_t)max_nI * sizeof(T)));
  cols = cols / 16 * 16;
  if (cols < 16) cols = 16;
  if (cols > max_nB) cols = (max_nB + 15) / 16 * 16;
  return cols;
}

template <typename T>
size_t leaf_smem_bytes(int max_nI, int max_nB, int max_w, int leaf, int d) {
  const int cols = leaf_panel_cols<T>(max_nI, max_nB, max_w, leaf, d);
  return leaf_fixed_smem<T>(max_nI, max_w, leaf, d) + (size_t)max_nI * cols * sizeof(T) + 16;
}

// A_II is the stencil restricted to the interior box of the leaf; in
// lexicographic order its half bandwidth is the box's x extent (2D) or x*y
// extent (3D), and its Cholesky factor stays inside that band, so
//   L        = banded chol(A_II)                      (band kept for the apply)
//   Z        = L^{-1} A_IB                            (scratch)
//   frame    = A_BB (this cell's share) - Z^T Z       (Eq. 2.1, Schur complement)
// reproduce Sec. 2.1 exactly.  A_IB has one entry per boundary DOF that faces
// the interior; it is kept as (interior index, value) for the apply.
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_leaf_elim(GeoDev G, LevelDev Lv, const double* diag, const double* off, int* status) {
  pdl_trigger();
  pdl_wait();   // what the previous kernel of the stream wrote
  extern __shared__ unsigned char smraw[];
  __shared__ int bad;
  const int c = blockIdx.x;
  const int nI = Lv.nI[c], nB = Lv.nB[c], n = nI + nB, w = Lv.band_w[c];
  const int w1 = w + 1;
  const int32_t* gid = Lv.gids + Lv.gid_off[c];
  const int64_t dbase = bind_cell_geo(Lv, c, G, diag, off);
  T* sband = (T*)smraw;
  size_t band_bytes = ((size_t)Lv.max_nI * (Lv.max_w + 1) * sizeof(T) + 15) & ~size_t(15);
  int* postab = (int*)(smraw + band_bytes);
  int tab = 1;
  for (int a = 0; a < G.d; ++a) tab *= G.leaf + 1;
  T* syrk_sm = (T*)((unsigned char*)postab + (((size_t)tab * sizeof(int) + 15) & ~size_t(15)));
  T* zp = syrk_sm + 2 * kKC * (kTile + 1);   // panel of Z columns, zp[k * pcols + j]
  const int pcols = leaf_panel_cols<T>(Lv.max_nI, Lv.max_nB, Lv.max_w, G.leaf, G.d);
  T* Z = (T*)Lv.zbuf + Lv.z_off[c];
  int ld;
  T* Fr = frame_of<T>(Lv, c, &ld);
  int* ci = Lv.cpl_i + Lv.b_off[c];
  T* ca = (T*)Lv.cpl_a + Lv.b_off[c];
  const int m = G.leaf, m1 = m + 1;
  int origin[3] = {0, 0, 0};
  {
    int64_t code = Lv.cell_code[c];
    for (int a = 0; a < G.d; ++a) {
      const int v = (int)(code % Lv.code_base);
      code /= Lv.code_base;
      origin[a] = ((v - 1) / 2) * m;
    }
  }
  if (threadIdx.x == 0) bad = 0;
  for (int i = threadIdx.x; i < tab; i += blockDim.x) postab[i] = -1;
  for (int i = threadIdx.x; i < nI * w1; i += blockDim.x) sband[i] = T(0);
  for (int64_t i = threadIdx.x; i < (int64_t)nB * nB; i += blockDim.x) Fr[i] = T(0);
  __syncthreads();
  for (int p = threadIdx.x; p < n; p += blockDim.x) {
    int x[3];
    coords1(G, gid[p] - dbase, x);
    int lin = 0, mul = 1;
    for (int a = 0; a < G.d; ++a) {
      lin += (x[a] - origin[a]) * mul;
      mul *= m1;
    }
    postab[lin] = p;
  }
  __syncthreads();
  // stencil entries: interior band, boundary couplings, this cell's share of A_BB
  for (int p = threadIdx.x; p < n; p += blockDim.x) {
    const int64_t g = gid[p] - dbase;
    int x[3];
    coords1(G, g, x);
    int lin = 0, mul = 1, lstride[3] = {1, 1, 1}, onplane = 0;
    for (int a = 0; a < G.d; ++a) {
      lin += (x[a] - origin[a]) * mul;
      lstride[a] = mul;
      mul *= m1;
      onplane += (x[a] % m == 0);
    }
    const int b = p - nI;
    if (p < nI) sband[p * w1] = T(diag[g]);
    else {
      Fr[b + (int64_t)b * ld] = T(diag[g] / double(1 << onplane));
      ci[b] = -1;
      ca[b] = T(0);
    }
    for (int a = 0; a < G.d; ++a) {
      const double share = double(1 << (onplane - (x[a] % m == 0)));
      const int lx = x[a] - origin[a];
      for (int dir = -1; dir <= 1; dir += 2) {
        if (dir > 0 && !(x[a] + 1 <= G.ns[a] && lx + 1 <= m)) continue;
        if (dir < 0 && !(x[a] - 1 >= 1 && lx - 1 >= 0)) continue;
        const int q = postab[lin + dir * lstride[a]];
        if (q < 0) continue;
        const double v = dir > 0 ? off[a * G.N + g] : off[a * G.N + g - G.stride[a]];
        if (p < nI) {
          if (q < nI && q > p) sband[p * w1 + (q - p)] = T(v);   // column p of A_II, below diagonal
        } else if (q < nI) {
          ci[b] = q;
          ca[b] = T(v);
        } else {
          Fr[b + (int64_t)(q - nI) * ld] = T(v / share);
        }
      }
    }
  }
  __syncthreads();
  // banded Cholesky, right-looking over columns (column k holds L[k..k+w, k])
  const bool cta_mode = w >= 32;
  if (cta_mode || threadIdx.x < 32) {
    const int nt = cta_mode ? blockDim.x : 32;
    for (int k = 0; k < nI; ++k) {
      T dkk = sband[k * w1];
      if (!(dkk > T(0))) {
        if (threadIdx.x == 0) bad = 1;
        dkk = T(1);
      }
      const T s = my_sqrt(dkk);
      const int wk = min(w, nI - 1 - k);
      if (cta_mode) __syncthreads(); else __syncwarp();
      for (int dd = 1 + threadIdx.x; dd <= wk; dd += nt) sband[k * w1 + dd] /= s;
      if (threadIdx.x == 0) sband[k * w1] = s;
      if (cta_mode) __syncthreads(); else __syncwarp();
      for (int idx = threadIdx.x; idx < wk * wk; idx += nt) {
        const int d1 = 1 + idx / wk, d2 = 1 + idx % wk;
        if (d2 > d1) continue;
        sband[(k + d2) * w1 + (d1 - d2)] -= sband[k * w1 + d1] * sband[k * w1 + d2];
      }
      if (cta_mode) __syncthreads(); else __syncwarp();
    }
  }
  __syncthreads();
  // Z = L^{-1} A_IB, stored Z[k*nB + b]; computed in shared-memory panels of
  // pcols boundary columns, one column per thread
  for (int b0 = 0; b0 < nB; b0 += pcols) {
    const int nc = min(pcols, nB - b0);
    for (int i = threadIdx.x; i < nI * pcols; i += blockDim.x) zp[i] = T(0);
    __syncthreads();
    for (int j = threadIdx.x; j < nc; j += blockDim.x) {
      const int b = b0 + j;
      const int i0 = ci[b];
      if (i0 < 0) continue;
      zp[i0 * pcols + j] = ca[b];
      for (int k = i0; k < nI; ++k) {
        const T zk = zp[k * pcols + j] / sband[k * w1];
        zp[k * pcols + j] = zk;
        const int wk = min(w, nI - 1 - k);
        for (int dd = 1; dd <= wk; ++dd) zp[(k + dd) * pcols + j] -= sband[k * w1 + dd] * zk;
      }
    }
    __syncthreads();
    for (int64_t i = threadIdx.x; i < (int64_t)nI * nc; i += blockDim.x) {
      const int k = (int)(i / nc), j = (int)(i % nc);
      Z[(int64_t)k * nB + b0 + j] = zp[k * pcols + j];
    }
    __syncthreads();
  }
  // frame -= Z^T Z
  cta_syrk_lower(Fr, ld, Z, nB, 0, nB, 0, nB, 0, nI, syrk_sm);
  T* band = (T*)Lv.band + Lv.band_off[c];
  for (int i = threadIdx.x; i < nI * w1; i += blockDim.x)
    band[i] = (i % w1 == 0) ? T(1) / sband[i] : sband[i];
  __syncthreads();
  if (threadIdx.x == 0 && bad) report(status, RHIF_ERR_NOT_SPD, 0, kKindCell, c);
}

// Streaming variant for leaves whose boundary fits one 64 x 64 register tile
// (2D): column k of the banded Cholesky, row k of Z = L^{-1} A_IB and the
// rank-1 update S += z_k z_k^T are done in one pass over k, keeping only a
// window of w+1 rows of Z in shared memory and S in registers (4 x 4 per
// thread).  The result equals the panel version's (same operations on the same
// entries, only Z is never stored).
constexpr int kStreamNB = 64;

template <typename T>
size_t leaf_stream_smem(int max_nI, int max_w, int leaf, int d) {
  int tab = 1;
  for (int a = 0; a < d; ++a) tab *= leaf + 1;
  size_t band = ((size_t)max_nI * (max_w + 1) * sizeof(T) + 15) & ~size_t(15);
  size_t win = ((size_t)(max_w + 1) * kStreamNB * sizeof(T) + 15) & ~size_t(15);
  size_t t = ((size_t)tab * sizeof(int) + 15) & ~size_t(15);
  size_t pairs = ((size_t)(max_w * (max_w + 1) / 2) * 2 * sizeof(short) + 15) & ~size_t(15);
  return band + win + t + pairs + 64;
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_leaf_stream(GeoDev G, LevelDev Lv, const double* diag, const double* off, int* status) {
  pdl_trigger();
  pdl_wait();   // what the previous kernel of the stream wrote
  extern __shared__ unsigned char smraw[];
  __shared__ int bad;
  __shared__ T s_piv, s_rpiv;
  const int c = blockIdx.x;
  const int nI = Lv.nI[c], nB = Lv.nB[c], n = nI + nB, w = Lv.band_w[c];
  const int w1 = w + 1;
  const int tid = threadIdx.x;
  const int32_t* gid = Lv.gids + Lv.gid_off[c];
  const int64_t dbase = bind_cell_geo(Lv, c, G, diag, off);
  unsigned char* p = smraw;
  T* sband = (T*)p;
  p += ((size_t)Lv.max_nI * (Lv.max_w + 1) * sizeof(T) + 15) & ~size_t(15);
  T* win = (T*)p;                                       // win[(k % w1) * 64 + b]
  p += ((size_t)(Lv.max_w + 1) * kStreamNB * sizeof(T) + 15) & ~size_t(15);
  int* postab = (int*)p;
  int tab = 1;
  for (int a = 0; a < G.d; ++a) tab *= G.leaf + 1;
  p += ((size_t)tab * sizeof(int) + 15) & ~size_t(15);
  short* pairs = (short*)p;                              // (d1, d2) with 1 <= d2 <= d1 <= w
  const int npair = w * (w + 1) / 2;
  int ld;
  T* Fr = frame_of<T>(Lv, c, &ld);
  int* ci = Lv.cpl_i + Lv.b_off[c];
  T* ca = (T*)Lv.cpl_a + Lv.b_off[c];
  const int m = G.leaf, m1 = m + 1;
  int origin[3] = {0, 0, 0};
  {
    int64_t code = Lv.cell_code[c];
    for (int a = 0; a < G.d; ++a) {
      const int v = (int)(code % Lv.code_base);
      code /= Lv.code_base;
      origin[a] = ((v - 1) / 2) * m;
    }
  }
  if (tid == 0) {
    bad = 0;
    int q = 0;
    for (int d1 = 1; d1 <= w; ++d1)
      for (int d2 = 1; d2 <= d1; ++d2) {
        pairs[2 * q] = (short)d1;
        pairs[2 * q + 1] = (short)d2;
        ++q;
      }
  }
  for (int i = tid; i < tab; i += blockDim.x) postab[i] = -1;
  for (int i = tid; i < nI * w1; i += blockDim.x) sband[i] = T(0);
  for (int i = tid; i < w1 * kStreamNB; i += blockDim.x) win[i] = T(0);
  for (int64_t i = tid; i < (int64_t)nB * nB; i += blockDim.x) Fr[i] = T(0);
  __syncthreads();
  for (int q = tid; q < n; q += blockDim.x) {
    int x[3];
    coords1(G, gid[q] - dbase, x);
    int lin = 0, mul = 1;
    for (int a = 0; a < G.d; ++a) {
      lin += (x[a] - origin[a]) * mul;
      mul *= m1;
    }
    postab[lin] = q;
  }
  __syncthreads();
  for (int q = tid; q < n; q += blockDim.x) {
    const int64_t g = gid[q] - dbase;
    int x[3];
    coords1(G, g, x);
    int lin = 0, mul = 1, lstride[3] = {1, 1, 1}, onplane = 0;
    for (int a = 0; a < G.d; ++a) {
      lin += (x[a] - origin[a]) * mul;
      lstride[a] = mul;
      mul *= m1;
      onplane += (x[a] % m == 0);
    }
    const int b = q - nI;
    if (q < nI) sband[q * w1] = T(diag[g]);
    else {
      Fr[b + (int64_t)b * ld] = T(diag[g] / double(1 << onplane));
      ci[b] = -1;
      ca[b] = T(0);
    }
    for (int a = 0; a < G.d; ++a) {
      const double share = double(1 << (onplane - (x[a] % m == 0)));
      const int lx = x[a] - origin[a];
      for (int dir = -1; dir <= 1; dir += 2) {
        if (dir > 0 && !(x[a] + 1 <= G.ns[a] && lx + 1 <= m)) continue;
        if (dir < 0 && !(x[a] - 1 >= 1 && lx - 1 >= 0)) continue;
        const int r = postab[lin + dir * lstride[a]];
        if (r < 0) continue;
        const double v = dir > 0 ? off[a * G.N + g] : off[a * G.N + g - G.stride[a]];
        if (q < nI) {
          if (r < nI && r > q) sband[q * w1 + (r - q)] = T(v);
        } else if (r < nI) {
          ci[b] = r;
          ca[b] = T(v);
        } else {
          Fr[b + (int64_t)(r - nI) * ld] = T(v / share);
        }
      }
    }
  }
  __syncthreads();
  // initial rows 0..w of the Z window: the single entry a_b of column b sits in row ci[b]
  for (int b = tid; b < nB; b += blockDim.x)
    if (ci[b] >= 0 && ci[b] <= w) win[(ci[b] % w1) * kStreamNB + b] = T(ca[b]);
  // fixed work assignment: Z-window column zb, rows 1 + zr0 + 4j; band pairs tid and tid + 256
  const int zb = tid & (kStreamNB - 1), zr0 = tid >> 6;
  const int my_ci = (tid < nB) ? ci[tid] : -1;
  const T my_ca = (tid < nB) ? T(ca[tid]) : T(0);
  int pd1[2] = {0, 0}, pd2[2] = {0, 0};
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int q = tid + h * kThreads;
    if (q < npair) {
      pd1[h] = pairs[2 * q];
      pd2[h] = pairs[2 * q + 1];
    }
  }
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int bq = 0; bq < 4; ++bq) acc[a][bq] = T(0);
  const int ti = (tid >> 4) * 4, tj = (tid & 15) * 4;   // this thread's 4 x 4 block of S
  int slot = 0;                                          // k % (w + 1)
  __syncthreads();
  for (int k = 0; k < nI; ++k) {
    const int wk = min(w, nI - 1 - k);
    T* zk = win + slot * kStreamNB;
    T* colk = sband + k * w1;
    // 1. pivot of column k
    if (tid == 0) {
      T dkk = colk[0];
      if (!(dkk > T(0))) {
        bad = 1;
        dkk = T(1);
      }
      s_piv = my_sqrt(dkk);
      s_rpiv = T(1) / s_piv;   // once, not per thread (FP64 divides are slow here)
      colk[0] = s_piv;
    }
    __syncthreads();
    const T rpiv = s_rpiv;
    // 2. scale column k of L and row k of Z
    if (tid >= 1 && tid <= wk) colk[tid] *= rpiv;
    if (tid < kStreamNB) zk[tid] *= rpiv;
    __syncthreads();
    // 3. trailing band update, Z rows k+1..k+wk, and S += z_k z_k^T
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int d1 = pd1[h], d2 = pd2[h];
      if (d1 && d1 <= wk) sband[(k + d2) * w1 + (d1 - d2)] -= colk[d1] * colk[d2];
    }
    {
      const T zv = zk[zb];
      int sl = slot + 1 + zr0;
      while (sl >= w1) sl -= w1;
      for (int dd = 1 + zr0; dd <= wk; dd += 4) {
        win[sl * kStreamNB + zb] -= colk[dd] * zv;
        sl += 4;
        while (sl >= w1) sl -= w1;
      }
    }
    {
      T zi[4], zj[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        zi[a] = zk[ti + a];
        zj[a] = zk[tj + a];
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int bq = 0; bq < 4; ++bq) acc[a][bq] += zi[a] * zj[bq];
    }
    __syncthreads();
    // 4. recycle row k's slot for row k + w + 1
    const int nr = k + w1;
    if (tid < kStreamNB) zk[tid] = (nr < nI && my_ci == nr) ? my_ca : T(0);
    slot = (slot + 1 == w1) ? 0 : slot + 1;
    __syncthreads();
  }
  // frame = A_BB share - S (lower triangle)
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int bq = 0; bq < 4; ++bq) {
      const int i = ti + a, j = tj + bq;
      if (i < nB && j < nB && i >= j) Fr[i + (int64_t)j * ld] -= acc[a][bq];
    }
  // band with reciprocal diagonal for the application
  T* band = (T*)Lv.band + Lv.band_off[c];
  for (int i = tid; i < nI * w1; i += blockDim.x)
    band[i] = T((i % w1 == 0) ? T(1) / sband[i] : sband[i]);
  __syncthreads();
  if (tid == 0 && bad) report(status, RHIF_ERR_NOT_SPD, 0, kKindCell, c);
}

// One warp per 2D leaf (interior box at most 15 wide, at most NBT <= 64
// boundary DOFs): the same column-by-column pass as k_leaf_stream, the same
// operations on the same entries in the same order, with no CTA barriers.
// The live parts of the band (columns k..k+15) and of Z = L^{-1} A_IB (rows
// k..k+15) sit in circular windows in shared memory; lane l owns Z columns l
// and l + 32 and keeps the matching columns of S = Z^T Z as register
// accumulators.  Columns of L leave the window as soon as they are final
// (reciprocal diagonal, as the application reads it).
constexpr int kLeafWarpW = 15;   // largest band half-width
constexpr int kLeafWarpCta = 4;  // warps (leaves) per CTA

template <typename T>
__host__ __device__ inline size_t leaf_warp_bytes(int max_nI, int leaf, int nbt) {
  const size_t tab = (size_t)(leaf + 1) * (leaf + 1) * sizeof(int);
  const size_t cols = (size_t)3 * max_nI * sizeof(T);
  const size_t win = 16 * 16 * sizeof(T) + (size_t)16 * nbt * sizeof(T);
  return ((tab + 15) & ~size_t(15)) + ((cols + 15) & ~size_t(15)) + ((win + 15) & ~size_t(15));
}

template <typename T, int NBT>
__global__ void __launch_bounds__(32 * kLeafWarpCta)
k_leaf_warp(GeoDev G, LevelDev Lv, const double* diag, const double* off, int* status) {
  pdl_trigger();
  pdl_wait();   // what the previous kernel of the stream wrote
  constexpr int CPL = NBT / 32;   // boundary columns per lane
  extern __shared__ __align__(16) unsigned char smraw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = blockIdx.x * kLeafWarpCta + warp;
  if (c >= Lv.ncell) return;
  const int nI = Lv.nI[c], nB = Lv.nB[c], n = nI + nB, w = Lv.band_w[c];
  const int m = G.leaf, m1 = m + 1;
  unsigned char* base = smraw + (size_t)warp * leaf_warp_bytes<T>(Lv.max_nI, m, NBT);
  int* postab = (int*)base;
  base += ((size_t)m1 * m1 * sizeof(int) + 15) & ~size_t(15);
  T* dg = (T*)base;                 // A_II: diagonal, x-neighbour (d = 1), y-neighbour (d = w)
  T* ax = dg + Lv.max_nI;
  T* ay = ax + Lv.max_nI;
  base += ((size_t)3 * Lv.max_nI * sizeof(T) + 15) & ~size_t(15);
  T* bw = (T*)base;                 // band window: column k in slot k & 15, entry d = L[k+d, k]
  T* zw = bw + 256;                 // Z window: row k in slot k & 15 (NBT entries)
  const int32_t* gid = Lv.gids + Lv.gid_off[c];
  const int64_t dbase = bind_cell_geo(Lv, c, G, diag, off);
  int ld;
  T* Fr = frame_of<T>(Lv, c, &ld);
  int* ci = Lv.cpl_i + Lv.b_off[c];
  T* ca = (T*)Lv.cpl_a + Lv.b_off[c];
  int origin[2] = {0, 0};
  {
    int64_t code = Lv.cell_code[c];
    for (int a = 0; a < 2; ++a) {
      const int v = (int)(code % Lv.code_base);
      code /= Lv.code_base;
      origin[a] = ((v - 1) / 2) * m;
    }
  }
  // 1. stencil entries: interior columns, couplings, this cell's share of A_BB
  for (int i = lane; i < m1 * m1; i += 32) postab[i] = -1;
  for (int j = 0; j < nB; ++j)
    for (int i = lane; i < nB; i += 32) Fr[i + (int64_t)j * ld] = T(0);
  __syncwarp();
  for (int q = lane; q < n; q += 32) {
    int x[3];
    coords1(G, gid[q] - dbase, x);
    postab[(x[0] - origin[0]) + (x[1] - origin[1]) * m1] = q;
  }
  __syncwarp();
  for (int q = lane; q < n; q += 32) {
    const int64_t g = gid[q] - dbase;
    int x[3];
    coords1(G, g, x);
    const int lin = (x[0] - origin[0]) + (x[1] - origin[1]) * m1;
    const int onplane = (x[0] % m == 0) + (x[1] % m == 0);
    const int b = q - nI;
    if (q < nI) {
      dg[q] = T(diag[g]);
      ax[q] = T(0);
      ay[q] = T(0);
    } else {
      Fr[b + (int64_t)b * ld] = T(diag[g] / double(1 << onplane));
      ci[b] = -1;
      ca[b] = T(0);
    }
    for (int a = 0; a < 2; ++a) {
      const double share = double(1 << (onplane - (x[a] % m == 0)));
      const int lx = x[a] - origin[a];
      const int lstride = a == 0 ? 1 : m1;
      for (int dir = -1; dir <= 1; dir += 2) {
        if (dir > 0 && !(x[a] + 1 <= G.ns[a] && lx + 1 <= m)) continue;
        if (dir < 0 && !(x[a] - 1 >= 1 && lx - 1 >= 0)) continue;
        const int r = postab[lin + dir * lstride];
        if (r < 0) continue;
        const double v = dir > 0 ? off[a * G.N + g] : off[a * G.N + g - G.stride[a]];
        if (q < nI) {
          if (r < nI && r > q) (a == 0 ? ax : ay)[q] = T(v);
        } else if (r < nI) {
          ci[b] = r;
          ca[b] = T(v);
        } else {
          Fr[b + (int64_t)(r - nI) * ld] = T(v / share);
        }
      }
    }
  }
  __syncwarp();
  // 2. initial windows: band columns 0..15, Z rows 0..15 (A_IB has one entry per column)
  for (int i = lane; i < 256; i += 32) {
    const int col = i >> 4, d = i & 15;
    T v = T(0);
    if (col < nI) {
      if (d == 0) v = dg[col];
      if (d == 1) v += ax[col];
      if (d == w) v += ay[col];
    }
    bw[i] = v;
  }
  int my_ci[CPL];
  T my_ca[CPL];
#pragma unroll
  for (int h = 0; h < CPL; ++h) {
    const int b = lane + 32 * h;
    my_ci[h] = b < nB ? ci[b] : -1;
    my_ca[h] = b < nB ? ca[b] : T(0);
  }
  for (int r = 0; r < 16; ++r)
#pragma unroll
    for (int h = 0; h < CPL; ++h) zw[r * NBT + lane + 32 * h] = my_ci[h] == r ? my_ca[h] : T(0);
  // trailing-update pairs (d1, d2), 1 <= d2 <= d1 <= w, four per lane
  int pd1[4], pd2[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int q = lane + 32 * u;
    int d1 = 1, rem = q;
    while (rem >= d1) {
      rem -= d1;
      ++d1;
    }
    pd1[u] = d1 <= w ? d1 : 0;
    pd2[u] = rem + 1;
  }
  T acc[CPL][NBT];
#pragma unroll
  for (int h = 0; h < CPL; ++h)
#pragma unroll
    for (int i = 0; i < NBT; ++i) acc[h][i] = T(0);
  int bad = 0;
  T* band = (T*)Lv.band + Lv.band_off[c];
  const int w1 = w + 1;
  __syncwarp();
  // 3. column k of the band Cholesky, row k of Z, S += z_k z_k^T
#pragma unroll 1
  for (int k = 0; k < nI; ++k) {
    const int wk = min(w, nI - 1 - k);
    T* colk = bw + (k & 15) * 16;
    T* zk_row = zw + (k & 15) * NBT;
    T dkk = colk[0];
    if (!(dkk > T(0))) {
      bad = 1;
      dkk = T(1);
    }
    const T sp = my_sqrt(dkk);
    const T rp = T(1) / sp;
    __syncwarp();
    if (lane == 0) colk[0] = sp;
    else if (lane <= wk) colk[lane] *= rp;
    T zk[CPL];
#pragma unroll
    for (int h = 0; h < CPL; ++h) {
      zk[h] = zk_row[lane + 32 * h] * rp;
      zk_row[lane + 32 * h] = zk[h];
    }
    __syncwarp();
    if (lane <= w) band[(int64_t)k * w1 + lane] = lane == 0 ? T(1) / sp : (lane <= wk ? colk[lane] : T(0));
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int d1 = pd1[u], d2 = pd2[u];
      if (d1 && d1 <= wk) bw[((k + d2) & 15) * 16 + (d1 - d2)] -= colk[d1] * colk[d2];
    }
    for (int d = 1; d <= wk; ++d) {
      const T l = colk[d];
      T* zr = zw + ((k + d) & 15) * NBT + lane;
#pragma unroll
      for (int h = 0; h < CPL; ++h) zr[32 * h] -= l * zk[h];
    }
#pragma unroll
    for (int i4 = 0; i4 < NBT; i4 += 4) {
      T zi[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) zi[e] = zk_row[i4 + e];
#pragma unroll
      for (int h = 0; h < CPL; ++h)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[h][i4 + e] += zi[e] * zk[h];
    }
    __syncwarp();
    // slot k becomes column / row k + 16
    const int nc = k + 16;
    if (lane < 16) {
      T v = T(0);
      if (nc < nI) {
        if (lane == 0) v = dg[nc];
        if (lane == 1) v += ax[nc];
        if (lane == w) v += ay[nc];
      }
      colk[lane] = v;
    }
#pragma unroll
    for (int h = 0; h < CPL; ++h) zk_row[lane + 32 * h] = my_ci[h] == nc ? my_ca[h] : T(0);
    __syncwarp();
  }
  // 4. frame = A_BB share - S, lower triangle written as rows j >= i of column i
#pragma unroll
  for (int h = 0; h < CPL; ++h) {
    const int j = lane + 32 * h;
#pragma unroll
    for (int i = 0; i < NBT; ++i)
      if (i <= j && j < nB) Fr[j + (int64_t)i * ld] -= acc[h][i];
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) report(status, RHIF_ERR_NOT_SPD, 0, kKindCell, c);
}

// ---------------------------------------------------------------------------
// level >= 1 fronts: extend-add of the children's frames, children in a fixed order
// ---------------------------------------------------------------------------

// Extend-add of child slot `slot` of every parent cell: the child's Schur
// complement (lower triangle of its frame) is added into the parent front
// through the position map.  A child's positions map to distinct parent
// positions, so the CTAs of one launch (a chunk of one child's entries each)
// write disjoint entries; slots run as successive launches, so the sum over
// the children of a parent is taken in slot order, as a fixed-order gather.
template <typename T>
__global__ void k_extend_add(LevelDev cur, LevelDev prev, int slot, int chunk) {
  pdl_trigger();
  pdl_wait();   // what the previous kernel of the stream wrote
  const int c = blockIdx.y;
  const int k = cur.ea_off[c] + slot;
  if (k >= cur.ea_off[c + 1]) return;
  const int n = cur.nI[c] + cur.nB[c];
  T* F = (T*)cur.front + cur.front_off[c];
  const int pc = cur.ea_child[k];
  const int* map = cur.ea_map + cur.ea_map_off[k];
  const int nbc = prev.nB[pc];
  int ldc;
  const T* Fc = frame_of<T>(prev, pc, &ldc);
  const int64_t e0 = (int64_t)blockIdx.x * chunk, e1 = min(e0 + chunk, (int64_t)nbc * nbc);
  for (int64_t idx = e0 + threadIdx.x; idx < e1; idx += blockDim.x) {
    const int i = (int)(idx % nbc), j = (int)(idx / nbc);
    if (i < j) continue;
    const int pi = map[i], pj = map[j];
    if (pi < 0 || pj < 0) continue;
    const int r = max(pi, pj), q = min(pi, pj);
    F[r + (int64_t)q * n] += Fc[i + (int64_t)j * ldc];
  }
}

// One CTA per parent cell, for fronts whose children's frames are small: the
// front is zeroed, then the children's frames are added in slot order (the
// order of the per-slot launches above), with a barrier between children
// (two children can share entries of the front).  One launch replaces the
// memset and the per-slot launches.
constexpr int kEaCellThreads = 512;

template <typename T>
__global__ void __launch_bounds__(kEaCellThreads) k_extend_add_cell(LevelDev cur, LevelDev prev) {
  pdl_trigger();
  pdl_wait();   // what the previous kernel of the stream wrote
  const int c = blockIdx.x;
  const int n = cur.nI[c] + cur.nB[c];
  T* F = (T*)cur.front + cur.front_off[c];
  for (int64_t idx = threadIdx.x; idx < (int64_t)n * n; idx += blockDim.x) F[idx] = T(0);
  for (int k = cur.ea_off[c]; k < cur.ea_off[c + 1]; ++k) {
    __syncthreads();
    const int pc = cur.ea_child[k];
    const int* map = cur.ea_map + cur.ea_map_off[k];
    const int nbc = prev.nB[pc];
    int ldc;
    const T* Fc = frame_of<T>(prev, pc, &ldc);
    for (int64_t idx = threadIdx.x; idx < (int64_t)nbc * nbc; idx += blockDim.x) {
      const int i = (int)(idx % nbc), j = (int)(idx / nbc);
      if (i < j) continue;
      const int pi = map[i], pj = map[j];
      if (pi < 0 || pj < 0) continue;
      const int r = max(pi, pj), q = min(pi, pj);
      F[r + (int64_t)q * n] += Fc[i + (int64_t)j * ldc];
    }
  }
}

// Leaf bands with w <= kBandInvW: replace the in-block entries of every
// diagonal w x w block of L (blocks start at multiples of w) by the entries
// of its inverse X (lower triangular; the diagonal slots already hold
// 1/L_kk = X_kk).  One warp per cell, lane c computes column c of X by
// forward substitution, X[r,c] = -(1/L_rr) sum_{k=c}^{r-1} L[r,k] X[k,c].
template <typename T>
__global__ void k_band_block_inverse(LevelDev Lv) {
  pdl_trigger();
  pdl_wait();   // what the previous kernel of the stream wrote
  const int lane = threadIdx.x & 31;
  const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (c >= Lv.ncell) return;
  const int n = Lv.nI[c], w = Lv.band_w[c];
  if (w < 1 || w > kBandInvW) return;
  const int w1 = w + 1;
  T* band = (T*)Lv.band + Lv.band_off[c];
  for (int s0 = 0; s0 < n; s0 += w) {
    const int B = min(w, n - s0);
    T x[kBandInvW];
    if (lane < B) {
      x[lane] = band[(s0 + lane) * w1];
      for (int r = lane + 1; r < B; ++r) {
        T s = T(0);
        for (int k = lane; k < r; ++k) s += band[(s0 + k) * w1 + (r - k)] * x[k];
        x[r] = -s * band[(s0 + r) * w1];
      }
    }
    __syncwarp();
    if (lane < B)
      for (int r = lane + 1; r < B; ++r) band[(s0 + lane) * w1 + (r - lane)] = x[r];
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// cell elimination (Sec. 2.1) of dense fronts: partial Cholesky
// ---------------------------------------------------------------------------

template <typename T>
__global__ void __launch_bounds__(kThreads) k_partial_chol(LevelDev Lv, int* status) {
  pdl_trigger();
  pdl_wait();   // what the previous kernel of the stream wrote
  extern __shared__ unsigned char smraw[];
  T* sm = (T*)smraw;
  const int c = blockIdx.x;
  const int nI = Lv.nI[c], n = nI + Lv.nB[c];
  T* F = (T*)Lv.front + Lv.front_off[c];
  if (!cta_partial_chol(F, n, n, nI, sm) && threadIdx.x == 0)
    report(status, RHIF_ERR_NOT_SPD, Lv.level, kKindCell, c);
}

// ---------------------------------------------------------------------------
// cell elimination of large fronts, spread over many CTAs: one launch per
// 32-column panel factors the diagonal block and scales the panel (one CTA per
// front), the next updates the trailing columns still to be eliminated tile by
// tile (one CTA per 64 x 64 tile of every front), and a final launch forms the
// Schur complement of the boundary block, C_BB -= W W^T, tile by tile.
// ---------------------------------------------------------------------------

// Panel at p0 of every front, in two launches: the nb x nb diagonal block
// (one CTA per front) and the rows below it (one CTA per 256 rows of a front,
// the factored block staged in shared memory).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_front_pdiag(LevelDev Lv, int p0, int* status) {
  pdl_trigger();
  pdl_wait();   // what the previous kernel of the stream wrote
  extern __shared__ unsigned char smraw[];
  const int c = blockIdx.x;
  const int nI = Lv.nI[c], n = nI + Lv.nB[c];
  if (p0 >= nI) return;
  T* F = (T*)Lv.front + Lv.front_off[c];
  const int nb = min(kNB, nI - p0);
  if (!cta_diag_chol(F, n, p0, nb, (T*)smraw) && threadIdx.x == 0)
    report(status, RHIF_ERR_NOT_SPD, Lv.level, kKindCell, c);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_front_prows(LevelDev Lv, int p0) {
  pdl_trigger();
  pdl_wait();   // what the previous kernel of the stream wrote
  extern __shared__ unsigned char smraw[];
  T* D = (T*)smraw;
  const int c = blockIdx.y;
  const int nI = Lv.nI[c], n = nI + Lv.nB[c];
  if (p0 >= nI) return;
  const int nb = min(kNB, nI - p0);
  const int r0 = p0 + nb + blockIdx.x * kThreads;
  if (r0 >= n) return;
  T* F = (T*)Lv.front + Lv.front_off[c];
  for (int idx = threadIdx.x; idx < nb * nb; idx += blockDim.x) {
    const int i = idx % nb, j = idx / nb;
    D[i * (kNB + 1) + j] = (i >= j) ? F[(p0 + i) + (int64_t)(p0 + j) * n] : T(0);
  }
  __syncthreads();
  cta_panel_rows(F, n, r0, min(n, r0 + kThreads), p0, nb, D);
}

__host__ __device__ inline int64_t trail_tiles(int nI, int n, int p0) {
  if (p0 >= nI) return 0;
  const int p1 = min(p0 + kNB, nI);
  const int64_t tr = (n - p1 + kTile - 1) / kTile, tc = (nI - p1 + kTile - 1) / kTile;
  return tr * tc;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_front_trailing(LevelDev Lv, int p0) {
  pdl_trigger();
  pdl_wait();   // what the previous kernel of the stream wrote
  extern __shared__ unsigned char smraw[];
  int64_t bid = blockIdx.x;
  int c = 0;
  for (; c < Lv.ncell; ++c) {
    const int64_t t = trail_tiles(Lv.nI[c], Lv.nI[c] + Lv.nB[c], p0);
    if (bid < t) break;
    bid -= t;
  }
  if (c >= Lv.ncell) return;
  const int nI = Lv.nI[c], n = nI + Lv.nB[c];
  const int p1 = min(p0 + kNB, nI);
  const int tc = (nI - p1 + kTile - 1) / kTile;
  const int a = (int)(bid / tc), b = (int)(bid % tc);
  if (b > a) return;   // above the diagonal
  T* F = (T*)Lv.front + Lv.front_off[c];
  cta_syrk_tile(F, n, F, n, p1 + a * kTile, p1 + b * kTile, n, nI, p0, p1, (T*)smraw);
}

__host__ __device__ inline int64_t schur_tiles(int nI, int nB) {
  if (nI == 0 || nB == 0) return 0;
  const int64_t t = (nB + kTile - 1) / kTile;
  return t * t;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_front_schur(LevelDev Lv) {
  pdl_trigger();
  pdl_wait();   // what the previous kernel of the stream wrote
  extern __shared__ unsigned char smraw[];
  int64_t bid = blockIdx.x;
  int c = 0;
  for (; c < Lv.ncell; ++c) {
    const int64_t t = schur_tiles(Lv.nI[c], Lv.nB[c]);
    if (bid < t) break;
    bid -= t;
  }
  if (c >= Lv.ncell) return;
  const int nI = Lv.nI[c], nB = Lv.nB[c], n = nI + nB;
  const int t = (nB + kTile - 1) / kTile;
  const int a = (int)(bid / t), b = (int)(bid % t);
  if (b > a) return;
  T* F = (T*)Lv.front + Lv.front_off[c];
  cta_syrk_tile(F, n, F, n, nI + a * kTile, nI + b * kTile, n, n, 0, nI, (T*)smraw);
}

// Explicit inverse of the interior factor L of large fronts, for the
// many-CTA application of the factor: one CTA per (cell, 64-column block J)
// solves L X[:, J] = E[:, J] by 64-row blocks from the diagonal down
// (tile product with the rows above, then a per-column solve with the
// diagonal block staged in shared memory) into X (per-cell offset xoff[c],
// column-major, leading dimension nI); k_front_inv_store then overwrites the
// lower triangle of L with X.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_front_trinv(LevelDev Lv, T* X, const int64_t* xoff) {
  pdl_trigger();
  pdl_wait();   // what the previous kernel of the stream wrote
  extern __shared__ unsigned char smraw[];
  const int c = blockIdx.y;
  const int nI = Lv.nI[c], n = nI + Lv.nB[c];
  const int J0 = blockIdx.x * kTile;
  if (J0 >= nI) return;
  cta_trinv_block((const T*)Lv.front + Lv.front_off[c], n, nI, X + xoff[c], nI, J0, (T*)smraw);
}

// L_g^{-1} of every preconditioned group, one CTA per (group, 64-column
// block), into Ph.Linv (same layout as Lbuf, upper triangle zero).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_group_trinv(LevelDev Lv, PhaseDev Ph) {
  pdl_trigger();
  pdl_wait();   // what the previous kernel of the stream wrote
  extern __shared__ unsigned char smraw[];
  const int b = blockIdx.y;
  const int sz = Lv.group_size[Ph.pre_group[b]];
  const int J0 = blockIdx.x * kTile;
  if (J0 >= sz) return;
  const T* Lg = (const T*)Ph.Lbuf + Ph.pre_off[b];
  T* X = (T*)Ph.Linv + Ph.pre_off[b];
  const int nc = min(kTile, sz - J0);
  for (int idx = threadIdx.x; idx < J0 * nc; idx += blockDim.x)
    X[(idx % J0) + (int64_t)(J0 + idx / J0) * sz] = T(0);
  cta_trinv_block(Lg, sz, sz, X, sz, J0, (T*)smraw);
}

// L_rr^{-1} of every skeletonization unit (the leading r x r block of its
// record, r = n - rank), one CTA per (unit, 64-column block), into X laid out
// like the records.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_unit_trinv(LevelDev Lv, PhaseDev Ph, T* X) {
  pdl_trigger();
  pdl_wait();   // what the previous kernel of the stream wrote
  extern __shared__ unsigned char smraw[];
  const int u = blockIdx.y;
  const int n = Lv.group_size[Ph.u_group[u]];
  const int r = n - Ph.rank[u];
  const int J0 = blockIdx.x * kTile;
  if (J0 >= r) return;
  const T* Fu = (const T*)Ph.rec + Ph.u_rec_off[u];
  cta_trinv_block(Fu, n, r, X + Ph.u_rec_off[u], n, J0, (T*)smraw);
}

// Lower triangle of every unit's L_rr^{-1} from X back into its record.
template <typename T>
__global__ void k_unit_inv_store(LevelDev Lv, PhaseDev Ph, const T* X) {
  pdl_trigger();
  pdl_wait();   // what the previous kernel of the stream wrote
  const int u = blockIdx.y;
  const int n = Lv.group_size[Ph.u_group[u]];
  const int r = n - Ph.rank[u];
  T* Fu = (T*)Ph.rec + Ph.u_rec_off[u];
  const T* Xu = X + Ph.u_rec_off[u];
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < r * r; idx += gridDim.x * blockDim.x) {
    const int i = idx % r, j = idx / r;
    if (i >= j) Fu[i + (int64_t)j * n] = Xu[i + (int64_t)j * n];
  }
}

// Inverses of lower-triangular blocks of order m <= 32, one warp each, the
// block staged in shared memory: lane c forms column c of X = L^{-1} by
// forward substitution.  UNIT: the leading r x r block of every unit record,
// in place; otherwise every L_g into Ph.Linv (upper triangle zero; the
// block-Jacobi factors of at most 32 DOFs get theirs from k_precond_diag_warp).
template <typename T>
constexpr int trinv_warps() { return sizeof(T) == 4 ? 4 : 2; }   // 33.8 KB of static shared memory

template <typename T, bool UNIT>
__global__ void __launch_bounds__(32 * trinv_warps<T>()) k_trinv_warp(LevelDev Lv, PhaseDev Ph, int count) {
  pdl_trigger();
  pdl_wait();   // what the previous kernel of the stream wrote
  constexpr int W = trinv_warps<T>();
  __shared__ T Ls[W][32][33];
  __shared__ T Xs[W][32][33];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int item = blockIdx.x * W + warp;
  if (item >= count) return;
  const T* L;
  T* out;
  int m, ld;
  if (UNIT) {
    const int n = Lv.group_size[Ph.u_group[item]];
    m = n - Ph.rank[item];
    ld = n;
    out = (T*)Ph.rec + Ph.u_rec_off[item];
    L = out;
  } else {
    m = Lv.group_size[Ph.pre_group[item]];
    ld = m;
    L = (const T*)Ph.Lbuf + Ph.pre_off[item];
    out = (T*)Ph.Linv + Ph.pre_off[item];
  }
  T (*Lw)[33] = Ls[warp];
  T (*Xw)[33] = Xs[warp];
  for (int idx = lane; idx < m * m; idx += 32) {
    const int i = idx % m, j = idx / m;
    Lw[i][j] = i >= j ? L[i + (int64_t)j * ld] : T(0);
  }
  __syncwarp();
  const int c = lane;
  for (int i = 0; i < m; ++i) {
    if (c <= i) {
      T v = i == c ? T(1) : T(0);
      for (int j = c; j < i; ++j) v -= Lw[i][j] * Xw[j][c];
      Xw[i][c] = v / Lw[i][i];
    }
  }
  __syncwarp();
  for (int idx = lane; idx < m * m; idx += 32) {
    const int i = idx % m, j = idx / m;
    if (i >= j) out[i + (int64_t)j * ld] = Xw[i][j];
    else if (!UNIT) out[i + (int64_t)j * ld] = T(0);
  }
}

template <typename T>
__global__ void k_front_inv_store(LevelDev Lv, const T* X, const int64_t* xoff) {
  pdl_trigger();
  pdl_wait();   // what the previous kernel of the stream wrote
  const int c = blockIdx.y;
  const int nI = Lv.nI[c], n = nI + Lv.nB[c];
  T* F = (T*)Lv.front + Lv.front_off[c];
  const T* Xc = X + xoff[c];
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < (int64_t)nI * nI;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx % nI), j = (int)(idx / nI);
    if (i >= j) F[i + (int64_t)j * n] = Xc[idx];
  }
}

// ---------------------------------------------------------------------------
// block Jacobi preconditioning (Sec. 2.3)
// ---------------------------------------------------------------------------

// L_g = chol(sum over the cells holding g of their diagonal block of g); with
// the diagonal local preconditioner (Sec. 5: any local preconditioner may
// replace block Cholesky) only the diagonal of that block is assembled, so
// L_g = diag(A_gg)^{1/2} and every later step sees a diagonal L_g.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_precond_diag(LevelDev Lv, PhaseDev Ph, int* status) {
  pdl_trigger();
  pdl_wait();   // what the previous kernel of the stream wrote
  extern __shared__ unsigned char smraw[];
  T* sm = (T*)smraw;
  const int b = blockIdx.x;
  const int g = Ph.pre_group[b];
  const int sz = Lv.group_size[g];
  T* Lg = (T*)Ph.Lbuf + Ph.pre_off[b];
  for (int64_t idx = threadIdx.x; idx < (int64_t)sz * sz; idx += blockDim.x) {
    const int i = (int)(idx % sz), j = (int)(idx / sz);
    T s = T(0);
    if (i == j || (i > j && !Ph.diag_only)) {
      for (int k = Lv.group_cell_off[g]; k < Lv.group_cell_off[g + 1]; ++k) {
        int ld;
        const T* fr = frame_of<T>(Lv, Lv.group_cell[k], &ld);
        const int pos = Lv.group_pos[k];
        s += fr[(pos + i) + (int64_t)(pos + j) * ld];
      }
    }
    Lg[idx] = s;
  }
  __syncthreads();
  if (!cta_partial_chol(Lg, sz, sz, sz, sm) && threadIdx.x == 0)
    report(status, RHIF_ERR_NOT_SPD, Lv.level, kKindGroup, g);
}

// Groups of at most 32 DOFs, one warp each: L_g = chol(sum over the cells
// holding g of their diagonal block of g) (written to Lbuf) and L_g^{-1}
// (written to Linv), the block staged in shared memory, lane = row.
template <typename T>
constexpr int pdiag_warps() { return sizeof(T) == 4 ? 4 : 2; }   // 33.8 KB of static shared memory

template <typename T>
__global__ void __launch_bounds__(32 * pdiag_warps<T>())
k_precond_diag_warp(LevelDev Lv, PhaseDev Ph, int* status) {
  pdl_trigger();
  pdl_wait();   // what the previous kernel of the stream wrote
  constexpr int W = pdiag_warps<T>();
  __shared__ T Ls[W][32][33];
  __shared__ T Xs[W][32][33];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int b = blockIdx.x * W + warp;
  if (b >= Ph.npre) return;
  const int g = Ph.pre_group[b];
  const int sz = Lv.group_size[g];
  T (*A)[33] = Ls[warp];
  T (*X)[33] = Xs[warp];
  for (int idx = lane; idx < sz * sz; idx += 32) {
    const int i = idx % sz, j = idx / sz;
    T v = T(0);
    if (i == j || (i > j && !Ph.diag_only))
      for (int k = Lv.group_cell_off[g]; k < Lv.group_cell_off[g + 1]; ++k) {
        int ld;
        const T* fr = frame_of<T>(Lv, Lv.group_cell[k], &ld);
        const int pos = Lv.group_pos[k];
        v += fr[(pos + i) + (int64_t)(pos + j) * ld];
      }
    A[i][j] = v;
  }
  __syncwarp();
  int bad = 0;
  for (int k = 0; k < sz; ++k) {   // right-looking, lane = row
    T piv = A[k][k];
    if (!(piv > T(0))) {
      bad = 1;
      piv = T(1);
    }
    const T d = my_sqrt(piv);
    __syncwarp();
    if (lane == k) A[k][k] = d;
    else if (lane > k && lane < sz) A[lane][k] /= d;
    __syncwarp();
    if (lane > k && lane < sz) {
      const T lik = A[lane][k];
      for (int j = k + 1; j <= lane; ++j) A[lane][j] -= lik * A[j][k];
    }
    __syncwarp();
  }
  if (bad && lane == 0) report(status, RHIF_ERR_NOT_SPD, Lv.level, kKindGroup, g);
  const int c = lane;   // column c of X = L^{-1} by forward substitution
  for (int i = 0; i < sz; ++i) {
    if (c <= i && c < sz) {
      T v = i == c ? T(1) : T(0);
      for (int j = c; j < i; ++j) v -= A[i][j] * X[j][c];
      X[i][c] = v / A[i][i];
    }
  }
  __syncwarp();
  T* Lg = (T*)Ph.Lbuf + Ph.pre_off[b];
  T* Xg = (T*)Ph.Linv + Ph.pre_off[b];
  for (int idx = lane; idx < sz * sz; idx += 32) {
    const int i = idx % sz, j = idx / sz;
    Lg[idx] = i >= j ? A[i][j] : T(0);
    Xg[idx] = i >= j ? X[i][j] : T(0);
  }
}

// frame <- D^{-1} frame D^{-T}, D = block diag of the L_g of the frame's groups.
// stage: work on a symmetric copy in shared memory with an odd leading
// dimension (the row pass walks along rows of the copy, one column per
// thread: an even one puts a warp's accesses in one bank).  xstage: the
// L_g^{-1} of the cell's segments are copied beside it, max_group^2 apart.
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_precond_scale(LevelDev Lv, PhaseDev Ph, int stage, int xstage) {
  pdl_trigger();
  pdl_wait();   // what the previous kernel of the stream wrote
  extern __shared__ unsigned char smraw[];
  const int c = blockIdx.x;
  int gld;
  T* Fg = frame_of<T>(Lv, c, &gld);
  const int nb = Lv.nB[c];
  T* Fr = Fg;
  int ld = gld;
  const int s0 = Lv.seg_off[c], s1 = Lv.seg_off[c + 1];
  const int64_t mg2 = (int64_t)Lv.max_group * Lv.max_group;
  T* Xs = nullptr;
  if (stage) {   // work on a full symmetric copy in shared memory
    Fr = (T*)smraw;
    ld = nb | 1;
    for (int64_t idx = threadIdx.x; idx < (int64_t)nb * nb; idx += blockDim.x) {
      const int i = (int)(idx % nb), j = (int)(idx / nb);
      Fr[i + (int64_t)j * ld] = sym_at(Fg, gld, i, j);
    }
    if (xstage && Ph.Linv && !Ph.diag_only) {
      Xs = (T*)(smraw + round16((size_t)Lv.max_nB * (Lv.max_nB | 1) * sizeof(T)));
      for (int q = s0; q < s1; ++q) {
        const int g = Lv.seg_group[q];
        const int pi = Ph.group_pre[g];
        if (pi < 0) continue;
        const int sz = Lv.group_size[g];
        const T* src = (const T*)Ph.Linv + Ph.pre_off[pi];
        T* dst = Xs + (q - s0) * mg2;
        for (int i = threadIdx.x; i < sz * sz; i += blockDim.x) dst[i] = src[i];
      }
    }
  } else {
    for (int64_t idx = threadIdx.x; idx < (int64_t)nb * nb; idx += blockDim.x) {
      const int i = (int)(idx % nb), j = (int)(idx / nb);
      if (i < j) Fr[i + (int64_t)j * ld] = Fr[j + (int64_t)i * ld];
    }
  }
  __syncthreads();
  const int64_t work = (int64_t)(s1 - s0) * nb;
  // rows: F[g, :] <- L_g^{-1} F[g, :]
  for (int64_t t = threadIdx.x; t < work; t += blockDim.x) {
    const int s = s0 + (int)(t / nb), j = (int)(t % nb);
    const int g = Lv.seg_group[s];
    const int pi = Ph.group_pre[g];
    if (pi < 0) continue;
    const int sz = Lv.group_size[g];
    const int pos = Lv.seg_pos[s];
    T* col = Fr + (int64_t)j * ld + pos;
    if (Ph.diag_only) {   // diagonal L_g: scale the rows
      const T* Dg = (const T*)(Ph.Linv ? Ph.Linv : Ph.Lbuf) + Ph.pre_off[pi];
      for (int a = 0; a < sz; ++a)
        col[a] = Ph.Linv ? col[a] * Dg[a + (int64_t)a * sz] : col[a] / Dg[a + (int64_t)a * sz];
      continue;
    }
    if (Ph.Linv) {   // col <- L_g^{-1} col as a product, bottom up in place
      const T* Xg = Xs ? Xs + (s - s0) * mg2 : (const T*)Ph.Linv + Ph.pre_off[pi];
      for (int a = sz - 1; a >= 0; --a) {
        T v = T(0);
        for (int q = 0; q <= a; ++q) v += Xg[a + (int64_t)q * sz] * col[q];
        col[a] = v;
      }
      continue;
    }
    const T* Lg = (const T*)Ph.Lbuf + Ph.pre_off[pi];
    for (int a = 0; a < sz; ++a) {
      T v = col[a];
      for (int q = 0; q < a; ++q) v -= Lg[a + (int64_t)q * sz] * col[q];
      col[a] = v / Lg[a + (int64_t)a * sz];
    }
  }
  __syncthreads();
  // columns: F[:, g] <- F[:, g] L_g^{-T}
  for (int64_t t = threadIdx.x; t < work; t += blockDim.x) {
    const int s = s0 + (int)(t / nb), i = (int)(t % nb);
    const int g = Lv.seg_group[s];
    const int pi = Ph.group_pre[g];
    if (pi < 0) continue;
    const int sz = Lv.group_size[g];
    const int pos = Lv.seg_pos[s];
    T* row = Fr + i + (int64_t)pos * ld;
    if (Ph.diag_only) {   // diagonal L_g: scale the columns
      const T* Dg = (const T*)(Ph.Linv ? Ph.Linv : Ph.Lbuf) + Ph.pre_off[pi];
      for (int a = 0; a < sz; ++a)
        row[(int64_t)a * ld] = Ph.Linv ? row[(int64_t)a * ld] * Dg[a + (int64_t)a * sz]
                                       : row[(int64_t)a * ld] / Dg[a + (int64_t)a * sz];
      continue;
    }
    if (Ph.Linv) {   // row <- row L_g^{-T} as a product, right to left in place
      const T* Xg = Xs ? Xs + (s - s0) * mg2 : (const T*)Ph.Linv + Ph.pre_off[pi];
      for (int a = sz - 1; a >= 0; --a) {
        T v = T(0);
        for (int q = 0; q <= a; ++q) v += Xg[a + (int64_t)q * sz] * row[(int64_t)q * ld];
        row[(int64_t)a * ld] = v;
      }
      continue;
    }
    const T* Lg = (const T*)Ph.Lbuf + Ph.pre_off[pi];
    for (int a = 0; a < sz; ++a) {
      T v = row[(int64_t)a * ld];
      for (int q = 0; q < a; ++q) v -= Lg[a + (int64_t)q * sz] * row[(int64_t)q * ld];
      row[(int64_t)a * ld] = v / Lg[a + (int64_t)a * sz];
    }
  }
  if (stage) {
    __syncthreads();
    for (int64_t idx = threadIdx.x; idx < (int64_t)nb * nb; idx += blockDim.x) {
      const int i = (int)(idx % nb), j = (int)(idx / nb);
      Fg[i + (int64_t)j * gld] = Fr[i + (int64_t)j * ld];
    }
  }
}

// Large frames: D^{-1} F D^{-T} spread over many CTAs.  The frame is first
// made symmetric; then one CTA per (cell, preconditioned segment g, block of
// 64 columns) applies L_g^{-1} to the rows of g, and one CTA per (cell,
// segment h, block of 64 rows) applies L_h^{-T} to the columns of h, both as
// tile products with the explicit inverses computed with the L_g.

template <typename T>
__global__ void k_frame_symmetrize(LevelDev Lv) {
  pdl_trigger();
  pdl_wait();   // what the previous kernel of the stream wrote
  for (int c = blockIdx.y; c < Lv.ncell; c += gridDim.y) {
    int ld;
    T* Fr = frame_of<T>(Lv, c, &ld);
    const int nb = Lv.nB[c];
    const int64_t total = (int64_t)nb * nb;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
      const int i = (int)(idx % nb), j = (int)(idx / nb);
      if (i < j) Fr[i + (int64_t)j * ld] = Fr[j + (int64_t)i * ld];
    }
  }
}

// Task `bid` of the tile-product scaling: the (cell, segment) pair whose
// 64-wide blocks hold it (binary search of the prefix sums) and the block.
__device__ inline void scale_task_of(const PhaseDev& Ph, int64_t bid, int* cell, int* seg,
                                     int* blk) {
  int lo = 0, hi = Ph.nscale_task - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (Ph.scale_off[mid] <= bid) lo = mid;
    else hi = mid - 1;
  }
  *cell = Ph.scale_task[2 * lo];
  *seg = Ph.scale_task[2 * lo + 1];
  *blk = (int)(bid - Ph.scale_off[lo]);
}

// F[g, J] <- L_g^{-1} F[g, J] for the 64 columns J of the task's block, as
// tile products with the explicit inverse; row tiles bottom-up so the update
// is in place (a row tile depends only on the rows above and at it).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_frame_rows_tp(LevelDev Lv, PhaseDev Ph) {
  pdl_trigger();
  pdl_wait();   // what the previous kernel of the stream wrote
  extern __shared__ unsigned char smraw[];
  T* sm = (T*)smraw;
  int c, q, blk;
  scale_task_of(Ph, blockIdx.x, &c, &q, &blk);
  int ld;
  T* Fr = frame_of<T>(Lv, c, &ld);
  const int nb = Lv.nB[c];
  const int g = Lv.seg_group[q], pos = Lv.seg_pos[q], sz = Lv.group_size[g];
  const T* Li = (const T*)Ph.Linv + Ph.pre_off[Ph.group_pre[g]];
  const int j0 = blk * kTile, ncol = min(kTile, nb - j0);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  auto fa = [&](int i, int k) { return Li[i + (int64_t)k * sz]; };
  auto fb = [&](int k, int j) { return Fr[(pos + k) + (int64_t)(j0 + j) * ld]; };
  for (int ti = ((sz - 1) / kTile) * kTile; ti >= 0; ti -= kTile) {
    T acc[4][4];
    cta_tile_product<T, false, true>(ti, 0, sz, ncol, min(sz, ti + kTile), fa, fb, sm, acc);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int i = ti + ty + 16 * a, j = tx + 16 * b;
        if (i < sz && j < ncol) Fr[(pos + i) + (int64_t)(j0 + j) * ld] = acc[a][b];
      }
  }
}

// F[I, h] <- F[I, h] L_h^{-T} for the 64 rows I of the task's block; column
// tiles right to left so the update is in place.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_frame_cols_tp(LevelDev Lv, PhaseDev Ph) {
  pdl_trigger();
  pdl_wait();   // what the previous kernel of the stream wrote
  extern __shared__ unsigned char smraw[];
  T* sm = (T*)smraw;
  int c, q, blk;
  scale_task_of(Ph, blockIdx.x, &c, &q, &blk);
  int ld;
  T* Fr = frame_of<T>(Lv, c, &ld);
  const int nb = Lv.nB[c];
  const int h = Lv.seg_group[q], pos = Lv.seg_pos[q], sz = Lv.group_size[h];
  const T* Li = (const T*)Ph.Linv + Ph.pre_off[Ph.group_pre[h]];
  const int i0 = blk * kTile, nrow = min(kTile, nb - i0);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  auto fa = [&](int i, int k) { return Fr[(i0 + i) + (int64_t)(pos + k) * ld]; };
  auto fb = [&](int k, int j) { return Li[j + (int64_t)k * sz]; };
  for (int tj = ((sz - 1) / kTile) * kTile; tj >= 0; tj -= kTile) {
    T acc[4][4];
    cta_tile_product<T>(0, tj, nrow, sz, min(sz, tj + kTile), fa, fb, sm, acc);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int i = ty + 16 * a, j = tj + tx + 16 * b;
        if (i < nrow && j < sz) Fr[(i0 + i) + (int64_t)(pos + j) * ld] = acc[a][b];
      }
  }
}

// ---------------------------------------------------------------------------
// skeletonization (Sec. 2.2) of one unit per CTA
// ---------------------------------------------------------------------------

template <typename T> __device__ inline T my_abs(T x) { return x < T(0) ? -x : x; }

// Row layout of A_{R,g} for unit group g: the other separator groups of the
// holding cells, each group once (first appearance in holding-cell order),
// with each group's position in every holding cell's frame.  Thread 0 builds
// the tables; the caller synchronizes.
struct SkelRows {
  int nrg;
  int group[kMaxRowGroupsDev];
  int row0[kMaxRowGroupsDev + 1];
  int pos[kMaxRowGroupsDev][kMaxSlotsDev];
};

__device__ inline void skel_row_groups(const LevelDev& Lv, int g, int nrow, int* status,
                                       SkelRows* R, bool leader) {
  if (!leader) return;
  const int c0 = Lv.group_cell_off[g], nslot = Lv.group_cell_off[g + 1] - c0;
  int nrg = 0, row = 0;
  for (int s = 0; s < nslot; ++s) {
    const int c = Lv.group_cell[c0 + s];
    for (int q = Lv.seg_off[c]; q < Lv.seg_off[c + 1]; ++q) {
      const int sg = Lv.seg_group[q];
      if (sg == g) continue;
      int f = -1;
      for (int i = 0; i < nrg; ++i)
        if (R->group[i] == sg) f = i;
      if (f < 0) {
        if (nrg >= kMaxRowGroupsDev) continue;
        f = nrg++;
        R->group[f] = sg;
        R->row0[f] = row;
        row += Lv.group_size[sg];
        for (int t = 0; t < kMaxSlotsDev; ++t) R->pos[f][t] = -1;
      }
      R->pos[f][s] = Lv.seg_pos[q];
    }
  }
  R->row0[nrg] = row;
  R->nrg = nrg;
  if (row != nrow) report(status, RHIF_ERR_BAD_ARG, Lv.level, kKindUnit, g);
}

// Rows [ra, rb) of A_{R,g} (n columns), summed over the holding cells in cell
// order; element (i, j) lands in D[(i - ra) * drs + j * dcs].  Dead DOFs give
// zero rows.
template <typename T>
__device__ void skel_gather_rows(const LevelDev& Lv, const uint8_t* alive, int g, int n, int nrow,
                                 const SkelRows& R, int ra, int rb, T* D, int64_t drs,
                                 int64_t dcs, int t0, int nt) {
  const int c0 = Lv.group_cell_off[g], nslot = Lv.group_cell_off[g + 1] - c0;
  for (int f = 0; f < R.nrg; ++f) {
    const int r0 = R.row0[f];
    const int lo = max(r0, ra), hi = min(min(R.row0[f + 1], rb), nrow);
    if (lo >= hi) continue;
    const int sg = R.group[f];
    const int32_t* sgid = Lv.bucket + Lv.group_start[sg];
    const int cnt = hi - lo;
    for (int idx = t0; idx < cnt * n; idx += nt) {
      const int o = lo - r0 + idx % cnt, j = idx / cnt;
      T v = T(0);
      if (alive[sgid[o]]) {
        for (int s = 0; s < nslot; ++s) {
          const int pos = R.pos[f][s];
          if (pos < 0) continue;
          int ld;
          const T* fr = frame_of<T>(Lv, Lv.group_cell[c0 + s], &ld);
          v += sym_at(fr, ld, pos + o, Lv.group_pos[c0 + s] + j);
        }
      }
      D[(int64_t)(lo - ra + idx % cnt) * drs + (int64_t)j * dcs] = v;
    }
  }
}

// A_gg summed over the holding cells; entries idx = first, first+step, ...
template <typename T>
__device__ void skel_gather_diag(const LevelDev& Lv, int g, int n, T* Aee, int64_t first,
                                 int64_t step) {
  const int c0 = Lv.group_cell_off[g], c1 = Lv.group_cell_off[g + 1];
  for (int64_t idx = first; idx < (int64_t)n * n; idx += step) {
    const int i = (int)(idx % n), j = (int)(idx / n);
    T v = T(0);
    for (int k = c0; k < c1; ++k) {
      int ld;
      const T* fr = frame_of<T>(Lv, Lv.group_cell[k], &ld);
      const int pos = Lv.group_pos[k];
      v += sym_at(fr, ld, pos + i, pos + j);
    }
    Aee[idx] = v;
  }
}

// Pivot rule of the CPQR, taken by warp 0 from the column norms nrm[j..n):
// stop once the largest remaining norm is <= tol * |R_11|; otherwise take the
// column with the smallest original index among those within a relative
// 1e-12 of the largest (ties broken by the original column order).
template <typename T>
__device__ void skel_pivot(const T* nrm, const int* sperm, int j, int n, double tol, T* s_r11,
                           int* s_stop, int* s_p) {
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  T mx = T(0);
  for (int c = j + lane; c < n; c += 32) mx = nrm[c] > mx ? nrm[c] : mx;
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const T y = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = y > mx ? y : mx;
  }
  const T r11 = j == 0 ? my_sqrt(mx) : *s_r11;
  // NaN norms (a breakdown earlier in the level, reported by its own kernel)
  // stop the decomposition instead of producing a pivot outside the columns
  int stop = (r11 == T(0)) || !(mx == mx) || !(r11 == r11) || (my_sqrt(mx) <= T(tol) * r11);
  int best = -1, bo = 0x7fffffff;
  if (!stop) {
    const T thr = T(1.0 - 1e-12) * mx;
    for (int c = j + lane; c < n; c += 32)
      if (nrm[c] >= thr && sperm[c] < bo) {
        bo = sperm[c];
        best = c;
      }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      const int ob = __shfl_xor_sync(0xffffffffu, bo, o);
      const int oc = __shfl_xor_sync(0xffffffffu, best, o);
      if (ob < bo) {
        bo = ob;
        best = oc;
      }
    }
    if (best < 0) stop = 1;
  }
  if (lane == 0) {
    if (j == 0) *s_r11 = r11;
    *s_stop = stop;
    *s_p = best;
  }
}

// Steps after the CPQR of unit u (rank k, R(i, j) = M[i * mrs + j * mcs] for
// i < k): T = R11^{-1} R12, the zeroing of Eq. (2.2) in (redundant, skeleton)
// order
//   [rd,rd] = A_rr - A_sr^T T - T^T [sk,rd],  [sk,rd] = A_sr - A_ss T,  [sk,sk] = A_ss,
// elimination of the redundant DOFs (Sec. 2.1 on the zeroed block), and the
// frame updates: the skeleton block of the first holding cell takes the new
// value, the others drop theirs.  One CTA of kThreads threads.
template <typename T>
__device__ void skel_finish(const LevelDev& Lv, const PhaseDev& Ph, int u, int g, int n, int k,
                            const T* M, int64_t mrs, int64_t mcs, const T* Aee, const int* sperm,
                            T* sm, int* status) {
  const int tid = threadIdx.x, r = n - k;
  const int tx = tid & 15, ty = tid >> 4;
  T* Fu = (T*)Ph.rec + Ph.u_rec_off[u];
  T* Tm = Fu + pad4e((int64_t)n * n);
  const int c0 = Lv.group_cell_off[g], c1 = Lv.group_cell_off[g + 1];
  auto R = [&](int i, int j) { return M[(int64_t)i * mrs + (int64_t)j * mcs]; };

  // interpolation matrix T = R11^{-1} R12 (k x r), by 64-row blocks from the
  // bottom: T[I,:] = R_II^{-1} (R12[I,:] - R[I, J] T[J,:]) with J the rows below I
  if (r > 0 && k > 0) {
    for (int ib = ((k - 1) / kTile) * kTile; ib >= 0; ib -= kTile) {
      const int ie = min(ib + kTile, k);
      auto fa = [&](int i, int q) { return R(i, ie + q); };
      auto fb = [&](int q, int a) { return Tm[(ie + q) + (int64_t)a * k]; };
      for (int tj = 0; tj < r; tj += kTile) {
        T acc[4][4];
        cta_tile_product(ib, tj, ie, r, k - ie, fa, fb, sm, acc);
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            const int i = ib + ty + 16 * a, c = tj + tx + 16 * b;
            if (i < ie && c < r) Tm[i + (int64_t)c * k] = R(i, k + c) - acc[a][b];
          }
      }
      T* Rb = sm;   // R_II, [kTile][kTile + 1]
      const int nb = ie - ib;
      for (int idx = tid; idx < nb * nb; idx += blockDim.x) {
        const int i = idx / nb, q = idx % nb;
        Rb[i * (kTile + 1) + q] = q >= i ? R(ib + i, ib + q) : T(0);
      }
      __syncthreads();
      for (int a = tid; a < r; a += blockDim.x) {
        T* col = Tm + (int64_t)a * k + ib;
        for (int i = nb - 1; i >= 0; --i) {
          T t = col[i];
          for (int q = i + 1; q < nb; ++q) t -= Rb[i * (kTile + 1) + q] * col[q];
          col[i] = t / Rb[i * (kTile + 1) + i];
        }
      }
      __syncthreads();
    }
  }

  // [sk,rd] = A_sr - A_ss T
  auto a_ss = [&](int q, int p) { return Aee[sperm[q] + (int64_t)sperm[p] * n]; };
  auto t_el = [&](int p, int a) { return Tm[p + (int64_t)a * k]; };
  for (int ti = 0; ti < k; ti += kTile)
    for (int tj = 0; tj < r; tj += kTile) {
      T acc[4][4];
      cta_tile_product(ti, tj, k, r, k, a_ss, t_el, sm, acc);
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int q = ti + ty + 16 * a, c = tj + tx + 16 * b;
          if (q < k && c < r) Fu[(r + q) + (int64_t)c * n] = a_ss(q, k + c) - acc[a][b];
        }
    }
  __syncthreads();
  // [rd,rd] = A_rr - [A_sr^T, T^T] [T; [sk,rd]]  (lower triangle)
  auto fa = [&](int a, int q) {
    return q < k ? Aee[sperm[q] + (int64_t)sperm[k + a] * n] : Tm[(q - k) + (int64_t)a * k];
  };
  auto fb = [&](int q, int b) {
    return q < k ? Tm[q + (int64_t)b * k] : Fu[(r + q - k) + (int64_t)b * n];
  };
  for (int ti = 0; ti < r; ti += kTile)
    for (int tj = 0; tj <= ti; tj += kTile) {
      T acc[4][4];
      cta_tile_product(ti, tj, r, r, 2 * k, fa, fb, sm, acc);
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int i = ti + ty + 16 * a, j = tj + tx + 16 * b;
          if (i < r && j <= i) Fu[i + (int64_t)j * n] = a_ss(k + i, k + j) - acc[a][b];
        }
    }
  for (int64_t idx = tid; idx < (int64_t)k * k; idx += blockDim.x) {
    const int q = (int)(idx % k), p = (int)(idx / k);
    if (q < p) continue;
    Fu[(r + q) + (int64_t)(r + p) * n] = a_ss(q, p);
  }
  __syncthreads();

  // eliminate the redundant DOFs
  if (!cta_partial_chol(Fu, n, n, r, sm) && tid == 0)
    report(status, RHIF_ERR_NOT_SPD, Lv.level, kKindUnit, g);
  __syncthreads();

  for (int64_t idx = tid; idx < (int64_t)k * k; idx += blockDim.x) {
    const int q = (int)(idx % k), p = (int)(idx / k);
    if (q < p) continue;
    const T val = Fu[(r + q) + (int64_t)(r + p) * n];
    for (int kk = c0; kk < c1; ++kk) {
      int ld;
      T* fr = frame_of<T>(Lv, Lv.group_cell[kk], &ld);
      const int pos = Lv.group_pos[kk];
      const int bq = pos + sperm[q], bp = pos + sperm[p];
      fr[max(bq, bp) + (int64_t)min(bq, bp) * ld] = kk == c0 ? val : T(0);
    }
  }
  int* perm_out = Ph.perm + Ph.u_perm_off[u];
  for (int i = tid; i < n; i += blockDim.x) perm_out[i] = sperm[i];
  if (tid == 0) Ph.rank[u] = k;
}

// Skeletonization (Sec. 2.2) of one unit per CTA: gather A_{R,g}, CPQR with
// exact norms recomputed at every step, then skel_finish.  M lives in shared
// memory when mstage is set.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_skel(LevelDev Lv, PhaseDev Ph, uint8_t* alive,
                                                   double tol, int* status, int mstage) {
  pdl_trigger();
  pdl_wait();   // what the previous kernel of the stream wrote
  extern __shared__ unsigned char smraw[];
  T* sm = (T*)smraw;                                   // partial-Cholesky / tile workspace
  T* nrm = sm + partial_chol_smem_elems();             // [max_n]
  int* sperm = (int*)(nrm + Ph.max_n);                 // [max_n]
  __shared__ int s_k, s_stop, s_p;
  __shared__ T s_r11;
  __shared__ SkelRows rows;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int u = blockIdx.x;
  const int g = Ph.u_group[u];
  const int n = Lv.group_size[g];
  const int nrow = Ph.u_nrow[u];
  const int ldm = nrow > 0 ? nrow : 1;
  T* M = (T*)Ph.Mbuf + Ph.u_m_off[u];
  if (mstage) M = (T*)((unsigned char*)(sperm + Ph.max_n) + 16 - (((size_t)(sperm + Ph.max_n)) & 15));
  T* Aee = M + (int64_t)nrow * n;

  skel_row_groups(Lv, g, nrow, status, &rows, tid == 0);
  __syncthreads();
  skel_gather_rows(Lv, alive, g, n, nrow, rows, 0, nrow, M, 1, ldm, tid, blockDim.x);
  skel_gather_diag(Lv, g, n, Aee, tid, blockDim.x);
  for (int i = tid; i < n; i += blockDim.x) sperm[i] = i;
  if (tid == 0) {
    s_k = 0;
    s_r11 = T(0);
  }
  __syncthreads();

  const int steps = min(nrow, n);
  for (int j = 0; j < steps; ++j) {
    for (int c = j + warp; c < n; c += nwarps) {
      T s = T(0);
      for (int i = j + lane; i < nrow; i += 32) {
        const T v = M[i + (int64_t)c * ldm];
        s += v * v;
      }
      s = warp_sum(s);
      if (lane == 0) nrm[c] = s;
    }
    __syncthreads();
    skel_pivot(nrm, sperm, j, n, tol, &s_r11, &s_stop, &s_p);
    __syncthreads();
    if (s_stop) break;
    const int p = s_p;
    if (p != j) {
      for (int i = tid; i < nrow; i += blockDim.x) {
        const T a = M[i + (int64_t)j * ldm];
        M[i + (int64_t)j * ldm] = M[i + (int64_t)p * ldm];
        M[i + (int64_t)p * ldm] = a;
      }
      if (tid == 0) {
        const int t = sperm[j]; sperm[j] = sperm[p]; sperm[p] = t;
        const T q = nrm[j]; nrm[j] = nrm[p]; nrm[p] = q;
      }
    }
    __syncthreads();
    const T x0 = M[j + (int64_t)j * ldm];
    const T nx = my_sqrt(nrm[j]);
    const T alpha = x0 < T(0) ? nx : -nx;
    const T v0 = x0 - alpha;
    const T tau = T(1) / (nx * (nx + my_abs(x0)));
    for (int c = j + 1 + warp; c < n; c += nwarps) {
      T s = T(0);
      for (int i = j + 1 + lane; i < nrow; i += 32) s += M[i + (int64_t)j * ldm] * M[i + (int64_t)c * ldm];
      s = warp_sum(s);
      const T w = (s + v0 * M[j + (int64_t)c * ldm]) * tau;
      __syncwarp();
      for (int i = j + lane; i < nrow; i += 32) {
        const T vi = (i == j) ? v0 : M[i + (int64_t)j * ldm];
        M[i + (int64_t)c * ldm] -= w * vi;
      }
    }
    __syncthreads();
    if (tid == 0) {
      M[j + (int64_t)j * ldm] = alpha;
      s_k = j + 1;
    }
    __syncthreads();
  }
  skel_finish(Lv, Ph, u, g, n, s_k, M, 1, ldm, Aee, sperm, sm, status);
}

// Skeletonization of small units (n <= 32) with one warp per unit: lane c
// owns column c of A_{R,g} (shared memory, odd leading dimension), so the
// CPQR needs no block barriers; the column norms for the next step are taken
// from the updated values in the same pass (an exact recomputation, not a
// downdate).  The zeroing and the elimination of the redundant DOFs run in the
// warp too, on an n x n copy in shared memory.  Same rank rule and pivot rule
// as k_skel.
__host__ __device__ inline size_t skel_warp_bytes(int max_n, int64_t max_m, size_t elem) {
  const size_t rows = (sizeof(SkelRows) + 15) & ~size_t(15);
  const size_t mcap = (size_t)max_m + max_n;   // (nrow + 1) * n covers the odd leading dimension
  const size_t mreg = (((size_t)max_n * max_n > mcap ? (size_t)max_n * max_n : mcap) * elem + 15) & ~size_t(15);
  const size_t sq = (((size_t)max_n * max_n) * elem + 15) & ~size_t(15);
  return rows + 128 + mreg + 2 * sq;
}

template <typename T>
__global__ void __launch_bounds__(256) k_skel_warp(LevelDev Lv, PhaseDev Ph, uint8_t* alive,
                                                   double tol, int* status, int per_warp) {
  pdl_trigger();
  pdl_wait();   // what the previous kernel of the stream wrote
  extern __shared__ __align__(16) unsigned char smraw[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int u = blockIdx.x * (blockDim.x >> 5) + wid;
  if (u >= Ph.nunit) return;   // whole warps only; no block barriers below
  unsigned char* base = smraw + (size_t)wid * per_warp;
  SkelRows* rows = (SkelRows*)base;
  int* sp = (int*)(base + ((sizeof(SkelRows) + 15) & ~size_t(15)));
  T* M = (T*)((unsigned char*)sp + 128);
  const int g = Ph.u_group[u];
  const int n = Lv.group_size[g];
  const int nrow = Ph.u_nrow[u];
  const int ld = nrow | 1;
  const int64_t mreg = (((int64_t)ld * n > (int64_t)n * n ? (int64_t)ld * n : (int64_t)n * n) + 3) & ~int64_t(3);
  T* Aee = M + mreg;
  T* Ts = Aee + pad4e((int64_t)n * n);
  T* Fs = M;   // reused for the zeroed block once R and T are done

  skel_row_groups(Lv, g, nrow, status, rows, lane == 0);
  __syncwarp();
  skel_gather_rows(Lv, alive, g, n, nrow, *rows, 0, nrow, M, 1, ld, lane, 32);
  skel_gather_diag(Lv, g, n, Aee, lane, 32);
  if (lane < n) sp[lane] = lane;
  __syncwarp();

  const bool own = lane < n;
  T* col = M + (int64_t)lane * ld;
  T nrm = T(0);
  if (own) {
    T a0 = T(0), a1 = T(0);
    int i = 0;
    for (; i + 1 < nrow; i += 2) { a0 += col[i] * col[i]; a1 += col[i + 1] * col[i + 1]; }
    if (i < nrow) a0 += col[i] * col[i];
    nrm = a0 + a1;
  }
  T r11 = T(0);
  int k = 0;
  const int steps = min(nrow, n);
  for (int j = 0; j < steps; ++j) {
    // pivot: largest norm, ties within 1e-12 relative to the smallest original index
    const bool cand = own && lane >= j;
    T mx = cand ? nrm : T(0);
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      const T y = __shfl_xor_sync(0xffffffffu, mx, o);
      mx = y > mx ? y : mx;
    }
    if (j == 0) r11 = my_sqrt(mx);
    if (r11 == T(0) || !(mx == mx) || !(r11 == r11) || my_sqrt(mx) <= T(tol) * r11) break;
    const T thr = T(1.0 - 1e-12) * mx;
    int key = (cand && nrm >= thr) ? sp[lane] : 0x7fffffff, p = lane;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      const int ok = __shfl_xor_sync(0xffffffffu, key, o);
      const int op = __shfl_xor_sync(0xffffffffu, p, o);
      if (ok < key || (ok == key && op < p)) { key = ok; p = op; }
    }
    if (key == 0x7fffffff || p < j || p >= n) break;   // no candidate (NaN norms)
    if (p != j) {
      for (int i = lane; i < nrow; i += 32) {
        const T a = M[i + (int64_t)j * ld];
        M[i + (int64_t)j * ld] = M[i + (int64_t)p * ld];
        M[i + (int64_t)p * ld] = a;
      }
      const T nj = __shfl_sync(0xffffffffu, nrm, p), np = __shfl_sync(0xffffffffu, nrm, j);
      if (lane == j) nrm = nj;
      if (lane == p) nrm = np;
      if (lane == 0) { const int t = sp[j]; sp[j] = sp[p]; sp[p] = t; }
    }
    __syncwarp();
    const T x0 = M[j + (int64_t)j * ld];
    const T nx = my_sqrt(__shfl_sync(0xffffffffu, nrm, j));
    const T alpha = x0 < T(0) ? nx : -nx;
    const T v0 = x0 - alpha;
    const T tau = T(1) / (nx * (nx + my_abs(x0)));
    const T* vj = M + (int64_t)j * ld;
    if (own && lane > j) {
      T s0 = T(0), s1 = T(0);
      int i = j + 1;
      for (; i + 1 < nrow; i += 2) { s0 += vj[i] * col[i]; s1 += vj[i + 1] * col[i + 1]; }
      if (i < nrow) s0 += vj[i] * col[i];
      const T w = ((s0 + s1) + v0 * col[j]) * tau;
      col[j] -= w * v0;
      T n0 = T(0), n1 = T(0);
      i = j + 1;
      for (; i + 1 < nrow; i += 2) {
        const T b0 = col[i] - w * vj[i], b1 = col[i + 1] - w * vj[i + 1];
        col[i] = b0;
        col[i + 1] = b1;
        n0 += b0 * b0;
        n1 += b1 * b1;
      }
      if (i < nrow) {
        const T b0 = col[i] - w * vj[i];
        col[i] = b0;
        n0 += b0 * b0;
      }
      nrm = n0 + n1;
    }
    __syncwarp();
    if (lane == 0) M[j + (int64_t)j * ld] = alpha;
    __syncwarp();
    k = j + 1;
  }
  const int r = n - k;
  // T = R11^{-1} R12 (k x r), one column per lane
  if (lane < r) {
    for (int i = k - 1; i >= 0; --i) {
      T t = M[i + (int64_t)(k + lane) * ld];
      for (int q = i + 1; q < k; ++q) t -= M[i + (int64_t)q * ld] * Ts[q + lane * k];
      Ts[i + lane * k] = t / M[i + (int64_t)i * ld];
    }
  }
  __syncwarp();
  // zeroing (Eq. 2.2) into Fs in (redundant, skeleton) order
  auto a_ss = [&](int q, int p2) { return Aee[sp[q] + sp[p2] * n]; };
  if (lane < r) {
    for (int q = 0; q < k; ++q) {
      T v = a_ss(q, k + lane);
      for (int p2 = 0; p2 < k; ++p2) v -= a_ss(q, p2) * Ts[p2 + lane * k];
      Fs[(r + q) + lane * n] = v;
    }
  }
  __syncwarp();
  if (lane < r) {
    const int b = lane;
    for (int a = b; a < r; ++a) {
      T v = a_ss(k + a, k + b);
      for (int q = 0; q < k; ++q)
        v -= Ts[q + a * k] * Fs[(r + q) + b * n] + a_ss(q, k + a) * Ts[q + b * k];
      Fs[a + b * n] = v;
    }
  }
  if (lane < k)
    for (int q = lane; q < k; ++q) Fs[(r + q) + (r + lane) * n] = a_ss(q, lane);
  __syncwarp();
  // eliminate the redundant DOFs: right-looking Cholesky of the first r columns
  bool bad = false;
  for (int pc = 0; pc < r; ++pc) {
    T d = Fs[pc + pc * n];
    if (!(d > T(0))) { bad = true; d = T(1); }
    const T sd = my_sqrt(d);
    __syncwarp();
    if (lane == pc) Fs[pc + pc * n] = sd;
    if (lane > pc && lane < n) Fs[lane + pc * n] /= sd;
    __syncwarp();
    if (lane > pc && lane < n) {
      const T lip = Fs[lane + pc * n];
      for (int jj = pc + 1; jj <= lane; ++jj) Fs[lane + jj * n] -= lip * Fs[jj + pc * n];
    }
    __syncwarp();
  }
  if (bad && lane == 0) report(status, RHIF_ERR_NOT_SPD, Lv.level, kKindUnit, g);
  // outputs: unit front, T, frames, permutation, rank
  T* Fu = (T*)Ph.rec + Ph.u_rec_off[u];
  T* Tm = Fu + pad4e((int64_t)n * n);
  for (int idx = lane; idx < n * n; idx += 32) {
    const int i = idx % n, jj = idx / n;
    if (i >= jj) Fu[idx] = Fs[idx];
  }
  for (int idx = lane; idx < k * r; idx += 32) Tm[idx] = Ts[idx];
  const int c0 = Lv.group_cell_off[g], c1 = Lv.group_cell_off[g + 1];
  for (int idx = lane; idx < k * k; idx += 32) {
    const int q = idx % k, p2 = idx / k;
    if (q < p2) continue;
    const T val = Fs[(r + q) + (r + p2) * n];
    for (int kk = c0; kk < c1; ++kk) {
      int ldf;
      T* fr = frame_of<T>(Lv, Lv.group_cell[kk], &ldf);
      const int pos = Lv.group_pos[kk];
      const int bq = pos + sp[q], bp = pos + sp[p2];
      fr[max(bq, bp) + (int64_t)min(bq, bp) * ldf] = kk == c0 ? val : T(0);
    }
  }
  int* perm_out = Ph.perm + Ph.u_perm_off[u];
  if (lane < n) perm_out[lane] = sp[lane];
  if (lane == 0) Ph.rank[u] = k;
}

// Row length (elements) of the per-rank partial-sum tables of k_skel_cluster:
// a multiple of 4, so every row is a whole number of 16-byte vectors.
__host__ __device__ inline int skel_cluster_ldp(int max_n) { return (max_n + 3) & ~3; }

// Skeletonization of one unit per thread-block cluster of C CTAs, for units
// whose A_{R,g} does not fit in one CTA's shared memory.  CTA q owns rows
// [q*sr, (q+1)*sr) of A_{R,g} (sr = ceil(nrow / C)), stored row-major and
// staged in its shared memory when they fit; each thread owns whole columns,
// so column sums need no shuffles and row loads are coalesced.  At each CPQR
// step every CTA pushes its partial column norms and Householder dot products
// into the shared memory of every CTA of the cluster (remote stores, no
// remote loads); after a cluster barrier each CTA sums the C partials in rank
// order from its own copy, so all CTAs take bitwise the same pivot and
// stopping decisions.  Two cluster barriers per step: after the partial norms
// (pivot) and after the partial dots (update).  The cluster barriers are
// hardware barriers that every CTA reaches the same number of times.  Rank 0
// then runs skel_finish on R written back to global memory.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_skel_cluster(LevelDev Lv, PhaseDev Ph, uint8_t* alive,
                                                           double tol, int* status,
                                                           int64_t slice_cap) {
  pdl_trigger();
  pdl_wait();   // what the previous kernel of the stream wrote
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks(), cr = (int)cl.block_rank();
  const int ldp = skel_cluster_ldp(Ph.max_n);
  extern __shared__ unsigned char smraw[];
  T* sm = (T*)smraw;
  T* nrm = sm + partial_chol_smem_elems();   // [ldp] column norms over the cluster
  T* pnall = nrm + ldp;                      // [C][ldp] partial norms of each rank
  T* pdall = pnall + (int64_t)C * ldp;       // [C][ldp] partial Householder dots
  int* sperm = (int*)(pdall + (int64_t)C * ldp);   // [ldp]
  T* slice = (T*)((unsigned char*)(sperm + ldp) + 16 - (((size_t)(sperm + ldp)) & 15));
  __shared__ int s_k, s_stop, s_p;
  __shared__ T s_r11, s_x0;
  __shared__ SkelRows rows;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int u = blockIdx.x / C;
  const int g = Ph.u_group[u];
  const int n = Lv.group_size[g];
  const int nrow = Ph.u_nrow[u];
  T* Mg = (T*)Ph.Mbuf + Ph.u_m_off[u];       // row-major nrow x n while this kernel runs
  T* Aee = Mg + (int64_t)nrow * n;
  const int sr = (nrow + C - 1) / C;
  const int i0 = min(nrow, cr * sr), i1 = min(nrow, i0 + sr);
  const bool stage = (int64_t)sr * n <= slice_cap;
  T* Ms = stage ? slice : Mg + (int64_t)i0 * n;   // row i of this CTA at Ms[(i - i0) * n]
  auto at = [&](int i, int c) -> T& { return Ms[(int64_t)(i - i0) * n + c]; };
  // copy this rank's row of buf (columns >= c0) into the same row of every
  // other rank, 16 bytes per store; rows are ldp elements (16-byte multiples)
  auto bcast = [&](T* buf, int c0) {
    const int v0 = (c0 * (int)sizeof(T)) / 16, v1 = (n * (int)sizeof(T) + 15) / 16;
    const int nv = v1 - v0;
    const uint4* src = (const uint4*)(buf + (int64_t)cr * ldp);
    for (int idx = tid; idx < (C - 1) * nv; idx += nth) {
      const int q = idx / nv, v = v0 + idx % nv;
      uint4* dst = (uint4*)cl.map_shared_rank(buf + (int64_t)cr * ldp, q < cr ? q : q + 1);
      dst[v] = src[v];
    }
  };

  skel_row_groups(Lv, g, nrow, status, &rows, tid == 0);
  __syncthreads();
  skel_gather_rows(Lv, alive, g, n, nrow, rows, i0, i1, Ms, n, 1, tid, nth);
  skel_gather_diag(Lv, g, n, Aee, (int64_t)cr * nth + tid, (int64_t)C * nth);
  for (int i = tid; i < n; i += nth) sperm[i] = i;
  if (tid == 0) {
    s_k = 0;
    s_r11 = T(0);
  }
  __syncthreads();
  T* myn = pnall + (int64_t)cr * ldp;
  T* myd = pdall + (int64_t)cr * ldp;
  for (int c = tid; c < n; c += nth) {
    T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
    int i = i0;
    for (; i + 3 < i1; i += 4) {
      const T a0 = at(i, c), a1 = at(i + 1, c), a2 = at(i + 2, c), a3 = at(i + 3, c);
      s0 += a0 * a0; s1 += a1 * a1; s2 += a2 * a2; s3 += a3 * a3;
    }
    for (; i < i1; ++i) {
      const T a0 = at(i, c);
      s0 += a0 * a0;
    }
    myn[c] = (s0 + s1) + (s2 + s3);
  }
  __syncthreads();
  bcast(pnall, 0);
  cl.sync();

  const int steps = min(nrow, n);
  for (int j = 0; j < steps; ++j) {
    for (int c = j + tid; c < n; c += nth) {
      T s = T(0);
      for (int q = 0; q < C; ++q) s += pnall[(int64_t)q * ldp + c];
      nrm[c] = s;
    }
    __syncthreads();
    skel_pivot(nrm, sperm, j, n, tol, &s_r11, &s_stop, &s_p);
    __syncthreads();
    if (s_stop) break;
    const int p = s_p;
    if (p != j) {
      for (int i = i0 + tid; i < i1; i += nth) {
        const T a = at(i, j);
        at(i, j) = at(i, p);
        at(i, p) = a;
      }
      if (tid == 0) {
        const int t = sperm[j]; sperm[j] = sperm[p]; sperm[p] = t;
        const T q = nrm[j]; nrm[j] = nrm[p]; nrm[p] = q;
      }
    }
    __syncthreads();
    const int owner = j / sr;
    const bool own_j = cr == owner;   // i0 <= j < i1
    const T nx = my_sqrt(nrm[j]);
    T v0 = T(0);
    if (own_j) {
      const T x0 = at(j, j);
      v0 = x0 - (x0 < T(0) ? nx : -nx);
      if (tid < C) *cl.map_shared_rank(&s_x0, tid) = x0;
    }
    const int ia = max(i0, j + 1);
    for (int c = j + 1 + tid; c < n; c += nth) {
      T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
      int i = ia;
      for (; i + 3 < i1; i += 4) {
        s0 += at(i, j) * at(i, c);
        s1 += at(i + 1, j) * at(i + 1, c);
        s2 += at(i + 2, j) * at(i + 2, c);
        s3 += at(i + 3, j) * at(i + 3, c);
      }
      for (; i < i1; ++i) s0 += at(i, j) * at(i, c);
      const T s = (s0 + s1) + (s2 + s3);
      myd[c] = own_j ? s + v0 * at(j, c) : s;
    }
    __syncthreads();
    bcast(pdall, j + 1);
    cl.sync();
    const T x0 = s_x0;
    const T alpha = x0 < T(0) ? nx : -nx;
    v0 = x0 - alpha;
    const T tau = T(1) / (nx * (nx + my_abs(x0)));
    for (int c = j + 1 + tid; c < n; c += nth) {
      T s = T(0);
      for (int q = 0; q < C; ++q) s += pdall[(int64_t)q * ldp + c];
      const T w = s * tau;
      if (own_j) at(j, c) -= w * v0;   // row j: v_j = v0, excluded from the next norms
      T n0 = T(0), n1 = T(0), n2 = T(0), n3 = T(0);
      int i = ia;
      for (; i + 3 < i1; i += 4) {
        const T b0 = at(i, c) - w * at(i, j);
        const T b1 = at(i + 1, c) - w * at(i + 1, j);
        const T b2 = at(i + 2, c) - w * at(i + 2, j);
        const T b3 = at(i + 3, c) - w * at(i + 3, j);
        at(i, c) = b0; at(i + 1, c) = b1; at(i + 2, c) = b2; at(i + 3, c) = b3;
        n0 += b0 * b0; n1 += b1 * b1; n2 += b2 * b2; n3 += b3 * b3;
      }
      for (; i < i1; ++i) {
        const T b0 = at(i, c) - w * at(i, j);
        at(i, c) = b0;
        n0 += b0 * b0;
      }
      myn[c] = (n0 + n1) + (n2 + n3);
    }
    __syncthreads();
    bcast(pnall, j + 1);
    if (tid == 0) {
      if (own_j) at(j, j) = alpha;
      s_k = j + 1;
    }
    cl.sync();
  }
  const int k = s_k;
  if (stage) {   // R rows back to global memory (row-major) for the finishing CTA
    const int rb = min(i1, k);
    for (int64_t idx = tid; idx < (int64_t)max(rb - i0, 0) * n; idx += nth)
      Mg[(int64_t)i0 * n + idx] = Ms[idx];
  }
  cl.sync();
  if (cr != 0) return;
  skel_finish(Lv, Ph, u, g, n, k, (const T*)Mg, (int64_t)n, (int64_t)1, (const T*)Aee, sperm, sm,
              status);
}

// ---------------------------------------------------------------------------
// FP64 leaf fallback of the FP32 factor: condition estimate of every leaf
// ---------------------------------------------------------------------------

// kappa_1(B) = ||B||_1 ||B^{-1}||_1 of the Jacobi-scaled leaf block
// B = D A_II D, D = diag(A_II)^{-1/2}, from the leaf's banded FP32 factor
// (A_II = L L^T; band column k: 1/L_kk, L[k+1..k+w, k]).  The leaves this
// runs on are 2D (at most 64 boundary DOFs): A_II is the five-point stencil
// of the interior box in lexicographic order (x-neighbours at +-1 within a
// row of w, y-neighbours at +-w), so D and ||B||_1 come from the stencil form
// itself; ||B^{-1}||_1 comes from one application of
// B^{-1} = S L^{-T} L^{-1} S (S = D^{-1}) to the vector of ones, exact for
// these M-matrices (see below).  One warp per leaf; a leaf whose estimate
// exceeds `thresh` or is not finite is appended to list (*count entries).
template <typename T>
__global__ void __launch_bounds__(128) k_leaf_cond(GeoDev G, LevelDev Lv, const double* diag,
                                                   const double* off, double thresh, int* list,
                                                   int* count, int per_warp) {
  pdl_trigger();
  pdl_wait();   // what the previous kernel of the stream wrote
  extern __shared__ __align__(16) unsigned char smraw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = blockIdx.x * (blockDim.x >> 5) + warp;
  if (c >= Lv.ncell) return;
  const int n = Lv.nI[c], w = Lv.band_w[c];
  const int32_t* gid = Lv.gids + Lv.gid_off[c];
  const int64_t dbase = bind_cell_geo(Lv, c, G, diag, off);
  // the band is read where the leaf elimination left it (staging it in shared
  // memory limited the resident leaves to about half of them)
  const T* band = (const T*)Lv.band + Lv.band_off[c];
  T* sd = (T*)(smraw + (size_t)warp * per_warp);   // S = sqrt(diag A_II)
  T* y = sd + Lv.max_nI;
  // entries of A_II from the stencil form (interior in lexicographic order:
  // x-neighbours at +-1 inside a row of w, y-neighbours at +-w)
  // (in T: FP64 arithmetic is scarce on this GPU and the estimate needs no more)
  for (int i = lane; i < n; i += 32) sd[i] = my_sqrt(T(diag[gid[i] - dbase]));
  __syncwarp();
  // ||B||_1: row sums of |d_i a_ij d_j|
  T norm1 = T(0);
  for (int i = lane; i < n; i += 32) {
    const int64_t g = gid[i] - dbase;
    const int ix = i % w;
    const T ri = T(1) / sd[i];
    T rs = T(1);
    if (ix + 1 < w && i + 1 < n) rs += fabs(T(off[g])) * ri / sd[i + 1];
    if (ix > 0) rs += fabs(T(off[g - 1])) * ri / sd[i - 1];
    if (i + w < n) rs += fabs(T(off[G.N + g])) * ri / sd[i + w];
    if (i >= w) rs += fabs(T(off[G.N + g - G.stride[1]])) * ri / sd[i - w];
    norm1 = fmax(norm1, rs);
  }
  for (int o = 16; o > 0; o >>= 1) norm1 = fmax(norm1, __shfl_xor_sync(0xffffffffu, norm1, o));
  auto binv = [&](T* v) {   // v <- S L^{-T} L^{-1} S v
    for (int i = lane; i < n; i += 32) v[i] *= sd[i];
    __syncwarp();
    if (w >= 1 && w <= 31) {
      warp_band_fwd_blk(band, n, w, v);
      warp_band_bwd_blk(band, n, w, v);
    } else {
      warp_band_fwd(band, n, w, v);
      warp_band_bwd(band, n, w, v);
    }
    for (int i = lane; i < n; i += 32) v[i] *= sd[i];
    __syncwarp();
  };
  // ||B^{-1}||_1 = max_i (B^{-1} 1)_i: B is an M-matrix (unit diagonal,
  // nonpositive off-diagonal entries: the five-point stencil has positive
  // edge weights), so B^{-1} >= 0 entrywise and its largest column sum is the
  // largest entry of B^{-1} applied to the vector of ones (B = B^T).  A
  // negative entry (not an M-matrix) leaves max |.|, a lower bound.
  for (int i = lane; i < n; i += 32) y[i] = T(1);
  __syncwarp();
  binv(y);
  T est = T(0);
  for (int i = lane; i < n; i += 32) est = fmax(est, fabs(y[i]));
  for (int o = 16; o > 0; o >>= 1) est = fmax(est, __shfl_xor_sync(0xffffffffu, est, o));
  const double kappa = double(norm1) * double(est);
  if (lane == 0 && !(kappa <= thresh))   // above the threshold, or not finite
    list[atomicAdd(count, 1)] = c;          // compact list of the flagged leaves
}

void launch_leaf_cond(const GeoDev& G, const LevelDev& Lv, const double* diag, const double* off,
                      double thresh, int* list, int* count, cudaStream_t s) {
  if (!Lv.ncell) return;
  const int per = (int)(((size_t)2 * Lv.max_nI * sizeof(float) + 15) & ~size_t(15));
  launch_pdl(k_leaf_cond<float>, (Lv.ncell + 3) / 4, 128, 4 * per, s, G, Lv, diag, off, thresh, list,
                                                             count, per);
}

// FP64 re-elimination of the flagged leaves of an FP32 factor, spread over
// CTAs.  GB300 runs FP64 at a small fraction of its FP32 rate, so one CTA per
// leaf spends most of its time in the FP64 accumulation of S = Z^T Z
// (Z = L^{-1} A_IB, nB x nB).  Here CTA (leaf, t) takes the lower tile
// t = (I, J), I >= J, of the 64 x 64 boundary block in 16 x 16 tiles: every
// CTA of a leaf assembles and factors the band in FP64 (the column-by-column
// pass of k_leaf_stream, the same operations in the same order), carries the
// rows of Z only for the tile's 16 or 32 columns, and accumulates only its
// tile of S.  It writes its tile of the frame's lower triangle, the FP32
// A_BB share minus S, the difference taken in FP64 and rounded to FP32; tile
// 0 writes the band.  The couplings and the frame's upper triangle are the
// FP32 leaf kernel's, from the same stencil values.  The flagged leaves come
// as a list of count[0] cells; the grid's x loops over it.
constexpr int kRedoTile = 16;
constexpr int kRedoTiles = 10;   // lower tiles of the 64 x 64 block

__global__ void __launch_bounds__(kThreads)
k_leaf_redo64(GeoDev G, LevelDev Lv, const double* diag, const double* off, int* status,
              const int* list, const int* count) {
  pdl_trigger();
  pdl_wait();   // what the previous kernel of the stream wrote
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ int bad;
  __shared__ double s_piv, s_rpiv;
  __shared__ int sci[kStreamNB];
  __shared__ double sca[kStreamNB];
  __shared__ float abb[kRedoTile][kRedoTile + 1];
  const int tid = threadIdx.x;
  const int t = blockIdx.y;
  int I = 0;
  while ((I + 1) * (I + 2) / 2 <= t) ++I;
  const int J = t - I * (I + 1) / 2;
  const int ncol = I == J ? kRedoTile : 2 * kRedoTile;
  const int zc = tid & 31, zr0 = tid >> 5;                 // Z column, first row phase
  const int zb = zc < kRedoTile ? J * kRedoTile + zc : I * kRedoTile + (zc - kRedoTile);
  const int si = tid >> 4, sj = tid & 15;                  // this thread's entry of the S tile
  const int zi = I == J ? si : kRedoTile + si;             // their Z columns
  const int zj = sj;
  const int m = G.leaf, m1 = m + 1;
  int tab = 1;
  for (int a = 0; a < G.d; ++a) tab *= m1;
  const int nlist = *count;
  for (int li = blockIdx.x; li < nlist; li += gridDim.x) {
    const int c = list[li];
    const int nI = Lv.nI[c], nB = Lv.nB[c], n = nI + nB, w = Lv.band_w[c];
    const int w1 = w + 1;
    const int32_t* gid = Lv.gids + Lv.gid_off[c];
    const int64_t dbase = bind_cell_geo(Lv, c, G, diag, off);
    unsigned char* p = smraw;
    double* sband = (double*)p;
    p += round16((size_t)Lv.max_nI * (Lv.max_w + 1) * sizeof(double));
    double* win = (double*)p;                              // win[(k % w1) * 32 + zc]
    p += round16((size_t)(Lv.max_w + 1) * 32 * sizeof(double));
    int* postab = (int*)p;
    p += round16((size_t)tab * sizeof(int));
    short* pairs = (short*)p;                              // (d1, d2), 1 <= d2 <= d1 <= w
    const int npair = w * (w + 1) / 2;
    int origin[3] = {0, 0, 0};
    {
      int64_t code = Lv.cell_code[c];
      for (int a = 0; a < G.d; ++a) {
        const int v = (int)(code % Lv.code_base);
        code /= Lv.code_base;
        origin[a] = ((v - 1) / 2) * m;
      }
    }
    if (tid == 0) {
      bad = 0;
      int q = 0;
      for (int d1 = 1; d1 <= w; ++d1)
        for (int d2 = 1; d2 <= d1; ++d2) {
          pairs[2 * q] = (short)d1;
          pairs[2 * q + 1] = (short)d2;
          ++q;
        }
    }
    for (int i = tid; i < tab; i += blockDim.x) postab[i] = -1;
    for (int i = tid; i < nI * w1; i += blockDim.x) sband[i] = 0.0;
    for (int i = tid; i < w1 * 32; i += blockDim.x) win[i] = 0.0;
    for (int i = tid; i < kStreamNB; i += blockDim.x) {
      sci[i] = -1;
      sca[i] = 0.0;
    }
    abb[si][sj] = 0.0f;
    __syncthreads();
    for (int q = tid; q < n; q += blockDim.x) {
      int x[3];
      coords1(G, gid[q] - dbase, x);
      int lin = 0, mul = 1;
      for (int a = 0; a < G.d; ++a) {
        lin += (x[a] - origin[a]) * mul;
        mul *= m1;
      }
      postab[lin] = q;
    }
    __syncthreads();
    // the stencil of every DOF: band rows (interior), couplings and the
    // A_BB share of the tile (boundary)
    for (int q = tid; q < n; q += blockDim.x) {
      const int64_t g = gid[q] - dbase;
      int x[3];
      coords1(G, g, x);
      int lin = 0, mul = 1, lstride[3] = {1, 1, 1}, onplane = 0;
      for (int a = 0; a < G.d; ++a) {
        lin += (x[a] - origin[a]) * mul;
        lstride[a] = mul;
        mul *= m1;
        onplane += (x[a] % m == 0);
      }
      const int b = q - nI;
      const bool rowin = b >= I * kRedoTile && b < (I + 1) * kRedoTile;
      if (q < nI) sband[q * w1] = diag[g];
      else if (rowin && b >= J * kRedoTile && b < (J + 1) * kRedoTile)
        abb[b - I * kRedoTile][b - J * kRedoTile] = float(diag[g] / double(1 << onplane));
      for (int a = 0; a < G.d; ++a) {
        const double share = double(1 << (onplane - (x[a] % m == 0)));
        const int lx = x[a] - origin[a];
        for (int dir = -1; dir <= 1; dir += 2) {
          if (dir > 0 && !(x[a] + 1 <= G.ns[a] && lx + 1 <= m)) continue;
          if (dir < 0 && !(x[a] - 1 >= 1 && lx - 1 >= 0)) continue;
          const int r = postab[lin + dir * lstride[a]];
          if (r < 0) continue;
          const double v = dir > 0 ? off[a * G.N + g] : off[a * G.N + g - G.stride[a]];
          if (q < nI) {
            if (r < nI && r > q) sband[q * w1 + (r - q)] = v;
          } else if (r < nI) {
            sci[b] = r;
            sca[b] = double(float(v));   // the coupling as the FP32 factor stores it
          } else if (rowin) {
            const int j = r - nI;
            if (j >= J * kRedoTile && j < (J + 1) * kRedoTile && j <= b)
              abb[b - I * kRedoTile][j - J * kRedoTile] = float(v / share);
          }
        }
      }
    }
    __syncthreads();
    const int my_ci = (zc < ncol && zb < nB) ? sci[zb] : -1;
    const double my_ca = (zc < ncol && zb < nB) ? sca[zb] : 0.0;
    // initial rows 0..w of the Z window: the single entry of column zb in row ci
    if (zr0 == 0 && my_ci >= 0 && my_ci <= w) win[(my_ci % w1) * 32 + zc] = my_ca;
    int pd1[2] = {0, 0}, pd2[2] = {0, 0};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int q = tid + h * kThreads;
      if (q < npair) {
        pd1[h] = pairs[2 * q];
        pd2[h] = pairs[2 * q + 1];
      }
    }
    double acc = 0.0;
    int slot = 0;   // k % (w + 1)
    __syncthreads();
    for (int k = 0; k < nI; ++k) {
      const int wk = min(w, nI - 1 - k);
      double* zk = win + slot * 32;
      double* colk = sband + k * w1;
      if (tid == 0) {   // 1. pivot of column k
        double dkk = colk[0];
        if (!(dkk > 0.0)) {
          bad = 1;
          dkk = 1.0;
        }
        s_piv = my_sqrt(dkk);
        s_rpiv = 1.0 / s_piv;   // once, not per thread
        colk[0] = s_piv;
      }
      __syncthreads();
      const double rpiv = s_rpiv;
      // 2. scale column k of L and row k of Z
      if (tid >= 1 && tid <= wk) colk[tid] *= rpiv;
      if (tid < ncol) zk[tid] *= rpiv;
      __syncthreads();
      // 3. trailing band update, Z rows k+1..k+wk, the S tile
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int d1 = pd1[h], d2 = pd2[h];
        if (d1 && d1 <= wk) sband[(k + d2) * w1 + (d1 - d2)] -= colk[d1] * colk[d2];
      }
      if (zc < ncol) {
        const double zv = zk[zc];
        int sl = slot + 1 + zr0;
        while (sl >= w1) sl -= w1;
        for (int dd = 1 + zr0; dd <= wk; dd += 8) {
          win[sl * 32 + zc] -= colk[dd] * zv;
          sl += 8;
          while (sl >= w1) sl -= w1;
        }
      }
      acc += zk[zi] * zk[zj];
      __syncthreads();
      // 4. recycle row k's slot for row k + w + 1
      const int nr = k + w1;
      if (tid < ncol) zk[tid] = (nr < nI && my_ci == nr) ? my_ca : 0.0;
      slot = (slot + 1 == w1) ? 0 : slot + 1;
      __syncthreads();
    }
    int ld;
    float* Fr = frame_of<float>(Lv, c, &ld);
    const int i = I * kRedoTile + si, j = J * kRedoTile + sj;
    if (i < nB && j < nB && i >= j) Fr[i + (int64_t)j * ld] = float(double(abb[si][sj]) - acc);
    if (t == 0) {   // band with reciprocal diagonal for the application
      float* band = (float*)Lv.band + Lv.band_off[c];
      for (int e = tid; e < nI * w1; e += blockDim.x)
        band[e] = float((e % w1 == 0) ? 1.0 / sband[e] : sband[e]);
      if (tid == 0 && bad) report(status, RHIF_ERR_NOT_SPD, 0, kKindCell, c);
    }
    __syncthreads();
  }
}

static size_t leaf_redo_smem(int max_nI, int max_w, int leaf, int d) {
  int tab = 1;
  for (int a = 0; a < d; ++a) tab *= leaf + 1;
  return round16((size_t)max_nI * (max_w + 1) * sizeof(double)) +
         round16((size_t)(max_w + 1) * 32 * sizeof(double)) + round16((size_t)tab * sizeof(int)) +
         round16((size_t)(max_w * (max_w + 1) / 2) * 2 * sizeof(short));
}

// The flagged leaves (list[0 .. count[0]) of an FP32 factor eliminated again
// in FP64, results rounded to the FP32 storage.  The grid covers up to 64
// flagged leaves at once; more are taken in turns.
void launch_leaf_fp64_redo(const GeoDev& G, const LevelDev& Lv, const double* diag,
                           const double* off, int* status, const int* list, const int* count,
                           cudaStream_t s) {
  if (!Lv.ncell || Lv.max_nB > kStreamNB || Lv.max_w >= 32) return;
  const size_t sm = leaf_redo_smem(Lv.max_nI, Lv.max_w, G.leaf, G.d);
  const unsigned gx = (unsigned)std::min(Lv.ncell, 64);
  launch_pdl(k_leaf_redo64, dim3(gx, kRedoTiles), kThreads, sm, s, G, Lv, diag, off, status, list, count);
}

// Redundant DOFs leave the active set only after every ID of the phase has
// been taken (the IDs all read the same matrix, Sec. 2.2 parallel order).
__global__ void k_mark_dead(LevelDev Lv, PhaseDev Ph, uint8_t* alive) {
  pdl_trigger();
  pdl_wait();   // what the previous kernel of the stream wrote
  const int u = blockIdx.x;
  const int g = Ph.u_group[u];
  const int n = Lv.group_size[g], k = Ph.rank[u];
  const int32_t* gg = Lv.bucket + Lv.group_start[g];
  const int* perm = Ph.perm + Ph.u_perm_off[u];
  for (int i = k + threadIdx.x; i < n; i += blockDim.x) alive[gg[perm[i]]] = 0;
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------

static inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

void launch_stencil_from_csr(const GeoDev& G, const int64_t* rowptr, const int32_t* col,
                             const double* val, int64_t nnz, double* diag, double* off,
                             double* offb, int* status, cudaStream_t s) {
  if (G.N == 0) return;
  launch_pdl(k_stencil_from_csr, blocks_for(G.N, 256), 256, 0, s, G, rowptr, col, val, nnz, diag, off,
                                                           offb, status);
  launch_pdl(k_stencil_check, blocks_for(G.d * G.N, 256), 256, 0, s, G.d * G.N, off, offb, status);
}

void launch_expand_gids(const LevelDev& Lv, cudaStream_t s) {
  if (Lv.ncell) launch_pdl(k_expand_gids, Lv.ncell, 128, 0, s, Lv);
}

template <typename T>
static bool leaf_warp_fits(const GeoDev& G, const LevelDev& Lv, int nbt) {
  if (G.d != 2 || Lv.max_w > kLeafWarpW || Lv.max_nB > nbt) return false;
  if (nbt == 64 && sizeof(T) != 4) return false;   // 64 accumulator columns fit registers in FP32 only
  return kLeafWarpCta * leaf_warp_bytes<T>(Lv.max_nI, G.leaf, nbt) <= 48 * 1024;
}

bool leaf_elim_needs_z(const GeoDev& G, const LevelDev& Lv, size_t elem) {
  const bool warp = elem == 4 ? (leaf_warp_fits<float>(G, Lv, 32) || leaf_warp_fits<float>(G, Lv, 64))
                              : leaf_warp_fits<double>(G, Lv, 32);
  return !warp && Lv.max_nB > kStreamNB;
}

template <typename T>
void launch_leaf_elim(const GeoDev& G, const LevelDev& Lv, const double* diag, const double* off,
                      int* status, cudaStream_t s) {
  if (!Lv.ncell) return;
  if (leaf_warp_fits<T>(G, Lv, 32)) {
    const size_t sm = kLeafWarpCta * leaf_warp_bytes<T>(Lv.max_nI, G.leaf, 32);
    launch_pdl(k_leaf_warp<T, 32>, (Lv.ncell + kLeafWarpCta - 1) / kLeafWarpCta, 32 * kLeafWarpCta, sm, s,
        G, Lv, diag, off, status);
    return;
  }
  if constexpr (sizeof(T) == 4) {   // no FP64 instance of the 64-column kernel
    if (leaf_warp_fits<T>(G, Lv, 64)) {
      const size_t sm = kLeafWarpCta * leaf_warp_bytes<T>(Lv.max_nI, G.leaf, 64);
      launch_pdl(k_leaf_warp<T, 64>, (Lv.ncell + kLeafWarpCta - 1) / kLeafWarpCta, 32 * kLeafWarpCta, sm, s,
          G, Lv, diag, off, status);
      return;
    }
  }
  if (Lv.max_nB <= kStreamNB) {
    const size_t sm = leaf_stream_smem<T>(Lv.max_nI, Lv.max_w, G.leaf, G.d);
    launch_pdl(k_leaf_stream<T>, Lv.ncell, kThreads, sm, s, G, Lv, diag, off, status);
    return;
  }
  const size_t sm = leaf_smem_bytes<T>(Lv.max_nI, Lv.max_nB, Lv.max_w, G.leaf, G.d);
  launch_pdl(k_leaf_elim<T>, Lv.ncell, kThreads, sm, s, G, Lv, diag, off, status);
}

template <typename T>
int launch_extend_add(const LevelDev& cur, const LevelDev& prev, int64_t front_total, int slots,
                      cudaStream_t s) {
  if (!cur.ncell) return 0;
  const int64_t nb = prev.max_nB;
  if (nb * nb * slots <= 128 * 1024) {   // small frames: one CTA per parent, one launch
    launch_pdl(k_extend_add_cell<T>, cur.ncell, kEaCellThreads, 0, s, cur, prev);
    return 1;
  }
  cudaMemsetAsync(cur.front, 0, (size_t)front_total * sizeof(T), s);
  const int chunk = 16 * kThreads;
  const unsigned chunks = (unsigned)((nb * nb + chunk - 1) / chunk);
  if (!chunks) return 0;
  for (int slot = 0; slot < slots; ++slot)
    launch_pdl(k_extend_add<T>, dim3(chunks, cur.ncell), kThreads, 0, s, cur, prev, slot, chunk);
  return slots;
}

template <typename T>
void launch_front_invert(const LevelDev& Lv, T* X, const int64_t* xoff, cudaStream_t s) {
  if (!Lv.ncell || !Lv.max_nI) return;
  const unsigned nb = (unsigned)((Lv.max_nI + kTile - 1) / kTile);
  launch_pdl(k_front_trinv<T>, dim3(nb, Lv.ncell), kThreads, kTile * (kTile + 1) * sizeof(T), s, Lv, X, xoff);
  launch_pdl(k_front_inv_store<T>, dim3(64, Lv.ncell), 256, 0, s, Lv, X, xoff);
}

template <typename T>
void launch_band_block_inverse(const LevelDev& Lv, cudaStream_t s) {
  if (!Lv.ncell) return;   // per-cell test inside: the apply decides per cell too
  launch_pdl(k_band_block_inverse<T>, (Lv.ncell + 7) / 8, 256, 0, s, Lv);
}

template <typename T>
void launch_partial_chol(const LevelDev& Lv, int* status, cudaStream_t s) {
  if (!Lv.ncell) return;
  launch_pdl(k_partial_chol<T>, Lv.ncell, kThreads, partial_chol_smem_elems() * sizeof(T), s, Lv, status);
}

template <typename T>
void launch_front_panel(const LevelDev& Lv, int p0, int* status, cudaStream_t s) {
  const size_t sm = kNB * (kNB + 1) * sizeof(T);
  launch_pdl(k_front_pdiag<T>, Lv.ncell, kThreads, sm, s, Lv, p0, status);
  const int rows = Lv.max_n - p0;
  if (rows > 0)
    launch_pdl(k_front_prows<T>, dim3((rows + kThreads - 1) / kThreads, Lv.ncell), kThreads, sm, s, Lv, p0);
}

template <typename T>
void launch_front_trailing(const LevelDev& Lv, int p0, int64_t tiles, cudaStream_t s) {
  if (tiles > 0)
    launch_pdl(k_front_trailing<T>, (unsigned)tiles, kThreads, 2 * kKC * (kTile + 1) * sizeof(T), s, Lv, p0);
}

template <typename T>
void launch_front_schur(const LevelDev& Lv, int64_t tiles, cudaStream_t s) {
  if (tiles > 0)
    launch_pdl(k_front_schur<T>, (unsigned)tiles, kThreads, 2 * kKC * (kTile + 1) * sizeof(T), s, Lv);
}

int64_t front_trailing_tiles(int nI, int n, int p0) { return trail_tiles(nI, n, p0); }
int64_t front_schur_tiles(int nI, int nB) { return schur_tiles(nI, nB); }

template <typename T>
int launch_precond_diag(const LevelDev& Lv, const PhaseDev& Ph, int* status, cudaStream_t s) {
  if (!Ph.npre) return 0;
  if (Ph.Linv && Lv.max_group <= 32) {   // factor and inverse, one warp per group
    constexpr int W = pdiag_warps<T>();
    launch_pdl(k_precond_diag_warp<T>, (Ph.npre + W - 1) / W, 32 * W, 0, s, Lv, Ph, status);
    return 1;
  }
  launch_pdl(k_precond_diag<T>, Ph.npre, kThreads, partial_chol_smem_elems() * sizeof(T), s, Lv, Ph, status);
  if (!Ph.Linv) return 1;
  const unsigned nb = (unsigned)((Lv.max_group + kTile - 1) / kTile);
  launch_pdl(k_group_trinv<T>, dim3(nb, Ph.npre), kThreads, kTile * (kTile + 1) * sizeof(T), s, Lv, Ph);
  return 2;
}

template <typename T>
int launch_unit_invert(const LevelDev& Lv, const PhaseDev& Ph, T* X, cudaStream_t s) {
  if (!Ph.nunit) return 0;
  if (Ph.max_n <= 32) {
    constexpr int W = trinv_warps<T>();
    launch_pdl(k_trinv_warp<T, true>, (Ph.nunit + W - 1) / W, 32 * W, 0, s, Lv, Ph, Ph.nunit);
    return 1;
  }
  const unsigned nb = (unsigned)((Ph.max_n + kTile - 1) / kTile);
  launch_pdl(k_unit_trinv<T>, dim3(nb, Ph.nunit), kThreads, kTile * (kTile + 1) * sizeof(T), s, Lv, Ph, X);
  const unsigned chunks = (unsigned)((Ph.max_n * Ph.max_n + 255) / 256);
  launch_pdl(k_unit_inv_store<T>, dim3(chunks, Ph.nunit), 256, 0, s, Lv, Ph, X);
  return 2;
}

template <typename T>
void launch_precond_scale(const LevelDev& Lv, const PhaseDev& Ph, int max_seg, cudaStream_t s) {
  if (!(Ph.npre && Lv.ncell)) return;
  const size_t blk = round16((size_t)Lv.max_nB * (Lv.max_nB | 1) * sizeof(T));
  const size_t xb = (size_t)max_seg * Lv.max_group * Lv.max_group * sizeof(T);
  if (blk + xb <= 96 * 1024) {
    launch_pdl(k_precond_scale<T>, Lv.ncell, kThreads, blk + xb, s, Lv, Ph, 1, 1);
  } else if (blk <= 200 * 1024) {
    launch_pdl(k_precond_scale<T>, Lv.ncell, kThreads, blk, s, Lv, Ph, 1, 0);
  } else {
    launch_pdl(k_precond_scale<T>, Lv.ncell, kThreads, 0, s, Lv, Ph, 0, 0);
  }
}

template <typename T>
void launch_precond_scale_big(const LevelDev& Lv, const PhaseDev& Ph, int64_t tasks,
                              cudaStream_t s) {
  launch_pdl(k_frame_symmetrize<T>, dim3(64, min(Lv.ncell, 65535)), 256, 0, s, Lv);
  if (tasks <= 0) return;
  const size_t sm = 2 * kKC * (kTile + 1) * sizeof(T);
  launch_pdl(k_frame_rows_tp<T>, (unsigned)tasks, kThreads, sm, s, Lv, Ph);
  launch_pdl(k_frame_cols_tp<T>, (unsigned)tasks, kThreads, sm, s, Lv, Ph);
}

template <typename T>
size_t skel_smem_bytes(int max_n) {
  return partial_chol_smem_elems() * sizeof(T) + (size_t)max_n * (sizeof(T) + sizeof(int)) + 32;
}

template <typename T>
void launch_skel(const LevelDev& Lv, const PhaseDev& Ph, uint8_t* alive, double tol, int* status,
                 int64_t max_m_elems, cudaStream_t s) {
  if (!Ph.nunit) return;
  size_t sm = skel_smem_bytes<T>(Ph.max_n);
  const size_t mb = (size_t)max_m_elems * sizeof(T);
  const int mstage = sm + mb <= 200 * 1024;
  if (mstage) sm += mb;
  launch_pdl(k_skel<T>, Ph.nunit, kThreads, sm, s, Lv, Ph, alive, tol, status, mstage);
  launch_pdl(k_mark_dead, Ph.nunit, 32, 0, s, Lv, Ph, alive);
}

template <typename T>
bool launch_skel_warp(const LevelDev& Lv, const PhaseDev& Ph, uint8_t* alive, double tol,
                      int* status, int64_t max_m_elems, cudaStream_t s) {
  if (!Ph.nunit) return true;
  if (Ph.max_n > 32) return false;
  const size_t per = skel_warp_bytes(Ph.max_n, max_m_elems, sizeof(T));
  int wpc = (int)std::min<size_t>(8, (200 * 1024) / per);
  if (wpc < 1) return false;
  const unsigned grid = (unsigned)((Ph.nunit + wpc - 1) / wpc);
  launch_pdl(k_skel_warp<T>, grid, 32 * wpc, wpc * per, s, Lv, Ph, alive, tol, status, (int)per);
  launch_pdl(k_mark_dead, Ph.nunit, 32, 0, s, Lv, Ph, alive);
  return true;
}

template <typename T>
size_t skel_cluster_fixed_bytes(int max_n, int C) {
  const size_t ldp = skel_cluster_ldp(max_n);
  return (partial_chol_smem_elems() + (1 + 2 * (size_t)C) * ldp) * sizeof(T) + ldp * sizeof(int) +
         32;
}

template <typename T>
int skel_cluster_schedulable(int C, size_t smem) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(C);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, (void*)k_skel_cluster<T>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

template <typename T>
cudaError_t launch_skel_cluster(const LevelDev& Lv, const PhaseDev& Ph, uint8_t* alive, double tol,
                                int* status, int C, int64_t slice_cap, size_t smem,
                                cudaStream_t s) {
  if (!Ph.nunit) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3((unsigned)Ph.nunit * C);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_skel_cluster<T>, Lv, Ph, alive, tol, status, slice_cap);
  if (e != cudaSuccess) return e;
  launch_pdl(k_mark_dead, Ph.nunit, 32, 0, s, Lv, Ph, alive);
  return cudaGetLastError();
}

template <typename T>
int configure_factor_kernels() {
  const int big = 220 * 1024;
  cudaError_t e = cudaFuncSetAttribute(k_skel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_skel_cluster<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_skel_warp<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_skel_cluster<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_leaf_elim<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_precond_scale<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_leaf_stream<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_leaf_redo64, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_leaf_cond<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  return e == cudaSuccess ? 0 : -1;
}

#define RHIF_INST(T)                                                                              \
  template size_t leaf_smem_bytes<T>(int, int, int, int, int);                                    \
  template void launch_leaf_elim<T>(const GeoDev&, const LevelDev&, const double*, const double*, \
                                    int*, cudaStream_t);                                          \
  template int launch_extend_add<T>(const LevelDev&, const LevelDev&, int64_t, int, cudaStream_t); \
  template void launch_partial_chol<T>(const LevelDev&, int*, cudaStream_t);                      \
  template void launch_band_block_inverse<T>(const LevelDev&, cudaStream_t);                     \
  template int launch_unit_invert<T>(const LevelDev&, const PhaseDev&, T*, cudaStream_t);        \
  template void launch_front_invert<T>(const LevelDev&, T*, const int64_t*, cudaStream_t);       \
  template void launch_front_panel<T>(const LevelDev&, int, int*, cudaStream_t);                  \
  template void launch_front_trailing<T>(const LevelDev&, int, int64_t, cudaStream_t);            \
  template void launch_front_schur<T>(const LevelDev&, int64_t, cudaStream_t);                    \
  template int launch_precond_diag<T>(const LevelDev&, const PhaseDev&, int*, cudaStream_t);     \
  template void launch_precond_scale<T>(const LevelDev&, const PhaseDev&, int, cudaStream_t);          \
  template void launch_precond_scale_big<T>(const LevelDev&, const PhaseDev&, int64_t,            \
                                            cudaStream_t);                                        \
  template void launch_skel<T>(const LevelDev&, const PhaseDev&, uint8_t*, double, int*, int64_t, \
                               cudaStream_t);                                                     \
  template size_t skel_smem_bytes<T>(int);                                                        \
  template size_t skel_cluster_fixed_bytes<T>(int, int);                                          \
  template bool launch_skel_warp<T>(const LevelDev&, const PhaseDev&, uint8_t*, double, int*,     \
                                    int64_t, cudaStream_t);                                       \
  template int skel_cluster_schedulable<T>(int, size_t);                                          \
  template cudaError_t launch_skel_cluster<T>(const LevelDev&, const PhaseDev&, uint8_t*, double, \
                                              int*, int, int64_t, size_t, cudaStream_t);          \
  template int configure_factor_kernels<T>();

RHIF_INST(double)
RHIF_INST(float)

}  // namespace rhif
