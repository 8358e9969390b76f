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
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n && off[i] != offb[i]) report(status, RHIF_ERR_BAD_ARG, -1, kKindArg, (int)(i % 2147483647));
}

// ---------------------------------------------------------------------------
// level-0 fronts straight from the stencil
// ---------------------------------------------------------------------------

__device__ inline void coords1(const GeoDev& G, int64_t gid, int x[3]) {
  int64_t rem = gid;
  x[0] = x[1] = x[2] = 1;
  for (int a = 0; a < G.d; ++a) {
    x[a] = (int)(rem % G.ns[a]) + 1;
    rem /= G.ns[a];
  }
}

// Entry (i, j) of A is split equally among the leaf cells whose closure holds
// both i and j (a power of two, so the split is exact); the level matrix is
// the sum of the per-cell fronts.
template <typename T>
__global__ void k_front_leaf(GeoDev G, LevelDev Lv, const double* diag, const double* off,
                             int* status) {
  extern __shared__ int postab[];
  const int c = blockIdx.x;
  const int nI = Lv.nI[c], n = nI + Lv.nB[c];
  T* F = (T*)Lv.front + Lv.front_off[c];
  const int64_t* gid = Lv.gids + Lv.gid_off[c];
  const int m = G.leaf, m1 = G.leaf + 1;
  int origin[3] = {0, 0, 0};
  {
    int64_t code = Lv.cell_code[c];
    for (int a = 0; a < G.d; ++a) {
      const int v = (int)(code % Lv.code_base);
      code /= Lv.code_base;
      origin[a] = ((v - 1) / 2) * m;
    }
  }
  int tab = 1;
  for (int a = 0; a < G.d; ++a) tab *= m1;
  for (int i = threadIdx.x; i < tab; i += blockDim.x) postab[i] = -1;
  __syncthreads();
  for (int p = threadIdx.x; p < n; p += blockDim.x) {
    int x[3];
    coords1(G, gid[p], x);
    int lin = 0, mul = 1;
    for (int a = 0; a < G.d; ++a) {
      lin += (x[a] - origin[a]) * mul;
      mul *= m1;
    }
    postab[lin] = p;
  }
  for (int64_t idx = threadIdx.x; idx < (int64_t)n * n; idx += blockDim.x) F[idx] = T(0);
  __syncthreads();
  for (int p = threadIdx.x; p < n; p += blockDim.x) {
    const int64_t g = gid[p];
    int x[3];
    coords1(G, g, x);
    int lin = 0, mul = 1, lstride[3] = {1, 1, 1};
    int onplane = 0;
    for (int a = 0; a < G.d; ++a) {
      lin += (x[a] - origin[a]) * mul;
      lstride[a] = mul;
      mul *= m1;
      onplane += (x[a] % m == 0);
    }
    F[p + (int64_t)p * n] = T(diag[g] / double(1 << onplane));
    for (int a = 0; a < G.d; ++a) {
      const int others = onplane - (x[a] % m == 0);
      const double share = double(1 << others);
      const int lx = x[a] - origin[a];
      if (x[a] + 1 <= G.ns[a] && lx + 1 <= m) {
        const int q = postab[lin + lstride[a]];
        if (q >= 0) F[p + (int64_t)q * n] = T(off[a * G.N + g] / share);
      }
      if (x[a] - 1 >= 1 && lx - 1 >= 0) {
        const int q = postab[lin - lstride[a]];
        if (q >= 0) F[p + (int64_t)q * n] = T(off[a * G.N + g - G.stride[a]] / share);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// level >= 1 fronts: extend-add of the children's frames, children in a fixed order
// ---------------------------------------------------------------------------

template <typename T>
__global__ void k_extend_add(LevelDev cur, LevelDev prev) {
  const int c = blockIdx.x;
  const int n = cur.nI[c] + cur.nB[c];
  T* F = (T*)cur.front + cur.front_off[c];
  for (int64_t idx = threadIdx.x; idx < (int64_t)n * n; idx += blockDim.x) F[idx] = T(0);
  __syncthreads();
  for (int k = cur.ea_off[c]; k < cur.ea_off[c + 1]; ++k) {
    const int pc = cur.ea_child[k];
    const int* map = cur.ea_map + cur.ea_map_off[k];
    const int nIc = prev.nI[pc], nbc = prev.nB[pc], nc = nIc + nbc;
    const T* Fc = (const T*)prev.front + prev.front_off[pc] + nIc + (int64_t)nIc * nc;
    for (int64_t idx = threadIdx.x; idx < (int64_t)nbc * nbc; idx += blockDim.x) {
      const int i = (int)(idx % nbc), j = (int)(idx / nbc);
      if (i < j) continue;
      const int pi = map[i], pj = map[j];
      if (pi < 0 || pj < 0) continue;
      const int r = max(pi, pj), s = min(pi, pj);
      F[r + (int64_t)s * n] += Fc[i + (int64_t)j * nc];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// cell elimination (Sec. 2.1): partial Cholesky of every front
// ---------------------------------------------------------------------------

template <typename T>
__global__ void __launch_bounds__(kThreads) k_partial_chol(LevelDev Lv, int* status) {
  extern __shared__ unsigned char smraw[];
  T* sm = (T*)smraw;
  const int c = blockIdx.x;
  const int nI = Lv.nI[c], n = nI + Lv.nB[c];
  T* F = (T*)Lv.front + Lv.front_off[c];
  if (!cta_partial_chol(F, n, n, nI, sm) && threadIdx.x == 0)
    report(status, RHIF_ERR_NOT_SPD, Lv.level, Lv.level < 0 ? kKindRoot : kKindCell, c);
}

// ---------------------------------------------------------------------------
// block Jacobi preconditioning (Sec. 2.3)
// ---------------------------------------------------------------------------

template <typename T>
__device__ inline T* frame_of(const LevelDev& Lv, int c, int* ld) {
  const int nI = Lv.nI[c], n = nI + Lv.nB[c];
  *ld = n;
  return (T*)Lv.front + Lv.front_off[c] + nI + (int64_t)nI * n;
}

// L_g = chol(sum over the cells holding g of their diagonal block of g)
template <typename T>
__global__ void __launch_bounds__(kThreads) k_precond_diag(LevelDev Lv, PhaseDev Ph, int* status) {
  extern __shared__ unsigned char smraw[];
  T* sm = (T*)smraw;
  const int b = blockIdx.x;
  const int g = Ph.pre_group[b];
  const int sz = (int)(Lv.group_gid_off[g + 1] - Lv.group_gid_off[g]);
  T* Lg = (T*)Ph.Lbuf + Ph.pre_off[b];
  for (int64_t idx = threadIdx.x; idx < (int64_t)sz * sz; idx += blockDim.x) {
    const int i = (int)(idx % sz), j = (int)(idx / sz);
    T s = T(0);
    if (i >= j) {
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

// frame <- D^{-1} frame D^{-T}, D = block diag of the L_g of the frame's groups
template <typename T>
__global__ void __launch_bounds__(kThreads) k_precond_scale(LevelDev Lv, PhaseDev Ph) {
  const int c = blockIdx.x;
  int ld;
  T* Fr = frame_of<T>(Lv, c, &ld);
  const int nb = Lv.nB[c];
  for (int64_t idx = threadIdx.x; idx < (int64_t)nb * nb; idx += blockDim.x) {
    const int i = (int)(idx % nb), j = (int)(idx / nb);
    if (i < j) Fr[i + (int64_t)j * ld] = Fr[j + (int64_t)i * ld];
  }
  __syncthreads();
  const int s0 = Lv.seg_off[c], s1 = Lv.seg_off[c + 1];
  const int64_t work = (int64_t)(s1 - s0) * nb;
  // rows: F[g, :] <- L_g^{-1} F[g, :]
  for (int64_t t = threadIdx.x; t < work; t += blockDim.x) {
    const int s = s0 + (int)(t / nb), j = (int)(t % nb);
    const int g = Lv.seg_group[s];
    const int pi = Ph.group_pre[g];
    if (pi < 0) continue;
    const int sz = (int)(Lv.group_gid_off[g + 1] - Lv.group_gid_off[g]);
    const int pos = Lv.seg_pos[s];
    const T* Lg = (const T*)Ph.Lbuf + Ph.pre_off[pi];
    T* col = Fr + (int64_t)j * ld + pos;
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
    const int sz = (int)(Lv.group_gid_off[g + 1] - Lv.group_gid_off[g]);
    const int pos = Lv.seg_pos[s];
    const T* Lg = (const T*)Ph.Lbuf + Ph.pre_off[pi];
    T* row = Fr + i + (int64_t)pos * ld;
    for (int a = 0; a < sz; ++a) {
      T v = row[(int64_t)a * ld];
      for (int q = 0; q < a; ++q) v -= Lg[a + (int64_t)q * sz] * row[(int64_t)q * ld];
      row[(int64_t)a * ld] = v / Lg[a + (int64_t)a * sz];
    }
  }
}

// ---------------------------------------------------------------------------
// skeletonization (Sec. 2.2) of one unit per CTA
// ---------------------------------------------------------------------------

template <typename T> __device__ inline T my_abs(T x) { return x < T(0) ? -x : x; }

template <typename T>
__global__ void __launch_bounds__(kThreads) k_skel(LevelDev Lv, PhaseDev Ph, uint8_t* alive,
                                                   double tol, int* status) {
  extern __shared__ unsigned char smraw[];
  T* sm = (T*)smraw;                                   // partial-Cholesky workspace
  T* nrm = sm + partial_chol_smem_elems();             // [max_n]
  int* sperm = (int*)(nrm + Ph.max_n);                 // [max_n]
  __shared__ int s_k, s_stop, s_p;
  __shared__ T s_r11;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int u = blockIdx.x;
  const int g = Ph.u_group[u];
  const int64_t g0 = Lv.group_gid_off[g];
  const int n = (int)(Lv.group_gid_off[g + 1] - g0);
  const int64_t* gg = Lv.group_gids + g0;
  const int nrow = Ph.u_nrow[u];
  const int ldm = nrow > 0 ? nrow : 1;
  T* M = (T*)Ph.Mbuf + Ph.u_m_off[u];
  T* Aee = M + (int64_t)nrow * n;
  T* Fu = (T*)Ph.rec + Ph.u_rec_off[u];
  T* Tm = Fu + (int64_t)n * n;
  const int c0 = Lv.group_cell_off[g], c1 = Lv.group_cell_off[g + 1];

  // 1. gather A_{R,I} (rows summed over the cells holding them, in cell order) and A_II
  const int64_t rb = Ph.u_row_off[u];
  for (int64_t idx = tid; idx < (int64_t)nrow * n; idx += blockDim.x) {
    const int r = (int)(idx % nrow), j = (int)(idx / nrow);
    const int64_t gr = rb + r;
    T v = T(0);
    if (alive[Ph.u_row_gid[gr]]) {
      for (int64_t s = Ph.row_src_off[gr]; s < Ph.row_src_off[gr + 1]; ++s) {
        int ld;
        const T* fr = frame_of<T>(Lv, Ph.src_cell[s], &ld);
        v += sym_at(fr, ld, Ph.src_pos[s], Ph.src_upos[s] + j);
      }
    }
    M[r + (int64_t)j * ldm] = v;
  }
  for (int64_t idx = tid; idx < (int64_t)n * n; idx += blockDim.x) {
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
  for (int i = tid; i < n; i += blockDim.x) sperm[i] = i;
  if (tid == 0) {
    s_k = 0;
    s_r11 = T(0);
  }
  __syncthreads();

  // 2. column-pivoted Householder QR of M, norms recomputed at every step,
  //    stopped once the largest remaining column norm is <= tol * |R_11|
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
    if (tid == 0) {
      T mx = T(0);
      for (int c = j; c < n; ++c) mx = nrm[c] > mx ? nrm[c] : mx;
      if (j == 0) s_r11 = my_sqrt(mx);
      const int stop = (s_r11 == T(0)) || (my_sqrt(mx) <= T(tol) * s_r11);
      s_stop = stop;
      if (!stop) {
        const T thr = T(1.0 - 1e-12) * mx;
        int best = -1;
        for (int c = j; c < n; ++c)
          if (nrm[c] >= thr && (best < 0 || sperm[c] < sperm[best])) best = c;
        s_p = best;
      }
    }
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
  const int k = s_k;
  const int r = n - k;

  // 3. interpolation matrix T = R11^{-1} R12 (k x r)
  for (int a = tid; a < r; a += blockDim.x) {
    for (int i = k - 1; i >= 0; --i) {
      T t = M[i + (int64_t)(k + a) * ldm];
      for (int q = i + 1; q < k; ++q) t -= M[i + (int64_t)q * ldm] * Tm[q + (int64_t)a * k];
      Tm[i + (int64_t)a * k] = t / M[i + (int64_t)i * ldm];
    }
  }
  __syncthreads();

  // 4. zeroing (Eq. 2.2): Z^T A_II Z in (redundant, skeleton) order
  //    [rd,rd] = A_rr - T^T A_sr - A_sr^T T + T^T A_ss T ; [sk,rd] = A_sr - A_ss T ; [sk,sk] = A_ss
  for (int64_t idx = tid; idx < (int64_t)k * r; idx += blockDim.x) {
    const int q = (int)(idx % k), a = (int)(idx / k);
    T v = Aee[sperm[q] + (int64_t)sperm[k + a] * n];
    for (int p = 0; p < k; ++p) v -= Aee[sperm[q] + (int64_t)sperm[p] * n] * Tm[p + (int64_t)a * k];
    Fu[(r + q) + (int64_t)a * n] = v;
  }
  __syncthreads();
  for (int64_t idx = tid; idx < (int64_t)r * r; idx += blockDim.x) {
    const int a = (int)(idx % r), b = (int)(idx / r);
    if (a < b) continue;
    T v = Aee[sperm[k + a] + (int64_t)sperm[k + b] * n];
    for (int q = 0; q < k; ++q)
      v -= Tm[q + (int64_t)a * k] * Fu[(r + q) + (int64_t)b * n] +
           Aee[sperm[q] + (int64_t)sperm[k + a] * n] * Tm[q + (int64_t)b * k];
    Fu[a + (int64_t)b * n] = v;
  }
  for (int64_t idx = tid; idx < (int64_t)k * k; idx += blockDim.x) {
    const int q = (int)(idx % k), p = (int)(idx / k);
    if (q < p) continue;
    Fu[(r + q) + (int64_t)(r + p) * n] = Aee[sperm[q] + (int64_t)sperm[p] * n];
  }
  __syncthreads();

  // 5. eliminate the redundant DOFs (Sec. 2.1 applied to the zeroed block)
  if (!cta_partial_chol(Fu, n, n, r, sm) && tid == 0)
    report(status, RHIF_ERR_NOT_SPD, Lv.level, kKindUnit, g);
  __syncthreads();

  // 6. the skeleton block of the first holding cell takes the new value, the
  //    others drop theirs; redundant DOFs leave the active set
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
  for (int i = tid; i < n; i += blockDim.x) {
    perm_out[i] = sperm[i];
    if (i >= k) alive[gg[sperm[i]]] = 0;
  }
  if (tid == 0) Ph.rank[u] = k;
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------

static inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

void launch_stencil_from_csr(const GeoDev& G, const int64_t* rowptr, const int32_t* col,
                             const double* val, int64_t nnz, double* diag, double* off,
                             double* offb, int* status, cudaStream_t s) {
  if (G.N == 0) return;
  k_stencil_from_csr<<<blocks_for(G.N, 256), 256, 0, s>>>(G, rowptr, col, val, nnz, diag, off,
                                                           offb, status);
  k_stencil_check<<<blocks_for(G.d * G.N, 256), 256, 0, s>>>(G.d * G.N, off, offb, status);
}

template <typename T>
void launch_front_leaf(const GeoDev& G, const LevelDev& Lv, const double* diag, const double* off,
                       int* status, cudaStream_t s) {
  if (!Lv.ncell) return;
  int tab = 1;
  for (int a = 0; a < G.d; ++a) tab *= G.leaf + 1;
  k_front_leaf<T><<<Lv.ncell, kThreads, tab * sizeof(int), s>>>(G, Lv, diag, off, status);
}

template <typename T>
void launch_extend_add(const LevelDev& cur, const LevelDev& prev, cudaStream_t s) {
  if (!cur.ncell) return;
  k_extend_add<T><<<cur.ncell, kThreads, 0, s>>>(cur, prev);
}

template <typename T>
void launch_partial_chol(const LevelDev& Lv, int* status, cudaStream_t s) {
  if (!Lv.ncell) return;
  k_partial_chol<T><<<Lv.ncell, kThreads, partial_chol_smem_elems() * sizeof(T), s>>>(Lv, status);
}

template <typename T>
void launch_precond_diag(const LevelDev& Lv, const PhaseDev& Ph, int* status, cudaStream_t s) {
  if (Ph.npre)
    k_precond_diag<T><<<Ph.npre, kThreads, partial_chol_smem_elems() * sizeof(T), s>>>(Lv, Ph, status);
}

template <typename T>
void launch_precond_scale(const LevelDev& Lv, const PhaseDev& Ph, cudaStream_t s) {
  if (Ph.npre && Lv.ncell) k_precond_scale<T><<<Lv.ncell, kThreads, 0, s>>>(Lv, Ph);
}

template <typename T>
size_t skel_smem_bytes(int max_n) {
  return partial_chol_smem_elems() * sizeof(T) + (size_t)max_n * (sizeof(T) + sizeof(int)) + 16;
}

template <typename T>
void launch_skel(const LevelDev& Lv, const PhaseDev& Ph, uint8_t* alive, double tol, int* status,
                 cudaStream_t s) {
  if (!Ph.nunit) return;
  const size_t sm = skel_smem_bytes<T>(Ph.max_n);
  k_skel<T><<<Ph.nunit, kThreads, sm, s>>>(Lv, Ph, alive, tol, status);
}

template <typename T>
int configure_factor_kernels() {
  const int big = 200 * 1024;
  cudaError_t e = cudaFuncSetAttribute(k_skel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e != cudaSuccess) return -1;
  e = cudaFuncSetAttribute(k_front_leaf<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  return e == cudaSuccess ? 0 : -1;
}

#define RHIF_INST(T)                                                                              \
  template void launch_front_leaf<T>(const GeoDev&, const LevelDev&, const double*, const double*, \
                                     int*, cudaStream_t);                                          \
  template void launch_extend_add<T>(const LevelDev&, const LevelDev&, cudaStream_t);              \
  template void launch_partial_chol<T>(const LevelDev&, int*, cudaStream_t);                       \
  template void launch_precond_diag<T>(const LevelDev&, const PhaseDev&, int*, cudaStream_t);      \
  template void launch_precond_scale<T>(const LevelDev&, const PhaseDev&, cudaStream_t);           \
  template void launch_skel<T>(const LevelDev&, const PhaseDev&, uint8_t*, double, int*,           \
                               cudaStream_t);                                                      \
  template size_t skel_smem_bytes<T>(int);                                                         \
  template int configure_factor_kernels<T>();

RHIF_INST(double)
RHIF_INST(float)

}  // namespace rhif
