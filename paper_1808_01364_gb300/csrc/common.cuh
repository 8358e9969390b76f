// Device building blocks shared by the factorization and application kernels:
// status reporting, warp/CTA reductions, the CTA-wide blocked partial
// Cholesky of a dense front (Sec. 2.1 block elimination), and CTA-wide
// triangular solves.  All matrices are column-major; only the lower triangle
// of a symmetric matrix is read or written.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace rhif {

constexpr int kThreads = 256;   // threads per CTA of the dense kernels
constexpr int kNB = 32;         // panel width of the partial Cholesky
constexpr int kTile = 64;       // SYRK output tile
constexpr int kKC = 32;         // SYRK k-chunk

// status word layout (device int[8]): [0] error code, [1] level, [2] kind, [3] index
enum StatusKind { kKindCell = 1, kKindGroup = 2, kKindUnit = 3, kKindRoot = 4, kKindArg = 5 };

__device__ inline void report(int* status, int code, int level, int kind, int index) {
  if (atomicCAS(status, 0, code) == 0) {
    status[1] = level;
    status[2] = kind;
    status[3] = index;
  }
}

// ---------------------------------------------------------------------------
// Bulk global -> shared copies (cp.async.bulk, the TMA bulk path) completed on
// an mbarrier.  Source, destination and size must be multiples of 16 bytes;
// every factor block is padded so that they are.  Waits are bounded: after
// kWaitLimit polls the caller reports RHIF_ERR_TIMEOUT instead of spinning on.
// ---------------------------------------------------------------------------
constexpr int kWaitLimit = 1 << 22;

__device__ inline uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ inline void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ inline void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ inline void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Programmatic dependent launch (the sweeps of one F^{-1} application): a
// kernel lets the next one start as soon as all of its CTAs run
// (pdl_trigger), and the next one stages its factor blocks, which no sweep
// writes, before it waits for the previous kernel's completion and memory
// (pdl_wait) and only then reads the vectors.  Both are no-ops for a launch
// without the programmatic-serialization attribute.
__device__ inline void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ inline void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Launches a kernel of the factorization or of an F^{-1} sweep.  Small grids
// (at most kPdlMaxCtas CTAs: the upper levels, whose kernels are
// latency-bound) get programmatic stream serialization: the kernel may begin
// while the previous one on the stream finishes, and waits for it with
// pdl_wait before it reads what that kernel wrote (factorization kernels:
// first thing; sweeps: after staging their factor blocks).  Large grids are
// launched in plain stream order: there the waiting CTAs and their early
// staging slowed the running kernel down.
constexpr int64_t kPdlMaxCtas = 8 * 152;

template <typename... KArgs, typename... Args>
static void launch_pdl(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = (int64_t)grid.x * grid.y * grid.z <= kPdlMaxCtas ? 1 : 0;
  cudaLaunchKernelEx(&cfg, k, static_cast<KArgs>(args)...);
}

__device__ inline bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for phase `parity` of the barrier; false if it did not complete.
__device__ inline bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (int i = 0; i < kWaitLimit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

__host__ __device__ inline uint32_t round16(size_t bytes) { return (uint32_t)((bytes + 15) & ~size_t(15)); }
__host__ __device__ inline int64_t pad4e(int64_t n) { return (n + 3) & ~int64_t(3); }

template <typename T>
__device__ inline T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T> __device__ inline T my_sqrt(T x);
template <> __device__ inline double my_sqrt<double>(double x) { return sqrt(x); }
template <> __device__ inline float my_sqrt<float>(float x) { return sqrtf(x); }

// Element (i, j) of a symmetric matrix stored in its lower triangle.
template <typename T>
__device__ inline T sym_at(const T* A, int64_t ld, int i, int j) {
  return i >= j ? A[i + (int64_t)j * ld] : A[j + (int64_t)i * ld];
}

// One 64 x 64 output tile with corner (ti, tj):
// C[i,j] -= sum_{k in [k0,k1)} P[i,k] * P[j,k] for i in [ti, min(ti+64, r1)),
// j in [tj, min(tj+64, c1)), i >= j.  C and P are column-major (ldc, ldp); they
// may be the same matrix as long as the tile and the operand columns do not overlap.
template <typename T>
__device__ void cta_syrk_tile(T* C, int64_t ldc, const T* P, int64_t ldp, int ti, int tj, int r1,
                              int c1, int k0, int k1, T* sm) {
  T* si = sm;                          // [kKC][kTile+1]
  T* sj = sm + kKC * (kTile + 1);      // [kKC][kTile+1]
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
  for (int kc = k0; kc < k1; kc += kKC) {
    const int kk = min(kKC, k1 - kc);
    for (int idx = tid; idx < kTile * kKC; idx += kThreads) {
      const int i = idx % kTile, k = idx / kTile;
      const int gi = ti + i, gj = tj + i;
      si[k * (kTile + 1) + i] = (gi < r1 && k < kk) ? P[gi + (int64_t)(kc + k) * ldp] : T(0);
      sj[k * (kTile + 1) + i] = (gj < c1 && k < kk) ? P[gj + (int64_t)(kc + k) * ldp] : T(0);
    }
    __syncthreads();
    for (int k = 0; k < kk; ++k) {
      T av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = si[k * (kTile + 1) + ty + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = sj[k * (kTile + 1) + tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] += av[a] * bv[b];
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int i = ti + ty + 16 * a;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int j = tj + tx + 16 * b;
      if (i < r1 && j < c1 && i >= j) C[i + (int64_t)j * ldc] -= acc[a][b];
    }
  }
}

// C[i,j] -= sum_{k in [k0,k1)} P[i,k] * P[j,k] for i in [r0,r1), j in [c0,c1), i >= j,
// tile by tile with the whole CTA.
template <typename T>
__device__ void cta_syrk_lower(T* C, int64_t ldc, const T* P, int64_t ldp, int r0, int r1, int c0,
                               int c1, int k0, int k1, T* sm) {
  if (r0 >= r1 || c0 >= c1 || k0 >= k1) return;
  for (int ti = r0; ti < r1; ti += kTile) {
    for (int tj = c0; tj < c1; tj += kTile) {
      if (tj > ti + kTile - 1) break;   // tile entirely above the diagonal
      cta_syrk_tile(C, ldc, P, ldp, ti, tj, r1, c1, k0, k1, sm);
    }
  }
}

// One 64 x 64 tile of a general product: acc[a][b] = sum_{k < K} fa(i, k) * fb(k, j)
// for i = ti + ty + 16a < M, j = tj + tx + 16b < N (tx = tid % 16, ty = tid / 16);
// fa / fb are element accessors, so operands may be gathered, transposed or
// concatenated.  AK / BK: consecutive threads load consecutive k of A / B
// (operand contiguous along k) instead of consecutive rows / columns.
// Needs 2 * kKC * (kTile + 1) elements of shared memory.
template <typename T, bool AK = false, bool BK = false, class FA, class FB>
__device__ void cta_tile_product(int ti, int tj, int M, int N, int K, FA fa, FB fb, T* sm,
                                 T (&acc)[4][4]) {
  T* sa = sm;
  T* sb = sm + kKC * (kTile + 1);
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
  for (int kc = 0; kc < K; kc += kKC) {
    const int kk = min(kKC, K - kc);
    for (int idx = tid; idx < kTile * kKC; idx += kThreads) {
      const int i = AK ? idx / kKC : idx % kTile, k = AK ? idx % kKC : idx / kTile;
      sa[k * (kTile + 1) + i] = (ti + i < M && k < kk) ? fa(ti + i, kc + k) : T(0);
    }
    for (int idx = tid; idx < kTile * kKC; idx += kThreads) {
      const int i = BK ? idx / kKC : idx % kTile, k = BK ? idx % kKC : idx / kTile;
      sb[k * (kTile + 1) + i] = (tj + i < N && k < kk) ? fb(kc + k, tj + i) : T(0);
    }
    __syncthreads();
    for (int k = 0; k < kk; ++k) {
      T av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = sa[k * (kTile + 1) + ty + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = sb[k * (kTile + 1) + tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] += av[a] * bv[b];
    }
    __syncthreads();
  }
}

// Shared memory (elements of T) needed by cta_partial_chol.
constexpr int partial_chol_smem_elems() { return kNB * (kNB + 1) + 2 * kKC * (kTile + 1); }

// One panel of the blocked Cholesky: factor the nb x nb diagonal block at p0
// (warp 0) and scale the rows below it, rows (p0+nb .. n) <- rows * D^{-T}.
// Returns false if a pivot is not positive.  D is shared scratch of
// kNB*(kNB+1) elements.
// Factor the nb x nb diagonal block at p0 in place (warp 0, staged in D, a
// shared [kNB][kNB+1] array that keeps the factor on return).  Returns false
// if a pivot is not positive.
template <typename T>
__device__ bool cta_diag_chol(T* A, int64_t ld, int p0, int nb, T* D) {
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int idx = threadIdx.x; idx < nb * nb; idx += blockDim.x) {
    const int i = idx % nb, j = idx / nb;
    D[i * (kNB + 1) + j] = (i >= j) ? A[(p0 + i) + (int64_t)(p0 + j) * ld] : T(0);
  }
  __syncthreads();
  if (warp == 0) {
    for (int k = 0; k < nb; ++k) {
      T dkk = D[k * (kNB + 1) + k];
      if (!(dkk > T(0))) {
        if (lane == 0) bad = 1;
        dkk = T(1);
      }
      const T s = my_sqrt(dkk);
      __syncwarp();
      if (lane > k && lane < nb) D[lane * (kNB + 1) + k] /= s;
      if (lane == k) D[k * (kNB + 1) + k] = s;
      __syncwarp();
      if (lane > k && lane < nb) {
        const T lik = D[lane * (kNB + 1) + k];
        for (int j = k + 1; j <= lane; ++j) D[lane * (kNB + 1) + j] -= lik * D[j * (kNB + 1) + k];
      }
      __syncwarp();
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < nb * nb; idx += blockDim.x) {
    const int i = idx % nb, j = idx / nb;
    if (i >= j) A[(p0 + i) + (int64_t)(p0 + j) * ld] = D[i * (kNB + 1) + j];
  }
  __syncthreads();
  return bad == 0;
}

// Rows [r0, r1) of the panel at p0 (nb columns) <- rows * L_pp^{-T}, with the
// factored diagonal block in D; one row per thread.
template <typename T>
__device__ void cta_panel_rows(T* A, int64_t ld, int r0, int r1, int p0, int nb, const T* D) {
  for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
    T r[kNB];
#pragma unroll
    for (int j = 0; j < kNB; ++j) r[j] = (j < nb) ? A[i + (int64_t)(p0 + j) * ld] : T(0);
#pragma unroll
    for (int j = 0; j < kNB; ++j) {
      if (j < nb) {
        T s = r[j];
#pragma unroll
        for (int q = 0; q < j; ++q) s -= r[q] * D[j * (kNB + 1) + q];
        r[j] = s / D[j * (kNB + 1) + j];
      }
    }
#pragma unroll
    for (int j = 0; j < kNB; ++j)
      if (j < nb) A[i + (int64_t)(p0 + j) * ld] = r[j];
  }
}

// One panel of the blocked Cholesky: factor the nb x nb diagonal block at p0
// and scale the rows below it, rows (p0+nb .. n) <- rows * D^{-T}.  Returns
// false if a pivot is not positive.  D is shared scratch of kNB*(kNB+1)
// elements.
template <typename T>
__device__ bool cta_panel(T* A, int64_t ld, int n, int p0, int nb, T* D) {
  const bool ok = cta_diag_chol(A, ld, p0, nb, D);
  cta_panel_rows(A, ld, p0 + nb, n, p0, nb, D);
  __syncthreads();
  return ok;
}

// X[:, J0 : J0+64] = L^{-1} E[:, J0 : J0+64] for the n x n lower-triangular L
// (ld ldl), written to X (ld ldx) for rows J0..n: by 64-row blocks from the
// diagonal down, a tile product with the rows above and then a per-column
// solve with the diagonal block staged in shared memory.  Rows above J0 are
// not written.  sm: kTile*(kTile+1) >= 2*kKC*(kTile+1) elements.
template <typename T>
__device__ void cta_trinv_block(const T* L, int64_t ldl, int n, T* X, int64_t ldx, int J0, T* sm) {
  const int nc = min(kTile, n - J0);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  auto fa = [&](int i, int k) { return L[i + (int64_t)(J0 + k) * ldl]; };
  auto fb = [&](int k, int j) { return X[(J0 + k) + (int64_t)(J0 + j) * ldx]; };
  for (int I0 = J0; I0 < n; I0 += kTile) {
    const int nr = min(kTile, n - I0);
    T acc[4][4];
    cta_tile_product<T, false, true>(I0, 0, n, nc, I0 - J0, fa, fb, sm, acc);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int i = ty + 16 * a, j = tx + 16 * b;
        if (i < nr && j < nc)
          X[(I0 + i) + (int64_t)(J0 + j) * ldx] = (I0 + i == J0 + j ? T(1) : T(0)) - acc[a][b];
      }
    T* Rb = sm;   // L[I, I], [kTile][kTile + 1]
    for (int idx = tid; idx < nr * nr; idx += blockDim.x) {
      const int i = idx / nr, q = idx % nr;
      Rb[i * (kTile + 1) + q] = q <= i ? L[(I0 + i) + (int64_t)(I0 + q) * ldl] : T(0);
    }
    __syncthreads();
    // per-column forward solve, four threads per column: the sum over q < i
    // is split four ways and combined with two shuffles; every lane of a warp
    // takes part in every step (lanes past the block only skip the write)
    const int grp = tid >> 2, sub = tid & 3;
    for (int j0 = 0; j0 < nc; j0 += (int)blockDim.x / 4) {
      const int j = j0 + grp;
      const bool act = j < nc;
      T* col = X + (int64_t)(J0 + (act ? j : 0)) * ldx + I0;
      for (int i = 0; i < nr; ++i) {
        T part = T(0);
        if (act)
          for (int q = sub; q < i; q += 4) part += Rb[i * (kTile + 1) + q] * col[q];
        part += __shfl_xor_sync(0xffffffffu, part, 1);
        part += __shfl_xor_sync(0xffffffffu, part, 2);
        const T v = act ? (col[i] - part) / Rb[i * (kTile + 1) + i] : T(0);
        __syncwarp();
        if (act && sub == 0) col[i] = v;
        __syncwarp();
      }
    }
    __syncthreads();
  }
}

// Blocked partial Cholesky of the n x n SPD front A (lower triangle, ld):
// eliminates the first nI unknowns (Sec. 2.1, Eq. 2.1).  On return
//   A[0:nI, 0:nI]  holds L        with A_II = L L^T,
//   A[nI:n, 0:nI]  holds W = A_BI L^{-T} (= X^T of the paper),
//   A[nI:n, nI:n]  holds the Schur complement A_BB - W W^T.
// Returns false (and leaves garbage) if a pivot is not positive.
template <typename T>
__device__ bool cta_partial_chol(T* A, int64_t ld, int n, int nI, T* sm) {
  T* D = sm;                                   // [kNB][kNB+1] row-major
  T* syrk_sm = sm + kNB * (kNB + 1);
  bool ok = true;
  for (int p0 = 0; p0 < nI; p0 += kNB) {
    const int nb = min(kNB, nI - p0);
    const int p1 = p0 + nb;
    ok &= cta_panel(A, ld, n, p0, nb, D);
    // trailing update restricted to the columns still to be eliminated
    cta_syrk_lower(A, ld, A, ld, p1, n, p1, nI, p0, p1, syrk_sm);
    __syncthreads();
  }
  // Schur complement of the boundary block in one pass over k = 0..nI
  cta_syrk_lower(A, ld, A, ld, nI, n, nI, n, 0, nI, syrk_sm);
  __syncthreads();
  return ok;
}

// y <- L^{-1} y for the n x n lower-triangular L (ld), y in shared memory.
template <typename T>
__device__ void cta_trsv_lower(const T* L, int64_t ld, int n, T* y) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int b0 = 0; b0 < n; b0 += 32) {
    const int nb = min(32, n - b0);
    if (warp == 0) {
      T yi = lane < nb ? y[b0 + lane] : T(0);
      for (int k = 0; k < nb; ++k) {
        const T yk = __shfl_sync(0xffffffffu, yi, k) / L[(b0 + k) + (int64_t)(b0 + k) * ld];
        if (lane == k) yi = yk;
        else if (lane > k && lane < nb) yi -= L[(b0 + lane) + (int64_t)(b0 + k) * ld] * yk;
      }
      if (lane < nb) y[b0 + lane] = yi;
    }
    __syncthreads();
    for (int i = b0 + nb + threadIdx.x; i < n; i += blockDim.x) {
      T s = T(0);
      for (int k = 0; k < nb; ++k) s += L[i + (int64_t)(b0 + k) * ld] * y[b0 + k];
      y[i] -= s;
    }
    __syncthreads();
  }
}

// y <- L^{-T} y for the n x n lower-triangular L (ld), y in shared memory.
template <typename T>
__device__ void cta_trsv_lower_t(const T* L, int64_t ld, int n, T* y) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  if (n <= 0) return;
  for (int b0 = ((n - 1) / 32) * 32; b0 >= 0; b0 -= 32) {
    const int nb = min(32, n - b0);
    const int below = b0 + nb;
    for (int k = warp; k < nb; k += nwarps) {
      T s = T(0);
      for (int i = below + lane; i < n; i += 32) s += L[i + (int64_t)(b0 + k) * ld] * y[i];
      s = warp_sum(s);
      if (lane == 0) y[b0 + k] -= s;
    }
    __syncthreads();
    if (warp == 0) {
      T yi = lane < nb ? y[b0 + lane] : T(0);
      for (int k = nb - 1; k >= 0; --k) {
        T c = (lane > k && lane < nb) ? L[(b0 + lane) + (int64_t)(b0 + k) * ld] * yi : T(0);
        c = warp_sum(c);
        if (lane == k) yi = (yi - c) / L[(b0 + k) + (int64_t)(b0 + k) * ld];
      }
      if (lane < nb) y[b0 + lane] = yi;
    }
    __syncthreads();
  }
}

// y <- L^{-1} y with L banded (column k of band holds 1/L[k,k], L[k+1..k+w, k]); one warp.
template <typename T>
__device__ inline void warp_band_fwd(const T* band, int n, int w, T* y) {
  const int lane = threadIdx.x & 31;
  const int w1 = w + 1;
  for (int k = 0; k < n; ++k) {
    const T yk = y[k] * band[k * w1];
    __syncwarp();
    if (lane == 0) y[k] = yk;
    const int wk = min(w, n - 1 - k);
    for (int d = 1 + lane; d <= wk; d += 32) y[k + d] -= band[k * w1 + d] * yk;
    __syncwarp();
  }
}

// y <- L^{-T} y with L banded; one warp.
template <typename T>
__device__ inline void warp_band_bwd(const T* band, int n, int w, T* y) {
  const int lane = threadIdx.x & 31;
  const int w1 = w + 1;
  for (int k = n - 1; k >= 0; --k) {
    const int wk = min(w, n - 1 - k);
    T s = T(0);
    for (int d = 1 + lane; d <= wk; d += 32) s += band[k * w1 + d] * y[k + d];
    s = warp_sum(s);
    if (lane == 0) y[k] = (y[k] - s) * band[k * w1];
    __syncwarp();
  }
}


// Blocked forms for w <= 31: blocks of w rows, lane r owns row s + r.  The
// coupling of a block to the w rows before (after) it is one dot product per
// lane; the triangle inside the block is solved in registers with shuffles.
template <typename T>
__device__ inline void warp_band_fwd_blk(const T* band, int n, int w, T* y) {
  const int lane = threadIdx.x & 31;
  const int w1 = w + 1;
  for (int s0 = 0; s0 < n; s0 += w) {
    const int B = min(w, n - s0);
    const int i = s0 + lane;
    T acc = T(0);
    if (lane < B) {
      acc = y[i];
      for (int d = lane + 1; d <= w; ++d) {
        const int j = i - d;
        if (j < 0) break;
        acc -= band[j * w1 + d] * y[j];
      }
    }
    for (int c = 0; c < B; ++c) {
      const T yc = __shfl_sync(0xffffffffu, acc, c) * band[(s0 + c) * w1];
      if (lane == c) acc = yc;
      else if (lane > c && lane < B) acc -= band[(s0 + c) * w1 + (lane - c)] * yc;
    }
    if (lane < B) y[i] = acc;
    __syncwarp();
  }
}

template <typename T>
__device__ inline void warp_band_bwd_blk(const T* band, int n, int w, T* y) {
  const int lane = threadIdx.x & 31;
  const int w1 = w + 1;
  const int nblk = (n + w - 1) / w;
  for (int bi = nblk - 1; bi >= 0; --bi) {
    const int s0 = bi * w;
    const int B = min(w, n - s0);
    const int i = s0 + lane;
    T acc = T(0);
    if (lane < B) {
      acc = y[i];
      for (int d = B - lane; d <= w; ++d) {
        const int j = i + d;
        if (j >= n) break;
        acc -= band[i * w1 + d] * y[j];
      }
    }
    for (int c = B - 1; c >= 0; --c) {
      const T yc = __shfl_sync(0xffffffffu, acc, c) * band[(s0 + c) * w1];
      if (lane == c) acc = yc;
      else if (lane < c) acc -= band[(s0 + lane) * w1 + (c - lane)] * yc;
    }
    if (lane < B) y[i] = acc;
    __syncwarp();
  }
}

}  // namespace rhif
