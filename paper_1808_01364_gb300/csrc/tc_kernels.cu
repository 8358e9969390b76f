// Tensor-core (tcgen05) tile products for the dense Schur updates of large
// fronts (Sec. 2.1, C_BB -= W W^T and the trailing updates of the blocked
// elimination), with FP32 data on the 5th-generation tensor cores.
//
// One CTA of 128 threads (4 warps) computes a 128 x 64 tile D = A B^T with
// FP32 accumulation in tensor memory.  The operands are loaded by the threads
// in chunks of 32 along K (coalesced: the fronts are column-major, the tile's
// rows contiguous), converted, and stored in shared memory in the K-major
// no-swizzle core-matrix layout; two stages alternate, so the threads convert
// chunk c+1 while the tensor cores multiply chunk c.  Three operand kinds:
//  * TF32x3: each value split into a TF32 high part and a TF32 remainder
//    (a = hi + lo), products hi*hi + hi*lo + lo*hi (kind::tf32): about FP32
//    accuracy, which the Schur updates of high-contrast problems need when
//    the factor is to stay an FP32 factor;
//  * TF32: one kind::tf32 product of the rounded values (~2^-11 per product);
//  * BF16: one kind::f16 product with both operands rounded to BF16 (~2^-8
//    per product), FP32 accumulation;
// the last two trade factor accuracy for tensor-core rate and leave the
// accuracy to the FP64 PCG around the factor.  One elected thread issues the
// MMAs and commits each chunk to its stage's mbarrier; every wait is bounded,
// and on a timeout the CTA records RHIF_ERR_TIMEOUT, waits once more for its
// MMAs, frees its tensor memory and returns.
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"
#include "tables.h"
#include "../../include/rhif.h"

namespace rhif {
namespace tc {

constexpr int kM = 128, kN = 64, kK = 32;   // tile and K chunk
constexpr int kThreadsTc = 128;
constexpr uint32_t kTmemCols = 64;

// Shared-memory matrix descriptor, K-major, no swizzle: 8-row x 16-byte core
// matrices; lbo = byte step between core matrices along K, sbo = along M/N.
__device__ inline uint64_t sdesc(const void* p, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((smem_u32(p) >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;   // descriptor version of this architecture family
  return d;                 // base offset 0, layout type 0 (no swizzle)
}

// Instruction descriptors: D FP32 (bits 4-5 = 1), A and B both K-major, N/8
// at bit 17, M/16 at bit 24.  kind::tf32 takes TF32 (2) for A and B;
// kind::f16 takes BF16 (1) for both (A and B always of the same type).
constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}
constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ inline void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ inline void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ inline void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ inline void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ inline void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}

__device__ inline void mma_tf32(uint32_t dtm, uint64_t ad, uint64_t bd, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtm),
      "l"(ad), "l"(bd), "r"(id), "r"(acc)
      : "memory");
}

__device__ inline void mma_f16(uint32_t dtm, uint64_t ad, uint64_t bd, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtm),
      "l"(ad), "l"(bd), "r"(id), "r"(acc)
      : "memory");
}

__device__ inline void commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

// 16 consecutive accumulator columns of this thread's row (its warp's lanes).
__device__ inline void ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ inline void split_tf32(float x, float& hi, float& lo) {
  uint32_t h;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
  hi = __uint_as_float(h);
  lo = x - hi;
}

// byte offset of element (r, k) of an R x 32 K-major no-swizzle tile of
// 4-byte elements: core matrices of 8 rows x 4 elements, consecutive along K
// (LBO 128 bytes), 8-row groups 1024 bytes apart (SBO)
__device__ inline uint32_t core_off4(int r, int k) {
  return (uint32_t)(((r >> 3) * (kK / 4) + (k >> 2)) * 128 + (r & 7) * 16 + (k & 3) * 4);
}
// the same for 2-byte elements: core matrices of 8 rows x 8 elements (LBO
// 128 bytes), 8-row groups 512 bytes apart
__device__ inline uint32_t core_off2(int r, int k) {
  return (uint32_t)(((r >> 3) * (kK / 8) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

enum TcKind { kTcTf32x3 = 0, kTcTf32 = 1, kTcBf16 = 2 };
constexpr int kStages = 2;

// One stage holds the high and low planes of A (kM x kK) and B (kN x kK) as
// FP32 / TF32 values; BF16 tiles use the first half of the high planes.
struct TileSmem {
  float a_hi[kStages][kM * kK], a_lo[kStages][kM * kK];
  float b_hi[kStages][kN * kK], b_lo[kStages][kN * kK];
  uint64_t bar[kStages];
  uint32_t tmem;
};

// Convert chunk [k0, k0 + kK) of the operands into stage `st`.
template <int Kind, class FA, class FB>
__device__ inline void stage_chunk(TileSmem& S, int st, int M, int N, int k0, int kk, FA fa, FB fb) {
  const int tid = threadIdx.x;
  if constexpr (Kind == kTcBf16) {
    unsigned char* A2 = reinterpret_cast<unsigned char*>(S.a_hi[st]);
    unsigned char* B2 = reinterpret_cast<unsigned char*>(S.b_hi[st]);
    for (int idx = tid; idx < kM * kK / 2; idx += kThreadsTc) {
      const int k = 2 * (idx / kM), r = idx % kM;
      const float x0 = (r < M && k < kk) ? fa(r, k0 + k) : 0.f;
      const float x1 = (r < M && k + 1 < kk) ? fa(r, k0 + k + 1) : 0.f;
      *reinterpret_cast<__nv_bfloat162*>(A2 + core_off2(r, k)) = __floats2bfloat162_rn(x0, x1);
    }
    for (int idx = tid; idx < kN * kK / 2; idx += kThreadsTc) {
      const int k = 2 * (idx / kN), r = idx % kN;
      const float x0 = (r < N && k < kk) ? fb(r, k0 + k) : 0.f;
      const float x1 = (r < N && k + 1 < kk) ? fb(r, k0 + k + 1) : 0.f;
      *reinterpret_cast<__nv_bfloat162*>(B2 + core_off2(r, k)) = __floats2bfloat162_rn(x0, x1);
    }
  } else {
    for (int idx = tid; idx < kM * kK; idx += kThreadsTc) {
      const int k = idx / kM, r = idx % kM;
      const float x = (r < M && k < kk) ? fa(r, k0 + k) : 0.f;
      const uint32_t o = core_off4(r, k) >> 2;
      if constexpr (Kind == kTcTf32x3) {
        float hi, lo;
        split_tf32(x, hi, lo);
        S.a_hi[st][o] = hi;
        S.a_lo[st][o] = lo;
      } else {
        S.a_hi[st][o] = x;   // kind::tf32 reads the leading 19 bits
      }
    }
    for (int idx = tid; idx < kN * kK; idx += kThreadsTc) {
      const int k = idx / kN, r = idx % kN;
      const float x = (r < N && k < kk) ? fb(r, k0 + k) : 0.f;
      const uint32_t o = core_off4(r, k) >> 2;
      if constexpr (Kind == kTcTf32x3) {
        float hi, lo;
        split_tf32(x, hi, lo);
        S.b_hi[st][o] = hi;
        S.b_lo[st][o] = lo;
      } else {
        S.b_hi[st][o] = x;
      }
    }
  }
}

// The MMAs of one staged chunk (issued by one thread); acc0 = 0 for the
// first chunk (overwrite the accumulator).
template <int Kind>
__device__ inline void issue_chunk(TileSmem& S, int st, uint32_t tmem, bool first) {
  if constexpr (Kind == kTcBf16) {
    constexpr uint32_t idesc = idesc_bf16(kM, kN);
    const uint32_t lbo = 128, sbo = 8 * 64;   // 8 rows x 16 bytes x (kK / 8) core matrices
#pragma unroll
    for (int s = 0; s < kK / 16; ++s) {   // K = 16 BF16 (two core matrices) per MMA
      const uint32_t koff = s * 2 * 128;
      const uint64_t ad = sdesc((const char*)S.a_hi[st] + koff, lbo, sbo);
      const uint64_t bd = sdesc((const char*)S.b_hi[st] + koff, lbo, sbo);
      mma_f16(tmem, ad, bd, idesc, (!first || s > 0) ? 1u : 0u);
    }
  } else {
    constexpr uint32_t idesc = idesc_tf32(kM, kN);
    const uint32_t sbo = 8 * 128, lbo = 128;
#pragma unroll
    for (int s = 0; s < kK / 8; ++s) {   // K = 8 TF32 (two core matrices) per MMA
      const uint32_t koff = s * 2 * 128;
      const uint64_t ah = sdesc((const char*)S.a_hi[st] + koff, lbo, sbo);
      const uint64_t bh = sdesc((const char*)S.b_hi[st] + koff, lbo, sbo);
      mma_tf32(tmem, ah, bh, idesc, (!first || s > 0) ? 1u : 0u);
      if constexpr (Kind == kTcTf32x3) {
        const uint64_t al = sdesc((const char*)S.a_lo[st] + koff, lbo, sbo);
        const uint64_t bl = sdesc((const char*)S.b_lo[st] + koff, lbo, sbo);
        mma_tf32(tmem, ah, bl, idesc, 1u);
        mma_tf32(tmem, al, bh, idesc, 1u);
      }
    }
  }
}

// D (128 x 64) = sum_{k < K} fa(i, k) fb(j, k) over rows i < M of the tile,
// columns j < N (zero beyond), then epi(i, j, d) for every i < M, j < N.
// All 128 threads of the CTA must call it.  Returns false on a wait timeout.
template <int Kind, class FA, class FB, class EPI>
__device__ bool tile_product(TileSmem& S, int M, int N, int K, FA fa, FB fb, EPI epi) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) tmem_alloc(&S.tmem, kTmemCols);
  if (tid == 0) {
    mbar_init(&S.bar[0], 1);
    mbar_init(&S.bar[1], 1);
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = S.tmem;
  // bit st of `phase`: parity of stage st's next completion; bit st of
  // `pending`: a commit of stage st not yet waited for (bit masks, no local arrays)
  uint32_t phase = 0, pending = 0;
  bool ok = true;
  const int nchunk = (K + kK - 1) / kK;
  for (int c = 0; c < nchunk && ok; ++c) {
    const int st = c & 1;
    if (pending >> st & 1u) {   // the MMAs of chunk c - 2 still read this stage
      ok = __syncthreads_and(mbar_wait(&S.bar[st], phase >> st & 1u)) != 0;   // CTA-uniform
      phase ^= 1u << st;
      pending &= ~(1u << st);
      if (!ok) break;
      fence_after();
    }
    stage_chunk<Kind>(S, st, M, N, c * kK, min(kK, K - c * kK), fa, fb);
    fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      fence_after();
      issue_chunk<Kind>(S, st, tmem, c == 0);
      commit(&S.bar[st]);
    }
    pending |= 1u << st;
  }
  // drain: every stage with a commit in flight (on a timeout, once more with
  // the limit, so that no MMA still runs when the tensor memory is freed)
  for (int st = 0; st < kStages; ++st)
    if (pending >> st & 1u) {
      const bool w = __syncthreads_and(mbar_wait(&S.bar[st], phase >> st & 1u)) != 0;
      ok = ok && w;
    }
  fence_after();
  if (ok && K > 0) {
    // epilogue: warp w owns accumulator rows 32w .. 32w+31
    const int row = warp * 32 + lane;
#pragma unroll
    for (int c0 = 0; c0 < kN; c0 += 16) {
      float v[16];
      ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (row < M) {
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (c0 + j < N) epi(row, c0 + j, v[j]);
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kTmemCols);
  return ok;
}

// C (column-major, ldc) -= A B^T, A M x K (lda), B N x K (ldb), column-major.
template <int Kind>
__global__ void __launch_bounds__(kThreadsTc) k_tc_gemm_check(int M, int N, int K, const float* A,
                                                             int64_t lda, const float* B,
                                                             int64_t ldb, float* C, int64_t ldc,
                                                             int* status) {
  extern __shared__ __align__(128) unsigned char smraw[];
  TileSmem& S = *reinterpret_cast<TileSmem*>(smraw);
  const int i0 = blockIdx.x * kM, j0 = blockIdx.y * kN;
  auto fa = [&](int r, int k) { return A[(i0 + r) + (int64_t)k * lda]; };
  auto fb = [&](int r, int k) { return B[(j0 + r) + (int64_t)k * ldb]; };
  auto epi = [&](int r, int j, float d) { C[(i0 + r) + (int64_t)(j0 + j) * ldc] -= d; };
  if (!tile_product<Kind>(S, min(kM, M - i0), min(kN, N - j0), K, fa, fb, epi) &&
      threadIdx.x == 0)
    report(status, RHIF_ERR_TIMEOUT, -1, kKindArg, blockIdx.x);
}

// Schur complement of every front of the level on the tensor cores:
// F[B, B] -= W W^T with W = F[B, I] (rows nI.. of the first nI columns), one
// CTA per 128 x 64 tile (a, b) of the boundary block; tiles entirely above
// the diagonal exit at once, tiles crossing it update only i >= j.
template <int Kind>
__global__ void __launch_bounds__(kThreadsTc) k_front_schur_tc(LevelDev Lv, int* status) {
  extern __shared__ __align__(128) unsigned char smraw[];
  TileSmem& S = *reinterpret_cast<TileSmem*>(smraw);
  int64_t bid = blockIdx.x;
  int c = 0;
  int rt = 0, ct = 0;
  for (; c < Lv.ncell; ++c) {
    const int nB = Lv.nB[c];
    rt = (nB + kM - 1) / kM;
    ct = (nB + kN - 1) / kN;
    const int64_t t = Lv.nI[c] > 0 ? (int64_t)rt * ct : 0;
    if (bid < t) break;
    bid -= t;
  }
  if (c >= Lv.ncell) return;
  const int a = (int)(bid / ct), b = (int)(bid % ct);
  if (b * kN > a * kM + kM - 1) return;   // above the diagonal (uniform per CTA)
  const int nI = Lv.nI[c], nB = Lv.nB[c], n = nI + nB;
  float* F = (float*)Lv.front + Lv.front_off[c];
  const int i0 = nI + a * kM, j0 = nI + b * kN;
  auto fa = [&](int r, int k) { return F[(i0 + r) + (int64_t)k * n]; };
  auto fb = [&](int r, int k) { return F[(j0 + r) + (int64_t)k * n]; };
  auto epi = [&](int r, int j, float d) {
    if (i0 + r >= j0 + j) F[(i0 + r) + (int64_t)(j0 + j) * n] -= d;
  };
  if (!tile_product<Kind>(S, min(kM, n - i0), min(kN, n - j0), nI, fa, fb, epi) &&
      threadIdx.x == 0)
    report(status, RHIF_ERR_TIMEOUT, Lv.level, kKindCell, c);
}

}  // namespace tc

size_t tc_tile_smem_bytes() { return sizeof(tc::TileSmem) + 128; }

int64_t front_schur_tc_tiles(int nI, int nB) {
  if (nI == 0 || nB == 0) return 0;
  return (int64_t)((nB + tc::kM - 1) / tc::kM) * ((nB + tc::kN - 1) / tc::kN);
}

void launch_front_schur_tc(const LevelDev& Lv, int64_t tiles, int kind, int* status,
                           cudaStream_t s) {
  if (tiles <= 0) return;
  const unsigned g = (unsigned)tiles;
  const size_t sm = tc_tile_smem_bytes();
  if (kind == tc::kTcBf16)
    tc::k_front_schur_tc<tc::kTcBf16><<<g, tc::kThreadsTc, sm, s>>>(Lv, status);
  else if (kind == tc::kTcTf32)
    tc::k_front_schur_tc<tc::kTcTf32><<<g, tc::kThreadsTc, sm, s>>>(Lv, status);
  else
    tc::k_front_schur_tc<tc::kTcTf32x3><<<g, tc::kThreadsTc, sm, s>>>(Lv, status);
}

template <int Kind>
static cudaError_t configure_kind() {
  const int sm = (int)tc_tile_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(tc::k_tc_gemm_check<Kind>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(tc::k_front_schur_tc<Kind>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  return e;
}

int configure_tc_kernels() {
  cudaError_t e = configure_kind<tc::kTcTf32x3>();
  if (e == cudaSuccess) e = configure_kind<tc::kTcTf32>();
  if (e == cudaSuccess) e = configure_kind<tc::kTcBf16>();
  return e == cudaSuccess ? 0 : -1;
}

void launch_tc_gemm_check(int kind, int M, int N, int K, const float* A, int64_t lda,
                          const float* B, int64_t ldb, float* C, int64_t ldc, int* status,
                          cudaStream_t s) {
  dim3 grid((M + tc::kM - 1) / tc::kM, (N + tc::kN - 1) / tc::kN);
  const size_t sm = tc_tile_smem_bytes();
  if (kind == tc::kTcBf16)
    tc::k_tc_gemm_check<tc::kTcBf16><<<grid, tc::kThreadsTc, sm, s>>>(M, N, K, A, lda, B, ldb, C,
                                                                      ldc, status);
  else if (kind == tc::kTcTf32)
    tc::k_tc_gemm_check<tc::kTcTf32><<<grid, tc::kThreadsTc, sm, s>>>(M, N, K, A, lda, B, ldb, C,
                                                                      ldc, status);
  else
    tc::k_tc_gemm_check<tc::kTcTf32x3><<<grid, tc::kThreadsTc, sm, s>>>(M, N, K, A, lda, B, ldb,
                                                                        C, ldc, status);
}

}  // namespace rhif
