// PCG vector kernels of a merged batch of independent problems (Sec. 4 PCG,
// one instance per problem and right-hand side, all advanced by the same
// launches).  The vectors of the problems are concatenated (one column per
// right-hand side, leading dimension = total DOFs); a vector block never
// straddles two problems, so each block reads its problem's scalars and its
// partial sums belong to one problem.  Dots are deterministic: per-block
// partials, then a fixed-order sum over each problem's blocks.
#include "common.cuh"
#include "kernels.h"
#include "tables.h"

namespace rhif {

namespace {

constexpr int kBThreads = 256;

__device__ inline double bsum(double v) {
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

// scalars of (problem p, right-hand side r)
__device__ inline double* scal(double* sc, const VecSeg& S, int p, int r) {
  return sc + 8 * ((int64_t)r * S.nprob + p);
}

__global__ void k_bspmv(VecSeg S, const BatchGeo* bg, const double* x, int64_t ldx, double* y,
                        int64_t ldy, double* partial) {
  const int b = blockIdx.x, r = blockIdx.y;
  const int p = S.prob[b];
  const BatchGeo& P = bg[p];
  const double* xr = x + r * ldx + P.base;
  double* yr = y + r * ldy + P.base;
  double acc = 0.0;
  for (int64_t i = S.row0[b] - P.base + threadIdx.x; i < S.row1[b] - P.base; i += blockDim.x) {
    double s = P.diag[i] * xr[i];
    int64_t rem = i;
    for (int a = 0; a < P.G.d; ++a) {
      const int xa = (int)(rem % P.G.ns[a]);
      rem /= P.G.ns[a];
      const int64_t st = P.G.stride[a];
      if (xa + 1 < P.G.ns[a]) s += P.off[a * P.G.N + i] * xr[i + st];
      if (xa >= 1) s += P.off[a * P.G.N + i - st] * xr[i - st];
    }
    yr[i] = s;
    acc += s * xr[i];
  }
  if (partial) {
    const double t = bsum(acc);
    if (threadIdx.x == 0) partial[b + (int64_t)S.nblk * r] = t;
  }
}

__global__ void k_bdot_partial(VecSeg S, const double* a, int64_t lda, const double* c, int64_t ldc,
                               double* partial) {
  const int b = blockIdx.x, r = blockIdx.y;
  double acc = 0.0;
  for (int64_t i = S.row0[b] + threadIdx.x; i < S.row1[b]; i += blockDim.x)
    acc += a[i + r * lda] * c[i + r * ldc];
  const double t = bsum(acc);
  if (threadIdx.x == 0) partial[b + (int64_t)S.nblk * r] = t;
}

// one block per (problem, right-hand side): the modes of k_reduce
__global__ void k_breduce(VecSeg S, const double* partial, double* sc, int mode, double rtol) {
  const int p = blockIdx.x, r = blockIdx.y;
  double acc = 0.0;
  for (int b = S.pblk_off[p] + threadIdx.x; b < S.pblk_off[p + 1]; b += blockDim.x)
    acc += partial[b + (int64_t)S.nblk * r];
  const double s = bsum(acc);
  if (threadIdx.x != 0) return;
  double* C = scal(sc, S, p, r);
  switch (mode) {
    case 0: C[kScFF] = s; break;
    case 1: C[kScRZ] = s; break;
    case 2:
      C[kScPQ] = s;
      C[kScAlpha] = (C[kScDone] != 0.0 || s == 0.0) ? 0.0 : C[kScRZ] / s;
      break;
    case 3:
      C[kScRR] = s;
      if (C[kScDone] == 0.0 && sqrt(s) <= rtol * sqrt(C[kScFF])) C[kScDone] = 1.0;
      break;
    case 4:
      C[kScBeta] = (C[kScDone] != 0.0 || C[kScRZ] == 0.0) ? 0.0 : s / C[kScRZ];
      C[kScRZ] = s;
      break;
  }
}

__global__ void k_bupdate_xr(VecSeg S, const double* sc, double* x, int64_t ldx, double* rv,
                             int64_t ldr, const double* pv, int64_t ldp, const double* q,
                             int64_t ldq, double* partial) {
  const int b = blockIdx.x, r = blockIdx.y;
  const double* C = sc + 8 * ((int64_t)r * S.nprob + S.prob[b]);
  const double alpha = C[kScAlpha];
  const bool live = C[kScDone] == 0.0;
  double acc = 0.0;
  for (int64_t i = S.row0[b] + threadIdx.x; i < S.row1[b]; i += blockDim.x) {
    double ri = rv[i + r * ldr];
    if (live) {
      x[i + r * ldx] += alpha * pv[i + r * ldp];
      ri -= alpha * q[i + r * ldq];
      rv[i + r * ldr] = ri;
    }
    acc += ri * ri;
  }
  const double t = bsum(acc);
  if (threadIdx.x == 0) partial[b + (int64_t)S.nblk * r] = t;
}

__global__ void k_bupdate_p(VecSeg S, const double* sc, const double* z, int64_t ldz, double* pv,
                            int64_t ldp, int first) {
  const int b = blockIdx.x, r = blockIdx.y;
  const double* C = sc + 8 * ((int64_t)r * S.nprob + S.prob[b]);
  if (!first && C[kScDone] != 0.0) return;
  const double beta = first ? 0.0 : C[kScBeta];
  for (int64_t i = S.row0[b] + threadIdx.x; i < S.row1[b]; i += blockDim.x)
    pv[i + r * ldp] = first ? z[i + r * ldz] : z[i + r * ldz] + beta * pv[i + r * ldp];
}

// concatenated column r <- problem p's column r (src[p], N_p x nrhs, ld N_p)
// (gather) or the reverse (scatter)
__global__ void k_bgather(VecSeg S, const BatchGeo* bg, const double* const* src, double* y,
                          int64_t ldy) {
  const int b = blockIdx.x, r = blockIdx.y;
  const int p = S.prob[b];
  const int64_t base = bg[p].base, n = bg[p].G.N;
  const double* s = src[p] + r * n;
  for (int64_t i = S.row0[b] + threadIdx.x; i < S.row1[b]; i += blockDim.x)
    y[i + r * ldy] = s[i - base];
}

__global__ void k_bscatter(VecSeg S, const BatchGeo* bg, const double* x, int64_t ldx,
                           double* const* dst) {
  const int b = blockIdx.x, r = blockIdx.y;
  const int p = S.prob[b];
  const int64_t base = bg[p].base, n = bg[p].G.N;
  double* d = dst[p] + r * n;
  for (int64_t i = S.row0[b] + threadIdx.x; i < S.row1[b]; i += blockDim.x)
    d[i - base] = x[i + r * ldx];
}

}  // namespace

void batch_vec_blocks(const std::vector<int64_t>& base, const std::vector<int64_t>& n,
                      std::vector<int>& prob, std::vector<int64_t>& row0,
                      std::vector<int64_t>& row1, std::vector<int>& pblk_off) {
  prob.clear();
  row0.clear();
  row1.clear();
  pblk_off.assign(1, 0);
  for (size_t p = 0; p < n.size(); ++p) {
    for (int64_t i = 0; i < n[p]; i += kBatchRows) {
      prob.push_back((int)p);
      row0.push_back(base[p] + i);
      row1.push_back(base[p] + std::min<int64_t>(i + kBatchRows, n[p]));
    }
    pblk_off.push_back((int)prob.size());
  }
}

void launch_bspmv(const VecSeg& S, const BatchGeo* bg, const double* x, int64_t ldx, double* y,
                  int64_t ldy, int nrhs, double* partial, cudaStream_t s) {
  if (S.nblk) k_bspmv<<<dim3(S.nblk, nrhs), kBThreads, 0, s>>>(S, bg, x, ldx, y, ldy, partial);
}
void launch_bdot_partial(const VecSeg& S, const double* a, int64_t lda, const double* c,
                         int64_t ldc, int nrhs, double* partial, cudaStream_t s) {
  if (S.nblk) k_bdot_partial<<<dim3(S.nblk, nrhs), kBThreads, 0, s>>>(S, a, lda, c, ldc, partial);
}
void launch_breduce(const VecSeg& S, const double* partial, int nrhs, double* sc, int mode,
                    double rtol, cudaStream_t s) {
  if (S.nprob) k_breduce<<<dim3(S.nprob, nrhs), kBThreads, 0, s>>>(S, partial, sc, mode, rtol);
}
void launch_bupdate_xr(const VecSeg& S, int nrhs, const double* sc, double* x, int64_t ldx,
                       double* r, int64_t ldr, const double* p, int64_t ldp, const double* q,
                       int64_t ldq, double* partial, cudaStream_t s) {
  if (S.nblk)
    k_bupdate_xr<<<dim3(S.nblk, nrhs), kBThreads, 0, s>>>(S, sc, x, ldx, r, ldr, p, ldp, q, ldq,
                                                          partial);
}
void launch_bupdate_p(const VecSeg& S, int nrhs, const double* sc, const double* z, int64_t ldz,
                      double* p, int64_t ldp, int first, cudaStream_t s) {
  if (S.nblk) k_bupdate_p<<<dim3(S.nblk, nrhs), kBThreads, 0, s>>>(S, sc, z, ldz, p, ldp, first);
}
void launch_bgather(const VecSeg& S, const BatchGeo* bg, const double* const* src, double* y,
                    int64_t ldy, int nrhs, cudaStream_t s) {
  if (S.nblk) k_bgather<<<dim3(S.nblk, nrhs), kBThreads, 0, s>>>(S, bg, src, y, ldy);
}
void launch_bscatter(const VecSeg& S, const BatchGeo* bg, const double* x, int64_t ldx,
                     double* const* dst, int nrhs, cudaStream_t s) {
  if (S.nblk) k_bscatter<<<dim3(S.nblk, nrhs), kBThreads, 0, s>>>(S, bg, x, ldx, dst);
}

}  // namespace rhif
