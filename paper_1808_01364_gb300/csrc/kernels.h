// Host launchers of the CUDA kernels (factor_kernels.cu, apply_kernels.cu).
#pragma once
#include <cstdint>
#include <vector>
#include <cuda_runtime.h>

#include "tables.h"

namespace rhif {

// PCG scalar slots (8 doubles per right-hand side)
enum { kScRZ = 0, kScPQ = 1, kScRR = 2, kScFF = 3, kScAlpha = 4, kScDone = 5, kScBeta = 6 };

void launch_stencil_from_csr(const GeoDev& G, const int64_t* rowptr, const int32_t* col,
                             const double* val, int64_t nnz, double* diag, double* off,
                             double* offb, int* status, cudaStream_t s);
void launch_expand_gids(const LevelDev& Lv, cudaStream_t s);
template <typename T>
size_t leaf_smem_bytes(int max_nI, int max_nB, int max_w, int leaf, int d);
// Whether launch_leaf_elim takes the panel kernel, the one that keeps
// Z = L^{-1} A_IB in Lv.zbuf (nI x nB per cell); the others need no scratch.
bool leaf_elim_needs_z(const GeoDev& G, const LevelDev& Lv, size_t elem);
template <typename T>
void launch_leaf_elim(const GeoDev& G, const LevelDev& Lv, const double* diag, const double* off,
                      int* status, cudaStream_t s);
// In-place explicit inverses of the diagonal blocks of the leaf bands with
// w <= kBandInvW (other cells untouched).
template <typename T>
void launch_band_block_inverse(const LevelDev& Lv, cudaStream_t s);
// Zero the level's fronts and add the children's Schur complements, one
// launch per child slot (slots = most children of any cell); returns the
// number of kernel launches.
template <typename T>
int launch_extend_add(const LevelDev& cur, const LevelDev& prev, int64_t front_total, int slots,
                      cudaStream_t s);
// Overwrite the interior factor L of every front of the level with L^{-1}
// (X: scratch of sum_c nI_c^2 elements at per-cell offsets xoff).
template <typename T>
void launch_front_invert(const LevelDev& Lv, T* X, const int64_t* xoff, cudaStream_t s);
template <typename T>
void launch_partial_chol(const LevelDev& Lv, int* status, cudaStream_t s);
template <typename T>
void launch_front_panel(const LevelDev& Lv, int p0, int* status, cudaStream_t s);
template <typename T>
void launch_front_trailing(const LevelDev& Lv, int p0, int64_t tiles, cudaStream_t s);
template <typename T>
void launch_front_schur(const LevelDev& Lv, int64_t tiles, cudaStream_t s);
int64_t front_trailing_tiles(int nI, int n, int p0);
int64_t front_schur_tiles(int nI, int nB);
// Replaces the leading r x r block L_rr of every unit record of the phase by
// L_rr^{-1} (lower triangle), through X (scratch laid out like the records).
// Returns the number of launches.
template <typename T>
int launch_unit_invert(const LevelDev& Lv, const PhaseDev& Ph, T* X, cudaStream_t s);
template <typename T>
int launch_precond_diag(const LevelDev& Lv, const PhaseDev& Ph, int* status, cudaStream_t s);   // launches
template <typename T>
void launch_precond_scale(const LevelDev& Lv, const PhaseDev& Ph, int max_seg, cudaStream_t s);
// Tile-product scaling of large frames; needs Ph.Linv (filled by
// launch_precond_diag when non-null) and the scale_task tables; `tasks` is
// the total number of 64-wide blocks.
template <typename T>
void launch_precond_scale_big(const LevelDev& Lv, const PhaseDev& Ph, int64_t tasks,
                              cudaStream_t s);
template <typename T>
void launch_skel(const LevelDev& Lv, const PhaseDev& Ph, uint8_t* alive, double tol, int* status,
                 int64_t max_m_elems, cudaStream_t s);
template <typename T>
size_t skel_smem_bytes(int max_n);
// Skeletonization with one thread-block cluster of C CTAs per unit; each CTA
// stages its row slice of A_{R,g} in shared memory when it has at most
// slice_cap elements.  smem = skel_cluster_fixed_bytes + slice bytes.
// One warp per unit when every unit has n <= 32 and fits the warp's shared
// memory; returns false (nothing launched) otherwise.
template <typename T>
bool launch_skel_warp(const LevelDev& Lv, const PhaseDev& Ph, uint8_t* alive, double tol,
                      int* status, int64_t max_m_elems, cudaStream_t s);
template <typename T>
size_t skel_cluster_fixed_bytes(int max_n, int C);
template <typename T>
int skel_cluster_schedulable(int C, size_t smem);   // clusters that fit at once (0: none)
template <typename T>
cudaError_t launch_skel_cluster(const LevelDev& Lv, const PhaseDev& Ph, uint8_t* alive, double tol,
                                int* status, int C, int64_t slice_cap, size_t smem, cudaStream_t s);
template <typename T>
int configure_factor_kernels();

template <typename T>
void launch_apply_cell_up(const LevelDev& Lv, double* x, int64_t ldx, int nrhs, double* ubuf,
                          int64_t ldu, cudaStream_t s);
template <typename T>
void launch_apply_cell_down(const LevelDev& Lv, double* x, int64_t ldx, int nrhs, cudaStream_t s);
// Cell sweeps of a level whose fronts hold L^{-1} (launch_front_invert): two
// many-CTA launches per direction; tmp is a scratch column set (leading
// dimension ldu / ldt) of at least the level's DOF-list length.  Return the
// number of kernel launches.
template <typename T>
int launch_apply_big_up(const LevelDev& Lv, double* x, int64_t ldx, int nrhs, double* ubuf,
                        int64_t ldu, double* tmp, cudaStream_t s);
template <typename T>
int launch_apply_big_down(const LevelDev& Lv, double* x, int64_t ldx, int nrhs, double* tmp,
                          int64_t ldt, cudaStream_t s);
template <typename T>
void launch_apply_group_up(const LevelDev& Lv, const PhaseDev& Ph, int gather, double* x,
                           int64_t ldx, int nrhs, const double* ubuf, int64_t ldu, cudaStream_t s);
template <typename T>
void launch_apply_group_down(const LevelDev& Lv, const PhaseDev& Ph, double* x, int64_t ldx,
                             int nrhs, cudaStream_t s);
template <typename T>
int configure_apply_kernels();

int vec_blocks(int64_t N);
void launch_spmv(const GeoDev& G, const double* diag, const double* off, const double* x,
                 int64_t ldx, double* y, int64_t ldy, int nrhs, double* partial, cudaStream_t s);
void launch_dot_partial(int64_t N, const double* a, int64_t lda, const double* b, int64_t ldb,
                        int nrhs, double* partial, cudaStream_t s);
void launch_reduce(const double* partial, int nblk, int nrhs, double* sc, int mode, double rtol,
                   cudaStream_t s);
void launch_update_xr(int64_t N, int nrhs, const double* sc, double* x, int64_t ldx, double* r,
                      int64_t ldr, const double* p, int64_t ldp, const double* q, int64_t ldq,
                      double* partial, cudaStream_t s);
void launch_update_p(int64_t N, int nrhs, const double* sc, const double* z, int64_t ldz, double* p,
                     int64_t ldp, int first, cudaStream_t s);
void launch_sub(int64_t N, int nrhs, const double* a, int64_t lda, const double* b, int64_t ldb,
                double* y, int64_t ldy, cudaStream_t s);
void launch_scale(int64_t N, double* x, const double* alpha, cudaStream_t s);
void launch_pcg_kit_init(int* kit, int nrhs, int maxit, cudaStream_t s);
void launch_pcg_check(const double* sc, int nrhs, int* kit, int maxit,
                      cudaGraphConditionalHandle h, cudaStream_t s);
void launch_copy_cols(int64_t N, int nrhs, const double* a, int64_t lda, double* y, int64_t ldy,
                      cudaStream_t s);
void launch_assemble_fd(const GeoDev& G, const double* a_pix, const double* b_node, double b_const,
                        int64_t* rowptr, int32_t* col, double* val, cudaStream_t s);
void launch_exp(int64_t n, const double* x, double* y, cudaStream_t s);
void launch_grad_logcoef(const GeoDev& G, const double* a_pix, const double* u, const double* lam,
                         double* grad, cudaStream_t s);

// PCG vector kernels of a merged batch (batch_kernels.cu); S.prob etc. are
// device arrays, scalars are 8 doubles per (right-hand side, problem),
// right-hand side major
constexpr int64_t kBatchRows = 4096;   // rows of one vector block
void batch_vec_blocks(const std::vector<int64_t>& base, const std::vector<int64_t>& n,
                      std::vector<int>& prob, std::vector<int64_t>& row0,
                      std::vector<int64_t>& row1, std::vector<int>& pblk_off);
void launch_bspmv(const VecSeg& S, const BatchGeo* bg, const double* x, int64_t ldx, double* y,
                  int64_t ldy, int nrhs, double* partial, cudaStream_t s);
void launch_bdot_partial(const VecSeg& S, const double* a, int64_t lda, const double* c,
                         int64_t ldc, int nrhs, double* partial, cudaStream_t s);
void launch_breduce(const VecSeg& S, const double* partial, int nrhs, double* sc, int mode,
                    double rtol, cudaStream_t s);
void launch_bupdate_xr(const VecSeg& S, int nrhs, const double* sc, double* x, int64_t ldx,
                       double* r, int64_t ldr, const double* p, int64_t ldp, const double* q,
                       int64_t ldq, double* partial, cudaStream_t s);
void launch_bupdate_p(const VecSeg& S, int nrhs, const double* sc, const double* z, int64_t ldz,
                      double* p, int64_t ldp, int first, cudaStream_t s);
void launch_bgather(const VecSeg& S, const BatchGeo* bg, const double* const* src, double* y,
                    int64_t ldy, int nrhs, cudaStream_t s);
void launch_bscatter(const VecSeg& S, const BatchGeo* bg, const double* x, int64_t ldx,
                     double* const* dst, int nrhs, cudaStream_t s);

// FP64 leaf fallback of FP32 factors (factor_kernels.cu)
void launch_leaf_cond(const GeoDev& G, const LevelDev& Lv, const double* diag, const double* off,
                      double thresh, int* list, int* count, cudaStream_t s);
void launch_leaf_fp64_redo(const GeoDev& G, const LevelDev& Lv, const double* diag,
                           const double* off, int* status, const int* list, const int* count,
                           cudaStream_t s);

// tensor-core tile products (tc_kernels.cu)
size_t tc_tile_smem_bytes();
int configure_tc_kernels();
// kind: 0 = TF32 split in three products (about FP32), 1 = TF32, 2 = BF16
void launch_tc_gemm_check(int kind, int M, int N, int K, const float* A, int64_t lda,
                          const float* B, int64_t ldb, float* C, int64_t ldc, int* status,
                          cudaStream_t s);
// FP32 fronts: F[B,B] -= F[B,I] F[B,I]^T on the tensor cores, 128 x 64 tiles
int64_t front_schur_tc_tiles(int nI, int nB);
void launch_front_schur_tc(const LevelDev& Lv, int64_t tiles, int kind, int* status,
                           cudaStream_t s);

}  // namespace rhif
