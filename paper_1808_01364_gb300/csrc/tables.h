// Device views of one level plan (see plan.h), passed by value to kernels.
#pragma once
#include <cstdint>

namespace rhif {

constexpr int kMaxRowGroupsDev = 128;   // = kMaxRowGroups of plan.h
constexpr int kMaxSlotsDev = 4;
// Leaf bands with half bandwidth w <= kBandInvW store the explicit inverse of
// every diagonal w x w block in the block's in-band slots (see
// k_band_block_inverse and the leaf application).
constexpr int kBandInvW = 15;

struct GeoDev {
  int d, leaf;
  int ns[3];
  int64_t N;
  int64_t stride[3];
};

// One problem of a merged batch: its grid, the first of its DOFs in the
// concatenated numbering, and its stencil form (diagonal; forward-edge
// weights, d x N_p, axis-major).
struct BatchGeo {
  GeoDev G;
  int64_t base;
  const double* diag;
  const double* off;
};

// Vector blocks of a merged batch: block b covers rows [row0[b], row1[b]) of
// problem prob[b] in the concatenated numbering; problem p owns blocks
// pblk_off[p] .. pblk_off[p+1]-1.
struct VecSeg {
  int nblk, nprob;
  const int* prob;
  const int64_t* row0;
  const int64_t* row1;
  const int* pblk_off;
};

struct LevelDev {
  int level, ncell, ngroup;
  int width, code_base;      // cell width in grid intervals; base of the group code
  int max_nI, max_nB, max_n, max_group, max_w;
  const int32_t* bucket;     // active DOFs sorted by (code, index)
  const int64_t* cell_code;
  const int32_t* cell_start;
  const int* nI;
  const int* nB;
  const int64_t* gid_off;
  int32_t* gids;             // front-order DOF lists, expanded on the device
  const int64_t* b_off;
  const int64_t* front_off;  // level >= 1
  void* front;
  const int64_t* frame_off;
  const int* frame_ld;
  void* frame_base;          // level 0: frame buffer; level >= 1: == front
  // level 0 banded factors
  const int* band_w;
  const int64_t* band_off;
  void* band;                // nI x (w+1), column k holds L[k..k+w, k]
  const int64_t* z_off;
  void* zbuf;                // factorization scratch
  int* cpl_i;                // per B position (b_off): coupled interior index or -1
  void* cpl_a;               // per B position: A(b, I(b))
  // segments
  const int* seg_off;
  const int* seg_group;
  const int* seg_pos;
  // groups
  const int* group_t;
  const int32_t* group_start;
  const int* group_size;
  const int* group_cell_off;
  const int* group_cell;
  const int* group_pos;
  // extend-add
  const int* ea_off;
  const int* ea_child;
  const int64_t* ea_map_off;
  const int* ea_map;
  int* status;               // error word of the handle (timeouts of bulk copies)
  // merged batches: problem of each cell and the problems' grids (null for a
  // single problem: the kernels' GeoDev and stencil arguments apply)
  const int* cell_prob;
  const BatchGeo* bgeo;
};

struct PhaseDev {
  int unit_type, pre_min_type;
  int npre;
  int diag_only;            // diagonal local preconditioner: L_g = diag(A_gg)^{1/2}
  const int* pre_group;
  const int64_t* pre_off;
  const int* group_pre;    // per group of the level: index into pre_group or -1
  void* Lbuf;
  void* Linv;              // explicit L_g^{-1} (same layout as Lbuf) while scaling, else null
  const int* scale_task;   // (cell, segment) pairs of the tile-product scaling
  const int64_t* scale_off;  // prefix sums of their 64-wide column / row blocks
  int nscale_task;
  int nunit, max_n;
  const int* u_group;
  const int* u_nrow;
  const int64_t* u_m_off;
  void* Mbuf;
  const int64_t* u_rec_off;
  void* rec;
  const int64_t* u_perm_off;
  int* perm;
  int* rank;
  const int* group_unit;   // per group of the level: unit index or -1
};

}  // namespace rhif
