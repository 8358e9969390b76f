// Host-side level plan: the quadtree/octree grouping of the active DOFs
// (Sec. 3.1, Fig. 3; Sec. 3.2) turned into flat index tables for the kernels.
//
// At level l the cells are w = 2^l m intervals wide.  Along each axis a node
// coordinate x maps to v = 2*(x / w) + (x % w != 0): odd v lies inside cell
// (v-1)/2, even v on the plane between cells v/2-1 and v/2.  A group is the
// set of active DOFs with equal (v0,v1,v2) ("code"); its type t is the number
// of even components (0 = cell interior, 1 = edge/face, 2 = corner/3D edge,
// 3 = 3D corner).  All active DOFs are stored once, sorted by code and, inside
// a code, by ascending DOF index (the `bucket` array); cells and groups are
// ranges of it.
//
// Every cell owns a front over [I ; B]: its interior I followed by the
// separator groups of its closure (its "segments"), in code order.  The per-cell
// Schur complements ("frames", the B x B block after elimination) are kept
// unassembled: the level matrix is the sum over cells of their frames.
// Level 0 eliminates I with a banded Cholesky straight from the stencil and
// writes only the frames; levels >= 1 assemble dense fronts from the children's
// frames (extend-add).
#pragma once
#include <cstdint>
#include <vector>

namespace rhif {

struct Geometry {
  int d = 2;
  int ns[3] = {1, 1, 1};
  int64_t N = 0;
  int leaf = 8;
  int L = 0;             // number of levels; the root front is level L
  int64_t stride[3] = {1, 1, 1};
};

Geometry make_geometry(int d, const int* ns, int leaf);

// Largest number of distinct row groups of one skeletonization unit (see unit_rows).
constexpr int kMaxRowGroups = 128;
constexpr int kMaxSlots = 4;

struct UnitTable {
  std::vector<int> group;          // group index of each unit (groups of type t == unit_type)
  std::vector<int> nrow;           // |R|
  std::vector<int64_t> m_off;      // scratch: M (nrow x n) then A_ee (n x n)
  int64_t m_total = 0;
  std::vector<int64_t> rec_off;    // record: unit front (n x n, padded to 4) then T (k x (n-k))
  int64_t rec_total = 0;
  std::vector<int64_t> perm_off;   // pivot order (n ints)
  int64_t perm_total = 0;
  int max_n = 0;
  int64_t max_m = 0;               // largest (nrow + n) * n of the phase
};

struct PhasePlan {
  int unit_type = 1;                 // skeletonized groups: t == unit_type
  int pre_min_type = 1;              // preconditioned groups: t >= pre_min_type
  std::vector<int> pre_group;        // groups preconditioned in this phase
  std::vector<int64_t> pre_off;      // offset of L_g (|g|^2) in the phase's L buffer
  int64_t pre_total = 0;
  std::vector<int> group_pre;        // per group: index into pre_group or -1
  std::vector<int> group_unit;       // per group: unit index or -1
  UnitTable units;
  // Empties every table but keeps the storage.
  void clear();
};

struct LevelPlan {
  int level = 0, width = 0, code_base = 0;
  std::vector<int32_t> bucket;       // active DOFs sorted by (code, index)
  // cells
  std::vector<int64_t> cell_code;
  std::vector<int32_t> cell_start;   // bucket offset of the interior
  std::vector<int> nI, nB;
  std::vector<int64_t> gid_off;      // front-order DOF list offsets (ncell + 1), expanded on the device
  std::vector<int64_t> b_off;        // prefix sums of nB (ncell + 1)
  std::vector<int64_t> front_off;    // level >= 1: dense n x n front
  int64_t front_total = 0;
  std::vector<int64_t> frame_off;    // B x B frame (level 0: own buffer; else inside the front)
  std::vector<int> frame_ld;
  int64_t frame_total = 0;           // level 0 frame buffer size
  // level 0: banded leaf factors
  std::vector<int> band_w;           // half bandwidth of the interior block
  std::vector<int64_t> band_off;     // nI x (w+1) band of L
  int64_t band_total = 0;
  std::vector<int64_t> z_off;        // scratch nI x nB for L^{-1} A_IB
  int64_t z_total = 0;
  int max_nI = 0, max_nB = 0, max_n = 0, max_w = 0;
  // segments of each cell's B
  std::vector<int> seg_off;          // ncell + 1
  std::vector<int> seg_group, seg_pos;
  // groups (t >= 1)
  std::vector<int64_t> group_code;
  std::vector<int> group_t;
  std::vector<int32_t> group_start;  // bucket offset
  std::vector<int> group_size;
  std::vector<int> group_cell_off;   // ngroup + 1
  std::vector<int> group_cell, group_pos;
  int max_group = 0;
  // extend-add (level >= 1): children frames of the previous level
  std::vector<int> ea_off;           // ncell + 1
  std::vector<int> ea_child;
  std::vector<int64_t> ea_map_off;   // per child entry
  std::vector<int> ea_map;           // child B position -> parent front position, -1 = eliminated
  // batches (merge_plans): problem of each cell; empty for a single problem
  std::vector<int> cell_prob;
  // preconditioning + skeletonization passes (1, or 2 with 3D edge skeletonization)
  std::vector<PhasePlan> phases;
  std::vector<PhasePlan> phase_spare;   // storage of cleared phases, reused by build_level

  int ncell() const { return (int)nI.size(); }
  int ngroup() const { return (int)group_t.size(); }
  // Empties every table but keeps the storage (every field is listed here).
  void clear();
};

// Hands a plan that is no longer needed back to the calling thread's pool: the
// next build_level of the same level on that thread reuses its storage, so a
// refactorization of the same geometry touches no fresh pages.  The pool
// holds at most one plan per level.
void recycle_plan(LevelPlan&& P);

// Build the plan of level `level`.  At level 0 every DOF is active; above it
// the active DOFs are those of the previous level's separator groups whose
// flag in `keep` is set (indexed by position in prev->bucket; only the group
// ranges are read).  `prev` is the plan of level-1.  For level == G.L only the
// root front is built (no phases).
LevelPlan build_level(const Geometry& G, int level, const std::vector<uint8_t>& keep,
                      const LevelPlan* prev,
                      bool precondition, bool edge_skel);

// Offsets of one problem's part inside a merged plan (merge_plans).
struct PartBase {
  int64_t dof = 0;      // first DOF of the problem in the concatenated numbering
  int64_t bucket = 0;   // first bucket position
  int cell = 0, group = 0;
  int unit[2] = {0, 0};   // first unit of each phase
  int64_t perm[2] = {0, 0};
};

// Concatenate the plans of one level of several independent d-dimensional problems into
// one plan whose cells, groups and units are those of every part, in part
// order: every index is shifted by the part's base, DOF numbers by dof_base,
// storage offsets by the running totals, and cell/group codes re-encoded
// with the largest code base (codes are per-problem coordinates; only the
// cells' codes are read on the device).  prev_cell_base[p] is the first cell
// of part p in the merged plan of the previous level (extend-add children).
// A part whose plan is its root front (no phases) contributes no units.
// Writes each part's bases to `bases` and its problem index to cell_prob.
void merge_plans(int d, const std::vector<const LevelPlan*>& parts,
                 const std::vector<int>& part_prob, const std::vector<int64_t>& dof_base,
                 const std::vector<int>& prev_cell_base, LevelPlan& out,
                 std::vector<PartBase>& bases);

// Hands a merged plan that is no longer needed to the calling thread's pool
// of merged plans (one per level), reused by the next merge_plans of that level.
void recycle_merged_plan(LevelPlan&& P);

// Row layout of A_{R,I} for a unit: the distinct separator groups other than
// the unit itself, over the cells holding the unit in cell order, each cell's
// segments in code order; a group met again in a later cell is not repeated
// (its entries from every holding cell are summed into the same rows).
// Returns the number of rows.
int unit_row_count(const LevelPlan& P, int group);

}  // namespace rhif
