// Host-side level plan: the quadtree/octree grouping of the active DOFs
// (Sec. 3.1, Fig. 3; Sec. 3.2) turned into flat index tables for the kernels.
//
// At level l the cells are 2^l m intervals wide.  Along each axis a node
// coordinate x maps to v = 2*(x / w) + (x % w != 0): odd v lies inside cell
// (v-1)/2, even v on the plane between cells v/2-1 and v/2.  A group is the
// set of active DOFs with equal (v0,v1,v2); its type t is the number of even
// components (0 = cell interior, 1 = edge/face, 2 = corner/3D edge, 3 = 3D
// corner).  Group members are kept in ascending DOF index.
//
// Every cell owns a dense front over [I ; B]: its interior I followed by the
// separator groups of its closure B, in group-code order.  The per-cell
// Schur complements ("frames", the B x B block after elimination) are kept
// unassembled: the level matrix is the sum over cells of their frames.
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

struct UnitTable {
  // one row per skeletonization unit (groups of type t == unit_type)
  std::vector<int> group;          // group index
  std::vector<int> nrow;           // |R|
  std::vector<int64_t> row_off;    // into row_gid (nunit + 1)
  std::vector<int64_t> row_gid;    // DOF of each row of A_{R,I}
  std::vector<int64_t> row_src_off; // per row (over all units, +1): range into src_*
  std::vector<int> src_cell, src_pos, src_upos; // frame entries summed into a row, in cell order:
                                                // cell, row position and unit offset in that cell's B
  std::vector<int64_t> m_off;      // scratch offset: M (nrow x n) then A_ee (n x n)
  int64_t m_total = 0;
  std::vector<int64_t> rec_off;    // record offset: unit front (n x n) then T (n x n)
  int64_t rec_total = 0;
  std::vector<int64_t> perm_off;   // pivot order (n ints)
  int64_t perm_total = 0;
  int max_n = 0;
};

struct PhasePlan {
  int unit_type = 1;                 // skeletonized groups: t == unit_type
  int pre_min_type = 1;              // preconditioned groups: t >= pre_min_type
  bool precondition = true;
  std::vector<int> pre_group;        // groups preconditioned in this phase
  std::vector<int64_t> pre_off;      // offset of L_g (|g|^2) in the phase's L buffer
  int64_t pre_total = 0;
  std::vector<int> group_pre;        // per group: index into pre_group or -1
  std::vector<int> group_unit;       // per group: unit index or -1
  UnitTable units;
};

struct LevelPlan {
  int level = 0, width = 0;
  // cells
  std::vector<int64_t> cell_code;
  std::vector<int> nI, nB;
  std::vector<int64_t> front_off;    // element offsets; front of cell c is n x n, n = nI + nB
  int64_t front_total = 0;
  std::vector<int64_t> gid_off;      // into gids (ncell + 1): front order, I then B
  std::vector<int64_t> gids;
  std::vector<int64_t> b_off;        // prefix sums of nB (ncell + 1)
  int max_nI = 0, max_nB = 0, max_n = 0;
  // segments of each cell's B
  std::vector<int> seg_off;          // ncell + 1
  std::vector<int> seg_group, seg_pos;
  // groups (t >= 1)
  std::vector<int64_t> group_code;
  std::vector<int> group_t;
  std::vector<int64_t> group_gid_off;   // ngroup + 1
  std::vector<int64_t> group_gids;
  std::vector<int> group_cell_off;      // ngroup + 1
  std::vector<int> group_cell, group_pos;
  int max_group = 0;
  // extend-add (level >= 1): children frames of the previous level
  std::vector<int> ea_off;           // ncell + 1
  std::vector<int> ea_child;
  std::vector<int64_t> ea_map_off;   // per child entry
  std::vector<int> ea_map;           // child B position -> parent front position, -1 = eliminated
  // preconditioning + skeletonization passes (1, or 2 with 3D edge skeletonization)
  std::vector<PhasePlan> phases;

  int ncell() const { return (int)nI.size(); }
  int ngroup() const { return (int)group_t.size(); }
};

// Build the plan of level `level` from the active DOFs (alive[g] != 0).
// `prev` is the plan of level-1 (nullptr at level 0).  For level == G.L only
// the root front is built (no phases).
LevelPlan build_level(const Geometry& G, int level, const std::vector<uint8_t>& alive,
                      const LevelPlan* prev, bool precondition, bool edge_skel);

}  // namespace rhif
