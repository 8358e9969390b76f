// Merged level plans of a batch of independent problems: one set of index
// tables per level covering the cells, groups and units of every problem, so
// that each step of the level is one launch over the whole batch.  The cells
// of different problems never share a DOF, a group or a frame (the problems
// are independent), and the cells, blocks and units of a level commute
// (Secs. 2.1-2.3), so the merged level is the union of the parts' levels.
#include <algorithm>
#include <atomic>
#include <thread>

#include "host_pool.h"
#include "plan.h"

namespace rhif {

namespace {

int64_t pad4(int64_t n) { return (n + 3) & ~int64_t(3); }

// Re-encode a code of base `from` (d digits, x first) in base `to`.
int64_t recode(int64_t code, int from, int to, int d) {
  int64_t out = 0, mul = 1;
  for (int a = 0; a < d; ++a) {
    out += mul * (code % from);
    code /= from;
    mul *= to;
  }
  return out;
}

// dst[at + i] = src[i] + add
template <class V>
void put(V& dst, size_t at, const V& src, int64_t add) {
  typename V::value_type* o = dst.data() + at;
  const typename V::value_type* in = src.data();
  const size_t n = src.size();
  for (size_t i = 0; i < n; ++i) o[i] = (typename V::value_type)(in[i] + add);
}

// prefix array of n + 1 entries: the part's entries after its leading 0,
// shifted, at dst[at + 1 ..]
template <class V>
void put_prefix(V& dst, size_t at, const V& src, int64_t add) {
  for (size_t i = 1; i < src.size(); ++i) dst[at + i] = (typename V::value_type)(src[i] + add);
}

// index of -1 stays -1
template <class V>
void put_index(V& dst, size_t at, const V& src, int add) {
  for (size_t i = 0; i < src.size(); ++i) dst[at + i] = src[i] < 0 ? -1 : src[i] + add;
}

// merged plans of freed batch handles, one per level, for the next merge of
// the same level on this thread (same sizes: no fresh pages, no zero fill)
thread_local std::vector<LevelPlan> t_merged;

// Running offsets of one part inside the merged arrays.
struct At {
  int64_t bucket = 0, cells = 0, groups = 0, segs = 0, gcells = 0, ea = 0, map = 0;
  int64_t gid = 0, b = 0, front = 0, frame = 0, band = 0, z = 0;
  int64_t pre[2] = {0, 0}, pre_total[2] = {0, 0}, units[2] = {0, 0};
  int64_t m[2] = {0, 0}, rec[2] = {0, 0}, perm[2] = {0, 0};
};

}  // namespace

void merge_plans(int d, const std::vector<const LevelPlan*>& parts,
                 const std::vector<int>& part_prob, const std::vector<int64_t>& dof_base,
                 const std::vector<int>& prev_cell_base, LevelPlan& M,
                 std::vector<PartBase>& bases) {
  const size_t np = parts.size();
  {
    const int lvl = np ? parts[0]->level : -1;
    if (lvl >= 0 && lvl < (int)t_merged.size() && !t_merged[lvl].cell_prob.empty())
      M = std::move(t_merged[lvl]);   // every entry is rewritten below
    else
      M = LevelPlan();
    M.phase_spare.clear();
  }
  bases.assign(np, PartBase());
  if (!np) return;
  int base = 1;
  size_t nph = 0;
  for (const LevelPlan* P : parts) {
    base = std::max(base, P->code_base);
    nph = std::max(nph, P->phases.size());
  }
  M.level = parts[0]->level;
  M.width = parts[0]->width;
  M.code_base = base;
  M.max_nI = M.max_nB = M.max_n = M.max_w = M.max_group = 0;
  M.phases.resize(nph);
  for (PhasePlan& Q : M.phases) {
    Q.units.max_n = 0;
    Q.units.max_m = 0;
  }
  for (size_t i = 0; i < nph; ++i)
    for (const LevelPlan* P : parts)
      if (P->phases.size() > i) {
        M.phases[i].unit_type = P->phases[i].unit_type;
        M.phases[i].pre_min_type = P->phases[i].pre_min_type;
        break;
      }
  // 1. offsets of every part (serial prefix sums over the parts)
  std::vector<At> at(np + 1);
  for (size_t p = 0; p < np; ++p) {
    const LevelPlan& P = *parts[p];
    At& a = at[p];
    At& n = at[p + 1];
    n = a;
    n.bucket += P.bucket.size();
    n.cells += P.ncell();
    n.groups += P.ngroup();
    n.segs += P.seg_group.size();
    n.gcells += P.group_cell.size();
    n.ea += P.ea_child.size();
    n.map += P.ea_map.size();
    n.gid += P.gid_off.empty() ? 0 : P.gid_off.back();
    n.b += P.b_off.empty() ? 0 : P.b_off.back();
    n.front += pad4(P.front_total);
    n.frame += pad4(P.frame_total);
    n.band += pad4(P.band_total);
    n.z += pad4(P.z_total);
    for (size_t i = 0; i < nph; ++i) {
      if (P.phases.size() <= i) continue;
      const PhasePlan& R = P.phases[i];
      n.pre[i] += R.pre_group.size();
      n.pre_total[i] += pad4(R.pre_total);
      n.units[i] += R.units.group.size();
      n.m[i] += pad4(R.units.m_total);
      n.rec[i] += pad4(R.units.rec_total);
      n.perm[i] += R.units.perm_total;
    }
    PartBase& B = bases[p];
    B.dof = dof_base[p];
    B.bucket = a.bucket;
    B.cell = (int)a.cells;
    B.group = (int)a.groups;
    for (size_t i = 0; i < nph && i < 2; ++i) {
      B.unit[i] = (int)a.units[i];
      B.perm[i] = a.perm[i];
    }
  }
  const At& T = at[np];
  M.bucket.resize(T.bucket);
  M.cell_code.resize(T.cells);
  M.cell_start.resize(T.cells);
  M.nI.resize(T.cells);
  M.nB.resize(T.cells);
  M.gid_off.resize(T.cells + 1);
  M.gid_off[0] = 0;
  M.b_off.resize(T.cells + 1);
  M.b_off[0] = 0;
  M.front_off.resize(T.cells);
  M.frame_off.resize(T.cells);
  M.frame_ld.resize(T.cells);
  const bool leaf = M.level == 0;
  if (leaf) {
    M.band_w.resize(T.cells);
    M.band_off.resize(T.cells);
    M.z_off.resize(T.cells);
  }
  M.front_total = T.front;
  M.frame_total = T.frame;
  M.band_total = T.band;
  M.z_total = T.z;
  M.seg_off.resize(T.cells + 1);
  M.seg_off[0] = 0;
  M.seg_group.resize(T.segs);
  M.seg_pos.resize(T.segs);
  M.group_code.resize(T.groups);
  M.group_t.resize(T.groups);
  M.group_start.resize(T.groups);
  M.group_size.resize(T.groups);
  M.group_cell_off.resize(T.groups + 1);
  M.group_cell_off[0] = 0;
  M.group_cell.resize(T.gcells);
  M.group_pos.resize(T.gcells);
  const bool ea = M.level > 0;
  M.ea_off.resize(T.cells + 1);
  M.ea_off[0] = 0;
  if (ea) {
    M.ea_child.resize(T.ea);
    M.ea_map_off.resize(T.ea);
    M.ea_map.resize(T.map);
  }
  M.cell_prob.resize(T.cells);
  for (size_t i = 0; i < nph; ++i) {
    PhasePlan& Q = M.phases[i];
    Q.pre_group.resize(T.pre[i]);
    Q.pre_off.resize(T.pre[i]);
    Q.pre_total = T.pre_total[i];
    Q.group_pre.resize(T.groups);
    Q.group_unit.resize(T.groups);
    UnitTable& U = Q.units;
    U.group.resize(T.units[i]);
    U.nrow.resize(T.units[i]);
    U.m_off.resize(T.units[i]);
    U.rec_off.resize(T.units[i]);
    U.perm_off.resize(T.units[i]);
    U.m_total = T.m[i];
    U.rec_total = T.rec[i];
    U.perm_total = T.perm[i];
  }
  for (const LevelPlan* P : parts) {
    M.max_nI = std::max(M.max_nI, P->max_nI);
    M.max_nB = std::max(M.max_nB, P->max_nB);
    M.max_n = std::max(M.max_n, P->max_n);
    M.max_w = std::max(M.max_w, P->max_w);
    M.max_group = std::max(M.max_group, P->max_group);
    for (size_t i = 0; i < nph && i < P->phases.size(); ++i) {
      M.phases[i].units.max_n = std::max(M.phases[i].units.max_n, P->phases[i].units.max_n);
      M.phases[i].units.max_m = std::max(M.phases[i].units.max_m, P->phases[i].units.max_m);
    }
  }
  // 2. every part fills its own ranges (parallel over the parts)
  auto fill = [&](size_t p) {
    const LevelPlan& P = *parts[p];
    const At& a = at[p];
    const int64_t bk = a.bucket, c0 = a.cells, g0 = a.groups;
    put(M.bucket, bk, P.bucket, dof_base[p]);
    for (int c = 0; c < P.ncell(); ++c)
      M.cell_code[c0 + c] = recode(P.cell_code[c], P.code_base, base, d);
    put(M.cell_start, c0, P.cell_start, bk);
    put(M.nI, c0, P.nI, 0);
    put(M.nB, c0, P.nB, 0);
    put_prefix(M.gid_off, c0, P.gid_off, a.gid);
    put_prefix(M.b_off, c0, P.b_off, a.b);
    if (leaf) {
      put(M.front_off, c0, P.front_off, 0);
      put(M.frame_off, c0, P.frame_off, a.frame);
      put(M.band_w, c0, P.band_w, 0);
      put(M.band_off, c0, P.band_off, a.band);
      put(M.z_off, c0, P.z_off, a.z);
    } else {
      put(M.front_off, c0, P.front_off, a.front);
      put(M.frame_off, c0, P.frame_off, a.front);
    }
    put(M.frame_ld, c0, P.frame_ld, 0);
    put_prefix(M.seg_off, c0, P.seg_off, a.segs);
    put(M.seg_group, a.segs, P.seg_group, g0);
    put(M.seg_pos, a.segs, P.seg_pos, 0);
    for (int g = 0; g < P.ngroup(); ++g)
      M.group_code[g0 + g] = recode(P.group_code[g], P.code_base, base, d);
    put(M.group_t, g0, P.group_t, 0);
    put(M.group_start, g0, P.group_start, bk);
    put(M.group_size, g0, P.group_size, 0);
    put_prefix(M.group_cell_off, g0, P.group_cell_off, a.gcells);
    put(M.group_cell, a.gcells, P.group_cell, c0);
    put(M.group_pos, a.gcells, P.group_pos, 0);
    if (ea && !P.ea_off.empty()) {
      put_prefix(M.ea_off, c0, P.ea_off, a.ea);
      put(M.ea_child, a.ea, P.ea_child, prev_cell_base.empty() ? 0 : prev_cell_base[p]);
      put(M.ea_map_off, a.ea, P.ea_map_off, a.map);
      put(M.ea_map, a.map, P.ea_map, 0);
    } else {
      for (int c = 1; c <= P.ncell(); ++c) M.ea_off[c0 + c] = (int)a.ea;
    }
    std::fill(M.cell_prob.begin() + c0, M.cell_prob.begin() + c0 + P.ncell(), part_prob[p]);
    for (size_t i = 0; i < nph; ++i) {
      PhasePlan& Q = M.phases[i];
      UnitTable& U = Q.units;
      if (P.phases.size() <= i) {   // root front: no groups take part
        std::fill(Q.group_pre.begin() + g0, Q.group_pre.begin() + g0 + P.ngroup(), -1);
        std::fill(Q.group_unit.begin() + g0, Q.group_unit.begin() + g0 + P.ngroup(), -1);
        continue;
      }
      const PhasePlan& R = P.phases[i];
      put(Q.pre_group, a.pre[i], R.pre_group, g0);
      put(Q.pre_off, a.pre[i], R.pre_off, a.pre_total[i]);
      put_index(Q.group_pre, g0, R.group_pre, (int)a.pre[i]);
      put_index(Q.group_unit, g0, R.group_unit, (int)a.units[i]);
      const UnitTable& V = R.units;
      put(U.group, a.units[i], V.group, g0);
      put(U.nrow, a.units[i], V.nrow, 0);
      put(U.m_off, a.units[i], V.m_off, a.m[i]);
      put(U.rec_off, a.units[i], V.rec_off, a.rec[i]);
      put(U.perm_off, a.units[i], V.perm_off, a.perm[i]);
    }
  };
  HostPool::get().parallel_for((int64_t)np, 1, [&](int64_t p0, int64_t p1) {
    for (int64_t p = p0; p < p1; ++p) fill((size_t)p);
  });
}

void recycle_merged_plan(LevelPlan&& P) {
  if (P.level < 0 || P.level >= 64 || P.cell_prob.empty()) return;
  if ((int)t_merged.size() <= P.level) t_merged.resize(P.level + 1);
  t_merged[P.level] = std::move(P);
}

}  // namespace rhif
