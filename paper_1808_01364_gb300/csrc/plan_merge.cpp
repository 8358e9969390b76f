// Merged level plans of a batch of independent problems: one set of index
// tables per level covering the cells, groups and units of every problem, so
// that each step of the level is one launch over the whole batch.  The cells
// of different problems never share a DOF, a group or a frame (the problems
// are independent), and the cells, blocks and units of a level commute
// (Secs. 2.1-2.3), so the merged level is the union of the parts' levels.
#include <algorithm>

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

template <class V, class F>
void append(V& dst, const V& src, F f) {
  const size_t n0 = dst.size();
  dst.resize(n0 + src.size());
  for (size_t i = 0; i < src.size(); ++i) dst[n0 + i] = f(src[i]);
}

template <class V>
void append_plus(V& dst, const V& src, int64_t add) {
  append(dst, src, [add](typename V::value_type v) { return (typename V::value_type)(v + add); });
}

// prefix array (n + 1 entries, dst already holding its leading 0): append
// the part's entries after its own leading 0, shifted
template <class V>
void append_prefix(V& dst, const V& src, int64_t add) {
  for (size_t i = 1; i < src.size(); ++i) dst.push_back((typename V::value_type)(src[i] + add));
}

}  // namespace

void merge_plans(int d, const std::vector<const LevelPlan*>& parts,
                 const std::vector<int>& part_prob, const std::vector<int64_t>& dof_base,
                 const std::vector<int>& prev_cell_base, LevelPlan& M,
                 std::vector<PartBase>& bases) {
  M = LevelPlan();
  bases.assign(parts.size(), PartBase());
  if (parts.empty()) return;
  int base = 1;
  for (const LevelPlan* P : parts) base = std::max(base, P->code_base);
  M.level = parts[0]->level;
  M.width = parts[0]->width;
  M.code_base = base;
  size_t nph = 0;
  for (const LevelPlan* P : parts) nph = std::max(nph, P->phases.size());
  M.phases.resize(nph);
  for (size_t i = 0; i < nph; ++i) {
    for (const LevelPlan* P : parts)
      if (P->phases.size() > i) {
        M.phases[i].unit_type = P->phases[i].unit_type;
        M.phases[i].pre_min_type = P->phases[i].pre_min_type;
        break;
      }
  }
  M.gid_off.push_back(0);
  M.b_off.push_back(0);
  M.seg_off.push_back(0);
  M.group_cell_off.push_back(0);
  M.ea_off.push_back(0);
  for (size_t p = 0; p < parts.size(); ++p) {
    const LevelPlan& P = *parts[p];
    PartBase& B = bases[p];
    B.dof = dof_base[p];
    B.bucket = (int64_t)M.bucket.size();
    B.cell = M.ncell();
    B.group = M.ngroup();
    const int64_t gid_base = M.gid_off.back(), b_base = M.b_off.back();
    const int seg_base = M.seg_off.back(), gc_base = M.group_cell_off.back();
    const int ea_base = M.ea_off.back();
    const int64_t map_base = (int64_t)M.ea_map.size();
    const int64_t front_base = M.front_total, frame_base = M.frame_total;
    const int64_t band_base = M.band_total, z_base = M.z_total;
    append_plus(M.bucket, P.bucket, B.dof);
    append(M.cell_code, P.cell_code, [&](int64_t c) { return recode(c, P.code_base, base, d); });
    append_plus(M.cell_start, P.cell_start, B.bucket);
    append_plus(M.nI, P.nI, 0);
    append_plus(M.nB, P.nB, 0);
    append_prefix(M.gid_off, P.gid_off, gid_base);
    append_prefix(M.b_off, P.b_off, b_base);
    if (M.level == 0) {
      append_plus(M.frame_off, P.frame_off, frame_base);
      append_plus(M.front_off, P.front_off, 0);
    } else {
      append_plus(M.front_off, P.front_off, front_base);
      append_plus(M.frame_off, P.frame_off, front_base);
    }
    M.front_total += pad4(P.front_total);
    M.frame_total += pad4(P.frame_total);
    append_plus(M.frame_ld, P.frame_ld, 0);
    append_plus(M.band_w, P.band_w, 0);
    append_plus(M.band_off, P.band_off, band_base);
    M.band_total += pad4(P.band_total);
    append_plus(M.z_off, P.z_off, z_base);
    M.z_total += pad4(P.z_total);
    M.max_nI = std::max(M.max_nI, P.max_nI);
    M.max_nB = std::max(M.max_nB, P.max_nB);
    M.max_n = std::max(M.max_n, P.max_n);
    M.max_w = std::max(M.max_w, P.max_w);
    append_prefix(M.seg_off, P.seg_off, seg_base);
    append_plus(M.seg_group, P.seg_group, B.group);
    append_plus(M.seg_pos, P.seg_pos, 0);
    append(M.group_code, P.group_code, [&](int64_t c) { return recode(c, P.code_base, base, d); });
    append_plus(M.group_t, P.group_t, 0);
    append_plus(M.group_start, P.group_start, B.bucket);
    append_plus(M.group_size, P.group_size, 0);
    append_prefix(M.group_cell_off, P.group_cell_off, gc_base);
    append_plus(M.group_cell, P.group_cell, B.cell);
    append_plus(M.group_pos, P.group_pos, 0);
    M.max_group = std::max(M.max_group, P.max_group);
    if (!P.ea_off.empty()) {
      append_prefix(M.ea_off, P.ea_off, ea_base);
      append_plus(M.ea_child, P.ea_child, prev_cell_base.empty() ? 0 : prev_cell_base[p]);
      append_plus(M.ea_map_off, P.ea_map_off, map_base);
      append_plus(M.ea_map, P.ea_map, 0);
    } else {
      for (int c = 0; c < P.ncell(); ++c) M.ea_off.push_back(ea_base);
    }
    M.cell_prob.insert(M.cell_prob.end(), P.ncell(), part_prob[p]);
    for (size_t i = 0; i < nph; ++i) {
      PhasePlan& Q = M.phases[i];
      UnitTable& U = Q.units;
      B.unit[i] = (int)U.group.size();
      B.perm[i] = U.perm_total;
      if (P.phases.size() <= i) {   // root front: no groups take part
        Q.group_pre.insert(Q.group_pre.end(), P.ngroup(), -1);
        Q.group_unit.insert(Q.group_unit.end(), P.ngroup(), -1);
        continue;
      }
      const PhasePlan& R = P.phases[i];
      const int pre_base = (int)Q.pre_group.size();
      append_plus(Q.pre_group, R.pre_group, B.group);
      append_plus(Q.pre_off, R.pre_off, Q.pre_total);
      Q.pre_total += pad4(R.pre_total);
      append(Q.group_pre, R.group_pre, [&](int v) { return v < 0 ? -1 : v + pre_base; });
      append(Q.group_unit, R.group_unit, [&](int v) { return v < 0 ? -1 : v + B.unit[i]; });
      const UnitTable& V = R.units;
      append_plus(U.group, V.group, B.group);
      append_plus(U.nrow, V.nrow, 0);
      append_plus(U.m_off, V.m_off, U.m_total);
      U.m_total += pad4(V.m_total);
      append_plus(U.rec_off, V.rec_off, U.rec_total);
      U.rec_total += pad4(V.rec_total);
      append_plus(U.perm_off, V.perm_off, U.perm_total);
      U.perm_total += V.perm_total;
      U.max_n = std::max(U.max_n, V.max_n);
      U.max_m = std::max(U.max_m, V.max_m);
    }
  }
}

}  // namespace rhif
