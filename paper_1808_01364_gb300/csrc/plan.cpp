// Host-side level planner; see plan.h for the grouping rule (Sec. 3.1, 3.2).
#include "plan.h"

#include <algorithm>
#include <stdexcept>

namespace rhif {

Geometry make_geometry(int d, const int* ns, int leaf) {
  Geometry G;
  G.d = d;
  G.leaf = leaf;
  int need = 0;
  G.N = 1;
  for (int a = 0; a < 3; ++a) {
    G.ns[a] = a < d ? ns[a] : 1;
    if (a < d) need = std::max(need, ns[a] + 1);
  }
  for (int a = 0; a < d; ++a) G.N *= G.ns[a];
  G.stride[0] = 1;
  G.stride[1] = G.ns[0];
  G.stride[2] = (int64_t)G.ns[0] * G.ns[1];
  int L = 0;
  while ((int64_t)leaf << L < need) ++L;
  G.L = L;
  return G;
}

namespace {

struct Coder {
  int d, width, base;
  int64_t ncode;
  Coder(const Geometry& G, int level) : d(G.d) {
    width = G.leaf << level;
    const int nc = 1 << (G.L - level);   // cells per axis of the padded tree
    base = 2 * nc + 1;
    ncode = 1;
    for (int a = 0; a < d; ++a) ncode *= base;
  }
  // code of a DOF and its type
  inline int64_t code_of(const Geometry& G, int64_t gid, int* t) const {
    int64_t c = 0, mul = 1;
    int tt = 0;
    int64_t rem = gid;
    for (int a = 0; a < d; ++a) {
      const int x = (int)(rem % G.ns[a]) + 1;
      rem /= G.ns[a];
      const int v = 2 * (x / width) + (x % width != 0);
      tt += (v % 2 == 0);
      c += mul * v;
      mul *= base;
    }
    *t = tt;
    return c;
  }
  inline void split(int64_t code, int v[3]) const {
    for (int a = 0; a < 3; ++a) v[a] = 1;
    for (int a = 0; a < d; ++a) {
      v[a] = (int)(code % base);
      code /= base;
    }
  }
  inline int64_t join(const int v[3]) const {
    int64_t c = 0, mul = 1;
    for (int a = 0; a < d; ++a) {
      c += mul * v[a];
      mul *= base;
    }
    return c;
  }
  inline int type_of(int64_t code) const {
    int v[3];
    split(code, v);
    int t = 0;
    for (int a = 0; a < d; ++a) t += (v[a] % 2 == 0);
    return t;
  }
};

}  // namespace

LevelPlan build_level(const Geometry& G, int level, const std::vector<uint8_t>& alive,
                      const LevelPlan* prev, bool precondition, bool edge_skel) {
  LevelPlan P;
  P.level = level;
  Coder C(G, level);
  P.width = C.width;
  const int d = G.d;

  // bucket the active DOFs by group code (ascending DOF index inside a bucket)
  std::vector<int64_t> count(C.ncode + 1, 0);
  std::vector<int64_t> codes;
  std::vector<int64_t> act;
  act.reserve(G.N);
  for (int64_t g = 0; g < G.N; ++g)
    if (alive[g]) act.push_back(g);
  codes.resize(act.size());
  for (size_t i = 0; i < act.size(); ++i) {
    int t;
    codes[i] = C.code_of(G, act[i], &t);
    ++count[codes[i] + 1];
  }
  for (int64_t c = 0; c < C.ncode; ++c) count[c + 1] += count[c];
  std::vector<int64_t> bucket(act.size());
  {
    std::vector<int64_t> fill(count.begin(), count.end() - 1);
    for (size_t i = 0; i < act.size(); ++i) bucket[fill[codes[i]]++] = act[i];
  }
  auto bsize = [&](int64_t c) { return count[c + 1] - count[c]; };

  // cells: every cell whose closure holds an active DOF
  std::vector<int> cell_of_code(C.ncode, -1);
  {
    std::vector<uint8_t> mark(C.ncode, 0);
    for (int64_t c = 0; c < C.ncode; ++c) {
      if (!bsize(c)) continue;
      int v[3];
      C.split(c, v);
      // cells containing this group: odd v -> itself; even v -> v-1 and v+1
      int lo[3], hi[3];
      for (int a = 0; a < 3; ++a) {
        if (a >= d) { lo[a] = hi[a] = 1; continue; }
        if (v[a] % 2) lo[a] = hi[a] = v[a];
        else { lo[a] = v[a] - 1; hi[a] = v[a] + 1; }
      }
      for (int z = lo[2]; z <= hi[2]; z += 2)
        for (int y = lo[1]; y <= hi[1]; y += 2)
          for (int x = lo[0]; x <= hi[0]; x += 2) {
            int w[3] = {x, y, z};
            mark[C.join(w)] = 1;
          }
    }
    for (int64_t c = 0; c < C.ncode; ++c)
      if (mark[c]) {
        cell_of_code[c] = (int)P.cell_code.size();
        P.cell_code.push_back(c);
      }
  }
  const int ncell = (int)P.cell_code.size();

  // groups (t >= 1) in code order
  std::vector<int> group_of_code(C.ncode, -1);
  P.group_gid_off.push_back(0);
  for (int64_t c = 0; c < C.ncode; ++c) {
    if (!bsize(c)) continue;
    const int t = C.type_of(c);
    if (t == 0) continue;
    group_of_code[c] = (int)P.group_t.size();
    P.group_code.push_back(c);
    P.group_t.push_back(t);
    for (int64_t i = count[c]; i < count[c + 1]; ++i) P.group_gids.push_back(bucket[i]);
    P.group_gid_off.push_back((int64_t)P.group_gids.size());
    P.max_group = std::max<int>(P.max_group, (int)bsize(c));
  }
  const int ngroup = (int)P.group_t.size();
  std::vector<std::vector<std::pair<int, int>>> gcells(ngroup);

  // fronts: I then the separator groups of the closure, in code order
  P.gid_off.push_back(0);
  P.b_off.push_back(0);
  P.seg_off.push_back(0);
  int64_t foff = 0;
  for (int ci = 0; ci < ncell; ++ci) {
    const int64_t cc = P.cell_code[ci];
    int v[3];
    C.split(cc, v);
    const int nI = (int)bsize(cc);
    for (int64_t i = count[cc]; i < count[cc + 1]; ++i) P.gids.push_back(bucket[i]);
    int nB = 0;
    int dz = d >= 3 ? 1 : 0, dy = d >= 2 ? 1 : 0;
    for (int oz = -dz; oz <= dz; ++oz)
      for (int oy = -dy; oy <= dy; ++oy)
        for (int ox = -1; ox <= 1; ++ox) {
          if (ox == 0 && oy == 0 && oz == 0) continue;
          int w[3] = {v[0] + ox, v[1] + oy, v[2] + oz};
          const int64_t gc = C.join(w);
          const int gi = group_of_code[gc];
          if (gi < 0) continue;
          P.seg_group.push_back(gi);
          P.seg_pos.push_back(nB);
          gcells[gi].push_back({ci, nB});
          for (int64_t i = count[gc]; i < count[gc + 1]; ++i) P.gids.push_back(bucket[i]);
          nB += (int)bsize(gc);
        }
    P.nI.push_back(nI);
    P.nB.push_back(nB);
    const int n = nI + nB;
    P.front_off.push_back(foff);
    foff += (int64_t)n * n;
    P.gid_off.push_back((int64_t)P.gids.size());
    P.b_off.push_back(P.b_off.back() + nB);
    P.seg_off.push_back((int)P.seg_group.size());
    P.max_nI = std::max(P.max_nI, nI);
    P.max_nB = std::max(P.max_nB, nB);
    P.max_n = std::max(P.max_n, n);
  }
  P.front_total = foff;
  P.group_cell_off.push_back(0);
  for (int gi = 0; gi < ngroup; ++gi) {
    for (auto& pr : gcells[gi]) {
      P.group_cell.push_back(pr.first);
      P.group_pos.push_back(pr.second);
    }
    P.group_cell_off.push_back((int)P.group_cell.size());
  }

  // extend-add maps from the previous level's frames
  if (prev) {
    Coder Cp(G, level - 1);
    std::vector<int> prev_cell_of_code(Cp.ncode, -1);
    for (int i = 0; i < prev->ncell(); ++i) prev_cell_of_code[prev->cell_code[i]] = i;
    std::vector<int> pos_of_gid(G.N, -1);
    P.ea_off.push_back(0);
    for (int ci = 0; ci < ncell; ++ci) {
      const int64_t b = P.gid_off[ci], e = P.gid_off[ci + 1];
      for (int64_t i = b; i < e; ++i) pos_of_gid[P.gids[i]] = (int)(i - b);
      int v[3];
      C.split(P.cell_code[ci], v);
      int lo[3], hi[3];
      for (int a = 0; a < 3; ++a) {
        const int cidx = (v[a] - 1) / 2;
        if (a >= d) { lo[a] = hi[a] = 0; continue; }
        lo[a] = 2 * cidx;
        hi[a] = 2 * cidx + 1;
      }
      for (int z = lo[2]; z <= hi[2]; ++z)
        for (int y = lo[1]; y <= hi[1]; ++y)
          for (int x = lo[0]; x <= hi[0]; ++x) {
            int w[3] = {2 * x + 1, 2 * y + 1, 2 * z + 1};
            if (d < 3) w[2] = 1;
            if (d < 2) w[1] = 1;
            const int pc = prev_cell_of_code[Cp.join(w)];
            if (pc < 0) continue;
            P.ea_child.push_back(pc);
            P.ea_map_off.push_back((int64_t)P.ea_map.size());
            const int64_t pb = prev->gid_off[pc] + prev->nI[pc];
            for (int j = 0; j < prev->nB[pc]; ++j) {
              const int64_t g = prev->gids[pb + j];
              P.ea_map.push_back(alive[g] ? pos_of_gid[g] : -1);
            }
          }
      P.ea_off.push_back((int)P.ea_child.size());
      for (int64_t i = b; i < e; ++i) pos_of_gid[P.gids[i]] = -1;
    }
  }

  if (level >= G.L) return P;   // root front only

  // preconditioning + skeletonization passes
  const int npass = (d == 3 && edge_skel) ? 2 : 1;
  std::vector<int> row_of_gid(G.N, -1);
  for (int pass = 0; pass < npass; ++pass) {
    PhasePlan ph;
    ph.unit_type = pass == 0 ? 1 : 2;
    ph.pre_min_type = pass == 0 ? 1 : 2;
    ph.precondition = precondition;
    ph.group_pre.assign(ngroup, -1);
    ph.group_unit.assign(ngroup, -1);
    for (int gi = 0; gi < ngroup; ++gi) {
      const int sz = (int)(P.group_gid_off[gi + 1] - P.group_gid_off[gi]);
      if (precondition && P.group_t[gi] >= ph.pre_min_type) {
        ph.group_pre[gi] = (int)ph.pre_group.size();
        ph.pre_group.push_back(gi);
        ph.pre_off.push_back(ph.pre_total);
        ph.pre_total += (int64_t)sz * sz;
      }
    }
    UnitTable& U = ph.units;
    U.row_off.push_back(0);
    U.row_src_off.push_back(0);
    std::vector<std::vector<int>> rsrc;   // per row of the current unit: (cell, pos, upos) triples
    for (int gi = 0; gi < ngroup; ++gi) {
      if (P.group_t[gi] != ph.unit_type) continue;
      const int n = (int)(P.group_gid_off[gi + 1] - P.group_gid_off[gi]);
      ph.group_unit[gi] = (int)U.group.size();
      U.group.push_back(gi);
      int nrow = 0;
      const int64_t row_base = (int64_t)U.row_gid.size();
      rsrc.clear();
      for (int k = P.group_cell_off[gi]; k < P.group_cell_off[gi + 1]; ++k) {
        const int ci = P.group_cell[k];
        const int upos = P.group_pos[k];
        for (int s = P.seg_off[ci]; s < P.seg_off[ci + 1]; ++s) {
          const int sg = P.seg_group[s];
          if (sg == gi) continue;
          const int spos = P.seg_pos[s];
          const int64_t g0 = P.group_gid_off[sg];
          const int ssz = (int)(P.group_gid_off[sg + 1] - g0);
          for (int j = 0; j < ssz; ++j) {
            const int64_t g = P.group_gids[g0 + j];
            int r = row_of_gid[g];
            if (r < 0) {
              r = row_of_gid[g] = nrow++;
              U.row_gid.push_back(g);
              rsrc.emplace_back();
            }
            rsrc[r].push_back(ci);
            rsrc[r].push_back(spos + j);
            rsrc[r].push_back(upos);
          }
        }
      }
      for (int r = 0; r < nrow; ++r) {
        for (size_t q = 0; q < rsrc[r].size(); q += 3) {
          U.src_cell.push_back(rsrc[r][q]);
          U.src_pos.push_back(rsrc[r][q + 1]);
          U.src_upos.push_back(rsrc[r][q + 2]);
        }
        U.row_src_off.push_back((int64_t)U.src_cell.size());
      }
      for (int64_t i = row_base; i < (int64_t)U.row_gid.size(); ++i) row_of_gid[U.row_gid[i]] = -1;
      U.nrow.push_back(nrow);
      U.row_off.push_back((int64_t)U.row_gid.size());
      U.m_off.push_back(U.m_total);
      U.m_total += (int64_t)(nrow + n) * n;
      U.rec_off.push_back(U.rec_total);
      U.rec_total += 2 * (int64_t)n * n;
      U.perm_off.push_back(U.perm_total);
      U.perm_total += n;
      U.max_n = std::max(U.max_n, n);
    }
    P.phases.push_back(std::move(ph));
  }
  return P;
}

}  // namespace rhif
