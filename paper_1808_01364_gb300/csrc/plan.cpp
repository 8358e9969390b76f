// Host-side level planner; see plan.h for the grouping rule (Sec. 3.1, 3.2).
// Work is proportional to the number of group codes and segments, plus one
// pass over the active DOFs (closed form at level 0).
#include "plan.h"

#include <algorithm>

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
  inline int64_t code_of(const Geometry& G, int64_t gid) const {
    int64_t c = 0, mul = 1;
    int64_t rem = gid;
    for (int a = 0; a < d; ++a) {
      const int x = (int)(rem % G.ns[a]) + 1;
      rem /= G.ns[a];
      c += mul * (2 * (x / width) + (x % width != 0));
      mul *= base;
    }
    return c;
  }
  // per-axis code values v(x) = 2 * (x / width) + (x % width != 0), x = 1..ns
  std::vector<int> axis_table(const Geometry& G, int a) const {
    std::vector<int> t(G.ns[a]);
    for (int x = 1; x <= G.ns[a]; ++x) t[x - 1] = 2 * (x / width) + (x % width != 0);
    return t;
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
};

// Node coordinates [lo, hi] (1-based) of axis value v at cell width w.
inline void vrange(int v, int w, int ns, int* lo, int* hi) {
  const int q = v / 2;
  if (v % 2) {
    *lo = q * w + 1;
    *hi = std::min((q + 1) * w - 1, ns);
  } else {
    *lo = q * w;
    *hi = q * w;
    if (*lo < 1 || *lo > ns) *hi = *lo - 1;
  }
}

// Element counts are padded to multiples of 4 so that every factor block
// starts on a 16-byte boundary (bulk shared-memory copies need it).
inline int64_t pad4(int64_t n) { return (n + 3) & ~int64_t(3); }

}  // namespace

int unit_row_count(const LevelPlan& P, int g) {
  int seen[kMaxRowGroups];
  int nseen = 0, rows = 0;
  for (int k = P.group_cell_off[g]; k < P.group_cell_off[g + 1]; ++k) {
    const int c = P.group_cell[k];
    for (int s = P.seg_off[c]; s < P.seg_off[c + 1]; ++s) {
      const int sg = P.seg_group[s];
      if (sg == g) continue;
      bool dup = false;
      for (int i = 0; i < nseen; ++i) dup |= seen[i] == sg;
      if (dup) continue;
      if (nseen < kMaxRowGroups) seen[nseen++] = sg;
      rows += P.group_size[sg];
    }
  }
  return rows;
}

LevelPlan build_level(const Geometry& G, int level, const std::vector<int32_t>& active,
                      const std::vector<uint8_t>& alive, const LevelPlan* prev,
                      bool precondition, bool edge_skel) {
  LevelPlan P;
  P.level = level;
  const Coder C(G, level);
  P.width = C.width;
  P.code_base = C.base;
  const int d = G.d, w = C.width;

  // 1. active DOFs sorted by (code, index)
  std::vector<int64_t> cstart(C.ncode + 1, 0);
  if (level == 0) {
    P.bucket.resize(G.N);
    int64_t pos = 0;
    const int vz1 = d == 3 ? C.base - 1 : 1, vz0 = d == 3 ? 0 : 1;
    for (int vz = vz0; vz <= vz1; ++vz) {
      int zlo = 1, zhi = 1;
      if (d == 3) vrange(vz, w, G.ns[2], &zlo, &zhi);
      for (int vy = 0; vy < C.base; ++vy) {
        int ylo, yhi;
        vrange(vy, w, G.ns[1], &ylo, &yhi);
        for (int vx = 0; vx < C.base; ++vx) {
          int xlo, xhi;
          vrange(vx, w, G.ns[0], &xlo, &xhi);
          int v[3] = {vx, vy, vz};
          cstart[C.join(v)] = pos;
          for (int z = zlo; z <= zhi; ++z)
            for (int y = ylo; y <= yhi; ++y) {
              const int64_t base = (int64_t)(y - 1) * G.ns[0] + (int64_t)(z - 1) * G.ns[0] * G.ns[1];
              for (int x = xlo; x <= xhi; ++x) P.bucket[pos++] = (int32_t)(base + x - 1);
            }
        }
      }
    }
    cstart[C.ncode] = pos;
  } else {
    std::vector<int64_t> code(active.size());
    std::vector<int64_t> cnt(C.ncode + 1, 0);
    std::vector<int> tab[3];
    for (int a = 0; a < d; ++a) tab[a] = C.axis_table(G, a);
    const int64_t n0 = G.ns[0], n01 = (int64_t)G.ns[0] * G.ns[1];
    for (size_t i = 0; i < active.size(); ++i) {
      const int64_t g = active[i];
      int64_t c;
      if (d == 2) {
        const int64_t y = g / n0;
        c = tab[0][g - y * n0] + C.base * tab[1][y];
      } else {
        const int64_t z = g / n01, r = g - z * n01, y = r / n0;
        c = tab[0][r - y * n0] + C.base * (tab[1][y] + (int64_t)C.base * tab[2][z]);
      }
      code[i] = c;
      ++cnt[c + 1];
    }
    for (int64_t c = 0; c < C.ncode; ++c) cnt[c + 1] += cnt[c];
    cstart = cnt;
    P.bucket.resize(active.size());
    for (size_t i = 0; i < active.size(); ++i) P.bucket[cnt[code[i]]++] = active[i];
    // ascending DOF index within every code
    for (int64_t c = 0; c < C.ncode; ++c)
      if (cstart[c + 1] - cstart[c] > 1)
        std::sort(P.bucket.begin() + cstart[c], P.bucket.begin() + cstart[c + 1]);
  }
  auto csize = [&](int64_t c) { return (int)(cstart[c + 1] - cstart[c]); };

  // 2. cells: every cell whose closure holds an active DOF
  std::vector<int> cell_of_code(C.ncode, -1);
  {
    std::vector<uint8_t> mark(C.ncode, 0);
    for (int64_t c = 0; c < C.ncode; ++c) {
      if (!csize(c)) continue;
      int v[3];
      C.split(c, v);
      int lo[3], hi[3];
      for (int a = 0; a < 3; ++a) {
        if (a >= d) { lo[a] = hi[a] = 1; continue; }
        if (v[a] % 2) lo[a] = hi[a] = v[a];
        else { lo[a] = v[a] - 1; hi[a] = v[a] + 1; }
      }
      for (int z = lo[2]; z <= hi[2]; z += 2)
        for (int y = lo[1]; y <= hi[1]; y += 2)
          for (int x = lo[0]; x <= hi[0]; x += 2) {
            int u[3] = {x, y, z};
            mark[C.join(u)] = 1;
          }
    }
    for (int64_t c = 0; c < C.ncode; ++c)
      if (mark[c]) {
        cell_of_code[c] = (int)P.cell_code.size();
        P.cell_code.push_back(c);
      }
  }
  const int ncell = (int)P.cell_code.size();

  // 3. groups (t >= 1) in code order
  std::vector<int> group_of_code(C.ncode, -1);
  for (int64_t c = 0; c < C.ncode; ++c) {
    if (!csize(c)) continue;
    int v[3];
    C.split(c, v);
    int t = 0;
    for (int a = 0; a < d; ++a) t += (v[a] % 2 == 0);
    if (t == 0) continue;
    group_of_code[c] = (int)P.group_t.size();
    P.group_code.push_back(c);
    P.group_t.push_back(t);
    P.group_start.push_back((int32_t)cstart[c]);
    P.group_size.push_back(csize(c));
    P.max_group = std::max(P.max_group, csize(c));
  }
  const int ngroup = (int)P.group_t.size();

  // 4. cells: interior range, separator segments, storage offsets
  P.cell_start.reserve(ncell);
  P.nI.reserve(ncell);
  P.nB.reserve(ncell);
  P.seg_off.reserve(ncell + 1);
  P.seg_off.push_back(0);
  P.gid_off.push_back(0);
  P.b_off.push_back(0);
  std::vector<int> gcount(ngroup + 1, 0);
  const int dz = d >= 3 ? 1 : 0;
  for (int ci = 0; ci < ncell; ++ci) {
    const int64_t cc = P.cell_code[ci];
    int v[3];
    C.split(cc, v);
    const int nI = csize(cc);
    int nB = 0;
    for (int oz = -dz; oz <= dz; ++oz)
      for (int oy = -1; oy <= 1; ++oy)
        for (int ox = -1; ox <= 1; ++ox) {
          if (ox == 0 && oy == 0 && oz == 0) continue;
          int u[3] = {v[0] + ox, v[1] + oy, v[2] + oz};
          const int gi = group_of_code[C.join(u)];
          if (gi < 0) continue;
          P.seg_group.push_back(gi);
          P.seg_pos.push_back(nB);
          ++gcount[gi + 1];
          nB += P.group_size[gi];
        }
    const int n = nI + nB;
    P.cell_start.push_back((int32_t)cstart[cc]);
    P.nI.push_back(nI);
    P.nB.push_back(nB);
    P.seg_off.push_back((int)P.seg_group.size());
    P.gid_off.push_back(P.gid_off.back() + n);
    P.b_off.push_back(P.b_off.back() + nB);
    if (level == 0) {
      int bw = 1;   // interior box: half bandwidth = its x extent (2D) or x*y extent (3D)
      for (int a = 0; a < d - 1; ++a) {
        int lo, hi;
        vrange(v[a], w, G.ns[a], &lo, &hi);
        bw *= std::max(hi - lo + 1, 0);
      }
      if (nI == 0) bw = 0;
      P.band_w.push_back(bw);
      P.band_off.push_back(P.band_total);
      P.band_total += pad4((int64_t)nI * (bw + 1));
      P.z_off.push_back(P.z_total);
      P.z_total += pad4((int64_t)nI * nB);
      P.frame_off.push_back(P.frame_total);
      P.frame_ld.push_back(nB);
      P.frame_total += pad4((int64_t)nB * nB);
      P.front_off.push_back(0);
      P.max_w = std::max(P.max_w, bw);
    } else {
      P.front_off.push_back(P.front_total);
      P.frame_off.push_back(P.front_total + nI + (int64_t)nI * n);
      P.frame_ld.push_back(n);
      P.front_total += pad4((int64_t)n * n);
    }
    P.max_nI = std::max(P.max_nI, nI);
    P.max_nB = std::max(P.max_nB, nB);
    P.max_n = std::max(P.max_n, n);
  }
  for (int gi = 0; gi < ngroup; ++gi) gcount[gi + 1] += gcount[gi];
  P.group_cell_off.assign(gcount.begin(), gcount.end());
  P.group_cell.resize(gcount[ngroup]);
  P.group_pos.resize(gcount[ngroup]);
  {
    std::vector<int> fill(gcount.begin(), gcount.end() - 1);
    for (int ci = 0; ci < ncell; ++ci)
      for (int s = P.seg_off[ci]; s < P.seg_off[ci + 1]; ++s) {
        const int gi = P.seg_group[s];
        P.group_cell[fill[gi]] = ci;
        P.group_pos[fill[gi]] = P.seg_pos[s];
        ++fill[gi];
      }
  }

  // 5. extend-add maps from the previous level's frames
  if (prev) {
    const Coder Cp(G, level - 1);
    std::vector<int> prev_cell_of_code(Cp.ncode, -1);
    for (int i = 0; i < prev->ncell(); ++i) prev_cell_of_code[prev->cell_code[i]] = i;
    // DOF -> front position, all -1 between cells (thread-local, reused by later calls)
    static thread_local std::vector<int> pos_scratch;
    if ((int64_t)pos_scratch.size() < G.N) pos_scratch.assign(G.N, -1);
    std::vector<int>& pos_of_gid = pos_scratch;
    P.ea_off.push_back(0);
    for (int ci = 0; ci < ncell; ++ci) {
      const int nI = P.nI[ci];
      for (int i = 0; i < nI; ++i) pos_of_gid[P.bucket[P.cell_start[ci] + i]] = i;
      for (int s = P.seg_off[ci]; s < P.seg_off[ci + 1]; ++s) {
        const int g = P.seg_group[s];
        for (int o = 0; o < P.group_size[g]; ++o)
          pos_of_gid[P.bucket[P.group_start[g] + o]] = nI + P.seg_pos[s] + o;
      }
      int v[3];
      C.split(P.cell_code[ci], v);
      int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
      for (int a = 0; a < d; ++a) {
        lo[a] = v[a] - 1;          // child cell indices 2p and 2p+1 of parent p = (v-1)/2
        hi[a] = v[a];
      }
      for (int z = lo[2]; z <= hi[2]; ++z)
        for (int y = lo[1]; y <= hi[1]; ++y)
          for (int x = lo[0]; x <= hi[0]; ++x) {
            int u[3] = {2 * x + 1, 2 * y + 1, 2 * z + 1};
            const int pc = prev_cell_of_code[Cp.join(u)];
            if (pc < 0) continue;
            P.ea_child.push_back(pc);
            P.ea_map_off.push_back((int64_t)P.ea_map.size());
            const size_t base = P.ea_map.size();
            P.ea_map.resize(base + prev->nB[pc], -1);
            for (int s = prev->seg_off[pc]; s < prev->seg_off[pc + 1]; ++s) {
              const int g = prev->seg_group[s];
              const int pos = prev->seg_pos[s];
              for (int o = 0; o < prev->group_size[g]; ++o) {
                const int32_t gid = prev->bucket[prev->group_start[g] + o];
                P.ea_map[base + pos + o] = alive[gid] ? pos_of_gid[gid] : -1;
              }
            }
          }
      P.ea_off.push_back((int)P.ea_child.size());
      for (int i = 0; i < nI; ++i) pos_of_gid[P.bucket[P.cell_start[ci] + i]] = -1;
      for (int s = P.seg_off[ci]; s < P.seg_off[ci + 1]; ++s) {
        const int g = P.seg_group[s];
        for (int o = 0; o < P.group_size[g]; ++o) pos_of_gid[P.bucket[P.group_start[g] + o]] = -1;
      }
    }
  }

  if (level >= G.L) return P;   // root front only

  // 6. preconditioning + skeletonization passes
  const int npass = (d == 3 && edge_skel) ? 2 : 1;
  for (int pass = 0; pass < npass; ++pass) {
    PhasePlan ph;
    ph.unit_type = pass == 0 ? 1 : 2;
    ph.pre_min_type = pass == 0 ? 1 : 2;
    ph.group_pre.assign(ngroup, -1);
    ph.group_unit.assign(ngroup, -1);
    UnitTable& U = ph.units;
    for (int gi = 0; gi < ngroup; ++gi) {
      const int sz = P.group_size[gi];
      if (precondition && P.group_t[gi] >= ph.pre_min_type) {
        ph.group_pre[gi] = (int)ph.pre_group.size();
        ph.pre_group.push_back(gi);
        ph.pre_off.push_back(ph.pre_total);
        ph.pre_total += pad4((int64_t)sz * sz);
      }
      if (P.group_t[gi] == ph.unit_type) {
        ph.group_unit[gi] = (int)U.group.size();
        U.group.push_back(gi);
        const int nrow = unit_row_count(P, gi);
        U.nrow.push_back(nrow);
        U.m_off.push_back(U.m_total);
        U.m_total += (int64_t)(nrow + sz) * sz;
        U.max_m = std::max<int64_t>(U.max_m, (int64_t)(nrow + sz) * sz);
        U.rec_off.push_back(U.rec_total);
        U.rec_total += 2 * pad4((int64_t)sz * sz);
        U.perm_off.push_back(U.perm_total);
        U.perm_total += sz;
        U.max_n = std::max(U.max_n, sz);
      }
    }
    P.phases.push_back(std::move(ph));
  }
  return P;
}

}  // namespace rhif
