// Host-side level planner; see plan.h for the grouping rule (Sec. 3.1, 3.2).
// Work is proportional to the number of group codes and segments, plus one
// pass over the DOFs of the previous level's separator groups (closed form at
// level 0).
#include "plan.h"

#include <algorithm>

#include "host_pool.h"

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

void LevelPlan::clear() {
  level = width = code_base = 0;
  // bucket and ea_map keep their sizes: build_level rewrites every entry, so a
  // recycled plan of the same size is not zero-filled first
  bucket.resize(bucket.size());
  cell_code.clear();
  cell_start.clear();
  nI.clear();
  nB.clear();
  gid_off.clear();
  b_off.clear();
  front_off.clear();
  front_total = 0;
  frame_off.clear();
  frame_ld.clear();
  frame_total = 0;
  band_w.clear();
  band_off.clear();
  band_total = 0;
  z_off.clear();
  z_total = 0;
  max_nI = max_nB = max_n = max_w = 0;
  seg_off.clear();
  seg_group.clear();
  seg_pos.clear();
  group_code.clear();
  group_t.clear();
  group_start.clear();
  group_size.clear();
  group_cell_off.clear();
  group_cell.clear();
  group_pos.clear();
  max_group = 0;
  ea_off.clear();
  ea_child.clear();
  ea_map_off.clear();
  cell_prob.clear();
  for (auto& ph : phases) phase_spare.push_back(std::move(ph));   // keeps their storage
  phases.clear();
}

void PhasePlan::clear() {
  unit_type = pre_min_type = 1;
  pre_group.clear();
  pre_off.clear();
  pre_total = 0;
  group_pre.clear();
  group_unit.clear();
  UnitTable& U = units;
  U.group.clear();
  U.nrow.clear();
  U.m_off.clear();
  U.m_total = 0;
  U.rec_off.clear();
  U.rec_total = 0;
  U.perm_off.clear();
  U.perm_total = 0;
  U.max_n = 0;
  U.max_m = 0;
}

namespace {
// per-thread storage reused across calls: recycled plans (one per level) and
// the planner's temporaries
struct PlanScratch {
  std::vector<LevelPlan> pool;
  std::vector<int64_t> cstart, cnt, gcode;
  std::vector<int> gpos_off, newpos, src, cell_of_code, group_of_code, prev_cell_of_code;
  std::vector<int> gna, cg, cgoff, nseg, nrow;
  std::vector<uint8_t> mark;
};
thread_local PlanScratch t_scratch;
}  // namespace

void recycle_plan(LevelPlan&& P) {
  auto& pool = t_scratch.pool;
  if (P.level < 0 || P.level >= 64) return;
  if ((int)pool.size() <= P.level) pool.resize(P.level + 1);
  pool[P.level] = std::move(P);
}

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

LevelPlan build_level(const Geometry& G, int level, const std::vector<uint8_t>& keep, const LevelPlan* prev,
                      bool precondition, bool edge_skel) {
  PlanScratch& X = t_scratch;
  LevelPlan P;
  if (level < (int)X.pool.size()) {
    P = std::move(X.pool[level]);
    X.pool[level] = LevelPlan();
    P.clear();
  }
  P.level = level;
  const Coder C(G, level);
  P.width = C.width;
  P.code_base = C.base;
  const int d = G.d, w = C.width;

  // 1. active DOFs sorted by (code, index); for level >= 1 also, per
  // separator group of level - 1, its code here (gcode) and, per DOF of those
  // groups (numbered group by group, gpos_off), its bucket position or -1
  std::vector<int64_t>& cstart = X.cstart;
  cstart.assign(C.ncode + 1, 0);
  std::vector<int64_t>& gcode = X.gcode;
  std::vector<int>& gpos_off = X.gpos_off;
  std::vector<int>& newpos = X.newpos;
  HostPool& pool = HostPool::get();
  if (level == 0) {
    // code sizes in code order (vx fastest), then the rows (vy, vz) filled in parallel
    P.bucket.resize(G.N);
    const int vz1 = d == 3 ? C.base - 1 : 1, vz0 = d == 3 ? 0 : 1;
    std::vector<int> ext[3];
    for (int a = 0; a < 3; ++a) {
      ext[a].assign(C.base, 1);
      if (a >= d) continue;
      for (int v = 0; v < C.base; ++v) {
        int lo, hi;
        vrange(v, w, G.ns[a], &lo, &hi);
        ext[a][v] = std::max(hi - lo + 1, 0);
      }
    }
    int64_t pos = 0;
    for (int vz = vz0; vz <= vz1; ++vz)
      for (int vy = 0; vy < C.base; ++vy)
        for (int vx = 0; vx < C.base; ++vx) {
          int v[3] = {vx, vy, vz};
          cstart[C.join(v)] = pos;
          pos += (int64_t)ext[0][vx] * ext[1][vy] * (d == 3 ? ext[2][vz] : 1);
        }
    cstart[C.ncode] = pos;
    const int nrows = (vz1 - vz0 + 1) * C.base;
    pool.parallel_for(nrows, 16, [&](int64_t r0, int64_t r1) {
      for (int64_t row = r0; row < r1; ++row) {
        const int vz = vz0 + (int)(row / C.base), vy = (int)(row % C.base);
        int zlo = 1, zhi = 1, ylo, yhi;
        if (d == 3) vrange(vz, w, G.ns[2], &zlo, &zhi);
        vrange(vy, w, G.ns[1], &ylo, &yhi);
        for (int vx = 0; vx < C.base; ++vx) {
          int xlo, xhi;
          vrange(vx, w, G.ns[0], &xlo, &xhi);
          int v[3] = {vx, vy, vz};
          int64_t q = cstart[C.join(v)];
          for (int z = zlo; z <= zhi; ++z)
            for (int y = ylo; y <= yhi; ++y) {
              const int64_t base = (int64_t)(y - 1) * G.ns[0] + (int64_t)(z - 1) * G.ns[0] * G.ns[1];
              for (int x = xlo; x <= xhi; ++x) P.bucket[q++] = (int32_t)(base + x - 1);
            }
        }
      }
    });
  } else {
    // Every DOF of a separator group of level - 1 lands in the same code at
    // this level (an open interval of width w/2 lies inside one interval of
    // width w, and a plane x = q w/2 is either a plane or an interior line),
    // so codes and counts go group by group, and each code is filled from its
    // groups (in group order) independently of the others.
    const Coder Cp(G, level - 1);
    const int pg = prev->ngroup();
    gcode.resize(pg);
    std::vector<int>& gna = X.gna;
    gna.resize(pg);
    pool.parallel_for(pg, 1024, [&](int64_t g0, int64_t g1) {
      for (int64_t g = g0; g < g1; ++g) {
        int v[3];
        Cp.split(prev->group_code[g], v);
        for (int a = 0; a < d; ++a) v[a] = (v[a] % 2 == 0) ? v[a] / 2 : 2 * (((v[a] - 1) / 2) / 2) + 1;
        gcode[g] = C.join(v);
        const uint8_t* kp = keep.data() + prev->group_start[g];
        int na = 0;
        for (int o = 0; o < prev->group_size[g]; ++o) na += kp[o] != 0;
        gna[g] = na;
      }
    });
    gpos_off.resize(pg + 1);
    gpos_off[0] = 0;
    std::vector<int>& cgoff = X.cgoff;   // groups of each code, stable
    cgoff.assign(C.ncode + 1, 0);
    for (int g = 0; g < pg; ++g) {
      gpos_off[g + 1] = gpos_off[g] + prev->group_size[g];
      cstart[gcode[g] + 1] += gna[g];
      ++cgoff[gcode[g] + 1];
    }
    for (int64_t c = 0; c < C.ncode; ++c) {
      cstart[c + 1] += cstart[c];
      cgoff[c + 1] += cgoff[c];
    }
    std::vector<int>& cg = X.cg;
    cg.resize(pg);
    {
      std::vector<int>& fillp = X.nseg;   // reused as a cursor here
      fillp.assign(cgoff.begin(), cgoff.end() - 1);
      for (int g = 0; g < pg; ++g) cg[fillp[gcode[g]]++] = g;
    }
    P.bucket.resize(cstart[C.ncode]);
    newpos.resize(gpos_off[pg]);
    std::vector<int>& src = X.src;
    src.resize(P.bucket.size());
    // ascending DOF index within every code; newpos follows the moves.  The
    // survivors of a group are compacted without branches (the flags are
    // data-dependent): first their offsets, with the new position of every
    // DOF, then the copy.
    pool.parallel_for(C.ncode, 256, [&](int64_t c0, int64_t c1) {
      std::vector<int64_t> key;
      std::vector<int> loc;
      for (int64_t c = c0; c < c1; ++c) {
        int64_t q = cstart[c];
        for (int t = cgoff[c]; t < cgoff[c + 1]; ++t) {
          const int g = cg[t];
          const int gs = prev->group_size[g], gp = gpos_off[g];
          const int32_t* __restrict__ gb = prev->bucket.data() + prev->group_start[g];
          const uint8_t* __restrict__ kp = keep.data() + prev->group_start[g];
          int* __restrict__ np = newpos.data() + gp;
          if ((int)loc.size() < gs) loc.resize(gs);
          int* __restrict__ lo = loc.data();
          int cnt = 0;
          for (int o = 0; o < gs; ++o) {
            const int k = kp[o] != 0;
            lo[cnt] = o;   // overwritten by the next DOF unless this one survives
            np[o] = k ? (int)q + cnt : -1;
            cnt += k;
          }
          int32_t* __restrict__ bq = P.bucket.data() + q;
          int* __restrict__ sq = src.data() + q;
          for (int j = 0; j < cnt; ++j) {
            bq[j] = gb[lo[j]];
            sq[j] = gp + lo[j];
          }
          q += cnt;
        }
        const int64_t a = cstart[c], b = cstart[c + 1];
        if (b - a > 1 && !std::is_sorted(P.bucket.begin() + a, P.bucket.begin() + b)) {
          key.resize(b - a);
          for (int64_t i = a; i < b; ++i) key[i - a] = ((int64_t)P.bucket[i] << 32) | (uint32_t)src[i];
          std::sort(key.begin(), key.end());
          for (int64_t i = a; i < b; ++i) {
            P.bucket[i] = (int32_t)(key[i - a] >> 32);
            src[i] = (int)(key[i - a] & 0xffffffff);
          }
          for (int64_t i = a; i < b; ++i) newpos[src[i]] = (int)i;
        }
      }
    });
  }
  auto csize = [&](int64_t c) { return (int)(cstart[c + 1] - cstart[c]); };

  // 2. cells: every cell whose closure holds an active DOF.  Codes are walked
  // as (v0, v1, v2) loops in code order (code = v0 + base v1 + base^2 v2).
  const int64_t s1 = C.base, s2 = d == 3 ? (int64_t)C.base * C.base : 0;
  const int vz_end = d == 3 ? C.base : 1;
  std::vector<int>& cell_of_code = X.cell_of_code;
  cell_of_code.assign(C.ncode, -1);
  for (int vz = d == 3 ? 1 : 0; vz < vz_end; vz += 2)
    for (int vy = 1; vy < C.base; vy += 2)
      for (int vx = 1; vx < C.base; vx += 2) {
        const int64_t c = vx + s1 * vy + s2 * vz;
        bool any = false;
        for (int oz = d == 3 ? -1 : 0; oz <= (d == 3 ? 1 : 0) && !any; ++oz)
          for (int oy = -1; oy <= 1 && !any; ++oy)
            for (int ox = -1; ox <= 1 && !any; ++ox) any = csize(c + ox + s1 * oy + s2 * oz) > 0;
        if (!any) continue;
        cell_of_code[c] = (int)P.cell_code.size();
        P.cell_code.push_back(c);
      }
  const int ncell = (int)P.cell_code.size();

  // 3. groups (t >= 1) in code order
  std::vector<int>& group_of_code = X.group_of_code;
  group_of_code.assign(C.ncode, -1);
  for (int vz = 0; vz < vz_end; ++vz)
    for (int vy = 0; vy < C.base; ++vy)
      for (int vx = 0; vx < C.base; ++vx) {
        const int64_t c = vx + s1 * vy + s2 * vz;
        const int sz = csize(c);
        const int t = (vx % 2 == 0) + (vy % 2 == 0) + (d == 3 && vz % 2 == 0);
        if (!sz || t == 0) continue;
        group_of_code[c] = (int)P.group_t.size();
        P.group_code.push_back(c);
        P.group_t.push_back(t);
        P.group_start.push_back((int32_t)cstart[c]);
        P.group_size.push_back(sz);
        P.max_group = std::max(P.max_group, sz);
      }
  const int ngroup = (int)P.group_t.size();

  // 4. cells: interior range, separator segments, storage offsets (segment
  // counts per cell in parallel, offsets in order, segments in parallel)
  const int dz = d >= 3 ? 1 : 0;
  P.cell_start.resize(ncell);
  P.nI.resize(ncell);
  P.nB.resize(ncell);
  if (level == 0) P.band_w.resize(ncell);
  std::vector<int>& nseg = X.nseg;
  nseg.resize(ncell);
  auto cell_segments = [&](int ci, int* sg, int* sp) {   // returns the count; fills if sg
    int v[3];
    C.split(P.cell_code[ci], v);
    int cnt = 0, nB = 0;
    for (int oz = -dz; oz <= dz; ++oz)
      for (int oy = -1; oy <= 1; ++oy)
        for (int ox = -1; ox <= 1; ++ox) {
          if (ox == 0 && oy == 0 && oz == 0) continue;
          int u[3] = {v[0] + ox, v[1] + oy, v[2] + oz};
          const int gi = group_of_code[C.join(u)];
          if (gi < 0) continue;
          if (sg) {
            sg[cnt] = gi;
            sp[cnt] = nB;
          }
          ++cnt;
          nB += P.group_size[gi];
        }
    P.nB[ci] = nB;
    return cnt;
  };
  pool.parallel_for(ncell, 256, [&](int64_t c0, int64_t c1) {
    for (int64_t ci = c0; ci < c1; ++ci) {
      const int64_t cc = P.cell_code[ci];
      nseg[ci] = cell_segments((int)ci, nullptr, nullptr);
      P.cell_start[ci] = (int32_t)cstart[cc];
      P.nI[ci] = csize(cc);
      if (level == 0) {
        int v[3];
        C.split(cc, v);
        int bw = 1;   // interior box: half bandwidth = its x extent (2D) or x*y extent (3D)
        for (int a = 0; a < d - 1; ++a) {
          int lo, hi;
          vrange(v[a], w, G.ns[a], &lo, &hi);
          bw *= std::max(hi - lo + 1, 0);
        }
        P.band_w[ci] = P.nI[ci] == 0 ? 0 : bw;
      }
    }
  });
  P.seg_off.resize(ncell + 1);
  P.gid_off.resize(ncell + 1);
  P.b_off.resize(ncell + 1);
  P.front_off.resize(ncell);
  P.frame_off.resize(ncell);
  P.frame_ld.resize(ncell);
  if (level == 0) {
    P.band_off.resize(ncell);
    P.z_off.resize(ncell);
  }
  P.seg_off[0] = 0;
  P.gid_off[0] = 0;
  P.b_off[0] = 0;
  for (int ci = 0; ci < ncell; ++ci) {
    const int nI = P.nI[ci], nB = P.nB[ci], n = nI + nB;
    P.seg_off[ci + 1] = P.seg_off[ci] + nseg[ci];
    P.gid_off[ci + 1] = P.gid_off[ci] + n;
    P.b_off[ci + 1] = P.b_off[ci] + nB;
    if (level == 0) {
      const int bw = P.band_w[ci];
      P.band_off[ci] = P.band_total;
      P.band_total += pad4((int64_t)nI * (bw + 1));
      P.z_off[ci] = P.z_total;
      P.z_total += pad4((int64_t)nI * nB);
      P.frame_off[ci] = P.frame_total;
      P.frame_ld[ci] = nB;
      P.frame_total += pad4((int64_t)nB * nB);
      P.front_off[ci] = 0;
      P.max_w = std::max(P.max_w, bw);
    } else {
      P.front_off[ci] = P.front_total;
      P.frame_off[ci] = P.front_total + nI + (int64_t)nI * n;
      P.frame_ld[ci] = n;
      P.front_total += pad4((int64_t)n * n);
    }
    P.max_nI = std::max(P.max_nI, nI);
    P.max_nB = std::max(P.max_nB, nB);
    P.max_n = std::max(P.max_n, n);
  }
  P.seg_group.resize(P.seg_off[ncell]);
  P.seg_pos.resize(P.seg_off[ncell]);
  pool.parallel_for(ncell, 256, [&](int64_t c0, int64_t c1) {
    for (int64_t ci = c0; ci < c1; ++ci)
      cell_segments((int)ci, P.seg_group.data() + P.seg_off[ci], P.seg_pos.data() + P.seg_off[ci]);
  });
  std::vector<int> gcount(ngroup + 1, 0);
  for (int sgi : P.seg_group) ++gcount[sgi + 1];
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

  // 5. extend-add maps from the previous level's frames.  A child segment's
  // DOFs all sit in one code here: the parent's interior or one of its
  // segments, found once per child segment.
  if (prev) {
    const Coder Cp(G, level - 1);
    std::vector<int>& prev_cell_of_code = X.prev_cell_of_code;
    prev_cell_of_code.assign(Cp.ncode, -1);
    for (int i = 0; i < prev->ncell(); ++i) prev_cell_of_code[prev->cell_code[i]] = i;
    // children of every cell, then one allocation of the whole map
    P.ea_off.assign(1, 0);
    int64_t map_total = 0;
    for (int ci = 0; ci < ncell; ++ci) {
      int v[3];
      C.split(P.cell_code[ci], v);
      for (int z = d == 3 ? v[2] - 1 : 0; z <= (d == 3 ? v[2] : 0); ++z)
        for (int y = v[1] - 1; y <= v[1]; ++y)
          for (int x = v[0] - 1; x <= v[0]; ++x) {
            int u[3] = {2 * x + 1, 2 * y + 1, 2 * z + 1};
            const int pc = prev_cell_of_code[Cp.join(u)];
            if (pc < 0) continue;
            P.ea_child.push_back(pc);
            P.ea_map_off.push_back(map_total);
            map_total += prev->nB[pc];
          }
      P.ea_off.push_back((int)P.ea_child.size());
    }
    P.ea_map.resize(map_total);   // every slot is written below
    pool.parallel_for(ncell, 128, [&](int64_t c0, int64_t c1) {
    for (int64_t ci = c0; ci < c1; ++ci) {
      const int nI = P.nI[ci];
      for (int k = P.ea_off[ci]; k < P.ea_off[ci + 1]; ++k) {
        const int pc = P.ea_child[k];
        const int64_t base = P.ea_map_off[k];
            for (int s = prev->seg_off[pc]; s < prev->seg_off[pc + 1]; ++s) {
              const int g = prev->seg_group[s];
              const int64_t gc = gcode[g];
              int64_t shift = 0;   // parent position = bucket position + shift
              bool found = false;
              if (gc == P.cell_code[ci]) {
                shift = -(int64_t)P.cell_start[ci];
                found = true;
              } else {
                const int pg = group_of_code[gc];
                for (int t = P.seg_off[ci]; t < P.seg_off[ci + 1] && !found; ++t)
                  if (P.seg_group[t] == pg) {
                    shift = nI + P.seg_pos[t] - (int64_t)P.group_start[pg];
                    found = true;
                  }
              }
              const int gs = prev->group_size[g];
              const int* __restrict__ np = newpos.data() + gpos_off[g];
              int* __restrict__ out = P.ea_map.data() + base + prev->seg_pos[s];
              if (!found) {   // no DOF of the segment reaches this front
                std::fill(out, out + gs, -1);
                continue;
              }
              const int sh = (int)shift;   // front positions and bucket offsets fit in int
              for (int o = 0; o < gs; ++o) {
                const int v = np[o];
                out[o] = v >= 0 ? v + sh : -1;
              }
            }
      }
    }
    });
  }

  if (level >= G.L) return P;   // root front only

  // 6. preconditioning + skeletonization passes
  const int npass = (d == 3 && edge_skel) ? 2 : 1;
  std::vector<int>& nrow_of = X.nrow;   // unit row counts of the unit groups, in parallel
  nrow_of.assign(ngroup, 0);
  pool.parallel_for(ngroup, 1024, [&](int64_t g0, int64_t g1) {
    for (int64_t gi = g0; gi < g1; ++gi)
      if (P.group_t[gi] <= npass) nrow_of[gi] = unit_row_count(P, (int)gi);
  });
  for (int pass = 0; pass < npass; ++pass) {
    PhasePlan ph;
    if (!P.phase_spare.empty()) {   // storage of a recycled plan's phase
      ph = std::move(P.phase_spare.back());
      P.phase_spare.pop_back();
      ph.clear();
    }
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
        const int nrow = nrow_of[gi];
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
