// Host-only self-check of the level planner (plan.cpp): builds every level of
// a grid with seeded synthetic survivor flags and checks the plan against the
// definitions it encodes (Sec. 3.1, Fig. 3: cells, separator groups, the
// front order [interior; segments]), recomputed here from DOF coordinates:
//   * the bucket holds each active DOF once, ordered by (code, DOF index),
//     the code being 2 (x / w) + (x % w != 0) per axis at cell width w;
//   * a cell's interior is the range of its own code; its segments are the
//     nonempty separator codes adjacent to it, in code order, at the prefix
//     positions of their sizes; every group lists exactly the cells that hold
//     it, at the positions those cells give it;
//   * every extend-add map entry sends a surviving child-frame DOF to the
//     position of the same DOF in the parent front, and a dropped one to -1;
//   * a second build from recycled storage gives the same tables.
// No device work: the function runs on any host.
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/rhif.h"
#include "plan.h"

namespace rhif {
void set_error_detail(const std::string& msg);
}

namespace {

using rhif::Geometry;
using rhif::LevelPlan;

uint64_t splitmix(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

int64_t code_of(const Geometry& G, int level, int64_t gid, int* v) {
  const int w = G.leaf << level;
  const int64_t base = 2 * (int64_t(1) << (G.L - level)) + 1;
  int64_t rem = gid, code = 0, mul = 1;
  for (int a = 0; a < 3; ++a) v[a] = 1;
  for (int a = 0; a < G.d; ++a) {
    const int x = (int)(rem % G.ns[a]) + 1;
    rem /= G.ns[a];
    v[a] = 2 * (x / w) + (x % w != 0);
    code += mul * v[a];
    mul *= base;
  }
  return code;
}

struct Fail {
  std::string msg;
  bool operator()(bool ok, int level, const char* what) {
    if (!ok && msg.empty()) {
      char b[160];
      std::snprintf(b, sizeof(b), "plan self-check: level %d: %s", level, what);
      msg = b;
    }
    return ok;
  }
};

// DOF at front position p of cell ci
int32_t front_gid(const LevelPlan& P, int ci, int p) {
  const int nI = P.nI[ci];
  if (p < nI) return P.bucket[P.cell_start[ci] + p];
  for (int s = P.seg_off[ci]; s < P.seg_off[ci + 1]; ++s) {
    const int g = P.seg_group[s];
    const int q = p - nI - P.seg_pos[s];
    if (q >= 0 && q < P.group_size[g]) return P.bucket[P.group_start[g] + q];
  }
  return -1;
}

bool same(const LevelPlan& A, const LevelPlan& B) {
  return A.bucket == B.bucket && A.cell_code == B.cell_code && A.cell_start == B.cell_start &&
         A.nI == B.nI && A.nB == B.nB && A.seg_off == B.seg_off && A.seg_group == B.seg_group &&
         A.seg_pos == B.seg_pos && A.group_code == B.group_code && A.group_start == B.group_start &&
         A.group_size == B.group_size && A.group_cell_off == B.group_cell_off &&
         A.group_cell == B.group_cell && A.group_pos == B.group_pos && A.ea_off == B.ea_off &&
         A.ea_child == B.ea_child && A.ea_map_off == B.ea_map_off && A.ea_map == B.ea_map &&
         A.front_off == B.front_off && A.frame_off == B.frame_off && A.band_off == B.band_off &&
         A.phases.size() == B.phases.size();
}

// Seeded survivor flags of level `lvl` (a share `keep` of each skeletonized
// group's DOFs), by bucket position; also cleared in `alive` (by DOF index).
void survivors(const Geometry& G, const LevelPlan& P, int lvl, bool edge, double keep, uint64_t& rng,
               std::vector<uint8_t>& keepv, std::vector<uint8_t>* alive) {
  keepv.assign(P.bucket.size(), 1);
  if (lvl >= G.L) return;
  for (int g = 0; g < P.ngroup(); ++g) {
    if (P.group_t[g] > (edge ? 2 : 1)) continue;
    for (int o = 0; o < P.group_size[g]; ++o) {
      const double u = (splitmix(rng) >> 11) * (1.0 / 9007199254740992.0);
      if (u >= keep) {
        keepv[P.group_start[g] + o] = 0;
        if (alive) (*alive)[P.bucket[P.group_start[g] + o]] = 0;
      }
    }
  }
}

}  // namespace

extern "C" int rhif_plan_selfcheck(int dim, const int* ns, int leaf, double keep, uint64_t seed,
                                   int edge_skel_3d, int64_t* levels_checked) {
  if ((dim != 2 && dim != 3) || !ns || leaf < 2 || !(keep >= 0.0 && keep <= 1.0)) {
    rhif::set_error_detail("plan self-check: bad argument");
    return RHIF_ERR_BAD_ARG;
  }
  for (int a = 0; a < dim; ++a)
    if (ns[a] < 1) {
      rhif::set_error_detail("plan self-check: bad grid");
      return RHIF_ERR_BAD_ARG;
    }
  const Geometry G = rhif::make_geometry(dim, ns, leaf);
  const bool edge = dim == 3 && edge_skel_3d;
  Fail fail;
  uint64_t rng = seed;
  std::vector<LevelPlan> plans;
  std::vector<uint8_t> keepv;
  std::vector<uint8_t> alive(G.N, 1);   // by DOF index, for the checks
  if (levels_checked) *levels_checked = 0;
  for (int lvl = 0; lvl <= G.L && fail.msg.empty(); ++lvl) {
    plans.push_back(rhif::build_level(G, lvl, keepv, lvl ? &plans[lvl - 1] : nullptr, true, edge));
    const LevelPlan& P = plans.back();
    // 1. bucket: the active DOFs once each, ordered by (code, index)
    int64_t nactive = G.N;
    if (lvl > 0) {
      nactive = 0;
      const LevelPlan& Q = plans[lvl - 1];
      for (int g = 0; g < Q.ngroup(); ++g)
        for (int o = 0; o < Q.group_size[g]; ++o) nactive += alive[Q.bucket[Q.group_start[g] + o]];
    }
    fail((int64_t)P.bucket.size() == nactive, lvl, "bucket size differs from the active count");
    std::vector<uint8_t> seen(G.N, 0);
    std::vector<int64_t> sep_codes;   // nonempty separator codes, ascending
    int64_t prev_code = -1;
    int32_t prev_gid = -1;
    for (int32_t gid : P.bucket) {
      if (!fail(gid >= 0 && gid < G.N && !seen[gid], lvl, "bucket repeats a DOF")) break;
      seen[gid] = 1;
      int v[3];
      const int64_t c = code_of(G, lvl, gid, v);
      fail(lvl == 0 || alive[gid], lvl, "bucket holds an eliminated DOF");
      fail(c > prev_code || (c == prev_code && gid > prev_gid), lvl, "bucket not ordered by (code, index)");
      int t = 0;
      for (int a = 0; a < G.d; ++a) t += (v[a] % 2 == 0);
      if (t >= 1 && c != prev_code) sep_codes.push_back(c);
      prev_code = c;
      prev_gid = gid;
    }
    fail(P.group_code == sep_codes, lvl, "groups differ from the nonempty separator codes");
    // 2. cells and their segments: every nonempty separator code adjacent to
    // the cell, in code order, at the prefix positions of the sizes
    std::vector<std::vector<std::pair<int, int>>> holders(P.ngroup());
    const int64_t base = 2 * (int64_t(1) << (G.L - lvl)) + 1;
    for (int ci = 0; ci < P.ncell() && fail.msg.empty(); ++ci) {
      int vc[3] = {1, 1, 1};
      {
        int64_t cc = P.cell_code[ci];
        for (int a = 0; a < G.d; ++a) {
          vc[a] = (int)(cc % base);
          cc /= base;
        }
      }
      for (int i = 0; i < P.nI[ci]; ++i) {
        int v[3];
        fail(code_of(G, lvl, P.bucket[P.cell_start[ci] + i], v) == P.cell_code[ci], lvl,
             "interior DOF outside its cell's code");
      }
      std::vector<int64_t> adj;   // expected segments
      for (int64_t sc : sep_codes) {
        int64_t r = sc;
        bool near = true;
        for (int a = 0; a < G.d; ++a) {
          const int va = (int)(r % base);
          r /= base;
          near &= va >= vc[a] - 1 && va <= vc[a] + 1;
        }
        if (near) adj.push_back(sc);
      }
      fail(P.seg_off[ci + 1] - P.seg_off[ci] == (int)adj.size(), lvl, "cell has a wrong number of segments");
      int pos = 0;
      for (int s = P.seg_off[ci]; s < P.seg_off[ci + 1]; ++s) {
        const int g = P.seg_group[s];
        const int k = s - P.seg_off[ci];
        fail(k < (int)adj.size() && P.group_code[g] == adj[k], lvl, "segment is not the next adjacent separator code");
        fail(P.seg_pos[s] == pos, lvl, "segment position is not the prefix of sizes");
        holders[g].push_back({ci, pos});
        pos += P.group_size[g];
      }
      fail(P.nB[ci] == pos, lvl, "nB differs from the segment sizes");
    }
    for (int g = 0; g < P.ngroup() && fail.msg.empty(); ++g) {
      const int k0 = P.group_cell_off[g], k1 = P.group_cell_off[g + 1];
      fail(k1 - k0 == (int)holders[g].size(), lvl, "group lists a wrong number of cells");
      for (int k = k0; k < k1 && k - k0 < (int)holders[g].size(); ++k)
        fail(P.group_cell[k] == holders[g][k - k0].first && P.group_pos[k] == holders[g][k - k0].second, lvl,
             "group's (cell, position) list differs from the cells' segments");
    }
    // 3. extend-add maps: surviving child-frame DOFs land on the same DOF
    if (lvl > 0 && fail.msg.empty()) {
      const LevelPlan& Q = plans[lvl - 1];
      for (int ci = 0; ci < P.ncell(); ++ci)
        for (int k = P.ea_off[ci]; k < P.ea_off[ci + 1]; ++k) {
          const int pc = P.ea_child[k];
          const int* map = P.ea_map.data() + P.ea_map_off[k];
          for (int j = 0; j < Q.nB[pc]; ++j) {
            const int32_t gid = front_gid(Q, pc, Q.nI[pc] + j);
            if (!alive[gid])
              fail(map[j] == -1, lvl, "dropped DOF mapped into a parent front");
            else
              fail(map[j] >= 0 && map[j] < P.nI[ci] + P.nB[ci] && front_gid(P, ci, map[j]) == gid, lvl,
                   "surviving DOF mapped to another DOF of the parent front");
          }
        }
    }
    survivors(G, P, lvl, edge, keep, rng, keepv, &alive);
    if (fail.msg.empty() && levels_checked) *levels_checked = lvl + 1;
  }
  // 4. the same survivors again, from recycled storage
  if (fail.msg.empty()) {
    std::vector<LevelPlan> first = plans;
    for (auto& P : plans) rhif::recycle_plan(std::move(P));
    std::vector<LevelPlan> again;
    uint64_t r2 = seed;
    keepv.clear();
    for (int lvl = 0; lvl <= G.L && fail.msg.empty(); ++lvl) {
      again.push_back(rhif::build_level(G, lvl, keepv, lvl ? &again[lvl - 1] : nullptr, true, edge));
      fail(same(again.back(), first[lvl]), lvl, "rebuild from recycled storage differs");
      survivors(G, again.back(), lvl, edge, keep, r2, keepv, nullptr);
    }
  }
  if (!fail.msg.empty()) {
    rhif::set_error_detail(fail.msg);
    return RHIF_ERR_CHECK;
  }
  return RHIF_OK;
}
