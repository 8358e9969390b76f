// Device views of one level plan (see plan.h), passed by value to kernels.
#pragma once
#include <cstdint>

namespace rhif {

struct GeoDev {
  int d, leaf;
  int ns[3];
  int64_t N;
  int64_t stride[3];
};

struct LevelDev {
  int level, ncell, ngroup;
  int width, code_base;      // cell width in grid intervals; base of the group code
  const int64_t* cell_code;
  int max_nI, max_nB, max_n, max_group;
  const int64_t* front_off;
  const int* nI;
  const int* nB;
  const int64_t* gid_off;
  const int64_t* gids;
  const int64_t* b_off;
  const int* seg_off;
  const int* seg_group;
  const int* seg_pos;
  const int* group_t;
  const int64_t* group_gid_off;
  const int64_t* group_gids;
  const int* group_cell_off;
  const int* group_cell;
  const int* group_pos;
  const int* ea_off;
  const int* ea_child;
  const int64_t* ea_map_off;
  const int* ea_map;
  void* front;   // element type of the factor
};

struct PhaseDev {
  int unit_type, pre_min_type;
  int npre;
  const int* pre_group;
  const int64_t* pre_off;
  const int* group_pre;    // per group of the level: index into pre_group or -1
  void* Lbuf;
  int nunit, max_n;
  const int* u_group;
  const int* u_nrow;
  const int64_t* u_row_off;
  const int64_t* u_row_gid;
  const int64_t* row_src_off;
  const int* src_cell;
  const int* src_pos;
  const int* src_upos;
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
