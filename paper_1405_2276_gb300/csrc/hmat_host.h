// Host-side result of the H-matrix construction (cluster order throughout).
#pragma once

#include <stdint.h>

#include <utility>
#include <vector>

struct HCluster {
  int64_t begin = 0, end = 0;  // point range in cluster order
  double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
  int child[2] = {-1, -1};
  int level = 0;
  int parent = -1;
};

// Low-rank block Gamma(t, s) ~= sum_l u_l v_l^T, stored column by column:
// u[l*|t| + i], v[l*|s| + j].
struct HFar {
  int t = 0, s = 0, k = 0;
  std::vector<double> u, v;
};

struct HostHmat {
  int64_t n = 0;
  int dim = 0;
  std::vector<HCluster> cl;
  std::vector<double> pts;                 // cluster order
  std::vector<HFar> far;                   // t before s
  std::vector<std::pair<int, int>> near;   // leaf pairs, t <= s
  std::vector<int64_t> near_off;           // offsets into near_val
  std::vector<double> near_val;            // |t| x |s| row-major per pair
  double build_seconds = 0;
};
