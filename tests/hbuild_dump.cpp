// Test harness (host only): runs the library's host-side H-matrix
// construction (csrc/hbuild.cpp) on points read from a file and writes the
// result -- permutation, cluster tree, low-rank blocks, near pairs and their
// dense tiles -- as one binary file of int64 / double records, for
// tests/test_hbuild_host.py to check against the oracle's Matern kernel.
//
// usage: hbuild_dump points.bin n dim nu ell sigma2 leaf eta aca_tol k_cap out.bin
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "common.h"
#include "hmat_host.h"

static void put_i(FILE* f, int64_t v) { fwrite(&v, sizeof v, 1, f); }
static void put_d(FILE* f, double v) { fwrite(&v, sizeof v, 1, f); }

int main(int argc, char** argv) {
  if (argc != 12) {
    fprintf(stderr, "usage: %s points.bin n dim nu ell sigma2 leaf eta aca_tol k_cap out.bin\n", argv[0]);
    return 2;
  }
  const int64_t n = atoll(argv[2]);
  const int dim = atoi(argv[3]);
  std::vector<double> pts((size_t)n * dim);
  FILE* fp = fopen(argv[1], "rb");
  if (!fp || fread(pts.data(), sizeof(double), pts.size(), fp) != pts.size()) return 3;
  fclose(fp);
  fkf_matern k{};
  k.nu = atof(argv[4]);
  k.ell = atof(argv[5]);
  k.sigma2 = atof(argv[6]);
  fkf_hparams hp{};
  hp.leaf = atoi(argv[7]);
  hp.eta = atof(argv[8]);
  hp.aca_tol = atof(argv[9]);
  hp.k_cap = atoi(argv[10]);
  HostHmat* H = nullptr;
  std::vector<int64_t> perm;
  if (hmat_build_host(nullptr, pts.data(), n, dim, k, hp, &H, perm) != FKF_OK) return 4;
  FILE* f = fopen(argv[11], "wb");
  if (!f) return 5;
  for (int64_t v : perm) put_i(f, v);
  put_i(f, (int64_t)H->cl.size());
  for (const HCluster& c : H->cl) {
    put_i(f, c.begin);
    put_i(f, c.end);
    put_i(f, c.child[0]);
    put_i(f, c.child[1]);
    for (int a = 0; a < 3; a++) put_d(f, c.lo[a]);
    for (int a = 0; a < 3; a++) put_d(f, c.hi[a]);
  }
  put_i(f, (int64_t)H->far.size());
  for (const HFar& b : H->far) {
    put_i(f, b.t);
    put_i(f, b.s);
    put_i(f, b.k);
    for (double v : b.u) put_d(f, v);
    for (double v : b.v) put_d(f, v);
  }
  put_i(f, (int64_t)H->near.size());
  for (size_t i = 0; i < H->near.size(); i++) {
    put_i(f, H->near[i].first);
    put_i(f, H->near[i].second);
  }
  for (double v : H->near_val) put_d(f, v);
  fclose(f);
  hmat_free_host(H);
  return 0;
}
