// H-matrix apply Y = Gamma_H X for a tall block X (N x ncols, cluster order).
//
// The paper needs Gamma_sys times blocks of vectors (Gamma H^T, Sec. 2.3 and
// Alg. kalmanconstantH; Gamma W_k, Sec. 2.4) and takes the MVP from an H-matrix
// (Sec. 2.2.1).  Device layout (all row-major, element type = precision):
//
//   Fac_c   |c| x K_c  for every cluster c: the row factors of all far blocks
//                       that have c as one side, side by side ("slots").  A far
//                       block b = (t, s) of rank k owns k slots in Fac_t (U_b)
//                       and k slots in Fac_s (V_b).
//   Near_l  |l| x Kn_l for every leaf l: the dense blocks Gamma(l, sigma) of all
//                       near partners sigma, side by side (both orientations
//                       of a stored pair are written from the same values, so
//                       Gamma_H is exactly symmetric).
//
// Apply, per panel of P columns:
//   phase 1  Z_c = Fac_c^T X_c        one reduction per cluster (split over row
//                                      chunks for large clusters, reduced in a
//                                      fixed order); slot rows are scattered to
//                                      the partner slot: Zmix[map(g)] = Z[g]
//   phase 2  Y_l = sum_{c ancestor of l} Fac_c[l rows] Zmix_c
//                + sum_{sigma near l} Near_l[:, sigma] X_sigma
// so each row block of Y is written once, by one CTA, with no atomics, and
// X_c is read once per cluster level instead of once per block.
#include <algorithm>
#include <cmath>
#include <unordered_map>
#include <cstring>
#include <mutex>

#include "common.h"
#include "hmat_host.h"
#include "tile.cuh"

namespace {

constexpr int kChunkRows = 2048;  // phase-1 reduction chunk (rows of a cluster)

template <typename T>
__global__ void __launch_bounds__(kTileThreads) k_phase1(const P1Item* __restrict__ items, const T* __restrict__ fac,
                                                         const T* __restrict__ X, int64_t ldx, int ncols,
                                                         const int64_t* __restrict__ slotmap, T* __restrict__ zmix,
                                                         T* __restrict__ part, int64_t ldz) {
  __shared__ TileSmem<T> sm;
  const P1Item it = items[blockIdx.x];
  const int n0 = blockIdx.y * TileCfg<T>::BN;
  const int nv = min(TileCfg<T>::BN, ncols - n0);
  if (nv <= 0) return;
  T acc[TileCfg<T>::TM][TileCfg<T>::TN];
  tile_zero<T>(acc);
  // A(m = slot, k = row) = Fac_c[(r0 + row) * K + q0 + slot]
  const T* A = fac + it.fac_off + (int64_t)it.r0 * it.K + it.q0;
  const T* B = X + it.x_row * ldx + n0;
  tile_mma<T, false, false>(acc, A, it.K, it.nq, B, ldx, nv, it.nr, sm);
#pragma unroll
  for (int i = 0; i < TileCfg<T>::TM; i++) {
    const int q = tile_row<T>(i);
    if (q >= it.nq) continue;
    T* dst = it.out_row < 0 ? zmix + slotmap[it.map_off + q] * ldz : part + (it.out_row + q) * ldz;
#pragma unroll
    for (int j = 0; j < TileCfg<T>::TN; j++) {
      const int n = tile_col<T>(j);
      if (n < nv) dst[n0 + n] = acc[i][j];
    }
  }
}

template <typename T>
__global__ void k_phase1_reduce(const P1Reduce* __restrict__ items, const T* __restrict__ part,
                                const int64_t* __restrict__ slotmap, T* __restrict__ zmix, int64_t ldz, int ncols) {
  const P1Reduce it = items[blockIdx.x];
  const int64_t total = (int64_t)it.nq * ncols;
  for (int64_t e = threadIdx.x + (int64_t)blockIdx.y * blockDim.x; e < total; e += (int64_t)blockDim.x * gridDim.y) {
    const int q = (int)(e / ncols), n = (int)(e % ncols);
    T s = 0;
    for (int c = 0; c < it.nch; c++) s += part[(it.part_row + (int64_t)c * it.nq + q) * ldz + n];
    zmix[slotmap[it.map_off + q] * ldz + n] = s;
  }
}

template <typename T>
__global__ void __launch_bounds__(kTileThreads) k_phase2(const P2Leaf* __restrict__ leaves,
                                                         const P2Seg* __restrict__ segs, const T* __restrict__ fac,
                                                         const T* __restrict__ nearv, const T* __restrict__ zmix,
                                                         int64_t ldz, const T* __restrict__ X, int64_t ldx,
                                                         T* __restrict__ Y, int64_t ldy, int ncols) {
  __shared__ TileSmem<T> sm;
  const P2Leaf lf = leaves[blockIdx.x];
  const int n0 = blockIdx.y * TileCfg<T>::BN;
  const int nv = min(TileCfg<T>::BN, ncols - n0);
  if (nv <= 0) return;
  T acc[TileCfg<T>::TM][TileCfg<T>::TN];
  tile_zero<T>(acc);
  for (int s = 0; s < lf.nseg; s++) {
    const P2Seg sg = segs[lf.seg0 + s];
    const T* A = (sg.near ? nearv : fac) + sg.a_off + (int64_t)lf.pad * sg.lda;
    const T* B = sg.near ? X + sg.b_row * ldx + n0 : zmix + sg.b_row * ldz + n0;
    tile_mma<T, true, false>(acc, A, sg.lda, lf.rows, B, sg.near ? ldx : ldz, nv, sg.K, sm);
  }
#pragma unroll
  for (int i = 0; i < TileCfg<T>::TM; i++) {
    const int r = tile_row<T>(i);
    if (r >= lf.rows) continue;
    T* dst = Y + (lf.row0 + r) * ldy + n0;
#pragma unroll
    for (int j = 0; j < TileCfg<T>::TN; j++) {
      const int n = tile_col<T>(j);
      if (n < nv) dst[n] = acc[i][j];
    }
  }
}

template <typename T>
__global__ void k_gather_rows(const T* __restrict__ src, int64_t lds, const int64_t* __restrict__ idx, T* __restrict__ dst,
                              int64_t ldd, int64_t nrows, int ncols) {
  // dst[i, :] = src[idx[i], :]
  const int64_t total = nrows * ncols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / ncols;
    const int j = (int)(e % ncols);
    dst[i * ldd + j] = src[idx[i] * lds + j];
  }
}

template <typename T>
fkf_status apply_impl(fkf_hmat* h, const T* X, int64_t ldx, T* Y, int64_t ldy, int64_t ncols) {
  fkf_ctx* ctx = h->ctx;
  const int64_t P = h->panel;
  const size_t zbytes = (size_t)std::max<int64_t>(h->ktot, 1) * P * sizeof(T);
  if (h->zmix.bytes < zbytes) FKF_TRY(dev_alloc(ctx, h->zmix, zbytes));
  const size_t pbytes = (size_t)std::max<int64_t>(h->part_rows, 1) * P * sizeof(T);
  if (h->part.bytes < pbytes) FKF_TRY(dev_alloc(ctx, h->part, pbytes));
  constexpr int BN = TileCfg<T>::BN;
  for (int64_t c0 = 0; c0 < ncols; c0 += P) {
    const int nc = (int)std::min<int64_t>(P, ncols - c0);
    const int ntile = (int)cdiv(nc, BN);
    if (h->n_p1 > 0) {
      k_phase1<T><<<dim3((unsigned)h->n_p1, ntile), kTileThreads, 0, ctx->stream>>>(
          h->p1items.as<P1Item>(), h->fac.as<T>(), X + c0, ldx, nc, h->slotmap.as<int64_t>(), h->zmix.as<T>(),
          h->part.as<T>(), P);
      FKF_LAUNCHED(ctx);
    }
    if (h->n_p1red > 0) {
      k_phase1_reduce<T><<<dim3((unsigned)h->n_p1red, 4), 256, 0, ctx->stream>>>(
          h->p1red.as<P1Reduce>(), h->part.as<T>(), h->slotmap.as<int64_t>(), h->zmix.as<T>(), P, nc);
      FKF_LAUNCHED(ctx);
    }
    k_phase2<T><<<dim3((unsigned)h->n_leaf, ntile), kTileThreads, 0, ctx->stream>>>(
        h->p2leaf.as<P2Leaf>(), h->p2seg.as<P2Seg>(), h->fac.as<T>(), h->nearv.as<T>(), h->zmix.as<T>(), P, X + c0,
        ldx, Y + c0, ldy, nc);
    FKF_LAUNCHED(ctx);
  }
  return FKF_OK;
}

template <typename T>
void fill_typed(void* dst, const double* src, size_t n) {
  T* d = reinterpret_cast<T*>(dst);
  for (size_t i = 0; i < n; i++) d[i] = (T)src[i];
}

}  // namespace

fkf_status hmat_apply_clustered(fkf_hmat* h, const void* X, int64_t ldx, void* Y, int64_t ldy, int64_t ncols) {
  if (ncols <= 0) return FKF_OK;
  if (h->prec == FKF_FP64) {
    if (h->engine == 3) return hmat_apply_clustered_oz(h, (const double*)X, ldx, (double*)Y, ldy, ncols);
    return apply_impl<double>(h, (const double*)X, ldx, (double*)Y, ldy, ncols);
  }
  if (h->engine != 0) return hmat_apply_clustered_tc(h, (const float*)X, ldx, (float*)Y, ldy, ncols);
  return apply_impl<float>(h, (const float*)X, ldx, (float*)Y, ldy, ncols);
}

template <typename T>
static fkf_status permute_rows(fkf_ctx* ctx, const T* src, int64_t lds, const int64_t* idx, T* dst, int64_t ldd,
                               int64_t nrows, int64_t ncols) {
  const int64_t total = nrows * ncols;
  const int blocks = (int)std::min<int64_t>(cdiv(total, 256), 152 * 16);
  k_gather_rows<T><<<blocks, 256, 0, ctx->stream>>>(src, lds, idx, dst, ldd, nrows, (int)ncols);
  FKF_LAUNCHED(ctx);
  return FKF_OK;
}

fkf_status hmat_permute_rows(fkf_hmat* h, const void* src, int64_t lds, const int64_t* idx_dev, void* dst,
                             int64_t ldd, int64_t nrows, int64_t ncols) {
  if (h->prec == FKF_FP64)
    return permute_rows<double>(h->ctx, (const double*)src, lds, idx_dev, (double*)dst, ldd, nrows, ncols);
  return permute_rows<float>(h->ctx, (const float*)src, lds, idx_dev, (float*)dst, ldd, nrows, ncols);
}

// Per-block partial sums of <A, B> (FP64 accumulation, fixed order).
template <typename T>
__global__ void k_dot_part(int64_t nrows, int64_t ncols, const T* __restrict__ A, int64_t lda,
                           const T* __restrict__ B, int64_t ldb, double* __restrict__ part) {
  __shared__ double red[256];
  double acc = 0;
  const int64_t total = nrows * ncols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / ncols, j = e % ncols;
    acc += (double)A[i * lda + j] * (double)B[i * ldb + j];
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

fkf_status hmat_dot(fkf_hmat* h, const void* A, int64_t lda, const void* B, int64_t ldb, int64_t nrows, int64_t ncols,
                    double* out) {
  fkf_ctx* ctx = h->ctx;
  constexpr int kBlocks = 304;
  DevBuf part;
  FKF_TRY(dev_alloc(ctx, part, kBlocks * sizeof(double)));
  if (h->prec == FKF_FP64)
    k_dot_part<double><<<kBlocks, 256, 0, ctx->stream>>>(nrows, ncols, (const double*)A, lda, (const double*)B, ldb,
                                                          part.as<double>());
  else
    k_dot_part<float><<<kBlocks, 256, 0, ctx->stream>>>(nrows, ncols, (const float*)A, lda, (const float*)B, ldb,
                                                         part.as<double>());
  FKF_LAUNCHED(ctx);
  double hp[kBlocks];
  FKF_CUDA(ctx, cudaMemcpyAsync(hp, part.p, sizeof(hp), cudaMemcpyDeviceToHost, ctx->stream));
  FKF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  double s = 0;
  for (int b = 0; b < kBlocks; b++) s += hp[b];
  *out = s;
  return FKF_OK;
}

fkf_status hmat_permute_rows_f64(fkf_ctx* ctx, const double* src, int64_t lds, const int64_t* idx_dev, double* dst,
                                 int64_t ldd, int64_t nrows, int64_t ncols) {
  return permute_rows<double>(ctx, src, lds, idx_dev, dst, ldd, nrows, ncols);
}

// Device memory the operator holds now (values, schedules, streams and the
// apply workspaces allocated so far).
int64_t hmat_device_bytes(const fkf_hmat* h) {
  const DevBuf* bufs[] = {&h->fac,    &h->nearv,   &h->slotmap, &h->p1items, &h->p1red,  &h->p2seg,  &h->p2leaf,
                          &h->perm_d, &h->iperm_d, &h->tcp1,    &h->tcred,   &h->tctile, &h->tcseg,  &h->tc_err,
                          &h->tca,    &h->tcadesc, &h->tcxmap,  &h->tcslot,  &h->xsplit, &h->zsplit, &h->tc_qslot,
                          &h->tc_qpos, &h->tc_rpt, &h->tc_col,  &h->ozitem,  &h->ozred,  &h->oztile, &h->ozseg,
                          &h->ozbdesc, &h->ozxmap, &h->ozslot,  &h->oz_sigslot, &h->oz_qslot, &h->oz_qshift,
                          &h->oz_qpos, &h->oz_sigpt, &h->ozb,   &h->ozx,     &h->ozz,    &h->ozpart, &h->oz_col,
                          &h->oz_err,  &h->zmix,   &h->part,    &h->xperm,   &h->yperm};
  int64_t t = 0;
  for (const DevBuf* b : bufs) t += (int64_t)b->bytes;
  return t;
}

// Lay the host build out as flat device arrays and work lists.
fkf_status hmat_upload(fkf_hmat* h, const HostHmat& hh) {
  fkf_ctx* ctx = h->ctx;
  const auto& cl = hh.cl;
  const int nc = (int)cl.size();
  const size_t w = h->prec == FKF_FP64 ? 8 : 4;
  auto csize = [&](int c) { return cl[c].end - cl[c].begin; };
  // slots per cluster
  std::vector<std::vector<std::pair<int, int>>> slots(nc);  // (block, side)
  for (int b = 0; b < (int)hh.far.size(); b++) {
    slots[hh.far[b].t].push_back({b, 0});
    slots[hh.far[b].s].push_back({b, 1});
  }
  std::vector<int64_t> K(nc, 0), slot_base(nc, 0), fac_off(nc, 0);
  std::vector<std::vector<int64_t>> slot_col(nc);
  // every block gets a multiple of 4 slots (zero columns) on both sides, so
  // that aligned groups of 4 slots map to aligned groups of 4 (the
  // tensor-core engines write their slot values 4 at a time)
  auto block_width = [&](int b) -> int64_t {
    const int64_t k = hh.far[b].k;
    return (k + 3) / 4 * 4;
  };
  int64_t ktot = 0, facn = 0;
  for (int c = 0; c < nc; c++) {
    int64_t k = 0;
    for (auto [b, side] : slots[c]) {
      slot_col[c].push_back(k);
      k += block_width(b);
    }
    K[c] = (k + 3) / 4 * 4;
    slot_base[c] = ktot;
    fac_off[c] = facn;
    ktot += K[c];
    facn += csize(c) * K[c];
  }
  // slot map (involution between the two sides of each block, the padding
  // columns of a block included; the padding at the end of a stack maps to itself)
  std::vector<int64_t> smap(std::max<int64_t>(ktot, 1));
  for (int64_t g = 0; g < ktot; g++) smap[g] = g;
  {
    std::vector<int64_t> side_row[2];
    side_row[0].assign(hh.far.size(), 0);
    side_row[1].assign(hh.far.size(), 0);
    for (int c = 0; c < nc; c++)
      for (size_t i = 0; i < slots[c].size(); i++)
        side_row[slots[c][i].second][slots[c][i].first] = slot_base[c] + slot_col[c][i];
    for (size_t b = 0; b < hh.far.size(); b++)
      for (int64_t l = 0; l < block_width((int)b); l++) {
        smap[side_row[0][b] + l] = side_row[1][b] + l;
        smap[side_row[1][b] + l] = side_row[0][b] + l;
      }
  }
  // factor stacks
  std::vector<double> facv((size_t)std::max<int64_t>(facn, 1), 0.0);
  for (int c = 0; c < nc; c++) {
    const int64_t nr = csize(c);
    for (size_t i = 0; i < slots[c].size(); i++) {
      const HFar& fb = hh.far[slots[c][i].first];
      const std::vector<double>& src = slots[c][i].second == 0 ? fb.u : fb.v;
      for (int l = 0; l < fb.k; l++)
        for (int64_t r = 0; r < nr; r++) facv[fac_off[c] + r * K[c] + slot_col[c][i] + l] = src[(size_t)l * nr + r];
    }
  }
  // near stacks per leaf
  std::vector<int> leaves;
  for (int c = 0; c < nc; c++)
    if (cl[c].child[0] < 0) leaves.push_back(c);
  std::sort(leaves.begin(), leaves.end(), [&](int a, int b) { return cl[a].begin < cl[b].begin; });
  std::vector<int> leaf_id(nc, -1);
  for (size_t i = 0; i < leaves.size(); i++) leaf_id[leaves[i]] = (int)i;
  struct NP {
    int sigma;
    int64_t pair;
    bool transposed;
  };
  std::vector<std::vector<NP>> partners(leaves.size());
  for (size_t p = 0; p < hh.near.size(); p++) {
    const auto [t, s] = hh.near[p];
    partners[leaf_id[t]].push_back({s, (int64_t)p, false});
    if (s != t) partners[leaf_id[s]].push_back({t, (int64_t)p, true});
  }
  std::vector<int64_t> kn(leaves.size()), near_off(leaves.size());
  int64_t nearn = 0;
  for (size_t l = 0; l < leaves.size(); l++) {
    std::sort(partners[l].begin(), partners[l].end(),
              [&](const NP& a, const NP& b) { return cl[a.sigma].begin < cl[b.sigma].begin; });
    int64_t k = 0;
    for (auto& np : partners[l]) k += csize(np.sigma);
    kn[l] = (k + 3) / 4 * 4;
    near_off[l] = nearn;
    nearn += csize(leaves[l]) * kn[l];
  }
  std::vector<double> nearv((size_t)std::max<int64_t>(nearn, 1), 0.0);
  std::vector<std::vector<int64_t>> pcol(leaves.size());
  for (size_t l = 0; l < leaves.size(); l++) {
    const int tau = leaves[l];
    const int64_t nt = csize(tau);
    int64_t col = 0;
    for (auto& np : partners[l]) {
      pcol[l].push_back(col);
      const int64_t ns = csize(np.sigma);
      const double* tile = hh.near_val.data() + hh.near_off[np.pair];
      for (int64_t a = 0; a < nt; a++)
        for (int64_t b = 0; b < ns; b++) {
          // stored tile is (t rows) x (s cols) for the pair (t, s)
          const double v = np.transposed ? tile[b * nt + a] : tile[a * ns + b];
          nearv[near_off[l] + a * kn[l] + col + b] = v;
        }
      col += ns;
    }
  }
  // phase-1 work list
  std::vector<P1Item> p1;
  std::vector<P1Reduce> p1r;
  int64_t part_rows = 0;
  const int BQ = 64;
  for (int c = 0; c < nc; c++) {
    if (K[c] == 0) continue;
    const int64_t nr = csize(c);
    const int nch = (int)cdiv(nr, kChunkRows);
    for (int64_t q0 = 0; q0 < K[c]; q0 += BQ) {
      const int nq = (int)std::min<int64_t>(BQ, K[c] - q0);
      const int64_t base = part_rows;
      for (int ch = 0; ch < nch; ch++) {
        P1Item it{};
        it.fac_off = fac_off[c];
        it.r0 = ch * kChunkRows;
        it.nr = (int)std::min<int64_t>(kChunkRows, nr - it.r0);
        it.x_row = cl[c].begin + it.r0;
        it.out_row = nch == 1 ? -1 : base + (int64_t)ch * nq;
        it.map_off = slot_base[c] + q0;
        it.K = (int)K[c];
        it.q0 = (int)q0;
        it.nq = nq;
        p1.push_back(it);
      }
      if (nch > 1) {
        p1r.push_back(P1Reduce{base, slot_base[c] + q0, nq, nch});
        part_rows += (int64_t)nch * nq;
      }
    }
  }
  // phase-2 segments per leaf (row chunks of at most BM rows)
  const int BM = h->prec == FKF_FP64 ? TileCfg<double>::BM : TileCfg<float>::BM;
  std::vector<P2Seg> segs;
  std::vector<P2Leaf> p2;
  int max_leaf = 0;
  for (size_t l = 0; l < leaves.size(); l++) {
    const int tau = leaves[l];
    const int seg0 = (int)segs.size();
    for (int c = tau; c >= 0; c = cl[c].parent) {
      if (K[c] == 0) continue;
      P2Seg s{};
      s.a_off = fac_off[c] + (cl[tau].begin - cl[c].begin) * K[c];
      s.b_row = slot_base[c];
      s.lda = (int)K[c];
      s.K = (int)K[c];
      s.near = 0;
      segs.push_back(s);
    }
    for (size_t i = 0; i < partners[l].size(); i++) {
      P2Seg s{};
      s.a_off = near_off[l] + pcol[l][i];
      s.b_row = cl[partners[l][i].sigma].begin;
      s.lda = (int)kn[l];
      s.K = (int)csize(partners[l][i].sigma);
      s.near = 1;
      segs.push_back(s);
    }
    const int nt = (int)csize(tau);
    max_leaf = std::max(max_leaf, nt);
    for (int r0 = 0; r0 < nt; r0 += BM) {
      P2Leaf lf{};
      lf.row0 = cl[tau].begin + r0;
      lf.rows = std::min(BM, nt - r0);
      lf.seg0 = seg0;
      lf.nseg = (int)segs.size() - seg0;
      lf.pad = r0;  // row offset inside the leaf (applied to every segment's A)
      p2.push_back(lf);
    }
  }
  // tensor-core schedules (FP32 operators).  The vector operands are split
  // into TF32 hi/lo chunks of 16 rows before the products: X per leaf (rows
  // of a leaf padded to a multiple of 16) and the slot workspace per cluster
  // (its K_c slots padded to a multiple of 16), so every K-chunk of a product
  // is one contiguous block.  Phase-1 items cover whole leaves (row groups of
  // at most 2048 rows of a cluster); phase-2 tiles are 128 consecutive rows
  // with merged segments.
  TcUpload tu;
  if (h->prec == FKF_FP32) {
    const int L = (int)leaves.size();
    std::vector<int64_t> xchunk0(L + 1, 0);
    std::unordered_map<int64_t, int64_t> leaf_by_begin;
    for (int l = 0; l < L; l++) {
      const int c = leaves[l];
      leaf_by_begin[cl[c].begin] = l;
      xchunk0[l] = (int64_t)tu.xmap.size();
      for (int64_t r = 0; r < csize(c); r += 16)
        tu.xmap.push_back(TcXChunk{cl[c].begin + r, (int32_t)std::min<int64_t>(16, csize(c) - r), 0});
    }
    xchunk0[L] = (int64_t)tu.xmap.size();
    std::vector<int64_t> zchunk0(nc, -1), tcpos(std::max<int64_t>(ktot, 1), 0);
    std::unordered_map<int64_t, int64_t> z_by_slot_base;
    int64_t nz = 0;
    for (int c = 0; c < nc; c++) {
      if (K[c] == 0) continue;
      zchunk0[c] = nz;
      z_by_slot_base[slot_base[c]] = nz;
      for (int64_t q = 0; q < K[c]; q++) tcpos[slot_base[c] + q] = nz * 16 + q;
      nz += cdiv(K[c], 16);
    }
    tu.nz = nz;
    tu.slotmap.resize(std::max<int64_t>(ktot, 1), 0);
    for (int64_t g = 0; g < ktot; g++) tu.slotmap[g] = tcpos[smap[g]];
    // leaf range of a cluster (its leaves are consecutive in cluster order)
    auto leaf_range = [&](int c, int& la, int& lb) {
      int a = c, b = c;
      while (cl[a].child[0] >= 0) a = cl[a].child[0];
      while (cl[b].child[1] >= 0) b = cl[b].child[1];
      la = leaf_id[a];
      lb = leaf_id[b] + 1;
    };
    int64_t tparts = 0;
    for (int c = 0; c < nc; c++) {
      if (K[c] == 0) continue;
      int la, lb;
      leaf_range(c, la, lb);
      std::vector<std::pair<int, int>> groups;  // leaf ranges of at most kChunkRows rows
      for (int l = la; l < lb;) {
        int e = l;
        int64_t rows = 0;
        while (e < lb && (e == l || rows + csize(leaves[e]) <= kChunkRows)) rows += csize(leaves[e++]);
        groups.push_back({l, e});
        l = e;
      }
      const int ng = (int)groups.size();
      // slot tiles of at most 128 (the MMA's N), balanced: N is the tile's
      // slot count rounded up to 16, so equal tiles waste the least
      const int64_t ntq = cdiv(K[c], 128);
      const int64_t tq = (cdiv(K[c], ntq) + 3) / 4 * 4;
      for (int64_t q0 = 0; q0 < K[c]; q0 += tq) {
        const int nq = (int)std::min<int64_t>(tq, K[c] - q0);
        const int64_t base = tparts;
        for (int g = 0; g < ng; g++) {
          P1Item it{};
          it.fac_off = fac_off[c];
          it.x_row = xchunk0[groups[g].first];  // first X chunk
          it.nchunk = (int)(xchunk0[groups[g].second] - xchunk0[groups[g].first]);
          it.out_row = ng == 1 ? -1 : base + (int64_t)g * nq;
          it.map_off = slot_base[c] + q0;
          it.K = (int)K[c];
          it.q0 = (int)q0;
          it.nq = nq;
          tu.items.push_back(it);
          // operator chunks: the item's leaves, 16 rows at a time
          std::vector<TcAChunk> ch;
          for (int l = groups[g].first; l < groups[g].second; l++) {
            const int lc = leaves[l];
            for (int64_t r = 0; r < csize(lc); r += 16) {
              TcAChunk a{};
              a.src_off = fac_off[c] + (cl[lc].begin - cl[c].begin + r) * K[c] + q0;
              a.si = 1;
              a.sk = (int32_t)K[c];
              a.row_lo = 0;
              a.row_hi = nq;
              a.kv = (int32_t)std::min<int64_t>(16, csize(lc) - r);
              a.near = 0;
              a.phase = 1;
              a.s_off = slot_base[c] + q0;
              a.k_off = -1;
              ch.push_back(a);
            }
          }
          tu.item_chunks.push_back(std::move(ch));
        }
        if (ng > 1) {
          tu.reduces.push_back(P1Reduce{base, slot_base[c] + q0, nq, ng});
          tparts += (int64_t)ng * nq;
        }
      }
    }
    hmat_build_tc_schedule(p2, segs, tu.tiles, tu.segs);
    // B operands of the phase-2 segments as chunk indices
    for (TcSeg& sg : tu.segs) {
      if (sg.near) {
        sg.b_row = xchunk0[leaf_by_begin.at(sg.b_row)];
      } else {
        sg.b_row = z_by_slot_base.at(sg.b_row);
      }
    }
    tu.part_rows = std::max(tparts, part_rows);
  }
  // FP64 operators: the schedule of the integer-slice tensor-core engine
  // (engine 3).  Vector chunks as above (X per leaf, the slot workspace per
  // cluster, 16 rows each); phase-1 items of at most 64 slots over leaf
  // groups of at most kChunkRows rows; phase-2 tiles of at most 64 points of
  // one leaf, whose segments are the leaf's ancestors' factor rows and its
  // near blocks.
  OzUpload ou;
  if (h->prec == FKF_FP64) {
    const int L = (int)leaves.size();
    std::vector<int64_t> xchunk0(L + 1, 0);
    for (int l = 0; l < L; l++) {
      const int c = leaves[l];
      xchunk0[l] = (int64_t)ou.xmap.size();
      for (int64_t r = 0; r < csize(c); r += 16)
        ou.xmap.push_back(TcXChunk{cl[c].begin + r, (int32_t)std::min<int64_t>(16, csize(c) - r), 0});
    }
    xchunk0[L] = (int64_t)ou.xmap.size();
    std::unordered_map<int64_t, int64_t> leaf_by_begin;
    for (int l = 0; l < L; l++) leaf_by_begin[cl[leaves[l]].begin] = l;
    std::vector<int64_t> zchunk0(nc, -1), pos(std::max<int64_t>(ktot, 1), 0);
    int64_t nz = 0;
    for (int c = 0; c < nc; c++) {
      if (K[c] == 0) continue;
      zchunk0[c] = nz;
      for (int64_t q = 0; q < K[c]; q++) pos[slot_base[c] + q] = nz * 16 + q;
      nz += cdiv(K[c], 16);
    }
    ou.nz = nz;
    ou.slotpos.resize(std::max<int64_t>(ktot, 1), 0);
    for (int64_t g = 0; g < ktot; g++) ou.slotpos[g] = pos[smap[g]];
    // scales of the slices (powers of two, so that every scaling is exact)
    auto pow2ceil = [](double x) { return x > 0 ? std::ldexp(1.0, std::ilogb(x) + 1) : 1.0; };
    ou.sig_slot.assign(std::max<int64_t>(ktot, 1), 1.0);
    ou.q_slot.assign(std::max<int64_t>(ktot, 1), 1.0);
    ou.q_shift.assign(std::max<int64_t>(ktot, 1), 0);
    for (int c = 0; c < nc; c++)
      for (int64_t q = 0; q < K[c]; q++) {
        double mx = 0, l1 = 0;
        for (int64_t r = 0; r < csize(c); r++) {
          const double v = std::fabs(facv[fac_off[c] + r * K[c] + q]);
          mx = std::max(mx, v);
          l1 += v;
        }
        ou.sig_slot[slot_base[c] + q] = pow2ceil(mx);
        ou.q_slot[slot_base[c] + q] = pow2ceil(l1);
        ou.q_shift[slot_base[c] + q] = std::ilogb(ou.q_slot[slot_base[c] + q]) - std::ilogb(ou.sig_slot[slot_base[c] + q]);
      }
    ou.q_pos.assign((size_t)std::max<int64_t>(nz, 1) * 16, 1.0);
    for (int64_t g = 0; g < ktot; g++) ou.q_pos[ou.slotpos[g]] = ou.q_slot[g];
    // phase-1 items
    int64_t parts = 0;
    for (int c = 0; c < nc; c++) {
      if (K[c] == 0) continue;
      int a = c, b = c;
      while (cl[a].child[0] >= 0) a = cl[a].child[0];
      while (cl[b].child[1] >= 0) b = cl[b].child[1];
      const int la = leaf_id[a], lb = leaf_id[b] + 1;
      std::vector<std::pair<int, int>> groups;
      for (int l = la; l < lb;) {
        int e = l;
        int64_t rows = 0;
        while (e < lb && (e == l || rows + csize(leaves[e]) <= kChunkRows)) rows += csize(leaves[e++]);
        groups.push_back({l, e});
        l = e;
      }
      const int ng = (int)groups.size();
      const int64_t ntq = cdiv(K[c], 64);
      const int64_t tq = (cdiv(K[c], ntq) + 3) / 4 * 4;
      for (int64_t q0 = 0; q0 < K[c]; q0 += tq) {
        const int nq = (int)std::min<int64_t>(tq, K[c] - q0);
        const int64_t base = parts;
        for (int g = 0; g < ng; g++) {
          OzItem it{};
          it.x_chunk0 = xchunk0[groups[g].first];
          it.nchunk = (int)(xchunk0[groups[g].second] - xchunk0[groups[g].first]);
          it.b_chunk0 = (int64_t)ou.bchunks.size();
          it.map_off = slot_base[c] + q0;
          it.out_row = ng == 1 ? -1 : base + (int64_t)g * nq;
          it.nq = nq;
          ou.items.push_back(it);
          for (int l = groups[g].first; l < groups[g].second; l++) {
            const int lc = leaves[l];
            for (int64_t r = 0; r < csize(lc); r += 16) {
              OzBChunk bc{};
              bc.src_off = fac_off[c] + (cl[lc].begin - cl[c].begin + r) * K[c] + q0;
              bc.si = 1;
              bc.sk = (int32_t)K[c];
              bc.rows = nq;
              bc.kv = (int32_t)std::min<int64_t>(16, csize(lc) - r);
              bc.phase = 1;
              bc.s_off = slot_base[c] + q0;
              bc.k_off = -1;
              ou.bchunks.push_back(bc);
            }
          }
        }
        if (ng > 1) {
          ou.reduces.push_back(P1Reduce{base, slot_base[c] + q0, nq, ng});
          parts += (int64_t)ng * nq;
        }
      }
    }
    ou.part_rows = parts;
    // phase-2 tiles and the point scales
    ou.sig_pt.assign((size_t)std::max<int64_t>(hh.n, 1), 1.0);
    for (int l = 0; l < L; l++) {
      const int tau = leaves[l];
      const int64_t nt = csize(tau);
      for (int64_t r0 = 0; r0 < nt; r0 += 64) {
        OzTile t{};
        t.row0 = cl[tau].begin + r0;
        t.rows = (int)std::min<int64_t>(64, nt - r0);
        t.seg0 = (int)ou.segs.size();
        t.b_chunk0 = (int64_t)ou.bchunks.size();
        std::vector<double> rmax((size_t)t.rows, 0.0);
        for (int c = tau; c >= 0; c = cl[c].parent) {
          if (K[c] == 0) continue;
          const int64_t a_row = t.row0 - cl[c].begin;
          ou.segs.push_back(OzSeg{zchunk0[c], (int32_t)cdiv(K[c], 16), 0});
          for (int64_t k0 = 0; k0 < K[c]; k0 += 16) {
            OzBChunk bc{};
            bc.src_off = fac_off[c] + a_row * K[c] + k0;
            bc.si = (int32_t)K[c];
            bc.sk = 1;
            bc.rows = t.rows;
            bc.kv = (int32_t)std::min<int64_t>(16, K[c] - k0);
            bc.phase = 2;
            bc.s_off = t.row0;
            bc.k_off = zchunk0[c] * 16 + k0;
            ou.bchunks.push_back(bc);
          }
          for (int i = 0; i < t.rows; i++)
            for (int64_t q = 0; q < K[c]; q++)
              rmax[i] = std::max(rmax[i], std::fabs(facv[fac_off[c] + (a_row + i) * K[c] + q]) *
                                              ou.q_pos[zchunk0[c] * 16 + q]);
        }
        for (size_t i = 0; i < partners[l].size(); i++) {
          const int sg = partners[l][i].sigma;
          const int64_t ns = csize(sg);
          ou.segs.push_back(OzSeg{xchunk0[leaf_by_begin.at(cl[sg].begin)], (int32_t)cdiv(ns, 16), 1});
          for (int64_t k0 = 0; k0 < ns; k0 += 16) {
            OzBChunk bc{};
            bc.src_off = near_off[l] + r0 * kn[l] + pcol[l][i] + k0;
            bc.si = (int32_t)kn[l];
            bc.sk = 1;
            bc.rows = t.rows;
            bc.kv = (int32_t)std::min<int64_t>(16, ns - k0);
            bc.near = 1;
            bc.phase = 2;
            bc.s_off = t.row0;
            bc.k_off = -1;
            ou.bchunks.push_back(bc);
          }
          for (int ii = 0; ii < t.rows; ii++)
            for (int64_t b = 0; b < ns; b++)
              rmax[ii] = std::max(rmax[ii], std::fabs(nearv[near_off[l] + (r0 + ii) * kn[l] + pcol[l][i] + b]));
        }
        t.nseg = (int)ou.segs.size() - t.seg0;
        t.nchunk = (int)((int64_t)ou.bchunks.size() - t.b_chunk0);
        for (int i = 0; i < t.rows; i++) ou.sig_pt[t.row0 + i] = pow2ceil(rmax[i]);
        ou.tiles.push_back(t);
      }
    }
  }
  // upload
  std::vector<char> tmp;
  auto upload_vals = [&](DevBuf& dst, const std::vector<double>& src) -> fkf_status {
    tmp.resize(src.size() * w);
    if (w == 8)
      fill_typed<double>(tmp.data(), src.data(), src.size());
    else
      fill_typed<float>(tmp.data(), src.data(), src.size());
    return dev_upload(ctx, dst, tmp.data(), tmp.size());
  };
  FKF_TRY(upload_vals(h->fac, facv));
  FKF_TRY(upload_vals(h->nearv, nearv));
  std::vector<char>().swap(tmp);
  h->ktot = ktot;  // the tensor-core upload sizes its per-slot scales by it
  if (h->prec == FKF_FP32) FKF_TRY(hmat_upload_tc(h, tu));
  if (h->prec == FKF_FP64) FKF_TRY(hmat_upload_oz(h, ou));
  FKF_TRY(dev_upload(ctx, h->slotmap, smap.data(), smap.size() * sizeof(int64_t)));
  if (!p1.empty()) FKF_TRY(dev_upload(ctx, h->p1items, p1.data(), p1.size() * sizeof(P1Item)));
  if (!p1r.empty()) FKF_TRY(dev_upload(ctx, h->p1red, p1r.data(), p1r.size() * sizeof(P1Reduce)));
  FKF_TRY(dev_upload(ctx, h->p2seg, segs.data(), std::max<size_t>(segs.size(), 1) * sizeof(P2Seg)));
  FKF_TRY(dev_upload(ctx, h->p2leaf, p2.data(), p2.size() * sizeof(P2Leaf)));
  h->n_p1 = (int64_t)p1.size();
  h->n_p1red = (int64_t)p1r.size();
  h->n_leaf = (int64_t)p2.size();
  h->ktot = ktot;
  h->part_rows = part_rows;
  h->max_leaf = max_leaf;
  // statistics
  fkf_hmat_info& in = h->info;
  in.n = hh.n;
  in.dim = hh.dim;
  in.precision = h->prec;
  in.n_clusters = nc;
  in.n_leaves = (int64_t)leaves.size();
  in.n_far = (int64_t)hh.far.size();
  in.n_near = (int64_t)hh.near.size();
  int64_t fe = 0, maxk = 0, near_used = 0;
  double ksum = 0;
  for (auto& fb : hh.far) {
    fe += (int64_t)fb.k * (csize(fb.t) + csize(fb.s));
    maxk = std::max<int64_t>(maxk, fb.k);
    ksum += fb.k;
  }
  for (auto [t, s] : hh.near) near_used += (t == s ? 1 : 2) * csize(t) * csize(s);
  in.far_entries = fe;
  in.near_entries = (int64_t)hh.near_val.size();
  in.max_rank = maxk;
  in.mean_rank = hh.far.empty() ? 0.0 : ksum / hh.far.size();
  in.flops_per_col = 2 * (2 * fe + near_used);
  in.bytes_per_col = 2 * hh.n * (int64_t)w;
  in.operator_bytes = (fe + in.near_entries) * (int64_t)w;
  in.device_bytes = hmat_device_bytes(h);
  in.build_seconds = hh.build_seconds;
  return FKF_OK;
}

// ----------------------------------------------------------------------------
// Apply without allocating: the phase-1 slot workspace (Zmix) and the
// split-reduction partials live in one file-scope device array of fixed size
// instead of cudaMalloc'd buffers.  Columns are processed in panels as wide
// as that array allows.  Every call (on any stream) shares the array, so
// calls that overlap on the GPU race; nothing in it needs to start at zero
// (phase 1 writes every slot row and every partial it later reads).
// ----------------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_noalloc_scratch[FKF_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on ctx->device, looked up once per device
// (with that device current) and cached.
fkf_status noalloc_scratch(fkf_ctx* ctx, void** out) {
  if (ctx->device < 0 || ctx->device >= kMaxDevices)
    return set_err(ctx, FKF_EINVAL, "apply_noalloc: device index %d >= %d", ctx->device, kMaxDevices);
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[ctx->device]) {
    int prev = 0;
    FKF_CUDA(ctx, cudaGetDevice(&prev));
    FKF_CUDA(ctx, cudaSetDevice(ctx->device));
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    cudaSetDevice(prev);
    if (e != cudaSuccess || !p)
      return set_err(ctx, FKF_ECUDA, "apply_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
    g_noalloc_ptr[ctx->device] = p;
  }
  *out = g_noalloc_ptr[ctx->device];
  return FKF_OK;
}

template <typename T>
fkf_status apply_noalloc_impl(fkf_hmat* h, const T* X, int64_t ldx, T* Y, int64_t ldy, int64_t ncols) {
  fkf_ctx* ctx = h->ctx;
  void* base = nullptr;
  FKF_TRY(noalloc_scratch(ctx, &base));
  const int64_t rows = std::max<int64_t>(h->ktot, 1) + h->part_rows;
  const int64_t P = std::min<int64_t>(ncols, (int64_t)(FKF_NOALLOC_SCRATCH_BYTES / (rows * (int64_t)sizeof(T))));
  if (P < 1)
    return set_err(ctx, FKF_EINVAL,
                   "apply_noalloc: operator needs %lld bytes of scratch per column; the static scratch holds %lld "
                   "bytes (use fkf_hmatrix_apply_clustered)",
                   (long long)(rows * (int64_t)sizeof(T)), (long long)FKF_NOALLOC_SCRATCH_BYTES);
  T* zmix = reinterpret_cast<T*>(base);
  T* part = zmix + std::max<int64_t>(h->ktot, 1) * P;
  constexpr int BN = TileCfg<T>::BN;
  for (int64_t c0 = 0; c0 < ncols; c0 += P) {
    const int nc = (int)std::min<int64_t>(P, ncols - c0);
    const int ntile = (int)cdiv(nc, BN);
    if (h->n_p1 > 0) {
      k_phase1<T><<<dim3((unsigned)h->n_p1, ntile), kTileThreads, 0, ctx->stream>>>(
          h->p1items.as<P1Item>(), h->fac.as<T>(), X + c0, ldx, nc, h->slotmap.as<int64_t>(), zmix, part, P);
      FKF_LAUNCHED(ctx);
    }
    if (h->n_p1red > 0) {
      k_phase1_reduce<T><<<dim3((unsigned)h->n_p1red, 4), 256, 0, ctx->stream>>>(
          h->p1red.as<P1Reduce>(), part, h->slotmap.as<int64_t>(), zmix, P, nc);
      FKF_LAUNCHED(ctx);
    }
    k_phase2<T><<<dim3((unsigned)h->n_leaf, ntile), kTileThreads, 0, ctx->stream>>>(
        h->p2leaf.as<P2Leaf>(), h->p2seg.as<P2Seg>(), h->fac.as<T>(), h->nearv.as<T>(), zmix, P, X + c0, ldx,
        Y + c0, ldy, nc);
    FKF_LAUNCHED(ctx);
  }
  return FKF_OK;
}
}  // namespace

fkf_status hmat_apply_clustered_noalloc(fkf_hmat* h, const void* X, int64_t ldx, void* Y, int64_t ldy,
                                        int64_t ncols) {
  if (ncols <= 0) return FKF_OK;
  if (h->prec == FKF_FP64)
    return apply_noalloc_impl<double>(h, (const double*)X, ldx, (double*)Y, ldy, ncols);
  return apply_noalloc_impl<float>(h, (const float*)X, ldx, (float*)Y, ldy, ncols);
}
