// H-apply of FP64 operators on the 5th-generation tensor cores (engine 3):
// FP64 products assembled from exact products of small integer slices, the
// error-free splitting of Ozaki, Ogita, Oishi and Rump ("Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 59, 2012), run as
// FP16 MMAs whose FP32 sums stay exact.
//
// Slices.  Every value is first scaled by a power of two (exact) into
// [-1, 1]: operator rows by a scale per row, vector columns by a scale per
// column.  A value x in [-1, 1] is then
//     x = sum_{i<7} d_i 2^(-7(i+1)) + r,   d_0 in [-128, 128], d_i in [-64, 63],
// the balanced base-128 digits of the integer rint(2^49 x) (|r| <= 2^-50),
// taken with integer operations: every d_i is an integer held exactly by
// FP16.  A dot product sum_k a_k b_k
// of two such values is sum_{i,j} 2^(-7(i+j+2)) S_ij with integer
// S_ij = sum_k d^a_{k,i} d^b_{k,j}.  The 28 products with i + j <= 6 are
// kept (the dropped ones lie below 2^-56 of the scales); those of one weight
// w = i + j accumulate in one FP32 TMEM accumulator.  Over a block of 512 K
// (32 chunks of 16) every partial sum of weight w <= 5 is an integer of
// magnitude <= 2^24, hence exact in FP32 (the MMA multiplies FP16 integers
// exactly).  Weights 0..3 are summed exactly: after each block the epilogue
// moves them into one 64-bit integer per output (sum_w T_w 2^(7(3-w)), below
// 2^44 per block) and releases their accumulators; weights 4..6 lie 2^-28 and
// further below weight 0, where the rounding of an FP32 sum (2^-24 of it) is
// below 2^-52 of the result, so they accumulate in TMEM over the whole tile,
// and the MMAs of the next block start on them while the epilogue moves the
// exact sums.  At the end of a tile everything is combined in FP64 with the
// scales.
//
// The products run in the tensor-core layout of happly_tc.cu, with the MMA
// roles of its phase 1 in both phases: the vector operand (X or the slot
// workspace; rows = 128 vector columns, K-major) is A, the operator (rows =
// 64 slots in phase 1, 64 points of one leaf in phase 2) is B, so the
// accumulator lanes are vector columns and every epilogue store is a row of
// consecutive vector columns.
//   phase 1  Z[n, g] = sum_{k in c} X[k, n] V[k, g]   for the slots g of a
//            cluster c, written (sliced, over the bound tau_n Q_g, with Q_g
//            >= the L1 norm of V's column) at the workspace position of the
//            partner slot, or as FP64 partial rows when the cluster's rows
//            are split over several leaf groups;
//   phase 2  Y[i, n] = sum_{far} U[i, g] Q_g Z'[n, g] + sum_{near} G[i, k] X'[k, n]
//            times tau_n and the row scale.
// One persistent CTA per SM, warp-specialised as in happly_tc.cu: a
// producer thread (two bulk copies per chunk), an MMA thread (28 MMAs per
// chunk), eight epilogue warps (two per TMEM lane quarter, one per half of
// the 64 operator rows).  Every mbarrier wait is bounded; an expired wait
// sets a flag, every role unwinds and the host reports FKF_ETIMEOUT.
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <type_traits>

#include "common.h"
#include "dense.h"
#include "umma.cuh"

namespace {

constexpr int kSl = 7;                   // slices per value
constexpr int kW = 7;                    // weights w = i + j kept (0 .. 6)
constexpr int kWx = 4;                   // weights 0 .. 3 are summed exactly (64-bit integers)
constexpr int kM = 128;                  // vector columns per tile (MMA M, TMEM lanes)
constexpr int kN = 64;                   // operator rows per tile (MMA N)
constexpr int kK = 16;                   // K per chunk = one kind::f16 MMA
constexpr int kAPlane = kM * kK * 2;     // one slice plane of a vector chunk (4 KB)
constexpr int kBPlane = kN * kK * 2;     // one slice plane of an operator chunk (2 KB)
constexpr int kAChunk = kSl * kAPlane;   // 28 KB
constexpr int kBChunk = kSl * kBPlane;   // 14 KB
constexpr int kStage = kAChunk + kBChunk;
constexpr int kStages = 4;
constexpr int kKBlock = 32;              // chunks per exact block (512 K)
constexpr uint32_t kSBO = 256;           // K-major FP16 core matrices: next 8-row group
constexpr int kEpiWarps = 8;
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr int kQ = 8;
constexpr uint32_t kTmemCols = 512;      // 7 weights x 64 columns used
constexpr uint32_t kMaxPolls = 1u << 22;
constexpr uint32_t kIdesc = umma::idesc_f16(kM, kN);
constexpr int FULL = 0, EMPTY = FULL + kStages, AF = EMPTY + kStages, AE = AF + 1, FIN = AE + 1, QF = FIN + 1,
              QE = QF + kQ, NBAR = QE + kQ;
constexpr int kBarBytes = 256;
constexpr int kTail = 512;
constexpr int kSmem = kStages * kStage + kTail;
static_assert(NBAR * 8 <= kBarBytes, "barrier area");
static_assert(kSmem <= 232448, "shared memory per CTA");

struct OzQ {
  int64_t id;   // tile index, -1: no more tiles
  int32_t nch;  // K-chunks of the tile
  int32_t pad;
};

struct OzSmem {
  uint8_t* base;
  uint64_t* bar;
  uint32_t* tmem_slot;
  int* fail;
  OzQ* q;
  uint32_t polls;
  __device__ __forceinline__ uint8_t* a(int s) const { return base + s * kStage; }
  __device__ __forceinline__ uint8_t* b(int s) const { return base + s * kStage + kAChunk; }
  __device__ __forceinline__ bool failed() const { return *reinterpret_cast<volatile int*>(fail) != 0; }
  __device__ __forceinline__ void set_fail() const { atomicExch(fail, 1); }
};

__device__ __forceinline__ bool wait_bar(const OzSmem& s, int i, uint32_t parity) {
  if (umma::mbar_wait(&s.bar[i], parity, s.polls)) return true;
  s.set_fail();
  return false;
}
__device__ __forceinline__ bool wait_unwind(const OzSmem& s, int i, uint32_t parity) {
  if (umma::mbar_wait(&s.bar[i], parity, kMaxPolls)) return true;
  s.set_fail();
  return false;
}

// byte offset of element (row, k) of one slice plane, K-major, no swizzle
__device__ __forceinline__ uint32_t off16(int row, int k) {
  return (uint32_t)((row >> 3) * kSBO + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// power of two >= |x| (1 for 0): the scale that maps a row or column into [-1, 1]
__device__ __forceinline__ double pow2_ceil(double x) {
  if (!(x > 0.0) || isinf(x)) return 1.0;
  int e;
  frexp(x, &e);  // x = f 2^e, f in [0.5, 1)
  return ldexp(1.0, e);
}

// x in [-1, 1] on the grid of the slices: rint(2^49 x) (the scaling by a
// power of two is exact; one conversion).
__device__ __forceinline__ int64_t grid49(double x) { return __double2ll_rn(x * 0x1p49); }

// The seven slices of z = rint(2^49 x), |z| <= 2^49, as FP16 bit patterns:
// balanced base-128 digits, z = sum_i d_i 128^(6-i), d_i in [-64, 63] for
// i >= 1 and |d_0| <= 128 (integer operations only).
__device__ __forceinline__ void digits7(int64_t z, uint16_t (&d)[kSl]) {
#pragma unroll
  for (int i = kSl - 1; i > 0; i--) {
    const int64_t r = ((z + 64) & 127) - 64;
    d[i] = __half_as_ushort(__int2half_rn((int)r));
    z = (z - r) >> 7;
  }
  d[0] = __half_as_ushort(__int2half_rn((int)z));
}

// ---- work descriptions ----------------------------------------------------
struct OzPh1 {
  const OzItem* items;
  const uint8_t* xs;  // sliced X of the pass
  const uint8_t* ops; // sliced operator stream
  uint8_t* zs;        // sliced slot workspace of the pass
  double* part;       // FP64 partial rows (clusters over several leaf groups)
  int64_t ldp;
  const int64_t* slotpos;
  const double* sig;  // per natural slot: row scale of its operator column
  const int32_t* qsh; // per natural slot: log2(bound of its products / sig)
  int nct, ncols;
};

struct OzPh2 {
  const OzTile* tiles;
  const OzSeg* segs;
  const uint8_t* xs;
  const uint8_t* zs;
  const uint8_t* ops;
  double* Y;
  int64_t ldy;
  const double* sig;  // per point
  const double* tau;  // per column of the pass
  int nct, ncols;
};

// Dense GEMM C = alpha op(A) op(B) + beta C: tile (row tile w of 128 rows of
// C, column tile ct of 64 columns); op(A) sliced per row (A chunks of row
// tile w: as + (w * nch + c) * kAChunk), op(B) sliced per column of C (B
// chunks of column tile ct: bs + (ct * nch + c) * kBChunk).
struct OzPhGemm {
  const uint8_t* as;
  const uint8_t* bs;
  double* C;
  int64_t ldc;
  const double* sa;  // row scales of op(A)
  const double* sb;  // column scales of op(B)
  double alpha, beta;
  int M, N, nch;
  int nct;
};

__device__ __forceinline__ int tile_nch(const OzPh1& p, int64_t w) { return p.items[w].nchunk; }
__device__ __forceinline__ int tile_nch(const OzPh2& p, int64_t w) { return p.tiles[w].nchunk; }
__device__ __forceinline__ int tile_nch(const OzPhGemm& p, int64_t) { return p.nch; }

// ---- roles ----------------------------------------------------------------
__device__ __forceinline__ bool next_tile(const OzSmem& s, int qi, int64_t& id, int& nch) {
  const int slot = qi % kQ;
  if (!wait_bar(s, QF + slot, (uint32_t)(qi / kQ) & 1)) return false;
  volatile OzQ* e = &s.q[slot];
  id = e->id;
  nch = e->nch;
  umma::mbar_arrive(&s.bar[QE + slot]);
  return id >= 0;
}

// One chunk (vector chunk a, operator chunk b) into stage st of the g-th
// chunk overall.  Returns false when the CTA failed.
__device__ __forceinline__ bool load_chunk(const OzSmem& s, int64_t& g, const uint8_t* a, const uint8_t* b) {
  const int st = (int)(g % kStages);
  if (s.failed()) return false;
  if (g >= kStages && !wait_bar(s, EMPTY + st, (uint32_t)((g / kStages) - 1) & 1)) return false;
  umma::mbar_arrive_expect_tx(&s.bar[FULL + st], (uint32_t)kStage);
  umma::bulk_g2s(s.a(st), a, (uint32_t)kAChunk, &s.bar[FULL + st]);
  umma::bulk_g2s(s.b(st), b, (uint32_t)kBChunk, &s.bar[FULL + st]);
  g++;
  return true;
}

template <class Ph>
__device__ __forceinline__ void producer(const OzSmem& s, const Ph& ph, int64_t ntiles, unsigned long long* counter,
                                         int64_t& g) {
  g = 0;
  for (int qi = 0;; qi++) {
    const int64_t raw = (int64_t)atomicAdd(counter, 1ull);
    const int64_t id = raw < ntiles ? raw : -1;
    const int64_t w = id >= 0 ? id / ph.nct : 0;
    const int ct = id >= 0 ? (int)(id % ph.nct) : 0;
    const int nch = id >= 0 ? tile_nch(ph, w) : 0;
    const int slot = qi % kQ;
    if (qi >= kQ && !wait_bar(s, QE + slot, (uint32_t)((qi / kQ) - 1) & 1)) return;
    volatile OzQ* e = &s.q[slot];
    e->id = id;
    e->nch = nch;
    umma::mbar_arrive(&s.bar[QF + slot]);
    if (id < 0) return;
    if constexpr (std::is_same<Ph, OzPhGemm>::value) {
      for (int c = 0; c < nch; c++)
        if (!load_chunk(s, g, ph.as + (w * nch + c) * (int64_t)kAChunk, ph.bs + ((int64_t)ct * nch + c) * kBChunk))
          return;
    } else if constexpr (std::is_same<Ph, OzPh1>::value) {
      const OzItem it = ph.items[w];
      for (int c = 0; c < nch; c++)
        if (!load_chunk(s, g, ph.xs + ((it.x_chunk0 + c) * ph.nct + ct) * (int64_t)kAChunk,
                        ph.ops + (it.b_chunk0 + c) * (int64_t)kBChunk))
          return;
    } else {
      const OzTile t = ph.tiles[w];
      int64_t bc = t.b_chunk0;
      for (int j = 0; j < t.nseg; j++) {
        const OzSeg sg = ph.segs[t.seg0 + j];
        const uint8_t* base = sg.near ? ph.xs : ph.zs;
        for (int c = 0; c < sg.nch; c++, bc++)
          if (!load_chunk(s, g, base + ((sg.a0 + c) * ph.nct + ct) * (int64_t)kAChunk,
                          ph.ops + bc * (int64_t)kBChunk))
            return;
      }
    }
  }
}

// The products of one chunk for the weights [w0, w1): weight w accumulates
// at TMEM column 64 w.  Weights below kWx start afresh at the first chunk of
// every 512-K block (their sums stay exact integers within a block and are
// moved to 64-bit registers after it); the others accumulate over the whole
// tile and start afresh at its first chunk.
__device__ __forceinline__ void issue_weights(const uint8_t* a, const uint8_t* b, uint32_t tmem, int w0, int w1,
                                              bool block_start, bool tile_start) {
  // descriptors of plane 0; plane i starts i planes further on (the start
  // address field holds addr >> 4 and stays below 2^14 inside shared memory)
  const uint64_t ad0 = umma::smem_desc(umma::smem_u32(a), kSBO), bd0 = umma::smem_desc(umma::smem_u32(b), kSBO);
#pragma unroll
  for (int w = 0; w < kW; w++) {
    if (w < w0 || w >= w1) continue;
    const bool fresh = w < kWx ? block_start : tile_start;
#pragma unroll
    for (int i = 0; i <= w; i++) {
      const int j = w - i;
      umma::mma_f16(tmem + (uint32_t)(w * kN), ad0 + (uint64_t)(i * (kAPlane >> 4)),
                    bd0 + (uint64_t)(j * (kBPlane >> 4)), kIdesc, (fresh && i == 0) ? 0u : 1u);
    }
  }
}

__device__ __forceinline__ void mma_issuer(const OzSmem& s, uint32_t tmem) {
  int64_t g = 0;  // chunks consumed
  int64_t fl = 0; // blocks handed to the epilogue
  int tl = 0, nch = 0;
  int64_t id;
  bool ok = true;
  for (; ok && next_tile(s, tl, id, nch); tl++) {
    if (nch == 0) {  // nothing to multiply: the epilogue writes zeros
      if (fl > 0 && !wait_bar(s, AE, (uint32_t)((fl - 1) & 1))) break;
      umma::mbar_arrive(&s.bar[AF]);
      fl++;
      continue;
    }
    for (int c = 0; c < nch; c++) {
      const int st = (int)(g % kStages);
      if (s.failed() || !wait_bar(s, FULL + st, (uint32_t)(g / kStages) & 1)) {
        ok = false;
        break;
      }
      umma::fence_after_sync();
      const bool block_start = c % kKBlock == 0;
      if (block_start && fl > 0) {
        // inside a tile the weights kept in TMEM go on while the epilogue moves the
        // exact sums of the previous block; at a tile start the epilogue reads all seven
        if (c > 0) issue_weights(s.a(st), s.b(st), tmem, kWx, kW, false, false);
        if (!wait_bar(s, AE, (uint32_t)((fl - 1) & 1))) {
          ok = false;
          break;
        }
        umma::fence_after_sync();
        issue_weights(s.a(st), s.b(st), tmem, 0, c > 0 ? kWx : kW, true, c == 0);
      } else {
        issue_weights(s.a(st), s.b(st), tmem, 0, kW, block_start, c == 0);
      }
      umma::commit(&s.bar[EMPTY + st]);
      g++;
      if (c % kKBlock == kKBlock - 1 || c == nch - 1) {
        umma::commit(&s.bar[AF]);
        fl++;
      }
    }
  }
  // every MMA issued here has completed before TMEM is released
  umma::commit(&s.bar[FIN]);
  wait_unwind(s, FIN, 0);
}

// Epilogue: warp (quarter q, half h) owns TMEM lanes 32 q .. (vector columns
// of the tile) and operator rows 32 h .. 32 h + 31 of every weight.
template <class Ph>
__device__ __forceinline__ void epilogue(const OzSmem& s, const Ph& ph, uint32_t tmem) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int quarter = warp & 3, half = (warp - 2) >> 2;
  const int vcol = 32 * quarter + lane;  // vector column within the column tile
  int64_t fl = 0;
  int tl = 0, nch = 0;
  int64_t id;
  for (; next_tile(s, tl, id, nch); tl++) {
    const int64_t w = id / ph.nct;
    const int ct = (int)(id % ph.nct);
    // H-apply: vector column of the pass; GEMM: the row of C
    const int col = std::is_same<Ph, OzPhGemm>::value ? (int)w * kM + vcol : ct * kM + vcol;
    // weights 0..3: exact integers, summed as sum_w T_w 2^(7(3-w)) in 64 bits (units of
    // 2^-21; at most 2^44 per block); weights 4..6 (summed over the tile in TMEM) in FP32 as
    // T_4 + T_5 2^-7 + T_6 2^-14 (units of 2^-28)
    int64_t acc[32];
    float low[32];
#pragma unroll
    for (int i = 0; i < 32; i++) {
      acc[i] = 0;
      low[i] = 0.f;
    }
    const int nblk = nch > 0 ? (nch + kKBlock - 1) / kKBlock : 1;
    bool ok = true;
    for (int blk = 0; blk < nblk; blk++, fl++) {
      if (!wait_bar(s, AF, (uint32_t)(fl & 1))) {
        ok = false;
        break;
      }
      umma::fence_after_sync();
      if (s.failed()) {
        ok = false;
        break;
      }
      if (nch > 0) {
        const bool last = blk == nblk - 1;
#pragma unroll
        for (int wt = 0; wt < kW; wt++) {
          if (wt >= kWx && !last) continue;
#pragma unroll
          for (int hh = 0; hh < 2; hh++) {
            float v[16];
            umma::tmem_ld16(tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(wt * kN + 32 * half + 16 * hh), v);
#pragma unroll
            for (int i = 0; i < 16; i++) {
              if (wt < kWx)
                acc[16 * hh + i] += (int64_t)__float2int_rn(v[i]) << (7 * (kWx - 1 - wt));
              else
                low[16 * hh + i] += v[i] * (wt == 4 ? 1.f : (wt == 5 ? 0.0078125f : 0.00006103515625f));
            }
          }
        }
      }
      umma::fence_before_sync();
      umma::mbar_arrive(&s.bar[AE]);
    }
    if (!ok) break;
    if constexpr (std::is_same<Ph, OzPhGemm>::value) {
      if (col >= ph.M) continue;
      const double sc = ph.alpha * ph.sa[col] * 0x1p-14;
      double* crow = ph.C + (int64_t)col * ph.ldc;
#pragma unroll
      for (int i = 0; i < 32; i++) {
        const int n = ct * kN + 32 * half + i;
        if (n < ph.N) {
          const double r = (double)acc[i] * 0x1p-21 + (double)low[i] * 0x1p-28;
          const double v = sc * ph.sb[n] * r;
          crow[n] = ph.beta == 0.0 ? v : fma(ph.beta, crow[n], v);
        }
      }
    } else if constexpr (std::is_same<Ph, OzPh2>::value) {
      if (col >= ph.ncols) continue;
      const OzTile t = ph.tiles[w];
      const double sc = ph.tau[col] * 0x1p-14;
#pragma unroll
      for (int i = 0; i < 32; i++) {
        const int n = 32 * half + i;
        if (n < t.rows) {
          const double r = (double)acc[i] * 0x1p-21 + (double)low[i] * 0x1p-28;
          ph.Y[(t.row0 + n) * ph.ldy + col] = sc * ph.sig[t.row0 + n] * r;
        }
      }
    } else {
      if (col >= ph.ncols) continue;
      const OzItem it = ph.items[w];
#pragma unroll
      for (int u = 0; u < 8; u++) {  // aligned groups of 4 slots
        const int n0 = 32 * half + 4 * u;
        if (n0 >= it.nq) continue;
        if (it.out_row >= 0) {  // FP64 partial rows: Z / tau_n
#pragma unroll
          for (int e = 0; e < 4; e++) {
            const double r = (double)acc[4 * u + e] * 0x1p-21 + (double)low[4 * u + e] * 0x1p-28;
            ph.part[(it.out_row + n0 + e) * ph.ldp + col] = ph.sig[it.map_off + n0 + e] * 0x1p-14 * r;
          }
          continue;
        }
        // Z / (tau_n Q_g) on the 2^-49 grid: (acc 2^14 + low 2^7) / 2^s with
        // s = log2(Q_g / sig_g) >= 0, in integers
        int64_t z[4];
#pragma unroll
        for (int e = 0; e < 4; e++) {
          const int sh = ph.qsh[it.map_off + n0 + e];
          const int64_t t = (acc[4 * u + e] << 14) + __float2ll_rn(low[4 * u + e] * 128.f);
          z[e] = sh > 0 ? (t + (int64_t(1) << (sh - 1))) >> sh : t;
        }
        const int64_t p = ph.slotpos[it.map_off + n0];  // 4 consecutive aligned positions
        uint8_t* ch = ph.zs + ((p >> 4) * ph.nct + ct) * (int64_t)kAChunk + off16(vcol, (int)(p & 15));
        // balanced base-128 digits (as digits7), plane by plane, least significant first
#pragma unroll
        for (int i = kSl - 1; i >= 0; i--) {
          uint32_t h[4];
#pragma unroll
          for (int e = 0; e < 4; e++) {
            const int64_t r = i > 0 ? ((z[e] + 64) & 127) - 64 : z[e];
            h[e] = __half_as_ushort(__int2half_rn((int)r));
            z[e] = (z[e] - r) >> 7;
          }
          *reinterpret_cast<uint2*>(ch + i * kAPlane) = make_uint2(h[0] | (h[1] << 16), h[2] | (h[3] << 16));
        }
      }
    }
  }
}

template <class Ph>
__global__ void __launch_bounds__(kThreads, 1)
    k_oz_apply(const Ph ph, int64_t ntiles, unsigned long long* __restrict__ counter, int* __restrict__ err,
               uint32_t max_polls) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  OzSmem s;
  s.base = smem_raw;
  uint8_t* tail = smem_raw + kStages * kStage;
  s.bar = reinterpret_cast<uint64_t*>(tail);
  s.tmem_slot = reinterpret_cast<uint32_t*>(tail + kBarBytes);
  s.fail = reinterpret_cast<int*>(tail + kBarBytes + 8);
  s.q = reinterpret_cast<OzQ*>(tail + kBarBytes + 16);
  s.polls = max_polls;
  const int warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    for (int i = FULL; i < AF; i++) umma::mbar_init(&s.bar[i], 1);
    umma::mbar_init(&s.bar[AF], 1);
    umma::mbar_init(&s.bar[AE], 32 * kEpiWarps);
    umma::mbar_init(&s.bar[FIN], 1);
    for (int i = QF; i < QE; i++) umma::mbar_init(&s.bar[i], 1);
    for (int i = QE; i < NBAR; i++) umma::mbar_init(&s.bar[i], 1 + 32 * kEpiWarps);
    *s.fail = 0;
    umma::fence_mbar_init();
  }
  if (warp == 1) umma::tmem_alloc(s.tmem_slot, kTmemCols);
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tmem = *s.tmem_slot;
  if (warp == 0) {
    if ((threadIdx.x & 31) == 0) {
      int64_t g = 0;
      producer<Ph>(s, ph, ntiles, counter, g);
      // no exit (nor unwind) while a bulk copy into this CTA's shared memory is in flight
      for (int64_t i = g > kStages ? g - kStages : 0; i < g; i++)
        wait_unwind(s, FULL + (int)(i % kStages), (uint32_t)(i / kStages) & 1);
    }
  } else if (warp == 1) {
    if ((threadIdx.x & 31) == 0) mma_issuer(s, tmem);
    __syncwarp();
  } else {
    epilogue<Ph>(s, ph, tmem);
  }
  umma::fence_before_sync();
  __syncthreads();
  if (threadIdx.x == 0 && s.failed()) atomicExch(err, 1);
  if (warp == 1) {
    umma::fence_after_sync();
    umma::tmem_dealloc(tmem, kTmemCols);
  }
}

// ---- slicing ----------------------------------------------------------------
// Operator chunks: thread (row n, 8 k) of chunk c; 7 planes of 64 x 16.
__global__ void __launch_bounds__(128) k_oz_build_b(const OzBChunk* __restrict__ d, int64_t n,
                                                    const double* __restrict__ fac, const double* __restrict__ nearv,
                                                    const double* __restrict__ sig_slot,
                                                    const double* __restrict__ sig_pt,
                                                    const double* __restrict__ q_pos, uint8_t* __restrict__ out) {
  const int row = threadIdx.x & 63, kg = threadIdx.x >> 6;
  for (int64_t c = blockIdx.x; c < n; c += gridDim.x) {
    const OzBChunk ch = d[c];
    const double* src = ch.near ? nearv : fac;
    const double rs = row < ch.rows ? 1.0 / (ch.phase == 1 ? sig_slot[ch.s_off + row] : sig_pt[ch.s_off + row]) : 0.0;
    uint16_t sl[8][kSl];
#pragma unroll
    for (int u = 0; u < 8; u++) {
      const int k = 8 * kg + u;
      double x = 0.0;
      if (row < ch.rows && k < ch.kv) {
        x = src[ch.src_off + (int64_t)row * ch.si + (int64_t)k * ch.sk] * rs;
        if (ch.k_off >= 0) x *= q_pos[ch.k_off + k];
      }
      digits7(grid49(x), sl[u]);
    }
    uint8_t* base = out + c * (int64_t)kBChunk + off16(row, 8 * kg);
#pragma unroll
    for (int i = 0; i < kSl; i++)
      *reinterpret_cast<uint4*>(base + i * kBPlane) =
          make_uint4((uint32_t)sl[0][i] | ((uint32_t)sl[1][i] << 16), (uint32_t)sl[2][i] | ((uint32_t)sl[3][i] << 16),
                     (uint32_t)sl[4][i] | ((uint32_t)sl[5][i] << 16), (uint32_t)sl[6][i] | ((uint32_t)sl[7][i] << 16));
  }
}

// Column maxima of |X| (bit patterns of non-negative doubles order like the values).
__global__ void __launch_bounds__(256) k_oz_colmax(const double* __restrict__ X, int64_t ldx, int64_t rows, int ncols,
                                                   int64_t rows_per_block, unsigned long long* __restrict__ cmax) {
  const int col = blockIdx.x * 256 + threadIdx.x;
  if (col >= ncols) return;
  const int64_t r0 = (int64_t)blockIdx.y * rows_per_block;
  const int64_t r1 = min(rows, r0 + rows_per_block);
  double m = 0.0;
  for (int64_t r = r0; r < r1; r++) m = fmax(m, fabs(X[r * ldx + col]));
  atomicMax(&cmax[col], (unsigned long long)__double_as_longlong(m));
}

__global__ void k_oz_tau(const unsigned long long* __restrict__ cmax, int ncols, double* __restrict__ tau) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < ncols) tau[j] = pow2_ceil(__longlong_as_double((long long)cmax[j]));
}

// Sliced X of one pass: chunk x (blockIdx.x) of 16 rows, column tile ct
// (blockIdx.y) of 128 columns; thread (column n, 8 rows).
__global__ void __launch_bounds__(256) k_oz_split_x(const double* __restrict__ X, int64_t ldx, int ncols,
                                                    const TcXChunk* __restrict__ xmap, int nct,
                                                    const double* __restrict__ tau, uint8_t* __restrict__ out) {
  const TcXChunk xc = xmap[blockIdx.x];
  const int ct = blockIdx.y;
  const int n = threadIdx.x & 127, kg = threadIdx.x >> 7;
  const int col = ct * kM + n;
  const double sc = col < ncols ? 0x1p49 / tau[col] : 0.0;  // a power of two
  uint16_t sl[8][kSl];
#pragma unroll
  for (int u = 0; u < 8; u++) {
    const int k = 8 * kg + u;
    const double x = (k < xc.rows && col < ncols) ? X[(xc.row0 + k) * ldx + col] * sc : 0.0;
    digits7(__double2ll_rn(x), sl[u]);
  }
  uint8_t* base = out + ((int64_t)blockIdx.x * nct + ct) * kAChunk + off16(n, 8 * kg);
#pragma unroll
  for (int i = 0; i < kSl; i++)
    *reinterpret_cast<uint4*>(base + i * kAPlane) =
        make_uint4((uint32_t)sl[0][i] | ((uint32_t)sl[1][i] << 16), (uint32_t)sl[2][i] | ((uint32_t)sl[3][i] << 16),
                   (uint32_t)sl[4][i] | ((uint32_t)sl[5][i] << 16), (uint32_t)sl[6][i] | ((uint32_t)sl[7][i] << 16));
}

// Sum the FP64 partial rows of a cluster split over several leaf groups
// (Z / tau, fixed order), divide by the slot bound and write the slices into
// the workspace position of the partner slot.
__global__ void k_oz_reduce(const P1Reduce* __restrict__ items, const double* __restrict__ part, int64_t ldp,
                            const int64_t* __restrict__ slotpos, const double* __restrict__ qs, uint8_t* __restrict__ zs,
                            int nct, int ncols) {
  const P1Reduce it = items[blockIdx.x];
  const int64_t total = (int64_t)it.nq * ncols;
  for (int64_t e = threadIdx.x + (int64_t)blockIdx.y * blockDim.x; e < total; e += (int64_t)blockDim.x * gridDim.y) {
    const int q = (int)(e / ncols), n = (int)(e % ncols);
    double acc = 0.0;
    for (int c = 0; c < it.nch; c++) acc += part[(it.part_row + (int64_t)c * it.nq + q) * ldp + n];
    uint16_t d[kSl];
    digits7(grid49(acc / qs[it.map_off + q]), d);
    const int64_t p = slotpos[it.map_off + q];
    uint8_t* ch = zs + ((p >> 4) * nct + n / kM) * (int64_t)kAChunk + off16(n % kM, (int)(p & 15));
#pragma unroll
    for (int i = 0; i < kSl; i++) *reinterpret_cast<uint16_t*>(ch + i * kAPlane) = d[i];
  }
}

// Row maxima of |op(src)| for a transposed view (element (r, k) = src[k * ld + r]):
// grid (row blocks of 256, K blocks of kSegK); bit patterns of non-negative doubles.
constexpr int kSegK = 128;
__global__ void __launch_bounds__(256) k_oz_rowmax_t(const double* __restrict__ src, int64_t ld, int64_t rows,
                                                     int64_t K, unsigned long long* __restrict__ mx) {
  const int64_t r = (int64_t)blockIdx.x * 256 + threadIdx.x;
  if (r >= rows) return;
  const int64_t k0 = (int64_t)blockIdx.y * kSegK, k1 = min(K, k0 + kSegK);
  double m = 0.0;
  for (int64_t k = k0; k < k1; k++) m = fmax(m, fabs(src[k * ld + r]));
  atomicMax(&mx[r], (unsigned long long)__double_as_longlong(m));
}

// Row scales of op(src), rows x K: power of two >= max_k |op(src)[r][k]|.
// Contiguous rows (trans = 0): a warp per row; transposed: from the maxima mx.
__global__ void __launch_bounds__(256) k_oz_rowscale(const double* __restrict__ src, int64_t ld, int trans,
                                                     int64_t rows, int64_t K, const unsigned long long* __restrict__ mx,
                                                     double* __restrict__ s) {
  if (trans) {
    const int64_t r = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (r < rows) s[r] = pow2_ceil(__longlong_as_double((long long)mx[r]));
    return;
  }
  const int64_t r = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (r >= rows) return;
  double m = 0.0;
  for (int64_t k = lane; k < K; k += 32) m = fmax(m, fabs(src[r * ld + k]));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) s[r] = pow2_ceil(m);
}

// op(src) (rows x K) into chunks of TR rows x 16 K x 7 slice planes: chunk
// (row tile t, K chunk c) at out + (t * nch + c) * 7 * TR * 32 bytes,
// element (r, k) over its row scale s[r], zero outside rows x K.  Thread
// (row of the tile, 8 k).
template <int TR>
__global__ void __launch_bounds__(2 * TR) k_oz_slice_dense(const double* __restrict__ src, int64_t ld, int trans,
                                                           int64_t rows, int64_t K, int nch,
                                                           const double* __restrict__ s, uint8_t* __restrict__ out) {
  constexpr int kPlane = TR * kK * 2;
  const int64_t t = blockIdx.x;
  const int c = blockIdx.y;
  const int rl = threadIdx.x % TR, kg = threadIdx.x / TR;
  const int64_t r = t * TR + rl;
  const double sc = r < rows ? 0x1p49 / s[r] : 0.0;  // a power of two
  uint16_t sl[8][kSl];
#pragma unroll
  for (int u = 0; u < 8; u++) {
    const int64_t k = (int64_t)c * kK + 8 * kg + u;
    double x = 0.0;
    if (r < rows && k < K) x = (trans ? src[k * ld + r] : src[r * ld + k]) * sc;
    digits7(__double2ll_rn(x), sl[u]);
  }
  uint8_t* base = out + (t * nch + c) * (int64_t)(kSl * kPlane) + off16(rl, 8 * kg);
#pragma unroll
  for (int i = 0; i < kSl; i++)
    *reinterpret_cast<uint4*>(base + i * kPlane) =
        make_uint4((uint32_t)sl[0][i] | ((uint32_t)sl[1][i] << 16), (uint32_t)sl[2][i] | ((uint32_t)sl[3][i] << 16),
                   (uint32_t)sl[4][i] | ((uint32_t)sl[5][i] << 16), (uint32_t)sl[6][i] | ((uint32_t)sl[7][i] << 16));
}

// Scales and slices of one GEMM operand viewed as rows x K (trans: element
// (r, k) = src[k * ld + r]).
template <int TR>
fkf_status oz_operand(fkf_ctx* ctx, const double* src, int64_t ld, bool trans, int64_t rows, int64_t K, int nch,
                      double* s, unsigned long long* mx, uint8_t* out) {
  cudaStream_t st = ctx->stream;
  if (trans) {
    FKF_CUDA(ctx, cudaMemsetAsync(mx, 0, (size_t)rows * sizeof(unsigned long long), st));
    k_oz_rowmax_t<<<dim3((unsigned)cdiv(rows, 256), (unsigned)cdiv(K, kSegK)), 256, 0, st>>>(src, ld, rows, K, mx);
    FKF_LAUNCHED(ctx);
    k_oz_rowscale<<<(unsigned)cdiv(rows, 256), 256, 0, st>>>(src, ld, 1, rows, K, mx, s);
  } else {
    k_oz_rowscale<<<(unsigned)cdiv(rows, 8), 256, 0, st>>>(src, ld, 0, rows, K, nullptr, s);
  }
  FKF_LAUNCHED(ctx);
  k_oz_slice_dense<TR><<<dim3((unsigned)cdiv(rows, TR), (unsigned)nch), 2 * TR, 0, st>>>(src, ld, trans ? 1 : 0, rows,
                                                                                       K, nch, s, out);
  FKF_LAUNCHED(ctx);
  return FKF_OK;
}

fkf_status build_oz_stream(fkf_hmat* h) {
  fkf_ctx* ctx = h->ctx;
  if (h->n_ozb > 0) {
    FKF_TRY(dev_alloc(ctx, h->ozb, (size_t)h->n_ozb * kBChunk));
    const int grid = (int)std::min<int64_t>(h->n_ozb, 152 * 16);
    k_oz_build_b<<<grid, 128, 0, ctx->stream>>>(h->ozbdesc.as<OzBChunk>(), h->n_ozb, h->fac.as<double>(),
                                               h->nearv.as<double>(), h->oz_sigslot.as<double>(),
                                               h->oz_sigpt.as<double>(), h->oz_qpos.as<double>(),
                                               h->ozb.as<uint8_t>());
    FKF_LAUNCHED(ctx);
  }
  h->ozb_built = true;
  return FKF_OK;
}

}  // namespace

fkf_status hmat_upload_oz(fkf_hmat* h, OzUpload& ou) {
  fkf_ctx* ctx = h->ctx;
  auto up = [&](DevBuf& b, const void* p, size_t bytes) -> fkf_status {
    if (bytes == 0) return FKF_OK;
    return dev_upload(ctx, b, p, bytes);
  };
  FKF_TRY(up(h->ozitem, ou.items.data(), ou.items.size() * sizeof(OzItem)));
  FKF_TRY(up(h->ozred, ou.reduces.data(), ou.reduces.size() * sizeof(P1Reduce)));
  FKF_TRY(up(h->oztile, ou.tiles.data(), ou.tiles.size() * sizeof(OzTile)));
  FKF_TRY(up(h->ozseg, ou.segs.data(), ou.segs.size() * sizeof(OzSeg)));
  FKF_TRY(up(h->ozbdesc, ou.bchunks.data(), ou.bchunks.size() * sizeof(OzBChunk)));
  FKF_TRY(up(h->ozxmap, ou.xmap.data(), ou.xmap.size() * sizeof(TcXChunk)));
  FKF_TRY(up(h->ozslot, ou.slotpos.data(), ou.slotpos.size() * sizeof(int64_t)));
  FKF_TRY(up(h->oz_sigslot, ou.sig_slot.data(), ou.sig_slot.size() * sizeof(double)));
  FKF_TRY(up(h->oz_qslot, ou.q_slot.data(), ou.q_slot.size() * sizeof(double)));
  FKF_TRY(up(h->oz_qshift, ou.q_shift.data(), ou.q_shift.size() * sizeof(int32_t)));
  FKF_TRY(up(h->oz_qpos, ou.q_pos.data(), ou.q_pos.size() * sizeof(double)));
  FKF_TRY(up(h->oz_sigpt, ou.sig_pt.data(), ou.sig_pt.size() * sizeof(double)));
  h->n_ozitem = (int64_t)ou.items.size();
  h->n_ozred = (int64_t)ou.reduces.size();
  h->n_oztile = (int64_t)ou.tiles.size();
  h->n_ozb = (int64_t)ou.bchunks.size();
  h->n_ozx = (int64_t)ou.xmap.size();
  h->n_ozz = ou.nz;
  h->oz_part_rows = ou.part_rows;
  // columns per pass: a multiple of 128 that keeps the sliced slot workspace under ~16 GB
  int64_t panel = 1024;
  while (panel > kM && (double)std::max<int64_t>(h->n_ozz, 1) * (panel / kM) * kAChunk > 16e9) panel /= 2;
  h->oz_panel = panel;
  h->ozb_built = false;  // the sliced stream is written when engine 3 is first selected
  return FKF_OK;
}

fkf_status hmat_oz_check(fkf_hmat* h) {
  if (!h->oz_err.p) return FKF_OK;
  int e = 0;
  FKF_CUDA(h->ctx, cudaMemcpyAsync(&e, h->oz_err.p, 4, cudaMemcpyDeviceToHost, h->ctx->stream));
  FKF_CUDA(h->ctx, cudaStreamSynchronize(h->ctx->stream));
  if (e) {
    FKF_CUDA(h->ctx, cudaMemsetAsync(h->oz_err.p, 0, 4, h->ctx->stream));
    return set_err(h->ctx, FKF_ETIMEOUT, "FP64 tensor-core H-apply: an mbarrier wait expired");
  }
  return FKF_OK;
}

fkf_status hmat_oz_prepare(fkf_hmat* h) {
  if (h->prec != FKF_FP64) return set_err(h->ctx, FKF_EINVAL, "engine 3 needs an FP64 operator");
  if (!h->ozb_built) FKF_TRY(build_oz_stream(h));
  return FKF_OK;
}

fkf_status hmat_apply_clustered_oz(fkf_hmat* h, const double* X, int64_t ldx, double* Y, int64_t ldy,
                                   int64_t ncols) {
  fkf_ctx* ctx = h->ctx;
  cudaStream_t st = ctx->stream;
  FKF_TRY(hmat_oz_prepare(h));
  const int64_t P = h->oz_panel;
  const int64_t nct_max = cdiv(std::min(ncols, P), kM);
  if (h->ozx.bytes < (size_t)std::max<int64_t>(h->n_ozx, 1) * nct_max * kAChunk)
    FKF_TRY(dev_alloc(ctx, h->ozx, (size_t)std::max<int64_t>(h->n_ozx, 1) * nct_max * kAChunk));
  const size_t zbytes = (size_t)std::max<int64_t>(h->n_ozz, 1) * nct_max * kAChunk;
  if (h->ozz.bytes < zbytes) {
    // positions no product lands on (padding slots) are read as zeros
    FKF_TRY(dev_alloc(ctx, h->ozz, zbytes));
    FKF_CUDA(ctx, cudaMemsetAsync(h->ozz.p, 0, h->ozz.bytes, st));
  }
  if (h->oz_part_rows > 0 && h->ozpart.bytes < (size_t)h->oz_part_rows * P * sizeof(double))
    FKF_TRY(dev_alloc(ctx, h->ozpart, (size_t)h->oz_part_rows * P * sizeof(double)));
  if (h->oz_col.bytes < (size_t)P * 16) FKF_TRY(dev_alloc(ctx, h->oz_col, (size_t)P * 16));
  if (h->oz_err.bytes < 64) {
    FKF_TRY(dev_alloc(ctx, h->oz_err, 64));
    FKF_CUDA(ctx, cudaMemsetAsync(h->oz_err.p, 0, 64, st));
  }
  double* tau = h->oz_col.as<double>();
  unsigned long long* cmax = reinterpret_cast<unsigned long long*>(tau + P);
  unsigned long long* counters = reinterpret_cast<unsigned long long*>(h->oz_err.as<char>() + 16);
  int sms = 0;
  FKF_CUDA(ctx, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
  FKF_CUDA(ctx, cudaFuncSetAttribute(k_oz_apply<OzPh1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem));
  FKF_CUDA(ctx, cudaFuncSetAttribute(k_oz_apply<OzPh2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem));
  for (int64_t c0 = 0; c0 < ncols; c0 += P) {
    const int nc = (int)std::min<int64_t>(P, ncols - c0);
    const int nct = (int)cdiv(nc, kM);
    FKF_CUDA(ctx, cudaMemsetAsync(counters, 0, 2 * sizeof(unsigned long long), st));
    FKF_CUDA(ctx, cudaMemsetAsync(cmax, 0, (size_t)nc * sizeof(unsigned long long), st));
    const int64_t rpb = 2048;
    k_oz_colmax<<<dim3((unsigned)cdiv(nc, 256), (unsigned)cdiv(h->n, rpb)), 256, 0, st>>>(X + c0, ldx, h->n, nc, rpb,
                                                                                       cmax);
    FKF_LAUNCHED(ctx);
    k_oz_tau<<<(unsigned)cdiv(nc, 256), 256, 0, st>>>(cmax, nc, tau);
    FKF_LAUNCHED(ctx);
    if (h->n_ozx > 0) {
      k_oz_split_x<<<dim3((unsigned)h->n_ozx, (unsigned)nct), 256, 0, st>>>(X + c0, ldx, nc, h->ozxmap.as<TcXChunk>(),
                                                                           nct, tau, h->ozx.as<uint8_t>());
      FKF_LAUNCHED(ctx);
    }
    if (h->n_ozitem > 0) {
      const OzPh1 p1{h->ozitem.as<OzItem>(), h->ozx.as<uint8_t>(), h->ozb.as<uint8_t>(), h->ozz.as<uint8_t>(),
                     h->ozpart.as<double>(), P, h->ozslot.as<int64_t>(), h->oz_sigslot.as<double>(),
                     h->oz_qshift.as<int32_t>(), nct, nc};
      const int64_t nt = h->n_ozitem * nct;
      k_oz_apply<OzPh1><<<(unsigned)std::min<int64_t>(sms, nt), kThreads, kSmem, st>>>(p1, nt, counters,
                                                                                      h->oz_err.as<int>(), h->tc_polls);
      FKF_LAUNCHED(ctx);
    }
    if (h->n_ozred > 0) {
      k_oz_reduce<<<dim3((unsigned)h->n_ozred, 4), 256, 0, st>>>(h->ozred.as<P1Reduce>(), h->ozpart.as<double>(), P,
                                                                h->ozslot.as<int64_t>(), h->oz_qslot.as<double>(),
                                                                h->ozz.as<uint8_t>(), nct, nc);
      FKF_LAUNCHED(ctx);
    }
    if (ctx->ph2_mark && c0 + P >= ncols) {  // the last phase 2 of this apply starts here
      FKF_CUDA(ctx, cudaEventRecord(ctx->ph2_mark, st));
      ctx->ph2_marked = true;
    }
    const OzPh2 p2{h->oztile.as<OzTile>(), h->ozseg.as<OzSeg>(), h->ozx.as<uint8_t>(), h->ozz.as<uint8_t>(),
                   h->ozb.as<uint8_t>(), Y + c0, ldy, h->oz_sigpt.as<double>(), tau, nct, nc};
    const int64_t nt = h->n_oztile * nct;
    k_oz_apply<OzPh2><<<(unsigned)std::min<int64_t>(sms, nt), kThreads, kSmem, st>>>(p2, nt, counters + 1,
                                                                                    h->oz_err.as<int>(), h->tc_polls);
    FKF_LAUNCHED(ctx);
  }
  return FKF_OK;
}

fkf_status gemm_f64_tc(fkf_ctx* ctx, bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha, const double* A,
                       int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc,
                       OzGemmWs* wsp) {
  if (M <= 0 || N <= 0) return FKF_OK;
  if (K <= 0 || alpha == 0.0) return beta == 1.0 ? FKF_OK : scale_f64(ctx, M, N, beta, C, ldc);
  OzGemmWs& ws = wsp ? *wsp : ctx->ozgemm_ws;
  const int nch = (int)cdiv(K, kK);
  const int64_t nrt = cdiv(M, kM), nct = cdiv(N, kN);
  const size_t abytes = (size_t)nrt * nch * kAChunk, bbytes = (size_t)nct * nch * kBChunk;
  if (ws.as.bytes < abytes) FKF_TRY(dev_alloc(ctx, ws.as, abytes));
  if (ws.bs.bytes < bbytes) FKF_TRY(dev_alloc(ctx, ws.bs, bbytes));
  const size_t sbytes = (size_t)(M + N) * 16;
  if (ws.sc.bytes < sbytes) FKF_TRY(dev_alloc(ctx, ws.sc, sbytes));
  if (ws.ctl.bytes < 64) {
    FKF_TRY(dev_alloc(ctx, ws.ctl, 64));
    FKF_CUDA(ctx, cudaMemsetAsync(ws.ctl.p, 0, 64, ctx->stream));
  }
  double* sa = ws.sc.as<double>();
  double* sb = sa + M;
  unsigned long long* mx = reinterpret_cast<unsigned long long*>(sb + N);
  // op(A) by rows of C; op(B) by columns of C: element (n, k) = op(B)[k][n]
  FKF_TRY(oz_operand<kM>(ctx, A, lda, ta, M, K, nch, sa, mx, ws.as.as<uint8_t>()));
  FKF_TRY(oz_operand<kN>(ctx, B, ldb, !tb, N, K, nch, sb, mx + M, ws.bs.as<uint8_t>()));
  unsigned long long* counter = reinterpret_cast<unsigned long long*>(ws.ctl.as<char>() + 16);
  FKF_CUDA(ctx, cudaMemsetAsync(counter, 0, sizeof(unsigned long long), ctx->stream));
  int sms = 0;
  FKF_CUDA(ctx, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
  FKF_CUDA(ctx, cudaFuncSetAttribute(k_oz_apply<OzPhGemm>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem));
  const OzPhGemm ph{ws.as.as<uint8_t>(), ws.bs.as<uint8_t>(), C, ldc, sa, sb, alpha, beta, (int)M, (int)N, nch,
                    (int)nct};
  const int64_t nt = nrt * nct;
  k_oz_apply<OzPhGemm><<<(unsigned)std::min<int64_t>(sms, nt), kThreads, kSmem, ctx->stream>>>(
      ph, nt, counter, ws.ctl.as<int>(), kMaxPolls);
  FKF_LAUNCHED(ctx);
  return FKF_OK;
}

fkf_status gemm_f64_tc_check(fkf_ctx* ctx) {
  // the context stream's GEMMs, then the low-priority stream's
  const cudaStream_t streams[2] = {ctx->stream, ctx->side_lo};
  OzGemmWs* wss[2] = {&ctx->ozgemm_ws, &ctx->ozgemm_ws_lo};
  for (int i = 0; i < 2; i++) {
    if (!wss[i]->ctl.p || !streams[i]) continue;
    int e = 0;
    FKF_CUDA(ctx, cudaMemcpyAsync(&e, wss[i]->ctl.p, 4, cudaMemcpyDeviceToHost, streams[i]));
    FKF_CUDA(ctx, cudaStreamSynchronize(streams[i]));
    if (e) {
      FKF_CUDA(ctx, cudaMemsetAsync(wss[i]->ctl.p, 0, 4, streams[i]));
      FKF_CUDA(ctx, cudaStreamSynchronize(streams[i]));
      return set_err(ctx, FKF_ETIMEOUT, "FP64 tensor-core GEMM: an mbarrier wait expired");
    }
  }
  return FKF_OK;
}
