// H-apply on the 5th-generation tensor cores (FP32 operators).  Both phases
// of the two-phase apply run as 128 x 256 output tiles of tcgen05.mma
// kind::tf32 with FP32 accumulators in TMEM.  Every FP32 value x is split into
// hi = tf32(x) and lo = tf32(x - hi), and each product is accumulated as
// hi*hi + hi*lo + lo*hi (3xTF32), which keeps FP32-level accuracy.
//
// Both operands reach shared memory already split, in the tensor core's
// K-major core-matrix layout, one bulk copy per operand and K-chunk of 16:
//   * the operator (A): split once when the operator is built, as one stream
//     of 16 KB chunks (128 x 16 TF32 hi block, then lo) per phase-1 item and
//     per phase-2 tile;
//   * the vectors (B): X is split per column pass into 16-row chunks per leaf
//     (rows padded to a multiple of 16), and phase 1 writes its products
//     straight into the split slot workspace (16-slot chunks per cluster);
//     a chunk is 32 KB per 256-column tile (hi, then lo).
//
// One persistent CTA per SM, warp-specialised:
//   warp 0     producer (one thread): two bulk copies per chunk into one of
//              four stages, completion counted in bytes on full[s];
//   warp 1     MMA issuer (one thread): six MMAs per chunk (2 K-steps x 3
//              products), commits to empty[s], and to acc_full after a
//              tile's last chunk; also allocates and frees TMEM;
//   warps 2-9  epilogue: tcgen05.ld of the finished accumulator (two warps
//              per TMEM lane quarter, one per half of the columns), stores,
//              arrive on acc_empty.
// Two accumulators (2 x 256 TMEM columns) let the epilogue of one tile run
// under the MMAs of the next.  Tiles are taken in order from a global
// counter (the producer takes the next one and passes its index to the MMA
// and epilogue roles through a small queue in shared memory): CTAs running at
// once work on neighbouring tiles, which share operator chunks (the column
// tiles of one work item) and X or ancestors' slot chunks, in L2, and a CTA
// that drew short tiles takes more of them.  Every mbarrier wait is bounded: an expired wait sets a flag,
// every role leaves its loop, the MMA issuer waits (bounded) for its
// outstanding MMAs, TMEM is freed and the host sees the error flag.
#include <algorithm>
#include <cstring>

#include "common.h"
#include "umma.cuh"

// Pipeline depth (compile-time tuning knob).
#ifndef FKF_TC_STAGES
#define FKF_TC_STAGES 4
#endif

namespace {

constexpr int kM = 128;                    // tile rows = TMEM lanes
constexpr int kN = 256;                    // tile columns = MMA N
constexpr int kK = umma::kChunk;           // 16: K per chunk
constexpr int kABytes = kM * kK * 4;       // 8 KB: one TF32 half of an A chunk
constexpr int kAChunkBytes = 2 * kABytes;  // 16 KB: hi | lo
constexpr int kBBytes = kN * kK * 4;       // 16 KB: one TF32 half of a B chunk
constexpr int kBChunkBytes = 2 * kBBytes;  // 32 KB: hi | lo
constexpr int kStageBytes = kAChunkBytes + kBChunkBytes;  // 48 KB
constexpr int kS = FKF_TC_STAGES;
constexpr int kEpiWarps = 8;               // warps 2-9: two per TMEM lane quarter, one per column half
constexpr int kEpiLd = 33;                 // padded row of an epilogue staging tile (32 x 32 floats)
constexpr int kEpiBytes = kEpiWarps * 32 * kEpiLd * 4;
constexpr int kQ = 8;                      // tile-index queue (producer -> MMA, epilogue)
constexpr int kTail = 384;                 // barriers, TMEM address, flag, queue
constexpr int kSmemBytes = kS * kStageBytes + kTail + kEpiBytes;  // 225.4 KB for 4 stages
static_assert(kSmemBytes <= 232448, "shared memory per CTA");
constexpr int kProdWarp = 0, kMmaWarp = 1;
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr uint32_t kTmemCols = 2 * kN;
constexpr uint32_t kMaxPolls = 1u << 22;
constexpr uint32_t kIdesc = umma::idesc_tf32(kM, kN);

// barrier indices
constexpr int FULL = 0, EMPTY = FULL + kS, AF = EMPTY + kS, AE = AF + 2, FIN = AE + 2, QF = FIN + 1, QE = QF + kQ,
              NBAR = QE + kQ;
static_assert(NBAR * 8 <= 256, "barrier area");

struct Smem {
  uint8_t* base;
  uint64_t* bar;
  uint32_t* tmem_slot;
  int* fail;
  int64_t* q;  // [kQ] tile indices (-1: no more tiles)
  float* epi;  // kEpiWarps staging tiles

  __device__ __forceinline__ uint8_t* a(int s) const { return base + s * kStageBytes; }
  __device__ __forceinline__ uint8_t* b(int s) const { return base + s * kStageBytes + kAChunkBytes; }
  __device__ __forceinline__ bool failed() const { return *reinterpret_cast<volatile int*>(fail) != 0; }
  __device__ __forceinline__ void set_fail() const { atomicExch(fail, 1); }
};

__device__ __forceinline__ Smem smem_layout(uint8_t* base) {
  Smem s;
  s.base = base;
  uint8_t* tail = base + kS * kStageBytes;
  s.bar = reinterpret_cast<uint64_t*>(tail);
  s.tmem_slot = reinterpret_cast<uint32_t*>(tail + 256);
  s.fail = reinterpret_cast<int*>(tail + 264);
  s.q = reinterpret_cast<int64_t*>(tail + 272);
  s.epi = reinterpret_cast<float*>(tail + kTail);
  return s;
}

__device__ __forceinline__ bool wait_bar(const Smem& s, int i, uint32_t parity) {
  if (umma::mbar_wait(&s.bar[i], parity, kMaxPolls)) return true;
  s.set_fail();
  return false;
}

// ---- splitting into the tensor-core layout ----------------------------------
__device__ __forceinline__ void split4(float v0, float v1, float v2, float v3, uint4& h, uint4& l) {
  umma::split_tf32(v0, h.x, l.x);
  umma::split_tf32(v1, h.y, l.y);
  umma::split_tf32(v2, h.z, l.z);
  umma::split_tf32(v3, h.w, l.w);
}

__device__ __forceinline__ void put4(uint8_t* hi_base, uint8_t* lo_base, int row, int k, float v0, float v1, float v2,
                                     float v3) {
  uint4 h, l;
  split4(v0, v1, v2, v3, h, l);
  const uint32_t off = umma::chunk_offset(row, k);
  *reinterpret_cast<uint4*>(hi_base + off) = h;
  *reinterpret_cast<uint4*>(lo_base + off) = l;
}

// One value into a split B chunk (row = column n of the tile, k = row in chunk).
__device__ __forceinline__ void put1(uint8_t* chunk, int n, int k, float v) {
  uint32_t h, l;
  umma::split_tf32(v, h, l);
  const uint32_t off = umma::chunk_offset(n, k);
  *reinterpret_cast<uint32_t*>(chunk + off) = h;
  *reinterpret_cast<uint32_t*>(chunk + kBBytes + off) = l;
}

// Split X: chunk x (blockIdx.x) of 16 rows (xmap; without a map, rows 16x..
// of a matrix of urows rows), column tile ct (blockIdx.y) of 256 columns ->
// 32 KB at out + (x * nct + ct) * 32 KB.  Thread units are (column n, rows
// 4kq..4kq+3): a warp reads 32 consecutive floats of a row and writes 512
// contiguous bytes per half.
__global__ void __launch_bounds__(256) k_tc_split_x(const float* __restrict__ X, int64_t ldx, int ncols,
                                                    const TcXChunk* __restrict__ xmap, int64_t urows, int nct,
                                                    uint8_t* __restrict__ out) {
  TcXChunk xc;
  if (xmap) {
    xc = xmap[blockIdx.x];
  } else {
    xc.row0 = (int64_t)blockIdx.x * kK;
    xc.rows = (int)min((int64_t)kK, urows - xc.row0);
  }
  const int ct = blockIdx.y;
  uint8_t* chunk = out + ((int64_t)blockIdx.x * nct + ct) * kBChunkBytes;
#pragma unroll
  for (int i = 0; i < 4; i++) {
    const int u = threadIdx.x + 256 * i;
    const int n = u & (kN - 1), kq = u >> 8;
    const int col = ct * kN + n;
    float v[4];
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const int k = 4 * kq + j;
      v[j] = (k < xc.rows && col < ncols) ? X[(xc.row0 + k) * ldx + col] : 0.f;
    }
    put4(chunk, chunk + kBBytes, n, 4 * kq, v[0], v[1], v[2], v[3]);
  }
}

// Split a row-major matrix A (rows x K, ld lda) into operator chunks: tile t
// (blockIdx.x) of 128 rows, K chunk c (blockIdx.y) of 16 columns -> 16 KB at
// out + (t * nch + c) * 16 KB; rows >= rows and columns >= K are zero.  Thread
// units are (row, 4 columns): a warp reads 64-byte runs of 8 rows and writes
// 512 contiguous bytes per half.
__global__ void __launch_bounds__(256) k_tc_split_rows(const float* __restrict__ A, int64_t lda, int64_t rows, int K,
                                                       int nch, uint8_t* __restrict__ out) {
  const int64_t t = blockIdx.x;
  const int c = blockIdx.y;
  uint8_t* hi = out + (t * nch + c) * (int64_t)kAChunkBytes;
  const bool vec = ((reinterpret_cast<uintptr_t>(A) & 15) == 0) && (lda & 3) == 0;
#pragma unroll
  for (int i = 0; i < 2; i++) {
    const int u = threadIdx.x + 256 * i;
    const int kq = u & 3, row = u >> 2;
    const int64_t r = t * kM + row;
    const int k = c * kK + 4 * kq;
    float v[4] = {0.f, 0.f, 0.f, 0.f};
    if (r < rows) {
      const float* src = A + r * lda + k;
      if (vec && k + 4 <= K) {
        const float4 q = *reinterpret_cast<const float4*>(src);
        v[0] = q.x, v[1] = q.y, v[2] = q.z, v[3] = q.w;
      } else {
#pragma unroll
        for (int j = 0; j < 4; j++)
          if (k + j < K) v[j] = src[j];
      }
    }
    put4(hi, hi + kABytes, row, 4 * kq, v[0], v[1], v[2], v[3]);
  }
}

// ---- the two phases' work items -------------------------------------------
// Phase 2: tiles of 128 consecutive rows; B segments = chunks of the split
// slot workspace (far) or of the split X (near); output rows of Y.
struct Ph2 {
  const TcTile* tiles;
  const TcSeg* segs;
  const uint8_t* zsplit;
  const uint8_t* xsplit;
  float* Y;
  int64_t ldy;
  __device__ __forceinline__ int nchunk(int64_t w) const { return tiles[w].nchunk; }
  __device__ __forceinline__ int64_t a_chunk0(int64_t w) const { return tiles[w].a_chunk0; }
  __device__ __forceinline__ int nseg(int64_t w) const { return tiles[w].nseg; }
  // B chunks of segment j: base array, first chunk, count
  __device__ __forceinline__ const uint8_t* seg(int64_t w, int j, int64_t& c0, int& nc) const {
    const TcSeg sg = segs[tiles[w].seg0 + j];
    c0 = sg.b_row;
    nc = (sg.K + kK - 1) / kK;
    return sg.near ? xsplit : zsplit;
  }
  __device__ __forceinline__ float* row_dst(int64_t w, int row) const {
    const TcTile& t = tiles[w];
    return row < t.rows ? Y + (t.row0 + row) * ldy : nullptr;
  }
};

// Phase 1: items (cluster, 128-slot tile, group of whole leaves); one B
// segment (the leaves' X chunks); output slot rows into the split slot
// workspace through the slot map, or partial rows when the cluster has
// several leaf groups.
struct Ph1 {
  const P1Item* items;
  const uint8_t* xsplit;
  const int64_t* slotpos;
  uint8_t* zsplit;
  float* part;
  int64_t ldp;
  __device__ __forceinline__ int nchunk(int64_t w) const { return items[w].nchunk; }
  __device__ __forceinline__ int64_t a_chunk0(int64_t w) const { return items[w].a_chunk0; }
  __device__ __forceinline__ int nseg(int64_t) const { return 1; }
  __device__ __forceinline__ const uint8_t* seg(int64_t w, int, int64_t& c0, int& nc) const {
    const P1Item& it = items[w];
    c0 = it.x_row;
    nc = it.nchunk;
    return xsplit;
  }
};

// Dense GEMM C_p = A_p B[0:K_p, :] for up to two problems that share B:
// row tiles of 128 rows of A_p (split by k_tc_split_rows, tile-major, K
// chunks consecutive), B split like X in uniform 16-row chunks; tiles of
// problem 0 first.  Output rows of C_p.
struct PhGemm {
  const uint8_t* bsplit;
  float *C0, *C1;
  int64_t ldc0, ldc1;
  int64_t rows0, rows1;
  int64_t a1;   // first A chunk of problem 1 (problem 0 starts at 0)
  int64_t nw0;  // row tiles of problem 0
  int nch0, nch1;  // K chunks per tile
  // (fields selected, not indexed: a dynamic index into a kernel parameter
  // array would copy the parameters to local memory)
  __device__ __forceinline__ int nchunk(int64_t w) const { return w >= nw0 ? nch1 : nch0; }
  __device__ __forceinline__ int64_t a_chunk0(int64_t w) const {
    return w >= nw0 ? a1 + (w - nw0) * nch1 : w * nch0;
  }
  __device__ __forceinline__ int nseg(int64_t) const { return 1; }
  __device__ __forceinline__ const uint8_t* seg(int64_t w, int, int64_t& c0, int& nc) const {
    c0 = 0;
    nc = nchunk(w);
    return bsplit;
  }
  __device__ __forceinline__ float* row_dst(int64_t w, int row) const {
    const bool p = w >= nw0;
    const int64_t r = (p ? w - nw0 : w) * kM + row;
    return r < (p ? rows1 : rows0) ? (p ? C1 : C0) + r * (p ? ldc1 : ldc0) : nullptr;
  }
};

// ---- roles -----------------------------------------------------------------
// Next tile of this CTA: taken from the global counter by the producer and
// published in the queue; every consumer reads each queue entry once.
__device__ __forceinline__ bool next_tile(const Smem& s, int qi, int64_t& id) {
  const int slot = qi % kQ;
  if (!wait_bar(s, QF + slot, (uint32_t)(qi / kQ) & 1)) return false;
  id = *reinterpret_cast<volatile int64_t*>(&s.q[slot]);
  umma::mbar_arrive(&s.bar[QE + slot]);
  return id >= 0;
}

template <class Ph>
__device__ __forceinline__ void producer(const Smem& s, const Ph& ph, int64_t ntiles, int nct,
                                         const uint8_t* astream, unsigned long long* counter) {
  int64_t g = 0;
  for (int qi = 0;; qi++) {
    int64_t id = (int64_t)atomicAdd(counter, 1ull);
    if (id >= ntiles) id = -1;
    const int slot = qi % kQ;
    if (qi >= kQ && !wait_bar(s, QE + slot, (uint32_t)((qi / kQ) - 1) & 1)) return;
    *reinterpret_cast<volatile int64_t*>(&s.q[slot]) = id;
    umma::mbar_arrive(&s.bar[QF + slot]);
    if (id < 0) return;
    const int64_t w = id / nct;
    const int ct = (int)(id % nct);
    const uint8_t* ap = astream + ph.a_chunk0(w) * (int64_t)kAChunkBytes;
    const int ns = ph.nseg(w);
    for (int j = 0; j < ns; j++) {
      int64_t c0;
      int nc;
      const uint8_t* bsrc = ph.seg(w, j, c0, nc);
      for (int c = 0; c < nc; c++, g++) {
        if (s.failed()) return;
        const int st = (int)(g % kS);
        if (g >= kS && !wait_bar(s, EMPTY + st, (uint32_t)((g / kS) - 1) & 1)) return;
        umma::mbar_arrive_expect_tx(&s.bar[FULL + st], kStageBytes);
        umma::bulk_g2s(s.a(st), ap, kAChunkBytes, &s.bar[FULL + st]);
        umma::bulk_g2s(s.b(st), bsrc + ((c0 + c) * nct + ct) * (int64_t)kBChunkBytes, kBChunkBytes,
                       &s.bar[FULL + st]);
        ap += kAChunkBytes;
      }
    }
  }
}

__device__ __forceinline__ void issue_mma(const uint8_t* a, const uint8_t* b, uint32_t acc, bool first) {
  const uint32_t a_hi = umma::smem_u32(a), a_lo = a_hi + kABytes;
  const uint32_t b_hi = umma::smem_u32(b), b_lo = b_hi + kBBytes;
#pragma unroll
  for (int kk = 0; kk < kK / 8; kk++) {
    const uint32_t koff = kk * 2 * umma::kLBO;  // two core matrices along K per MMA
    umma::mma_tf32(acc, umma::smem_desc(a_hi + koff), umma::smem_desc(b_hi + koff), kIdesc,
                   (first && kk == 0) ? 0u : 1u);
    umma::mma_tf32(acc, umma::smem_desc(a_hi + koff), umma::smem_desc(b_lo + koff), kIdesc, 1u);
    umma::mma_tf32(acc, umma::smem_desc(a_lo + koff), umma::smem_desc(b_hi + koff), kIdesc, 1u);
  }
}

template <class Ph>
__device__ __forceinline__ void mma_issuer(const Smem& s, const Ph& ph, int64_t ntiles, int nct, uint32_t tmem) {
  int64_t g = 0;
  int tl = 0;
  bool ok = true;
  int64_t id;
  for (; ok && next_tile(s, tl, id); tl++) {
    const int nch = ph.nchunk(id / nct);
    const int b = tl & 1;
    if (tl >= 2 && !wait_bar(s, AE + b, (uint32_t)((tl >> 1) - 1) & 1)) break;
    umma::fence_after_sync();
    const uint32_t acc = tmem + (uint32_t)(b * kN);
    for (int c = 0; c < nch; c++, g++) {
      const int st = (int)(g % kS);
      if (s.failed() || !wait_bar(s, FULL + st, (uint32_t)(g / kS) & 1)) {
        ok = false;
        break;
      }
      umma::fence_after_sync();
      issue_mma(s.a(st), s.b(st), acc, c == 0);
      umma::commit(&s.bar[EMPTY + st]);
    }
    if (!ok) break;
    if (nch > 0)
      umma::commit(&s.bar[AF + b]);
    else
      umma::mbar_arrive(&s.bar[AF + b]);
  }
  // every MMA issued here has completed before TMEM is released
  umma::commit(&s.bar[FIN]);
  wait_bar(s, FIN, 0);
}

// Epilogue stores of one row's 32 columns [c0, c0 + 32) of a tile.
struct RowSinkY {  // phase 2: a row of Y
  float* dst;
  __device__ __forceinline__ void put(int c0, int nv, const float (&v)[32]) const {
    if (!dst) return;
    if (((reinterpret_cast<uintptr_t>(dst + c0) & 15) == 0) && c0 + 32 <= nv) {
#pragma unroll
      for (int i = 0; i < 32; i += 4)
        *reinterpret_cast<float4*>(dst + c0 + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
    } else {
#pragma unroll
      for (int i = 0; i < 32; i++)
        if (c0 + i < nv) dst[c0 + i] = v[i];
    }
  }
};

template <class Ph>
__device__ __forceinline__ void epilogue(const Smem& s, const Ph& ph, int64_t ntiles, int nct, int ncols,
                                         uint32_t tmem);

// Rows of a row-major output: Ph supplies the destination row (nullptr past
// the tile's rows) and nchunk (0: the tile is zero).
template <class Ph>
__device__ __forceinline__ void epilogue_rows(const Smem& s, const Ph& ph, int nct, int ncols, uint32_t tmem) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int quarter = warp & 3;  // TMEM lanes 32*quarter.. are this warp's
  const int half = (warp - 2) >> 2;
  const int row = 32 * quarter + lane;
  int tl = 0;
  int64_t id;
  for (; next_tile(s, tl, id); tl++) {
    const int b = tl & 1;
    if (!wait_bar(s, AF + b, (uint32_t)(tl >> 1) & 1)) break;
    umma::fence_after_sync();
    if (s.failed()) break;
    const int64_t w = id / nct;
    const int n0 = (int)(id % nct) * kN;
    const int nv = min(kN, ncols - n0);
    const bool zero = ph.nchunk(w) == 0;
    float* dst = ph.row_dst(w, row);
    const RowSinkY sink{dst ? dst + n0 : nullptr};
#pragma unroll 1
    for (int j = 4 * half; j < 4 * half + 4; j++) {
      float v[32];
      if (zero) {
#pragma unroll
        for (int i = 0; i < 32; i++) v[i] = 0.f;
      } else {
        umma::tmem_ld32(tmem + (uint32_t)(b * kN) + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(32 * j), v);
      }
      sink.put(32 * j, nv, v);
    }
    umma::fence_before_sync();
    umma::mbar_arrive(&s.bar[AE + b]);
  }
}

// phase 2: rows of Y
template <>
__device__ __forceinline__ void epilogue<Ph2>(const Smem& s, const Ph2& ph, int64_t, int nct, int ncols,
                                              uint32_t tmem) {
  epilogue_rows(s, ph, nct, ncols, tmem);
}

// dense GEMM: rows of C
template <>
__device__ __forceinline__ void epilogue<PhGemm>(const Smem& s, const PhGemm& ph, int64_t, int nct, int ncols,
                                                 uint32_t tmem) {
  epilogue_rows(s, ph, nct, ncols, tmem);
}

// phase 1: slot rows into the split slot workspace, or partial rows.  The
// slots of a tile come in aligned groups of 4 that map to 4 consecutive
// aligned positions of the split workspace (blocks have a multiple of 4
// slots), i.e. one 16-byte unit (4 k) per column: each warp stages its
// 32 rows x 32 columns in shared memory and writes whole units, a warp
// covering 512 contiguous bytes per hi/lo half.
template <>
__device__ __forceinline__ void epilogue<Ph1>(const Smem& s, const Ph1& ph, int64_t ntiles, int nct, int ncols,
                                              uint32_t tmem) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int quarter = warp & 3;
  const int half = (warp - 2) >> 2;
  const int row = 32 * quarter + lane;
  float* tile = s.epi + (warp - 2) * 32 * kEpiLd;
  int tl = 0;
  int64_t id;
  for (; next_tile(s, tl, id); tl++) {
    const int b = tl & 1;
    if (!wait_bar(s, AF + b, (uint32_t)(tl >> 1) & 1)) break;
    umma::fence_after_sync();
    if (s.failed()) break;
    const int64_t w = id / nct;
    const int ct = (int)(id % nct);
    const int n0 = ct * kN;
    const int nv = min(kN, ncols - n0);
    const P1Item& it = ph.items[w];
    const bool zero = it.nchunk == 0;
    const bool partial = it.out_row >= 0;
    RowSinkY psink{(partial && row < it.nq) ? ph.part + (it.out_row + row) * ph.ldp + n0 : nullptr};
    // split-workspace chunk and k of the 8 slot groups of this warp's rows
    uint8_t* gchunk[8];
    int gk[8];
#pragma unroll
    for (int q = 0; q < 8; q++) {
      const int r4 = 32 * quarter + 4 * q;
      gchunk[q] = nullptr;
      gk[q] = 0;
      if (!partial && r4 < it.nq) {
        const int64_t p = ph.slotpos[it.map_off + r4];
        gchunk[q] = ph.zsplit + ((p >> 4) * nct + ct) * (int64_t)kBChunkBytes;
        gk[q] = (int)(p & 12);
      }
    }
#pragma unroll 1
    for (int j = 4 * half; j < 4 * half + 4; j++) {
      float v[32];
      if (zero) {
#pragma unroll
        for (int i = 0; i < 32; i++) v[i] = 0.f;
      } else {
        umma::tmem_ld32(tmem + (uint32_t)(b * kN) + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(32 * j), v);
      }
      if (partial) {
        psink.put(32 * j, nv, v);
      } else {
#pragma unroll
        for (int i = 0; i < 32; i++) tile[lane * kEpiLd + i] = v[i];
        __syncwarp();
        const int n = 32 * j + lane;  // column of this lane
#pragma unroll
        for (int q = 0; q < 8; q++) {
          if (gchunk[q] && n < nv)
            put4(gchunk[q], gchunk[q] + kBBytes, n, gk[q], tile[(4 * q + 0) * kEpiLd + lane],
                 tile[(4 * q + 1) * kEpiLd + lane], tile[(4 * q + 2) * kEpiLd + lane], tile[(4 * q + 3) * kEpiLd + lane]);
        }
        __syncwarp();
      }
    }
    umma::fence_before_sync();
    umma::mbar_arrive(&s.bar[AE + b]);
  }
}

template <class Ph>
__global__ void __launch_bounds__(kThreads, 1)
    k_tc_apply(const Ph ph, int64_t nwork, int nct, int ncols, const uint8_t* __restrict__ astream,
               unsigned long long* __restrict__ counter, int* __restrict__ err) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  const Smem s = smem_layout(smem_raw);
  const int warp = threadIdx.x >> 5;
  const int64_t ntiles = nwork * nct;
  if (threadIdx.x == 0) {
    for (int i = FULL; i < EMPTY; i++) umma::mbar_init(&s.bar[i], 1);
    for (int i = EMPTY; i < AF; i++) umma::mbar_init(&s.bar[i], 1);
    for (int i = AF; i < AE; i++) umma::mbar_init(&s.bar[i], 1);
    for (int i = AE; i < FIN; i++) umma::mbar_init(&s.bar[i], 32 * kEpiWarps);
    umma::mbar_init(&s.bar[FIN], 1);
    for (int i = QF; i < QE; i++) umma::mbar_init(&s.bar[i], 1);
    for (int i = QE; i < NBAR; i++) umma::mbar_init(&s.bar[i], 1 + 32 * kEpiWarps);
    *s.fail = 0;
    umma::fence_mbar_init();
  }
  if (warp == kMmaWarp) umma::tmem_alloc(s.tmem_slot, kTmemCols);
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tmem = *s.tmem_slot;
  if (warp == kProdWarp) {
    if ((threadIdx.x & 31) == 0) producer(s, ph, ntiles, nct, astream, counter);
  } else if (warp == kMmaWarp) {
    if ((threadIdx.x & 31) == 0) mma_issuer(s, ph, ntiles, nct, tmem);
    __syncwarp();
  } else {
    epilogue<Ph>(s, ph, ntiles, nct, ncols, tmem);
  }
  umma::fence_before_sync();
  __syncthreads();
  if (threadIdx.x == 0 && s.failed()) atomicExch(err, 1);
  if (warp == kMmaWarp) {
    umma::fence_after_sync();
    umma::tmem_dealloc(tmem, kTmemCols);
  }
}

// Writes the split operator chunks: element (i, k) of chunk c (see TcAChunk)
// into its hi and lo blocks in the tensor-core layout.
__global__ void k_tc_build_a(const TcAChunk* __restrict__ d, int64_t n, const float* __restrict__ fac,
                             const float* __restrict__ nearv, uint8_t* __restrict__ out) {
  for (int64_t c = blockIdx.x; c < n; c += gridDim.x) {
    const TcAChunk ch = d[c];
    const float* src = ch.near ? nearv : fac;
    uint8_t* hi = out + c * kAChunkBytes;
    uint8_t* lo = hi + kABytes;
    for (int e = threadIdx.x; e < kM * kK / 4; e += blockDim.x) {
      const int i = e >> 2, kq = e & 3;
      float v[4];
#pragma unroll
      for (int u = 0; u < 4; u++) {
        const int k = 4 * kq + u;
        v[u] = (i >= ch.row_lo && i < ch.row_hi && k < ch.kv)
                   ? src[ch.src_off + (int64_t)(i - ch.row_lo) * ch.si + (int64_t)k * ch.sk]
                   : 0.f;
      }
      put4(hi, lo, i, 4 * kq, v[0], v[1], v[2], v[3]);
    }
  }
}

// Sum the partials of a cluster split into several leaf groups and write the
// slot rows into the split slot workspace.
__global__ void k_phase1_reduce_tc(const P1Reduce* __restrict__ items, const float* __restrict__ part, int64_t ldp,
                                   const int64_t* __restrict__ slotpos, uint8_t* __restrict__ zsplit, int nct,
                                   int ncols) {
  const P1Reduce it = items[blockIdx.x];
  const int64_t total = (int64_t)it.nq * ncols;
  for (int64_t e = threadIdx.x + (int64_t)blockIdx.y * blockDim.x; e < total; e += (int64_t)blockDim.x * gridDim.y) {
    const int q = (int)(e / ncols), n = (int)(e % ncols);
    float acc = 0.f;
    for (int c = 0; c < it.nch; c++) acc += part[(it.part_row + (int64_t)c * it.nq + q) * ldp + n];
    const int64_t p = slotpos[it.map_off + q];
    put1(zsplit + ((p >> 4) * nct + n / kN) * (int64_t)kBChunkBytes, n % kN, (int)(p & 15), acc);
  }
}

}  // namespace

// Tensor-core apply for an FP32 operator (cluster order).
fkf_status hmat_apply_clustered_tc(fkf_hmat* h, const float* X, int64_t ldx, float* Y, int64_t ldy, int64_t ncols) {
  fkf_ctx* ctx = h->ctx;
  const int64_t P = h->tc_panel;
  const int64_t nct_max = cdiv(P, kN);
  const size_t xbytes = (size_t)std::max<int64_t>(h->n_tcx, 1) * nct_max * kBChunkBytes;
  if (h->xsplit.bytes < xbytes) FKF_TRY(dev_alloc(ctx, h->xsplit, xbytes));
  const size_t zbytes = (size_t)std::max<int64_t>(h->n_tcz, 1) * nct_max * kBChunkBytes;
  if (h->zsplit.bytes < zbytes) {
    // padding slots of the split workspace are never written: they start (and stay) zero
    FKF_TRY(dev_alloc(ctx, h->zsplit, zbytes));
    FKF_CUDA(ctx, cudaMemsetAsync(h->zsplit.p, 0, zbytes, ctx->stream));
  }
  const size_t pbytes = (size_t)std::max<int64_t>(h->tc_part_rows, 1) * P * sizeof(float);
  if (h->part.bytes < pbytes) FKF_TRY(dev_alloc(ctx, h->part, pbytes));
  if (h->tc_err.bytes < 64) {
    FKF_TRY(dev_alloc(ctx, h->tc_err, 64));
    FKF_CUDA(ctx, cudaMemsetAsync(h->tc_err.p, 0, 64, ctx->stream));
  }
  // tile counters of the two phases at tc_err + 16, + 24 bytes
  unsigned long long* counters = reinterpret_cast<unsigned long long*>(h->tc_err.as<char>() + 16);
  int sms = 0;
  FKF_CUDA(ctx, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
  FKF_CUDA(ctx, cudaFuncSetAttribute(k_tc_apply<Ph1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes));
  FKF_CUDA(ctx, cudaFuncSetAttribute(k_tc_apply<Ph2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes));
  const uint8_t* astream = h->tca.as<uint8_t>();
  for (int64_t c0 = 0; c0 < ncols; c0 += P) {
    const int nc = (int)std::min<int64_t>(P, ncols - c0);
    const int nct = (int)cdiv(nc, kN);
    FKF_CUDA(ctx, cudaMemsetAsync(counters, 0, 2 * sizeof(unsigned long long), ctx->stream));
    if (h->n_tcx > 0) {
      k_tc_split_x<<<dim3((unsigned)h->n_tcx, (unsigned)nct), 256, 0, ctx->stream>>>(
          X + c0, ldx, nc, h->tcxmap.as<TcXChunk>(), 0, nct, h->xsplit.as<uint8_t>());
      FKF_LAUNCHED(ctx);
    }
    if (h->n_tcp1 > 0) {
      const Ph1 ph{h->tcp1.as<P1Item>(), h->xsplit.as<uint8_t>(), h->tcslot.as<int64_t>(), h->zsplit.as<uint8_t>(),
                   h->part.as<float>(), P};
      const int grid = (int)std::min<int64_t>(sms, h->n_tcp1 * nct);
      k_tc_apply<Ph1><<<grid, kThreads, kSmemBytes, ctx->stream>>>(ph, h->n_tcp1, nct, nc, astream, counters,
                                                                   h->tc_err.as<int>());
      FKF_LAUNCHED(ctx);
    }
    if (h->n_tcred > 0) {
      k_phase1_reduce_tc<<<dim3((unsigned)h->n_tcred, 4), 256, 0, ctx->stream>>>(
          h->tcred.as<P1Reduce>(), h->part.as<float>(), P, h->tcslot.as<int64_t>(), h->zsplit.as<uint8_t>(), nct, nc);
      FKF_LAUNCHED(ctx);
    }
    const Ph2 ph{h->tctile.as<TcTile>(), h->tcseg.as<TcSeg>(), h->zsplit.as<uint8_t>(), h->xsplit.as<uint8_t>(),
                 Y + c0, ldy};
    const int grid = (int)std::min<int64_t>(sms, h->n_tctile * nct);
    k_tc_apply<Ph2><<<grid, kThreads, kSmemBytes, ctx->stream>>>(ph, h->n_tctile, nct, nc, astream, counters + 1,
                                                                 h->tc_err.as<int>());
    FKF_LAUNCHED(ctx);
  }
  return FKF_OK;
}

fkf_status tc_gemm_f32(fkf_ctx* ctx, const TcGemmProblem* p, int np, const float* B, int64_t ldb, int64_t kb,
                       int ncols, TcGemmWs& ws) {
  if (np < 1 || np > 2) return set_err(ctx, FKF_EINVAL, "tc_gemm_f32: 1 or 2 problems");
  if (ncols <= 0) return FKF_OK;
  PhGemm ph{};
  int64_t nw[2] = {0, 0}, a0[2] = {0, 0}, achunks = 0;
  int nch[2] = {0, 0};
  for (int i = 0; i < np; i++) {
    if (p[i].K < 0 || p[i].K > kb || p[i].rows < 0) return set_err(ctx, FKF_EINVAL, "tc_gemm_f32: bad shape");
    nw[i] = cdiv(p[i].rows, kM);
    nch[i] = (int)cdiv(p[i].K, kK);
    a0[i] = achunks;
    achunks += nw[i] * nch[i];
  }
  ph.C0 = p[0].C, ph.ldc0 = p[0].ldc, ph.rows0 = p[0].rows, ph.nch0 = nch[0];
  if (np > 1) ph.C1 = p[1].C, ph.ldc1 = p[1].ldc, ph.rows1 = p[1].rows, ph.nch1 = nch[1], ph.a1 = a0[1];
  ph.nw0 = nw[0];
  const int64_t nwork = nw[0] + nw[1];
  if (nwork == 0) return FKF_OK;
  const int nct = (int)cdiv(ncols, kN);
  const int64_t nbx = cdiv(kb, kK);
  const size_t abytes = (size_t)std::max<int64_t>(achunks, 1) * kAChunkBytes;
  const size_t bbytes = (size_t)std::max<int64_t>(nbx, 1) * nct * kBChunkBytes;
  if (ws.asplit.bytes < abytes) FKF_TRY(dev_alloc(ctx, ws.asplit, abytes));
  if (ws.bsplit.bytes < bbytes) FKF_TRY(dev_alloc(ctx, ws.bsplit, bbytes));
  if (ws.ctl.bytes < 64) {
    FKF_TRY(dev_alloc(ctx, ws.ctl, 64));
    FKF_CUDA(ctx, cudaMemsetAsync(ws.ctl.p, 0, 64, ctx->stream));
  }
  unsigned long long* counter = reinterpret_cast<unsigned long long*>(ws.ctl.as<char>() + 16);
  FKF_CUDA(ctx, cudaMemsetAsync(counter, 0, sizeof(unsigned long long), ctx->stream));
  if (nbx > 0) {
    k_tc_split_x<<<dim3((unsigned)nbx, (unsigned)nct), 256, 0, ctx->stream>>>(B, ldb, ncols, nullptr, kb, nct,
                                                                              ws.bsplit.as<uint8_t>());
    FKF_LAUNCHED(ctx);
  }
  for (int i = 0; i < np; i++) {
    if (nw[i] == 0 || nch[i] == 0) continue;
    k_tc_split_rows<<<dim3((unsigned)nw[i], (unsigned)nch[i]), 256, 0, ctx->stream>>>(
        p[i].A, p[i].lda, p[i].rows, p[i].K, nch[i], ws.asplit.as<uint8_t>() + a0[i] * kAChunkBytes);
    FKF_LAUNCHED(ctx);
  }
  ph.bsplit = ws.bsplit.as<uint8_t>();
  int sms = 0;
  FKF_CUDA(ctx, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
  FKF_CUDA(ctx, cudaFuncSetAttribute(k_tc_apply<PhGemm>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes));
  const int grid = (int)std::min<int64_t>(sms, nwork * nct);
  k_tc_apply<PhGemm><<<grid, kThreads, kSmemBytes, ctx->stream>>>(ph, nwork, nct, ncols, ws.asplit.as<uint8_t>(),
                                                                  counter, ws.ctl.as<int>());
  FKF_LAUNCHED(ctx);
  return FKF_OK;
}

fkf_status tc_gemm_check(fkf_ctx* ctx, TcGemmWs& ws) {
  if (!ws.ctl.p) return FKF_OK;
  int e = 0;
  FKF_CUDA(ctx, cudaMemcpyAsync(&e, ws.ctl.p, 4, cudaMemcpyDeviceToHost, ctx->stream));
  FKF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (e) {
    FKF_CUDA(ctx, cudaMemsetAsync(ws.ctl.p, 0, 64, ctx->stream));
    return set_err(ctx, FKF_ETIMEOUT, "tensor-core GEMM: an mbarrier wait expired");
  }
  return FKF_OK;
}

fkf_status hmat_upload_tc(fkf_hmat* h, TcUpload& tu) {
  fkf_ctx* ctx = h->ctx;
  std::vector<TcAChunk> ch;
  // phase-1 items in the order of their first row (the items of all tree
  // levels that read the same X chunks run together and share them in L2),
  // longest first among equal starts
  std::vector<size_t> order(tu.items.size());
  for (size_t i = 0; i < order.size(); i++) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) {
    const P1Item &x = tu.items[a], &y = tu.items[b];
    return x.x_row != y.x_row ? x.x_row < y.x_row : x.nchunk > y.nchunk;
  });
  std::vector<P1Item> items;
  items.reserve(order.size());
  for (size_t i : order) {
    P1Item it = tu.items[i];
    it.a_chunk0 = (int64_t)ch.size();
    ch.insert(ch.end(), tu.item_chunks[i].begin(), tu.item_chunks[i].end());
    items.push_back(it);
  }
  for (TcTile& t : tu.tiles) {
    t.a_chunk0 = (int64_t)ch.size();
    int nch = 0;
    for (int j = 0; j < t.nseg; j++) {
      const TcSeg& sg = tu.segs[t.seg0 + j];
      for (int k0 = 0; k0 < sg.K; k0 += kK, nch++) {
        TcAChunk a{};
        a.src_off = sg.a_off + k0;
        a.si = sg.lda;
        a.sk = 1;
        a.row_lo = sg.row_lo;
        a.row_hi = sg.row_hi;
        a.kv = std::min(kK, sg.K - k0);
        a.near = sg.near;
        ch.push_back(a);
      }
    }
    t.nchunk = nch;
  }
  if (!items.empty()) FKF_TRY(dev_upload(ctx, h->tcp1, items.data(), items.size() * sizeof(P1Item)));
  if (!tu.reduces.empty())
    FKF_TRY(dev_upload(ctx, h->tcred, tu.reduces.data(), tu.reduces.size() * sizeof(P1Reduce)));
  if (!tu.tiles.empty()) FKF_TRY(dev_upload(ctx, h->tctile, tu.tiles.data(), tu.tiles.size() * sizeof(TcTile)));
  FKF_TRY(dev_upload(ctx, h->tcseg, tu.segs.data(), std::max<size_t>(tu.segs.size(), 1) * sizeof(TcSeg)));
  if (!tu.xmap.empty()) FKF_TRY(dev_upload(ctx, h->tcxmap, tu.xmap.data(), tu.xmap.size() * sizeof(TcXChunk)));
  FKF_TRY(dev_upload(ctx, h->tcslot, tu.slotmap.data(), tu.slotmap.size() * sizeof(int64_t)));
  h->n_tcp1 = (int64_t)items.size();
  h->n_tcred = (int64_t)tu.reduces.size();
  h->n_tctile = (int64_t)tu.tiles.size();
  h->n_tcx = (int64_t)tu.xmap.size();
  h->n_tcz = tu.nz;
  h->tc_part_rows = tu.part_rows;
  // columns per pass: keep the split slot workspace under ~24 GB
  int64_t panel = 1024;
  while (panel > kN && (double)h->n_tcz * (panel / kN) * kBChunkBytes > 24e9) panel /= 2;
  h->tc_panel = panel;
  h->n_tca = (int64_t)ch.size();
  FKF_TRY(dev_alloc(ctx, h->tca, (size_t)std::max<int64_t>(h->n_tca, 1) * kAChunkBytes));
  if (h->n_tca > 0) {
    DevBuf desc;
    FKF_TRY(dev_upload(ctx, desc, ch.data(), ch.size() * sizeof(TcAChunk)));
    const int grid = (int)std::min<int64_t>(h->n_tca, 152 * 8);
    k_tc_build_a<<<grid, 256, 0, ctx->stream>>>(desc.as<TcAChunk>(), h->n_tca, h->fac.as<float>(),
                                                h->nearv.as<float>(), h->tca.as<uint8_t>());
    FKF_LAUNCHED(ctx);
    FKF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  }
  h->engine = 1;
  return FKF_OK;
}

fkf_status hmat_tc_check(fkf_hmat* h) {
  if (!h->tc_err.p) return FKF_OK;
  int e = 0;
  FKF_CUDA(h->ctx, cudaMemcpyAsync(&e, h->tc_err.p, 4, cudaMemcpyDeviceToHost, h->ctx->stream));
  FKF_CUDA(h->ctx, cudaStreamSynchronize(h->ctx->stream));
  if (e) {
    FKF_CUDA(h->ctx, cudaMemsetAsync(h->tc_err.p, 0, 64, h->ctx->stream));
    return set_err(h->ctx, FKF_ETIMEOUT, "tensor-core H-apply: an mbarrier wait expired");
  }
  return FKF_OK;
}

// Build the tensor-core work lists from the per-leaf segment lists and the
// cluster factor layout (host).
void hmat_build_tc_schedule(const std::vector<P2Leaf>& leaves, const std::vector<P2Seg>& segs,
                            std::vector<TcTile>& tiles, std::vector<TcSeg>& tsegs) {
  size_t i = 0;
  while (i < leaves.size()) {
    TcTile t{};
    t.row0 = leaves[i].row0;
    t.seg0 = (int)tsegs.size();
    int rows = 0;
    while (i < leaves.size() && rows + leaves[i].rows <= 128 && leaves[i].row0 == t.row0 + rows) {
      const P2Leaf& lf = leaves[i];
      const int ro = rows;
      for (int k = 0; k < lf.nseg; k++) {
        const P2Seg& sg = segs[lf.seg0 + k];
        const int64_t a_off = sg.a_off + (int64_t)lf.pad * sg.lda;
        bool merged = false;
        for (size_t q = t.seg0; q < tsegs.size(); q++) {
          TcSeg& e = tsegs[q];
          if (e.near == sg.near && e.b_row == sg.b_row && e.K == sg.K && e.lda == sg.lda && e.row_hi == ro &&
              e.a_off + (int64_t)(e.row_hi - e.row_lo) * e.lda == a_off) {
            e.row_hi = ro + lf.rows;
            merged = true;
            break;
          }
        }
        if (!merged) {
          TcSeg e{};
          e.a_off = a_off;
          e.b_row = sg.b_row;
          e.lda = sg.lda;
          e.K = sg.K;
          e.near = sg.near;
          e.row_lo = ro;
          e.row_hi = ro + lf.rows;
          tsegs.push_back(e);
        }
      }
      rows += lf.rows;
      i++;
    }
    t.rows = rows;
    t.nseg = (int)tsegs.size() - t.seg0;
    tiles.push_back(t);
  }
}
