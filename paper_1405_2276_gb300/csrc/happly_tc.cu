// H-apply on the 5th-generation tensor cores (FP32 operators).  Both phases
// of the two-phase apply run as 128 x 256 output tiles of tcgen05.mma with
// FP32 accumulators in TMEM.  Every FP32 value is split into two terms and
// each product is accumulated as hi*hi + hi*lo + lo*hi, in one of two
// element formats:
//   F = 1 (3xTF32, kind::tf32): hi = tf32(x), lo = tf32(x - hi);
//   F = 2 (scaled 2xFP16, kind::f16, twice the MMA rate): x is first scaled
//     by a power of two (exact), hi = fp16(x s), lo = fp16(x s - hi).  The
//     scales keep every operand inside FP16's range with room for lo:
//     operator rows (per slot in phase 1, per point in phase 2), the slot
//     columns of phase 2 (inverse of the slot's phase-1 scale, so that the
//     slot products pass between the phases without rescaling), and the
//     columns of X (per apply); the phase-2 epilogue removes the point and
//     column scales.  Each term then carries 11 significant bits, the pair
//     22, as in 3xTF32, down to 2^-17 of its row's (column's) scale; smaller
//     elements keep an absolute error below 2^-25 of that scale.
//
// Both operands reach shared memory already split, in the tensor core's
// K-major core-matrix layout, one bulk copy per operand and K-chunk of 16:
//   * the operator (A): split once when the operator is built (or the
//     format changes), as one stream of chunks (128 x 16 hi block, then lo)
//     per phase-1 item and per phase-2 tile;
//   * the vectors (B): X is split per column pass into 16-row chunks per leaf
//     (rows padded to a multiple of 16), and phase 1 writes its products
//     straight into the split slot workspace (16-slot chunks per cluster).
// Phase 1 swaps the roles inside the MMA: the two 128-column halves of an X
// chunk are A and the operator chunk (slots) is B, with N = the item's slot
// count rounded up to 16, so that the accumulator lanes are vector columns.
//
// One persistent CTA per SM, warp-specialised:
//   warp 0     producer (one thread): two bulk copies per chunk into one of
//              the stages, completion counted in bytes on full[s];
//   warp 1     MMA issuer (one thread): three products per K-step, commits
//              to empty[s], and to acc_full after a tile's last chunk; also
//              allocates and frees TMEM;
//   warps 2-9  epilogue: tcgen05.ld of the finished accumulator (two warps
//              per TMEM lane quarter, one per half of the columns), stores,
//              arrive on acc_empty.
// Two accumulators (2 x 256 TMEM columns) let the epilogue of one tile run
// under the MMAs of the next.  Tiles are taken in order from a global
// counter (the producer takes the next one and passes its index to the MMA
// and epilogue roles through a small queue in shared memory): CTAs running at
// once work on neighbouring tiles, which share operator chunks (the column
// tiles of one work item) and X or ancestors' slot chunks, in L2, and a CTA
// that drew short tiles takes more of them.  Every mbarrier wait is bounded:
// an expired wait sets a flag, every role leaves its loop, the MMA issuer
// waits (bounded) for its outstanding MMAs, TMEM is freed and the host sees
// the error flag.
#include <cuda_fp16.h>

#include <algorithm>
#include <cstring>
#include <type_traits>

#include "common.h"
#include "umma.cuh"

// Chunks per pipeline stage and stage counts of the two formats
// (compile-time tuning knobs).  A stage's MMAs end with one commit, and each
// commit costs the MMA pipe a gap: fewer, larger stages keep it busier.
#ifndef FKF_TC_TF32_CHUNKS_PER_STAGE
#define FKF_TC_TF32_CHUNKS_PER_STAGE 1
#endif
#ifndef FKF_TC_STAGES_TF32
#define FKF_TC_STAGES_TF32 (4 / FKF_TC_TF32_CHUNKS_PER_STAGE)
#endif
// tcgen05 fence after each stage's full-barrier wait (the bulk copies and
// the MMAs are both async-proxy operations ordered by the mbarrier)
#ifndef FKF_TC_STAGE_FENCE
#define FKF_TC_STAGE_FENCE 1
#endif
#ifndef FKF_TC_F16_CHUNKS_PER_STAGE
#define FKF_TC_F16_CHUNKS_PER_STAGE 4
#endif
#ifndef FKF_TC_STAGES_F16
#define FKF_TC_STAGES_F16 (8 / FKF_TC_F16_CHUNKS_PER_STAGE)
#endif
// the second FP16 pipeline shape (kernel code 3) that the autotuner tries
#ifndef FKF_TC_F16_ALT_CHUNKS_PER_STAGE
#define FKF_TC_F16_ALT_CHUNKS_PER_STAGE 2
#endif
#ifndef FKF_TC_STAGES_F16_ALT
#define FKF_TC_STAGES_F16_ALT 4
#endif

namespace {

constexpr int kM = 128;           // tile rows = TMEM lanes
constexpr int kN = 256;           // tile columns = MMA N
constexpr int kK = umma::kChunk;  // 16: K per chunk
constexpr int kEpiWarps = 8;      // warps 2-9: two per TMEM lane quarter, one per column half
constexpr int kQ = 8;             // tile-index queue (producer -> MMA, epilogue)
constexpr int kBarBytes = 384;
constexpr int kTail = 640;        // barriers, TMEM address, flag, queue
constexpr int kProdWarp = 0, kMmaWarp = 1;
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr uint32_t kTmemCols = 2 * kN;
constexpr uint32_t kMaxPolls = 1u << 22;

// Kernel codes F: 1 = 3xTF32; 2 and 3 = the scaled 2xFP16 format with two
// pipeline shapes (2: four K-chunks per stage, two stages; 3: two chunks per
// stage, four stages), chosen per operator by hmat_autotune.  fmt_of(F) is
// the element format (1 or 2) of the split operands.
__host__ __device__ constexpr int fmt_of(int F) { return F == 1 ? 1 : 2; }

// Geometry of kernel code F's split chunks and pipeline.
template <int F>
struct Geo {
  static constexpr int kFmt = fmt_of(F);
  static constexpr int kEl = kFmt == 1 ? 4 : 2;    // bytes per element
  static constexpr int kPer = 16 / kEl;            // elements of one core-matrix row (16 bytes)
  static constexpr int kMmaK = kFmt == 1 ? 8 : 16; // K per MMA
  static constexpr int kABytes = kM * kK * kEl;    // one half (hi or lo) of an A chunk
  static constexpr int kAChunk = 2 * kABytes;
  static constexpr int kBBytes = kN * kK * kEl;    // one half of a B chunk (256 columns)
  static constexpr int kBChunk = 2 * kBBytes;
  static constexpr int kCPS = F == 1 ? FKF_TC_TF32_CHUNKS_PER_STAGE
                                     : (F == 2 ? FKF_TC_F16_CHUNKS_PER_STAGE
                                               : FKF_TC_F16_ALT_CHUNKS_PER_STAGE);  // chunks per stage
  static constexpr int kStage = kCPS * (kAChunk + kBChunk);
  static constexpr int kS = F == 1 ? FKF_TC_STAGES_TF32
                                   : (F == 2 ? FKF_TC_STAGES_F16 : FKF_TC_STAGES_F16_ALT);  // pipeline stages
  static constexpr uint32_t kSBO = (kK / kPer) * 128;  // next 8-row group
  static constexpr uint32_t kIdesc = kFmt == 1 ? umma::idesc_tf32(kM, kN) : umma::idesc_f16(kM, kN);
  // every epilogue stores straight from TMEM (no staging tiles): the room
  // left on the SM holds one FP64 tile CTA of concurrent work
  static constexpr int kSmemRows = kS * kStage + kTail;
  // barrier indices
  static constexpr int FULL = 0, EMPTY = FULL + kS, AF = EMPTY + kS, AE = AF + 2, FIN = AE + 2, QF = FIN + 1,
                       QE = QF + kQ, NBAR = QE + kQ;
  static_assert(kSmemRows <= 232448, "shared memory per CTA");
  static_assert(NBAR * 8 <= kBarBytes, "barrier area");
  // byte offset of element (row, k) in a K-major no-swizzle chunk of kK columns
  __device__ static __forceinline__ uint32_t off(int row, int k) {
    return (uint32_t)((row >> 3) * kSBO + (k / kPer) * 128 + (row & 7) * 16 + (k % kPer) * kEl);
  }
};

// Tile queue entry (producer -> MMA issuer, epilogue).
struct TileQ {
  int64_t id;  // packed (job, tile), -1: no more tiles
  int32_t nch; // K-chunks of the tile
  int32_t n;   // phase 1: MMA N (the item's slots rounded up to 16)
};

template <int F>
struct Smem {
  uint8_t* base;
  uint64_t* bar;
  uint32_t* tmem_slot;
  int* fail;
  uint32_t polls;  // poll limit of the pipeline waits (kMaxPolls unless a caller lowered it)
  TileQ* q;  // [kQ] tile entries (id -1: no more tiles)

  // stage s: the A chunks of its kCPS chunks (consecutive), then their B chunks
  __device__ __forceinline__ uint8_t* a(int s) const { return base + s * Geo<F>::kStage; }
  __device__ __forceinline__ uint8_t* b(int s) const {
    return base + s * Geo<F>::kStage + Geo<F>::kCPS * Geo<F>::kAChunk;
  }
  __device__ __forceinline__ bool failed() const { return *reinterpret_cast<volatile int*>(fail) != 0; }
  __device__ __forceinline__ void set_fail() const { atomicExch(fail, 1); }
};

template <int F>
__device__ __forceinline__ Smem<F> smem_layout(uint8_t* base) {
  Smem<F> s;
  s.base = base;
  uint8_t* tail = base + Geo<F>::kS * Geo<F>::kStage;
  s.bar = reinterpret_cast<uint64_t*>(tail);
  s.tmem_slot = reinterpret_cast<uint32_t*>(tail + kBarBytes);
  s.fail = reinterpret_cast<int*>(tail + kBarBytes + 8);
  s.q = reinterpret_cast<TileQ*>(tail + kBarBytes + 16);
  return s;
}

// A pipeline wait (stages, accumulators, tile queue): gives up after s.polls
// polls and marks the CTA failed, which makes every role unwind.
template <int F>
__device__ __forceinline__ bool wait_bar(const Smem<F>& s, int i, uint32_t parity) {
  if (umma::mbar_wait(&s.bar[i], parity, s.polls)) return true;
  s.set_fail();
  return false;
}

// An unwind wait (MMA completion before TMEM is released, bulk copies landed
// before the CTA exits): always the full kMaxPolls, whatever s.polls is.
template <int F>
__device__ __forceinline__ bool wait_bar_unwind(const Smem<F>& s, int i, uint32_t parity) {
  if (umma::mbar_wait(&s.bar[i], parity, kMaxPolls)) return true;
  s.set_fail();
  return false;
}

// ---- splitting into the tensor-core layout ----------------------------------
__device__ __forceinline__ void split_f16(float x, uint32_t& h, uint32_t& l) {
  const __half hh = __float2half_rn(x);
  const __half ll = __float2half_rn(x - __half2float(hh));
  h = __half_as_ushort(hh);
  l = __half_as_ushort(ll);
}

// kPer consecutive elements v[0..kPer) of one row, starting at k (a multiple
// of kPer): one 16-byte store per half.
template <int F>
__device__ __forceinline__ void put_unit(uint8_t* hi_base, uint8_t* lo_base, int row, int k, const float* v) {
  uint4 h, l;
  if constexpr (fmt_of(F) == 1) {
    umma::split_tf32(v[0], h.x, l.x);
    umma::split_tf32(v[1], h.y, l.y);
    umma::split_tf32(v[2], h.z, l.z);
    umma::split_tf32(v[3], h.w, l.w);
  } else {
    uint32_t a[8], b[8];
#pragma unroll
    for (int i = 0; i < 8; i++) split_f16(v[i], a[i], b[i]);
    h = make_uint4(a[0] | a[1] << 16, a[2] | a[3] << 16, a[4] | a[5] << 16, a[6] | a[7] << 16);
    l = make_uint4(b[0] | b[1] << 16, b[2] | b[3] << 16, b[4] | b[5] << 16, b[6] | b[7] << 16);
  }
  const uint32_t off = Geo<F>::off(row, k);
  *reinterpret_cast<uint4*>(hi_base + off) = h;
  *reinterpret_cast<uint4*>(lo_base + off) = l;
}

// Four consecutive elements of one row starting at k (a multiple of 4).
template <int F>
__device__ __forceinline__ void put4(uint8_t* hi_base, uint8_t* lo_base, int row, int k, float v0, float v1, float v2,
                                     float v3) {
  const uint32_t off = Geo<F>::off(row, k);
  if constexpr (fmt_of(F) == 1) {
    uint4 h, l;
    umma::split_tf32(v0, h.x, l.x);
    umma::split_tf32(v1, h.y, l.y);
    umma::split_tf32(v2, h.z, l.z);
    umma::split_tf32(v3, h.w, l.w);
    *reinterpret_cast<uint4*>(hi_base + off) = h;
    *reinterpret_cast<uint4*>(lo_base + off) = l;
  } else {
    uint32_t a[4], b[4];
    split_f16(v0, a[0], b[0]);
    split_f16(v1, a[1], b[1]);
    split_f16(v2, a[2], b[2]);
    split_f16(v3, a[3], b[3]);
    *reinterpret_cast<uint2*>(hi_base + off) = make_uint2(a[0] | a[1] << 16, a[2] | a[3] << 16);
    *reinterpret_cast<uint2*>(lo_base + off) = make_uint2(b[0] | b[1] << 16, b[2] | b[3] << 16);
  }
}

// One value into a split B chunk (row = column n of the tile, k = row in chunk).
template <int F>
__device__ __forceinline__ void put1(uint8_t* chunk, int n, int k, float v) {
  const uint32_t off = Geo<F>::off(n, k);
  uint32_t h, l;
  if constexpr (fmt_of(F) == 1) {
    umma::split_tf32(v, h, l);
    *reinterpret_cast<uint32_t*>(chunk + off) = h;
    *reinterpret_cast<uint32_t*>(chunk + Geo<F>::kBBytes + off) = l;
  } else {
    split_f16(v, h, l);
    *reinterpret_cast<uint16_t*>(chunk + off) = (uint16_t)h;
    *reinterpret_cast<uint16_t*>(chunk + Geo<F>::kBBytes + off) = (uint16_t)l;
  }
}

// Largest power of two <= x, limited to [2^-100, 2^100]; 1 for x that is not
// a positive finite number.
__device__ __forceinline__ float pow2_floor(float x) {
  if (!(x > 0.f) || isinf(x)) return 1.f;
  int e;
  frexpf(x, &e);  // x = f 2^e, f in [0.5, 1)
  return ldexpf(1.f, min(max(e - 1, -100), 100));
}

// Split X: chunk x (blockIdx.x) of 16 rows (xmap; without a map, rows 16x..
// of a matrix of urows rows), column tile ct (blockIdx.y) of 256 columns ->
// out + (x * nct + ct) * kBChunk; columns scaled by cscale (F = 2).  Thread
// units are (column n, kPer rows): a warp reads 32 consecutive floats of a
// row and writes 512 contiguous bytes per half.
template <int F>
__global__ void __launch_bounds__(256) k_tc_split_x(const float* __restrict__ X, int64_t ldx, int ncols,
                                                    const TcXChunk* __restrict__ xmap, int64_t urows, int nct,
                                                    const float* __restrict__ cscale, uint8_t* __restrict__ out) {
  using G = Geo<F>;
  TcXChunk xc;
  if (xmap) {
    xc = xmap[blockIdx.x];
  } else {
    xc.row0 = (int64_t)blockIdx.x * kK;
    xc.rows = (int)min((int64_t)kK, urows - xc.row0);
  }
  const int ct = blockIdx.y;
  uint8_t* chunk = out + ((int64_t)blockIdx.x * nct + ct) * G::kBChunk;
#pragma unroll
  for (int i = 0; i < kK / G::kPer; i++) {
    const int u = threadIdx.x + 256 * i;
    const int n = u & (kN - 1), kq = u >> 8;
    const int col = ct * kN + n;
    const float sc = (fmt_of(F) == 2 && col < ncols) ? cscale[col] : 1.f;
    float v[G::kPer];
#pragma unroll
    for (int j = 0; j < G::kPer; j++) {
      const int k = G::kPer * kq + j;
      v[j] = (k < xc.rows && col < ncols) ? X[(xc.row0 + k) * ldx + col] * sc : 0.f;
    }
    put_unit<F>(chunk, chunk + G::kBBytes, n, G::kPer * kq, v);
  }
}

// Sparse X (TcSparseX) into the split format of k_tc_split_x: thread per row
// i of X, the row's entries summed per column in their order (as a dense X
// built by adding them to a zero row would hold), times the column scale,
// split into the row's chunk; pos[p] receives the byte offset of the hi
// element written for entry p (repeated columns repeat it).  The rest of the
// split X must already be zero.
template <int F>
__global__ void __launch_bounds__(256) k_tc_scatter_x(int64_t n, const int64_t* __restrict__ colptr,
                                                      const int* __restrict__ crow, const double* __restrict__ cval,
                                                      int nct, const int* __restrict__ rowchunk,
                                                      const TcXChunk* __restrict__ xmap,
                                                      const float* __restrict__ cscale, uint8_t* __restrict__ out,
                                                      int64_t* __restrict__ pos) {
  using G = Geo<F>;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t p1 = colptr[i + 1];
  const int c = rowchunk[i];
  const int k = (int)(i - xmap[c].row0);
  for (int64_t p = colptr[i]; p < p1;) {
    const int col = crow[p];
    float v = 0.f;
    int64_t q = p;
    for (; q < p1 && crow[q] == col; q++) v += (float)cval[q];
    const int64_t base = ((int64_t)c * nct + col / kN) * G::kBChunk;
    put1<F>(out + base, col % kN, k, v * cscale[col]);
    const int64_t at = base + G::off(col % kN, k);
    for (; p < q; p++) pos[p] = at;
  }
}

// Zero the elements (hi and lo) a previous sparse split wrote: pos holds
// their offsets, -1 for entries that wrote none (dropped indices); offsets
// outside the split X of `bytes` bytes are skipped.
template <int F>
__global__ void k_tc_clear_x(const int64_t* __restrict__ pos, int64_t cnt, uint8_t* __restrict__ out,
                             int64_t bytes) {
  using G = Geo<F>;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= cnt) return;
  const int64_t at = pos[i];
  if (at < 0 || (at & (G::kEl - 1)) || at + G::kBBytes + G::kEl > bytes) return;
  if constexpr (G::kEl == 2) {
    *reinterpret_cast<uint16_t*>(out + at) = 0;
    *reinterpret_cast<uint16_t*>(out + at + G::kBBytes) = 0;
  } else {
    *reinterpret_cast<uint32_t*>(out + at) = 0;
    *reinterpret_cast<uint32_t*>(out + at + G::kBBytes) = 0;
  }
}

// Chunk of every row of X (each X chunk holds rows [row0, row0 + rows)).
__global__ void k_tc_rowchunk(const TcXChunk* __restrict__ xmap, int64_t nx, int* __restrict__ rowchunk) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= nx) return;
  const TcXChunk x = xmap[c];
  for (int k = 0; k < x.rows; k++) rowchunk[x.row0 + k] = (int)c;
}

// Column maxima of |X| (rows x ncols, ld ldx) as ordered float bits; grid
// (column blocks of 256, row blocks).
__global__ void __launch_bounds__(256) k_colmax(const float* __restrict__ X, int64_t ldx, int64_t rows, int ncols,
                                                int64_t rows_per_block, unsigned* __restrict__ cmax) {
  const int col = blockIdx.x * 256 + threadIdx.x;
  if (col >= ncols) return;
  const int64_t r0 = (int64_t)blockIdx.y * rows_per_block;
  const int64_t r1 = min(rows, r0 + rows_per_block);
  float m = 0.f;
  for (int64_t r = r0; r < r1; r++) m = fmaxf(m, fabsf(X[r * ldx + col]));
  atomicMax(&cmax[col], __float_as_uint(m));
}

// X column scales: the largest power of two with max |X_j| * s_j <= 1/2 (so
// that a phase-1 slot value, bounded by its operator row's scaled L1 bound
// 2^15 times max |X_j s_j|, stays below FP16's 65504); inverse scales after
// them.
__global__ void k_colscale(const unsigned* __restrict__ cmax, int ncols, float* __restrict__ cs) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ncols) return;
  const float s = pow2_floor(0.5f / __uint_as_float(cmax[j]));
  cs[j] = s;
  cs[ncols + j] = 1.f / s;
}

// Split a row-major matrix A (rows x K, ld lda) into operator chunks of
// kernel code F: tile t (blockIdx.x) of 128 rows, K chunk c (blockIdx.y) of 16
// columns -> out + (t * nch + c) * kAChunk; rows >= rows and columns >= K are
// zero; the FP16 format scales row r by rs[r].  Thread units are (row, kPer
// columns): a warp reads runs of 8 (TF32) or 4 (FP16) rows and writes 512
// contiguous bytes per half.
template <int F>
__global__ void __launch_bounds__(256) k_tc_split_rows(const float* __restrict__ A, int64_t lda, int64_t rows, int K,
                                                       int nch, const float* __restrict__ rs,
                                                       uint8_t* __restrict__ out) {
  using G = Geo<F>;
  constexpr int P = G::kPer, NU = kK / P;
  const int64_t t = blockIdx.x;
  const int c = blockIdx.y;
  uint8_t* hi = out + (t * nch + c) * (int64_t)G::kAChunk;
  const bool vec = ((reinterpret_cast<uintptr_t>(A) & 15) == 0) && (lda & 3) == 0;
#pragma unroll
  for (int i = 0; i < kM * NU / 256; i++) {
    const int u = threadIdx.x + 256 * i;
    const int kq = u % NU, row = u / NU;
    const int64_t r = t * kM + row;
    const int k = c * kK + P * kq;
    float v[P];
#pragma unroll
    for (int j = 0; j < P; j++) v[j] = 0.f;
    if (r < rows) {
      const float* src = A + r * lda + k;
      const float sc = (fmt_of(F) == 2 && rs) ? rs[r] : 1.f;
#pragma unroll
      for (int j0 = 0; j0 < P; j0 += 4) {
        if (vec && k + j0 + 4 <= K) {
          const float4 q = *reinterpret_cast<const float4*>(src + j0);
          v[j0] = q.x * sc, v[j0 + 1] = q.y * sc, v[j0 + 2] = q.z * sc, v[j0 + 3] = q.w * sc;
        } else {
#pragma unroll
          for (int j = j0; j < j0 + 4; j++)
            if (k + j < K) v[j] = src[j] * sc;
        }
      }
    }
    put_unit<F>(hi, hi + G::kABytes, row, P * kq, v);
  }
}

// Row scales of the FP16 format: the largest power of two with the row's max
// |element| <= 2^14 (one warp per row).
__global__ void __launch_bounds__(256) k_rowscale(const float* __restrict__ A, int64_t lda, int64_t rows, int K,
                                                  float* __restrict__ rs) {
  const int64_t r = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (r >= rows) return;
  float m = 0.f;
  for (int k = lane; k < K; k += 32) m = fmaxf(m, fabsf(A[r * lda + k]));
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) rs[r] = pow2_floor(16384.f / m);
}

// ---- the work items ----------------------------------------------------------
// Phase 2: tiles of 128 consecutive rows; B segments = chunks of the split
// slot workspace (far) or of the split X (near); output rows of Y, with the
// point and column scales removed (F = 2: rpt = point scales, cinv = inverse
// column scales of the pass).
struct Ph2 {
  const TcTile* tiles;
  const TcSeg* segs;
  const uint8_t* zsplit;
  const uint8_t* xsplit;
  float* Y;
  int64_t ldy;
  const float* rpt;
  const float* cinv;
  const uint8_t* astream;  // split operator stream
  int nct, ncols;          // column tiles and columns of the pass
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
  __device__ __forceinline__ float* row_dst(int64_t w, int row, float& rinv) const {
    const TcTile& t = tiles[w];
    if (row >= t.rows) return nullptr;
    rinv = rpt ? 1.f / rpt[t.row0 + row] : 1.f;
    return Y + (t.row0 + row) * ldy;
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
  const uint8_t* astream;
  int nct, ncols;
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
  int64_t a1;      // first A chunk of problem 1 (problem 0 starts at 0)
  int64_t nw0;     // row tiles of problem 0
  int nch0, nch1;  // K chunks per tile
  const float* cinv;  // inverse column scales of B (FP16 format), else null
  const uint8_t* astream;
  int nct, ncols;
  const float *rs0, *rs1;  // row scales of A_0, A_1 (FP16 format), else null
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
  __device__ __forceinline__ float* row_dst(int64_t w, int row, float& rinv) const {
    const bool p = w >= nw0;
    const int64_t r = (p ? w - nw0 : w) * kM + row;
    if (r >= (p ? rows1 : rows0)) return nullptr;
    const float* rs = p ? rs1 : rs0;
    rinv = rs ? 1.f / rs[r] : 1.f;
    return (p ? C1 : C0) + r * (p ? ldc1 : ldc0);
  }
};

// A set of jobs of one phase run by one persistent launch: one job (a
// filter's apply, passed by value) or a device list of jobs whose tiles are
// numbered consecutively (t0[j] = first global tile of job j).  Queue entries
// carry (job, tile within the job).
constexpr int kJobShift = 44;
constexpr int64_t kLocalMask = (int64_t(1) << kJobShift) - 1;

template <class Ph>
struct JobSet {
  Ph one;
  const Ph* list;
  const int64_t* t0;
  int nj;  // 0: the single job `one`
  __device__ __forceinline__ Ph get(int j) const { return nj ? list[j] : one; }
  __device__ __forceinline__ int64_t pack(int64_t id) const {
    if (!nj) return id;
    int lo = 0, hi = nj - 1;  // largest j with t0[j] <= id
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (t0[mid] <= id)
        lo = mid;
      else
        hi = mid - 1;
    }
    return ((int64_t)lo << kJobShift) | (id - t0[lo]);
  }
};

// ---- roles -----------------------------------------------------------------
// Slot count of a phase-1 item rounded up to the MMA's N granularity.
__device__ __forceinline__ int p1_n(int nq) { return (nq + 15) & ~15; }
// Halves of column tile ct that hold vector columns (the other is all zero).
__device__ __forceinline__ int p1_halves(int ncols, int ct) { return ncols - ct * kN > kN / 2 ? 2 : 1; }
// Next tile of this CTA: taken from the global counter by the producer and
// published in the queue; every consumer reads each queue entry once.
template <int F>
__device__ __forceinline__ bool next_tile(const Smem<F>& s, int qi, int64_t& id, int* nch = nullptr,
                                          int* n = nullptr) {
  using G = Geo<F>;
  const int slot = qi % kQ;
  if (!wait_bar(s, G::QF + slot, (uint32_t)(qi / kQ) & 1)) return false;
  volatile TileQ* e = &s.q[slot];
  id = e->id;
  if (nch) *nch = e->nch;
  if (n) *n = e->n;
  umma::mbar_arrive(&s.bar[G::QE + slot]);
  return id >= 0;
}

// A tile's chunks go kCPS to a stage (the last stage of a tile may hold
// fewer): one bulk copy for their A chunks (consecutive in the operator
// stream), one per B chunk.
// Returns through g the number of stages whose bulk copies it issued (each
// stage is issued whole: every exit is at a stage boundary).
template <int F, class Ph>
__device__ __forceinline__ void producer(const Smem<F>& s, const JobSet<Ph>& js, int64_t ntiles,
                                         unsigned long long* counter, int64_t& g) {
  using G = Geo<F>;
  g = 0;  // stages issued
  for (int qi = 0;; qi++) {
    const int64_t id = (int64_t)atomicAdd(counter, 1ull);
    const int64_t packed = id < ntiles ? js.pack(id) : -1;
    const int slot = qi % kQ;
    // the tile's chunk count (and phase 1's MMA N) travel with its index, so
    // the MMA issuer reads nothing from global memory between tiles
    Ph ph{};
    int64_t w = 0;
    int ct = 0, nch = 0, nn = 0;
    if (packed >= 0) {
      ph = js.get((int)(packed >> kJobShift));
      const int64_t lid = packed & kLocalMask;
      w = lid / ph.nct;
      ct = (int)(lid % ph.nct);
      nch = ph.nchunk(w);
      if constexpr (std::is_same<Ph, Ph1>::value) nn = p1_n(ph.items[w].nq);
    }
    if (qi >= kQ && !wait_bar(s, G::QE + slot, (uint32_t)((qi / kQ) - 1) & 1)) return;
    volatile TileQ* e = &s.q[slot];
    e->id = packed;
    e->nch = nch;
    e->n = nn;
    umma::mbar_arrive(&s.bar[G::QF + slot]);
    if (packed < 0) return;
    const int nct = ph.nct;
    const uint8_t* ap = ph.astream + ph.a_chunk0(w) * (int64_t)G::kAChunk;
    const int ns = ph.nseg(w);
    int t = 0, j = 0, nin = 0, st = 0;  // chunk of the tile, chunk within the stage, chunks in the stage
    for (int sg = 0; sg < ns; sg++) {
      int64_t c0;
      int nc;
      const uint8_t* bsrc = ph.seg(w, sg, c0, nc);
      for (int c = 0; c < nc; c++, t++) {
        if (j == 0) {
          if (s.failed()) return;
          st = (int)(g % G::kS);
          if (g >= G::kS && !wait_bar(s, G::EMPTY + st, (uint32_t)((g / G::kS) - 1) & 1)) return;
          nin = min(G::kCPS, nch - t);
          umma::mbar_arrive_expect_tx(&s.bar[G::FULL + st], (uint32_t)(nin * (G::kAChunk + G::kBChunk)));
          umma::bulk_g2s(s.a(st), ap, (uint32_t)(nin * G::kAChunk), &s.bar[G::FULL + st]);
          ap += nin * G::kAChunk;
        }
        umma::bulk_g2s(s.b(st) + j * G::kBChunk, bsrc + ((c0 + c) * nct + ct) * (int64_t)G::kBChunk, G::kBChunk,
                       &s.bar[G::FULL + st]);
        if (++j == nin) {
          j = 0;
          g++;
        }
      }
    }
  }
}

template <int F>
__device__ __forceinline__ void issue_mma(const uint8_t* a, const uint8_t* b, uint32_t acc, bool first) {
  using G = Geo<F>;
  // descriptors by offset from the chunk's first core matrix (see issue_mma_p1)
  const uint64_t ah0 = umma::smem_desc(umma::smem_u32(a), G::kSBO);
  const uint64_t bh0 = umma::smem_desc(umma::smem_u32(b), G::kSBO);
#pragma unroll
  for (int kk = 0; kk < kK / G::kMmaK; kk++) {
    const uint64_t koff = (uint64_t)((kk * 2 * umma::kLBO) >> 4);  // two core matrices along K per MMA
    const uint64_t ah = ah0 + koff, al = ah + (uint64_t)(G::kABytes >> 4);
    const uint64_t bh = bh0 + koff, bl = bh + (uint64_t)(G::kBBytes >> 4);
    const uint32_t acc0 = (first && kk == 0) ? 0u : 1u;
    if constexpr (fmt_of(F) == 1) {
      umma::mma_tf32(acc, ah, bh, G::kIdesc, acc0);
      umma::mma_tf32(acc, ah, bl, G::kIdesc, 1u);
      umma::mma_tf32(acc, al, bh, G::kIdesc, 1u);
    } else {
      umma::mma_f16(acc, ah, bh, G::kIdesc, acc0);
      umma::mma_f16(acc, ah, bl, G::kIdesc, 1u);
      umma::mma_f16(acc, al, bh, G::kIdesc, 1u);
    }
  }
}

// Phase 1 with the roles swapped: the 128-row halves of the split X chunk
// (rows = vector columns) are A (M = 128), the operator chunk (rows = slots)
// is B with N = the item's slot count rounded up to 16, and half h
// accumulates at TMEM column offset 128 h.  The accumulator lanes are then
// vector columns, so the epilogue writes the K-major split slot workspace
// without a transpose, and short slot tiles cost no padded MMA rows.
template <int F>
__device__ __forceinline__ void issue_mma_p1(const uint8_t* op, const uint8_t* x, uint32_t acc, bool first, int nh,
                                             uint32_t idesc) {
  using G = Geo<F>;
  // descriptors by offset from the chunk's first core matrix (the start
  // address field holds addr >> 4 and stays below 2^14 inside shared memory)
  const uint64_t bh0 = umma::smem_desc(umma::smem_u32(op), G::kSBO);
  const uint64_t ah0 = umma::smem_desc(umma::smem_u32(x), G::kSBO);
  for (int h = 0; h < nh; h++) {
    const uint32_t d = acc + (uint32_t)(h * (kN / 2));
#pragma unroll
    for (int kk = 0; kk < kK / G::kMmaK; kk++) {
      const uint64_t koff = (uint64_t)((kk * 2 * umma::kLBO) >> 4);
      const uint64_t ah = ah0 + (uint64_t)((h * (G::kBBytes / 2)) >> 4) + koff, al = ah + (uint64_t)(G::kBBytes >> 4);
      const uint64_t bh = bh0 + koff, bl = bh + (uint64_t)(G::kABytes >> 4);
      const uint32_t acc0 = (first && kk == 0) ? 0u : 1u;
      if constexpr (fmt_of(F) == 1) {
        umma::mma_tf32(d, ah, bh, idesc, acc0);
        umma::mma_tf32(d, ah, bl, idesc, 1u);
        umma::mma_tf32(d, al, bh, idesc, 1u);
      } else {
        umma::mma_f16(d, ah, bh, idesc, acc0);
        umma::mma_f16(d, ah, bl, idesc, 1u);
        umma::mma_f16(d, al, bh, idesc, 1u);
      }
    }
  }
}


template <int F, class Ph>
__device__ __forceinline__ void mma_issuer(const Smem<F>& s, const JobSet<Ph>& js, uint32_t tmem) {
  using G = Geo<F>;
  int64_t g = 0;
  int tl = 0;
  bool ok = true;
  int64_t id;
  int nch = 0, nn = 0;
  for (; ok && next_tile(s, tl, id, &nch, &nn); tl++) {
    int nh = 0;
    uint32_t idesc1 = 0;
    if constexpr (std::is_same<Ph, Ph1>::value) {
      const Ph ph = js.get((int)(id >> kJobShift));  // a kernel parameter unless the launch has a job list
      nh = p1_halves(ph.ncols, (int)((id & kLocalMask) % ph.nct));
      idesc1 = fmt_of(F) == 1 ? umma::idesc_tf32(kM, nn) : umma::idesc_f16(kM, nn);
    }
    const int b = tl & 1;
    if (tl >= 2 && !wait_bar(s, G::AE + b, (uint32_t)((tl >> 1) - 1) & 1)) break;
    umma::fence_after_sync();
    const uint32_t acc = tmem + (uint32_t)(b * kN);
    for (int c = 0; c < nch; g++) {
      const int st = (int)(g % G::kS);
      const int nin = min(G::kCPS, nch - c);
      if (s.failed() || !wait_bar(s, G::FULL + st, (uint32_t)(g / G::kS) & 1)) {
        ok = false;
        break;
      }
#if FKF_TC_STAGE_FENCE
      umma::fence_after_sync();
#endif
      for (int j = 0; j < nin; j++, c++) {
        if constexpr (std::is_same<Ph, Ph1>::value)
          issue_mma_p1<F>(s.a(st) + j * G::kAChunk, s.b(st) + j * G::kBChunk, acc, c == 0, nh, idesc1);
        else
          issue_mma<F>(s.a(st) + j * G::kAChunk, s.b(st) + j * G::kBChunk, acc, c == 0);
      }
      umma::commit(&s.bar[G::EMPTY + st]);
    }
    if (!ok) break;
    if (nch > 0)
      umma::commit(&s.bar[G::AF + b]);
    else
      umma::mbar_arrive(&s.bar[G::AF + b]);
  }
  // every MMA issued here has completed before TMEM is released
  umma::commit(&s.bar[G::FIN]);
  wait_bar_unwind(s, G::FIN, 0);
}

// Epilogue stores of one row's 32 columns [c0, c0 + 32) of a tile, times
// rinv * cinv[c] when cinv is given.
struct RowSinkY {
  float* dst;
  __device__ __forceinline__ void put(int c0, int nv, float (&v)[32], float rinv, const float* cinv) const {
    if (!dst) return;
    if (cinv) {
#pragma unroll
      for (int i = 0; i < 32; i++) v[i] *= rinv * (c0 + i < nv ? cinv[c0 + i] : 0.f);
    }
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

// Rows of a row-major output: Ph supplies the destination row (nullptr past
// the tile's rows) and its inverse scale, and nchunk (0: the tile is zero).
template <int F, class Ph>
__device__ __forceinline__ void epilogue_rows(const Smem<F>& s, const JobSet<Ph>& js, uint32_t tmem) {
  using G = Geo<F>;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int quarter = warp & 3;  // TMEM lanes 32*quarter.. are this warp's
  const int half = (warp - 2) >> 2;
  const int row = 32 * quarter + lane;
  int tl = 0;
  int64_t id;
  int nch = 0;
  for (; next_tile(s, tl, id, &nch); tl++) {
    const int b = tl & 1;
    // the tile's destination rows and scales are loaded while its MMAs run
    const Ph ph = js.get((int)(id >> kJobShift));
    const int64_t lid = id & kLocalMask;
    const int64_t w = lid / ph.nct;
    const int n0 = (int)(lid % ph.nct) * kN;
    const int nv = min(kN, ph.ncols - n0);
    const bool zero = nch == 0;
    float rinv = 1.f;
    float* dst = ph.row_dst(w, row, rinv);
    const RowSinkY sink{dst ? dst + n0 : nullptr};
    const float* cinv = ph.cinv ? ph.cinv + n0 : nullptr;
    if (!wait_bar(s, G::AF + b, (uint32_t)(tl >> 1) & 1)) break;
    umma::fence_after_sync();
    if (s.failed()) break;
    // a warp whose 32 rows are all past the tile's rows has nothing to store
    const int jend = __any_sync(0xffffffffu, dst != nullptr) ? 4 * half + 4 : 4 * half;
#pragma unroll 1
    for (int j = 4 * half; j < jend; j++) {
      float v[32];
      if (zero) {
#pragma unroll
        for (int i = 0; i < 32; i++) v[i] = 0.f;
      } else {
        umma::tmem_ld32(tmem + (uint32_t)(b * kN) + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(32 * j), v);
      }
      sink.put(32 * j, nv, v, rinv, cinv);
    }
    umma::fence_before_sync();
    umma::mbar_arrive(&s.bar[G::AE + b]);
  }
}

// Phase 1: slot values into the split slot workspace, or partial rows.  The
// accumulator of half h holds (vector column, slot): lane = column
// 128 h + 32 quarter + lane of the column tile, TMEM column = slot of the
// item.  A lane loads 32 slots of its column and stores them as the 16-row
// K-major chunks of the workspace: the slots of a tile come in aligned
// groups of 4 that map to 4 consecutive aligned positions (blocks have a
// multiple of 4 slots), i.e. 4 k of one workspace row; two groups that
// fill one 16-byte FP16 unit go out as one store per half.  Partial rows
// (clusters split over several leaf groups) are FP32 rows of the partial
// buffer.  (Slot values stay scaled: phase 2's operator columns carry the
// inverse scales.)
template <int F>
__device__ __forceinline__ void epilogue_p1(const Smem<F>& s, const JobSet<Ph1>& js, uint32_t tmem) {
  using G = Geo<F>;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int quarter = warp & 3;
  const int half = (warp - 2) >> 2;
  const int nl = half * (kN / 2) + 32 * quarter + lane;  // column within the column tile
  int tl = 0;
  int64_t id;
  int nch = 0;
  for (; next_tile(s, tl, id, &nch); tl++) {
    const int b = tl & 1;
    // the tile's descriptors and slot positions are loaded while its MMAs
    // run: lane L holds the workspace position of slot group L (slots 4L..)
    const Ph1 ph = js.get((int)(id >> kJobShift));
    const int64_t lid = id & kLocalMask;
    const int nct = ph.nct;
    const int64_t w = lid / nct;
    const int ct = (int)(lid % nct);
    const int n0 = ct * kN;
    const bool col_ok = n0 + nl < ph.ncols;
    const P1Item it = ph.items[w];
    const bool zero = nch == 0;
    const bool partial = it.out_row >= 0;
    const int64_t pl = (!partial && 4 * lane < it.nq) ? ph.slotpos[it.map_off + 4 * lane] : -1;
    if (!wait_bar(s, G::AF + b, (uint32_t)(tl >> 1) & 1)) break;
    umma::fence_after_sync();
    if (s.failed()) break;
    // the warps of an all-zero half (past the pass's columns) have nothing to load
    const bool active = half < p1_halves(ph.ncols, ct);
    const uint32_t tbase = tmem + (uint32_t)(b * kN + half * (kN / 2)) + ((uint32_t)(32 * quarter) << 16);
#pragma unroll 1
    for (int j = 0; active && 32 * j < it.nq; j++) {
      float v[32];
      if (zero) {
#pragma unroll
        for (int i = 0; i < 32; i++) v[i] = 0.f;
      } else {
        umma::tmem_ld32(tbase + (uint32_t)(32 * j), v);
      }
      int64_t p[8];  // workspace positions of this j's 8 slot groups (-1: none)
#pragma unroll
      for (int u = 0; u < 8; u++) p[u] = __shfl_sync(0xffffffffu, pl, 8 * j + u);
      if (!col_ok) continue;
      const int q0 = 32 * j;
      if (partial) {
        float* dst = ph.part + (it.out_row + q0) * ph.ldp + n0 + nl;
#pragma unroll
        for (int i = 0; i < 32; i++)
          if (q0 + i < it.nq) dst[(int64_t)i * ph.ldp] = v[i];
        continue;
      }
#pragma unroll
      for (int u = 0; u < 8; u += 2) {
        if (p[u] < 0) continue;
        uint8_t* ch = ph.zsplit + ((p[u] >> 4) * nct + ct) * (int64_t)G::kBChunk;
        // FP16: two groups that fill one 16-byte unit (positions p, p + 4 with p % 8 == 0)
        if (fmt_of(F) == 2 && p[u + 1] == p[u] + 4 && (p[u] & 7) == 0) {
          put_unit<F>(ch, ch + G::kBBytes, nl, (int)(p[u] & 12), &v[4 * u]);
          continue;
        }
        put4<F>(ch, ch + G::kBBytes, nl, (int)(p[u] & 12), v[4 * u], v[4 * u + 1], v[4 * u + 2], v[4 * u + 3]);
        if (p[u + 1] >= 0) {
          uint8_t* ch1 = ph.zsplit + ((p[u + 1] >> 4) * nct + ct) * (int64_t)G::kBChunk;
          put4<F>(ch1, ch1 + G::kBBytes, nl, (int)(p[u + 1] & 12), v[4 * u + 4], v[4 * u + 5], v[4 * u + 6],
                  v[4 * u + 7]);
        }
      }
    }
    umma::fence_before_sync();
    umma::mbar_arrive(&s.bar[G::AE + b]);
  }
}

template <int F, class Ph>
__device__ __forceinline__ void epilogue(const Smem<F>& s, const JobSet<Ph>& js, uint32_t tmem) {
  if constexpr (std::is_same<Ph, Ph1>::value)
    epilogue_p1<F>(s, js, tmem);
  else
    epilogue_rows<F>(s, js, tmem);
}

template <int F, class Ph>
__global__ void __launch_bounds__(kThreads, 1)
    k_tc_apply(const JobSet<Ph> js, int64_t ntiles, unsigned long long* __restrict__ counter, int* __restrict__ err,
               uint32_t max_polls) {
  using G = Geo<F>;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  Smem<F> s = smem_layout<F>(smem_raw);
  s.polls = max_polls;
  const int warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    for (int i = G::FULL; i < G::EMPTY; i++) umma::mbar_init(&s.bar[i], 1);
    for (int i = G::EMPTY; i < G::AF; i++) umma::mbar_init(&s.bar[i], 1);
    for (int i = G::AF; i < G::AE; i++) umma::mbar_init(&s.bar[i], 1);
    for (int i = G::AE; i < G::FIN; i++) umma::mbar_init(&s.bar[i], 32 * kEpiWarps);
    umma::mbar_init(&s.bar[G::FIN], 1);
    for (int i = G::QF; i < G::QE; i++) umma::mbar_init(&s.bar[i], 1);
    for (int i = G::QE; i < G::NBAR; i++) umma::mbar_init(&s.bar[i], 1 + 32 * kEpiWarps);
    *s.fail = 0;
    umma::fence_mbar_init();
  }
  if (warp == kMmaWarp) umma::tmem_alloc(s.tmem_slot, kTmemCols);
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tmem = *s.tmem_slot;
  if (warp == kProdWarp) {
    if ((threadIdx.x & 31) == 0) {
      int64_t g = 0;
      producer<F>(s, js, ntiles, counter, g);
      // the CTA does not exit (nor does a failed one unwind) while a bulk copy
      // into its shared memory is in flight: wait for the last phase issued to
      // each stage (a phase the MMA thread already consumed reads as complete)
      for (int64_t i = g > G::kS ? g - G::kS : 0; i < g; i++)
        wait_bar_unwind(s, G::FULL + (int)(i % G::kS), (uint32_t)(i / G::kS) & 1);
    }
  } else if (warp == kMmaWarp) {
    if ((threadIdx.x & 31) == 0) mma_issuer<F>(s, js, tmem);
    __syncwarp();
  } else {
    epilogue<F>(s, js, tmem);
  }
  umma::fence_before_sync();
  __syncthreads();
  if (threadIdx.x == 0 && s.failed()) atomicExch(err, 1);
  if (warp == kMmaWarp) {
    umma::fence_after_sync();
    umma::tmem_dealloc(tmem, kTmemCols);
  }
}

// ---- operator stream ---------------------------------------------------------
// Element (i, k) of chunk ch, unscaled (0 outside the chunk's rows and kv).
__device__ __forceinline__ bool chunk_row(const TcAChunk& ch, int i) {
  return (i >= ch.row_lo && i < ch.row_hi) || (i >= ch.row_lo2 && i < ch.row_hi2);
}
__device__ __forceinline__ float chunk_elem(const TcAChunk& ch, const float* fac, const float* nearv, int i, int k) {
  if (k >= ch.kv) return 0.f;
  const float* src = ch.near ? nearv : fac;
  if (i >= ch.row_lo && i < ch.row_hi) return src[ch.src_off + (int64_t)(i - ch.row_lo) * ch.si + (int64_t)k * ch.sk];
  if (i >= ch.row_lo2 && i < ch.row_hi2)
    return src[ch.src_off2 + (int64_t)(i - ch.row_lo2) * ch.si2 + (int64_t)k * ch.sk];
  return 0.f;
}

// Scale passes of format 2 over the chunks of one phase: per scale row (a
// natural slot in phase 1, a point in phase 2) the max |element| (phase 2:
// with the slot columns' inverse scales applied), and in phase 1 the number
// of columns.  One thread per chunk row.
__global__ void __launch_bounds__(128) k_tc_rowmax(const TcAChunk* __restrict__ d, int64_t n, int phase,
                                                   const float* __restrict__ fac, const float* __restrict__ nearv,
                                                   const float* __restrict__ qpos, unsigned* __restrict__ rmax,
                                                   int* __restrict__ cnt) {
  const int i = threadIdx.x;
  for (int64_t c = blockIdx.x; c < n; c += gridDim.x) {
    const TcAChunk ch = d[c];
    if (ch.phase != phase || !chunk_row(ch, i)) continue;
    float m = 0.f;
    for (int k = 0; k < ch.kv; k++) {
      float a = fabsf(chunk_elem(ch, fac, nearv, i, k));
      if (ch.k_off >= 0) a /= qpos[ch.k_off + k];
      m = fmaxf(m, a);
    }
    atomicMax(&rmax[ch.s_off + i], __float_as_uint(m));
    if (cnt) atomicAdd(&cnt[ch.s_off + i], ch.kv);
  }
}

// Slot scales: q_g = largest power of two with q_g * cnt_g * max|V_g| <= 2^15
// (so that q_g |V_g . x| <= 2^15 * max|x| <= 2^14 for column-scaled x),
// stored per natural slot and at the slot's workspace position.
__global__ void k_tc_qscale(int64_t nslots, const unsigned* __restrict__ vmax, const int* __restrict__ cnt,
                            const int64_t* __restrict__ slotpos, float* __restrict__ qslot,
                            float* __restrict__ qpos) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nslots) return;
  const float q = pow2_floor(32768.f / ((float)max(cnt[g], 1) * __uint_as_float(vmax[g])));
  qslot[g] = q;
  qpos[slotpos[g]] = q;
}

// Point scales: largest power of two with the row's max |element| <= 2^14.
__global__ void k_tc_rscale(int64_t n, const unsigned* __restrict__ rmax, float* __restrict__ r) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) r[i] = pow2_floor(16384.f / __uint_as_float(rmax[i]));
}

__global__ void k_fill_f32(int64_t n, float v, float* __restrict__ p) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

// Writes the split operator chunks in format F: element (i, k) of chunk c
// (see TcAChunk; format 2 with its row and column scales) into its hi and lo
// blocks in the tensor-core layout.
template <int F>
__global__ void k_tc_build_a(const TcAChunk* __restrict__ d, int64_t n, const float* __restrict__ fac,
                             const float* __restrict__ nearv, const float* __restrict__ qslot,
                             const float* __restrict__ rpt, const float* __restrict__ qpos,
                             uint8_t* __restrict__ out) {
  using G = Geo<F>;
  constexpr int NU = kK / G::kPer;
  for (int64_t c = blockIdx.x; c < n; c += gridDim.x) {
    const TcAChunk ch = d[c];
    uint8_t* hi = out + c * G::kAChunk;
    uint8_t* lo = hi + G::kABytes;
    for (int e = threadIdx.x; e < kM * NU; e += blockDim.x) {
      const int i = e / NU, kq = e % NU;
      float rs = 1.f;
      if (fmt_of(F) == 2 && chunk_row(ch, i))
        rs = ch.phase == 1 ? qslot[ch.s_off + i] : rpt[ch.s_off + i];
      float v[G::kPer];
#pragma unroll
      for (int u = 0; u < G::kPer; u++) {
        const int k = G::kPer * kq + u;
        float x = chunk_elem(ch, fac, nearv, i, k);
        if (fmt_of(F) == 2 && x != 0.f) {
          x *= rs;
          if (ch.k_off >= 0) x /= qpos[ch.k_off + k];
        }
        v[u] = x;
      }
      put_unit<F>(hi, lo, i, G::kPer * kq, v);
    }
  }
}

// Sum the partials of a cluster split into several leaf groups and write the
// slot rows into the split slot workspace.
template <int F>
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
    put1<F>(zsplit + ((p >> 4) * nct + n / kN) * (int64_t)Geo<F>::kBChunk, n % kN, (int)(p & 15), acc);
  }
}

fkf_status build_stream(fkf_hmat* h, int F);

// Buffers of an apply whose passes have up to nc columns (allocated or grown
// on first use; the slot workspace is cleared when it grows or its format
// changes).
template <int F>
fkf_status tc_buffers(fkf_hmat* h, int64_t nc, cudaStream_t st) {
  using G = Geo<F>;
  fkf_ctx* ctx = h->ctx;
  const int64_t P = h->tc_panel;
  const int64_t nct_max = cdiv(std::min(nc, P), kN);
  const size_t xbytes = (size_t)std::max<int64_t>(h->n_tcx, 1) * nct_max * G::kBChunk;
  if (h->xsplit.bytes < xbytes) {
    h->xs_count = -1;  // fresh memory: no known zero pattern
    FKF_TRY(dev_alloc(ctx, h->xsplit, xbytes));
  }
  const size_t zbytes = (size_t)std::max<int64_t>(h->n_tcz, 1) * nct_max * G::kBChunk;
  if (h->zsplit.bytes < zbytes || h->zsplit_fmt != fmt_of(F)) {
    // padding slots of the split workspace are never written: they start (and stay) zero
    if (h->zsplit.bytes < zbytes) FKF_TRY(dev_alloc(ctx, h->zsplit, zbytes));
    FKF_CUDA(ctx, cudaMemsetAsync(h->zsplit.p, 0, h->zsplit.bytes, st));
    h->zsplit_fmt = fmt_of(F);
  }
  const size_t pbytes = (size_t)std::max<int64_t>(h->tc_part_rows, 1) * P * sizeof(float);
  if (h->part.bytes < pbytes) FKF_TRY(dev_alloc(ctx, h->part, pbytes));
  if (h->tc_err.bytes < 64) {
    FKF_TRY(dev_alloc(ctx, h->tc_err, 64));
    FKF_CUDA(ctx, cudaMemsetAsync(h->tc_err.p, 0, 64, st));
  }
  // column maxima and scales of one pass (format 2)
  if (fmt_of(F) == 2 && h->tc_col.bytes < (size_t)P * 12) FKF_TRY(dev_alloc(ctx, h->tc_col, (size_t)P * 12));
  return FKF_OK;
}

// Split X of one pass (nc columns) on stream st; format 2 first computes the
// column scales (returned in cs: scales, then inverse scales) from the column
// maxima of |X|, scanned here unless the caller supplies them (cmax_in).
template <int F>
fkf_status tc_split_pass(fkf_hmat* h, const float* X, int64_t ldx, int nc, cudaStream_t st, float*& cs,
                         const unsigned* cmax_in) {
  using G = Geo<F>;
  fkf_ctx* ctx = h->ctx;
  const int64_t P = h->tc_panel;
  const int nct = (int)cdiv(nc, kN);
  cs = nullptr;
  if (fmt_of(F) == 2) {
    const unsigned* cmax = cmax_in;
    cs = h->tc_col.as<float>();
    if (!cmax) {
      unsigned* cm = reinterpret_cast<unsigned*>(h->tc_col.as<float>() + 2 * P);
      FKF_CUDA(ctx, cudaMemsetAsync(cm, 0, (size_t)nc * sizeof(unsigned), st));
      const int64_t rpb = 2048;
      k_colmax<<<dim3((unsigned)cdiv(nc, 256), (unsigned)cdiv(h->n, rpb)), 256, 0, st>>>(X, ldx, h->n, nc, rpb, cm);
      FKF_LAUNCHED(ctx);
      cmax = cm;
    }
    k_colscale<<<(unsigned)cdiv(nc, 256), 256, 0, st>>>(cmax, nc, cs);
    FKF_LAUNCHED(ctx);
  }
  if (h->n_tcx == 0) return FKF_OK;
  const TcSparseX* sx = fmt_of(F) == 2 ? h->ctx->x_sparse : nullptr;
  if (!sx) {
    h->xs_count = -1;
    k_tc_split_x<F><<<dim3((unsigned)h->n_tcx, (unsigned)nct), 256, 0, st>>>(X, ldx, nc, h->tcxmap.as<TcXChunk>(), 0,
                                                                             nct, cs, h->xsplit.as<uint8_t>());
    FKF_LAUNCHED(ctx);
    return FKF_OK;
  }
  // sparse X: zero what the previous sparse split wrote (or all of the pass's
  // split X when its content is unknown), then scatter the entries
  if (!cmax_in) return set_err(ctx, FKF_ESTATE, "sparse X without its column maxima");
  uint8_t* xs = h->xsplit.as<uint8_t>();
  if (h->tc_rowchunk.bytes < (size_t)h->n * sizeof(int)) {
    FKF_TRY(dev_alloc(ctx, h->tc_rowchunk, (size_t)h->n * sizeof(int)));
    k_tc_rowchunk<<<(unsigned)cdiv(h->n_tcx, 256), 256, 0, st>>>(h->tcxmap.as<TcXChunk>(), h->n_tcx,
                                                                h->tc_rowchunk.as<int>());
    FKF_LAUNCHED(ctx);
  }
  const int64_t xbytes = h->n_tcx * nct * (int64_t)G::kBChunk;
  const bool known = h->xs_count >= 0 && h->xs_nct == nct;
  if (known && h->xs_count > 0) {
    k_tc_clear_x<F><<<(unsigned)cdiv(h->xs_count, 256), 256, 0, st>>>(h->xs_pos.as<int64_t>(), h->xs_count, xs,
                                                                      xbytes);
    FKF_LAUNCHED(ctx);
  }
  h->xs_count = -1;  // until the scatter below is queued
  if (!known) FKF_CUDA(ctx, cudaMemsetAsync(xs, 0, (size_t)xbytes, st));
  if (h->xs_pos.bytes < (size_t)std::max<int64_t>(sx->nnz, 1) * sizeof(int64_t)) {
    // a larger record: the clear above has read the old one before it is freed
    FKF_CUDA(ctx, cudaStreamSynchronize(st));
    FKF_TRY(dev_alloc(ctx, h->xs_pos, (size_t)std::max<int64_t>(sx->nnz, 1) * sizeof(int64_t)));
  }
  // entries the CSC index dropped (column index outside [0, N)) record no offset
  if (sx->nnz > 0) FKF_CUDA(ctx, cudaMemsetAsync(h->xs_pos.p, 0xff, (size_t)sx->nnz * sizeof(int64_t), st));
  if (sx->n > 0) {
    k_tc_scatter_x<F><<<(unsigned)cdiv(sx->n, 256), 256, 0, st>>>(sx->n, sx->colptr, sx->crow, sx->cval, nct,
                                                                   h->tc_rowchunk.as<int>(), h->tcxmap.as<TcXChunk>(),
                                                                   cs, xs, h->xs_pos.as<int64_t>());
    FKF_LAUNCHED(ctx);
  }
  h->xs_count = sx->nnz;
  h->xs_nct = nct;
  return FKF_OK;
}

template <int F>
Ph1 tc_ph1(fkf_hmat* h, int nc) {
  return Ph1{h->tcp1.as<P1Item>(), h->xsplit.as<uint8_t>(), h->tcslot.as<int64_t>(), h->zsplit.as<uint8_t>(),
             h->part.as<float>(), h->tc_panel, h->tca.as<uint8_t>(), (int)cdiv(nc, kN), nc};
}

template <int F>
Ph2 tc_ph2(fkf_hmat* h, float* Y, int64_t ldy, int nc, const float* cs) {
  return Ph2{h->tctile.as<TcTile>(), h->tcseg.as<TcSeg>(), h->zsplit.as<uint8_t>(), h->xsplit.as<uint8_t>(),
             Y, ldy, fmt_of(F) == 2 ? h->tc_rpt.as<float>() : nullptr, fmt_of(F) == 2 ? cs + nc : nullptr,
             h->tca.as<uint8_t>(),
             (int)cdiv(nc, kN), nc};
}

template <int F>
fkf_status tc_reduce(fkf_hmat* h, int nc, cudaStream_t st) {
  if (h->n_tcred == 0) return FKF_OK;
  k_phase1_reduce_tc<F><<<dim3((unsigned)h->n_tcred, 4), 256, 0, st>>>(
      h->tcred.as<P1Reduce>(), h->part.as<float>(), h->tc_panel, h->tcslot.as<int64_t>(), h->zsplit.as<uint8_t>(),
      (int)cdiv(nc, kN), nc);
  FKF_LAUNCHED(h->ctx);
  return FKF_OK;
}

template <int F>
fkf_status apply_tc(fkf_hmat* h, const float* X, int64_t ldx, float* Y, int64_t ldy, int64_t ncols) {
  using G = Geo<F>;
  fkf_ctx* ctx = h->ctx;
  cudaStream_t st = ctx->stream;
  const int64_t P = h->tc_panel;
  if (ctx->x_sparse && (fmt_of(F) != 2 || ncols > P))
    return set_err(ctx, FKF_ESTATE, "sparse X needs the FP16 split engine and one column pass");
  FKF_TRY(tc_buffers<F>(h, ncols, st));
  // tile counters of the two phases at tc_err + 16, + 24 bytes
  unsigned long long* counters = reinterpret_cast<unsigned long long*>(h->tc_err.as<char>() + 16);
  int sms = 0;
  FKF_CUDA(ctx, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
  FKF_CUDA(ctx, cudaFuncSetAttribute(k_tc_apply<F, Ph1>, cudaFuncAttributeMaxDynamicSharedMemorySize, G::kSmemRows));
  FKF_CUDA(ctx, cudaFuncSetAttribute(k_tc_apply<F, Ph2>, cudaFuncAttributeMaxDynamicSharedMemorySize, G::kSmemRows));
  // the largest carveout (not the smallest that fits phase 2): the SM keeps room for one FP64 tile CTA
  FKF_CUDA(ctx, cudaFuncSetAttribute(k_tc_apply<F, Ph2>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     cudaSharedmemCarveoutMaxShared));
  for (int64_t c0 = 0; c0 < ncols; c0 += P) {
    const int nc = (int)std::min<int64_t>(P, ncols - c0);
    const int nct = (int)cdiv(nc, kN);
    FKF_CUDA(ctx, cudaMemsetAsync(counters, 0, 2 * sizeof(unsigned long long), st));
    float* cs = nullptr;
    FKF_TRY(tc_split_pass<F>(h, X + c0, ldx, nc, st, cs, ctx->x_colmax ? ctx->x_colmax + c0 : nullptr));
    if (h->n_tcp1 > 0) {
      const int grid = (int)std::min<int64_t>(sms, h->n_tcp1 * nct);
      k_tc_apply<F, Ph1><<<grid, kThreads, G::kSmemRows, st>>>(JobSet<Ph1>{tc_ph1<F>(h, nc), nullptr, nullptr, 0},
                                                            h->n_tcp1 * nct, counters, h->tc_err.as<int>(),
                                                            h->tc_polls);
      FKF_LAUNCHED(ctx);
    }
    FKF_TRY(tc_reduce<F>(h, nc, st));
    if (ctx->ph2_mark && c0 + P >= ncols) {  // the last phase 2 of this apply starts here
      FKF_CUDA(ctx, cudaEventRecord(ctx->ph2_mark, st));
      ctx->ph2_marked = true;
    }
    const int grid = (int)std::min<int64_t>(sms, h->n_tctile * nct);
    k_tc_apply<F, Ph2><<<grid, kThreads, G::kSmemRows, st>>>(JobSet<Ph2>{tc_ph2<F>(h, Y + c0, ldy, nc, cs), nullptr,
                                                                      nullptr, 0},
                                                          h->n_tctile * nct, counters + 1, h->tc_err.as<int>(),
                                                          h->tc_polls);
    FKF_LAUNCHED(ctx);
  }
  return FKF_OK;
}

// err -> every operator's tensor-core error flag
__global__ void k_err_fanout(const int* __restrict__ err, int* const* __restrict__ dst, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && *err) atomicExch(dst[i], 1);
}

template <int F>
fkf_status apply_tc_multi(fkf_ctx* ctx, fkf_hmat* const* hs, int nb, const float* const* X, const int64_t* ldx,
                          float* const* Y, const int64_t* ldy, const int64_t* ncols) {
  using G = Geo<F>;
  cudaStream_t st = ctx->stream;
  TcMultiWs& ws = ctx->multi_ws;
  std::vector<Ph1> p1;
  std::vector<Ph2> p2;
  std::vector<int64_t> t1{0}, t2{0};
  std::vector<int*> errs;
  std::vector<int> active;
  for (int f = 0; f < nb; f++) {
    fkf_hmat* h = hs[f];
    if (ncols[f] <= 0) continue;
    if (h->ctx->x_sparse && fmt_of(F) != 2)
      return set_err(ctx, FKF_ESTATE, "sparse X needs the FP16 split engine");
    if (h->tca_fmt != fmt_of(F)) FKF_TRY(build_stream(h, fmt_of(F)));
    FKF_TRY(tc_buffers<F>(h, ncols[f], st));
    const int nc = (int)ncols[f];
    const int nct = (int)cdiv(nc, kN);
    float* cs = nullptr;
    FKF_TRY(tc_split_pass<F>(h, X[f], ldx[f], nc, st, cs, h->ctx->x_colmax));
    if (h->n_tcp1 > 0) {
      p1.push_back(tc_ph1<F>(h, nc));
      t1.push_back(t1.back() + h->n_tcp1 * nct);
    }
    if (h->n_tctile > 0) {
      p2.push_back(tc_ph2<F>(h, Y[f], ldy[f], nc, cs));
      t2.push_back(t2.back() + h->n_tctile * nct);
    }
    errs.push_back(h->tc_err.as<int>());
    active.push_back(f);
  }
  if (active.empty()) return FKF_OK;
  // job lists: Ph1[], Ph2[], t1[], t2[], error flags[] (8-byte aligned pieces)
  auto al = [](size_t x) { return (x + 15) & ~size_t(15); };
  const size_t o1 = 0, o2 = al(o1 + p1.size() * sizeof(Ph1)), ot1 = al(o2 + p2.size() * sizeof(Ph2)),
               ot2 = al(ot1 + t1.size() * 8), oe = al(ot2 + t2.size() * 8), total = al(oe + errs.size() * 8);
  if (!ws.staged) FKF_CUDA(ctx, cudaEventCreateWithFlags(&ws.staged, cudaEventDisableTiming));
  FKF_CUDA(ctx, cudaEventSynchronize(ws.staged));  // the previous upload has left the staging buffer
  if (ws.staging_bytes < total) {
    if (ws.staging) cudaFreeHost(ws.staging);
    ws.staging = nullptr;
    ws.staging_bytes = 0;
    FKF_CUDA(ctx, cudaMallocHost(&ws.staging, total));
    ws.staging_bytes = total;
  }
  if (ws.jobs.bytes < total) FKF_TRY(dev_alloc(ctx, ws.jobs, total));
  if (ws.ctl.bytes < 64) FKF_TRY(dev_alloc(ctx, ws.ctl, 64));
  char* hb = static_cast<char*>(ws.staging);
  std::memcpy(hb + o1, p1.data(), p1.size() * sizeof(Ph1));
  std::memcpy(hb + o2, p2.data(), p2.size() * sizeof(Ph2));
  std::memcpy(hb + ot1, t1.data(), t1.size() * 8);
  std::memcpy(hb + ot2, t2.data(), t2.size() * 8);
  std::memcpy(hb + oe, errs.data(), errs.size() * 8);
  FKF_CUDA(ctx, cudaMemcpyAsync(ws.jobs.p, hb, total, cudaMemcpyHostToDevice, st));
  FKF_CUDA(ctx, cudaEventRecord(ws.staged, st));
  char* db = ws.jobs.as<char>();
  int* err = ws.ctl.as<int>();
  unsigned long long* counters = reinterpret_cast<unsigned long long*>(ws.ctl.as<char>() + 16);
  uint32_t polls = kMaxPolls;  // the smallest limit any operator of the batch asks for
  for (int f : active) polls = std::min(polls, hs[f]->tc_polls);
  FKF_CUDA(ctx, cudaMemsetAsync(ws.ctl.p, 0, 64, st));
  int sms = 0;
  FKF_CUDA(ctx, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
  FKF_CUDA(ctx, cudaFuncSetAttribute(k_tc_apply<F, Ph1>, cudaFuncAttributeMaxDynamicSharedMemorySize, G::kSmemRows));
  FKF_CUDA(ctx, cudaFuncSetAttribute(k_tc_apply<F, Ph2>, cudaFuncAttributeMaxDynamicSharedMemorySize, G::kSmemRows));
  // the largest carveout (not the smallest that fits phase 2): the SM keeps room for one FP64 tile CTA
  FKF_CUDA(ctx, cudaFuncSetAttribute(k_tc_apply<F, Ph2>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     cudaSharedmemCarveoutMaxShared));
  if (!p1.empty()) {
    const JobSet<Ph1> js{p1[0], reinterpret_cast<const Ph1*>(db + o1), reinterpret_cast<const int64_t*>(db + ot1),
                         (int)p1.size()};
    const int grid = (int)std::min<int64_t>(sms, t1.back());
    k_tc_apply<F, Ph1><<<grid, kThreads, G::kSmemRows, st>>>(js, t1.back(), counters, err, polls);
    FKF_LAUNCHED(ctx);
  }
  for (int f : active) FKF_TRY(tc_reduce<F>(hs[f], (int)ncols[f], st));
  for (int f : active) {  // each operator's context may ask to hear when phase 2 starts
    fkf_ctx* c = hs[f]->ctx;
    if (c->ph2_mark) {
      FKF_CUDA(ctx, cudaEventRecord(c->ph2_mark, st));
      c->ph2_marked = true;
    }
  }
  if (!p2.empty()) {
    const JobSet<Ph2> js{p2[0], reinterpret_cast<const Ph2*>(db + o2), reinterpret_cast<const int64_t*>(db + ot2),
                         (int)p2.size()};
    const int grid = (int)std::min<int64_t>(sms, t2.back());
    k_tc_apply<F, Ph2><<<grid, kThreads, G::kSmemRows, st>>>(js, t2.back(), counters + 1, err, polls);
    FKF_LAUNCHED(ctx);
  }
  k_err_fanout<<<1, 64, 0, st>>>(err, reinterpret_cast<int* const*>(db + oe), (int)errs.size());
  FKF_LAUNCHED(ctx);
  return FKF_OK;
}

// Rewrites the split operator stream in format F (format 2: scales first).
fkf_status build_stream(fkf_hmat* h, int F) {
  fkf_ctx* ctx = h->ctx;
  if (h->n_tca == 0) {
    h->tca_fmt = F;
    return FKF_OK;
  }
  const size_t need = (size_t)h->n_tca * (F == 1 ? Geo<1>::kAChunk : Geo<2>::kAChunk);
  if (h->tca.bytes < need) {
    h->tca_fmt = 0;  // the old stream is gone
    FKF_TRY(dev_alloc(ctx, h->tca, need));
  }
  const int grid = (int)std::min<int64_t>(h->n_tca, 152 * 8);
  const TcAChunk* d = h->tcadesc.as<TcAChunk>();
  if (F == 2) {
    // every natural slot (phase-1 row) has a scale: the slot count must be known
    if (h->n_tcp1 > 0 && h->ktot <= 0) return set_err(ctx, FKF_ESTATE, "tensor-core stream: slot count not set");
    const int64_t ns = std::max<int64_t>(h->ktot, 1), npos = std::max<int64_t>(h->n_tcz, 1) * 16;
    FKF_TRY(dev_alloc(ctx, h->tc_qslot, (size_t)ns * sizeof(float)));
    FKF_TRY(dev_alloc(ctx, h->tc_qpos, (size_t)npos * sizeof(float)));
    FKF_TRY(dev_alloc(ctx, h->tc_rpt, (size_t)std::max<int64_t>(h->n, 1) * sizeof(float)));
    DevBuf mx, cnt;
    FKF_TRY(dev_alloc(ctx, mx, (size_t)std::max(ns, h->n) * sizeof(unsigned)));
    FKF_TRY(dev_alloc(ctx, cnt, (size_t)ns * sizeof(int)));
    FKF_CUDA(ctx, cudaMemsetAsync(mx.p, 0, mx.bytes, ctx->stream));
    FKF_CUDA(ctx, cudaMemsetAsync(cnt.p, 0, cnt.bytes, ctx->stream));
    k_fill_f32<<<(unsigned)cdiv(npos, 256), 256, 0, ctx->stream>>>(npos, 1.f, h->tc_qpos.as<float>());
    FKF_LAUNCHED(ctx);
    k_tc_rowmax<<<grid, 128, 0, ctx->stream>>>(d, h->n_tca, 1, h->fac.as<float>(), h->nearv.as<float>(), nullptr,
                                              mx.as<unsigned>(), cnt.as<int>());
    FKF_LAUNCHED(ctx);
    if (h->ktot > 0) {
      k_tc_qscale<<<(unsigned)cdiv(h->ktot, 256), 256, 0, ctx->stream>>>(
          h->ktot, mx.as<unsigned>(), cnt.as<int>(), h->tcslot.as<int64_t>(), h->tc_qslot.as<float>(),
          h->tc_qpos.as<float>());
      FKF_LAUNCHED(ctx);
    }
    FKF_CUDA(ctx, cudaMemsetAsync(mx.p, 0, mx.bytes, ctx->stream));
    k_tc_rowmax<<<grid, 128, 0, ctx->stream>>>(d, h->n_tca, 2, h->fac.as<float>(), h->nearv.as<float>(),
                                              h->tc_qpos.as<float>(), mx.as<unsigned>(), nullptr);
    FKF_LAUNCHED(ctx);
    k_tc_rscale<<<(unsigned)cdiv(h->n, 256), 256, 0, ctx->stream>>>(h->n, mx.as<unsigned>(), h->tc_rpt.as<float>());
    FKF_LAUNCHED(ctx);
    k_tc_build_a<2><<<grid, 256, 0, ctx->stream>>>(d, h->n_tca, h->fac.as<float>(), h->nearv.as<float>(),
                                                   h->tc_qslot.as<float>(), h->tc_rpt.as<float>(),
                                                   h->tc_qpos.as<float>(), h->tca.as<uint8_t>());
    FKF_LAUNCHED(ctx);
    FKF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));  // before mx, cnt are freed
  } else {
    k_tc_build_a<1><<<grid, 256, 0, ctx->stream>>>(d, h->n_tca, h->fac.as<float>(), h->nearv.as<float>(), nullptr,
                                                   nullptr, nullptr, h->tca.as<uint8_t>());
    FKF_LAUNCHED(ctx);
    FKF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  }
  h->tca_fmt = F;
  return FKF_OK;
}

}  // namespace

bool hmat_sparse_x_ok(const fkf_hmat* h, int64_t ncols) {
  return h->prec == FKF_FP32 && h->engine == 2 && h->n_tcx > 0 && ncols > 0 && ncols <= h->tc_panel;
}

// Tensor-core apply for an FP32 operator (cluster order).
fkf_status hmat_apply_clustered_tc(fkf_hmat* h, const float* X, int64_t ldx, float* Y, int64_t ldy, int64_t ncols) {
  if (h->tca_fmt != h->engine) FKF_TRY(build_stream(h, h->engine));
  if (h->engine == 2)
    return h->tc_variant ? apply_tc<3>(h, X, ldx, Y, ldy, ncols) : apply_tc<2>(h, X, ldx, Y, ldy, ncols);
  return apply_tc<1>(h, X, ldx, Y, ldy, ncols);
}

namespace {
// deterministic test vectors in [-1, 1) (a 32-bit integer hash of the index)
__global__ void k_fill_hash(int64_t n, float* __restrict__ x) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t v = (uint32_t)i * 2654435761u;
    v ^= v >> 16;
    v *= 2246822519u;
    v ^= v >> 13;
    x[i] = (float)(v >> 8) * (2.0f / 16777216.0f) - 1.0f;
  }
}
}  // namespace

fkf_status hmat_autotune(fkf_hmat* h, int64_t ncols, int* variant, double* ms_best) {
  fkf_ctx* ctx = h->ctx;
  *variant = h->tc_variant;
  *ms_best = 0.0;
  if (h->prec != FKF_FP32 || h->engine != 2) return FKF_OK;
  const int64_t nc = std::max<int64_t>(1, std::min<int64_t>(ncols, h->tc_panel));
  DevBuf X, Y;
  FKF_TRY(dev_alloc(ctx, X, (size_t)h->n * nc * sizeof(float)));
  FKF_TRY(dev_alloc(ctx, Y, (size_t)h->n * nc * sizeof(float)));
  k_fill_hash<<<152 * 8, 256, 0, ctx->stream>>>(h->n * nc, X.as<float>());
  FKF_LAUNCHED(ctx);
  cudaEvent_t e0, e1;
  FKF_CUDA(ctx, cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return set_err(ctx, FKF_ECUDA, "autotune: event creation failed");
  }
  double best = -1.0;
  int vbest = 0;
  fkf_status st = FKF_OK;
  for (int v = 0; v < 2 && st == FKF_OK; v++) {
    h->tc_variant = v;
    st = hmat_apply_clustered_tc(h, X.as<float>(), nc, Y.as<float>(), nc, nc);  // warm
    if (st != FKF_OK) break;
    cudaEventRecord(e0, ctx->stream);
    for (int k = 0; k < 3 && st == FKF_OK; k++)
      st = hmat_apply_clustered_tc(h, X.as<float>(), nc, Y.as<float>(), nc, nc);
    cudaEventRecord(e1, ctx->stream);
    float ms = 0.f;
    if (st == FKF_OK && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
      st = set_err(ctx, FKF_ECUDA, "autotune: timing failed");
    if (st == FKF_OK && (best < 0 || ms / 3.0 < best)) best = ms / 3.0, vbest = v;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  FKF_TRY(st);
  FKF_TRY(hmat_tc_check(h));
  h->tc_variant = vbest;
  *variant = vbest;
  *ms_best = best;
  return FKF_OK;
}

bool hmat_tc_multi_ok(fkf_hmat* const* hs, int nb, const int64_t* ncols) {
  if (nb < 1) return false;
  const int F = hs[0]->engine;
  for (int f = 0; f < nb; f++) {
    const fkf_hmat* h = hs[f];
    if (h->prec != FKF_FP32 || h->engine != F || (F != 1 && F != 2) || ncols[f] > h->tc_panel ||
        h->ctx->device != hs[0]->ctx->device || h->tc_variant != hs[0]->tc_variant)
      return false;
    for (int g = 0; g < f; g++)
      if (hs[g] == h) return false;  // one operator's buffers serve one apply at a time
  }
  return true;
}

fkf_status hmat_apply_tc_multi(fkf_ctx* ctx, fkf_hmat* const* hs, int nb, const float* const* X, const int64_t* ldx,
                               float* const* Y, const int64_t* ldy, const int64_t* ncols) {
  if (!hmat_tc_multi_ok(hs, nb, ncols)) return set_err(ctx, FKF_EINVAL, "merged apply: operators not compatible");
  if (hs[0]->engine == 2)
    return hs[0]->tc_variant ? apply_tc_multi<3>(ctx, hs, nb, X, ldx, Y, ldy, ncols)
                             : apply_tc_multi<2>(ctx, hs, nb, X, ldx, Y, ldy, ncols);
  return apply_tc_multi<1>(ctx, hs, nb, X, ldx, Y, ldy, ncols);
}

fkf_status hmat_set_engine(fkf_hmat* h, int engine) {
  if (engine == 3) {
    FKF_TRY(hmat_oz_prepare(h));
    h->engine = 3;
    return FKF_OK;
  }
  if (engine != 0 && h->tca_fmt != engine) FKF_TRY(build_stream(h, engine));
  h->engine = engine;
  return FKF_OK;
}

namespace {
template <int F>
fkf_status tc_gemm_impl(fkf_ctx* ctx, const TcGemmProblem* p, int np, const float* B, int64_t ldb, int64_t kb,
                        int ncols, TcGemmWs& ws) {
  using G = Geo<F>;
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
  const size_t abytes = (size_t)std::max<int64_t>(achunks, 1) * G::kAChunk;
  const size_t bbytes = (size_t)std::max<int64_t>(nbx, 1) * nct * G::kBChunk;
  if (ws.asplit.bytes < abytes) FKF_TRY(dev_alloc(ctx, ws.asplit, abytes));
  if (ws.bsplit.bytes < bbytes) FKF_TRY(dev_alloc(ctx, ws.bsplit, bbytes));
  if (ws.ctl.bytes < 64) {
    FKF_TRY(dev_alloc(ctx, ws.ctl, 64));
    FKF_CUDA(ctx, cudaMemsetAsync(ws.ctl.p, 0, 64, ctx->stream));
  }
  unsigned long long* counter = reinterpret_cast<unsigned long long*>(ws.ctl.as<char>() + 16);
  FKF_CUDA(ctx, cudaMemsetAsync(counter, 0, sizeof(unsigned long long), ctx->stream));
  float* rs[2] = {nullptr, nullptr};
  float* cs = nullptr;
  if (fmt_of(F) == 2) {
    // row scales of A_0, A_1, then scales, inverse scales and maxima of B's columns
    const size_t sbytes = (size_t)(p[0].rows + (np > 1 ? p[1].rows : 0) + 3 * (int64_t)ncols + 4) * sizeof(float);
    if (ws.scales.bytes < sbytes) FKF_TRY(dev_alloc(ctx, ws.scales, sbytes));
    rs[0] = ws.scales.as<float>();
    rs[1] = rs[0] + p[0].rows;
    cs = rs[1] + (np > 1 ? p[1].rows : 0);
    unsigned* cmax = reinterpret_cast<unsigned*>(cs + 2 * ncols);
    for (int i = 0; i < np; i++)
      if (p[i].rows > 0) {
        k_rowscale<<<(unsigned)cdiv(p[i].rows, 8), 256, 0, ctx->stream>>>(p[i].A, p[i].lda, p[i].rows, p[i].K, rs[i]);
        FKF_LAUNCHED(ctx);
      }
    FKF_CUDA(ctx, cudaMemsetAsync(cmax, 0, (size_t)ncols * sizeof(unsigned), ctx->stream));
    if (kb > 0) {
      const int64_t rpb = 2048;
      k_colmax<<<dim3((unsigned)cdiv(ncols, 256), (unsigned)cdiv(kb, rpb)), 256, 0, ctx->stream>>>(B, ldb, kb, ncols,
                                                                                                    rpb, cmax);
      FKF_LAUNCHED(ctx);
    }
    k_colscale<<<(unsigned)cdiv(ncols, 256), 256, 0, ctx->stream>>>(cmax, ncols, cs);
    FKF_LAUNCHED(ctx);
    ph.rs0 = rs[0];
    ph.rs1 = np > 1 ? rs[1] : nullptr;
    ph.cinv = cs + ncols;
  }
  if (nbx > 0) {
    k_tc_split_x<F><<<dim3((unsigned)nbx, (unsigned)nct), 256, 0, ctx->stream>>>(B, ldb, ncols, nullptr, kb, nct, cs,
                                                                                 ws.bsplit.as<uint8_t>());
    FKF_LAUNCHED(ctx);
  }
  for (int i = 0; i < np; i++) {
    if (nw[i] == 0 || nch[i] == 0) continue;
    k_tc_split_rows<F><<<dim3((unsigned)nw[i], (unsigned)nch[i]), 256, 0, ctx->stream>>>(
        p[i].A, p[i].lda, p[i].rows, p[i].K, nch[i], rs[i], ws.asplit.as<uint8_t>() + a0[i] * G::kAChunk);
    FKF_LAUNCHED(ctx);
  }
  ph.bsplit = ws.bsplit.as<uint8_t>();
  ph.astream = ws.asplit.as<uint8_t>();
  ph.nct = nct;
  ph.ncols = ncols;
  int sms = 0;
  FKF_CUDA(ctx, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
  FKF_CUDA(ctx, cudaFuncSetAttribute(k_tc_apply<F, PhGemm>, cudaFuncAttributeMaxDynamicSharedMemorySize, G::kSmemRows));
  const int grid = (int)std::min<int64_t>(sms, nwork * nct);
  k_tc_apply<F, PhGemm><<<grid, kThreads, G::kSmemRows, ctx->stream>>>(JobSet<PhGemm>{ph, nullptr, nullptr, 0},
                                                                   nwork * nct, counter, ws.ctl.as<int>(), kMaxPolls);
  FKF_LAUNCHED(ctx);
  return FKF_OK;
}
}  // namespace

fkf_status tc_gemm_f32(fkf_ctx* ctx, const TcGemmProblem* p, int np, const float* B, int64_t ldb, int64_t kb,
                       int ncols, TcGemmWs& ws, int fmt) {
  if (np < 1 || np > 2) return set_err(ctx, FKF_EINVAL, "tc_gemm_f32: 1 or 2 problems");
  if (ncols <= 0) return FKF_OK;
  if (fmt == 1) return tc_gemm_impl<1>(ctx, p, np, B, ldb, kb, ncols, ws);
  return tc_gemm_impl<2>(ctx, p, np, B, ldb, kb, ncols, ws);
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
        a.src_off2 = sg.a_off2 + k0;
        a.si2 = sg.lda2;
        a.row_lo2 = sg.row_lo2;
        a.row_hi2 = sg.row_hi2;
        a.kv = std::min(kK, sg.K - k0);
        a.near = sg.near;
        a.phase = 2;
        a.s_off = t.row0;
        a.k_off = sg.near ? -1 : sg.b_row * kK + k0;
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
  // columns per pass: keep the split slot workspace (FP16 format, the default
  // engine's) under ~24 GB
  int64_t panel = 1024;
  while (panel > kN && (double)h->n_tcz * (panel / kN) * Geo<2>::kBChunk > 24e9) panel /= 2;
  h->tc_panel = panel;
  h->n_tca = (int64_t)ch.size();
  // the stream is sized for the format it holds (build_stream grows it for
  // the larger 3xTF32 chunks)
  h->tca.release();
  if (h->n_tca > 0) FKF_TRY(dev_upload(ctx, h->tcadesc, ch.data(), ch.size() * sizeof(TcAChunk)));
  FKF_TRY(build_stream(h, 2));
  h->engine = 2;
  return FKF_OK;
}

fkf_status hmat_tc_check(fkf_hmat* h) {
  if (h->prec == FKF_FP64) return hmat_oz_check(h);
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
        for (size_t q = t.seg0; q < tsegs.size() && !merged; q++) {
          TcSeg& e = tsegs[q];
          if (e.near != sg.near || e.b_row != sg.b_row || e.K != sg.K) continue;
          const bool two = e.row_hi2 > e.row_lo2;
          if (!two && e.lda == sg.lda && e.row_hi == ro && e.a_off + (int64_t)(e.row_hi - e.row_lo) * e.lda == a_off) {
            e.row_hi = ro + lf.rows;  // the rows continue the segment's A block
            merged = true;
          } else if (two && e.lda2 == sg.lda && e.row_hi2 == ro &&
                     e.a_off2 + (int64_t)(e.row_hi2 - e.row_lo2) * e.lda2 == a_off) {
            e.row_hi2 = ro + lf.rows;  // the rows continue its second A block
            merged = true;
          } else if (!two && sg.near && e.row_hi <= ro) {
            // the same near partner for a later leaf of the tile: its A block
            // becomes the segment's second row range (the B chunks are shared)
            e.a_off2 = a_off;
            e.lda2 = sg.lda;
            e.row_lo2 = ro;
            e.row_hi2 = ro + lf.rows;
            merged = true;
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
