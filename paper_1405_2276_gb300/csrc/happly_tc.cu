// H-apply on the 5th-generation tensor cores (FP32 operators).  Both phases
// of the two-phase apply run as 128 x 256 output tiles of tcgen05.mma
// kind::tf32 with FP32 accumulators in TMEM.  Every FP32 value x is split into
// hi = tf32(x) and lo = tf32(x - hi), and each product is accumulated as
// hi*hi + hi*lo + lo*hi (3xTF32), which keeps FP32-level accuracy.
//
// The operator side (A) is split once, when the operator is built: every
// phase-1 item and every phase-2 tile owns a stream of 16 KB chunks (a
// 128 x 16 TF32 hi block and its lo block, already in the tensor core's
// shared-memory layout), so a chunk reaches shared memory with one bulk copy.
// The vector side (B: rows of X or of the slot workspace) is copied as FP32
// with cp.async and split in shared memory by four producer warps.
//
// One persistent CTA per SM, warp-specialised:
//   warps 0-7  B producers: cp.async kR-1 chunks ahead (kR raw stages),
//              split into three hi/lo stages, arrive on full_b;
//   warp 8     A producer (one thread): bulk copies into four stages, full_a;
//   warp 9     MMA issuer (one thread): six MMAs per chunk (2 K-steps x 3
//              products), commits to empty_a / empty_b, and to acc_full after
//              a tile's last chunk; also allocates and frees TMEM;
//   warps 10-13 epilogue: tcgen05.ld of the finished accumulator, stores,
//              arrive on acc_empty.
// Two accumulators (2 x 256 TMEM columns) let the epilogue of one tile run
// under the MMAs of the next.  Tiles are dealt round-robin over the CTAs, the
// column tiles of one work item consecutively (they share its A stream
// through L2).  Every mbarrier wait is bounded: an expired wait sets a flag,
// every role leaves its loop, the MMA issuer waits (bounded) for its
// outstanding MMAs, TMEM is freed and the host sees the error flag.
#include <algorithm>
#include <cstring>

#include "common.h"
#include "umma.cuh"

// Pipeline depths (compile-time tuning knobs).
#ifndef FKF_TC_RAW_STAGES
#define FKF_TC_RAW_STAGES 3
#endif
#ifndef FKF_TC_A_PREFETCH
#define FKF_TC_A_PREFETCH 0
#endif
#ifndef FKF_TC_B_PREFETCH
#define FKF_TC_B_PREFETCH 0
#endif

namespace {

constexpr int kM = 128;                    // tile rows = TMEM lanes
constexpr int kN = 256;                    // tile columns = MMA N
constexpr int kK = umma::kChunk;           // 16: K per chunk
constexpr int kABytes = kM * kK * 4;       // 8 KB: one TF32 half of an A chunk
constexpr int kAChunkBytes = 2 * kABytes;  // 16 KB: hi | lo
constexpr int kBBytes = kN * kK * 4;       // 16 KB: one TF32 half of a B chunk, or the raw FP32 chunk
constexpr int kSA = 4;                     // A stages
constexpr int kSB = 3;                     // split B stages
constexpr int kR = FKF_TC_RAW_STAGES;      // raw B stages
constexpr int kAPrefetch = FKF_TC_A_PREFETCH;  // A chunks prefetched into L2 ahead of their copy (0: none)
constexpr int kBPrefetch = FKF_TC_B_PREFETCH;  // B chunks prefetched into L2 ahead of their copy (0: none)
constexpr int kSmemBytes = kSA * kAChunkBytes + kSB * 2 * kBBytes + kR * kBBytes + 256;  // 208.25 KB (kR = 3)
static_assert(kSmemBytes <= 232448, "shared memory per CTA");
constexpr int kBThreads = 256;             // warps 0-7: B producers, one column each
constexpr int kAWarp = 8, kMmaWarp = 9;    // warps 10-13: epilogue
constexpr int kThreads = 448;
constexpr uint32_t kTmemCols = 2 * kN;
constexpr uint32_t kMaxPolls = 1u << 22;
constexpr uint32_t kIdesc = umma::idesc_tf32(kM, kN);

// barrier indices
constexpr int FA = 0, EA = FA + kSA, FB = EA + kSA, EB = FB + kSB, AF = EB + kSB, AE = AF + 2, FIN = AE + 2,
              NBAR = FIN + 1;
static_assert(NBAR * 8 <= 192, "barrier area");

struct Smem {
  uint8_t* base;
  uint64_t* bar;
  uint32_t* tmem_slot;
  int* fail;
  __device__ __forceinline__ uint8_t* a(int s) const { return base + s * kAChunkBytes; }
  __device__ __forceinline__ uint8_t* bc(int s) const { return base + kSA * kAChunkBytes + s * 2 * kBBytes; }
  __device__ __forceinline__ uint8_t* braw(int s) const {
    return base + kSA * kAChunkBytes + kSB * 2 * kBBytes + s * kBBytes;
  }
  __device__ __forceinline__ bool failed() const { return *reinterpret_cast<volatile int*>(fail) != 0; }
  __device__ __forceinline__ void set_fail() const { atomicExch(fail, 1); }
};

__device__ __forceinline__ Smem smem_layout(uint8_t* base) {
  Smem s;
  s.base = base;
  uint8_t* tail = base + kSA * kAChunkBytes + kSB * 2 * kBBytes + kR * kBBytes;
  s.bar = reinterpret_cast<uint64_t*>(tail);
  s.tmem_slot = reinterpret_cast<uint32_t*>(tail + 192);
  s.fail = reinterpret_cast<int*>(tail + 224);
  return s;
}

__device__ __forceinline__ bool wait_bar(const Smem& s, int i, uint32_t parity) {
  if (umma::mbar_wait(&s.bar[i], parity, kMaxPolls)) return true;
  s.set_fail();
  return false;
}

// ---- B side: cp.async of FP32 chunks, split in shared memory ----------------
__device__ __forceinline__ void cp16(void* dst, const void* src, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(umma::smem_u32(dst)), "l"(src), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void cp4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(umma::smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// L2 prefetch of `bytes` (a multiple of 16) at a 16-byte aligned global address
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Barrier over the B-producer warps (named barrier 1) that also ORs a
// predicate across them, so that all of them take the same exit decision.
__device__ __forceinline__ bool bar_or_b(bool pred) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.b32 p, %1, 0;\n\t"
      "bar.red.or.pred q, 1, 256, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}\n"
      : "=r"(r)
      : "r"((uint32_t)pred)
      : "memory");
  return r != 0;
}

// A quad (4 floats) of `valid` leading elements from src into dst (16 bytes);
// src is read only where valid, the missing elements are stored as zeros.
__device__ __forceinline__ void copy_quad(void* dst, const float* src, int valid, bool vec) {
  if (valid <= 0) {
    *reinterpret_cast<float4*>(dst) = make_float4(0.f, 0.f, 0.f, 0.f);
  } else if (vec) {
    cp16(dst, src, 4 * min(valid, 4));
  } else {
#pragma unroll
    for (int u = 0; u < 4; u++) {
      float* d = reinterpret_cast<float*>(dst) + u;
      if (u < valid)
        cp4(d, src + u);
      else
        *d = 0.f;
    }
  }
}

// Raw B chunk: 16 rows (k) x 256 floats, quad q of row k at byte k * 1024 + q * 16.
// Copies of P(k, c) = P[(k0 + k) * ld + c] for k0 + k < kv, c < cv; thread t of kBThreads.
__device__ __forceinline__ void issue_b(uint8_t* raw, const float* P, int64_t ld, int cv, int k0, int kv, bool vec,
                                        int t) {
#pragma unroll
  for (int j = 0; j < (kK * kN / 4) / kBThreads; j++) {
    const int i = t + j * kBThreads;
    const int k = i / (kN / 4), q = i % (kN / 4);
    const bool kvld = k0 + k < kv;
    const int valid = kvld ? cv - 4 * q : 0;
    copy_quad(raw + k * (kN * 4) + q * 16, P + (int64_t)(kvld ? k0 + k : 0) * ld + 4 * q, valid, vec);
  }
}

__device__ __forceinline__ void put4(uint8_t* hi_base, uint8_t* lo_base, int row, int k, float v0, float v1, float v2,
                                     float v3) {
  uint4 h, l;
  umma::split_tf32(v0, h.x, l.x);
  umma::split_tf32(v1, h.y, l.y);
  umma::split_tf32(v2, h.z, l.z);
  umma::split_tf32(v3, h.w, l.w);
  const uint32_t off = umma::chunk_offset(row, k);
  *reinterpret_cast<uint4*>(hi_base + off) = h;
  *reinterpret_cast<uint4*>(lo_base + off) = l;
}

// Column t of a raw chunk -> (row = t, k = 0..15) of the split stage.  A
// warp reads 32 consecutive floats per k and writes 8 distinct rows per
// quarter-warp (no bank conflicts).
__device__ __forceinline__ void split_b(const uint8_t* raw, uint8_t* conv, int t) {
  static_assert(kBThreads == kN, "one B-producer thread per column");
  uint8_t* hi = conv;
  uint8_t* lo = conv + kBBytes;
  const float* r = reinterpret_cast<const float*>(raw) + t;
#pragma unroll
  for (int q = 0; q < 4; q++)
    put4(hi, lo, t, 4 * q, r[(4 * q + 0) * kN], r[(4 * q + 1) * kN], r[(4 * q + 2) * kN], r[(4 * q + 3) * kN]);
}

// ---- the two phases' work items -------------------------------------------
struct BSeg {
  const float* p;  // first row of the segment's B rows
  int64_t ld;
  int K;
};

// Phase 2: tiles of 128 consecutive rows; B segments = slot rows of the slot
// workspace (far) or rows of X (near); output rows of Y.
struct Ph2 {
  const TcTile* tiles;
  const TcSeg* segs;
  const float* zmix;
  int64_t ldz;
  const float* X;
  int64_t ldx;
  float* Y;
  int64_t ldy;
  __device__ __forceinline__ int nchunk(int64_t w) const { return tiles[w].nchunk; }
  __device__ __forceinline__ int64_t a_chunk0(int64_t w) const { return tiles[w].a_chunk0; }
  __device__ __forceinline__ int nseg(int64_t w) const { return tiles[w].nseg; }
  __device__ __forceinline__ BSeg seg(int64_t w, int j) const {
    const TcSeg sg = segs[tiles[w].seg0 + j];
    if (sg.near) return BSeg{X + sg.b_row * ldx, ldx, sg.K};
    return BSeg{zmix + sg.b_row * ldz, ldz, sg.K};
  }
  __device__ __forceinline__ float* row_ptr(int64_t w, int row) const {
    const TcTile& t = tiles[w];
    return row < t.rows ? Y + (t.row0 + row) * ldy : nullptr;
  }
};

// Phase 1: items (cluster, 128-slot tile, <= 2048-row chunk); one B segment
// (the chunk's rows of X); output slot rows scattered through the slot map,
// or partial rows when the cluster is split into several row chunks.
struct Ph1 {
  const P1Item* items;
  const float* X;
  int64_t ldx;
  const int64_t* slotmap;
  float* zmix;
  float* part;
  int64_t ldz;
  __device__ __forceinline__ int nchunk(int64_t w) const { return items[w].nchunk; }
  __device__ __forceinline__ int64_t a_chunk0(int64_t w) const { return items[w].a_chunk0; }
  __device__ __forceinline__ int nseg(int64_t) const { return 1; }
  __device__ __forceinline__ BSeg seg(int64_t w, int) const {
    const P1Item& it = items[w];
    return BSeg{X + it.x_row * ldx, ldx, it.nr};
  }
  __device__ __forceinline__ float* row_ptr(int64_t w, int row) const {
    const P1Item& it = items[w];
    if (row >= it.nq) return nullptr;
    return it.out_row < 0 ? zmix + slotmap[it.map_off + row] * ldz : part + (it.out_row + row) * ldz;
  }
};

// Walks this CTA's B chunks in order (tiles blockIdx.x, + gridDim.x, ...; in
// each, its segments' K-chunks), skipping tiles without chunks.
template <class Ph>
struct BCursor {
  const Ph* ph;
  int64_t ntiles;
  int nct, ncols;
  int64_t id, w;
  int j, nseg, k0, nv;
  BSeg sg;
  const float* base;
  bool vec, valid;

  __device__ __forceinline__ bool find_seg() {
    for (; j < nseg; j++) {
      sg = ph->seg(w, j);
      if (sg.K > 0) {
        const int n0 = (int)(id % nct) * kN;
        base = sg.p + n0;
        vec = (sg.ld % 4 == 0) && ((reinterpret_cast<uintptr_t>(base) & 15) == 0);
        return true;
      }
    }
    return false;
  }
  __device__ __forceinline__ void enter() {
    valid = false;
    for (; id < ntiles; id += gridDim.x) {
      w = id / nct;
      nv = min(kN, ncols - (int)(id % nct) * kN);
      nseg = ph->nseg(w);
      j = 0;
      k0 = 0;
      if (find_seg()) {
        valid = true;
        return;
      }
    }
  }
  __device__ __forceinline__ void start() {
    id = blockIdx.x;
    enter();
  }
  __device__ __forceinline__ void advance() {
    k0 += kK;
    if (k0 < sg.K) return;
    k0 = 0;
    j++;
    if (find_seg()) return;
    id += gridDim.x;
    enter();
  }
};

// ---- roles -----------------------------------------------------------------
template <class Ph>
__device__ __forceinline__ void b_producer(const Smem& s, const Ph& ph, int64_t ntiles, int nct, int ncols) {
  const int t = threadIdx.x;
  int64_t total = 0;
  for (int64_t id = blockIdx.x; id < ntiles; id += gridDim.x) total += ph.nchunk(id / nct);
  BCursor<Ph> cur;
  cur.ph = &ph;
  cur.ntiles = ntiles;
  cur.nct = nct;
  cur.ncols = ncols;
  cur.start();
  // a second cursor kBPrefetch chunks ahead of the copies: its 16 rows are
  // prefetched into L2 (one row per thread t < 16) when 16-byte aligned
  BCursor<Ph> pf = cur;
  if (kBPrefetch == 0) pf.valid = false;
  for (int i = 0; i < kBPrefetch && pf.valid; i++) pf.advance();
#pragma unroll
  for (int i = 0; i < kR - 1; i++) {
    if (cur.valid) {
      issue_b(s.braw(i), cur.base, cur.sg.ld, cur.nv, cur.k0, cur.sg.K, cur.vec, t);
      cur.advance();
    }
    cp_commit();
  }
  for (int64_t g = 0; g < total; g++) {
    cp_wait<kR - 2>();  // this thread's copies of chunk g have landed
    if (bar_or_b(s.failed())) break;  // everyone's copies of g have landed; raw stage of g-1 is free
    if (cur.valid) {
      issue_b(s.braw((int)((g + kR - 1) % kR)), cur.base, cur.sg.ld, cur.nv, cur.k0, cur.sg.K, cur.vec, t);
      cur.advance();
    }
    cp_commit();
    if (pf.valid) {
      if (t < kK && pf.vec && (pf.nv & 3) == 0 && pf.k0 + t < pf.sg.K)
        prefetch_l2(pf.base + (int64_t)(pf.k0 + t) * pf.sg.ld, (uint32_t)pf.nv * 4);
      pf.advance();
    }
    const int sb = (int)(g % kSB);
    if (g >= kSB) wait_bar(s, EB + sb, (uint32_t)((g / kSB) - 1) & 1);
    split_b(s.braw((int)(g % kR)), s.bc(sb), t);
    umma::fence_proxy_async();
    umma::mbar_arrive(&s.bar[FB + sb]);
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
}

template <class Ph>
__device__ __forceinline__ void a_producer(const Smem& s, const Ph& ph, int64_t ntiles, int nct,
                                           const uint8_t* astream) {
  int64_t g = 0;
  for (int64_t id = blockIdx.x; id < ntiles; id += gridDim.x) {
    const int64_t w = id / nct;
    const int nch = ph.nchunk(w);
    const int64_t a0 = ph.a_chunk0(w);
    for (int c = 0; c < nch; c++, g++) {
      if (s.failed()) return;
      const int sa = (int)(g % kSA);
      if (g >= kSA && !wait_bar(s, EA + sa, (uint32_t)((g / kSA) - 1) & 1)) return;
      umma::mbar_arrive_expect_tx(&s.bar[FA + sa], kAChunkBytes);
      umma::bulk_g2s(s.a(sa), astream + (a0 + c) * (int64_t)kAChunkBytes, kAChunkBytes, &s.bar[FA + sa]);
      if (kAPrefetch > 0 && c + kAPrefetch < nch) prefetch_l2(astream + (a0 + c + kAPrefetch) * (int64_t)kAChunkBytes, kAChunkBytes);
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
  for (int64_t id = blockIdx.x; ok && id < ntiles; id += gridDim.x, tl++) {
    const int nch = ph.nchunk(id / nct);
    const int b = tl & 1;
    if (tl >= 2 && !wait_bar(s, AE + b, (uint32_t)((tl >> 1) - 1) & 1)) break;
    umma::fence_after_sync();
    const uint32_t acc = tmem + (uint32_t)(b * kN);
    for (int c = 0; c < nch; c++, g++) {
      const int sa = (int)(g % kSA), sb = (int)(g % kSB);
      if (s.failed() || !wait_bar(s, FA + sa, (uint32_t)(g / kSA) & 1) ||
          !wait_bar(s, FB + sb, (uint32_t)(g / kSB) & 1)) {
        ok = false;
        break;
      }
      umma::fence_after_sync();
      issue_mma(s.a(sa), s.bc(sb), acc, c == 0);
      umma::commit(&s.bar[EA + sa]);
      umma::commit(&s.bar[EB + sb]);
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

template <class Ph>
__device__ __forceinline__ void epilogue(const Smem& s, const Ph& ph, int64_t ntiles, int nct, int ncols,
                                         uint32_t tmem) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int quarter = warp & 3;  // TMEM lanes 32*quarter.. are this warp's
  const int row = 32 * quarter + lane;
  int tl = 0;
  for (int64_t id = blockIdx.x; id < ntiles; id += gridDim.x, tl++) {
    const int b = tl & 1;
    if (!wait_bar(s, AF + b, (uint32_t)(tl >> 1) & 1)) break;
    umma::fence_after_sync();
    if (s.failed()) break;
    const int64_t w = id / nct;
    const int n0 = (int)(id % nct) * kN;
    const int nv = min(kN, ncols - n0);
    const bool zero = ph.nchunk(w) == 0;
    float* dst = ph.row_ptr(w, row);
    if (dst) dst += n0;
    const bool vec4 = dst && ((reinterpret_cast<uintptr_t>(dst) & 15) == 0);
#pragma unroll 1
    for (int j = 0; j < kN / 32; j++) {
      float v[32];
      if (zero) {
#pragma unroll
        for (int i = 0; i < 32; i++) v[i] = 0.f;
      } else {
        umma::tmem_ld32(tmem + (uint32_t)(b * kN) + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(32 * j), v);
      }
      if (dst) {
        const int c0 = 32 * j;
        if (vec4 && c0 + 32 <= nv) {
#pragma unroll
          for (int i = 0; i < 32; i += 4)
            *reinterpret_cast<float4*>(dst + c0 + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
        } else {
#pragma unroll
          for (int i = 0; i < 32; i++)
            if (c0 + i < nv) dst[c0 + i] = v[i];
        }
      }
    }
    umma::fence_before_sync();
    umma::mbar_arrive(&s.bar[AE + b]);
  }
}

template <class Ph>
__global__ void __launch_bounds__(kThreads, 1)
    k_tc_apply(const Ph ph, int64_t nwork, int nct, int ncols, const uint8_t* __restrict__ astream,
               int* __restrict__ err) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  const Smem s = smem_layout(smem_raw);
  const int warp = threadIdx.x >> 5;
  const int64_t ntiles = nwork * nct;
  if (threadIdx.x == 0) {
    for (int i = FA; i < EA; i++) umma::mbar_init(&s.bar[i], 1);
    for (int i = EA; i < FB; i++) umma::mbar_init(&s.bar[i], 1);
    for (int i = FB; i < EB; i++) umma::mbar_init(&s.bar[i], kBThreads);
    for (int i = EB; i < AF; i++) umma::mbar_init(&s.bar[i], 1);
    for (int i = AF; i < AE; i++) umma::mbar_init(&s.bar[i], 1);
    for (int i = AE; i < FIN; i++) umma::mbar_init(&s.bar[i], 128);
    umma::mbar_init(&s.bar[FIN], 1);
    *s.fail = 0;
    umma::fence_mbar_init();
  }
  if (warp == kMmaWarp) umma::tmem_alloc(s.tmem_slot, kTmemCols);
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tmem = *s.tmem_slot;
  if (warp < kBThreads / 32) {
    b_producer(s, ph, ntiles, nct, ncols);
  } else if (warp == kAWarp) {
    if ((threadIdx.x & 31) == 0) a_producer(s, ph, ntiles, nct, astream);
  } else if (warp == kMmaWarp) {
    if ((threadIdx.x & 31) == 0) mma_issuer(s, ph, ntiles, nct, tmem);
    __syncwarp();
  } else {
    epilogue(s, ph, ntiles, nct, ncols, tmem);
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

__global__ void k_phase1_reduce_tc(const P1Reduce* __restrict__ items, const float* __restrict__ part,
                                   const int64_t* __restrict__ slotmap, float* __restrict__ zmix, int64_t ldz,
                                   int ncols) {
  const P1Reduce it = items[blockIdx.x];
  const int64_t total = (int64_t)it.nq * ncols;
  for (int64_t e = threadIdx.x + (int64_t)blockIdx.y * blockDim.x; e < total; e += (int64_t)blockDim.x * gridDim.y) {
    const int q = (int)(e / ncols), n = (int)(e % ncols);
    float acc = 0.f;
    for (int c = 0; c < it.nch; c++) acc += part[(it.part_row + (int64_t)c * it.nq + q) * ldz + n];
    zmix[slotmap[it.map_off + q] * ldz + n] = acc;
  }
}

}  // namespace

// Tensor-core apply for an FP32 operator (cluster order).
fkf_status hmat_apply_clustered_tc(fkf_hmat* h, const float* X, int64_t ldx, float* Y, int64_t ldy, int64_t ncols) {
  fkf_ctx* ctx = h->ctx;
  const int64_t P = h->panel;
  const size_t zbytes = (size_t)std::max<int64_t>(h->ktot, 1) * P * sizeof(float);
  if (h->zmix.bytes < zbytes) FKF_TRY(dev_alloc(ctx, h->zmix, zbytes));
  const size_t pbytes = (size_t)std::max<int64_t>(h->tc_part_rows, 1) * P * sizeof(float);
  if (h->part.bytes < pbytes) FKF_TRY(dev_alloc(ctx, h->part, pbytes));
  if (h->tc_err.bytes < 64) {
    FKF_TRY(dev_alloc(ctx, h->tc_err, 64));
    FKF_CUDA(ctx, cudaMemsetAsync(h->tc_err.p, 0, 64, ctx->stream));
  }
  int sms = 0;
  FKF_CUDA(ctx, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
  FKF_CUDA(ctx, cudaFuncSetAttribute(k_tc_apply<Ph1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes));
  FKF_CUDA(ctx, cudaFuncSetAttribute(k_tc_apply<Ph2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes));
  const uint8_t* astream = h->tca.as<uint8_t>();
  for (int64_t c0 = 0; c0 < ncols; c0 += P) {
    const int nc = (int)std::min<int64_t>(P, ncols - c0);
    const int nct = (int)cdiv(nc, kN);
    if (h->n_tcp1 > 0) {
      const Ph1 ph{h->tcp1.as<P1Item>(), X + c0, ldx, h->slotmap.as<int64_t>(), h->zmix.as<float>(),
                   h->part.as<float>(), P};
      const int grid = (int)std::min<int64_t>(sms, h->n_tcp1 * nct);
      k_tc_apply<Ph1><<<grid, kThreads, kSmemBytes, ctx->stream>>>(ph, h->n_tcp1, nct, nc, astream,
                                                                   h->tc_err.as<int>());
      FKF_LAUNCHED(ctx);
    }
    if (h->n_tcred > 0) {
      k_phase1_reduce_tc<<<dim3((unsigned)h->n_tcred, 4), 256, 0, ctx->stream>>>(
          h->tcred.as<P1Reduce>(), h->part.as<float>(), h->slotmap.as<int64_t>(), h->zmix.as<float>(), P, nc);
      FKF_LAUNCHED(ctx);
    }
    const Ph2 ph{h->tctile.as<TcTile>(), h->tcseg.as<TcSeg>(), h->zmix.as<float>(), P, X + c0, ldx, Y + c0, ldy};
    const int grid = (int)std::min<int64_t>(sms, h->n_tctile * nct);
    k_tc_apply<Ph2><<<grid, kThreads, kSmemBytes, ctx->stream>>>(ph, h->n_tctile, nct, nc, astream,
                                                                 h->tc_err.as<int>());
    FKF_LAUNCHED(ctx);
  }
  return FKF_OK;
}

fkf_status hmat_build_tc_streams(fkf_hmat* h, std::vector<P1Item>& items, std::vector<TcTile>& tiles) {
  fkf_ctx* ctx = h->ctx;
  std::vector<TcAChunk> ch;
  // phase-1 items are dealt round-robin to persistent CTAs: longest first
  std::stable_sort(items.begin(), items.end(), [](const P1Item& a, const P1Item& b) { return a.nr > b.nr; });
  for (P1Item& it : items) {
    it.a_chunk0 = (int64_t)ch.size();
    it.nchunk = (int)cdiv(it.nr, kK);
    for (int c = 0; c < it.nchunk; c++) {
      TcAChunk a{};
      a.src_off = it.fac_off + (int64_t)(it.r0 + c * kK) * it.K + it.q0;
      a.si = 1;
      a.sk = it.K;
      a.row_lo = 0;
      a.row_hi = it.nq;
      a.kv = std::min(kK, it.nr - c * kK);
      a.near = 0;
      ch.push_back(a);
    }
  }
  for (TcTile& t : tiles) {
    t.a_chunk0 = (int64_t)ch.size();
    int nch = 0;
    for (int j = 0; j < t.nseg; j++) {
      const TcSeg& sg = h->tcseg_host[t.seg0 + j];
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
  if (!tiles.empty()) FKF_TRY(dev_upload(ctx, h->tctile, tiles.data(), tiles.size() * sizeof(TcTile)));
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
  return FKF_OK;
}

// Reads (and clears) the tensor-core wait-expiry flag; synchronises.
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
