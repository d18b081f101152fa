// Symmetric eigensolver (FP64) of the library's own, for the data-space
// generalized eigenproblem (Eq. ghep written in data space, Sec. 2.2.2) and the
// merge eigenproblem of Alg. lowrankaddition (step 4, Sec. 2.4):
//
//  1. Householder reduction to tridiagonal form T = Q_H^T A Q_H, blocked by
//     panels of kNB columns: the column steps of a panel run in one cooperative
//     kernel (grid-wide barriers between the column's phases: the column's
//     update with the panel's earlier reflectors, the reflector, the
//     symmetric product A v, the correction w), the trailing update
//     A -= V W^T + W V^T after the panel in one symmetric FP64 tile GEMM;
//  2. divide and conquer on T (Cuppen's splitting T = diag(T1, T2) + |b| u u^T):
//     leaves of at most kLeaf rows by implicit QL (one warp per leaf); each
//     merge sorts the children's eigenvalues, deflates (small components of
//     z, and pairs of close eigenvalues rotated until one component vanishes),
//     solves the secular equation 1/rho + sum z_i^2 / (d_i - lambda) = 0 for
//     every remaining root (one thread per root: a fit of the two nearest
//     poles by rational functions, safeguarded by bisection, with lambda kept
//     as an offset from its nearest pole), recomputes z from the roots
//     (Loewner's formula, which makes the eigenvectors orthogonal to working
//     precision), forms the eigenvectors of the rank-one update and applies
//     them to the children's eigenvectors with one FP64 GEMM;
//  3. back-transformation X = Q_H Z of the wanted eigenvectors, one block
//     reflector (I - V T V^T, compact WY form) per panel, by GEMMs.
//
// Every spin (the grid barrier) is bounded and sets an error flag; iteration
// counts are bounded.  Results: eigenvalues ascending; eigenvector j in row j.
#include <cooperative_groups.h>

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstring>

#include "dense.h"

namespace {

constexpr int kNB = 32;                  // panel width of the reduction and the back-transformation
constexpr int kLeaf = 32;                // largest leaf of the divide and conquer (one warp)
constexpr int kBT = 128;                 // reflectors per block of the back-transformation
constexpr size_t kPrepSmem = 216 * 1024;  // shared memory of the merge preparation (s <= 3949)                 // reflectors per block of the back-transformation
constexpr int kTrdThreads = 512;
constexpr int kTrdSmemV = 6144;            // reflector entries staged in shared memory (48 KB)
constexpr uint32_t kBarPolls = 1u << 24;  // bounded grid-barrier spin
constexpr double kEps = DBL_EPSILON;

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ double block_sum(double v, double* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  if (warp == 0) {
    double x = lane < nw ? sh[lane] : 0.0;
    x = warp_sum(x);
    if (lane == 0) sh[32] = x;
  }
  __syncthreads();
  const double r = sh[32];
  __syncthreads();
  return r;
}

// Grid-wide barrier of a cooperative launch (all CTAs co-resident): an
// arrival counter (monotonic: count = gen * gridDim.x after generation gen) and
// a generation flag that the last CTA to arrive publishes; the others spin on
// the flag.  The spin is bounded and records a failure in err.
__device__ void grid_barrier(unsigned* count, unsigned* flag, unsigned& gen, int* err) {
  __syncthreads();
  if (threadIdx.x == 0) {
    gen++;
    __threadfence();
    const unsigned prev = atomicAdd(count, 1u);
    if (prev == gen * gridDim.x - 1) {
      atomicExch(flag, gen);
    } else {
      uint32_t polls = 0;
      while (*reinterpret_cast<volatile unsigned*>(flag) < gen) {
        if (++polls > kBarPolls) {
          atomicExch(err, 1);
          break;
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
}

// Sum over the grid's CTAs of a per-CTA partial (part[0..G)), by the whole
// block (one load per thread, then a block reduction); every CTA obtains the
// same value (fixed order).
__device__ double grid_partials_sum(const double* part, int G, double* sh) {
  double v = 0;
  for (int q = threadIdx.x; q < G; q += blockDim.x) v += part[q];
  return block_sum(v, sh);
}

struct TrdArgs {
  double* A;     // n x n, row-major, symmetric (both triangles current in the trailing block)
  int64_t n;
  int64_t j0;    // first column of the panel
  int nbp;       // columns in the panel
  double* VW;    // n x 2kNB: [V | W] of the panel
  double* WV;    // n x 2kNB: [W | V]
  double* d;     // diagonal of T
  double* e;     // off-diagonal of T
  double* tau;   // reflector scalars
  double* col;   // n: current column
  double* vg;    // n: reflector
  double* pg;    // n: A v
  double* part;  // 3 * gridDim.x + gridDim.x * 2 kNB partial sums (one region per phase)
  unsigned* bar; // [0] arrival count, [1] generation flag
  int* err;
};

// One panel of the Householder reduction (lower form), by every SM (the
// column's symmetric product is FP64-FMA bound).  Column j of the panel
// (c = j - j0), with x = a[1:] the part below the diagonal:
//   a = A[j:, j] - V[j:, :c] W[j, :c]^T - W[j:, :c] V[j, :c]^T   (current column)
//   d_j = a_0; reflector H = I - tau v v^T with H x = beta e_1,
//   v = (x - beta e_1) / (alpha - beta), alpha = x_0
//   p = A[j+1:, j+1:] v - V (W^T v) - W (V^T v)                    (current matrix times v)
//   w = tau p - tau^2/2 (p^T v) v;  V[:, c] = v, W[:, c] = w
// Two grid barriers per column: the product starts from x as soon as the
// column is complete, A v = (A x - beta A e_1) / (alpha - beta), and W^T v,
// V^T v follow from W^T x, V^T x in the same way, so the reflector's scalars
// (from the column's norm) are formed after the same barrier.  The correction
// w of column c is formed at the start of column c + 1 by the CTA that owns
// each row there (every CTA forms the entry w_{j+1} that all of them need), and
// after the loop for the last column.  Partial sums go to one region per phase,
// so a region is rewritten only after every CTA has passed a later barrier.
// The reflector (below its leading 1) is stored in A[j+2:, j].
__global__ void __launch_bounds__(kTrdThreads) k_trd_panel(TrdArgs a) {
  __shared__ double sh[33];
  __shared__ double wv[2 * kNB];
  __shared__ double bc[4];
  extern __shared__ double vs[];  // x[0..n-j-1) when it fits
  const int64_t n = a.n;
  const int G = gridDim.x, b = blockIdx.x, t = threadIdx.x;
  const int lane = t & 31, warp = t >> 5, nw = blockDim.x >> 5;
  constexpr int L = 2 * kNB;
  double* partA = a.part;
  double* partC = a.part + G;
  double* partB = a.part + 2 * G;  // G x 2 kNB
  unsigned gen = 0;
  double tau_prev = 0, k2_prev = 0;  // column c - 1: w = tau p - k2 v
  int64_t s0 = 0, s1 = 0;            // rows [j+1, n) of this CTA (the product phase)
  for (int c = 0; c < a.nbp; c++) {
    const int64_t j = a.j0 + c;
    if (j >= n) break;
    // ---- phase A: w of column c - 1 and the current column on this CTA's rows
    // of [j, n); partial sums of |x[1:]|^2, W^T x and V^T x
    {
      const int64_t rows = n - j, R = (rows + G - 1) / G;
      const int64_t r0 = j + b * R, r1 = min(n, r0 + R);
      if (c > 0) {
        for (int64_t i = r0 + t; i < r1; i += blockDim.x) {
          const double w = tau_prev * a.pg[i] - k2_prev * a.vg[i];
          a.VW[i * L + kNB + c - 1] = w;
          a.WV[i * L + c - 1] = w;
        }
      }
      const double* Vj = a.VW + j * L;
      const double wjc = c > 0 ? tau_prev * a.pg[j] - k2_prev * a.vg[j] : 0.0;
      __syncthreads();
      // a warp per row; lane q < c forms the correction terms of column q
      const double vjq = lane < c ? (lane == c - 1 ? wjc : Vj[kNB + lane]) : 0.0;  // W[j][q]
      const double vjv = lane < c ? Vj[lane] : 0.0;                                // V[j][q]
      double ss = 0;
      double px = 0;  // lane q: W[:, q]^T x (q < c) or V[:, q - c]^T x (c <= q < 2c), this warp's rows
      double px2 = 0;  // the same for lane q + 32 (2c may reach 64)
      for (int64_t i = r0 + warp; i < r1; i += nw) {
        const double* Vi = a.VW + i * L;
        double corr = lane < c ? Vi[lane] * vjq + Vi[kNB + lane] * vjv : 0.0;
        corr = warp_sum(corr);
        const double v = a.A[j * n + i] - corr;  // A[i][j] = A[j][i]
        if (lane == 0) {
          a.col[i] = v;
          if (i >= j + 2) ss += v * v;
        }
        if (i >= j + 1) {
          // W[i][q] for q < c sits at Vi[kNB + q], V[i][q] at Vi[q]
          if (lane < 2 * c) px += (lane < c ? Vi[kNB + lane] : Vi[lane - c]) * v;
          if (lane + 32 < 2 * c) px2 += (lane + 32 < c ? Vi[kNB + lane + 32] : Vi[lane + 32 - c]) * v;
        }
      }
      ss = block_sum(ss, sh);
      if (t == 0) partA[b] = ss;
      // combine the warps' W^T x / V^T x partials in shared memory
      __shared__ double pxw[kTrdThreads / 32][2 * kNB];
      if (lane < 2 * c) pxw[warp][lane] = px;
      if (lane + 32 < 2 * c) pxw[warp][lane + 32] = px2;
      __syncthreads();
      if (t < 2 * c) {
        double acc = 0;
        for (int w2 = 0; w2 < nw; w2++) acc += pxw[w2][t];
        partB[(int64_t)b * L + t] = acc;
      }
    }
    grid_barrier(a.bar, a.bar + 1, gen, a.err);
    // ---- phase B: the reflector's scalars (every CTA, same partials, same order)
    const double s2 = grid_partials_sum(partA, G, sh);
    if (t == 0) {
      double beta = 0, tau = 0, scale = 0;
      if (j + 1 < n) {
        const double alpha = a.col[j + 1];
        if (s2 == 0.0) {
          beta = alpha;
        } else {
          beta = -copysign(sqrt(alpha * alpha + s2), alpha);
          tau = (beta - alpha) / beta;
          scale = 1.0 / (alpha - beta);
        }
      }
      bc[0] = tau;
      bc[1] = scale;
      bc[3] = beta;
      if (b == 0) {
        a.d[j] = a.col[j];
        if (j + 1 < n) {
          a.e[j] = beta;
          a.tau[j] = tau;
        }
      }
    }
    __syncthreads();
    if (j + 1 >= n) break;  // the last diagonal entry has no reflector (uniform over the grid)
    const double tau = bc[0], scale = bc[1], beta = bc[3];
    // W^T v = scale (W^T x - beta W[j+1, :]), V^T v likewise
    const double* Vn = a.VW + (j + 1) * L;
    for (int qq = warp; qq < 2 * c; qq += nw) {
      double acc = 0;
      for (int q = lane; q < G; q += 32) acc += partB[(int64_t)q * L + qq];
      acc = warp_sum(acc);
      if (lane == 0) {
        const double e1 = qq < c ? Vn[kNB + qq] : Vn[qq - c];
        wv[qq] = scale * (acc - beta * e1);
      }
    }
    const int64_t rows1 = n - j - 1, R1 = (rows1 + G - 1) / G;
    s0 = j + 1 + b * R1;
    s1 = min(n, s0 + R1);
    for (int64_t i = s0 + t; i < s1; i += blockDim.x) {
      const double v = (i == j + 1) ? 1.0 : a.col[i] * scale;
      a.vg[i] = v;
      a.VW[i * L + c] = v;
      a.WV[i * L + kNB + c] = v;
      if (i >= j + 2) a.A[i * n + j] = v;
    }
    // x = col[j+1..n) staged in shared memory when it fits
    const int64_t nv = n - j - 1;
    const bool vsm = nv <= kTrdSmemV;
    if (vsm)
      for (int64_t k = t; k < nv; k += blockDim.x) vs[k] = a.col[j + 1 + k];
    __syncthreads();
    // ---- phase C: p = scale (A x - beta A e_1) - V (W^T v) - W (V^T v), a warp per row
    double pv = 0;
    for (int64_t i = s0 + warp; i < s1; i += nw) {
      const double* Ai = a.A + i * n + j + 1;
      const double* xv = vsm ? vs : a.col + j + 1;
      double acc0 = 0, acc1 = 0, acc2 = 0, acc3 = 0;
      int64_t k = lane;
      for (; k + 96 < nv; k += 128) {
        acc0 += Ai[k] * xv[k];
        acc1 += Ai[k + 32] * xv[k + 32];
        acc2 += Ai[k + 64] * xv[k + 64];
        acc3 += Ai[k + 96] * xv[k + 96];
      }
      for (; k < nv; k += 32) acc0 += Ai[k] * xv[k];
      const double* Vi = a.VW + i * L;
      const double corr = lane < c ? Vi[lane] * wv[lane] + Vi[kNB + lane] * wv[c + lane] : 0.0;
      const double ax = warp_sum((acc0 + acc1) + (acc2 + acc3));
      const double cs = warp_sum(corr);
      if (lane == 0) {
        const double pi = scale * (ax - beta * Ai[0]) - cs;
        a.pg[i] = pi;
        pv += pi * ((i == j + 1) ? 1.0 : a.col[i] * scale);
      }
    }
    pv = block_sum(pv, sh);
    if (t == 0) partC[b] = pv;
    grid_barrier(a.bar, a.bar + 1, gen, a.err);
    // w = tau p - tau^2/2 (p^T v) v, formed at the start of the next column (or below)
    const double ptv = grid_partials_sum(partC, G, sh);
    tau_prev = tau;
    k2_prev = 0.5 * tau * tau * ptv;
  }
  // the panel's last correction column, on this CTA's rows of [j_last + 1, n)
  const int64_t jl = a.j0 + a.nbp - 1;
  if (jl + 1 < n) {
    for (int64_t i = s0 + t; i < s1; i += blockDim.x) {
      const double w = tau_prev * a.pg[i] - k2_prev * a.vg[i];
      a.VW[i * L + kNB + a.nbp - 1] = w;
      a.WV[i * L + a.nbp - 1] = w;
    }
  }
}

// d[p - 1] -= |e[p - 1]| and d[p] -= |e[p - 1]| at every split point p of the
// divide and conquer tree (Cuppen's splitting), in order.
__global__ void k_dc_split_d(int ns, const int* __restrict__ splits, double* __restrict__ d,
                             const double* __restrict__ e) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  for (int q = 0; q < ns; q++) {
    const int p = splits[q];
    const double bb = fabs(e[p - 1]);
    d[p - 1] -= bb;
    d[p] -= bb;
  }
}

// Leaves: implicit QL with a Wilkinson-type shift on a tridiagonal of s <=
// kLeaf rows, one warp per leaf.  Lane 0 runs the scalar recurrence of a sweep
// and records its rotations; every lane applies them to its row of Z.  The
// eigenvalues (ascending) go to D[off..], the eigenvectors to the diagonal
// block of Q (column q = eigenvector q).
__global__ void __launch_bounds__(32) k_dc_leaf(const int* __restrict__ loff, const int* __restrict__ lsize,
                                                 const double* __restrict__ d, const double* __restrict__ e,
                                                 double* __restrict__ D, double* __restrict__ Q, int64_t ldq,
                                                 int* __restrict__ err) {
  __shared__ double Z[kLeaf][kLeaf + 1];
  __shared__ double dd[kLeaf], ee[kLeaf], cs[2][kLeaf];
  __shared__ int lo_sh, perm[kLeaf];
  const int off = loff[blockIdx.x], s = lsize[blockIdx.x], lane = threadIdx.x;
  if (lane < s)
    for (int q = 0; q < s; q++) Z[lane][q] = (lane == q) ? 1.0 : 0.0;
  if (lane < s) {
    dd[lane] = d[off + lane];
    ee[lane] = lane < s - 1 ? e[off + lane] : 0.0;
  }
  __syncwarp();
  for (int l = 0; l < s; l++) {
    for (int iter = 0;; iter++) {
      int m = l;
      for (; m < s - 1; m++) {
        const double dm = fabs(dd[m]) + fabs(dd[m + 1]);
        if (fabs(ee[m]) <= kEps * dm) break;
      }
      if (m == l) break;
      if (iter >= 60) {
        if (lane == 0) atomicExch(err, 2);
        break;
      }
      if (lane == 0) {
        double g = (dd[l + 1] - dd[l]) / (2.0 * ee[l]);
        double r = hypot(g, 1.0);
        g = dd[m] - dd[l] + ee[l] / (g + copysign(r, g));
        double sn = 1.0, c = 1.0, p = 0.0;
        int i = m - 1;
        bool early = false;
        for (; i >= l; i--) {
          const double f = sn * ee[i], bb = c * ee[i];
          r = hypot(f, g);
          ee[i + 1] = r;
          if (r == 0.0) {
            dd[i + 1] -= p;
            ee[m] = 0.0;
            early = true;
            break;
          }
          sn = f / r;
          c = g / r;
          g = dd[i + 1] - p;
          r = (dd[i] - g) * sn + 2.0 * c * bb;
          p = sn * r;
          dd[i + 1] = g + p;
          g = c * r - bb;
          cs[0][i] = c;
          cs[1][i] = sn;
        }
        lo_sh = early ? i + 1 : l;
        if (!early) {
          dd[l] -= p;
          ee[l] = g;
          ee[m] = 0.0;
        }
      }
      __syncwarp();
      const int lo = lo_sh;
      if (lane < s) {
        for (int i = m - 1; i >= lo; i--) {
          const double c = cs[0][i], sn = cs[1][i];
          const double zi = Z[lane][i], zi1 = Z[lane][i + 1];
          Z[lane][i + 1] = sn * zi + c * zi1;
          Z[lane][i] = c * zi - sn * zi1;
        }
      }
      __syncwarp();
    }
  }
  if (lane == 0) {
    for (int q = 0; q < s; q++) perm[q] = q;
    for (int q = 1; q < s; q++) {  // insertion sort by eigenvalue
      const int x = perm[q];
      int p = q - 1;
      while (p >= 0 && dd[perm[p]] > dd[x]) {
        perm[p + 1] = perm[p];
        p--;
      }
      perm[p + 1] = x;
    }
  }
  __syncwarp();
  if (lane < s) {
    D[off + lane] = dd[perm[lane]];
    for (int q = 0; q < s; q++) Q[(int64_t)(off + lane) * ldq + off + q] = Z[lane][perm[q]];
  }
}

// Scratch of one merge (every array sized for the largest node, n).
struct DcMerge {
  int* perm;    // sorted position -> column of the node's block
  double* Dp;   // eigenvalues in sorted order (rotated ones updated)
  double* zp;   // z in sorted order
  int* gi;      // Givens rotations (sorted positions gi < gj)
  int* gj;
  double* gc;
  double* gs;
  int* nd;      // non-deflated positions, by ascending Dp
  int* df;      // deflated positions, by ascending Dp
  double* dk;   // Dp[nd]
  double* zk;   // zp[nd]
  int* orig;    // secular roots: lambda_j = dk[orig_j] + taus_j
  double* taus;
  double* lam;
  double* zh;   // Loewner z
  double* cnrm; // eigenvector column norms
  int* ctl;     // [0] K, [1] number of rotations, [2] deflated count, [3] error
  int* src;     // final position -> source (>= 0: non-deflated root, < 0: -1 - deflated index)
  double* rho;  // [0]
  int* iscr;    // 4 n ints of preparation scratch (when shared memory is too small)
  double* dscr; // n words of preparation scratch
};

// Order-preserving integer key of a double (compares of keys are integer
// compares; the serial scans below avoid long FP64 dependency chains).
__device__ __forceinline__ long long dkey(double x) {
  const long long b = __double_as_longlong(x);
  return b < 0 ? (b ^ 0x7fffffffffffffffLL) : b;
}

// Exclusive prefix sums of flags[0..s) into pos (block-wide; thread t takes a
// contiguous chunk); returns the total.
__device__ int block_scan_flags(const int* flags, int s, int* pos, int* cnt) {
  const int T = blockDim.x, t = threadIdx.x;
  const int chunk = (s + T - 1) / T, lo = min(s, t * chunk), hi = min(s, lo + chunk);
  int c = 0;
  for (int p = lo; p < hi; p++) c += flags[p];
  cnt[t] = c;
  __syncthreads();
  if (t == 0) {
    int acc = 0;
    for (int u = 0; u < T; u++) {
      const int x = cnt[u];
      cnt[u] = acc;
      acc += x;
    }
    cnt[T] = acc;
  }
  __syncthreads();
  int o = cnt[t];
  for (int p = lo; p < hi; p++) {
    pos[p] = o;
    o += flags[p];
  }
  const int total = cnt[T];
  __syncthreads();
  return total;
}

constexpr int kPrepThreads = 512;

// Merge preparation (one CTA; copies in shared memory when they fit): z from
// the children's eigenvectors, the children's sorted eigenvalue lists merged
// (on integer keys), deflation, the remaining poles and z compacted.
// Deflation (scan in ascending order of d): a pole with rho |z_j| <= tol is
// deflated; otherwise, with i the previous surviving pole, the rotation in the
// (i, j) plane that zeroes z_i is taken when |(d_j - d_i) c s| <= tol, which
// deflates i.  The tests of consecutive survivors are formed in parallel from
// the merged values; the serial walk recomputes a test only after a rotation
// changed its left pole.  Dynamic shared memory: kPrepWords(s) words of 8 bytes.
__global__ void __launch_bounds__(kPrepThreads) k_dc_prep(int64_t off, int s, int m, int64_t bidx,
                                                          const double* __restrict__ e,
                                                          const double* __restrict__ D,
                                                          const double* __restrict__ Q, int64_t ldq, DcMerge mg,
                                                          double* __restrict__ zc, int use_smem) {
  extern __shared__ double psm[];
  __shared__ int cnt[kPrepThreads + 1];
  __shared__ double shr[33];
  // shared memory (or the global scratch of the merge): Dp, zp, key (s words
  // each), then eight int arrays of s entries
  double* Dp = use_smem ? psm : mg.Dp;   // merged, then rotated
  double* zp = use_smem ? psm + s : mg.zp;
  long long* key = reinterpret_cast<long long*>(use_smem ? psm + 2 * s : mg.dscr);
  int* ib = use_smem ? reinterpret_cast<int*>(psm + 3 * s) : nullptr;
  int* perm = use_smem ? ib : mg.perm;
  int* defl = use_smem ? ib + s : mg.src;
  int* nd = use_smem ? ib + 2 * s : mg.nd;
  int* df = use_smem ? ib + 3 * s : mg.df;
  int* sv = use_smem ? ib + 4 * s : mg.iscr;        // survivors, in order
  int* flg = use_smem ? ib + 5 * s : mg.iscr + s;   // flags
  int* pos = use_smem ? ib + 6 * s : mg.iscr + 2 * s;
  int* rot = use_smem ? ib + 7 * s : mg.iscr + 3 * s;  // pair u (survivors u-1, u) rotates
  const int t = threadIdx.x, T = blockDim.x;
  const double beta = e[bidx];
  const double sgn = beta < 0 ? -1.0 : 1.0;
  const double inv2 = 0.70710678118654752440;
  const double rho = 2.0 * fabs(beta);
  for (int p = t; p < s; p += T) {
    zc[p] = (p < m ? Q[(off + m - 1) * ldq + off + p] : sgn * Q[(off + m) * ldq + off + p]) * inv2;
    key[p] = dkey(D[off + p]);
  }
  __syncthreads();
  // merge the two ascending lists (integer keys)
  if (t == 0) {
    mg.rho[0] = rho;
    int a = 0, b2 = m, q = 0;
    while (a < m || b2 < s) perm[q++] = (b2 >= s || (a < m && key[a] <= key[b2])) ? a++ : b2++;
  }
  __syncthreads();
  double dmax = 0, zmax = 0;
  for (int q = t; q < s; q += T) {
    Dp[q] = D[off + perm[q]];
    zp[q] = zc[perm[q]];
    dmax = fmax(dmax, fabs(Dp[q]));
    zmax = fmax(zmax, fabs(zp[q]));
  }
  // block maxima (the partial maxima are non-negative: reuse block_sum's shape)
  {
    const int lane = t & 31, warp = t >> 5, nw = T >> 5;
    for (int o = 16; o > 0; o >>= 1) {
      dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
      zmax = fmax(zmax, __shfl_xor_sync(0xffffffffu, zmax, o));
    }
    if (lane == 0) {
      shr[warp] = dmax;
      shr[16 + warp] = zmax;
    }
    __syncthreads();
    if (t == 0) {
      double a = 0, b = 0;
      for (int w = 0; w < nw; w++) {
        a = fmax(a, shr[w]);
        b = fmax(b, shr[16 + w]);
      }
      shr[32] = 8.0 * kEps * fmax(a, rho * b);
    }
    __syncthreads();
  }
  const double tol = shr[32];
  // survivors of the small-z test, compacted in order
  for (int q = t; q < s; q += T) flg[q] = rho * fabs(zp[q]) <= tol ? 0 : 1;
  __syncthreads();
  const int nsv = block_scan_flags(flg, s, pos, cnt);
  for (int q = t; q < s; q += T)
    if (flg[q]) sv[pos[q]] = q;
  __syncthreads();
  // the rotation test of each consecutive pair of survivors, from the merged values
  for (int u = t + 1; u < nsv; u += T) {
    const int i = sv[u - 1], j = sv[u];
    const double r = sqrt(zp[i] * zp[i] + zp[j] * zp[j]);
    rot[u] = fabs((Dp[j] - Dp[i]) * (zp[j] / r) * (zp[i] / r)) <= tol ? 1 : 0;
  }
  for (int q = t; q < s; q += T) defl[q] = flg[q] ? 0 : 1;
  __syncthreads();
  // serial walk over the survivors: rotations (recomputing a pair's test only
  // when the previous rotation changed its left pole)
  if (t == 0) {
    int ng = 0;
    bool changed = false;
    for (int u = 1; u < nsv; u++) {
      const int i = sv[u - 1], j = sv[u];
      bool take = rot[u] != 0;
      double r = 0, c = 0, sn = 0;
      if (take || changed) {
        r = sqrt(zp[i] * zp[i] + zp[j] * zp[j]);
        c = zp[j] / r;
        sn = -zp[i] / r;
        if (changed) take = fabs((Dp[j] - Dp[i]) * c * sn) <= tol;
      }
      changed = false;
      if (take) {
        zp[j] = r;
        zp[i] = 0.0;
        mg.gi[ng] = i;
        mg.gj[ng] = j;
        mg.gc[ng] = c;
        mg.gs[ng] = sn;
        ng++;
        const double di = Dp[i], dj = Dp[j];
        Dp[i] = di * c * c + dj * sn * sn;
        Dp[j] = di * sn * sn + dj * c * c;
        defl[i] = 1;
        changed = true;
      }
    }
    cnt[0] = ng;
  }
  __syncthreads();
  const int ng = cnt[0];
  __syncthreads();
  // non-deflated and deflated positions, each in position order, then by
  // ascending Dp (the rotations may have moved a value slightly)
  for (int q = t; q < s; q += T) flg[q] = defl[q] ? 0 : 1;
  __syncthreads();
  const int K = block_scan_flags(flg, s, pos, cnt);
  for (int q = t; q < s; q += T) {
    if (flg[q]) nd[pos[q]] = q;
    else df[q - pos[q]] = q;
    key[q] = dkey(Dp[q]);
  }
  __syncthreads();
  const int nf = s - K;
  if (t == 0) {
    for (int u = 1; u < K; u++) {
      const int x = nd[u];
      const long long kx = key[x];
      int v = u - 1;
      while (v >= 0 && key[nd[v]] > kx) {
        nd[v + 1] = nd[v];
        v--;
      }
      nd[v + 1] = x;
    }
  } else if (t == 32) {
    for (int u = 1; u < nf; u++) {
      const int x = df[u];
      const long long kx = key[x];
      int v = u - 1;
      while (v >= 0 && key[df[v]] > kx) {
        df[v + 1] = df[v];
        v--;
      }
      df[v + 1] = x;
    }
  }
  if (t == 64) {
    mg.ctl[0] = K;
    mg.ctl[1] = ng;
    mg.ctl[2] = nf;
  }
  __syncthreads();
  for (int u = t; u < K; u += T) {
    mg.dk[u] = Dp[nd[u]];
    mg.zk[u] = zp[nd[u]];
  }
  if (use_smem) {
    for (int p = t; p < s; p += T) {
      mg.perm[p] = perm[p];
      mg.Dp[p] = Dp[p];
    }
    for (int u = t; u < K; u += T) mg.nd[u] = nd[u];
    for (int u = t; u < nf; u += T) mg.df[u] = df[u];
  }
}

// QsT[q][r] = column perm[q] of the node's block (row r), then the deflation
// rotations applied in order (thread per row r).
__global__ void k_dc_gather_rotate(int64_t off, int s, const double* __restrict__ Q, int64_t ldq, DcMerge mg,
                                   double* __restrict__ QsT) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= s) return;
  const double* Qr = Q + (off + r) * ldq + off;
  for (int q = 0; q < s; q++) QsT[(int64_t)q * s + r] = Qr[mg.perm[q]];
  const int ng = mg.ctl[1];
  for (int g = 0; g < ng; g++) {
    const int i = mg.gi[g], j = mg.gj[g];
    const double c = mg.gc[g], sn = mg.gs[g];
    const double qi = QsT[(int64_t)i * s + r], qj = QsT[(int64_t)j * s + r];
    QsT[(int64_t)i * s + r] = c * qi + sn * qj;
    QsT[(int64_t)j * s + r] = -sn * qi + c * qj;
  }
}

// Root j of the secular equation F(l) = 1/rho + sum_i z_i^2 / (d_i - l) = 0
// (d ascending, rho > 0): in (d_j, d_j+1) for j < K-1, in (d_K-1, d_K-1 + rho
// |z|^2] for the last.  The root is carried as an offset tau from the nearer
// pole (origin), so that every difference d_i - lambda = (d_i - d_o) - tau is
// accurate.  Each iteration fits the poles left of the interval by
// c1 + s1/(d_j - l) and those right of it by c2 + s2/(d_j+1 - l) (value and
// derivative matched at the current point) and takes the root of the fit in
// the interval, falling back to bisection of the bracket.  One warp per root:
// the lanes split the sums over the poles.
__global__ void k_dc_secular(DcMerge mg, int* __restrict__ err) {
  const int K = mg.ctl[0];
  const int j = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (j >= K) return;
  const double rho = mg.rho[0];
  const double* dk = mg.dk;
  const double* zk = mg.zk;
  int o;
  double lo, hi;
  if (j < K - 1) {
    const double mid = 0.5 * (dk[j + 1] - dk[j]);
    double f = 0;
    for (int i = lane; i < K; i += 32) f += zk[i] * zk[i] / ((dk[i] - dk[j]) - mid);
    f = warp_sum(f) + 1.0 / rho;
    if (f >= 0) {
      o = j;
      lo = 0.0;
      hi = mid;
    } else {
      o = j + 1;
      lo = -mid;
      hi = 0.0;
    }
  } else {
    o = j;
    double z2 = 0;
    for (int i = lane; i < K; i += 32) z2 += zk[i] * zk[i];
    z2 = warp_sum(z2);
    lo = 0.0;
    hi = rho * z2;
  }
  const double dor = dk[o];
  double tau = 0.5 * (lo + hi);
  bool conv = false;
  for (int it = 0; it < 200; it++) {
    double F = 0, aF = 0, p1 = 0, dp1 = 0, p2 = 0, dp2 = 0;
    for (int i = lane; i < K; i += 32) {
      const double rdel = 1.0 / ((dk[i] - dor) - tau);
      const double tm = zk[i] * zk[i] * rdel;
      F += tm;
      aF += fabs(tm);
      if (i <= j) {
        p1 += tm;
        dp1 += tm * rdel;
      } else {
        p2 += tm;
        dp2 += tm * rdel;
      }
    }
    F = warp_sum(F) + 1.0 / rho;
    aF = warp_sum(aF) + 1.0 / rho;
    p1 = warp_sum(p1);
    dp1 = warp_sum(dp1);
    p2 = warp_sum(p2);
    dp2 = warp_sum(dp2);
    if (fabs(F) <= 8.0 * kEps * aF) {
      conv = true;
      break;
    }
    if (F < 0) lo = tau;
    else hi = tau;
    double eta;
    const double a1 = (dk[j] - dor) - tau;
    if (j < K - 1) {
      const double a2 = (dk[j + 1] - dor) - tau;
      const double s1 = dp1 * a1 * a1, s2 = dp2 * a2 * a2;
      const double c = 1.0 / rho + (p1 - s1 / a1) + (p2 - s2 / a2);
      // c (a1 - x)(a2 - x) + s1 (a2 - x) + s2 (a1 - x) = 0, root x in (a1, a2)
      const double qa = c, qb = -(c * (a1 + a2) + s1 + s2), qc = c * a1 * a2 + s1 * a2 + s2 * a1;
      eta = NAN;
      if (qa == 0.0) {
        if (qb != 0.0) eta = -qc / qb;
      } else {
        const double disc = fmax(qb * qb - 4.0 * qa * qc, 0.0);
        const double qq = -0.5 * (qb + copysign(sqrt(disc), qb));
        const double x1 = qq / qa, x2 = qq != 0.0 ? qc / qq : NAN;
        const double lo_x = fmin(a1, a2), hi_x = fmax(a1, a2);
        if (x1 > lo_x && x1 < hi_x) eta = x1;
        else if (x2 > lo_x && x2 < hi_x) eta = x2;
      }
    } else {
      const double s1 = dp1 * a1 * a1;
      const double c = 1.0 / rho + (p1 - s1 / a1);
      eta = c != 0.0 ? a1 + s1 / c : NAN;
    }
    double nt = tau + eta;
    if (!(nt > lo && nt < hi)) nt = 0.5 * (lo + hi);
    if (nt == tau) {
      conv = true;
      break;
    }
    tau = nt;
  }
  if (lane == 0) {
    if (!conv) atomicExch(err, 3);
    mg.orig[j] = o;
    mg.taus[j] = tau;
    mg.lam[j] = dor + tau;
  }
}

// Loewner: zh_i^2 = prod_j (lambda_j - d_i) / (rho prod_{j != i} (d_j - d_i)),
// as a product of ratios of order one; sign of z_i.  Warp per i: each lane
// multiplies a strided subset, the partial products are combined.
__global__ void k_dc_lowner(DcMerge mg) {
  const int K = mg.ctl[0];
  const int i = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (i >= K) return;
  const double* dk = mg.dk;
  const double di = dk[i];
  double prod = 1.0;
  for (int j = lane; j < K; j += 32) {
    const double lmd = (dk[mg.orig[j]] - di) + mg.taus[j];
    prod *= j == K - 1 ? lmd / mg.rho[0] : lmd / ((j < i ? dk[j] : dk[j + 1]) - di);
  }
  for (int o = 16; o > 0; o >>= 1) prod *= __shfl_xor_sync(0xffffffffu, prod, o);
  if (lane == 0) mg.zh[i] = copysign(sqrt(fmax(prod, 0.0)), mg.zk[i]);
}

// Column norms of u_j = zh / (d - lambda_j) (warp per column).
__global__ void k_dc_colnorm(DcMerge mg) {
  const int K = mg.ctl[0];
  const int j = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (j >= K) return;
  const double dor = mg.dk[mg.orig[j]], tj = mg.taus[j];
  double s = 0;
  for (int i = lane; i < K; i += 32) {
    const double u = mg.zh[i] / ((mg.dk[i] - dor) - tj);
    s += u * u;
  }
  s = warp_sum(s);
  if (lane == 0) mg.cnrm[j] = sqrt(s);
}

// UT[j][i] = zh_i / (d_i - lambda_j) / |u_j| (K x K, row j = u_j), and the
// non-deflated columns of QsT gathered: QselT[q][r] = QsT[nd[q]][r].
__global__ void k_dc_vectors(int s, DcMerge mg, double* __restrict__ UT, const double* __restrict__ QsT,
                             double* __restrict__ QselT) {
  const int K = mg.ctl[0];
  const int64_t tot = (int64_t)K * K, tot2 = (int64_t)K * s;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot + tot2;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (e < tot) {
      const int j = (int)(e / K), i = (int)(e % K);
      UT[e] = mg.zh[i] / ((mg.dk[i] - mg.dk[mg.orig[j]]) - mg.taus[j]) / mg.cnrm[j];
    } else {
      const int64_t f = e - tot;
      const int q = (int)(f / s), r = (int)(f % s);
      QselT[f] = QsT[(int64_t)mg.nd[q] * s + r];
    }
  }
}

// The node's eigenvalues in ascending order (roots and deflated values
// merged) and, per final position, the source column.
__global__ void k_dc_order(int64_t off, DcMerge mg, double* __restrict__ D) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  const int K = mg.ctl[0], nf = mg.ctl[2];
  int a = 0, b = 0, t = 0;
  while (a < K || b < nf) {
    const bool root = b >= nf || (a < K && mg.lam[a] <= mg.Dp[mg.df[b]]);
    if (root) {
      D[off + t] = mg.lam[a];
      mg.src[t] = a++;
    } else {
      D[off + t] = mg.Dp[mg.df[b]];
      mg.src[t] = -1 - b++;
    }
    t++;
  }
}

// Q block column t <- its source: QnT[q] (the q-th new eigenvector, K x s) or
// QsT[df[.]] (a deflated column).
__global__ void k_dc_assemble(int64_t off, int s, DcMerge mg, const double* __restrict__ QnT,
                              const double* __restrict__ QsT, double* __restrict__ Q, int64_t ldq) {
  const int64_t tot = (int64_t)s * s;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / s), t = (int)(e % s);
    const int sc = mg.src[t];
    Q[(off + r) * ldq + off + t] = sc >= 0 ? QnT[(int64_t)sc * s + r] : QsT[(int64_t)mg.df[-1 - sc] * s + r];
  }
}

// Block reflector of the back-transformation: Vp (rows x nbp, rows [j0+1, n))
// with the unit leading entries and the stored reflectors of columns
// j0 .. j0+nbp-1 of A.
__global__ void k_bt_vp(int64_t n, int64_t j0, int nbp, const double* __restrict__ A, double* __restrict__ Vp) {
  const int64_t rows = n - j0 - 1, tot = rows * nbp;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = j0 + 1 + e / nbp;
    const int c = (int)(e % nbp);
    const int64_t jc = j0 + c;
    Vp[e] = i == jc + 1 ? 1.0 : (i > jc + 1 ? A[i * n + jc] : 0.0);
  }
}

// Triangular factor of the compact WY form H_j0 ... H_j0+nbp-1 = I - V T V^T:
// T[c][c] = tau_c, T[0:c, c] = -tau_c T[0:c, 0:c] (V^T V)[0:c, c].  Row r of T
// depends only on row r and V^T V: a warp per row, its lanes splitting each
// sum (V^T V's strictly upper triangle packed in shared memory, G[q][c] at
// c(c-1)/2 + q; the warp's row of T in shared memory).
constexpr int kTfWarps = 16;
__global__ void __launch_bounds__(32 * kTfWarps) k_bt_tfactor(int nbp, const double* __restrict__ VtV,
                                                             const double* __restrict__ tau, double* __restrict__ T) {
  extern __shared__ double smt[];
  double* Gu = smt;                               // nbp (nbp - 1) / 2
  double* rows = smt + nbp * (nbp - 1) / 2;       // kTfWarps x nbp
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  for (int e = t; e < nbp * nbp; e += blockDim.x) {
    const int q = e / nbp, c = e % nbp;
    if (q < c) Gu[c * (c - 1) / 2 + q] = VtV[e];
  }
  __syncthreads();
  const int r = blockIdx.x * kTfWarps + w;
  if (r >= nbp) return;
  double* Tr = rows + w * nbp;
  for (int c = lane; c < nbp; c += 32) Tr[c] = c == r ? tau[r] : 0.0;
  __syncwarp();
  for (int c = r + 1; c < nbp; c++) {
    const double* gc = Gu + c * (c - 1) / 2;
    double acc = 0;
    for (int q = r + lane; q < c; q += 32) acc += Tr[q] * gc[q];
    acc = warp_sum(acc);
    if (lane == 0) Tr[c] = -tau[c] * acc;
    __syncwarp();
  }
  for (int c = lane; c < nbp; c += 32) T[(int64_t)r * nbp + c] = Tr[c];
}

__global__ void k_copy_cols(int64_t rows, int64_t cols, const double* __restrict__ src, int64_t lds,
                            double* __restrict__ dst, int64_t ldd) {
  const int64_t tot = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x)
    dst[(e / cols) * ldd + e % cols] = src[(e / cols) * lds + e % cols];
}

__global__ void k_transpose_into(int64_t rows, int64_t cols, const double* __restrict__ src, int64_t lds,
                                 double* __restrict__ dst, int64_t ldd) {
  const int64_t tot = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / cols, c = e % cols;
    dst[c * ldd + r] = src[r * lds + c];
  }
}

__global__ void k_symmetrize_full(int64_t n, double* __restrict__ A) {
  const int64_t tot = n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / n, j = e % n;
    if (j > i) {
      const double v = 0.5 * (A[i * n + j] + A[j * n + i]);
      A[i * n + j] = v;
      A[j * n + i] = v;
    }
  }
}

inline unsigned grid_for(int64_t tot, int threads = 256) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(cdiv(tot, threads), 152 * 16));
}

struct Node {
  int off, s, m;
};

void build_tree(int off, int s, std::vector<Node>& merges, std::vector<int>& loff, std::vector<int>& lsize) {
  if (s <= kLeaf) {
    loff.push_back(off);
    lsize.push_back(s);
    return;
  }
  const int m = s / 2;
  build_tree(off, m, merges, loff, lsize);
  build_tree(off + m, s - m, merges, loff, lsize);
  merges.push_back({off, s, m});  // post-order: children first
}

}  // namespace

// Eigen-decomposition of a symmetric n x n A (row-major; both triangles read
// and symmetrised): all eigenvalues ascending into w_dev (and w_host); the
// eigenvectors of the `want` largest (want <= n) into rows 0..want-1 of A,
// ascending, row q = eigenvector of w[n - want + q].
// Large FP64 products of the solver on the tensor cores (the integer-slice
// GEMM of the FP64 H-apply engine: 49 bits of every value relative to its row
// or column scale), the others on the FP64 tile GEMM.
static fkf_status gemm_big(fkf_ctx* ctx, bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha,
                           const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* C,
                           int64_t ldc) {
  if (ctx->fp64_tc && (double)M * N * K >= 1e8 && cdiv(M, 128) * cdiv(N, 64) >= 16)
    return gemm_f64_tc(ctx, ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
  return gemm_f64(ctx, ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
}

fkf_status eigh_own(fkf_ctx* ctx, int n, double* A, double* w_dev, std::vector<double>& w_host, DevBuf& ws,
                    int want) {
  cudaStream_t st = ctx->stream;
  w_host.assign(n, 0.0);
  if (n <= 0) return FKF_OK;
  want = std::max(0, std::min(want, n));
  const int64_t N = n, nn = N * N;
  const int64_t L = 2 * kNB;
  DevBuf gws;  // partial sums of the back-transformation's long products
  // workspace layout (doubles)
  int sms = 0;
  FKF_CUDA(ctx, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
  const int gmax = std::max(1, sms);
  const int64_t w_Q = nn, w_QsT = nn, w_QselT = nn, w_U = nn, w_Qn = nn;
  const int64_t w_X = N * std::max(want, 1);
  const int64_t w_VW = N * L, w_WV = N * L;
  const int64_t w_vec = 20 * N + 64;                       // d, e, tau, col, vg, pg, zc, the merge arrays
  const int64_t w_part = (int64_t)gmax * (3 + L) + 64;
  const int64_t w_small = 2 * kBT * kBT + N * kBT + kBT * std::max<int64_t>(want, 1) + 64;  // back-transformation
  const int64_t total = w_Q + w_QsT + w_QselT + w_U + w_Qn + w_X + w_VW + w_WV + w_vec + w_part + w_small;
  const size_t ints = (size_t)15 * N + 128;
  const size_t need = (size_t)total * 8 + ints * 4 + 256;
  if (ws.bytes < need) FKF_TRY(dev_alloc(ctx, ws, need));
  double* p = ws.as<double>();
  auto take = [&](int64_t k) {
    double* r = p;
    p += k;
    return r;
  };
  double* Q = take(w_Q);
  double* QsT = take(w_QsT);
  double* QselT = take(w_QselT);
  double* U = take(w_U);
  double* Qn = take(w_Qn);
  double* X = take(w_X);
  double* VW = take(w_VW);
  double* WV = take(w_WV);
  double* d = take(N);
  double* e = take(N);
  double* tau = take(N);
  double* col = take(N);
  double* vg = take(N);
  double* pg = take(N);
  DcMerge mg{};
  mg.Dp = take(N);
  mg.zp = take(N);
  mg.gc = take(N);
  mg.gs = take(N);
  mg.dk = take(N);
  mg.zk = take(N);
  mg.taus = take(N);
  mg.lam = take(N);
  mg.zh = take(N);
  mg.cnrm = take(N);
  mg.rho = take(8);
  double* zc = take(N);
  mg.dscr = take(N);
  double* part = take(w_part);
  double* Vp = take(N * kBT);
  double* Y1 = take(kBT * std::max<int64_t>(want, 1));
  double* VtV = take(kBT * kBT);
  double* Tf = take(kBT * kBT);
  int* ip = reinterpret_cast<int*>(p + 8);
  mg.perm = ip;
  mg.gi = ip + N;
  mg.gj = ip + 2 * N;
  mg.nd = ip + 3 * N;
  mg.df = ip + 4 * N;
  mg.orig = ip + 5 * N;
  mg.src = ip + 6 * N;
  int* loff_d = ip + 7 * N;
  int* lsize_d = ip + 8 * N;
  int* splits_d = ip + 9 * N;
  mg.ctl = ip + 10 * N;   // 8 ints
  mg.iscr = ip + 10 * N + 64;  // 4 N ints
  int* err = ip + 10 * N + 16;
  FKF_CUDA(ctx, cudaMemsetAsync(err, 0, 4 * sizeof(int), st));
  FKF_CUDA(ctx, cudaMemsetAsync(e, 0, N * 8, st));
  FKF_CUDA(ctx, cudaMemsetAsync(tau, 0, N * 8, st));
  k_symmetrize_full<<<grid_for(nn), 256, 0, st>>>(N, A);
  FKF_LAUNCHED(ctx);

  // ---- 1. tridiagonal reduction: one cooperative panel kernel over every SM per panel
  unsigned* bar = reinterpret_cast<unsigned*>(ip + 10 * N + 8);
  FKF_CUDA(ctx, cudaFuncSetAttribute(k_trd_panel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(kTrdSmemV * sizeof(double))));
  for (int64_t j0 = 0; j0 < N; j0 += kNB) {
    const int nbp = (int)std::min<int64_t>(kNB, N - j0);
    FKF_CUDA(ctx, cudaMemsetAsync(VW, 0, w_VW * 8, st));
    FKF_CUDA(ctx, cudaMemsetAsync(WV, 0, w_WV * 8, st));
    FKF_CUDA(ctx, cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), st));
    const int G = (int)std::max<int64_t>(4, std::min<int64_t>(gmax, (N - j0) / 8));
    TrdArgs ta{A, N, j0, nbp, VW, WV, d, e, tau, col, vg, pg, part, bar, err};
    void* args[] = {&ta};
    const size_t vsm = (size_t)std::min<int64_t>(N, kTrdSmemV) * sizeof(double);
    FKF_CUDA(ctx, cudaLaunchCooperativeKernel((const void*)k_trd_panel, dim3(G), dim3(kTrdThreads), args, vsm, st));
    ctx->launches++;
    const int64_t j1 = j0 + nbp;
    if (j1 < N) {
      // A[j1:, j1:] -= [V W] [W V]^T = V W^T + W V^T (large trailing blocks on the tensor
      // cores: both triangles computed, symmetric to rounding; the panel kernel reads rows)
      if (ctx->fp64_tc && N - j1 >= 512)
        FKF_TRY(gemm_f64_tc(ctx, false, true, N - j1, N - j1, L, -1.0, VW + j1 * L, L, WV + j1 * L, L, 1.0,
                            A + j1 * N + j1, N));
      else
        FKF_TRY(gemm_sym_f64(ctx, false, true, N - j1, L, -1.0, VW + j1 * L, L, WV + j1 * L, L, 1.0,
                             A + j1 * N + j1, N));
    }
  }

  // ---- 2. divide and conquer on the tridiagonal (d, e)
  std::vector<Node> merges;
  std::vector<int> loff, lsize, splits;
  build_tree(0, n, merges, loff, lsize);
  for (const Node& nd : merges) splits.push_back(nd.off + nd.m);
  FKF_CUDA(ctx, cudaMemsetAsync(Q, 0, nn * 8, st));
  FKF_CUDA(ctx, cudaMemcpyAsync(loff_d, loff.data(), loff.size() * 4, cudaMemcpyHostToDevice, st));
  FKF_CUDA(ctx, cudaMemcpyAsync(lsize_d, lsize.data(), lsize.size() * 4, cudaMemcpyHostToDevice, st));
  if (!splits.empty()) {
    FKF_CUDA(ctx, cudaMemcpyAsync(splits_d, splits.data(), splits.size() * 4, cudaMemcpyHostToDevice, st));
    k_dc_split_d<<<1, 32, 0, st>>>((int)splits.size(), splits_d, d, e);
    FKF_LAUNCHED(ctx);
  }
  double* Dv = w_dev;  // eigenvalues of the nodes, in place
  k_dc_leaf<<<(unsigned)loff.size(), 32, 0, st>>>(loff_d, lsize_d, d, e, Dv, Q, N, err);
  FKF_LAUNCHED(ctx);
  FKF_CUDA(ctx, cudaFuncSetAttribute(k_dc_prep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPrepSmem));
  for (const Node& nd : merges) {
    const int s = nd.s;
    const size_t psm = (size_t)s * (3 * sizeof(double) + 8 * sizeof(int));
    const int use_smem = psm <= kPrepSmem ? 1 : 0;
    k_dc_prep<<<1, kPrepThreads, use_smem ? psm : 0, st>>>(nd.off, s, nd.m, nd.off + nd.m - 1, e, Dv, Q, N, mg, zc,
                                                           use_smem);
    FKF_LAUNCHED(ctx);
    int hc[3] = {0, 0, 0};
    FKF_CUDA(ctx, cudaMemcpyAsync(hc, mg.ctl, sizeof(hc), cudaMemcpyDeviceToHost, st));
    k_dc_gather_rotate<<<(unsigned)cdiv(s, 128), 128, 0, st>>>(nd.off, s, Q, N, mg, QsT);
    FKF_LAUNCHED(ctx);
    FKF_CUDA(ctx, cudaStreamSynchronize(st));
    const int K = hc[0];
    if (K > 0) {
      const unsigned wb = (unsigned)cdiv((int64_t)K * 32, 128);  // a warp per root / index
      k_dc_secular<<<wb, 128, 0, st>>>(mg, err);
      FKF_LAUNCHED(ctx);
      k_dc_lowner<<<wb, 128, 0, st>>>(mg);
      FKF_LAUNCHED(ctx);
      k_dc_colnorm<<<wb, 128, 0, st>>>(mg);
      FKF_LAUNCHED(ctx);
      k_dc_vectors<<<grid_for((int64_t)K * K + (int64_t)K * s), 256, 0, st>>>(s, mg, U, QsT, QselT);
      FKF_LAUNCHED(ctx);
      // QnT (K x s) = UT QselT: row q = the q-th new eigenvector in the node's basis
      FKF_TRY(gemm_big(ctx, false, false, K, s, K, 1.0, U, K, QselT, s, 0.0, Qn, s));
    }
    k_dc_order<<<1, 32, 0, st>>>(nd.off, mg, Dv);
    FKF_LAUNCHED(ctx);
    k_dc_assemble<<<grid_for((int64_t)s * s), 256, 0, st>>>(nd.off, s, mg, Qn, QsT, Q, N);
    FKF_LAUNCHED(ctx);
  }

  // ---- 3. back-transformation of the wanted eigenvectors (the last `want` columns of Q)
  if (want > 0) {
    const int64_t k = want;
    k_copy_cols<<<grid_for(N * k), 256, 0, st>>>(N, k, Q + (N - k), N, X, k);
    FKF_LAUNCHED(ctx);
    const int64_t nref = N - 1;  // reflectors 0 .. n-2
    FKF_CUDA(ctx, cudaFuncSetAttribute(k_bt_tfactor, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (kBT * (kBT - 1) / 2 + kTfWarps * kBT) * (int)sizeof(double)));
    for (int64_t j0 = nref > 0 ? ((nref - 1) / kBT) * kBT : -1; j0 >= 0; j0 -= kBT) {
      const int nbp = (int)std::min<int64_t>(kBT, nref - j0);
      const int64_t rows = N - j0 - 1;
      if (rows <= 0 || nbp <= 0) continue;
      k_bt_vp<<<grid_for(rows * nbp), 256, 0, st>>>(N, j0, nbp, A, Vp);
      FKF_LAUNCHED(ctx);
      FKF_TRY(gram_f64(ctx, nbp, nbp, rows, Vp, nbp, Vp, nbp, VtV, nbp, gws));
      k_bt_tfactor<<<(unsigned)cdiv(nbp, kTfWarps), 32 * kTfWarps,
                     (size_t)(nbp * (nbp - 1) / 2 + kTfWarps * nbp) * sizeof(double), st>>>(nbp, VtV, tau + j0, Tf);
      FKF_LAUNCHED(ctx);
      double* Xs = X + (j0 + 1) * k;
      // X[j0+1:] -= V (T (V^T X[j0+1:]))
      if (ctx->fp64_tc && (double)nbp * k * rows >= 1e8 && cdiv(k, 64) >= 16)
        FKF_TRY(gemm_f64_tc(ctx, true, false, nbp, k, rows, 1.0, Vp, nbp, Xs, k, 0.0, Y1, k));
      else
        FKF_TRY(gram_f64(ctx, nbp, k, rows, Vp, nbp, Xs, k, Y1, k, gws));
      FKF_TRY(gemm_f64(ctx, false, false, nbp, k, nbp, 1.0, Tf, nbp, Y1, k, 0.0, QselT, k));
      FKF_TRY(gemm_big(ctx, false, false, rows, k, nbp, -1.0, Vp, nbp, QselT, k, 1.0, Xs, k));
    }
    // eigenvector q (column q of X) -> row q of A
    k_transpose_into<<<grid_for(N * k), 256, 0, st>>>(N, k, X, k, A, N);
    FKF_LAUNCHED(ctx);
  }
  int herr = 0;
  FKF_CUDA(ctx, cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  FKF_CUDA(ctx, cudaMemcpyAsync(w_host.data(), w_dev, N * 8, cudaMemcpyDeviceToHost, st));
  FKF_CUDA(ctx, cudaStreamSynchronize(st));
  FKF_TRY(gemm_f64_tc_check(ctx));
  if (herr) return set_err(ctx, FKF_ENOCONV, "symmetric eigensolver: %s (n=%d)",
                           herr == 1 ? "a grid barrier timed out" : (herr == 2 ? "QL did not converge" :
                                                                                  "secular equation did not converge"),
                           n);
  return FKF_OK;
}
