// Many small 3-way dense decompositions in one persistent launch: every
// thread-block cluster runs the whole N-GMRES solve (Algorithm 1: Step I the
// ALS sweep of Section 2.3, Step II the window least squares of Section 2.1
// with delta I, Step III the More-Thuente search of Section 2.4 on the line
// polynomial) of one request at a time, and takes the next request from a
// device queue when it finishes.  Cross-CTA steps meet at cluster barriers
// (barrier.cluster with release/acquire), so a request costs no kernel
// launches per iteration and its iterations never wait on the host.
//
// Work split inside a cluster of C CTAs (rank k):
//   * rows: CTA k owns rows [k I_n / C, (k+1) I_n / C) of every factor, of
//     every iterate and gradient block, and of M^(n); everything row-wise
//     (ALS updates, gradients, normalisation, window pushes, N-GMRES
//     combination) touches only its own rows;
//   * fibers: the tensor is read as T[j][i3] (j = i1 I2 + i2, the last index
//     fastest); CTA k owns fibers [k J / C, (k+1) J / C);
//   * sums (Grams, M^(3), window dots, column norms, slopes, f) are written
//     as per-CTA partials and added in rank order after a barrier, by every
//     CTA that needs them (the same order everywhere, so every CTA takes the
//     same decisions).
//
// Passes over T per iteration (one each, all CTAs): Y = T x_3 A^(3) for the
// sweep's modes 1 and 2; M^(3) of the swept point; Y' = T x_3 Abar^(3) for
// ubar's modes 1 and 2 (M^(3)(ubar) is the swept M^(3) with the
// normalisation's column scales); Z = T x_3 [Abar^(3) | D^(3)] for the line
// polynomial and the accepted point's modes 1 and 2; M^(3) at the accepted
// point.
//
// Precision per request phase: mixed (products and their sums over at most
// a few hundred terms in FP32 on the CUDA cores, partial sums added in FP64;
// Grams, solves, window least squares, f and the line search in FP64),
// then an FP64 phase that restarts the window from the FP64 gradient and runs
// to tol (the polish); or FP64 throughout.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <map>
#include <mutex>
#include <vector>

#include "cp_internal.cuh"
#include "linesearch.cuh"
#include "mt_device.cuh"
#include "newton.cuh"

namespace cpg {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxR = 32;      // rank limit
constexpr int kMaxW = 32;      // window limit
constexpr int kHLd = kMaxW + 1; // row stride of the window system in shared memory
constexpr int kMaxC = 8;       // cluster size limit (portable clusters)
constexpr int kMaxI = 256;     // side limit
constexpr int kMaxIR = 8192;   // I_n R limit (the M^(3) accumulators live in shared memory)
constexpr int kColW = 16;      // columns per register tile in the passes
constexpr int kBsCols = 32;    // columns of the factor staged at once for Y = T x_3 B
constexpr int kFlush = 8;      // chunks between FP64 flushes of the FP32 accumulators
constexpr int kTile = 128;     // window elements per shared-memory tile
constexpr int kTileLd = kTile + 1;

enum { STOP_RUN = 0, STOP_TOL = 1, STOP_MAXIT = 2, STOP_STALL = 3, STOP_NONFINITE = 4 };
enum { PH_MIXED = 1, PH_FP64 = 2, PH_DONE = 3 };
// scal[] slots
enum { S_F = 0, S_FBAR = 1, S_BETA = 2, S_ACCEPT = 3, S_PARK = 4, S_NSCAL = 8 };

struct ManyCtl {
  int iters, fg_evals, als_sweeps, restarts, ls_failures, ls_trials, accepts;
  int mixed_iters, fp64_iters;
  int phase;          // PH_*
  int start;          // 2: normalise the start point, then start a phase; 1: start a phase; 0: iterate
  int stop;           // STOP_* of the last test
  int status;         // cp_status of the request
  int win_start, win_m;
  int since_best;
  int ysrc;           // T x_3 A^(3)(u) for the next sweep: 0 none, 1 in Y (stride R),
                      // 2 in Y2 (stride R), 3 the first R columns of Y (stride 2R)
  double best, gn, f;
};

struct ManyReq {
  const void* T;      // T[j][i3], J x I3, j = i1 I2 + i2 (modes 1, 2, 3 of the paper)
  int t64;            // T holds doubles
  int I1, I2, I3, J, R, P;
  int off2, off3;     // element offsets of A^(2), A^(3) in an iterate
  double normT2;
  double tol, tol_mixed, eps;
  int maxit, w, polish, stall;
  cp_ls_opts ls, ls_mixed;
  double *u, *g, *ub, *gb, *uh, *d, *x, *U, *G;
  double* Y;          // J x 2R (floats in the mixed phase)
  double* Y2;         // J x R: T x_3 A^(3) of the accepted point's normalisation
  double *M1, *M2, *M3, *M3s;   // M^(n) at the current point; the swept point's M^(3)
  double *V1, *V2;    // line-search variants of modes 1, 2: 4 x I1 x R, 4 x I2 x R
  double* K;          // w x w: g_a^T g_b of the window's gradients by ring slot (mixed phase)
  double* part;       // kMaxC x part_ld partials: two large regions of big_ld, two of 128 scalars
  int part_ld, big_ld;
  double *Gu, *Gs, *Gb, *Gad, *Gdd, *Gx;   // Grams (3 x R x R): u, swept, ubar, ubar^T d, d^T d, x
  double* scal;
  ManyCtl* ctl;
};

struct ManyQueue {
  int next;
  int ntasks;
  unsigned long long budget_ns;   // a cluster parks its request after this long
};

// Small shared state of one CTA.
struct EngSh {
  ManyReq q;
  ManyCtl c;
  double A[kMaxR * kMaxR];        // Gammabar and its inverse
  double A0[kMaxR * kMaxR];       // a copy for the ridge retry
  double H[kMaxW * kHLd];         // window system, rows padded against bank conflicts
  double rhs[kMaxW];
  double alpha[kMaxW];
  double nu[3 * kMaxR];
  double scale[3 * kMaxR];
  double key[kMaxR];
  double lam[kMaxR];
  double sc2[3 * kMaxR];          // second set of scales (the other normalisation of a step)
  double poly[8];
  double red[kWarps];
  double redn[kWarps * 8];
  double bcast[8];
  int order[kMaxR];
  int order2[kMaxR];
  double gp[kThreads];            // Gram partials of the row groups
  unsigned long long t0;
  int task;
  int flag;
};

// ---------------------------------------------------------------- cluster

__device__ __forceinline__ unsigned cl_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cl_size() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cl_id() {
  unsigned r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return r;
}
// Every thread of every CTA of the cluster; global and shared writes before
// it are visible to the cluster's threads after it.
__device__ __forceinline__ void cl_sync() {
  asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}
__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int lo_of(int n, int k, int C) { return (int)(((long long)n * k) / C); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the CTA (fixed order); every thread gets it.
__device__ double cta_sum(double v, EngSh& sh) {
  v = warp_sum(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh.red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) s += sh.red[w];
  return s;
}

// NV sums over the CTA at once (NV <= 8, fixed order); every thread gets them.
template <int NV>
__device__ void cta_sums(double* v, EngSh& sh) {
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
  __syncthreads();
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) sh.redn[(threadIdx.x >> 5) * 8 + k] = v[k];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) s += sh.redn[w * 8 + k];
    v[k] = s;
  }
}

// Sum over the cluster's partials part[c * ld + k] in rank order.
__device__ __forceinline__ double psum(const double* part, int ld, int C, int k) {
  double s = 0.0;
  for (int c = 0; c < C; ++c) s += part[(size_t)c * ld + k];
  return s;
}


__device__ __forceinline__ float fmat(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmat(double a, double b, double c) { return __fma_rn(a, b, c); }

// ------------------------------------------------------------ passes over T

// Asynchronous copies global -> shared (cp.async, sm_80 and later): every
// thread issues its share of a tile, so hundreds of loads are in flight.
__device__ __forceinline__ void cp_async_el(float* dst, const float* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_el(double* dst, const double* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// Wait until at most N of this thread's newest copy groups are in flight.
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Tiles of T staged per step: 128 bytes of a row (32 floats, 16 doubles) for
// Y = T x_3 B; whole rows of kTF fibers (32 for floats, 16 for doubles) for M^(3).
template <typename TT>
struct Stage {
  static constexpr int kIC = 128 / (int)sizeof(TT);   // i3 per sub-tile in Y = T x_3 B
  static constexpr int kTF = 128 / (int)sizeof(TT);   // fibers per chunk in M^(3) at I3 = kMaxI
};
// M^(3)'s shared regions: the two T chunks and the Khatri-Rao rows.
constexpr size_t kTchBytes = 2 * (size_t)Stage<float>::kTF * kMaxI * sizeof(float);
constexpr size_t kKRBytes = 16384;

// Y[j][c0 + c] = sum_{i3} T[j][i3] B[i3][c] for the CTA's fibers j, where B
// is A (I3 x R) or [A | D] (I3 x 2R); Y has row stride ys (AT elements).
// Threads own fibers (blocks of 256); T arrives in 256-fiber x kIC-column
// sub-tiles (128 bytes of a row), double-buffered by cp.async from every
// thread and stored with row stride kIC + 1, so that a warp reading one
// column of its 32 rows hits 32 banks; the factor columns (32 at a time) are
// read as broadcasts; two kColW-column register tiles per thread.  (Measured
// against two fibers per thread with 64-byte sub-tiles and against a
// three-deep ring: 8-10 % faster than either on 64^3 and 128^3, R = 16.)
template <typename TT, typename AT>
__device__ __noinline__ void pass_y(const TT* __restrict__ T, int J, int I3, int R, const double* __restrict__ A,
                                    const double* __restrict__ D, AT* __restrict__ Y, int ys, int rk, int C, AT* Bs,
                                    TT* Tst) {
  constexpr int kIC = Stage<TT>::kIC, kLd = kIC + 1;
  const int ncol = D ? 2 * R : R;
  const int jlo = lo_of(J, rk, C), jhi = lo_of(J, rk + 1, C);
  const int nsub = (I3 + kIC - 1) / kIC;
  TT* const buf1 = Tst + kThreads * kLd;
  for (int c0 = 0; c0 < ncol; c0 += kBsCols) {
    const int nc = min(kBsCols, ncol - c0);
    const int ncp = (nc + kColW - 1) / kColW * kColW;
    __syncthreads();
    for (int e = threadIdx.x; e < I3 * ncp; e += kThreads) {
      const int i = e / ncp, c = e - (e / ncp) * ncp;
      const int cc = c0 + c;
      double v = 0.0;
      if (c < nc) v = cc < R ? A[(size_t)i * R + cc] : D[(size_t)i * R + cc - R];
      Bs[e] = (AT)v;
    }
    __syncthreads();
    const bool two = ncp > kColW;
    for (int jb = jlo; jb < jhi; jb += kThreads) {
      const int nrow = min(kThreads, jhi - jb);
      auto issue = [&](int sc, TT* dst) {
        const int i0 = sc * kIC, ni = min(kIC, I3 - i0);
        for (int e = threadIdx.x; e < kThreads * kIC; e += kThreads) {
          const int f = e / kIC, i = e - (e / kIC) * kIC;
          if (f < nrow && i < ni) cp_async_el(dst + f * kLd + i, T + (size_t)(jb + f) * I3 + i0 + i);
        }
        cp_async_commit();
      };
      AT acc0[kColW], acc1[kColW];
#pragma unroll
      for (int k = 0; k < kColW; ++k) {
        acc0[k] = (AT)0;
        acc1[k] = (AT)0;
      }
      issue(0, Tst);
      for (int sc = 0; sc < nsub; ++sc) {
        if (sc + 1 < nsub) {
          issue(sc + 1, ((sc + 1) & 1) ? buf1 : Tst);
          cp_async_wait<1>();
        } else {
          cp_async_wait<0>();
        }
        __syncthreads();
        const int i0 = sc * kIC, ni = min(kIC, I3 - i0);
        const TT* trow = ((sc & 1) ? buf1 : Tst) + threadIdx.x * kLd;
        const AT* b = Bs + (size_t)i0 * ncp;
        if (two) {
          for (int i = 0; i < ni; ++i) {
            const AT t = (AT)trow[i];
#pragma unroll
            for (int k = 0; k < kColW; ++k) {
              acc0[k] = fmat(t, b[k], acc0[k]);
              acc1[k] = fmat(t, b[kColW + k], acc1[k]);
            }
            b += ncp;
          }
        } else {
          for (int i = 0; i < ni; ++i) {
            const AT t = (AT)trow[i];
#pragma unroll
            for (int k = 0; k < kColW; ++k) acc0[k] = fmat(t, b[k], acc0[k]);
            b += ncp;
          }
        }
        __syncthreads();
      }
      if ((int)threadIdx.x < nrow) {
        AT* yrow = Y + (size_t)(jb + threadIdx.x) * ys + c0;
#pragma unroll
        for (int k = 0; k < kColW; ++k) {
          if (k < nc) yrow[k] = acc0[k];
          if (two && kColW + k < nc) yrow[kColW + k] = acc1[k];
        }
      }
    }
  }
}

// The CTA's partial of M^(3)(A, B): out[i3][r] = sum_{j in its fibers}
// T[j][i3] A[j / I2][r] B[j % I2][r] (I3 x R doubles).  T arrives in chunks
// of kTF whole rows (contiguous in memory), double-buffered by cp.async from
// every thread; each chunk's Khatri-Rao rows are formed in shared memory.
// Lanes own i3 (32-row x kColW-column output tiles); with at most kWarps
// tiles each gets kWarps / tiles warps that take every (kWarps / tiles)-th
// fiber of a chunk, with more a warp keeps two tiles.  Register sums are
// FP32 (or FP64) and are added into FP64 shared totals, one set per fiber
// group, every kFlush kTF fibers; the groups are added in order at the end.
// A chunk holds F = kTF 2^k fibers, as many as the two T buffers and the
// Khatri-Rao rows allow (up to kFlush kTF), so short rows come in longer
// chunks (fewer barriers and Khatri-Rao builds per fiber); the flush points
// and each group's fibers do not depend on F.  (Measured against 64-row
// tiles with the next chunk's Khatri-Rao rows loaded ahead and against a
// three-deep ring: 8-10 % faster.)
template <typename TT, typename AT>
__device__ __noinline__ void pass_m3(const TT* __restrict__ T, int J, int I2, int I3, int R, const double* __restrict__ A,
                                     const double* __restrict__ B, double* __restrict__ out, int rk, int C, TT* Tst,
                                     AT* KRs, double* Ms) {
  constexpr int kTF = Stage<TT>::kTF;
  const int Rp = (R + kColW - 1) / kColW * kColW;
  int F = kTF;
  while (2 * F <= kFlush * kTF && 2 * (size_t)(2 * F) * I3 * sizeof(TT) <= kTchBytes &&
         (size_t)(2 * F) * Rp * sizeof(AT) <= kKRBytes)
    F *= 2;
  const int flush_every = kFlush * kTF / F;
  const int nib = (I3 + 31) / 32, nct = Rp / kColW;
  const int units = nib * nct;
  const int wpu = units <= kWarps ? kWarps / units : 1;
  const int IR = I3 * R;
  const int jlo = lo_of(J, rk, C), jhi = lo_of(J, rk + 1, C);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = warp % wpu;
  TT* const buf1 = Tst + kTchBytes / 2 / sizeof(TT);
  for (int e = threadIdx.x; e < wpu * IR; e += kThreads) Ms[e] = 0.0;
  AT acc[2][kColW];
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int k = 0; k < kColW; ++k) acc[u][k] = (AT)0;
  auto issue = [&](int j0, TT* dst) {
    const int n = min(F, jhi - j0) * I3;
    const TT* src = T + (size_t)j0 * I3;
    for (int e = threadIdx.x; e < n; e += kThreads) cp_async_el(dst + e, src + e);
    cp_async_commit();
  };
  const int nch = (jhi - jlo + F - 1) / F;
  if (nch > 0) issue(jlo, Tst);
  int chunks = 0;
  for (int c = 0; c < nch; ++c) {
    const int j0 = jlo + c * F;
    const int nf = min(F, jhi - j0);
    for (int e = threadIdx.x; e < F * Rp; e += kThreads) {
      const int f = e / Rp, r = e - (e / Rp) * Rp;
      AT v = (AT)0;
      if (f < nf && r < R) {
        const int j = j0 + f;
        const int i1 = j / I2, i2 = j - (j / I2) * I2;
        v = (AT)A[(size_t)i1 * R + r] * (AT)B[(size_t)i2 * R + r];
      }
      KRs[e] = v;
    }
    if (c + 1 < nch) {
      issue(j0 + F, ((c + 1) & 1) ? buf1 : Tst);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const TT* tb = (c & 1) ? buf1 : Tst;
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int unit = units <= kWarps ? (u == 0 && warp < units * wpu ? warp / wpu : units) : warp + u * kWarps;
      if (unit < units) {
        const int ib = unit / nct, ct = unit - (unit / nct) * nct;
        const int i3 = ib * 32 + lane;
        const bool ok = i3 < I3;
        const TT* tcol = tb + (ok ? i3 : 0);
        const AT* b = KRs + ct * kColW;
        int f = grp;
        // four fibers at a time, their T values loaded first (the same
        // order of additions as one at a time)
        for (; f + 3 * wpu < nf; f += 4 * wpu) {
          AT t[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) t[q] = ok ? (AT)tcol[(f + q * wpu) * I3] : (AT)0;
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const AT* bf = b + (f + q * wpu) * Rp;
#pragma unroll
            for (int k = 0; k < kColW; ++k) acc[u][k] = fmat(t[q], bf[k], acc[u][k]);
          }
        }
        for (; f < nf; f += wpu) {
          const AT t = ok ? (AT)tcol[f * I3] : (AT)0;
          const AT* bf = b + f * Rp;
#pragma unroll
          for (int k = 0; k < kColW; ++k) acc[u][k] = fmat(t, bf[k], acc[u][k]);
        }
      }
    }
    if (++chunks == flush_every || c + 1 == nch) {
      chunks = 0;
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int unit = units <= kWarps ? (u == 0 && warp < units * wpu ? warp / wpu : units) : warp + u * kWarps;
        if (unit < units) {
          const int ib = unit / nct, ct = unit - (unit / nct) * nct;
          const int i3 = ib * 32 + lane;
          if (i3 < I3) {
#pragma unroll
            for (int k = 0; k < kColW; ++k) {
              const int r = ct * kColW + k;
              if (r < R) Ms[grp * IR + r * I3 + i3] += (double)acc[u][k];
            }
          }
        }
#pragma unroll
        for (int k = 0; k < kColW; ++k) acc[u][k] = (AT)0;
      }
    }
    __syncthreads();
  }
  __syncthreads();
  for (int e = threadIdx.x; e < IR; e += kThreads) {
    const int i3 = e / R, r = e - (e / R) * R;
    double v = 0.0;
    for (int g = 0; g < wpu; ++g) v += Ms[g * IR + r * I3 + i3];
    out[e] = v;
  }
}

// Rows of M^(1) from Y = T x_3 (.): out[i1][r] = sum_{i2} Y[(i1 I2 + i2) ys + c0 + r] B[i2][r]
// for the CTA's rows i1 (and the same for the D columns at c0 + R with dv).
template <typename AT>
__device__ void contract_m1(const AT* __restrict__ Y, int ys, int c0, int I1, int I2, int R,
                            const double* __restrict__ B, double* __restrict__ out, int rk, int C) {
  const int lo = lo_of(I1, rk, C), hi = lo_of(I1, rk + 1, C);
  for (int e = threadIdx.x; e < (hi - lo) * R; e += kThreads) {
    const int i1 = lo + e / R, r = e - (e / R) * R;
    const AT* y = Y + (size_t)i1 * I2 * ys + c0 + r;
    AT s = (AT)0;
    for (int i2 = 0; i2 < I2; ++i2) s = fmat(y[(size_t)i2 * ys], (AT)B[(size_t)i2 * R + r], s);
    out[(size_t)i1 * R + r] = (double)s;
  }
}

// Rows of M^(2) from Y: out[i2][r] = sum_{i1} Y[(i1 I2 + i2) ys + c0 + r] A[i1][r]
// for the CTA's rows i2.
template <typename AT>
__device__ void contract_m2(const AT* __restrict__ Y, int ys, int c0, int I1, int I2, int R,
                            const double* __restrict__ A, double* __restrict__ out, int rk, int C) {
  const int lo = lo_of(I2, rk, C), hi = lo_of(I2, rk + 1, C);
  for (int e = threadIdx.x; e < (hi - lo) * R; e += kThreads) {
    const int i2 = lo + e / R, r = e - (e / R) * R;
    const AT* y = Y + (size_t)i2 * ys + c0 + r;
    AT s = (AT)0;
    for (int i1 = 0; i1 < I1; ++i1) s = fmat(y[(size_t)i1 * I2 * ys], (AT)A[(size_t)i1 * R + r], s);
    out[(size_t)i2 * R + r] = (double)s;
  }
}

// The line search's variants of modes 1 and 2 from Z = T x_3 [Abar^(3) | D^(3)]
// (row stride 2R): V1[v][i1][r], v = 2 c + b, sums over i2 of Z_c B_b with
// B_0 = Abar^(2), B_1 = D^(2); V2[v][i2][r], v = 2 c + a, sums over i1 of
// Z_c A_a with A_0 = Abar^(1), A_1 = D^(1) (c = 0: Abar^(3) columns, 1: D^(3)).
template <typename AT>
__device__ void contract_variants(const AT* __restrict__ Z, int I1, int I2, int R, const double* __restrict__ Ab1,
                                  const double* __restrict__ D1, const double* __restrict__ Ab2,
                                  const double* __restrict__ D2, double* __restrict__ V1, double* __restrict__ V2,
                                  int rk, int C) {
  const int zs = 2 * R;
  {
    const int lo = lo_of(I1, rk, C), hi = lo_of(I1, rk + 1, C);
    for (int e = threadIdx.x; e < (hi - lo) * R; e += kThreads) {
      const int i1 = lo + e / R, r = e - (e / R) * R;
      const AT* z = Z + (size_t)i1 * I2 * zs + r;
      AT s00 = 0, s01 = 0, s10 = 0, s11 = 0;
      for (int i2 = 0; i2 < I2; ++i2) {
        const AT za = z[(size_t)i2 * zs], zd = z[(size_t)i2 * zs + R];
        const AT ba = (AT)Ab2[(size_t)i2 * R + r], bd = (AT)D2[(size_t)i2 * R + r];
        s00 = fmat(za, ba, s00);
        s01 = fmat(za, bd, s01);
        s10 = fmat(zd, ba, s10);
        s11 = fmat(zd, bd, s11);
      }
      const size_t o = (size_t)i1 * R + r, st = (size_t)I1 * R;
      V1[o] = (double)s00;
      V1[st + o] = (double)s01;
      V1[2 * st + o] = (double)s10;
      V1[3 * st + o] = (double)s11;
    }
  }
  {
    const int lo = lo_of(I2, rk, C), hi = lo_of(I2, rk + 1, C);
    for (int e = threadIdx.x; e < (hi - lo) * R; e += kThreads) {
      const int i2 = lo + e / R, r = e - (e / R) * R;
      const AT* z = Z + (size_t)i2 * zs + r;
      AT s00 = 0, s01 = 0, s10 = 0, s11 = 0;
      for (int i1 = 0; i1 < I1; ++i1) {
        const AT za = z[(size_t)i1 * I2 * zs], zd = z[(size_t)i1 * I2 * zs + R];
        const AT aa = (AT)Ab1[(size_t)i1 * R + r], ad = (AT)D1[(size_t)i1 * R + r];
        s00 = fmat(za, aa, s00);
        s01 = fmat(za, ad, s01);
        s10 = fmat(zd, aa, s10);
        s11 = fmat(zd, ad, s11);
      }
      const size_t o = (size_t)i2 * R + r, st = (size_t)I2 * R;
      V2[o] = (double)s00;
      V2[st + o] = (double)s01;
      V2[2 * st + o] = (double)s10;
      V2[3 * st + o] = (double)s11;
    }
  }
}

// ------------------------------------------------------------ FP64 helpers

// Partial X^T Y over rows [lo, hi) of two I x R row-major matrices.  For
// R^2 below the block size and long row ranges the rows are dealt
// round-robin to up to kThreads / R^2 thread groups of at least 16 rows
// each (shorter dependent FMA chains) whose sums are added in group order
// through gp (kThreads doubles of shared memory).
__device__ void gram_part(const double* __restrict__ X, const double* __restrict__ Yv, int lo, int hi, int R,
                          double* __restrict__ out, double* gp) {
  const int RR = R * R;
  const int G = min(RR < kThreads ? kThreads / RR : 1, (hi - lo) / 16);
  if (G <= 1) {
    for (int e = threadIdx.x; e < RR; e += kThreads) {
      const int r = e / R, s = e - (e / R) * R;
      double acc = 0.0;
      for (int i = lo; i < hi; ++i) acc = fma(X[(size_t)i * R + r], Yv[(size_t)i * R + s], acc);
      out[e] = acc;
    }
    return;
  }
  const int t = threadIdx.x;
  double acc = 0.0;
  if (t < G * RR) {
    const int g = t / RR, e = t - (t / RR) * RR;
    const int r = e / R, s = e - (e / R) * R;
    for (int i = lo + g; i < hi; i += G) acc = fma(X[(size_t)i * R + r], Yv[(size_t)i * R + s], acc);
  }
  __syncthreads();
  gp[t] = acc;
  __syncthreads();
  for (int e = t; e < RR; e += kThreads) {
    double v = 0.0;
    for (int g = 0; g < G; ++g) v += gp[g * RR + e];
    out[e] = v;
  }
  __syncthreads();
}

// In-place inverse of the SPD matrix A (R x R, shared) by Gauss-Jordan
// elimination without pivoting; false (the same in every thread) when a
// pivot is not positive and finite.
__device__ bool spd_inverse(double* A, int R) {
  for (int k = 0; k < R; ++k) {
    __syncthreads();
    const double p = A[k * R + k];
    if (!(p > 0.0) || !isfinite(p)) return false;
    const double ip = recip_nr(p);
    constexpr int kPer = kMaxR * kMaxR / kThreads;
    double v[kPer];
#pragma unroll
    for (int c = 0; c < kPer; ++c) {
      const int e = threadIdx.x + c * kThreads;
      double a = 0.0;
      if (e < R * R) {
        const int i = e / R, j = e - (e / R) * R;
        a = A[e];
        if (i == k && j == k)
          a = ip;
        else if (i == k)
          a *= ip;
        else if (j == k)
          a = -a * ip;
        else
          a = fma(-A[i * R + k] * ip, A[k * R + j], a);
      }
      v[c] = a;
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < kPer; ++c) {
      const int e = threadIdx.x + c * kThreads;
      if (e < R * R) A[e] = v[c];
    }
  }
  __syncthreads();
  return true;
}

// sh.A <- inverse of sh.A0 (Gammabar), retrying once with the ridge
// 1e-12 trace / R (the reading of the ALS mode solve used throughout).
__device__ bool gammabar_inverse(int R, EngSh& sh) {
  __syncthreads();
  for (int e = threadIdx.x; e < R * R; e += kThreads) sh.A[e] = sh.A0[e];
  if (spd_inverse(sh.A, R)) return true;
  double tr = 0.0;
  for (int r = 0; r < R; ++r) tr += sh.A0[r * R + r];
  const double ridge = 1e-12 * tr / R;
  __syncthreads();
  for (int e = threadIdx.x; e < R * R; e += kThreads) {
    const int i = e / R, j = e - (e / R) * R;
    sh.A[e] = sh.A0[e] + (i == j ? ridge : 0.0);
  }
  return spd_inverse(sh.A, R);
}

// sh.A0 = Ga o Gb (Hadamard product of two R x R Grams).
__device__ void hadamard_into(const double* Ga, const double* Gb, int R, double* out) {
  __syncthreads();
  for (int e = threadIdx.x; e < R * R; e += kThreads) out[e] = Ga[e] * Gb[e];
  __syncthreads();
}

// Normalisation scales and term order (Section 2.3) from the column sums of
// squares s[n R + r] of the three factors: nu = ||a_r^(n)||, lambda_r =
// prod_n nu, scale = lambda^(1/3) / nu (1 for a term with a zero column),
// order = stable sort by decreasing lambda (NaN last).
__device__ void norm_scales(const double* s, int R, EngSh& sh, double* scale, int* order) {
  __syncthreads();
  for (int t = threadIdx.x; t < 3 * R; t += kThreads) {
    const double v = s[t];
    const double y = v > 0.0 ? rsqrt_nr(v) : 0.0;
    sh.nu[t] = v * y;
    scale[t] = y;
  }
  __syncthreads();
  for (int r = threadIdx.x; r < R; r += kThreads) {
    double l = 1.0;
    bool zero = false;
    for (int n = 0; n < 3; ++n) {
      l *= sh.nu[n * R + r];
      if (sh.nu[n * R + r] == 0.0) zero = true;
    }
    if (zero) l = 0.0;
    const double root = cbrt(l);
    for (int n = 0; n < 3; ++n) scale[n * R + r] = zero ? 1.0 : root * scale[n * R + r];
    sh.lam[r] = l;
    sh.key[r] = isnan(l) ? -INFINITY : l;
  }
  __syncthreads();
  for (int r = threadIdx.x; r < R; r += kThreads) {
    int rank = 0;
    for (int q = 0; q < R; ++q)
      if (sh.key[q] > sh.key[r] || (sh.key[q] == sh.key[r] && q < r)) ++rank;
    order[rank] = r;
  }
  __syncthreads();
}

// Grams of the normalised point: out_n[p][q] = G_n[o_p][o_q] s_n[o_p] s_n[o_q].
__device__ void grams_normalised(const double* G, int R, const double* scale, const int* order, double* out) {
  for (int e = threadIdx.x; e < 3 * R * R; e += kThreads) {
    const int n = e / (R * R), pq = e - n * R * R;
    const int p = pq / R, q = pq - (pq / R) * R;
    const int op = order[p], oq = order[q];
    out[e] = G[(size_t)n * R * R + op * R + oq] * scale[n * R + op] * scale[n * R + oq];
  }
}

// sum_{r,s} prod_n G_n[r][s] = ||[[A]]||^2 (Eq. fA), by the whole CTA.
__device__ double model_norm2(const double* G, int R, EngSh& sh) {
  double part = 0.0;
  for (int e = threadIdx.x; e < R * R; e += kThreads)
    part += G[e] * G[(size_t)R * R + e] * G[2 * (size_t)R * R + e];
  return cta_sum(part, sh);
}

// Cholesky solve of (H + delta I) alpha = rhs in shared memory by warp 0
// (m <= 32): the N-GMRES normal equations (Eq. normal with delta I).  alpha
// = 0 when max diag H = 0.
__device__ void window_solve(int m, double eps, EngSh& sh) {
  __syncthreads();
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    double dmax = 0.0;
    for (int j = 0; j < m; ++j) dmax = fmax(dmax, sh.H[j * kHLd + j]);
    if (dmax == 0.0) {
      if (lane < m) sh.alpha[lane] = 0.0;
    } else {
      const double delta = eps * dmax;
      if (lane < m) sh.H[lane * kHLd + lane] += delta;
      __syncwarp();
      // right-looking Cholesky, lower triangle in place (lane = row)
      // (Newton-refined square roots and reciprocals: each IEEE FP64 divide
      // or sqrt is a serial chain of ~650 cycles in this one-warp solve)
      for (int k = 0; k < m; ++k) {
        // 1/sqrt first: the pivot and its reciprocal from one Newton chain
        const double hk = sh.H[k * kHLd + k];
        const double idk = rsqrt_nr(hk);   // NaN for a pivot <= 0 (not positive definite)
        const double dk = hk * idk;
        __syncwarp();
        if (lane == k) {
          sh.H[k * kHLd + k] = dk;
          sh.sc2[k] = idk;
        }
        if (lane > k && lane < m) sh.H[lane * kHLd + k] *= idk;
        __syncwarp();
        if (lane > k && lane < m) {
          const double lk = sh.H[lane * kHLd + k];
          for (int j = k + 1; j <= lane; ++j) sh.H[lane * kHLd + j] -= lk * sh.H[j * kHLd + k];
        }
        __syncwarp();
      }
      // L y = rhs, then L^T alpha = y
      double y = lane < m ? sh.rhs[lane] : 0.0;
      for (int k = 0; k < m; ++k) {
        const double yk = __shfl_sync(0xffffffffu, y, k) * sh.sc2[k];
        if (lane == k) y = yk;
        if (lane > k && lane < m) y -= sh.H[lane * kHLd + k] * yk;
      }
      double a = y;
      for (int k = m - 1; k >= 0; --k) {
        const double ak = __shfl_sync(0xffffffffu, a, k) * sh.sc2[k];
        if (lane == k) a = ak;
        if (lane < k) a -= sh.H[k * kHLd + lane] * ak;
      }
      if (lane < m) sh.alpha[lane] = a;
    }
  }
  __syncthreads();
}

// Window ring slot of window row j (oldest first).
__device__ __forceinline__ int ring(int start, int j, int w) { return (start + j) % w; }

// ------------------------------------------------------------ request steps

struct Rows {
  int lo[3], hi[3], off[3], I[3];
};

__device__ __forceinline__ Rows rows_of(const ManyReq& q, int rk, int C) {
  Rows w;
  w.I[0] = q.I1;
  w.I[1] = q.I2;
  w.I[2] = q.I3;
  w.off[0] = 0;
  w.off[1] = q.off2;
  w.off[2] = q.off3;
  for (int n = 0; n < 3; ++n) {
    w.lo[n] = lo_of(w.I[n], rk, C);
    w.hi[n] = lo_of(w.I[n], rk + 1, C);
  }
  return w;
}

// f(e, n, i, r) for the CTA's elements of an iterate (its rows of every mode).
template <class F>
__device__ __forceinline__ void for_own(const Rows& w, int R, F f) {
  for (int n = 0; n < 3; ++n) {
    const int cnt = (w.hi[n] - w.lo[n]) * R;
    for (int k = threadIdx.x; k < cnt; k += kThreads) {
      const int i = w.lo[n] + k / R, r = k - (k / R) * R;
      f(w.off[n] + i * R + r, n, i, r);
    }
  }
}

// Shared memory of the passes (the large region):
// Y = T x_3 B: the factor columns (kMaxI x kBsCols) and two staging tiles
// (256 fibers x (kIC + 1) elements of T); M^(3): two chunks of rows of T
// (kTF rows of the longest side each, more rows of shorter ones), the
// Khatri-Rao rows, the FP64 totals.
constexpr size_t kBsBytes = (size_t)kMaxI * kBsCols * sizeof(double);
constexpr size_t kTstBytes = 2 * (size_t)kThreads * (Stage<double>::kIC + 1) * sizeof(double) + 256;

// T x_3 A into the Y buffer: row stride ys, columns c0 .. c0 + R - 1.
template <typename AT>
__device__ void do_pass_y(const ManyReq& q, const double* A, int ys, int c0, int rk, int C, char* big) {
  AT* Bs = (AT*)big;
  AT* Y = (AT*)q.Y + c0;
  if (q.t64)
    pass_y<double, AT>((const double*)q.T, q.J, q.I3, q.R, A, nullptr, Y, ys, rk, C, Bs, (double*)(big + kBsBytes));
  else
    pass_y<float, AT>((const float*)q.T, q.J, q.I3, q.R, A, nullptr, Y, ys, rk, C, Bs, (float*)(big + kBsBytes));
}

template <typename AT>
__device__ void do_pass_m3(const ManyReq& q, const double* A, const double* B, double* out, int rk, int C,
                           char* big) {
  AT* KRs = (AT*)(big + kTchBytes);
  double* Ms = (double*)(big + kTchBytes + kKRBytes);
  if (q.t64)
    pass_m3<double, AT>((const double*)q.T, q.J, q.I2, q.I3, q.R, A, B, out, rk, C, (double*)big, KRs, Ms);
  else
    pass_m3<float, AT>((const float*)q.T, q.J, q.I2, q.I3, q.R, A, B, out, rk, C, (float*)big, KRs, Ms);
}

// Gradient rows G^(n) = -M^(n) + A^(n) Gammabar^(n) (Eq. Gn) of the CTA's
// rows, Gammabar^(n) from the Grams G (3 x R x R) of the point v.
__device__ void grad_rows(const ManyReq& q, const Rows& w, const double* v, const double* G, const double* M1,
                          const double* M2, const double* M3, double* g, EngSh& sh) {
  const int R = q.R, RR = R * R;
  for (int n = 0; n < 3; ++n) {
    hadamard_into(G + (size_t)((n + 1) % 3) * RR, G + (size_t)((n + 2) % 3) * RR, R, sh.A0);
    const double* Mn = n == 0 ? M1 : n == 1 ? M2 : M3;
    const int cnt = (w.hi[n] - w.lo[n]) * R;
    for (int k = threadIdx.x; k < cnt; k += kThreads) {
      const int i = w.lo[n] + k / R, r = k - (k / R) * R;
      const double* a = v + w.off[n] + (size_t)i * R;
      double s = -Mn[(size_t)i * R + r];
      for (int kk = 0; kk < R; ++kk) s = fma(a[kk], sh.A0[kk * R + r], s);
      g[w.off[n] + (size_t)i * R + r] = s;
    }
  }
  __syncthreads();
}

// ALS update of the CTA's rows of mode n: dst rows = M rows Gammabar^-1 (sh.A).
__device__ void als_rows(const double* M, int R, int lo, int hi, double* dst, const EngSh& sh) {
  __syncthreads();
  for (int k = threadIdx.x; k < (hi - lo) * R; k += kThreads) {
    const int i = lo + k / R, r = k - (k / R) * R;
    const double* m = M + (size_t)i * R;
    double s = 0.0;
    for (int kk = 0; kk < R; ++kk) s = fma(m[kk], sh.A[kk * R + r], s);
    dst[(size_t)i * R + r] = s;
  }
  __syncthreads();
}

// Push the CTA's elements of (u, g) into the window (slot 0 after a reset)
// and return its partial of ||g||^2.
__device__ double window_push(const ManyReq& q, const Rows& w, const double* u, const double* g, int slot) {
  double part = 0.0;
  double* Us = q.U + (size_t)slot * q.P;
  double* Gs_ = q.G + (size_t)slot * q.P;
  for_own(w, q.R, [&](int e, int, int, int) {
    const double gv = g[e];
    Us[e] = u[e];
    Gs_[e] = gv;
    part = fma(gv, gv, part);
  });
  return part;
}

__device__ __forceinline__ int push_slot(const ManyCtl& c, int w, bool reset) {
  if (reset) return 0;
  return c.win_m < w ? (c.win_start + c.win_m) % w : c.win_start;
}

enum TailKind { T_BEGIN = 0, T_ACCEPT = 1, T_KEEP = 2 };

// End of a phase start or an iteration: ||g||, f, window bookkeeping,
// counters and the stopping test (the same in every CTA), the park
// decision (CTA 0's clock), the control block to global memory.  The
// partials of ||g||^2 (and of <A^(3), M^(3)> for T_BEGIN / T_ACCEPT) are in
// the scalar region A, slots 2 and 1.  Returns true when the cluster leaves
// this request (finished or parked).
__device__ bool tail(EngSh& sh, int rk, int C, int kind, bool reset, unsigned long long t0,
                     unsigned long long budget) {
  const ManyReq& q = sh.q;
  const int SCA = 2 * q.big_ld;
  if (rk == 0 && threadIdx.x == 0) q.scal[S_PARK] = (gtimer() - t0 > budget) ? 1.0 : 0.0;
  cl_sync();
  const double gg = psum(q.part + SCA + 2, q.part_ld, C, 0);
  double f;
  if (kind == T_KEEP) {
    f = sh.bcast[0];
  } else {
    const double inner = psum(q.part + SCA + 1, q.part_ld, C, 0);
    const double model = model_norm2(kind == T_ACCEPT ? q.Gx : q.Gu, q.R, sh);
    f = 0.5 * (q.normT2 - 2.0 * inner + model);
  }
  const bool park = q.scal[S_PARK] != 0.0;
  __syncthreads();
  if (threadIdx.x == 0) {
    ManyCtl& c = sh.c;
    const bool mixed = c.phase == PH_MIXED;
    if (reset) {
      c.win_start = 0;
      c.win_m = 1;
    } else if (c.win_m < q.w) {
      c.win_m += 1;
    } else {
      c.win_start = (c.win_start + 1) % q.w;
    }
    if (kind == T_BEGIN) {
      c.best = INFINITY;
      c.since_best = 0;
      c.fg_evals += 1;
      c.start = 0;
    } else {
      c.iters += 1;
      if (mixed)
        c.mixed_iters += 1;
      else
        c.fp64_iters += 1;
    }
    const double gn = sqrt(gg) / q.P;
    c.gn = gn;
    c.f = f;
    int stop = STOP_RUN;
    if (!isfinite(gn))
      stop = STOP_NONFINITE;
    else if (gn < (mixed ? q.tol_mixed : q.tol))
      stop = STOP_TOL;
    else if (c.iters >= q.maxit)
      stop = STOP_MAXIT;
    else if (mixed) {
      if (gn < c.best) {
        c.best = gn;
        c.since_best = 0;
      } else if (++c.since_best >= q.stall) {
        stop = STOP_STALL;
      }
    }
    c.stop = stop;
    if (stop != STOP_RUN) {
      if (mixed && q.polish && (stop == STOP_TOL || stop == STOP_STALL)) {
        c.phase = PH_FP64;
        c.start = 1;
      } else {
        c.phase = PH_DONE;
        if (stop == STOP_NONFINITE) c.status = CP_ERR_NONFINITE;
      }
    }
    if (rk == 0) {
      *q.ctl = c;
      q.scal[S_F] = f;
    }
  }
  __syncthreads();
  return sh.c.phase == PH_DONE || park;
}

// Phase start: (start == 2) u = normalise(x), x holding the initial guess
// (R5 of the readings: the solve starts from the normalised guess); f and g
// at u in this phase's precision; the window becomes {(u, g)}.
template <typename AT>
__device__ bool run_start(EngSh& sh, char* big, int rk, int C, unsigned long long t0, unsigned long long budget) {
  const ManyReq& q = sh.q;
  const int R = q.R, RR = R * R, ld = q.part_ld;
  const int BA = 0, BB = q.big_ld, SCA = 2 * q.big_ld;
  double* my = q.part + (size_t)rk * ld;
  const Rows w = rows_of(q, rk, C);
  if (sh.c.start == 2) {
    for (int n = 0; n < 3; ++n) gram_part(q.x + w.off[n], q.x + w.off[n], w.lo[n], w.hi[n], R, my + BA + n * RR, sh.gp);
    cl_sync();
    for (int t = threadIdx.x; t < 3 * R; t += kThreads) {
      const int n = t / R, r = t - (t / R) * R;
      sh.sc2[t] = psum(q.part + BA, ld, C, n * RR + r * R + r);
    }
    norm_scales(sh.sc2, R, sh, sh.scale, sh.order);
    for_own(w, R, [&](int e, int n, int i, int r) {
      const int o = sh.order[r];
      q.u[e] = q.x[w.off[n] + (size_t)i * R + o] * sh.scale[n * R + o];
    });
    if (rk == 0) {
      for (int e = threadIdx.x; e < 3 * RR; e += kThreads) q.Gx[e] = psum(q.part + BA, ld, C, e);
      __syncthreads();
      grams_normalised(q.Gx, R, sh.scale, sh.order, q.Gu);
    }
    cl_sync();
  }
  const double* u = q.u;
  do_pass_y<AT>(q, u + q.off3, R, 0, rk, C, big);
  cl_sync();
  contract_m1<AT>((const AT*)q.Y, R, 0, q.I1, q.I2, R, u + q.off2, q.M1, rk, C);
  contract_m2<AT>((const AT*)q.Y, R, 0, q.I1, q.I2, R, u, q.M2, rk, C);
  do_pass_m3<AT>(q, u, u + q.off2, my + BB, rk, C, big);
  cl_sync();
  double inner = 0.0;
  for (int k = threadIdx.x; k < (w.hi[2] - w.lo[2]) * R; k += kThreads) {
    const int e = w.lo[2] * R + k;
    const double m = psum(q.part + BB, ld, C, e);
    q.M3[e] = m;
    inner = fma(u[q.off3 + e], m, inner);
  }
  inner = cta_sum(inner, sh);
  grad_rows(q, w, u, q.Gu, q.M1, q.M2, q.M3, q.g, sh);
  const double gpart = cta_sum(window_push(q, w, u, q.g, 0), sh);
  if (threadIdx.x == 0) {
    my[SCA + 1] = inner;
    my[SCA + 2] = gpart;
    sh.c.ysrc = 1;
  }
  return tail(sh, rk, C, T_BEGIN, true, t0, budget);
}

// The "keep" ends of an iteration: after a restart (reset) or a search that
// found no acceptable step, u = ubar with its f, g and Grams.
__device__ bool keep_ubar(EngSh& sh, int rk, int C, bool reset, int ysrc, unsigned long long t0,
                          unsigned long long budget) {
  const ManyReq& q = sh.q;
  const Rows w = rows_of(q, rk, C);
  if (threadIdx.x == 0) sh.c.ysrc = ysrc;
  for_own(w, q.R, [&](int e, int, int, int) {
    q.u[e] = q.ub[e];
    q.g[e] = q.gb[e];
  });
  if (rk == 0)
    for (int e = threadIdx.x; e < 3 * q.R * q.R; e += kThreads) q.Gu[e] = q.Gb[e];
  __syncthreads();
  const double gpart = cta_sum(window_push(q, w, q.u, q.g, push_slot(sh.c, q.w, reset)), sh);
  if (threadIdx.x == 0) q.part[(size_t)rk * q.part_ld + 2 * q.big_ld + 2] = gpart;
  return tail(sh, rk, C, T_KEEP, reset, t0, budget);
}

// One iteration of Algorithm 1 from u (with g(u), Grams of u, window).
template <typename AT>
__device__ bool run_iter(EngSh& sh, char* big, int rk, int C, unsigned long long t0, unsigned long long budget) {
  const ManyReq& q = sh.q;
  const int R = q.R, RR = R * R, ld = q.part_ld;
  const int BA = 0, BB = q.big_ld, SCA = 2 * q.big_ld, SCB = SCA + 128;
  double* my = q.part + (size_t)rk * ld;
  const Rows w = rows_of(q, rk, C);
  const double* u = q.u;
  double* sw = q.uh;   // the swept point (unnormalised), later uhat
  auto fail_spd = [&]() {
    if (threadIdx.x == 0) {
      sh.c.status = CP_ERR_NOT_SPD;
      sh.c.phase = PH_DONE;
      if (rk == 0) *q.ctl = sh.c;
    }
    __syncthreads();
    return true;
  };

  // ---- Step I: the ALS sweep (Section 2.3), modes 1 and 2 from Y = T x_3 A^(3)
  // (kept from the previous iteration when it made u: see ysrc)
  const int ysrc = sh.c.ysrc;
  const AT* Ysw = ysrc == 2 ? (const AT*)q.Y2 : (const AT*)q.Y;
  const int ysw = ysrc == 3 ? 2 * R : R;
  if (ysrc == 0) {
    do_pass_y<AT>(q, u + q.off3, R, 0, rk, C, big);
    cl_sync();
  }
  hadamard_into(q.Gu + RR, q.Gu + 2 * RR, R, sh.A0);
  if (!gammabar_inverse(R, sh)) return fail_spd();
  contract_m1<AT>(Ysw, ysw, 0, q.I1, q.I2, R, u + q.off2, q.M1, rk, C);
  als_rows(q.M1, R, w.lo[0], w.hi[0], sw, sh);
  gram_part(sw, sw, w.lo[0], w.hi[0], R, my + BA, sh.gp);
  cl_sync();
  __syncthreads();
  for (int e = threadIdx.x; e < RR; e += kThreads) {
    const double g1 = psum(q.part + BA, ld, C, e);
    sh.A0[e] = g1 * q.Gu[2 * RR + e];
    if (rk == 0) q.Gs[e] = g1;
  }
  if (!gammabar_inverse(R, sh)) return fail_spd();
  contract_m2<AT>(Ysw, ysw, 0, q.I1, q.I2, R, sw, q.M2, rk, C);
  als_rows(q.M2, R, w.lo[1], w.hi[1], sw + q.off2, sh);
  gram_part(sw + q.off2, sw + q.off2, w.lo[1], w.hi[1], R, my + BB, sh.gp);
  cl_sync();
  if (rk == 0)
    for (int e = threadIdx.x; e < RR; e += kThreads) q.Gs[RR + e] = psum(q.part + BB, ld, C, e);
  do_pass_m3<AT>(q, sw, sw + q.off2, my + BA, rk, C, big);
  cl_sync();
  for (int k = threadIdx.x; k < (w.hi[2] - w.lo[2]) * R; k += kThreads) {
    const int e = w.lo[2] * R + k;
    q.M3s[e] = psum(q.part + BA, ld, C, e);
  }
  hadamard_into(q.Gs, q.Gs + RR, R, sh.A0);
  if (!gammabar_inverse(R, sh)) return fail_spd();
  als_rows(q.M3s, R, w.lo[2], w.hi[2], sw + q.off3, sh);
  gram_part(sw + q.off3, sw + q.off3, w.lo[2], w.hi[2], R, my + BB, sh.gp);
  cl_sync();

  // ---- ubar = normalise(swept) (R3, R4); its Grams and M^(3) follow
  for (int t = threadIdx.x; t < 3 * R; t += kThreads) {
    const int n = t / R, r = t - (t / R) * R;
    sh.sc2[t] = n < 2 ? q.Gs[(size_t)n * RR + r * R + r] : psum(q.part + BB, ld, C, r * R + r);
  }
  norm_scales(sh.sc2, R, sh, sh.scale, sh.order);
  if (rk == 0) {
    for (int e = threadIdx.x; e < RR; e += kThreads) q.Gs[2 * RR + e] = psum(q.part + BB, ld, C, e);
    __syncthreads();
    grams_normalised(q.Gs, R, sh.scale, sh.order, q.Gb);
  }
  for_own(w, R, [&](int e, int n, int i, int r) {
    const int o = sh.order[r];
    q.ub[e] = sw[w.off[n] + (size_t)i * R + o] * sh.scale[n * R + o];
  });
  for (int k = threadIdx.x; k < (w.hi[2] - w.lo[2]) * R; k += kThreads) {
    const int i = w.lo[2] + k / R, p = k - (k / R) * R;
    const int o = sh.order[p];
    q.M3[(size_t)i * R + p] = q.M3s[(size_t)i * R + o] * sh.scale[o] * sh.scale[R + o];
  }
  cl_sync();

  // ---- f and g at ubar: modes 1 and 2 from Y' = T x_3 Abar^(3), kept in
  // the first R columns of Y (row stride 2R) for the line search's Z
  const double* ub = q.ub;
  do_pass_y<AT>(q, ub + q.off3, 2 * R, 0, rk, C, big);
  cl_sync();
  contract_m1<AT>((const AT*)q.Y, 2 * R, 0, q.I1, q.I2, R, ub + q.off2, q.M1, rk, C);
  contract_m2<AT>((const AT*)q.Y, 2 * R, 0, q.I1, q.I2, R, ub, q.M2, rk, C);
  __syncthreads();
  grad_rows(q, w, ub, q.Gb, q.M1, q.M2, q.M3, q.gb, sh);
  {
    double inner = 0.0;
    for (int k = threadIdx.x; k < (w.hi[2] - w.lo[2]) * R; k += kThreads) {
      const int e = w.lo[2] * R + k;
      inner = fma(ub[q.off3 + e], q.M3[e], inner);
    }
    inner = cta_sum(inner, sh);
    if (threadIdx.x == 0) my[SCA] = inner;
  }

  // ---- Step II: window dots over the CTA's elements (p_j = gbar - g_j).
  // The FP64 phase forms P^T P and P^T gbar directly.  The mixed phase keeps
  // the window Gram K_jl = g_j^T g_l between iterations and forms only
  // c_j = gbar^T g_j, gbar^T gbar and the newest entry's row of K (2m + 1
  // dots instead of m(m + 3)/2); then (P^T P)_jl = gbar^T gbar - c_j - c_l
  // + K_jl.  The cancellation in that sum costs about u |g|^2 / |p|^2 of
  // relative accuracy, far below the FP32-level error of the mixed phase's
  // gradients.
  constexpr bool kGramKept = sizeof(AT) == sizeof(float);
  const int m = sh.c.win_m, wstart = sh.c.win_start;
  const int npairs = m * (m + 1) / 2, ntask = npairs + m;
  if (kGramKept) {
    // task t < m: gbar . g_t; t = m: gbar . gbar; m < t <= 2m: g_{m-1} . g_{t-m-1}.
    // Each task's elements are split over S threads (k = s, s + S, ...),
    // whose sums are added in order at the end.
    double* tile = (double*)big;                 // m x kTileLd, then gbar
    double* gt = tile + (size_t)kMaxW * kTileLd;
    const int nt = 2 * m + 1;
    const int S = kThreads / nt;
    const int t = threadIdx.x;
    const int task = t / S, sidx = t - (t / S) * S;
    int ta = -1, tb = -1;                        // tile rows; m is gbar
    if (task < m) {
      ta = m;
      tb = task;
    } else if (task == m) {
      ta = m;
      tb = m;
    } else if (task < nt) {
      ta = m - 1;
      tb = task - m - 1;
    }
    double acc = 0.0;
    for (int n = 0; n < 3; ++n) {
      const int e_lo = w.off[n] + w.lo[n] * R, e_hi = w.off[n] + w.hi[n] * R;
      for (int e0 = e_lo; e0 < e_hi; e0 += kTile) {
        const int ne = min(kTile, e_hi - e0);
        __syncthreads();
        for (int x = threadIdx.x; x < m * kTile; x += kThreads) {
          const int j = x / kTile, k = x - (x / kTile) * kTile;
          tile[j * kTileLd + k] = k < ne ? q.G[(size_t)ring(wstart, j, q.w) * q.P + e0 + k] : 0.0;
        }
        for (int k = threadIdx.x; k < kTile; k += kThreads) gt[k] = k < ne ? q.gb[e0 + k] : 0.0;
        __syncthreads();
        if (ta >= 0) {
          const double* a = ta == m ? gt : tile + ta * kTileLd;
          const double* b = tb == m ? gt : tile + tb * kTileLd;
          double v = acc;
          for (int k = sidx; k < ne; k += S) v = fma(a[k], b[k], v);
          acc = v;
        }
      }
    }
    __syncthreads();
    sh.gp[t] = acc;
    __syncthreads();
    for (int k = threadIdx.x; k < nt; k += kThreads) {
      double v = 0.0;
      for (int s2 = 0; s2 < S; ++s2) v += sh.gp[k * S + s2];
      my[BA + k] = v;
    }
  } else {
    double* tile = (double*)big;                 // m x kTileLd, then gbar
    double* gt = tile + (size_t)kMaxW * kTileLd;
    double acc[3] = {0.0, 0.0, 0.0};
    int ta[3], tb[3];
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      const int t = threadIdx.x + s * kThreads;
      ta[s] = -1;
      tb[s] = -1;
      if (t < npairs) {
        int j = 0, rem = t;
        while (rem >= m - j) {
          rem -= m - j;
          ++j;
        }
        ta[s] = j;
        tb[s] = j + rem;
      } else if (t < ntask) {
        ta[s] = t - npairs;   // rhs_j: against gbar
        tb[s] = -2;
      }
    }
    for (int n = 0; n < 3; ++n) {
      const int e_lo = w.off[n] + w.lo[n] * R, e_hi = w.off[n] + w.hi[n] * R;
      for (int e0 = e_lo; e0 < e_hi; e0 += kTile) {
        const int ne = min(kTile, e_hi - e0);
        __syncthreads();
        for (int x = threadIdx.x; x < m * kTile; x += kThreads) {
          const int j = x / kTile, k = x - (x / kTile) * kTile;
          double v = 0.0;
          if (k < ne) v = q.gb[e0 + k] - q.G[(size_t)ring(wstart, j, q.w) * q.P + e0 + k];
          tile[j * kTileLd + k] = v;
        }
        for (int k = threadIdx.x; k < kTile; k += kThreads) gt[k] = k < ne ? q.gb[e0 + k] : 0.0;
        __syncthreads();
#pragma unroll
        for (int s = 0; s < 3; ++s) {
          if (ta[s] >= 0) {
            const double* a = tile + ta[s] * kTileLd;
            const double* b = tb[s] == -2 ? gt : tile + tb[s] * kTileLd;
            double v = acc[s];
            for (int k = 0; k < ne; ++k) v = fma(a[k], b[k], v);
            acc[s] = v;
          }
        }
      }
    }
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      const int t = threadIdx.x + s * kThreads;
      if (t < ntask) my[BA + t] = t < npairs ? acc[s] : -acc[s];
    }
  }
  cl_sync();
  // f(ubar); the normal equations, solved in every CTA
  {
    const double inner = psum(q.part + SCA, ld, C, 0);
    const double model = model_norm2(q.Gb, R, sh);
    if (threadIdx.x == 0) sh.bcast[0] = 0.5 * (q.normT2 - 2.0 * inner + model);
  }
  if (kGramKept) {
    const double gg = psum(q.part + BA, ld, C, m);
    for (int t = threadIdx.x; t < ntask; t += kThreads) {
      if (t < npairs) {
        int j = 0, rem = t;
        while (rem >= m - j) {
          rem -= m - j;
          ++j;
        }
        const int l = j + rem;   // j <= l
        const double kjl = l == m - 1 ? psum(q.part + BA, ld, C, m + 1 + j)
                                      : q.K[(size_t)ring(wstart, j, q.w) * q.w + ring(wstart, l, q.w)];
        const double v = gg - psum(q.part + BA, ld, C, j) - psum(q.part + BA, ld, C, l) + kjl;
        sh.H[j * kHLd + l] = v;
        sh.H[l * kHLd + j] = v;
      } else {
        const int j = t - npairs;
        sh.rhs[j] = psum(q.part + BA, ld, C, j) - gg;
      }
    }
    if (rk == 0) {
      const int sn = ring(wstart, m - 1, q.w);
      for (int l = threadIdx.x; l < m; l += kThreads) {
        const int sl = ring(wstart, l, q.w);
        const double v = psum(q.part + BA, ld, C, m + 1 + l);
        q.K[(size_t)sn * q.w + sl] = v;
        q.K[(size_t)sl * q.w + sn] = v;
      }
    }
  } else {
    for (int t = threadIdx.x; t < ntask; t += kThreads) {
      const double v = psum(q.part + BA, ld, C, t);
      if (t < npairs) {
        int j = 0, rem = t;
        while (rem >= m - j) {
          rem -= m - j;
          ++j;
        }
        const int l = j + rem;
        sh.H[j * kHLd + l] = v;
        sh.H[l * kHLd + j] = v;
      } else {
        sh.rhs[t - npairs] = v;
      }
    }
  }
  window_solve(m, q.eps, sh);
  // uhat = ubar + sum_j alpha_j (ubar - u_j) (Eq. accel), and its column sums of squares
  {
    double cs = 0.0;
    const int tR = (int)threadIdx.x < 3 * R ? (int)threadIdx.x : -1;
    for_own(w, R, [&](int e, int, int, int) {
      const double b = ub[e];
      double acc = 0.0;
#pragma unroll 4
      for (int j = 0; j < m; ++j) acc += sh.alpha[j] * (b - q.U[(size_t)ring(wstart, j, q.w) * q.P + e]);
      sw[e] = b + acc;
    });
    __syncthreads();
    if (tR >= 0) {
      const int n = tR / R, r = tR - (tR / R) * R;
      for (int i = w.lo[n]; i < w.hi[n]; ++i) {
        const double v = sw[w.off[n] + (size_t)i * R + r];
        cs = fma(v, v, cs);
      }
      my[SCB + tR] = cs;
    }
  }
  cl_sync();
  // normalise uhat (R6); d = uhat - ubar, the slope g(ubar)^T d; the line
  // search's Grams ubar^T d and d^T d
  for (int t = threadIdx.x; t < 3 * R; t += kThreads) sh.sc2[t] = psum(q.part + SCB, ld, C, t);
  norm_scales(sh.sc2, R, sh, sh.scale, sh.order);
  {
    double sl = 0.0;
    for_own(w, R, [&](int e, int n, int i, int r) {
      const int o = sh.order[r];
      const double dv = sw[w.off[n] + (size_t)i * R + o] * sh.scale[n * R + o] - ub[e];
      q.d[e] = dv;
      sl = fma(q.gb[e], dv, sl);
    });
    sl = cta_sum(sl, sh);
    if (threadIdx.x == 0) my[SCA] = sl;
  }
  __syncthreads();
  for (int n = 0; n < 3; ++n) {
    gram_part(ub + w.off[n], q.d + w.off[n], w.lo[n], w.hi[n], R, my + BB + n * RR, sh.gp);
    gram_part(q.d + w.off[n], q.d + w.off[n], w.lo[n], w.hi[n], R, my + BB + (3 + n) * RR, sh.gp);
  }
  cl_sync();
  const double slope = psum(q.part + SCA, ld, C, 0);
  const bool restart = !(slope < 0.0);
  if (threadIdx.x == 0) {
    sh.c.als_sweeps += 1;
    sh.c.fg_evals += 1;
    if (restart) sh.c.restarts += 1;
  }
  __syncthreads();
  // (after a restart the Y buffer still holds Y' = T x_3 Abar^(3))
  if (restart) return keep_ubar(sh, rk, C, true, 3, t0, budget);   // R7

  // ---- Step III: the line polynomial phi(beta) = f(ubar + beta d)
  if (rk == 0)
    for (int e = threadIdx.x; e < 3 * RR; e += kThreads) {
      q.Gad[e] = psum(q.part + BB, ld, C, e);
      q.Gdd[e] = psum(q.part + BB, ld, C, 3 * RR + e);
    }
  // Z = T x_3 [Abar^(3) | D^(3)]: the D columns beside Y'
  do_pass_y<AT>(q, q.d + q.off3, 2 * R, R, rk, C, big);
  cl_sync();
  contract_variants<AT>((const AT*)q.Y, q.I1, q.I2, R, ub, q.d, ub + q.off2, q.d + q.off2, q.V1, q.V2, rk, C);
  __syncthreads();
  // <T, [[A_a, B_b, C_c]]> partials: sum over the CTA's rows of mode 1 of A_a V1[2c + b]
  {
    double s8[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const size_t st1 = (size_t)q.I1 * R;
    for (int k = threadIdx.x; k < (w.hi[0] - w.lo[0]) * R; k += kThreads) {
      const int e = w.lo[0] * R + k;
      const double fa = ub[e], fd = q.d[e];
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const double m = q.V1[v * st1 + e];
        s8[v] = fma(fa, m, s8[v]);
        s8[4 + v] = fma(fd, m, s8[4 + v]);
      }
    }
    cta_sums<8>(s8, sh);
    if (threadIdx.x == 0)
#pragma unroll
      for (int k = 0; k < 8; ++k) my[SCB + k] = s8[k];
  }
  cl_sync();
  if (rk == 0) {
    // E(beta) = ||[[ubar + beta d]]||^2 = sum_{r,s} prod_n (a_n + b_n beta + c_n beta^2)
    double e7[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int e = threadIdx.x; e < RR; e += kThreads) {
      const int r = e / R, s2 = e - (e / R) * R;
      double qd[3][3];
#pragma unroll
      for (int n = 0; n < 3; ++n) {
        qd[n][0] = q.Gb[(size_t)n * RR + e];
        qd[n][1] = q.Gad[(size_t)n * RR + e] + q.Gad[(size_t)n * RR + s2 * R + r];
        qd[n][2] = q.Gdd[(size_t)n * RR + e];
      }
      // the product of the three quadratics, coefficient by coefficient
      double p4[5] = {0, 0, 0, 0, 0};
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) p4[i + j] = fma(qd[0][i], qd[1][j], p4[i + j]);
      double p6[7] = {0, 0, 0, 0, 0, 0, 0};
#pragma unroll
      for (int i = 0; i < 5; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) p6[i + j] = fma(p4[i], qd[2][j], p6[i + j]);
#pragma unroll
      for (int k = 0; k < 7; ++k) e7[k] += p6[k];
    }
    cta_sums<7>(e7, sh);
    if (threadIdx.x == 0) {
      double poly[7];
      for (int k = 0; k < 7; ++k) poly[k] = 0.5 * e7[k];
#pragma unroll
      for (int k8 = 0; k8 < 8; ++k8) {
        const int a = k8 >> 2, v = k8 & 3;
        const int b = v & 1, c = v >> 1;
        poly[a + b + c] -= psum(q.part + SCB, ld, C, k8);
      }
      poly[0] += 0.5 * q.normT2;
      MTState st;
      mtdev::mt_init(st, poly[0], poly[1], sh.c.phase == PH_MIXED ? q.ls_mixed : q.ls);
      while (!st.done) {
        const double b = st.stp;
        double f = poly[6], g = 6.0 * poly[6];
        for (int k = 5; k >= 1; --k) {
          f = fma(f, b, poly[k]);
          g = fma(g, b, k * poly[k]);
        }
        f = fma(f, b, poly[0]);
        mtdev::mt_advance(&st, &f, &g);
      }
      const bool accept = st.nfev > 0 && (st.info == 1 || st.f <= st.f0 + st.ftol * st.stp_eval * st.g0);
      q.scal[S_BETA] = st.stp_eval;
      q.scal[S_ACCEPT] = accept ? 1.0 : 0.0;
      q.scal[5] = (double)st.nfev;
      q.scal[6] = (double)st.info;
      sh.bcast[1] = accept ? 1.0 : 0.0;
      sh.bcast[2] = st.stp_eval;
    }
    __syncthreads();
    if (sh.bcast[1] != 0.0) {
      const double beta = sh.bcast[2];
      for (int e = threadIdx.x; e < 3 * RR; e += kThreads) {
        const int n = e / RR, rs = e - n * RR;
        const int r = rs / R, s2 = rs - (rs / R) * R;
        const double a1 = q.Gad[e] + q.Gad[(size_t)n * RR + s2 * R + r];
        q.Gx[e] = fma(beta, fma(beta, q.Gdd[e], a1), q.Gb[e]);
      }
    }
  }
  cl_sync();
  const double beta = q.scal[S_BETA];
  const bool accept = q.scal[S_ACCEPT] != 0.0;
  if (threadIdx.x == 0) {
    sh.c.ls_trials += (int)q.scal[5];
    if ((int)q.scal[6] != 1) sh.c.ls_failures += 1;
    if (accept) {
      sh.c.accepts += 1;
      sh.c.fg_evals += 1;
    }
  }
  __syncthreads();
  // (Z's first R columns are T x_3 Abar^(3))
  if (!accept) return keep_ubar(sh, rk, C, false, 3, t0, budget);   // R10

  // ---- the accepted point x = ubar + beta d: M^(1), M^(2) from the variants
  for_own(w, R, [&](int e, int, int, int) { q.x[e] = fma(beta, q.d[e], ub[e]); });
  {
    const double b2 = beta * beta;
    const size_t s1 = (size_t)q.I1 * R, s2 = (size_t)q.I2 * R;
    for (int k = threadIdx.x; k < (w.hi[0] - w.lo[0]) * R; k += kThreads) {
      const int e = w.lo[0] * R + k;
      q.M1[e] = q.V1[e] + beta * (q.V1[s1 + e] + q.V1[2 * s1 + e]) + b2 * q.V1[3 * s1 + e];
    }
    for (int k = threadIdx.x; k < (w.hi[1] - w.lo[1]) * R; k += kThreads) {
      const int e = w.lo[1] * R + k;
      q.M2[e] = q.V2[e] + beta * (q.V2[s2 + e] + q.V2[2 * s2 + e]) + b2 * q.V2[3 * s2 + e];
    }
  }
  cl_sync();
  do_pass_m3<AT>(q, q.x, q.x + q.off2, my + BA, rk, C, big);
  cl_sync();
  double inner = 0.0;
  for (int k = threadIdx.x; k < (w.hi[2] - w.lo[2]) * R; k += kThreads) {
    const int e = w.lo[2] * R + k;
    const double mv = psum(q.part + BA, ld, C, e);
    q.M3[e] = mv;
    inner = fma(q.x[q.off3 + e], mv, inner);
  }
  inner = cta_sum(inner, sh);
  grad_rows(q, w, q.x, q.Gx, q.M1, q.M2, q.M3, sw, sh);
  // u, g = normalise(x, g(x)) (R8), with the scales from x's Grams
  for (int t = threadIdx.x; t < 3 * R; t += kThreads) {
    const int n = t / R, r = t - (t / R) * R;
    sh.sc2[t] = q.Gx[(size_t)n * RR + r * R + r];
  }
  norm_scales(sh.sc2, R, sh, sh.scale, sh.order);
  for_own(w, R, [&](int e, int n, int i, int r) {
    const int o = sh.order[r];
    const size_t src = w.off[n] + (size_t)i * R + o;
    const double sc = sh.scale[n * R + o];
    q.u[e] = q.x[src] * sc;
    q.g[e] = sw[src] / sc;
  });
  if (rk == 0) grams_normalised(q.Gx, R, sh.scale, sh.order, q.Gu);
  // the next sweep's Y = T x_3 A^(3)(u): u's A^(3) is x's, scaled and
  // reordered, and T x_3 x^(3) = Z_ubar + beta Z_d (the line-search pass)
  {
    const int jlo = lo_of(q.J, rk, C), jhi = lo_of(q.J, rk + 1, C);
    const AT* Z = (const AT*)q.Y;
    AT* Y2 = (AT*)q.Y2;
    const AT b = (AT)beta;
    for (int k = threadIdx.x; k < (jhi - jlo) * R; k += kThreads) {
      const int j = jlo + k / R, p = k - (k / R) * R;
      const int o = sh.order[p];
      const AT* z = Z + (size_t)j * 2 * R;
      Y2[(size_t)j * R + p] = fmat(b, z[R + o], z[o]) * (AT)sh.scale[2 * R + o];
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) sh.c.ysrc = 2;
  const double gpart = cta_sum(window_push(q, w, q.u, q.g, push_slot(sh.c, q.w, false)), sh);
  if (threadIdx.x == 0) {
    my[SCA + 1] = inner;
    my[SCA + 2] = gpart;
  }
  return tail(sh, rk, C, T_ACCEPT, false, t0, budget);
}

// ------------------------------------------------------------------ kernel

// Persistent: each cluster takes requests from the queue (tasks[next++]) and
// runs their solves; a cluster stops taking new ones once its CTA 0 has run
// for budget_ns, and parks its current request at the end of the iteration
// in which that happens (the request's state stays in its buffers).
__global__ void __launch_bounds__(kThreads, 1)
    many_kernel(const ManyReq* __restrict__ reqs, const int* __restrict__ tasks, ManyQueue* queue,
                int* cluster_task) {
  extern __shared__ __align__(128) unsigned char dyn_smem[];
  EngSh& sh = *reinterpret_cast<EngSh*>(dyn_smem);
  char* big = reinterpret_cast<char*>(dyn_smem) + (sizeof(EngSh) + 127) / 128 * 128;
  const int rk = (int)cl_rank(), C = (int)cl_size();
  const unsigned cid = cl_id();
  if (threadIdx.x == 0) sh.t0 = gtimer();
  __syncthreads();
  const unsigned long long t0 = sh.t0;
  const unsigned long long budget = queue->budget_ns;
  const int ntasks = queue->ntasks;
  for (;;) {
    if (rk == 0 && threadIdx.x == 0) {
      int t = ntasks;
      if (gtimer() - t0 <= budget) t = atomicAdd(&queue->next, 1);
      cluster_task[cid] = t;
    }
    cl_sync();
    if (threadIdx.x == 0) sh.task = *(volatile int*)&cluster_task[cid];
    __syncthreads();
    const int t = sh.task;
    cl_sync();
    if (t >= ntasks) break;
    if (threadIdx.x == 0) {
      sh.q = reqs[tasks[t]];
      sh.c = *sh.q.ctl;
    }
    __syncthreads();
    for (;;) {
      if (sh.c.phase == PH_DONE) break;
      bool leave;
      if (sh.c.start)
        leave = sh.c.phase == PH_MIXED ? run_start<float>(sh, big, rk, C, t0, budget)
                                       : run_start<double>(sh, big, rk, C, t0, budget);
      else
        leave = sh.c.phase == PH_MIXED ? run_iter<float>(sh, big, rk, C, t0, budget)
                                       : run_iter<double>(sh, big, rk, C, t0, budget);
      if (leave) break;
    }
  }
}

size_t engine_smem() {
  size_t bigb = std::max<size_t>(kBsBytes + kTstBytes, kTchBytes + kKRBytes + (size_t)kMaxIR * sizeof(double));
  bigb = std::max<size_t>(bigb, ((size_t)kMaxW * kTileLd + kTile) * sizeof(double));
  return (sizeof(EngSh) + 127) / 128 * 128 + bigb;
}

}  // namespace
}  // namespace cpg

// ------------------------------------------------------------------- host

namespace cpg {

namespace {

constexpr int kStallDefault = 800;
constexpr int kProbeIters = 6;        // iterations a tuning probe runs
constexpr int kGroups = 4;            // cluster sizes 1, 2, 4, 8

int64_t big_ld_of(int I3, int R) {
  int64_t b = std::max<int64_t>((int64_t)I3 * R, 6 * (int64_t)R * R);
  b = std::max<int64_t>(b, (int64_t)kMaxW * (kMaxW + 1) / 2 + kMaxW);
  return (b + 31) / 32 * 32;
}

// Bytes of one request's state; with base, the pointers of q are set.
size_t job_layout(ManyReq& q, char* base) {
  const int64_t P = q.P, R = q.R, RR = R * R;
  const int64_t big = big_ld_of(q.I3, q.R);
  const int64_t ld = 2 * big + 256;
  size_t n = 0;
  auto take = [&](int64_t cnt) -> double* {
    double* p = base ? (double*)(base + n * sizeof(double)) : nullptr;
    n += (size_t)((cnt + 15) / 16 * 16);   // 128-byte aligned pieces
    return p;
  };
  q.u = take(P);
  q.g = take(P);
  q.ub = take(P);
  q.gb = take(P);
  q.uh = take(P);
  q.d = take(P);
  q.x = take(P);
  q.U = take((int64_t)q.w * P);
  q.G = take((int64_t)q.w * P);
  q.Y = take((int64_t)q.J * 2 * R);
  q.Y2 = take((int64_t)q.J * R);
  q.M1 = take(q.I1 * R);
  q.M2 = take(q.I2 * R);
  q.M3 = take(q.I3 * R);
  q.M3s = take(q.I3 * R);
  q.V1 = take(4 * q.I1 * R);
  q.V2 = take(4 * q.I2 * R);
  q.K = take((int64_t)q.w * q.w);
  q.part = take(kMaxC * ld);
  q.Gu = take(3 * RR);
  q.Gs = take(3 * RR);
  q.Gb = take(3 * RR);
  q.Gad = take(3 * RR);
  q.Gdd = take(3 * RR);
  q.Gx = take(3 * RR);
  q.scal = take(16);
  q.part_ld = (int)ld;
  q.big_ld = (int)big;
  return n * sizeof(double);
}

void fill_req(ManyReq& q, const cp_tensor* t, const cp_solve_opts& o) {
  q = ManyReq{};
  q.T = t->Tn[0];
  q.t64 = t->dtype == CP_DTYPE_F64 ? 1 : 0;
  q.I1 = (int)t->dims[0];
  q.I2 = (int)t->dims[1];
  q.I3 = (int)t->dims[2];
  q.J = q.I1 * q.I2;
  q.R = o.R;
  q.P = (q.I1 + q.I2 + q.I3) * o.R;
  q.off2 = q.I1 * o.R;
  q.off3 = (q.I1 + q.I2) * o.R;
  q.normT2 = t->norm2;
  q.tol = o.tol;
  q.tol_mixed = o.tol * (o.mixed_tol_factor > 0.0 ? o.mixed_tol_factor : 1.0);
  q.eps = o.eps;
  q.maxit = o.maxit;
  q.w = o.w;
  q.polish = o.polish ? 1 : 0;
  q.stall = o.mixed_stall > 0 ? o.mixed_stall : kStallDefault;
  q.ls = o.ls;
  q.ls_mixed = o.ls;
  if (o.mixed_maxfev > 0 && o.mixed_maxfev < o.ls.maxfev) q.ls_mixed.maxfev = o.mixed_maxfev;
}

ManyCtl initial_ctl(const cp_solve_opts& o) {
  ManyCtl c{};
  c.phase = o.prec == CP_FP64 ? PH_FP64 : PH_MIXED;
  c.start = 2;
  c.best = INFINITY;
  c.status = CP_OK;
  return c;
}

// Cluster sizes chosen by the tuner, per (device, ceil log2 entries,
// ceil log2 R, precision) bucket; shared by every context of the process.
struct TuneKey {
  int dev, lk, lr, prec;
  bool operator<(const TuneKey& o) const {
    if (dev != o.dev) return dev < o.dev;
    if (lk != o.lk) return lk < o.lk;
    if (lr != o.lr) return lr < o.lr;
    return prec < o.prec;
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, int> g_tune;

int ceil_log2(int64_t v) {
  int l = 0;
  while (((int64_t)1 << l) < v) ++l;
  return l;
}

TuneKey tune_key(int dev, const cp_tensor* t, const cp_solve_opts& o) {
  return TuneKey{dev, ceil_log2(t->K), ceil_log2(o.R), o.prec == CP_FP64 ? 0 : 1};
}

}  // namespace

// Why a request cannot run on the engine (nullptr when it can).
const char* many_unsupported_dims(int kind, int N, const int64_t* dims, const cp_solve_opts& o) {
  if (kind != 0 || N != 3) return "the engine takes 3-way dense tensors";
  if (o.R < 1 || o.R > kMaxR) return "rank above 32";
  if (o.w < 1 || o.w > kMaxW) return "window above 32";
  for (int n = 0; n < 3; ++n) {
    if (dims[n] < 1 || dims[n] > kMaxI) return "a side above 256";
    if (dims[n] * o.R > kMaxIR) return "I_n R above 8192";
  }
  return nullptr;
}

const char* many_unsupported(const cp_tensor* t, const cp_solve_opts& o) {
  if (!t) return "no tensor";
  return many_unsupported_dims(t->kind, t->N, t->dims, o);
}

// Device bytes of one request's engine state.
size_t many_state_bytes(const int64_t* dims, const cp_solve_opts& o) {
  ManyReq q{};
  q.I1 = (int)dims[0];
  q.I2 = (int)dims[1];
  q.I3 = (int)dims[2];
  q.J = q.I1 * q.I2;
  q.R = o.R;
  q.P = (q.I1 + q.I2 + q.I3) * o.R;
  q.w = o.w;
  return job_layout(q, nullptr) + 4096;
}

// The engine: request states, the device descriptor table, the launch
// rounds.  Not thread-safe (one owner thread).
struct ManyEngine {
  struct Job {
    bool used = false, running = false;
    bool in_round = false;             // launched in the round in flight
    ManyReq q{};
    void* mem = nullptr;
    int C = 1;
    const cp_tensor* t = nullptr;
    int iters = 0;
  };
  cp_ctx* ctx = nullptr;
  int cap = 0;
  int maxcl[kGroups] = {0, 0, 0, 0};
  size_t smem = 0;
  cudaStream_t es = nullptr;          // rounds, read-back, results
  cudaStream_t us = nullptr;          // admissions (allocation, uploads), never behind a round
  cudaEvent_t up_ev = nullptr;        // the last admission's uploads
  cudaStream_t gs[kGroups] = {};
  cudaEvent_t fork = nullptr, join[kGroups] = {}, round_ev = nullptr, pa = nullptr, pb = nullptr;
  ManyReq* req_d = nullptr;          // cap + 1 descriptors (the last one for tuning probes)
  ManyCtl* ctl_d = nullptr;          // cap + 1
  char* qbuf_d = nullptr;
  size_t qstride = 0;
  ManyCtl* ctl_h = nullptr;          // pinned: control blocks read back after a round
  ManyCtl* ctl_up = nullptr;         // pinned: initial control blocks to upload
  int* tasks_h = nullptr;            // pinned, kGroups x cap
  ManyQueue* q_h = nullptr;          // pinned, kGroups
  std::vector<Job> jobs;
  bool in_flight = false;
  int launched_rounds = 0;
  int max_ctas = 0;                  // CTAs one round may use (<= 0: as many as fit)
  unsigned long long round_ns = 500ull * 1000 * 1000;   // cp_solve_many's round length

  ~ManyEngine() { destroy(); }

  cp_status create(cp_ctx* c, int capacity) {
    ctx = c;
    cap = std::max(1, capacity);
    smem = engine_smem();
    CP_CUDA(cudaSetDevice(ctx->device));
    CP_CUDA(cudaFuncSetAttribute(many_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    CP_CUDA(cudaStreamCreateWithFlags(&es, cudaStreamNonBlocking));
    CP_CUDA(cudaStreamCreateWithFlags(&us, cudaStreamNonBlocking));
    CP_CUDA(cudaEventCreateWithFlags(&up_ev, cudaEventDisableTiming));
    for (int k = 0; k < kGroups; ++k) {
      CP_CUDA(cudaStreamCreateWithFlags(&gs[k], cudaStreamNonBlocking));
      CP_CUDA(cudaEventCreateWithFlags(&join[k], cudaEventDisableTiming));
    }
    CP_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    CP_CUDA(cudaEventCreateWithFlags(&round_ev, cudaEventDisableTiming));
    CP_CUDA(cudaEventCreate(&pa));
    CP_CUDA(cudaEventCreate(&pb));
    for (int k = 0; k < kGroups; ++k) {
      const int C = 1 << k;
      cudaLaunchConfig_t cfg{};
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = (unsigned)C;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.gridDim = dim3((unsigned)C);
      cfg.blockDim = dim3(kThreads);
      cfg.dynamicSmemBytes = smem;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      int n = 0;
      if (cudaOccupancyMaxActiveClusters(&n, many_kernel, &cfg) != cudaSuccess) {
        (void)cudaGetLastError();
        n = 0;
      }
      maxcl[k] = n;
    }
    if (maxcl[0] < 1) {
      set_error("cp_solve_many: the engine kernel cannot be resident");
      return CP_ERR_CUDA;
    }
    const int mx = std::max({maxcl[0], maxcl[1], maxcl[2], maxcl[3], 1});
    qstride = (sizeof(ManyQueue) + 64 + (size_t)(cap + 1 + mx) * sizeof(int) + 255) / 256 * 256;
    CP_CUDA(cudaMallocAsync((void**)&req_d, sizeof(ManyReq) * (cap + 1), es));
    CP_CUDA(cudaMallocAsync((void**)&ctl_d, sizeof(ManyCtl) * (cap + 1), es));
    CP_CUDA(cudaMallocAsync((void**)&qbuf_d, qstride * (kGroups + 1), es));
    CP_CUDA(cudaMallocHost((void**)&ctl_h, sizeof(ManyCtl) * (cap + 1)));
    CP_CUDA(cudaMallocHost((void**)&ctl_up, sizeof(ManyCtl) * (cap + 1)));
    CP_CUDA(cudaMallocHost((void**)&tasks_h, sizeof(int) * (size_t)(kGroups + 1) * (cap + 1)));
    CP_CUDA(cudaMallocHost((void**)&q_h, sizeof(ManyQueue) * (kGroups + 1)));
    jobs.resize((size_t)cap);
    return CP_OK;
  }

  void destroy() {
    if (es) cudaStreamSynchronize(es);
    for (auto& j : jobs)
      if (j.mem) cudaFreeAsync(j.mem, es);
    jobs.clear();
    if (req_d) cudaFreeAsync(req_d, es);
    if (ctl_d) cudaFreeAsync(ctl_d, es);
    if (qbuf_d) cudaFreeAsync(qbuf_d, es);
    req_d = nullptr;
    ctl_d = nullptr;
    qbuf_d = nullptr;
    if (es) cudaStreamSynchronize(es);
    if (ctl_h) cudaFreeHost(ctl_h);
    if (ctl_up) cudaFreeHost(ctl_up);
    ctl_up = nullptr;
    if (tasks_h) cudaFreeHost(tasks_h);
    if (q_h) cudaFreeHost(q_h);
    ctl_h = nullptr;
    tasks_h = nullptr;
    q_h = nullptr;
    for (int k = 0; k < kGroups; ++k) {
      if (gs[k]) cudaStreamDestroy(gs[k]);
      if (join[k]) cudaEventDestroy(join[k]);
      gs[k] = nullptr;
      join[k] = nullptr;
    }
    if (fork) cudaEventDestroy(fork);
    if (round_ev) cudaEventDestroy(round_ev);
    if (pa) cudaEventDestroy(pa);
    if (pb) cudaEventDestroy(pb);
    fork = round_ev = pa = pb = nullptr;
    if (us) {
      cudaStreamSynchronize(us);
      cudaStreamDestroy(us);
    }
    if (up_ev) cudaEventDestroy(up_ev);
    us = nullptr;
    up_ev = nullptr;
    if (es) cudaStreamDestroy(es);
    es = nullptr;
  }

  // One launch of cluster size C over ntasks requests (tasks_h + group
  // offset already filled) on stream s, queue block g.
  cp_status launch(int g, int C, int ntasks, unsigned long long budget_ns, cudaStream_t s, int cta_cap = 0) {
    char* qb = qbuf_d + (size_t)g * qstride;
    ManyQueue* qd = (ManyQueue*)qb;
    int* tasks_d = (int*)(qb + sizeof(ManyQueue) + 64);
    int* ctask_d = tasks_d + cap + 1;
    q_h[g] = ManyQueue{0, ntasks, budget_ns};
    const int k = C == 1 ? 0 : C == 2 ? 1 : C == 4 ? 2 : 3;
    int nclusters = std::min(maxcl[k], ntasks);
    if (cta_cap > 0) nclusters = std::max(1, std::min(nclusters, cta_cap / C));
    if (nclusters < 1) {
      set_error("cp_solve_many: clusters of %d CTAs cannot be resident", C);
      return CP_ERR_CUDA;
    }
    CP_CUDA(cudaMemcpyAsync(qd, &q_h[g], sizeof(ManyQueue), cudaMemcpyHostToDevice, s));
    CP_CUDA(cudaMemcpyAsync(tasks_d, tasks_h + (size_t)g * (cap + 1), sizeof(int) * ntasks, cudaMemcpyHostToDevice, s));
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)(nclusters * C));
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    CP_CUDA(cudaLaunchKernelEx(&cfg, many_kernel, (const ManyReq*)req_d, (const int*)tasks_d, qd, ctask_d));
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return CP_OK;
  }

  // Cluster size for a request: the tuned one for its bucket.  The first
  // request of a bucket times kProbeIters iterations of itself with each
  // cluster size (scratch state, descriptor slot cap); among the sizes whose
  // time is within 1.5x of the fastest, the one with the least SM time
  // (C x elapsed) is kept: the fewest CTAs that do not stretch the
  // request's latency by more than half.
  cp_status tuned_cluster(const cp_tensor* t, const cp_solve_opts& o, const double* u0, int* out) {
    const TuneKey key = tune_key(ctx->device, t, o);
    {
      std::lock_guard<std::mutex> lock(g_tune_mu);
      auto it = g_tune.find(key);
      if (it != g_tune.end()) {
        *out = it->second;
        return CP_OK;
      }
    }
    ManyReq q;
    fill_req(q, t, o);
    q.maxit = std::min(o.maxit, kProbeIters);
    q.tol = 0.0;
    q.tol_mixed = 0.0;
    void* mem = nullptr;
    CP_CUDA(cudaMallocAsync(&mem, job_layout(q, nullptr), es));
    (void)job_layout(q, (char*)mem);
    q.ctl = ctl_d + cap;
    const ManyCtl c0 = initial_ctl(o);
    double best = INFINITY;
    int bestC = 1;
    double tms[kGroups] = {INFINITY, INFINITY, INFINITY, INFINITY};
    cp_status st = CP_OK;
    for (int pass = 0; pass < 2 && st == CP_OK; ++pass) {
      for (int k = 0; k < kGroups && st == CP_OK; ++k) {
        const int C = 1 << k;
        if (maxcl[k] < 1 || (pass == 0 && k > 0)) continue;   // pass 0: one warm-up launch
        // the probe uses descriptor and control slot cap and queue block kGroups
        ctl_up[cap] = c0;
        char* qb = qbuf_d + (size_t)kGroups * qstride;
        ManyQueue* qd = (ManyQueue*)qb;
        int* tasks_d = (int*)(qb + sizeof(ManyQueue) + 64);
        int* ctask_d = tasks_d + cap + 1;
        q_h[kGroups] = ManyQueue{0, 1, ~0ull >> 1};
        tasks_h[(size_t)kGroups * (cap + 1)] = cap;
        cudaLaunchConfig_t cfg{};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)C;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3((unsigned)C);
        cfg.blockDim = dim3(kThreads);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = es;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        cudaError_t e = cudaMemcpyAsync(q.ctl, &ctl_up[cap], sizeof(ManyCtl), cudaMemcpyHostToDevice, es);
        if (e == cudaSuccess) e = cudaMemcpyAsync(req_d + cap, &q, sizeof(ManyReq), cudaMemcpyHostToDevice, es);
        if (e == cudaSuccess) e = cudaMemcpyAsync(q.x, u0, sizeof(double) * q.P, cudaMemcpyDefault, es);
        if (e == cudaSuccess) e = cudaMemcpyAsync(qd, &q_h[kGroups], sizeof(ManyQueue), cudaMemcpyHostToDevice, es);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(tasks_d, tasks_h + (size_t)kGroups * (cap + 1), sizeof(int), cudaMemcpyHostToDevice, es);
        if (e == cudaSuccess) e = cudaEventRecord(pa, es);
        if (e == cudaSuccess)
          e = cudaLaunchKernelEx(&cfg, many_kernel, (const ManyReq*)req_d, (const int*)tasks_d, qd, ctask_d);
        g_launches.fetch_add(1, std::memory_order_relaxed);
        if (e == cudaSuccess) e = cudaEventRecord(pb, es);
        if (e == cudaSuccess) e = cudaEventSynchronize(pb);
        if (e != cudaSuccess) {
          st = cuda_fail(e, "cp_solve_many: tuning probe", __FILE__, __LINE__);
          break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, pa, pb);
        if (pass == 1) tms[k] = ms;
      }
    }
    cudaFreeAsync(mem, es);
    if (st != CP_OK) return st;
    double tmin = INFINITY;
    for (int k = 0; k < kGroups; ++k) tmin = std::min(tmin, tms[k]);
    for (int k = 0; k < kGroups; ++k) {
      const int C = 1 << k;
      if (tms[k] <= 1.5 * tmin && (double)C * tms[k] < best) {
        best = (double)C * tms[k];
        bestC = C;
      }
    }
    {
      std::lock_guard<std::mutex> lock(g_tune_mu);
      g_tune[key] = bestC;
    }
    *out = bestC;
    return CP_OK;
  }

  // Admit a request (its tensor complete on the device).  cluster: 1, 2, 4,
  // 8, or 0 for the tuned size.
  cp_status add(const cp_tensor* t, const cp_solve_opts& o, const double* u0, int cluster, int* slot) {
    int k = -1;
    for (int i = 0; i < cap; ++i)
      if (!jobs[i].used) {
        k = i;
        break;
      }
    if (k < 0) {
      set_error("cp_solve_many: engine full");
      return CP_ERR_BUSY;
    }
    int C = cluster;
    if (C == 0) CP_TRY(tuned_cluster(t, o, u0, &C));
    Job& j = jobs[k];
    fill_req(j.q, t, o);
    void* mem = nullptr;
    // on the admission stream: a host upload on es would wait for the round
    // in flight (pageable copies return only when done)
    CP_CUDA(cudaMallocAsync(&mem, job_layout(j.q, nullptr), us));
    (void)job_layout(j.q, (char*)mem);
    j.q.ctl = ctl_d + k;
    j.mem = mem;
    j.C = C;
    j.t = t;
    j.used = true;
    j.running = true;
    j.iters = 0;
    // (ctl_h belongs to the round read-back, which may still be in flight)
    ctl_up[k] = initial_ctl(o);
    CP_CUDA(cudaMemcpyAsync(j.q.x, u0, sizeof(double) * j.q.P, cudaMemcpyDefault, us));
    CP_CUDA(cudaMemcpyAsync(ctl_d + k, &ctl_up[k], sizeof(ManyCtl), cudaMemcpyHostToDevice, us));
    CP_CUDA(cudaMemcpyAsync(req_d + k, &j.q, sizeof(ManyReq), cudaMemcpyHostToDevice, us));
    CP_CUDA(cudaEventRecord(up_ev, us));   // the next round waits for it
    // pageable sources above: the copies have been taken before they return
    *slot = k;
    return CP_OK;
  }

  int running() const {
    int n = 0;
    for (const auto& j : jobs) n += j.running ? 1 : 0;
    return n;
  }

  // Enqueue one round: every running request, grouped by cluster size, one
  // launch per group on its own stream (least iterations first), then the
  // control blocks back to the host.  Non-blocking.
  cp_status launch_round(unsigned long long budget_ns) {
    CP_CUDA(cudaStreamWaitEvent(es, up_ev, 0));
    CP_CUDA(cudaEventRecord(fork, es));
    int left = max_ctas;   // shared by the groups, larger clusters first
    for (int g = kGroups - 1; g >= 0; --g) {
      const int C = 1 << g;
      std::vector<int> ids;
      for (int i = 0; i < cap; ++i)
        if (jobs[i].running && jobs[i].C == C) ids.push_back(i);
      if (ids.empty()) continue;
      std::stable_sort(ids.begin(), ids.end(), [&](int a, int b) { return jobs[a].iters < jobs[b].iters; });
      for (int i : ids) jobs[i].in_round = true;
      std::copy(ids.begin(), ids.end(), tasks_h + (size_t)g * (cap + 1));
      CP_CUDA(cudaStreamWaitEvent(gs[g], fork, 0));
      const int cap_g = max_ctas > 0 ? std::max(left, C) : 0;
      CP_TRY(launch(g, C, (int)ids.size(), budget_ns, gs[g], cap_g));
      if (max_ctas > 0) left -= std::min((int)ids.size(), std::max(1, cap_g / C)) * C;
      CP_CUDA(cudaEventRecord(join[g], gs[g]));
      CP_CUDA(cudaStreamWaitEvent(es, join[g], 0));
    }
    CP_CUDA(cudaMemcpyAsync(ctl_h, ctl_d, sizeof(ManyCtl) * cap, cudaMemcpyDeviceToHost, es));
    CP_CUDA(cudaEventRecord(round_ev, es));
    in_flight = true;
    ++launched_rounds;
    return CP_OK;
  }

  // After a round: true when it has finished; `finished` receives the
  // requests that are done.
  cp_status poll(bool block, bool* idle, std::vector<int>* finished) {
    *idle = true;
    if (!in_flight) return CP_OK;
    const cudaError_t e = block ? cudaEventSynchronize(round_ev) : cudaEventQuery(round_ev);
    if (e == cudaErrorNotReady) {
      *idle = false;
      return CP_OK;
    }
    in_flight = false;
    if (e != cudaSuccess) return cuda_fail(e, "cp_solve_many: engine round", __FILE__, __LINE__);
    for (int i = 0; i < cap; ++i) {
      Job& j = jobs[i];
      if (!j.running || !j.in_round) continue;   // admitted after the round was launched
      j.in_round = false;
      j.iters = ctl_h[i].iters;
      if (ctl_h[i].phase == PH_DONE) {
        j.running = false;
        if (finished) finished->push_back(i);
      }
    }
    return CP_OK;
  }

  // Result of a finished request: u (host or device), report, status.  With
  // sync false the copy of u is only enqueued (the caller synchronises es).
  cp_status result(int k, double* u_out, cp_solve_report* rep, cp_status* status, bool sync = true) {
    const Job& j = jobs[k];
    const ManyCtl& c = ctl_h[k];
    CP_CUDA(cudaMemcpyAsync(u_out, j.q.u, sizeof(double) * j.q.P, cudaMemcpyDefault, es));
    if (sync) CP_CUDA(cudaStreamSynchronize(es));
    if (rep) {
      cp_solve_report r{};
      r.iters = c.iters;
      r.fg_evals = c.fg_evals;
      r.als_sweeps = c.als_sweeps;
      r.restarts = c.restarts;
      r.ls_failures = c.ls_failures;
      r.converged = (c.stop == STOP_TOL && c.status == CP_OK) ? 1 : 0;
      r.mixed_iters = c.mixed_iters;
      r.fp64_iters = c.fp64_iters;
      r.f = c.f;
      r.gnorm_over_P = c.gn;
      r.normT2 = j.t->norm2;
      r.ls_trials = c.ls_trials;
      *rep = r;
    }
    cp_status st = (cp_status)c.status;
    if (st == CP_OK && c.stop != STOP_TOL) st = CP_ERR_MAXIT;
    if (status) *status = st;
    return CP_OK;
  }

  void release(int k) {
    Job& j = jobs[k];
    if (j.mem) cudaFreeAsync(j.mem, es);
    j = Job();
  }
};

ManyEngine* many_engine_create(cp_ctx* ctx, int capacity, cp_status* st) {
  ManyEngine* e = new ManyEngine();
  *st = e->create(ctx, capacity);
  if (*st != CP_OK) {
    delete e;
    return nullptr;
  }
  return e;
}
void many_engine_destroy(ManyEngine* e) { delete e; }
cp_status many_engine_add(ManyEngine* e, const cp_tensor* t, const cp_solve_opts& o, const double* u0, int* slot) {
  return e->add(t, o, u0, 0, slot);
}
cudaStream_t many_engine_stream(ManyEngine* e) { return e->es; }
int many_engine_running(ManyEngine* e) { return e->running(); }
void many_engine_set_cta_cap(ManyEngine* e, int max_ctas) { e->max_ctas = max_ctas; }
bool many_engine_in_flight(ManyEngine* e) { return e->in_flight; }
cp_status many_engine_launch(ManyEngine* e, double budget_s) {
  return e->launch_round((unsigned long long)(budget_s * 1e9));
}
cp_status many_engine_poll(ManyEngine* e, bool block, bool* idle, std::vector<int>* finished) {
  return e->poll(block, idle, finished);
}
cp_status many_engine_result(ManyEngine* e, int slot, double* u_out, cp_solve_report* rep, cp_status* st) {
  return e->result(slot, u_out, rep, st);
}
void many_engine_release(ManyEngine* e, int slot) { e->release(slot); }

cp_status many_solve(cp_ctx* ctx, int nreq, const cp_tensor* const* ts, const cp_solve_opts* opts,
                     double* const* u, cp_solve_report* reps, int cluster) {
  if (!ctx || nreq < 0 || (nreq > 0 && (!ts || !opts || !u)) || cluster < 0 || cluster > kMaxC ||
      (cluster & (cluster - 1))) {
    set_error("cp_solve_many: bad arguments");
    return CP_ERR_ARG;
  }
  if (nreq == 0) return CP_OK;
  CP_CUDA(cudaSetDevice(ctx->device));
  for (int i = 0; i < nreq; ++i) {
    if (!ts[i] || !u[i] || ts[i]->device != ctx->device) {
      set_error("cp_solve_many: request %d: null tensor or iterate, or tensor on another device", i);
      return CP_ERR_ARG;
    }
    const char* why = many_unsupported(ts[i], opts[i]);
    if (why) {
      set_error("cp_solve_many: request %d: %s", i, why);
      return CP_ERR_UNSUPPORTED;
    }
    const cp_solve_opts& o = opts[i];
    if (!(o.tol > 0.0) || o.maxit < 0 || !(o.eps >= 0.0) || o.ls.maxfev < 1) {
      set_error("cp_solve_many: request %d: bad options", i);
      return CP_ERR_ARG;
    }
  }
  CP_CUDA(cudaStreamSynchronize(ctx->stream));   // the tensors are complete
  const auto t0 = std::chrono::steady_clock::now();
  // the context keeps its engine (streams, pinned buffers, descriptor table)
  // between calls; a larger batch replaces it
  ManyEngine* ep = static_cast<ManyEngine*>(ctx->many);
  if (!ep || ep->cap < nreq) {
    const unsigned long long round_ns = ep ? ep->round_ns : 500ull * 1000 * 1000;
    if (ep) many_engine_destroy(ep);
    ctx->many = nullptr;
    cp_status cst = CP_OK;
    ep = many_engine_create(ctx, std::max(nreq, 64), &cst);
    if (!ep) return cst;
    ep->round_ns = round_ns;
    ctx->many = ep;
  }
  ManyEngine& e = *ep;
  struct Release {
    ManyEngine& e;
    ~Release() {
      for (int k = 0; k < e.cap; ++k)
        if (e.jobs[k].used) e.release(k);
    }
  } release_all{e};
  std::vector<int> slot((size_t)nreq, -1);
  std::vector<double> t_done((size_t)nreq, 0.0);
  cp_status st = CP_OK;
  for (int i = 0; i < nreq && st == CP_OK; ++i) st = e.add(ts[i], opts[i], u[i], cluster, &slot[i]);
  while (st == CP_OK && e.running() > 0) {
    st = e.launch_round(e.round_ns);
    if (st != CP_OK) break;
    bool idle = false;
    std::vector<int> fin;
    st = e.poll(true, &idle, &fin);
    const double now = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    for (int k : fin) t_done[(size_t)k] = now;   // slot k is request k (added in order)
  }
  cp_status first = st;
  std::vector<cp_solve_report> rr((size_t)nreq);
  std::vector<cp_status> rst((size_t)nreq, CP_OK), cst((size_t)nreq, CP_OK);
  for (int i = 0; i < nreq && st == CP_OK; ++i) cst[i] = e.result(slot[i], u[i], &rr[i], &rst[i], false);
  if (st == CP_OK) {
    const cudaError_t ce = cudaStreamSynchronize(e.es);
    if (ce != cudaSuccess) first = cuda_fail(ce, "cp_solve_many: solutions", __FILE__, __LINE__);
  }
  for (int i = 0; i < nreq && st == CP_OK; ++i) {
    cp_solve_report r = rr[i];
    const cp_status rs = rst[i];
    const cp_status c = cst[i];
    r.t_total_s = t_done[(size_t)slot[i]];
    if (reps) reps[i] = r;
    if (first == CP_OK) {
      if (c != CP_OK) {
        first = c;
      } else if (rs != CP_OK) {
        if (rs == CP_ERR_MAXIT)
          set_error("cp_solve_many: request %d: tol not met after %d iterations (||g||/P = %.3e)", i, r.iters,
                    r.gnorm_over_P);
        else
          set_error("cp_solve_many: request %d: %s", i,
                    rs == CP_ERR_NOT_SPD ? "Gammabar not positive definite" : "non-finite gradient");
        first = rs;
      }
    }
  }
  return first;
}

cp_status many_plan(cp_ctx* ctx, const cp_tensor* t, const cp_solve_opts* o, const double* u0, int* cluster) {
  if (!ctx || !t || !o || !u0 || !cluster) {
    set_error("cp_many_plan: bad arguments");
    return CP_ERR_ARG;
  }
  const char* why = many_unsupported(t, *o);
  if (why) {
    set_error("cp_many_plan: %s", why);
    return CP_ERR_UNSUPPORTED;
  }
  CP_CUDA(cudaSetDevice(ctx->device));
  CP_CUDA(cudaStreamSynchronize(ctx->stream));
  ManyEngine* ep = static_cast<ManyEngine*>(ctx->many);
  if (!ep) {
    cp_status cst = CP_OK;
    ep = many_engine_create(ctx, 64, &cst);
    if (!ep) return cst;
    ctx->many = ep;
  }
  return ep->tuned_cluster(t, *o, u0, cluster);
}

}  // namespace cpg

extern "C" cp_status cp_solve_many(cp_ctx* ctx, int nreq, const cp_tensor* const* tensors, const cp_solve_opts* opts,
                                   double* const* u, cp_solve_report* reps, int cluster) {
  return cpg::many_solve(ctx, nreq, tensors, opts, u, reps, cluster);
}

extern "C" cp_status cp_many_set_round(cp_ctx* ctx, double seconds) {
  if (!ctx || !(seconds > 0.0) || seconds > 3600.0) {
    cpg::set_error("cp_many_set_round: bad arguments");
    return CP_ERR_ARG;
  }
  if (!ctx->many) {
    cp_status cst = CP_OK;
    cpg::ManyEngine* e = cpg::many_engine_create(ctx, 64, &cst);
    if (!e) return cst;
    ctx->many = e;
  }
  static_cast<cpg::ManyEngine*>(ctx->many)->round_ns = (unsigned long long)(seconds * 1e9);
  return CP_OK;
}

extern "C" cp_status cp_many_plan(cp_ctx* ctx, const cp_tensor* t, const cp_solve_opts* opts, const double* u0,
                                  int* cluster) {
  return cpg::many_plan(ctx, t, opts, u0, cluster);
}
