// Sparse (COO) tensors (Section 4): per-mode sorted copies and the sparse
// MTTKRP M^(n) = T_(n) Phibar^(n) over the nonzeros only (Section 2.3).
//
// Build, for every mode n (once per tensor):
//   * stable LSD radix sort (4-bit digits, written here) of the nonzero
//     indices by the cyclic key (i_n, i_{n+1}, ..., i_{n-1}): one stable pass
//     per digit, components taken from least to most significant;
//   * segments = runs of equal i_n (head flags + exclusive scan);
//   * work units = segments cut into chunks of at most kUnit nonzeros;
//   * the other coordinates as int32 planes and the values, in sorted order.
// MTTKRP: one warp per unit (its nonzeros share one output row).  FP32
// products: "vector groups" of lanes per nonzero, each lane reading one
// 16-byte piece of every gathered factor row; FP64 products: a staged form
// (the warp reads 32 nonzeros' values and coordinates at once, then groups
// of R lanes gather the rows entry by entry).  Either way the products are
// summed per lane and the lanes combined by shuffles in a fixed order (no
// atomics); a last kernel adds the units of each segment in order into M.
// Rows without nonzeros are zero.
#include <algorithm>
#include <vector>

#include "cp_internal.cuh"

namespace cpg {

cp_status sumsq(cp_ctx* ctx, const void* x, cp_dtype dt, int64_t n, double* d_out);

namespace {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kBins = 16;
constexpr int kUnit = 256;            // nonzeros per MTTKRP work unit

// ------------------------------------------------------------- scans (int64)
// Exclusive scan, tile of 2048 per block: block sums, then a one-block scan
// of the sums, then the per-tile scans with the carried offset.
__global__ void tile_sum_kernel(const int64_t* __restrict__ in, int64_t n, int64_t* __restrict__ sums) {
  __shared__ int64_t sh[kSortThreads];
  const int64_t base = (int64_t)blockIdx.x * kSortTile + threadIdx.x * kSortItems;
  int64_t s = 0;
  for (int i = 0; i < kSortItems; ++i)
    if (base + i < n) s += in[base + i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int st = kSortThreads / 2; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) sh[threadIdx.x] += sh[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) sums[blockIdx.x] = sh[0];
}

// In-place exclusive scan of x[0..n) by one block of 1024 threads; total to *total.
__global__ void single_block_scan_kernel(int64_t* __restrict__ x, int64_t n, int64_t* total) {
  __shared__ int64_t sh[1024];
  const int64_t per = (n + 1023) / 1024;
  const int64_t b = threadIdx.x * per;
  const int64_t e = min(n, b + per);
  int64_t s = 0;
  for (int64_t k = b; k < e; ++k) s += x[k];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    int64_t v = (int)threadIdx.x >= off ? sh[threadIdx.x - off] : 0;
    __syncthreads();
    sh[threadIdx.x] += v;
    __syncthreads();
  }
  int64_t run = threadIdx.x ? sh[threadIdx.x - 1] : 0;
  for (int64_t k = b; k < e; ++k) {
    const int64_t v = x[k];
    x[k] = run;
    run += v;
  }
  if (threadIdx.x == 1023 && total) *total = sh[1023];
}

__global__ void tile_scan_kernel(const int64_t* __restrict__ in, int64_t n,
                                 const int64_t* __restrict__ offs, int64_t* __restrict__ out) {
  __shared__ int64_t sh[kSortThreads];
  const int64_t base = (int64_t)blockIdx.x * kSortTile + threadIdx.x * kSortItems;
  int64_t v[kSortItems];
  int64_t s = 0;
  for (int i = 0; i < kSortItems; ++i) {
    v[i] = base + i < n ? in[base + i] : 0;
    s += v[i];
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int off = 1; off < kSortThreads; off <<= 1) {
    int64_t t = (int)threadIdx.x >= off ? sh[threadIdx.x - off] : 0;
    __syncthreads();
    sh[threadIdx.x] += t;
    __syncthreads();
  }
  int64_t run = offs[blockIdx.x] + (threadIdx.x ? sh[threadIdx.x - 1] : 0);
  for (int i = 0; i < kSortItems; ++i) {
    if (base + i < n) out[base + i] = run;
    run += v[i];
  }
}

// ----------------------------------------------------------------- radix sort
__device__ __forceinline__ int digit_of(const int64_t* coords, int N, int c, int shift, int64_t idx) {
  return (int)((coords[idx * N + c] >> shift) & (kBins - 1));
}

__global__ void radix_hist_kernel(const int64_t* __restrict__ perm, const int64_t* __restrict__ coords,
                                  int N, int c, int shift, int64_t n, int64_t* __restrict__ hist,
                                  int64_t ntiles) {
  __shared__ int cnt[kBins];
  if (threadIdx.x < kBins) cnt[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kSortTile + threadIdx.x * kSortItems;
  for (int i = 0; i < kSortItems; ++i)
    if (base + i < n) atomicAdd(&cnt[digit_of(coords, N, c, shift, perm[base + i])], 1);
  __syncthreads();
  if (threadIdx.x < kBins) hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

// Stable scatter: thread t owns items [t*8, t*8+8) of the tile, in order.
__global__ void radix_scatter_kernel(const int64_t* __restrict__ perm_in,
                                     const int64_t* __restrict__ coords, int N, int c, int shift,
                                     int64_t n, const int64_t* __restrict__ hist_scan,
                                     int64_t ntiles, int64_t* __restrict__ perm_out) {
  __shared__ int cnt[kBins * kSortThreads];   // [bin][thread]
  __shared__ int tsum[kSortThreads];
  const int64_t base = (int64_t)blockIdx.x * kSortTile + threadIdx.x * kSortItems;
  int64_t item[kSortItems];
  int dig[kSortItems];
  int local[kBins];
#pragma unroll
  for (int b = 0; b < kBins; ++b) local[b] = 0;
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) {
    if (base + i < n) {
      item[i] = perm_in[base + i];
      dig[i] = digit_of(coords, N, c, shift, item[i]);
      local[dig[i]]++;
    } else {
      dig[i] = -1;
    }
  }
#pragma unroll
  for (int b = 0; b < kBins; ++b) cnt[b * kSortThreads + threadIdx.x] = local[b];
  __syncthreads();
  // exclusive scan of cnt in (bin, thread) order: thread t scans entries
  // [t*16, t*16+16), then a block scan of the per-thread sums.
  int run = 0;
  int vals[kBins];
#pragma unroll
  for (int k = 0; k < kBins; ++k) {
    vals[k] = cnt[threadIdx.x * kBins + k];
    run += vals[k];
  }
  tsum[threadIdx.x] = run;
  __syncthreads();
  for (int off = 1; off < kSortThreads; off <<= 1) {
    int t = (int)threadIdx.x >= off ? tsum[threadIdx.x - off] : 0;
    __syncthreads();
    tsum[threadIdx.x] += t;
    __syncthreads();
  }
  int ex = threadIdx.x ? tsum[threadIdx.x - 1] : 0;
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kBins; ++k) {
    cnt[threadIdx.x * kBins + k] = ex;
    ex += vals[k];
  }
  __syncthreads();
  int pos[kBins];
#pragma unroll
  for (int b = 0; b < kBins; ++b)
    pos[b] = cnt[b * kSortThreads + threadIdx.x] - cnt[b * kSortThreads];
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) {
    if (dig[i] >= 0) {
      const int b = dig[i];
      const int64_t dst = hist_scan[(int64_t)b * ntiles + blockIdx.x] + pos[b];
      pos[b]++;
      perm_out[dst] = item[i];
    }
  }
}

__global__ void iota_kernel(int64_t* __restrict__ p, int64_t n) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    p[k] = k;
}

__global__ void range_check_kernel(const int64_t* __restrict__ coords, int64_t nnz, int N,
                                   const int64_t* __restrict__ dims, int* status) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz * N;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int n = (int)(k % N);
    const int64_t v = coords[k];
    if (v < 0 || v >= dims[n]) record_status(status, CP_ERR_SHAPE);
  }
}

// Segment heads of the sorted order: flag[e] = 1 if i_n changes at e.
__global__ void head_flags_kernel(const int64_t* __restrict__ perm, const int64_t* __restrict__ coords,
                                  int N, int n, int64_t nnz, int64_t* __restrict__ flag) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = coords[perm[e] * N + n];
    flag[e] = (e == 0 || coords[perm[e - 1] * N + n] != r) ? 1 : 0;
  }
}

// Duplicate check on a fully sorted order: neighbours must differ somewhere.
__global__ void dup_check_kernel(const int64_t* __restrict__ perm, const int64_t* __restrict__ coords,
                                 int N, int64_t nnz, int* status) {
  for (int64_t e = 1 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t* a = coords + perm[e - 1] * N;
    const int64_t* b = coords + perm[e] * N;
    bool same = true;
    for (int k = 0; k < N; ++k) same = same && (a[k] == b[k]);
    if (same) record_status(status, CP_ERR_SHAPE);
  }
}

__global__ void segments_kernel(const int64_t* __restrict__ perm, const int64_t* __restrict__ coords, int N,
                                int n, int64_t nnz, const int64_t* __restrict__ flag,
                                const int64_t* __restrict__ segidx, int64_t* __restrict__ seg_ptr,
                                int32_t* __restrict__ seg_row) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
    if (flag[e]) {
      const int64_t s = segidx[e];
      seg_ptr[s] = e;
      seg_row[s] = (int32_t)coords[perm[e] * N + n];
    }
  }
}

__global__ void units_count_kernel(const int64_t* __restrict__ seg_ptr, int64_t nseg, int64_t* __restrict__ cnt) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nseg; s += (int64_t)gridDim.x * blockDim.x)
    cnt[s] = (seg_ptr[s + 1] - seg_ptr[s] + kUnit - 1) / kUnit;
}

__global__ void units_fill_kernel(const int64_t* __restrict__ seg_ptr, int64_t nseg,
                                  const int64_t* __restrict__ ubase, int64_t* __restrict__ unit_start,
                                  int64_t nunits, int64_t nnz) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nseg; s += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = seg_ptr[s], e = seg_ptr[s + 1];
    int64_t u = ubase[s];
    for (int64_t k = b; k < e; k += kUnit) unit_start[u++] = k;
    if (s == nseg - 1) unit_start[nunits] = nnz;
  }
}

__global__ void gather_sorted_kernel(const int64_t* __restrict__ perm, const int64_t* __restrict__ coords,
                                     const float* __restrict__ vals, int N, int n, int64_t nnz,
                                     int32_t* __restrict__ other, float* __restrict__ svals) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = perm[e];
    svals[e] = vals[p];
    for (int j = 0; j < N - 1; ++j) other[(int64_t)j * nnz + e] = (int32_t)coords[p * N + (n + 1 + j) % N];
  }
}

// ------------------------------------------------------------------- MTTKRP
struct Tables {
  const void* A[CP_MAX_N - 1];   // factor of the j-th other mode (cyclic order), row stride RP
};

// Copy factor m of u into a padded table (row stride RP) of type TT.
template <typename TT>
__global__ void table_kernel(const double* __restrict__ A, int64_t I, int R, int RP, TT* __restrict__ out) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < I * RP; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = k / RP;
    const int r = (int)(k - i * RP);
    out[k] = r < R ? (TT)A[i * R + r] : (TT)0;
  }
}

// 16-byte vector types of the factor-row reads.
template <typename TT>
struct VecOf;
template <>
struct VecOf<float> {
  using V = float4;
  static constexpr int kW = 4;
  __device__ static void put(const V& x, float* d) { d[0] = x.x; d[1] = x.y; d[2] = x.z; d[3] = x.w; }
};
template <>
struct VecOf<double> {
  using V = double2;
  static constexpr int kW = 2;
  __device__ static void put(const V& x, double* d) { d[0] = x.x; d[1] = x.y; }
};

// Staged form for R <= 32.  The warp first reads the next 32 nonzeros of its
// unit lane by lane (coalesced values and coordinates, all in flight at
// once); then its G = 32 / R groups of R lanes take those nonzeros in turn,
// kUn per group at a time, each group getting a nonzero's value and
// coordinates from the lane that read them by shuffle and gathering the
// factor rows with lane r reading entry r (one contiguous R-wide read per
// row).  Group g adds the products of its nonzeros in order; the G group
// sums are added in a fixed order at the end.
template <typename TT, int NO, int kUn>
__global__ void __launch_bounds__(256) mttkrp_coo_staged_kernel(const int32_t* __restrict__ other,
                                                                const float* __restrict__ vals, int64_t nnz,
                                                                const int64_t* __restrict__ unit_start,
                                                                int64_t nunits, Tables tab, int R, int RP,
                                                                double* __restrict__ partial) {
  const int lane = threadIdx.x & 31;
  const int64_t unit = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (unit >= nunits) return;
  const int64_t b = unit_start[unit], e = unit_start[unit + 1];
  const int G = 32 / R;
  const int g = lane / R;
  const int r = lane - g * R;
  const bool active = g < G;
  TT acc = (TT)0;
  for (int64_t base = b; base < e; base += 32) {
    const int64_t k = base + lane;
    const bool in = k < e;
    const float vl = in ? vals[k] : 0.f;
    int32_t co[NO];
#pragma unroll
    for (int j = 0; j < NO; ++j) co[j] = in ? other[(int64_t)j * nnz + k] : 0;
    const int cnt = (int)min((int64_t)32, e - base);
    for (int q0 = 0; q0 < cnt; q0 += G * kUn) {
      TT v[kUn], x[kUn][NO];
#pragma unroll
      for (int u = 0; u < kUn; ++u) {
        const int q = q0 + u * G + g;               // this group's nonzero
        const bool use = active && q < cnt;
        // every lane takes part in every shuffle; the predicate applies after
        const float vq = __shfl_sync(0xffffffffu, vl, q & 31);
        v[u] = use ? (TT)vq : (TT)0;
#pragma unroll
        for (int j = 0; j < NO; ++j) {
          const int32_t i = __shfl_sync(0xffffffffu, co[j], q & 31);
          x[u][j] = use ? ((const TT*)tab.A[j])[(int64_t)i * RP + r] : (TT)0;
        }
      }
#pragma unroll
      for (int u = 0; u < kUn; ++u) {
        TT p = v[u];
#pragma unroll
        for (int j = 0; j < NO - 1; ++j) p *= x[u][j];
        acc = fma(p, x[u][NO - 1], acc);
      }
    }
  }
  // add the group sums in order: lane r (group 0) gathers groups 1..G-1
  double s0 = (double)acc;
  for (int q = 1; q < G; ++q) s0 += (double)__shfl_sync(0xffffffffu, acc, (lane + q * R) & 31);
  if (g == 0) partial[unit * R + r] = s0;
}

// Vector-group form.  Each nonzero is handled by LP lanes; lane h of a group
// owns the row entries [h CH, h CH + CH) (CH = NV 16-byte vectors: NV x 4
// FP32 or NV x 2 FP64 values), so a warp instruction gathers 32 / LP rows,
// each as contiguous 16-byte pieces, and all kUn x (N - 1) row reads of a
// lane are issued before its products.  A unit's nonzeros all belong to one
// output row: each lane sums its CH ranks over the nonzeros it took, the
// lanes holding the same ranks are added by a butterfly (a fixed order), and
// lanes 0..LP-1 write the unit's R sums.  Table rows are RP entries apart, RP
// a multiple of 32 bytes, so every vector read stays inside its row.
template <typename TT, int NO, int LP, int NV, int kUn>
__global__ void __launch_bounds__(256) mttkrp_coo_vgroup_kernel(const int32_t* __restrict__ other,
                                                                const float* __restrict__ vals, int64_t nnz,
                                                                const int64_t* __restrict__ unit_start,
                                                                int64_t nunits, Tables tab, int R, int RP,
                                                                double* __restrict__ partial) {
  using VT = VecOf<TT>;
  using V = typename VT::V;
  constexpr int kW = VT::kW, kCh = NV * kW, kNpw = 32 / LP;
  const int lane = threadIdx.x & 31;
  const int64_t unit = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (unit >= nunits) return;
  const int64_t b = unit_start[unit], e = unit_start[unit + 1];
  const int slot = lane / LP;                 // this lane's nonzero within a warp step
  const int h = lane - slot * LP;             // this lane's chunk of ranks
  const bool cols = h * kCh < R;
  TT acc[kCh];
#pragma unroll
  for (int l = 0; l < kCh; ++l) acc[l] = (TT)0;
  for (int64_t k0 = b + slot; k0 < e; k0 += (int64_t)kNpw * kUn) {
    TT v[kUn];
    V x[kUn][NO][NV];
#pragma unroll
    for (int u = 0; u < kUn; ++u) {
      const int64_t k = k0 + (int64_t)u * kNpw;
      const bool in = k < e;
      v[u] = in ? (TT)vals[k] : (TT)0;
#pragma unroll
      for (int j = 0; j < NO; ++j) {
        if (in && cols) {
          const int64_t i = other[(int64_t)j * nnz + k];
          const V* src = reinterpret_cast<const V*>((const TT*)tab.A[j] + i * RP + h * kCh);
#pragma unroll
          for (int q = 0; q < NV; ++q) x[u][j][q] = __ldg(src + q);
        } else {
#pragma unroll
          for (int q = 0; q < NV; ++q) x[u][j][q] = V{};
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kUn; ++u) {
#pragma unroll
      for (int hv = 0; hv < NV; ++hv) {
        TT p[kW], y[kW];
#pragma unroll
        for (int l = 0; l < kW; ++l) p[l] = v[u];
#pragma unroll
        for (int j = 0; j < NO - 1; ++j) {
          VT::put(x[u][j][hv], y);
#pragma unroll
          for (int l = 0; l < kW; ++l) p[l] *= y[l];
        }
        VT::put(x[u][NO - 1][hv], y);
#pragma unroll
        for (int l = 0; l < kW; ++l) acc[hv * kW + l] = fma(p[l], y[l], acc[hv * kW + l]);
      }
    }
  }
  // lanes h, h + LP, h + 2 LP, ... hold the same ranks: butterfly over them
#pragma unroll
  for (int l = 0; l < kCh; ++l) {
#pragma unroll
    for (int o = 16; o >= LP; o >>= 1) acc[l] += __shfl_xor_sync(0xffffffffu, acc[l], o);
  }
  if (lane < LP && cols) {
#pragma unroll
    for (int l = 0; l < kCh; ++l)
      if (h * kCh + l < R) partial[unit * R + h * kCh + l] = (double)acc[l];
  }
}

__global__ void zero_kernel(double* __restrict__ x, int64_t n) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    x[k] = 0.0;
}

// M[seg_row[s], :] = sum of the partials of the units of segment s.
__global__ void coo_finalize_kernel(const int64_t* __restrict__ seg_unit, int64_t nseg,
                                    const int32_t* __restrict__ seg_row, const double* __restrict__ partial,
                                    int R, double* __restrict__ M) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nseg * R; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = k / R;
    const int r = (int)(k - s * R);
    double v = 0.0;
    for (int64_t u = seg_unit[s]; u < seg_unit[s + 1]; ++u) v += partial[u * R + r];
    M[(int64_t)seg_row[s] * R + r] = v;
  }
}

inline int blocks_for(cp_ctx* ctx, int64_t n, int threads = 256) {
  int64_t b = (n + threads - 1) / threads;
  b = std::min<int64_t>(b, 16 * (int64_t)ctx->num_sms);
  return (int)std::max<int64_t>(b, 1);
}

cp_status exclusive_scan(cp_ctx* ctx, const int64_t* in, int64_t* out, int64_t n, int64_t* d_total) {
  const int64_t ntiles = std::max<int64_t>(1, (n + kSortTile - 1) / kSortTile);
  int64_t* sums = nullptr;
  CP_TRY(ws_alloc(ctx, (void**)&sums, sizeof(int64_t) * (size_t)ntiles));
  tile_sum_kernel<<<(unsigned)ntiles, kSortThreads, 0, ctx->stream>>>(in, n, sums);
  CP_LAUNCH_CHECK();
  single_block_scan_kernel<<<1, 1024, 0, ctx->stream>>>(sums, ntiles, d_total);
  CP_LAUNCH_CHECK();
  tile_scan_kernel<<<(unsigned)ntiles, kSortThreads, 0, ctx->stream>>>(in, n, sums, out);
  CP_LAUNCH_CHECK();
  ws_free(ctx, sums);
  return CP_OK;
}

int bits_for(int64_t dim) {
  int b = 0;
  while (b < 63 && (((int64_t)1 << b) < dim)) ++b;
  return b;
}

// Stable sort of perm (identity on entry) by the cyclic key starting at mode n.
cp_status sort_mode(cp_ctx* ctx, const cp_tensor* t, const int64_t* coords, int n, int64_t* perm,
                    int64_t* tmp) {
  const int64_t nnz = t->nnz;
  const int64_t ntiles = (nnz + kSortTile - 1) / kSortTile;
  int64_t* hist = nullptr;
  CP_TRY(ws_alloc(ctx, (void**)&hist, sizeof(int64_t) * (size_t)kBins * ntiles));
  iota_kernel<<<blocks_for(ctx, nnz), 256, 0, ctx->stream>>>(perm, nnz);
  CP_LAUNCH_CHECK();
  int64_t* a = perm;
  int64_t* b = tmp;
  for (int k = t->N - 1; k >= 0; --k) {
    const int c = (n + k) % t->N;
    const int bits = bits_for(t->dims[c]);
    for (int shift = 0; shift < bits; shift += 4) {
      radix_hist_kernel<<<(unsigned)ntiles, kSortThreads, 0, ctx->stream>>>(a, coords, t->N, c, shift, nnz,
                                                                            hist, ntiles);
      CP_LAUNCH_CHECK();
      CP_TRY(exclusive_scan(ctx, hist, hist, (int64_t)kBins * ntiles, nullptr));
      radix_scatter_kernel<<<(unsigned)ntiles, kSortThreads, 0, ctx->stream>>>(a, coords, t->N, c, shift, nnz,
                                                                               hist, ntiles, b);
      CP_LAUNCH_CHECK();
      std::swap(a, b);
    }
  }
  if (a != perm)
    CP_CUDA(cudaMemcpyAsync(perm, a, sizeof(int64_t) * nnz, cudaMemcpyDeviceToDevice, ctx->stream));
  ws_free(ctx, hist);
  return CP_OK;
}

}  // namespace

cp_status coo_build(cp_ctx* ctx, cp_tensor* t, const int64_t* coords, const float* vals) {
  const int64_t nnz = t->nnz;
  const int N = t->N;
  // ||T||^2 over the nonzeros
  {
    double* d = nullptr;
    CP_TRY(ws_alloc(ctx, (void**)&d, sizeof(double)));
    if (nnz > 0) {
      CP_TRY(sumsq(ctx, vals, CP_DTYPE_F32, nnz, d));
      CP_CUDA(cudaMemcpyAsync(ctx->h_pinned, d, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
      CP_CUDA(cudaStreamSynchronize(ctx->stream));
      t->norm2 = ctx->h_pinned[0];
    } else {
      t->norm2 = 0.0;
    }
    ws_free(ctx, d);
  }
  int64_t* d_dims = nullptr;
  CP_TRY(ws_alloc(ctx, (void**)&d_dims, sizeof(int64_t) * CP_MAX_N));
  for (int n = 0; n < N; ++n) ((int64_t*)ctx->h_pinned)[n] = t->dims[n];
  CP_CUDA(cudaMemcpyAsync(d_dims, ctx->h_pinned, sizeof(int64_t) * N, cudaMemcpyHostToDevice, ctx->stream));
  if (nnz > 0) {
    range_check_kernel<<<blocks_for(ctx, nnz * N), 256, 0, ctx->stream>>>(coords, nnz, N, d_dims, ctx->d_status);
    CP_LAUNCH_CHECK();
    CP_TRY(read_status(ctx));
  }
  int64_t* tmp = nullptr;
  int64_t* flag = nullptr;
  CP_TRY(ws_alloc(ctx, (void**)&tmp, sizeof(int64_t) * (size_t)(nnz + 1)));
  CP_TRY(ws_alloc(ctx, (void**)&flag, sizeof(int64_t) * (size_t)(2 * nnz + 2)));
  int64_t* segidx = flag + nnz + 1;
  for (int n = 0; n < N; ++n) {
    CooMode& md = t->modes[n];
    CP_CUDA(cudaMalloc(&md.perm, sizeof(int64_t) * (size_t)std::max<int64_t>(nnz, 1)));
    CP_CUDA(cudaMalloc(&md.vals, sizeof(float) * (size_t)std::max<int64_t>(nnz, 1)));
    CP_CUDA(cudaMalloc(&md.other, sizeof(int32_t) * (size_t)std::max<int64_t>(nnz * (N - 1), 1)));
    if (nnz == 0) {
      md.nseg = 0;
      md.nunits = 0;
      CP_CUDA(cudaMalloc(&md.seg_ptr, sizeof(int64_t)));
      CP_CUDA(cudaMemsetAsync(md.seg_ptr, 0, sizeof(int64_t), ctx->stream));
      CP_CUDA(cudaMalloc(&md.seg_row, sizeof(int32_t)));
      CP_CUDA(cudaMalloc(&md.seg_unit, sizeof(int64_t)));
      CP_CUDA(cudaMemsetAsync(md.seg_unit, 0, sizeof(int64_t), ctx->stream));
      CP_CUDA(cudaMalloc(&md.unit_start, sizeof(int64_t)));
      CP_CUDA(cudaMemsetAsync(md.unit_start, 0, sizeof(int64_t), ctx->stream));
      continue;
    }
    CP_TRY(sort_mode(ctx, t, coords, n, md.perm, tmp));
    if (n == 0) {
      dup_check_kernel<<<blocks_for(ctx, nnz), 256, 0, ctx->stream>>>(md.perm, coords, N, nnz, ctx->d_status);
      CP_LAUNCH_CHECK();
      CP_TRY(read_status(ctx));
    }
    head_flags_kernel<<<blocks_for(ctx, nnz), 256, 0, ctx->stream>>>(md.perm, coords, N, n, nnz, flag);
    CP_LAUNCH_CHECK();
    int64_t* d_total = tmp + nnz;
    CP_TRY(exclusive_scan(ctx, flag, segidx, nnz, d_total));
    CP_CUDA(cudaMemcpyAsync(ctx->h_pinned, d_total, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream));
    CP_CUDA(cudaStreamSynchronize(ctx->stream));
    md.nseg = ((int64_t*)ctx->h_pinned)[0];
    CP_CUDA(cudaMalloc(&md.seg_ptr, sizeof(int64_t) * (size_t)(md.nseg + 1)));
    CP_CUDA(cudaMalloc(&md.seg_row, sizeof(int32_t) * (size_t)md.nseg));
    segments_kernel<<<blocks_for(ctx, nnz), 256, 0, ctx->stream>>>(md.perm, coords, N, n, nnz, flag, segidx,
                                                                   md.seg_ptr, md.seg_row);
    CP_LAUNCH_CHECK();
    ((int64_t*)ctx->h_pinned)[0] = nnz;
    CP_CUDA(cudaMemcpyAsync(md.seg_ptr + md.nseg, ctx->h_pinned, sizeof(int64_t), cudaMemcpyHostToDevice,
                            ctx->stream));
    // work units
    CP_CUDA(cudaMalloc(&md.seg_unit, sizeof(int64_t) * (size_t)(md.nseg + 1)));
    units_count_kernel<<<blocks_for(ctx, md.nseg), 256, 0, ctx->stream>>>(md.seg_ptr, md.nseg, flag);
    CP_LAUNCH_CHECK();
    CP_TRY(exclusive_scan(ctx, flag, md.seg_unit, md.nseg, md.seg_unit + md.nseg));
    CP_CUDA(cudaMemcpyAsync(ctx->h_pinned, md.seg_unit + md.nseg, sizeof(int64_t), cudaMemcpyDeviceToHost,
                            ctx->stream));
    CP_CUDA(cudaStreamSynchronize(ctx->stream));
    md.nunits = ((int64_t*)ctx->h_pinned)[0];
    CP_CUDA(cudaMalloc(&md.unit_start, sizeof(int64_t) * (size_t)(md.nunits + 1)));
    units_fill_kernel<<<blocks_for(ctx, md.nseg), 256, 0, ctx->stream>>>(md.seg_ptr, md.nseg, md.seg_unit,
                                                                         md.unit_start, md.nunits, nnz);
    CP_LAUNCH_CHECK();
    gather_sorted_kernel<<<blocks_for(ctx, nnz), 256, 0, ctx->stream>>>(md.perm, coords, vals, N, n, nnz,
                                                                        md.other, md.vals);
    CP_LAUNCH_CHECK();
  }
  CP_CUDA(cudaStreamSynchronize(ctx->stream));
  ws_free(ctx, flag);
  ws_free(ctx, tmp);
  ws_free(ctx, d_dims);
  return read_status(ctx);
}

void tensor_free_coo(cp_tensor* t) {
  for (int n = 0; n < CP_MAX_N; ++n) {
    CooMode& md = t->modes[n];
    cudaFree(md.perm);
    cudaFree(md.seg_ptr);
    cudaFree(md.seg_row);
    cudaFree(md.other);
    cudaFree(md.vals);
    cudaFree(md.seg_unit);
    cudaFree(md.unit_start);
    md = CooMode();
  }
}

// 16-byte vectors per lane and factor row in the vector-group kernel (one:
// two 16-byte reads of one lane fall into the same 32-byte sector and
// doubled the L1 sector requests, 43.0 against 28.7 us per mode)
constexpr int kVecPerLane = 1;

template <typename TT, int NO>
static cp_status launch_coo(cp_ctx* ctx, const cp_tensor* t, const CooMode& md, const Tables& tab, int R, int RP,
                            double* partial) {
  const int64_t threads = 256;
  const int64_t blocks = (md.nunits * 32 + threads - 1) / threads;
  if (blocks == 0) return CP_OK;
  TimerScope ts(ctx, 2);
  const dim3 g((unsigned)blocks), bl((unsigned)threads);
  if (sizeof(TT) == 8 && R <= 32) {
    // FP64 products: the staged kernel (154 us per mode of the 2e6-nonzero
    // rank-10 tensor against 175 us for the vector groups; FP64 is the bound)
    mttkrp_coo_staged_kernel<TT, NO, 4><<<g, bl, 0, ctx->stream>>>(md.other, md.vals, t->nnz, md.unit_start,
                                                                    md.nunits, tab, R, RP, partial);
  } else {
    // FP32 products (and FP64 above rank 32): the vector groups (28.7 us per
    // mode at 2e6 nonzeros, 2.64 ms at 2e8), lanes per nonzero enough
    // 16-byte chunks for the R ranks, a power of two
    constexpr int NV = kVecPerLane;
    const int ch = NV * 16 / (int)sizeof(TT);
    int LP = 1;
    while (LP * ch < R) LP *= 2;
#define CP_VG(lp) mttkrp_coo_vgroup_kernel<TT, NO, lp, NV, 2><<<g, bl, 0, ctx->stream>>>( \
    md.other, md.vals, t->nnz, md.unit_start, md.nunits, tab, R, RP, partial)
    switch (LP) {
      case 1: CP_VG(1); break;
      case 2: CP_VG(2); break;
      case 4: CP_VG(4); break;
      case 8: CP_VG(8); break;
      case 16: CP_VG(16); break;
      default: CP_VG(32); break;
    }
#undef CP_VG
  }
  CP_LAUNCH_CHECK();
  return CP_OK;
}

template <typename TT>
static cp_status dispatch_coo(cp_ctx* ctx, const cp_tensor* t, const CooMode& md, const Tables& tab, int R,
                              int RP, double* partial) {
  switch (t->N - 1) {
    case 1: return launch_coo<TT, 1>(ctx, t, md, tab, R, RP, partial);
    case 2: return launch_coo<TT, 2>(ctx, t, md, tab, R, RP, partial);
    case 3: return launch_coo<TT, 3>(ctx, t, md, tab, R, RP, partial);
    case 4: return launch_coo<TT, 4>(ctx, t, md, tab, R, RP, partial);
    case 5: return launch_coo<TT, 5>(ctx, t, md, tab, R, RP, partial);
    case 6: return launch_coo<TT, 6>(ctx, t, md, tab, R, RP, partial);
    default: return launch_coo<TT, 7>(ctx, t, md, tab, R, RP, partial);
  }
}

cp_status mttkrp_sparse(cp_ctx* ctx, const cp_tensor* t, const Layout& L, const double* u, int mode,
                        double* out, cp_precision prec) {
  const int R = L.R;
  const int N = t->N;
  const CooMode& md = t->modes[mode];
  // rows without nonzeros are zero (a kernel, so that graph bodies hold kernel nodes only)
  zero_kernel<<<blocks_for(ctx, t->dims[mode] * R), 256, 0, ctx->stream>>>(out, t->dims[mode] * R);
  CP_LAUNCH_CHECK();
  if (t->nnz == 0) return CP_OK;
  const bool f32 = prec != CP_FP64;
  const size_t esz = f32 ? sizeof(float) : sizeof(double);
  // table rows padded to a multiple of 32 bytes (whole sectors per gathered row)
  const int per_sector = (int)(32 / esz);
  const int RP = (R + per_sector - 1) / per_sector * per_sector;
  size_t tab_elems = 0;
  for (int j = 0; j < N - 1; ++j) tab_elems += (size_t)t->dims[(mode + 1 + j) % N] * RP;
  char* tabmem = nullptr;
  double* partial = nullptr;
  CP_TRY(ws_alloc(ctx, (void**)&tabmem, esz * tab_elems + 256));
  CP_TRY(ws_alloc(ctx, (void**)&partial, sizeof(double) * (size_t)md.nunits * R + 16));
  Tables tab;
  size_t off = 0;
  for (int j = 0; j < N - 1; ++j) {
    const int m = (mode + 1 + j) % N;
    void* dst = tabmem + off * esz;
    const int64_t I = t->dims[m];
    if (f32)
      table_kernel<float><<<blocks_for(ctx, I * RP), 256, 0, ctx->stream>>>(u + L.off[m], I, R, RP, (float*)dst);
    else
      table_kernel<double><<<blocks_for(ctx, I * RP), 256, 0, ctx->stream>>>(u + L.off[m], I, R, RP, (double*)dst);
    CP_LAUNCH_CHECK();
    tab.A[j] = dst;
    off += (size_t)I * RP;
  }
  if (f32)
    CP_TRY(dispatch_coo<float>(ctx, t, md, tab, R, RP, partial));
  else
    CP_TRY(dispatch_coo<double>(ctx, t, md, tab, R, RP, partial));
  coo_finalize_kernel<<<blocks_for(ctx, md.nseg * R), 256, 0, ctx->stream>>>(md.seg_unit, md.nseg, md.seg_row,
                                                                             partial, R, out);
  CP_LAUNCH_CHECK();
  ws_free(ctx, partial);
  ws_free(ctx, tabmem);
  return CP_OK;
}

}  // namespace cpg
