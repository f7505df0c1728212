// Dense MTTKRP on the sm_103a tensor cores (tcgen05), bf16x3 split products
// with FP32 accumulation in tensor memory.
//
// M^(n) = T_(n) Phibar^(n) (Section 2.3, Eq. Gn) is a GEMM with rows i of
// T_(n) (I_n of them), contraction over kbar (prod of the other dims) and R
// columns.  T_(n) is kept as two bf16 planes, hi = bf16(T) and
// lo = bf16(T - hi), so that T ~= hi + lo to about 2^-17 relative.  The
// Khatri-Rao tile KR[kbar, r] = prod_{m != n} A_m[i_m, r] is formed on the fly
// in shared memory from FP32 copies of the factors and split the same way.
// Each 16-deep step issues three MMAs, hi*hi + hi*lo + lo*hi, into an FP32
// accumulator in tensor memory (the lo*lo term, ~2^-18 relative, is
// dropped); successive contraction tiles rotate over up to four accumulators
// that the epilogue adds in registers (see kMaxAcc).
//
// T_(n) is stored pre-tiled: every 128-row x 64-column tile of each plane is
// one contiguous block of rows x 128 bytes, already in the 128-byte-swizzled
// K-major order the tensor cores read (16-byte chunk c of row r at chunk
// c ^ (r & 7)), hi block then lo block, tiles of one column range for all
// row tiles next to each other.  A stage is then filled by two plain bulk
// copies of contiguous memory, which keeps whole DRAM pages in use (a 2-D
// box of 128 rows x 128 bytes from a row-major matrix touches 128 pages).
//
// CTA layout (192 threads, one CTA per SM):
//   warp 0     producer: bulk copies of the hi / lo blocks of one tile per
//              stage into a ring of `stages` shared-memory stages.
//   warp 1     TMEM allocation and the MMA issuer (one thread).
//   warps 2-5  build the Khatri-Rao hi/lo tiles of each stage (SW128,
//              K-major), then drain the accumulators (tcgen05.ld) and write
//              the CTA's partial I x R sums.
// The grid splits the contraction range (split-K) and the rows into 128-row
// groups; one launch may hold the MTTKRPs of several modes (jobs), the CTAs
// shared among them.  The consumers of the per-CTA partial sums add them in
// a fixed order: in FP32 in the solver's kernels (ALS update, f/g finish,
// line-search coefficients, variant sums), in FP64 in the stand-alone
// MTTKRP's reduction.
// Every mbarrier wait is bounded; on a timeout the CTA records
// CP_ERR_TIMEOUT in the device status word and winds down.

#include <algorithm>

#include "cp_internal.cuh"
#include "reduce.cuh"

namespace cpg {

namespace {

constexpr int kBM = 128;                 // rows per M tile = TMEM lanes
constexpr int kBK = 64;                  // contraction elements per tile (128 bytes of bf16)
constexpr int kThreads = 192;
constexpr uint32_t kTileBytes = kBM * kBK * 2;   // one plane, one M tile: 16 KB
constexpr int kMaxTilesPerCta = 1;       // M tiles handled by one CTA
constexpr unsigned long long kWaitNs = 2000000000ull;   // 2 s bound on any wait
constexpr int kMaxDynSmem = 227 * 1024;
// Accumulators per row tile: the MMAs of contraction tile i go into TMEM
// accumulator i % nacc, and the epilogue adds the nacc of them in FP32
// registers (round-to-nearest).  The tensor-core FP32 accumulation loses
// accuracy in proportion to the number of products added into one
// accumulator: measured as ||g_mixed - g_FP64|| / P at a converged 256^3
// R=16 point, the gradient error grew about linearly with a CTA's tiles
// (1.1e-8 at 7, 2.4e-8 at 14, 7.5e-8 at 43 tiles, one accumulator).
constexpr int kMaxAcc = 4;

// One MTTKRP of a launch (a launch may run the MTTKRPs of several modes:
// CTAs cta0 .. cta0 + gx * mgroups - 1 are this job's, gx contraction
// slices per row group).
struct TcJob {
  const uint8_t* tiles;       // pre-tiled hi / lo planes of T_(n)
  int64_t I;
  int64_t Kbar;
  int64_t ktiles;             // total contraction tiles
  int64_t ktiles_per_cta;
  int cta0, gx;
  const float* tab[CP_MAX_N - 1];    // FP32 factors of the other modes, row stride rs
  const float* tabd[CP_MAX_N - 1];   // FP32 D factors (nvar > 1)
  int64_t dimo[CP_MAX_N - 1];
  uint32_t tab_soff[CP_MAX_N - 1];   // offsets (floats) of the tables in shared memory
  uint32_t tabd_soff[CP_MAX_N - 1];
  uint32_t tab_cpy[CP_MAX_N - 1];    // bytes copied per table (multiple of 16)
  uint32_t tab_bytes;                // sum of the copies
  float* partial;                    // [gx][I][outc]
};

struct TcParams {
  int njobs;
  TcJob job[CP_MAX_N];
  int R, RP;
  int ntm;                    // M tiles per CTA
  int stages;
  int nother;
  // Khatri-Rao variants: 1, or 2^nother when the other modes' factors are
  // each either A (bit clear) or D (bit set): column v rs + r of the result
  // is T_(n) times prod_j (bit j of v ? D_j : A_j)[:, r]
  int nvar;
  int outc;                          // output columns: R, or nvar * rs
  int tab_smem;                      // 1: builders read the tables from shared memory
  int rs;                            // table row stride in floats (R rounded up to 4)
  int* status;
  uint32_t ncols;             // TMEM columns allocated
  int nacc;                   // accumulators per row tile (1 .. kMaxAcc)
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t a) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}

__device__ __forceinline__ void mbar_arrive_tx(uint32_t a, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase with the given parity; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity, int* status) {
  if (mbar_try(a, parity)) return true;
  const unsigned long long t0 = gtimer();
  while (!mbar_try(a, parity)) {
    if (gtimer() - t0 > kWaitNs) {
      record_status(status, CP_ERR_TIMEOUT);
      return false;
    }
  }
  return true;
}

// Untiled bulk copy global -> shared (16-byte aligned addresses, size a
// multiple of 16), completing on an mbarrier.
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(dst), "l"((unsigned long long)src), "r"(bytes), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (SBO), descriptor version 1.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;              // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;    // stride byte offset
  d |= (uint64_t)1 << 46;              // version
  d |= (uint64_t)2 << 61;              // SWIZZLE_128B
  return d;
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
      ::"r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

// 16 columns of this warp's 32 TMEM lanes, without waiting for them
// (tcgen05.wait::ld before the registers are read).
__device__ __forceinline__ void tmem_ld16_async(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr)
      : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

template <int NO>
__global__ void __launch_bounds__(kThreads, 1)
    mttkrp_tc_kernel(const __grid_constant__ TcParams p) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* gbase = smem_raw + (base - raw);
  const int S = p.stages;
  const uint32_t b_bytes = (uint32_t)p.RP * 128u;
  const uint32_t stage_bytes = (uint32_t)p.ntm * 2u * kTileBytes + 2u * b_bytes;
  const uint32_t bars = base + (uint32_t)S * stage_bytes;
  auto full_bar = [&](int s) { return bars + 8u * (uint32_t)s; };
  auto empty_bar = [&](int s) { return bars + 8u * (uint32_t)(S + s); };
  const uint32_t done_bar = bars + 16u * (uint32_t)S;
  const uint32_t tab_bar = done_bar + 8u;
  const uint32_t tmem_slot = tab_bar + 8u;
  const uint32_t tab_saddr = (tmem_slot + 8u + 15u) & ~15u;   // factor tables (16-byte aligned)
  volatile uint32_t* tmem_slot_ptr = (volatile uint32_t*)(gbase + (tmem_slot - base));

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  // this CTA's job, contraction slice and row group
  int jb = 0;
  while (jb + 1 < p.njobs && (int)blockIdx.x >= p.job[jb + 1].cta0) ++jb;
  const TcJob& J = p.job[jb];
  const int local = (int)blockIdx.x - J.cta0;
  const int kslice = local % J.gx;
  const int64_t kt0 = (int64_t)kslice * J.ktiles_per_cta;
  const int64_t kt1 = min(J.ktiles, kt0 + J.ktiles_per_cta);
  const int nk = (int)max((int64_t)0, kt1 - kt0);
  const int64_t row0 = (int64_t)(local / J.gx) * (kBM * kMaxTilesPerCta);

  // tile kt of row tile m: hi block (rows x 128 bytes) then lo block, at
  // kt (2 I 128) + m (2 128 128) bytes; stage i of this CTA holds tile kt0 + i
  auto issue_stage = [&](int i) {
    const int s = i % S;
    const int64_t kt = kt0 + i;
    const uint32_t st = base + (uint32_t)s * stage_bytes;
    uint32_t bytes = 0;
    for (int mt = 0; mt < p.ntm; ++mt)
      bytes += 2u * 128u * (uint32_t)max((int64_t)0, min((int64_t)kBM, J.I - (row0 + mt * kBM)));
    mbar_arrive_tx(full_bar(s), bytes);
    for (int mt = 0; mt < p.ntm; ++mt) {
      const int64_t r0 = row0 + mt * kBM;
      if (r0 >= J.I) break;
      const uint32_t blk = 128u * (uint32_t)min((int64_t)kBM, J.I - r0);
      const uint8_t* src = J.tiles + kt * (2 * J.I * 128) + r0 * 256;
      bulk_load(st + (uint32_t)mt * kTileBytes, src, blk, full_bar(s));
      bulk_load(st + (uint32_t)(p.ntm + mt) * kTileBytes, src + blk, blk, full_bar(s));
    }
  };
  // one stage issued before the rest of the set-up (more would queue the
  // factor tables, which the builders need first, behind T: measured slower)
  const int npre = min(1, nk);
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(full_bar(s), 2);
      mbar_init(empty_bar(s), 1);
    }
    mbar_init(done_bar, 1);
    mbar_init(tab_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    fence_proxy_async();
    // the planes of T are never written by a kernel: the first stage streams
    // in while TMEM is allocated and before the wait for the preceding
    // kernel (programmatic dependent launch)
    for (int i = 0; i < npre; ++i) issue_stage(i);
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tmem_slot),
                 "r"(p.ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot_ptr;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      // the factor tables (written by the preceding kernel) once it is done,
      // then the remaining tiles of T
      CP_PDL_WAIT();
      CP_PDL_TRIGGER();
      if (p.tab_smem) {
        mbar_arrive_tx(tab_bar, J.tab_bytes);
#pragma unroll
        for (int j = 0; j < NO; ++j) {
          bulk_load(tab_saddr + 4u * J.tab_soff[j], J.tab[j], J.tab_cpy[j], tab_bar);
          if (p.nvar > 1) bulk_load(tab_saddr + 4u * J.tabd_soff[j], J.tabd[j], J.tab_cpy[j], tab_bar);
        }
      }
      int issued = npre;
      for (int i = npre; i < nk; ++i) {
        const int s = i % S;
        const uint32_t ph = (uint32_t)((i / S) & 1);
        if (!mbar_wait(empty_bar(s), ph ^ 1u, p.status)) break;
        issue_stage(i);
        ++issued;
      }
      // let copies still in flight land before the CTA can exit
      for (int i = max(0, issued - S); i < issued; ++i)
        mbar_wait(full_bar(i % S), (uint32_t)((i / S) & 1), p.status);
      if (p.tab_smem) mbar_wait(tab_bar, 0u, p.status);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(kBM, p.RP);
      for (int i = 0; i < nk; ++i) {
        const int s = i % S;
        const uint32_t ph = (uint32_t)((i / S) & 1);
        if (!mbar_wait(full_bar(s), ph, p.status)) break;
        tc_fence_after();
        const uint32_t st = base + (uint32_t)s * stage_bytes;
        const uint32_t bhi = st + 2u * (uint32_t)p.ntm * kTileBytes;
        const uint32_t blo = bhi + b_bytes;
        for (int mt = 0; mt < p.ntm; ++mt) {
          // accumulator i % nacc of row tile mt; its first tile starts it
          const int a = i % p.nacc;
          const uint32_t d = tmem + (uint32_t)((a * p.ntm + mt) * p.RP);
          const uint32_t ahi = st + (uint32_t)mt * kTileBytes;
          const uint32_t alo = st + (uint32_t)(p.ntm + mt) * kTileBytes;
#pragma unroll
          for (int j = 0; j < kBK / 16; ++j) {
            const uint32_t off = (uint32_t)j * 32u;
            mma_bf16(d, sdesc_sw128(ahi + off), sdesc_sw128(bhi + off), idesc, (i >= p.nacc || j > 0) ? 1u : 0u);
            mma_bf16(d, sdesc_sw128(ahi + off), sdesc_sw128(blo + off), idesc, 1u);
            mma_bf16(d, sdesc_sw128(alo + off), sdesc_sw128(bhi + off), idesc, 1u);
          }
        }
        mma_commit(empty_bar(s));
      }
      mma_commit(done_bar);
    }
  } else {
    // ------------------------------------------------- Khatri-Rao tile builders
    CP_PDL_WAIT();      // the tables may be read from global memory; the epilogue writes it
    CP_PDL_TRIGGER();
    const int t = threadIdx.x - 64;            // 0..127
    const int kk = t & (kBK - 1);              // contraction element within the tile
    const int half = t >> 6;                   // which half of the column groups
    const int rs = p.rs;                       // FP32 table row stride (multiple of 4)
    uint32_t dim32[NO];
#pragma unroll
    for (int j = 0; j < NO; ++j) dim32[j] = (uint32_t)J.dimo[j];
    // four consecutive ranks of table row `ro` (float offset) of mode j: 16-byte
    // loads from shared memory (or through the read-only path when the tables
    // stay in global memory)
    auto ld4 = [&](int j, bool dtab, uint32_t ro) -> float4 {
      if (p.tab_smem) {
        float4 v;
        const uint32_t a = tab_saddr + 4u * ((dtab ? J.tabd_soff[j] : J.tab_soff[j]) + ro);
        asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                     : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                     : "r"(a));
        return v;
      }
      return __ldg(reinterpret_cast<const float4*>((dtab ? J.tabd[j] : J.tab[j]) + ro));
    };
    // column c of the B tile, SW128 K-major: hi = bf16(x), lo = bf16(x - hi)
    auto put = [&](uint8_t* bhi, uint8_t* blo, uint32_t c, float x) {
      const __nv_bfloat16 h = __float2bfloat16_rn(x);
      const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
      const uint32_t off = c * 128u + ((((uint32_t)kk >> 3) ^ (c & 7u)) << 4) + ((uint32_t)kk & 7u) * 2u;
      *(__nv_bfloat16*)(bhi + off) = h;
      *(__nv_bfloat16*)(blo + off) = l;
    };
    if (p.nvar > 1) {
      // padding columns outc .. RP-1 stay zero in every stage
      for (int s = 0; s < S; ++s) {
        uint8_t* bhi = gbase + (size_t)s * stage_bytes + 2u * (uint32_t)p.ntm * kTileBytes;
        for (int r = p.outc + half; r < p.RP; r += 2) put(bhi, bhi + b_bytes, (uint32_t)r, 0.f);
      }
    }
    const bool tabs_ok = !p.tab_smem || mbar_wait(tab_bar, 0u, p.status);
    for (int i = 0; i < nk; ++i) {
      const int s = i % S;
      const uint32_t ph = (uint32_t)((i / S) & 1);
      const bool ok = tabs_ok && mbar_wait(empty_bar(s), ph ^ 1u, p.status);
      if (ok) {
        uint8_t* st = gbase + (size_t)s * stage_bytes;
        uint8_t* bhi = st + 2u * (uint32_t)p.ntm * kTileBytes;
        uint8_t* blo = bhi + b_bytes;
        const int64_t kb64 = (kt0 + i) * kBK + kk;
        const bool in = kb64 < J.Kbar;
        uint32_t rowo[NO];                     // float offset of each factor row
        uint32_t rem = (uint32_t)(in ? kb64 : 0);
#pragma unroll
        for (int j = NO - 1; j >= 0; --j) {
          const uint32_t q = rem / dim32[j];
          rowo[j] = (rem - q * dim32[j]) * (uint32_t)rs;
          rem = q;
        }
        if (NO <= 3 && p.nvar > 1) {
          // all 2^NO products of four ranks by doubling: after mode j the list
          // index holds the A/D choice of modes 0..j in its bits (variants
          // are built for up to 4-way tensors); variant v fills columns
          // v rs .. v rs + rs - 1
          constexpr int V = 1 << (NO <= 3 ? NO : 0);
          const int G = rs >> 2, gh = (G + 1) >> 1;
          const int g1 = min(G, (half + 1) * gh);
          for (int g = half * gh; g < g1; ++g) {
            float4 vals[V];
            vals[0] = in ? make_float4(1.f, 1.f, 1.f, 1.f) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int j = 0; j < (NO <= 3 ? NO : 0); ++j) {
              const float4 a = ld4(j, false, rowo[j] + 4u * g);
              const float4 dd = ld4(j, true, rowo[j] + 4u * g);
#pragma unroll
              for (int q = 0; q < (1 << j); ++q) {
                float4& lo = vals[q];
                float4& up = vals[q + (1 << j)];
                up = make_float4(lo.x * dd.x, lo.y * dd.y, lo.z * dd.z, lo.w * dd.w);
                lo = make_float4(lo.x * a.x, lo.y * a.y, lo.z * a.z, lo.w * a.w);
              }
            }
#pragma unroll
            for (int v = 0; v < V; ++v) {
              const uint32_t c = (uint32_t)(v * rs + 4 * g);
              put(bhi, blo, c, vals[v].x);
              put(bhi, blo, c + 1, vals[v].y);
              put(bhi, blo, c + 2, vals[v].z);
              put(bhi, blo, c + 3, vals[v].w);
            }
          }
        } else {
          // columns in groups of four; groups past the table rows are zero
          const int gh = p.RP >> 3;
#pragma unroll 2
          for (int g = half * gh; g < (half + 1) * gh; ++g) {
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (in && 4 * g < rs) {
              v = ld4(0, false, rowo[0] + 4u * g);
#pragma unroll
              for (int j = 1; j < NO; ++j) {
                const float4 w = ld4(j, false, rowo[j] + 4u * g);
                v = make_float4(v.x * w.x, v.y * w.y, v.z * w.z, v.w * w.w);
              }
            }
            const uint32_t c = 4u * g;
            put(bhi, blo, c, v.x);
            put(bhi, blo, c + 1, v.y);
            put(bhi, blo, c + 2, v.z);
            put(bhi, blo, c + 3, v.w);
          }
        }
      }
      fence_proxy_async();
      // all 128 builders agree on success before the stage is published, so
      // a timeout in one thread stops every builder at the same tile
      uint32_t all_ok;
      asm volatile(
          "{\n\t.reg .pred pin, pout;\n\t"
          "setp.ne.u32 pin, %1, 0;\n\t"
          "bar.red.and.pred pout, 1, 128, pin;\n\t"
          "selp.u32 %0, 1, 0, pout;\n\t}"
          : "=r"(all_ok)
          : "r"((uint32_t)ok)
          : "memory");
      if (!all_ok) break;
      if (t == 0) mbar_arrive(full_bar(s));
    }
    // ------------------------------------------------------------ epilogue
    const bool done = mbar_wait(done_bar, 0u, p.status);
    tc_fence_after();
    const int q = warp & 3;                    // TMEM lane quarter of this warp
    const int64_t rin = q * 32 + lane;
    for (int mt = 0; mt < p.ntm; ++mt) {
      const int64_t row = row0 + mt * kBM + rin;
      for (int c = 0; c < p.RP; c += 16) {
        // the accumulators that received tiles (all of them unless nk < nacc):
        // their loads issued together, one wait
        const int na = min(p.nacc, nk);
        const uint32_t lane_col = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(mt * p.RP + c);
        const uint32_t astep = (uint32_t)(p.ntm * p.RP);
        uint32_t v[kMaxAcc][16];
#pragma unroll
        for (int a = 0; a < kMaxAcc; ++a)
          if (a < na) tmem_ld16_async(lane_col + (uint32_t)a * astep, v[a]);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        float sum[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          float s = 0.f;
#pragma unroll
          for (int a = 0; a < kMaxAcc; ++a)
            if (a < na) s = a == 0 ? __uint_as_float(v[a][e]) : s + __uint_as_float(v[a][e]);
          sum[e] = s;
        }
        if (done && row < J.I && nk > 0) {
          float* out = J.partial + ((int64_t)kslice * J.I + row) * p.outc;
#pragma unroll
          for (int e = 0; e < 16; ++e)
            if (c + e < p.outc) out[c + e] = sum[e];
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(p.ncols) : "memory");
  }
}

// Variant MTTKRPs from the tensor-core partial sums: out[v][i][r] is the
// FP32 sum, over the CTAs in index order, of column v rs + r of row i.
__global__ void variant_sum_kernel(const float* __restrict__ part, int count, int64_t I, int outc, int rs, int R,
                                   int nvar, double* __restrict__ out) {
  CP_PDL_ENTRY();
  const int64_t n = (int64_t)nvar * I * R;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = e / (I * R);
    const int64_t rem = e - v * I * R;
    const int64_t i = rem / R;
    const int r = (int)(rem - i * R);
    out[e] = (double)strided_sum(part + i * outc + v * rs + r, 0, count, 1, I * (int64_t)outc);
  }
}

// Pre-tiled planes: one thread per (column tile kt, row i, 16-byte chunk c)
// writes eight hi and eight lo values, hi = bf16(x), lo = bf16(x - hi),
// zero past Kbar.  Tile (kt, m) starts at kt (2 I 128) + m (2 128 128)
// bytes; its hi block has rows x 128 bytes with chunk c of row r at
// position c ^ (r & 7), and the lo block follows.
template <typename TT>
__global__ void split_tiles_kernel(const TT* __restrict__ src, int64_t I, int64_t Kbar, int64_t ktiles,
                                   uint8_t* __restrict__ out, int transposed = 0) {
  const int64_t total = ktiles * I * 8;
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < total; o += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(o & 7);
    const int64_t ri = o >> 3;
    const int64_t i = ri % I;
    const int64_t kt = ri / I;
    const int64_t m = i / kBM;
    const int r = (int)(i - m * kBM);
    const int64_t rows = min((int64_t)kBM, I - m * kBM);
    uint32_t h[4], l[4];
#pragma unroll
    for (int q = 0; q < 8; q += 2) {
      const int64_t k = kt * kBK + c * 8 + q;
      // element (i, k) of the I x Kbar matrix: row-major, or stored as its
      // transpose (Kbar x I row-major)
      const double x0 = k < Kbar ? (double)(transposed ? src[k * I + i] : src[i * Kbar + k]) : 0.0;
      const double x1 = k + 1 < Kbar ? (double)(transposed ? src[(k + 1) * I + i] : src[i * Kbar + k + 1]) : 0.0;
      const __nv_bfloat16 h0 = __double2bfloat16(x0), h1 = __double2bfloat16(x1);
      const __nv_bfloat16 l0 = __double2bfloat16(x0 - (double)__bfloat162float(h0));
      const __nv_bfloat16 l1 = __double2bfloat16(x1 - (double)__bfloat162float(h1));
      h[q / 2] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
      l[q / 2] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
    }
    uint8_t* tile = out + kt * (2 * I * 128) + m * (2 * kBM * 128);
    const int64_t pos = (int64_t)r * 128 + (int64_t)((c ^ (r & 7)) << 4);
    *reinterpret_cast<uint4*>(tile + pos) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(tile + rows * 128 + pos) = make_uint4(l[0], l[1], l[2], l[3]);
  }
}

struct MixedMode {
  bool ready = false;
};

}  // namespace

// Per-tensor mixed-precision state lives beside the handle (indexed by mode).
struct TcState {
  MixedMode mode[CP_MAX_N];
  // planes of T seen as a matrix for the dimension tree: [0] rows over modes
  // 1..N-1, contraction over mode 0; [1] rows over modes 0..N-2,
  // contraction over mode N-1
  void* gemm_tiles[2] = {nullptr, nullptr};
};

static TcState* tc_state(cp_tensor* t) {
  return reinterpret_cast<TcState*>(t->tc_state);
}

void tensor_free_mixed(cp_tensor* t, cudaStream_t s) {
  for (int n = 0; n < CP_MAX_N; ++n) {
    if (t->Ttile[n]) cudaFreeAsync(t->Ttile[n], s);
    t->Ttile[n] = nullptr;
  }
  if (tc_state(t))
    for (void*& g : tc_state(t)->gemm_tiles)
      if (g) cudaFreeAsync(g, s);
  delete tc_state(t);
  t->tc_state = nullptr;
}

static cp_status ensure_planes(cp_ctx* ctx, cp_tensor* t, int n) {
  if (!t->tc_state) t->tc_state = new TcState();
  MixedMode& mm = tc_state(t)->mode[n];
  if (mm.ready) return CP_OK;
  const int64_t I = t->dims[n];
  const int64_t Kb = kbar(t, n);
  const int64_t ktiles = (Kb + kBK - 1) / kBK;
  const size_t bytes = (size_t)ktiles * 2 * (size_t)I * 128;
  CP_CUDA(cudaMallocAsync(&t->Ttile[n], bytes, ctx->stream));
  const int64_t work = ktiles * I * 8;
  const int64_t blocks = std::min<int64_t>((work + 255) / 256, 16 * (int64_t)ctx->num_sms);
  if (t->dtype == CP_DTYPE_F64)
    split_tiles_kernel<double><<<(unsigned)blocks, 256, 0, ctx->stream>>>((const double*)t->Tn[n], I, Kb, ktiles,
                                                                         (uint8_t*)t->Ttile[n]);
  else
    split_tiles_kernel<float><<<(unsigned)blocks, 256, 0, ctx->stream>>>((const float*)t->Tn[n], I, Kb, ktiles,
                                                                        (uint8_t*)t->Ttile[n]);
  CP_LAUNCH_CHECK();
  mm.ready = true;
  return CP_OK;
}

// Planes of T as the matrix of a dimension-tree GEMM (see TcState): which =
// 0 contracts mode 0 (rows = prod of dims 1..N-1, the transpose of T_(1)),
// which = 1 contracts mode N-1 (rows = prod of dims 0..N-2, T_(1) itself,
// the row-major tensor).
static cp_status ensure_gemm_planes(cp_ctx* ctx, cp_tensor* t, int which) {
  if (!t->tc_state) t->tc_state = new TcState();
  void*& tiles = tc_state(t)->gemm_tiles[which];
  if (tiles) return CP_OK;
  const int64_t K = which == 0 ? t->dims[0] : t->dims[t->N - 1];
  const int64_t rows = t->K / K;
  const int64_t ktiles = (K + kBK - 1) / kBK;
  CP_CUDA(cudaMallocAsync(&tiles, (size_t)ktiles * 2 * (size_t)rows * 128, ctx->stream));
  const int64_t work = ktiles * rows * 8;
  const int64_t blocks = std::min<int64_t>((work + 255) / 256, 16 * (int64_t)ctx->num_sms);
  if (t->dtype == CP_DTYPE_F64)
    split_tiles_kernel<double><<<(unsigned)blocks, 256, 0, ctx->stream>>>((const double*)t->Tn[0], rows, K, ktiles,
                                                                         (uint8_t*)tiles, which == 0);
  else
    split_tiles_kernel<float><<<(unsigned)blocks, 256, 0, ctx->stream>>>((const float*)t->Tn[0], rows, K, ktiles,
                                                                        (uint8_t*)tiles, which == 0);
  CP_LAUNCH_CHECK();
  return CP_OK;
}

typedef void (*TcKernel)(TcParams);

static TcKernel tc_kernel_for(int nother) {
  switch (nother) {
    case 1: return mttkrp_tc_kernel<1>;
    case 2: return mttkrp_tc_kernel<2>;
    case 3: return mttkrp_tc_kernel<3>;
    case 4: return mttkrp_tc_kernel<4>;
    case 5: return mttkrp_tc_kernel<5>;
    case 6: return mttkrp_tc_kernel<6>;
    default: return mttkrp_tc_kernel<7>;
  }
}

static cp_status set_smem_attr() {
  static bool attr_set = false;
  if (!attr_set) {
    for (int no = 1; no <= CP_MAX_N - 1; ++no)
      CP_CUDA(cudaFuncSetAttribute(tc_kernel_for(no), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   kMaxDynSmem));
    attr_set = true;
  }
  return CP_OK;
}

cp_status prepare_mixed(cp_ctx* ctx, cp_tensor* t) {
  if (t->kind != 0) return CP_OK;
  for (int n = 0; n < t->N; ++n) CP_TRY(ensure_planes(ctx, t, n));
  CP_TRY(set_smem_attr());
  CP_CUDA(cudaStreamSynchronize(ctx->stream));
  return CP_OK;
}

cp_status prepare_dimtree(cp_ctx* ctx, cp_tensor* t) {
  if (t->kind != 0 || t->N != 3) return CP_OK;
  CP_TRY(ensure_gemm_planes(ctx, t, 0));
  CP_TRY(ensure_gemm_planes(ctx, t, 1));
  CP_TRY(set_smem_attr());
  CP_CUDA(cudaStreamSynchronize(ctx->stream));
  return CP_OK;
}

// Padded FP32 copy of the factors of u (one launch for all modes).
static cp_status factors_f32(cp_ctx* ctx, const Layout& L, const double* u, float** buf, F32Off* o) {
  int64_t total = 0;
  *o = f32_layout(L, &total);
  CP_TRY(ws_alloc(ctx, (void**)buf, sizeof(float) * (size_t)total + 64));
  return f32_copy(ctx, L, u, *o, total, *buf);
}

static cp_status tc_plan_launch(cp_ctx* ctx, TcParams& p, const int64_t* work, int64_t work_sum,
                                const int64_t* mgroups, size_t tab_max, uint32_t stage_bytes, Parts* parts);

// The MTTKRPs of modes[0..nmodes) in one launch of the tensor-core kernel
// (FP32 factors u32 at offsets o; with nvar > 1 the Khatri-Rao variants of
// u32 and d32); per mode the partial sums (gx x I x outc floats) in parts[k].
// The CTAs (one per SM) are shared among the modes in proportion to their
// tiles of T.
static cp_status mttkrp_tc_multi(cp_ctx* ctx, cp_tensor* t, const Layout& L, const float* u32, const F32Off& o,
                                 const int* modes, int nmodes, Parts* parts, const float* d32 = nullptr,
                                 int nvar = 1) {
  if (nmodes < 1 || nmodes > t->N) {
    set_error("mixed MTTKRP: %d modes in one launch", nmodes);
    return CP_ERR_ARG;
  }
  // the factor tables are bulk-copied and read as float4: 16-byte aligned
  if (((uintptr_t)u32 & 15u) || ((uintptr_t)d32 & 15u)) {
    set_error("mixed MTTKRP: FP32 factor copies must be 16-byte aligned");
    return CP_ERR_ARG;
  }
  for (int k = 0; k < nmodes; ++k) CP_TRY(ensure_planes(ctx, t, modes[k]));
  const int R = L.R;
  const int outc = nvar > 1 ? nvar * o.rs : R;
  const int RP = std::max(16, (outc + 15) / 16 * 16);
  if (RP > 256 || (nvar > 1 && (nvar != (1 << (t->N - 1)) || !d32))) {
    set_error("mixed MTTKRP: %d Khatri-Rao variants of rank %d not supported", nvar, R);
    return CP_ERR_UNSUPPORTED;
  }
  TcParams p{};
  p.njobs = nmodes;
  p.R = R;
  p.RP = RP;
  p.nvar = nvar;
  p.outc = outc;
  p.rs = o.rs;
  p.nother = t->N - 1;
  p.status = ctx->d_status;
  int64_t mtiles_max = 1;
  for (int k = 0; k < nmodes; ++k) mtiles_max = std::max<int64_t>(mtiles_max, (t->dims[modes[k]] + kBM - 1) / kBM);
  p.ntm = (int)std::min<int64_t>(mtiles_max, kMaxTilesPerCta);
  const uint32_t stage_bytes = (uint32_t)p.ntm * 2u * kTileBytes + 2u * (uint32_t)RP * 128u;
  // factor tables of the other modes: bulk-copied to shared memory when they
  // fit (the same choice for every job of the launch)
  size_t tab_max = 0;
  int64_t work[CP_MAX_N], work_sum = 0, mgroups[CP_MAX_N];
  for (int k = 0; k < nmodes; ++k) {
    const int mode = modes[k];
    TcJob& J = p.job[k];
    J.tiles = (const uint8_t*)t->Ttile[mode];
    J.I = t->dims[mode];
    J.Kbar = kbar(t, mode);
    J.ktiles = (J.Kbar + kBK - 1) / kBK;
    size_t tab_bytes = 0;
    int j = 0;
    for (int m = 0; m < t->N; ++m) {
      if (m == mode) continue;
      const uint32_t cpy = (uint32_t)((size_t)t->dims[m] * o.rs * sizeof(float));   // multiple of 16
      J.tab[j] = u32 + o.off[m];
      J.dimo[j] = t->dims[m];
      J.tab_soff[j] = (uint32_t)(tab_bytes / sizeof(float));
      J.tab_cpy[j] = cpy;
      tab_bytes += cpy;
      if (nvar > 1) {
        J.tabd[j] = d32 + o.off[m];
        J.tabd_soff[j] = (uint32_t)(tab_bytes / sizeof(float));
        tab_bytes += cpy;
      }
      ++j;
    }
    J.tab_bytes = (uint32_t)tab_bytes;
    tab_max = std::max(tab_max, tab_bytes);
    const int64_t mt = (J.I + kBM - 1) / kBM;
    mgroups[k] = (mt + kMaxTilesPerCta - 1) / kMaxTilesPerCta;
    work[k] = J.ktiles * mt;
    work_sum += work[k];
  }
  return tc_plan_launch(ctx, p, work, work_sum, mgroups, tab_max, stage_bytes, parts);
}

// Plan and launch the jobs of p (their tiles, sizes and tables set; p's R,
// RP, nvar, outc, rs, nother, status and ntm set): shared-memory stages,
// accumulators, each job's split of its contraction range over its share of
// the SMs, and the per-job partial sums (gx x I x outc floats, in parts).
static cp_status tc_plan_launch(cp_ctx* ctx, TcParams& p, const int64_t* work, int64_t work_sum,
                                const int64_t* mgroups, size_t tab_max, uint32_t stage_bytes, Parts* parts) {
  const int nmodes = p.njobs;
  const int RP = p.RP;
  const int outc = p.outc;
  const int R = p.R;
  const size_t fixed = 1024 + 256 + 64;          // alignment slack, barriers, TMEM slot
  p.tab_smem = (tab_max <= 96 * 1024 && (size_t)kMaxDynSmem >= fixed + tab_max + 2 * (size_t)stage_bytes) ? 1 : 0;
  const size_t avail = (size_t)kMaxDynSmem - fixed - (p.tab_smem ? tab_max : 0);
  p.stages = (int)std::min<size_t>(6, avail / stage_bytes);
  if (p.stages < 2) {
    set_error("mixed MTTKRP: rank %d too large for the shared-memory pipeline", R);
    return CP_ERR_UNSUPPORTED;
  }
  // as many accumulators (up to kMaxAcc) as the 512 TMEM columns hold
  p.nacc = 1;
  while (p.nacc < kMaxAcc && 2 * p.nacc * p.ntm * RP <= 512) p.nacc *= 2;
  uint32_t cols = 32;
  while (cols < (uint32_t)(p.nacc * p.ntm * RP)) cols <<= 1;
  p.ncols = cols;
  // contraction slices per row group: the job's share of the SMs
  int cta = 0;
  for (int k = 0; k < nmodes; ++k) {
    TcJob& J = p.job[k];
    const double share = (double)ctx->num_sms * (double)work[k] / (double)std::max<int64_t>(1, work_sum);
    const int64_t target = std::max<int64_t>(1, (int64_t)(share / (double)mgroups[k]));
    J.ktiles_per_cta = std::max<int64_t>(1, (J.ktiles + target - 1) / target);
    J.gx = (int)((J.ktiles + J.ktiles_per_cta - 1) / J.ktiles_per_cta);
    J.cta0 = cta;
    cta += J.gx * (int)mgroups[k];
  }
  for (int k = 0; k < nmodes; ++k) {
    TcJob& J = p.job[k];
    float* partial = nullptr;
    CP_TRY(ws_alloc(ctx, (void**)&partial, sizeof(float) * (size_t)J.gx * J.I * outc));
    J.partial = partial;
    parts[k] = Parts{partial, J.gx, 1};
  }
  const size_t smem = (size_t)p.stages * stage_bytes + fixed + (p.tab_smem ? tab_max : 0);
  CP_TRY(set_smem_attr());
  {
    TimerScope ts(ctx, 0);
    (void)launch_pdl(tc_kernel_for(p.nother), dim3(cta), dim3(kThreads), smem, ctx->stream, p);
  }
  CP_LAUNCH_CHECK();
  return CP_OK;
}

static cp_status mttkrp_tc_launch(cp_ctx* ctx, cp_tensor* t, const Layout& L, const float* u32, const F32Off& o,
                                  int mode, Parts* parts, const float* d32 = nullptr, int nvar = 1) {
  return mttkrp_tc_multi(ctx, t, L, u32, o, &mode, 1, parts, d32, nvar);
}

static cp_status mttkrp_tc_core(cp_ctx* ctx, cp_tensor* t, const Layout& L, const float* u32, const F32Off& o,
                                int mode, double* out) {
  Parts pt;
  CP_TRY(mttkrp_tc_launch(ctx, t, L, u32, o, mode, &pt));
  CP_TRY(reduce_parts<float>(ctx, (const float*)pt.p, pt.count, L.dims[mode] * L.R, out));
  ws_free(ctx, const_cast<void*>(pt.p));
  return CP_OK;
}

cp_status mttkrp_tc_parts(cp_ctx* ctx, cp_tensor* t, const Layout& L, const float* u32, const F32Off& o, int mode,
                          Parts* out) {
  return mttkrp_tc_launch(ctx, t, L, u32, o, mode, out);
}

cp_status mttkrp_tc_variants(cp_ctx* ctx, cp_tensor* t, const Layout& L, const float* a32, const float* d32,
                             const F32Off& o, const int* modes, int nmodes, Parts* out) {
  return mttkrp_tc_multi(ctx, t, L, a32, o, modes, nmodes, out, d32, 1 << (L.N - 1));
}

bool tc_variants_supported(const Layout& L) {
  if (L.N < 2 || L.N > 4) return false;
  return ((1 << (L.N - 1)) * ((L.R + 3) & ~3) + 15) / 16 * 16 <= 256;
}

cp_status mttkrp_dense_mixed(cp_ctx* ctx, cp_tensor* t, const Layout& L, const double* u, int mode, double* out) {
  float* u32 = nullptr;
  F32Off o;
  CP_TRY(factors_f32(ctx, L, u, &u32, &o));
  CP_TRY(mttkrp_tc_core(ctx, t, L, u32, o, mode, out));
  ws_free(ctx, u32);
  return CP_OK;
}

// Modes first..N-1 into M_all (packed like u), one FP32 conversion of u.
cp_status mttkrp_dense_mixed_modes(cp_ctx* ctx, cp_tensor* t, const Layout& L, const double* u, int first,
                                   double* M_all) {
  float* u32 = nullptr;
  F32Off o;
  CP_TRY(factors_f32(ctx, L, u, &u32, &o));
  for (int n = first; n < L.N; ++n) CP_TRY(mttkrp_tc_core(ctx, t, L, u32, o, n, M_all + L.off[n]));
  ws_free(ctx, u32);
  return CP_OK;
}

// The Khatri-Rao variant MTTKRPs of the listed modes in one tensor-core
// launch (see cp_mttkrp_variants); out holds, per mode, nvar blocks of
// I_mode x R doubles.
cp_status mttkrp_dense_mixed_variants(cp_ctx* ctx, cp_tensor* t, const Layout& L, const double* u, const double* d,
                                      const int* modes, int nmodes, double* out) {
  int64_t acc32 = 0;
  const F32Off o = f32_layout(L, &acc32);
  float *a32 = nullptr, *d32 = nullptr;
  CP_TRY(ws_alloc(ctx, (void**)&a32, sizeof(float) * (size_t)acc32 + 64));
  CP_TRY(ws_alloc(ctx, (void**)&d32, sizeof(float) * (size_t)acc32 + 64));
  CP_TRY(f32_copy(ctx, L, u, o, acc32, a32));
  CP_TRY(f32_copy(ctx, L, d, o, acc32, d32));
  Parts pts[CP_MAX_N];
  CP_TRY(mttkrp_tc_variants(ctx, t, L, a32, d32, o, modes, nmodes, pts));
  const int nvar = 1 << (L.N - 1);
  size_t off = 0;
  for (int k = 0; k < nmodes; ++k) {
    const int64_t I = L.dims[modes[k]];
    const int64_t n = (int64_t)nvar * I * L.R;
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 4 * ctx->num_sms));
    (void)launch_pdl(variant_sum_kernel, dim3(blocks), dim3(256), 0, ctx->stream, (const float*)pts[k].p,
                     pts[k].count, I, nvar * o.rs, o.rs, L.R, nvar, out + off);
    CP_LAUNCH_CHECK();
    off += (size_t)n;
  }
  for (int k = 0; k < nmodes; ++k) ws_free(ctx, const_cast<void*>(pts[k].p));
  ws_free(ctx, d32);
  ws_free(ctx, a32);
  return CP_OK;
}

// ---------------------------------------------------------------------------
// Dimension tree for 3-way tensors: one pass over T makes
//   W = T x_c A^(c)   (I_a x I_b x R, FP32; c the first or the last mode),
// from which the MTTKRPs of the two other modes follow by contracting W with
// one factor each (a = the slower of them in T's order, b the faster):
//   M^(a)[i, r] = sum_j W[i, j, r] F_b[j, r],   M^(b)[j, r] = sum_i W[i, j, r] F_a[i, r],
// the same index sums as Eq. Gn's M^(n) = T_(n) Phibar^(n), regrouped.  W is a
// GEMM (rows (i_a, i_b), contraction i_c, R columns) on the tensor-core
// kernel with the one factor as its Khatri-Rao tile; the contractions run in
// FP64 on W's FP32 values and FP64 factors.
// ---------------------------------------------------------------------------
namespace {

// out[a, r] = sum_b W[a B + b, r] F[b, r] in FP32 (W one FP32 buffer, A B x R;
// F the FP32 factor copy, row stride rs), written as FP64.  One block per a;
// thread t = q R + r takes b = q, q + Q, ... (Q = 256 / R), kU of them with
// all their reads issued before the FMAs; the Q sums of each r are added in
// q order.
constexpr int kContractU = 8;

__global__ void __launch_bounds__(256) contract_fast_kernel(const float* __restrict__ W, int A, int B, int R,
                                                            const float* __restrict__ F, int rs,
                                                            double* __restrict__ out) {
  CP_PDL_ENTRY();
  __shared__ float red[256];
  const int Q = 256 / R;
  const int t = threadIdx.x;
  const int q = t / R, r = t - q * R;
  const int nb = q < Q ? (B - q + Q - 1) / Q : 0;       // this thread's b count
  const int wstep = Q * R, fstep = Q * rs;
  for (int a = blockIdx.x; a < A; a += gridDim.x) {
    const float* wp = W + ((size_t)a * B + q) * R + r;
    const float* fp = F + (size_t)q * rs + r;
    float acc = 0.f;
    for (int k0 = 0; k0 < nb; k0 += kContractU) {
      float w[kContractU], f[kContractU];
#pragma unroll
      for (int u = 0; u < kContractU; ++u) {
        const bool in = k0 + u < nb;
        w[u] = in ? __ldg(wp + (size_t)(k0 + u) * wstep) : 0.f;
        f[u] = in ? __ldg(fp + (size_t)(k0 + u) * fstep) : 0.f;
      }
#pragma unroll
      for (int u = 0; u < kContractU; ++u) acc = fmaf(w[u], f[u], acc);
    }
    red[t] = acc;
    __syncthreads();
    if (t < R) {
      float sum = 0.f;
      for (int k = 0; k < Q; ++k) sum += red[k * R + t];
      out[(size_t)a * R + t] = (double)sum;
    }
    __syncthreads();
  }
}

// out[b, r] = sum_a W[a B + b, r] F[a, r] in FP32, written as FP64.  Block x
// covers 32 consecutive (b, r) elements (one per lane); warp w of 32 takes
// a = w, w + 32, ..., kU of them with all their reads issued before the FMAs;
// the 32 warp sums are added in warp order.
__global__ void __launch_bounds__(1024) contract_slow_kernel(const float* __restrict__ W, int A, int B, int R,
                                                             const float* __restrict__ F, int rs,
                                                             double* __restrict__ out) {
  CP_PDL_ENTRY();
  __shared__ float red[32][33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int BR = B * R;
  const int e = blockIdx.x * 32 + lane;                 // b R + r
  const bool in = e < BR;
  const int r = in ? e % R : 0;
  const int na = in && w < A ? (A - w + 31) / 32 : 0;   // this thread's a count
  const float* wp = W + (size_t)w * BR + e;
  const float* fp = F + (size_t)w * rs + r;
  const size_t wstep = (size_t)32 * BR, fstep = (size_t)32 * rs;
  float acc = 0.f;
  for (int k0 = 0; k0 < na; k0 += kContractU) {
    float x[kContractU], f[kContractU];
#pragma unroll
    for (int u = 0; u < kContractU; ++u) {
      const bool ok = k0 + u < na;
      x[u] = ok ? __ldg(wp + (k0 + u) * wstep) : 0.f;
      f[u] = ok ? __ldg(fp + (k0 + u) * fstep) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < kContractU; ++u) acc = fmaf(x[u], f[u], acc);
  }
  red[w][lane] = acc;
  __syncthreads();
  if (w == 0 && in) {
    float sum = 0.f;
#pragma unroll 8
    for (int k = 0; k < 32; ++k) sum += red[k][lane];
    out[e] = (double)sum;
  }
}

// W = sum of `count` FP32 partials (pitch n) into one FP32 buffer, in order.
__global__ void sum_parts_f32_kernel(const float* __restrict__ part, int count, int64_t n, float* __restrict__ out) {
  CP_PDL_ENTRY();
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int c = 0; c < count; ++c) s += part[(int64_t)c * n + k];
    out[k] = s;
  }
}

}  // namespace

// The dimension tree's GEMM W = T_mat F (rows x K, K x R) as a persistent
// tensor-core kernel: W has many rows and a short contraction (one mode's
// length), so each CTA (one per SM) takes 128-row tiles m = blockIdx.x,
// blockIdx.x + gridDim.x, ... with one TMEM accumulator per tile, two of
// them alternating, so that a tile's epilogue overlaps the next tile's MMAs;
// the B operand (F split into bf16 hi / lo, all nk contraction tiles) is
// built once into shared memory, and the tiles of T stream through a ring of
// stages as in the MTTKRP kernel.  Warps: 0 bulk-copy producer, 1 TMEM and
// MMA issuer, 2-5 B builders and then the epilogue.  Every wait is bounded.
struct GemmParams {
  const uint8_t* tiles;   // pre-tiled hi / lo planes of the rows x K matrix
  int64_t rows;
  int K, nk;              // contraction length and tiles of 64
  const float* F;         // K x rs FP32 (row stride rs floats)
  int rs, R, RP;
  int stages;
  uint32_t ncols;         // TMEM columns (two accumulators of RP)
  float* W;               // rows x R FP32
  int* status;
};
constexpr int kGemmMaxTiles = 8;        // contraction tiles held in shared memory (K <= 512)

__global__ void __launch_bounds__(kThreads, 1) dimtree_gemm_kernel(const __grid_constant__ GemmParams p) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* gbase = smem_raw + (base - raw);
  const uint32_t b_bytes = (uint32_t)p.RP * 128u;     // one plane of one B tile
  const uint32_t btile = 2u * b_bytes;                 // hi then lo (a multiple of 1024 bytes)
  const uint32_t abase = base + (uint32_t)p.nk * btile;
  const uint32_t stage_bytes = 2u * kTileBytes;        // hi then lo A tile
  const int S = p.stages;
  const uint32_t bars = abase + (uint32_t)S * stage_bytes;
  auto full_bar = [&](int s) { return bars + 8u * (uint32_t)s; };
  auto empty_bar = [&](int s) { return bars + 8u * (uint32_t)(S + s); };
  auto accf_bar = [&](int b) { return bars + 16u * (uint32_t)S + 8u * (uint32_t)b; };
  auto acce_bar = [&](int b) { return bars + 16u * (uint32_t)S + 16u + 8u * (uint32_t)b; };
  const uint32_t bready_bar = bars + 16u * (uint32_t)S + 32u;
  const uint32_t tmem_slot = bready_bar + 8u;
  volatile uint32_t* tmem_slot_ptr = (volatile uint32_t*)(gbase + (tmem_slot - base));
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t mtiles = (p.rows + kBM - 1) / kBM;
  const int nm = blockIdx.x < mtiles ? (int)((mtiles - blockIdx.x + gridDim.x - 1) / gridDim.x) : 0;
  // stage i: contraction tile kt = i mod nk of this CTA's row tile i / nk
  auto issue_stage = [&](int i) {
    const int j = i / p.nk, kt = i - (i / p.nk) * p.nk;
    const int s = i % S;
    const int64_t m = blockIdx.x + (int64_t)j * gridDim.x;
    const uint32_t blk = 128u * (uint32_t)min((int64_t)kBM, p.rows - m * kBM);
    const uint32_t st = abase + (uint32_t)s * stage_bytes;
    const uint8_t* src = p.tiles + (int64_t)kt * (2 * p.rows * 128) + m * (2 * kBM * 128);
    mbar_arrive_tx(full_bar(s), 2u * blk);
    bulk_load(st, src, blk, full_bar(s));
    bulk_load(st + kTileBytes, src + blk, blk, full_bar(s));
  };
  const int ntot = nm * p.nk;
  const int npre = min(1, ntot);   // one stage issued before the rest of the set-up

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(accf_bar(b), 1);
      mbar_init(acce_bar(b), 128);
    }
    mbar_init(bready_bar, 128);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    fence_proxy_async();
    // T's planes are never written by a kernel: the first stage streams in
    // while TMEM is allocated and before the wait for the preceding kernel
    for (int i = 0; i < npre; ++i) issue_stage(i);
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tmem_slot),
                 "r"(p.ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot_ptr;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      CP_PDL_WAIT();
      CP_PDL_TRIGGER();
      int issued = npre;
      for (int i = npre; i < ntot; ++i) {
        const int s = i % S;
        if (!mbar_wait(empty_bar(s), (uint32_t)(((i / S) & 1) ^ 1), p.status)) break;
        issue_stage(i);
        ++issued;
      }
      // let copies still in flight land before the CTA can exit
      for (int i = max(0, issued - S); i < issued; ++i)
        mbar_wait(full_bar(i % S), (uint32_t)((i / S) & 1), p.status);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0 && mbar_wait(bready_bar, 0u, p.status)) {
      tc_fence_after();
      const uint32_t idesc = idesc_bf16(kBM, p.RP);
      bool ok = true;
      for (int j = 0; j < nm && ok; ++j) {
        const int buf = j & 1;
        if (!mbar_wait(acce_bar(buf), (uint32_t)(((j >> 1) & 1) ^ 1), p.status)) break;
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(buf * p.RP);
        for (int kt = 0; kt < p.nk; ++kt) {
          const int i = j * p.nk + kt;
          const int s = i % S;
          if (!mbar_wait(full_bar(s), (uint32_t)((i / S) & 1), p.status)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t ahi = abase + (uint32_t)s * stage_bytes;
          const uint32_t alo = ahi + kTileBytes;
          const uint32_t bhi = base + (uint32_t)kt * btile;
          const uint32_t blo = bhi + b_bytes;
#pragma unroll
          for (int q = 0; q < kBK / 16; ++q) {
            const uint32_t off = (uint32_t)q * 32u;
            mma_bf16(d, sdesc_sw128(ahi + off), sdesc_sw128(bhi + off), idesc, (kt > 0 || q > 0) ? 1u : 0u);
            mma_bf16(d, sdesc_sw128(ahi + off), sdesc_sw128(blo + off), idesc, 1u);
            mma_bf16(d, sdesc_sw128(alo + off), sdesc_sw128(bhi + off), idesc, 1u);
          }
          mma_commit(empty_bar(s));
        }
        if (ok) mma_commit(accf_bar(buf));
      }
    }
  } else {
    // --------------------------------------------- B tiles, then the epilogue
    CP_PDL_WAIT();      // F is written by the preceding kernel
    CP_PDL_TRIGGER();
    // thread t takes groups g = t, t + 128, ... of four columns of one
    // contraction element (a 16-byte read of F), eight groups in flight
    const int t = threadIdx.x - 64;              // 0..127
    const int gpr = p.RP >> 2;                   // column groups per contraction element
    const int ngroups = p.nk * kBK * gpr;
    for (int g0 = t; g0 < ngroups; g0 += 128 * 8) {
      float4 v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int g = g0 + 128 * u;
        const int kappa = g / gpr;
        const int c4 = (g - kappa * gpr) * 4;
        v[u] = (g < ngroups && kappa < p.K && c4 < p.rs)
                   ? __ldg(reinterpret_cast<const float4*>(p.F + (int64_t)kappa * p.rs + c4))
                   : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int g = g0 + 128 * u;
        if (g >= ngroups) break;
        const int kappa = g / gpr;
        const int c4 = (g - kappa * gpr) * 4;
        const int kt = kappa / kBK;
        const uint32_t kk = (uint32_t)(kappa - kt * kBK);
        uint8_t* bhi = gbase + (size_t)kt * btile;
        const float xs[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const uint32_t c = (uint32_t)(c4 + q);
          const float x = (int)c < p.R ? xs[q] : 0.f;
          const __nv_bfloat16 h = __float2bfloat16_rn(x);
          const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
          const uint32_t off = c * 128u + (((kk >> 3) ^ (c & 7u)) << 4) + (kk & 7u) * 2u;
          *(__nv_bfloat16*)(bhi + off) = h;
          *(__nv_bfloat16*)(bhi + b_bytes + off) = l;
        }
      }
    }
    fence_proxy_async();
    mbar_arrive(bready_bar);
    const int qd = warp & 3;                     // TMEM lane quarter of this warp
    for (int j = 0; j < nm; ++j) {
      const int buf = j & 1;
      if (!mbar_wait(accf_bar(buf), (uint32_t)((j >> 1) & 1), p.status)) break;
      tc_fence_after();
      const int64_t row = (blockIdx.x + (int64_t)j * gridDim.x) * kBM + qd * 32 + lane;
      for (int c = 0; c < p.RP; c += 16) {
        uint32_t v[16];
        tmem_ld16_async(tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)(buf * p.RP + c), v);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (row < p.rows) {
          float* out = p.W + row * p.R;
#pragma unroll
          for (int e = 0; e < 16; ++e)
            if (c + e < p.R) out[c + e] = __uint_as_float(v[e]);
        }
      }
      tc_fence_before();
      mbar_arrive(acce_bar(buf));
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(p.ncols) : "memory");
  }
}

// W = T x_c A^(c) on the tensor cores: one job, the factor's FP32 copy (row
// stride rs) as its only table; the partial sums (gx x rows x R FP32) in *W.
static cp_status tc_gemm_launch(cp_ctx* ctx, cp_tensor* t, int which, const float* F32, int rs, int R, Parts* W) {
  if ((uintptr_t)F32 & 15u) {
    set_error("dimension tree: FP32 factor copy must be 16-byte aligned");
    return CP_ERR_ARG;
  }
  CP_TRY(ensure_gemm_planes(ctx, t, which));
  const int64_t K = which == 0 ? t->dims[0] : t->dims[t->N - 1];
  const int64_t rows = t->K / K;
  {
    GemmParams g{};
    g.tiles = (const uint8_t*)tc_state(t)->gemm_tiles[which];
    g.rows = rows;
    g.K = (int)K;
    g.nk = (int)((K + kBK - 1) / kBK);
    g.F = F32;
    g.rs = rs;
    g.R = R;
    g.RP = std::max(16, (R + 15) / 16 * 16);
    const size_t btiles = (size_t)g.nk * 2 * g.RP * 128;
    const size_t fixed = 1024 + 256;
    const size_t stages = ((size_t)kMaxDynSmem - fixed - std::min(btiles, (size_t)kMaxDynSmem)) / (2 * kTileBytes);
    if (g.nk <= kGemmMaxTiles && btiles <= 96 * 1024 && stages >= 2) {
      g.stages = (int)std::min<size_t>(6, stages);
      g.ncols = 32;
      while (g.ncols < (uint32_t)(2 * g.RP)) g.ncols <<= 1;
      g.status = ctx->d_status;
      float* Wout = nullptr;
      CP_TRY(ws_alloc(ctx, (void**)&Wout, sizeof(float) * (size_t)rows * R));
      g.W = Wout;
      static bool attr = false;
      if (!attr) {
        CP_CUDA(cudaFuncSetAttribute(dimtree_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem));
        attr = true;
      }
      const int64_t mtiles = (rows + kBM - 1) / kBM;
      const unsigned grid = (unsigned)std::min<int64_t>(mtiles, ctx->num_sms);
      const size_t smem = fixed + btiles + (size_t)g.stages * 2 * kTileBytes;
      {
        TimerScope ts(ctx, 0);
        (void)launch_pdl(dimtree_gemm_kernel, dim3(grid), dim3(kThreads), smem, ctx->stream, g);
      }
      CP_LAUNCH_CHECK();
      *W = Parts{Wout, 1, 1};
      return CP_OK;
    }
  }
  TcParams p{};
  p.njobs = 1;
  p.R = R;
  p.RP = std::max(16, (R + 15) / 16 * 16);
  p.nvar = 1;
  p.outc = R;
  p.rs = rs;
  p.nother = 1;
  p.status = ctx->d_status;
  p.ntm = 1;
  const uint32_t stage_bytes = 2u * kTileBytes + 2u * (uint32_t)p.RP * 128u;
  TcJob& J = p.job[0];
  J.tiles = (const uint8_t*)tc_state(t)->gemm_tiles[which];
  J.I = rows;
  J.Kbar = K;
  J.ktiles = (K + kBK - 1) / kBK;
  J.tab[0] = F32;
  J.dimo[0] = K;
  J.tab_soff[0] = 0;
  J.tab_cpy[0] = (uint32_t)((size_t)K * rs * sizeof(float));
  J.tab_bytes = J.tab_cpy[0];
  const int64_t mg = (rows + kBM - 1) / kBM;
  const int64_t work = J.ktiles * mg;
  return tc_plan_launch(ctx, p, &work, work, &mg, J.tab_cpy[0], stage_bytes, W);
}

cp_status dimtree_w(cp_ctx* ctx, cp_tensor* t, const Layout& L, const float* u32, const F32Off& o32, int contracted,
                    Parts* W) {
  if (t->kind != 0 || t->N != 3 || (contracted != 0 && contracted != 2)) {
    set_error("dimension tree: 3-way dense tensors, first or last mode only");
    return CP_ERR_UNSUPPORTED;
  }
  CP_TRY(tc_gemm_launch(ctx, t, contracted == 0 ? 0 : 1, u32 + o32.off[contracted], o32.rs, L.R, W));
  if (W->count > 1) {
    // the split-K form (contractions too long for the persistent kernel):
    // one FP32 buffer for the contractions
    const int64_t n = t->K / t->dims[contracted] * L.R;
    float* one = nullptr;
    CP_TRY(ws_alloc(ctx, (void**)&one, sizeof(float) * (size_t)n));
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 4 * ctx->num_sms));
    (void)launch_pdl(sum_parts_f32_kernel, dim3(blocks), dim3(256), 0, ctx->stream, (const float*)W->p, W->count, n,
                     one);
    CP_LAUNCH_CHECK();
    ws_free(ctx, const_cast<void*>(W->p));
    *W = Parts{one, 1, 1};
  }
  return CP_OK;
}

cp_status dimtree_contract(cp_ctx* ctx, const cp_tensor* t, const Layout& L, const Parts& W, int contracted,
                           int mode, const float* u32, const F32Off& o32, double* out) {
  // W's rows: (i_a, i_b) with a < b the two modes other than `contracted`
  const int a = contracted == 0 ? 1 : 0;
  const int b = contracted == 2 ? 1 : 2;
  const int64_t A = t->dims[a], B = t->dims[b];
  const int R = L.R;
  if (R > 256 || !W.f32 || W.count != 1 || (int64_t)A * B * R >= ((int64_t)1 << 31)) {
    set_error("dimension tree: rank %d / partials not supported", R);
    return CP_ERR_UNSUPPORTED;
  }
  if (mode == a) {
    const unsigned blocks = (unsigned)std::min<int64_t>(A, 8 * (int64_t)ctx->num_sms);
    (void)launch_pdl(contract_fast_kernel, dim3(blocks), dim3(256), 0, ctx->stream, (const float*)W.p, (int)A, (int)B,
                     R, u32 + o32.off[b], o32.rs, out);
  } else if (mode == b) {
    const unsigned blocks = (unsigned)((B * R + 31) / 32);
    (void)launch_pdl(contract_slow_kernel, dim3(blocks), dim3(1024), 0, ctx->stream, (const float*)W.p, (int)A, (int)B,
                     R, u32 + o32.off[a], o32.rs, out);
  } else {
    set_error("dimension tree: mode %d is not one W serves", mode);
    return CP_ERR_ARG;
  }
  CP_LAUNCH_CHECK();
  return CP_OK;
}

}  // namespace cpg
