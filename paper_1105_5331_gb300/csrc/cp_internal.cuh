// Internal declarations shared by the library's translation units.
// Nothing here is part of the C ABI (include/cp.h is).
#pragma once

#include <cuda_runtime.h>
#include <utility>
#include <cuda_bf16.h>

#include <atomic>
#include <cstdint>
#include <cstdio>
#include <vector>

#include "../../include/cp.h"

#define CP_MAX_N 8
#define CP_MAX_R 64       // largest rank the kernels accept
#define CP_MAX_W 64       // largest N-GMRES window

namespace cpg {

// ---------------------------------------------------------------- errors
void set_error(const char* fmt, ...);
cp_status cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define CP_CUDA(expr)                                                         \
  do {                                                                        \
    cudaError_t e__ = (expr);                                                 \
    if (e__ != cudaSuccess) return cpg::cuda_fail(e__, #expr, __FILE__, __LINE__); \
  } while (0)

extern std::atomic<unsigned long long> g_launches;

#define CP_LAUNCH_CHECK()                                                     \
  do {                                                                        \
    cpg::g_launches.fetch_add(1, std::memory_order_relaxed);                  \
    cudaError_t e__ = cudaGetLastError();                                     \
    if (e__ != cudaSuccess) return cpg::cuda_fail(e__, "kernel launch", __FILE__, __LINE__); \
  } while (0)

#define CP_TRY(expr)                                                          \
  do {                                                                        \
    cp_status s__ = (expr);                                                   \
    if (s__ != CP_OK) return s__;                                             \
  } while (0)

// Device status word: kernels record the first error (cp_status value) they
// meet with atomicCAS; the host reads and clears it at sync points.
__device__ __forceinline__ void record_status(int* st, int code) {
  if (st) atomicCAS(st, 0, code);
}

// Mode bookkeeping of an iterate u = [A^(1); ...; A^(N)].
struct Layout {
  int N = 0;
  int R = 0;
  int64_t dims[CP_MAX_N] = {0};
  int64_t off[CP_MAX_N + 1] = {0};   // element offset of A^(n) in u; off[N] = P
  int64_t P() const { return off[N]; }
  void set(int N_, const int64_t* d, int R_) {
    N = N_;
    R = R_;
    off[0] = 0;
    for (int n = 0; n < N; ++n) {
      dims[n] = d[n];
      off[n + 1] = off[n] + d[n] * R;
    }
  }
};

// Pointers of the factor matrices of one iterate, passed to kernels by value.
struct FactorPtrs {
  const double* A[CP_MAX_N];
  int64_t I[CP_MAX_N];
  int N;
  int R;
};

// Split-K partial sums of one mode's MTTKRP: M[e] = sum_{c < count} p[c * n + e]
// (n = I_mode * R), FP32 or FP64.
struct Parts {
  const void* p = nullptr;
  int count = 0;
  int f32 = 0;
};

// FP32 copy of an iterate for the tensor-core MTTKRP: factor n starts at
// float offset off[n]; its rows are rs = R rounded up to 4 floats apart (16
// bytes, for vector loads) with zero padding.
struct F32Off {
  int64_t off[CP_MAX_N];
  int rs;
};

inline F32Off f32_layout(const Layout& L, int64_t* total) {
  F32Off o{};
  o.rs = (L.R + 3) & ~3;
  int64_t acc = 0;
  for (int n = 0; n < L.N; ++n) {
    o.off[n] = acc;
    acc += L.dims[n] * o.rs;
  }
  *total = acc;
  return o;
}

inline FactorPtrs factor_ptrs(const Layout& L, const double* u) {
  FactorPtrs f;
  f.N = L.N;
  f.R = L.R;
  for (int n = 0; n < CP_MAX_N; ++n) {
    f.A[n] = n < L.N ? u + L.off[n] : nullptr;
    f.I[n] = n < L.N ? L.dims[n] : 0;
  }
  return f;
}

}  // namespace cpg

// ------------------------------------------------------------------ handles
struct cp_ctx {
  int device = 0;
  // solver contexts only: 3-way dense mixed-precision MTTKRP pairs come from
  // a dimension tree (one pass over T for two modes)
  bool dimtree = false;
  void* many = nullptr;             // the cluster engine cp_solve_many keeps between calls
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int num_sms = 0;
  int* d_status = nullptr;          // device status word
  unsigned* d_counter = nullptr;    // last-block counters (zero between kernels): [0] stream, [1] aux
  // Second stream for work that overlaps the MTTKRP (the Gram inverse of
  // the next ALS mode), and the events that fork it from / join it to
  // `stream`; inside a stream capture they become graph edges.
  cudaStream_t aux = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  double* h_pinned = nullptr;       // small pinned host scratch (1024 doubles)
  int* h_pinned_i = nullptr;        // small pinned host scratch (64 ints)
  // Bump arena for workspace while capturing graphs whose bodies may hold
  // only kernel nodes: ws_alloc hands out arena space, ws_free does nothing.
  // With arena_measure set, pointers are placeholders and only the peak
  // offset is recorded.
  bool arena_on = false;
  bool arena_measure = false;
  char* arena_base = nullptr;
  size_t arena_cap = 0;
  size_t arena_off = 0;
  // Kernel timers (cp_ctx_timer_*): CUDA events around the MTTKRP kernels.
  struct KTimer {
    cudaEvent_t a[64], b[64];
    int n = 0;
    double ms = 0.0;
    int count = 0;
    bool made = false;
  };
  bool timing = false;
  KTimer ktimer[3];
};

namespace cpg {

// Brackets one kernel launch on ctx->stream with events when timing is on
// (never inside a stream capture).
struct TimerScope {
  cp_ctx* c;
  int kind;
  bool on = false;
  TimerScope(cp_ctx* ctx, int k) : c(ctx), kind(k) {
    if (!c->timing) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(c->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
    cp_ctx::KTimer& t = c->ktimer[kind];
    if (!t.made) {
      for (int i = 0; i < 64; ++i) {
        cudaEventCreate(&t.a[i]);
        cudaEventCreate(&t.b[i]);
      }
      t.made = true;
    }
    if (t.n == 64) {
      for (int i = 0; i < 64; ++i) {
        float ms = 0.f;
        cudaEventSynchronize(t.b[i]);
        cudaEventElapsedTime(&ms, t.a[i], t.b[i]);
        t.ms += ms;
      }
      t.n = 0;
    }
    cudaEventRecord(t.a[t.n], c->stream);
    on = true;
  }
  ~TimerScope() {
    if (!on) return;
    cp_ctx::KTimer& t = c->ktimer[kind];
    cudaEventRecord(t.b[t.n], c->stream);
    ++t.n;
    ++t.count;
  }
};

}  // namespace cpg

struct cp_ctx_timer_tag {};

struct CooMode {
  int64_t nseg = 0;
  int64_t nunits = 0;
  int64_t* perm = nullptr;       // nnz: position in the input order
  int64_t* seg_ptr = nullptr;    // nseg + 1
  int32_t* seg_row = nullptr;    // nseg: the i_n of each segment
  int64_t* seg_unit = nullptr;   // nseg + 1: first work unit of each segment
  int64_t* unit_start = nullptr; // nunits + 1: first nonzero of each work unit
  int32_t* other = nullptr;      // (N-1) x nnz: other coordinates, cyclic order n+1..n-1
  float* vals = nullptr;         // nnz values in sorted order
};

struct cp_tensor {
  int kind = 0;                  // 0 dense, 1 coo
  int N = 0;
  int device = 0;
  int64_t dims[CP_MAX_N] = {0};
  int64_t K = 0;                 // prod dims (dense)
  double norm2 = 0.0;            // ||T||_F^2
  cp_dtype dtype = CP_DTYPE_F32;
  // dense: per-mode matricised copies T_(n), row-major I_n x Kbar_n
  void* Tn[CP_MAX_N] = {nullptr};
  // dense mixed precision: per-mode bf16 hi/lo planes of T_(n) with a row
  // pitch padded to a multiple of 64 elements (created on first use)
  void* Ttile[CP_MAX_N] = {nullptr};   // mixed precision: pre-tiled bf16 hi / lo planes of T_(n)
  void* tc_state = nullptr;      // tensor maps of the planes (dense_tc.cu)
  // coo
  int64_t nnz = 0;
  CooMode modes[CP_MAX_N];
};

namespace cpg {

inline int64_t kbar(const cp_tensor* t, int n) { return t->K / t->dims[n]; }

// --------------------------------------------------------- kernel entry points
// Dense MTTKRP, FP64 arithmetic.  Writes out (I_n x R).
cp_status mttkrp_dense_f64(cp_ctx* ctx, const cp_tensor* t, const Layout& L, const double* u,
                           int mode, double* out);
// Dense MTTKRP, bf16x3 split products on tcgen05 tensor cores, FP32 accumulate.
cp_status mttkrp_dense_mixed(cp_ctx* ctx, cp_tensor* t, const Layout& L, const double* u,
                             int mode, double* out);
// Mixed MTTKRP of modes first..N-1 into M_all (packed like u).
cp_status mttkrp_dense_mixed_modes(cp_ctx* ctx, cp_tensor* t, const Layout& L, const double* u,
                                   int first, double* M_all);
// Sparse MTTKRP from the mode-sorted copy (FP64 or FP32 products).
cp_status mttkrp_sparse(cp_ctx* ctx, const cp_tensor* t, const Layout& L, const double* u,
                        int mode, double* out, cp_precision prec);
cp_status coo_build(cp_ctx* ctx, cp_tensor* t, const int64_t* d_coords, const float* d_vals);

cp_status mttkrp_any(cp_ctx* ctx, const cp_tensor* t, const Layout& L, const double* u, int mode,
                     double* out, cp_precision prec);
// Khatri-Rao variant MTTKRPs of the listed modes along u + beta d (the
// semantics and out layout of cp_mttkrp_variants).
cp_status mttkrp_variants_any(cp_ctx* ctx, const cp_tensor* t, const Layout& L, const double* u, const double* d,
                              const int* modes, int nmodes, double* out, cp_precision prec);
cp_status mttkrp_dense_mixed_variants(cp_ctx* ctx, cp_tensor* t, const Layout& L, const double* u, const double* d,
                                      const int* modes, int nmodes, double* out);
cp_status mttkrp_tc_variants(cp_ctx* ctx, cp_tensor* t, const Layout& L, const float* a32, const float* d32,
                             const F32Off& o, const int* modes, int nmodes, Parts* out);
bool tc_variants_supported(const Layout& L);
// Dimension tree (3-way dense, mixed precision): W = T x_c A^(c) on the
// tensor cores (in *W), and the MTTKRP of `mode` (one of the two modes other
// than c) from W and the other factor's FP32 copy (u32, f32_layout), summed
// in FP32 and written as FP64.
cp_status prepare_dimtree(cp_ctx* ctx, cp_tensor* t);
cp_status dimtree_w(cp_ctx* ctx, cp_tensor* t, const Layout& L, const float* u32, const F32Off& o32, int contracted,
                    Parts* W);
cp_status dimtree_contract(cp_ctx* ctx, const cp_tensor* t, const Layout& L, const Parts& W, int contracted,
                           int mode, const float* u32, const F32Off& o32, double* out);

// Normalise src (and gsrc) into dst (and gdst); lambda (R) optional.  With
// grams (N x R x R, the Grams of src) the column norms come from their
// diagonals instead of a pass over src.
// With m0_src the M^(1) of src follows the normalisation into m0_dst (its
// columns reordered and scaled by the other modes' scales).
// With grams_out the Grams of dst (from grams), with xi_src / xi_dst the
// inverse of Gammabar^(1) (and its ok flag) follow the normalisation too;
// with ml_src / ml_dst the last mode's M^(N), like M^(1).  dst32
// (nullable): the padded FP32 copy of dst (f32_layout; padding untouched).
cp_status normalize_into(cp_ctx* ctx, const Layout& L, const double* src, double* dst,
                         const double* gsrc, double* gdst, double* lambda, const double* grams = nullptr,
                         const double* m0_src = nullptr, double* m0_dst = nullptr, double* grams_out = nullptr,
                         const double* xi_src = nullptr, double* xi_dst = nullptr, const double* ml_src = nullptr,
                         double* ml_dst = nullptr, float* dst32 = nullptr);

// Window-indexed N-GMRES Step II.  win (device) = {start, m}; window row j
// (oldest first) is ring slot (start + j) % cap.
// With L and colsq, the combine pass also writes the column sums of squares
// of uhat per block, colsq[n][S][R] (S blocks, returned in *S_out; colsq needs
// N x (2 x SMs + 1) x R doubles).
cp_status ngmres_core(cp_ctx* ctx, int64_t P, const int* win, int cap, const double* U,
                      const double* G, const double* ubar, const double* gbar, double eps,
                      double* uhat, double* alpha, const Layout* L = nullptr, double* colsq = nullptr,
                      int* S_out = nullptr);
// Push (u, g) into the window ring (or reset it to {(u, g)}).
cp_status window_update(cp_ctx* ctx, int* win, int cap, bool reset, int64_t P, const double* u,
                        const double* g, double* U, double* G);
// Create the bf16 planes of every mode before graph capture.
cp_status prepare_mixed(cp_ctx* ctx, cp_tensor* t);
// Free every buffer of t in stream order on s and delete the handle.
void tensor_release(cp_tensor* t, cudaStream_t s);
bool on_device(const void* p);
cp_status dense_build(cp_ctx* ctx, cp_tensor* t, const void* d_data);

// Deterministic FP64 dot product: out = x . y (device scalar).
cp_status dot(cp_ctx* ctx, int64_t n, const double* x, const double* y, double* out);
// Device scalar helpers.
cp_status axpy_scalar(cp_ctx* ctx, int64_t n, const double* x0, const double* d,
                      const double* stp, double* x);  // x = x0 + (*stp) d
cp_status sub_vec(cp_ctx* ctx, int64_t n, const double* a, const double* b, double* out);  // a - b

// Full cp_fg with workspace.
cp_status fg_eval(cp_ctx* ctx, const cp_tensor* t, const Layout& L, const double* u, double* f,
                  double* g, cp_precision prec);
// MTTKRP of one mode as split-K partial sums (u32: FP32 copy of u for the
// tensor-core path, may be null otherwise).
cp_status mttkrp_parts(cp_ctx* ctx, cp_tensor* t, const Layout& L, const double* u, const float* u32,
                       const F32Off& o32, int mode, cp_precision prec, Parts* out);
// Gram jobs out = X^T Y (X, Y: I x R row-major; sym: X == Y, both triangles
// written), one launch on stream s; counter: a zeroed last-block counter
// owned by s.
struct GramJob {
  const double* X;
  const double* Y;
  int64_t I;
  double* out;
  int sym;
  const double* D = nullptr;     // optional: both operands read as fma(*stp, D, .)
  const double* stp = nullptr;
};
constexpr int kMaxGramJobs = 3 * CP_MAX_N;
cp_status grams_jobs(cp_ctx* ctx, cudaStream_t s, unsigned* counter, int R, const GramJob* jobs, int njobs);
// Grams A_m^T A_m of modes mode_lo .. mode_lo + nmodes - 1 of u into grams[m].
cp_status grams_of(cp_ctx* ctx, cudaStream_t s, unsigned* counter, const Layout& L, const double* u, int mode_lo,
                   int nmodes, double* grams);
// ALS sweep in place on u: per mode, the Gram inverse on ctx->aux overlapped
// with the MTTKRP, then a row-parallel update.  grams (N x R x R) ends with
// the Grams of the updated factors (grams_valid: it holds u's on entry).
// m0 (nullable): M^(1) of u, used for the first mode instead of an MTTKRP;
// xi0 (nullable): the inverse of u's Gammabar^(1) and its ok flag (R*R
// doubles, then an int), used instead of forming it.
// mlast_out (nullable): receives the last mode's M^(N) (I_N x R), formed
// from the updated modes 1..N-1 and so also M^(N) of the swept point.
// u32_io (nullable): the padded FP32 copy of u (f32_layout), used instead of
// making one and kept up to date with the sweep.
cp_status als_sweep_v2(cp_ctx* ctx, const cp_tensor* t, const Layout& L, double* u, cp_precision prec,
                       double* grams, bool grams_valid, const double* m0 = nullptr, const double* xi0 = nullptr,
                       double* mlast_out = nullptr, float* u32_io = nullptr);
// Inverse of Gammabar^(n) from grams (N x R x R) on stream s into xi (R*R
// doubles, then an int ok flag).
cp_status gram_inverse_launch(cp_ctx* ctx, cudaStream_t s, const double* grams, const Layout& L, int n, double* xi);
// M^(n) supplied to fg_eval_ex instead of MTTKRP passes, per mode
// (nullable): M^(n) itself (nvar = 1), or the Khatri-Rao variants of a
// line search, M^(n)(base + beta d) = sum_v beta^popc(v) m[n][v I_n R + .]
// with beta = *beta (the model is multilinear in the factors).
struct MGiven {
  const double* m[CP_MAX_N] = {};
  int nvar = 1;
  const double* beta = nullptr;
};

// Fused f/g at x = base (+ (*stp) d when d is given; x written); with gd
// (and d) also g . d.
// grams_out: the Grams of the point (N x R x R); m0_out: its M^(1) (I_1 x R);
// mg: modes whose M is supplied instead of an MTTKRP pass (MGiven).
// grams_ls (with d): the Grams of base and d from a line search (ls_poly's
// grams_out); the Grams of x = base + stp d follow from them without a pass
// over the factors.  x32_in (without d): the padded FP32 copy of base,
// used instead of making one.
// grams_in: the Grams of the point when already known (no Gram pass);
// xi0_out: the inverse of its Gammabar^(1) with the ok flag (as
// gram_inverse_launch), formed on the aux stream beside the MTTKRPs.
cp_status fg_eval_ex(cp_ctx* ctx, const cp_tensor* t, const Layout& L, const double* base,
                     const double* d, const double* stp, double* x, double* f, double* g,
                     cp_precision prec, double* gd, double* grams_out = nullptr, double* m0_out = nullptr,
                     const MGiven* mg = nullptr, const double* grams_in = nullptr, double* xi0_out = nullptr,
                     const double* grams_ls = nullptr, const float* x32_in = nullptr);

// Padded FP32 copy (f32_layout) of the packed FP64 iterate u, on ctx->stream.
cp_status f32_copy(cp_ctx* ctx, const Layout& L, const double* u, const F32Off& o, int64_t total, float* out);

// Programmatic dependent launch.  Kernels of the solve start with
// CP_PDL_ENTRY(): wait until the kernel before them in the stream has
// completed and its writes are visible (a no-op when they were launched
// without the attribute), then let the next kernel of the stream begin to
// launch, so that its launch and block scheduling overlap this kernel's run.
// Nothing before the wait touches global memory.
#define CP_PDL_WAIT() asm volatile("griddepcontrol.wait;" ::: "memory")
#define CP_PDL_TRIGGER() asm volatile("griddepcontrol.launch_dependents;" ::: "memory")
#define CP_PDL_ENTRY() \
  do {                 \
    CP_PDL_WAIT();     \
    CP_PDL_TRIGGER();  \
  } while (0)

extern bool g_pdl;   // launch with the programmatic attribute (CP_PDL=0 turns it off)

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args&&... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = g_pdl ? 1 : 0;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

// Workspace (stream-ordered on ctx->stream, or on s for the _on forms).
cp_status ws_alloc(cp_ctx* ctx, void** p, size_t bytes);
void ws_free(cp_ctx* ctx, void* p);
cp_status ws_alloc_on(cp_ctx* ctx, cudaStream_t s, void** p, size_t bytes);
void ws_free_on(cp_ctx* ctx, cudaStream_t s, void* p);

cp_status read_status(cp_ctx* ctx);

// The cluster engine (many.cu).
struct ManyEngine;
void many_engine_destroy(ManyEngine* e);

}  // namespace cpg
