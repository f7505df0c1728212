// C ABI (include/cp.h): argument validation, handle management and dispatch
// to the kernels.  No computation happens here.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include <cstdlib>

#include "cp_internal.cuh"
#include "linesearch.cuh"

namespace cpg {

static thread_local char g_err[1024] = "";
std::atomic<unsigned long long> g_launches{0};
bool g_pdl = [] {
  const char* e = getenv("CP_PDL");
  return !(e && e[0] == '0');
}();

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

cp_status cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
  set_error("%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
  return e == cudaErrorMemoryAllocation ? CP_ERR_OOM : CP_ERR_CUDA;
}

cp_status ws_alloc(cp_ctx* ctx, void** p, size_t bytes) { return ws_alloc_on(ctx, ctx->stream, p, bytes); }

void ws_free(cp_ctx* ctx, void* p) { ws_free_on(ctx, ctx->stream, p); }

cp_status ws_alloc_on(cp_ctx* ctx, cudaStream_t s, void** p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (ctx->arena_on) {
    const size_t off = (ctx->arena_off + 255) & ~(size_t)255;
    if (!ctx->arena_measure && off + bytes > ctx->arena_cap) {
      set_error("workspace arena too small (%zu + %zu > %zu)", off, bytes, ctx->arena_cap);
      return CP_ERR_OOM;
    }
    *p = (ctx->arena_measure ? (char*)(uintptr_t)4096 : ctx->arena_base) + off;
    ctx->arena_off = off + bytes;
    return CP_OK;
  }
  cudaError_t e = cudaMallocAsync(p, bytes, s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync(workspace)", __FILE__, __LINE__);
  return CP_OK;
}

void ws_free_on(cp_ctx* ctx, cudaStream_t s, void* p) {
  if (p && !ctx->arena_on) cudaFreeAsync(p, s);
}

cp_status read_status(cp_ctx* ctx) {
  int code = 0;
  CP_CUDA(cudaMemcpyAsync(ctx->h_pinned_i, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost,
                          ctx->stream));
  CP_CUDA(cudaStreamSynchronize(ctx->stream));
  code = ctx->h_pinned_i[0];
  if (code != 0) {
    CP_CUDA(cudaMemsetAsync(ctx->d_status, 0, sizeof(int), ctx->stream));
    CP_CUDA(cudaStreamSynchronize(ctx->stream));
    set_error("device reported status %d", code);
    return (cp_status)code;
  }
  return CP_OK;
}

cp_status dense_build(cp_ctx* ctx, cp_tensor* t, const void* d_data);
cp_status solve_impl(cp_ctx* ctx, const cp_tensor* t, const cp_solve_opts* o, double* u_user,
                     bool user_on_device, cp_solve_report* rep);


void tensor_free_coo(cp_tensor* t);
void tensor_free_mixed(cp_tensor* t, cudaStream_t s);

// Free every buffer of t in stream order on `s` (no device-wide sync) and
// delete the handle.  The caller guarantees no queued work still uses t.
void tensor_release(cp_tensor* t, cudaStream_t s) {
  for (int n = 0; n < CP_MAX_N; ++n)
    if (t->Tn[n]) cudaFreeAsync(t->Tn[n], s);
  tensor_free_mixed(t, s);
  tensor_free_coo(t);
  delete t;
}

bool on_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static cp_status use_device(cp_ctx* ctx) {
  int cur = -1;
  CP_CUDA(cudaGetDevice(&cur));
  if (cur != ctx->device) CP_CUDA(cudaSetDevice(ctx->device));
  return CP_OK;
}

static cp_status check_R(int R) {
  if (R < 1 || R > CP_MAX_R) {
    set_error("rank R = %d outside [1, %d]", R, CP_MAX_R);
    return CP_ERR_ARG;
  }
  return CP_OK;
}

}  // namespace cpg

using namespace cpg;

#define CP_NULLCHECK(p)                                  \
  do {                                                   \
    if (!(p)) {                                          \
      cpg::set_error("%s: null argument '%s'", __func__, #p); \
      return CP_ERR_ARG;                                 \
    }                                                    \
  } while (0)

extern "C" {

const char* cp_last_error(void) { return cpg::g_err; }

unsigned long long cp_kernel_launches(void) { return cpg::g_launches.load(); }

cp_status cp_ctx_create(int device, void* cuda_stream, cp_ctx** out) {
  CP_NULLCHECK(out);
  *out = nullptr;
  int ndev = 0;
  CP_CUDA(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) {
    set_error("device %d not present (%d devices)", device, ndev);
    return CP_ERR_ARG;
  }
  CP_CUDA(cudaSetDevice(device));
  cp_ctx* c = new (std::nothrow) cp_ctx();
  if (!c) return CP_ERR_OOM;
  c->device = device;
  CP_CUDA(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device));
  if (cuda_stream) {
    c->stream = (cudaStream_t)cuda_stream;
  } else {
    CP_CUDA(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
    c->own_stream = true;
  }
  CP_CUDA(cudaMalloc(&c->d_status, sizeof(int)));
  CP_CUDA(cudaMalloc(&c->d_counter, 4 * sizeof(unsigned)));
  CP_CUDA(cudaMemset(c->d_counter, 0, 4 * sizeof(unsigned)));
  CP_CUDA(cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking));
  CP_CUDA(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
  CP_CUDA(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
  CP_CUDA(cudaMemset(c->d_status, 0, sizeof(int)));
  CP_CUDA(cudaMallocHost(&c->h_pinned, sizeof(double) * 1024));
  CP_CUDA(cudaMallocHost(&c->h_pinned_i, sizeof(int) * 64));
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  *out = c;
  return CP_OK;
}

void cp_ctx_destroy(cp_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  if (c->many) cpg::many_engine_destroy(static_cast<cpg::ManyEngine*>(c->many));
  if (c->own_stream) cudaStreamDestroy(c->stream);
  if (c->aux) cudaStreamDestroy(c->aux);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  cudaFree(c->d_status);
  cudaFree(c->d_counter);
  cudaFreeHost(c->h_pinned);
  cudaFreeHost(c->h_pinned_i);
  delete c;
}

cp_status cp_ctx_sync(cp_ctx* c) {
  CP_NULLCHECK(c);
  CP_TRY(use_device(c));
  CP_CUDA(cudaStreamSynchronize(c->stream));
  return read_status(c);
}

void* cp_ctx_stream(cp_ctx* c) { return c ? (void*)c->stream : nullptr; }

cp_status cp_ctx_timer_enable(cp_ctx* c, int enable) {
  CP_NULLCHECK(c);
  CP_TRY(use_device(c));
  CP_CUDA(cudaStreamSynchronize(c->stream));
  c->timing = enable != 0;
  for (auto& t : c->ktimer) {
    t.n = 0;
    t.ms = 0.0;
    t.count = 0;
  }
  return CP_OK;
}

cp_status cp_ctx_timer_read(cp_ctx* c, int which, double* total_ms, int* launches) {
  CP_NULLCHECK(c);
  if (which < 0 || which > 2) {
    set_error("cp_ctx_timer_read: kernel family %d unknown", which);
    return CP_ERR_ARG;
  }
  CP_TRY(use_device(c));
  CP_CUDA(cudaStreamSynchronize(c->stream));
  cp_ctx::KTimer& t = c->ktimer[which];
  for (int i = 0; i < t.n; ++i) {
    float ms = 0.f;
    CP_CUDA(cudaEventElapsedTime(&ms, t.a[i], t.b[i]));
    t.ms += ms;
  }
  t.n = 0;
  if (total_ms) *total_ms = t.ms;
  if (launches) *launches = t.count;
  return CP_OK;
}

cp_status cp_tensor_dense(cp_ctx* ctx, int N, const int64_t* dims, cp_dtype dtype, const void* data,
                          cp_tensor** out) {
  CP_NULLCHECK(ctx);
  CP_NULLCHECK(dims);
  CP_NULLCHECK(data);
  CP_NULLCHECK(out);
  *out = nullptr;
  if (N < 2 || N > CP_MAX_N) {
    set_error("tensor order N = %d outside [2, %d]", N, CP_MAX_N);
    return CP_ERR_ARG;
  }
  if (dtype != CP_DTYPE_F32 && dtype != CP_DTYPE_F64) {
    set_error("unknown dtype %d", (int)dtype);
    return CP_ERR_ARG;
  }
  int64_t K = 1;
  for (int n = 0; n < N; ++n) {
    if (dims[n] < 1 || dims[n] > (int64_t)1 << 31) {
      set_error("dim %d = %lld out of range", n, (long long)dims[n]);
      return CP_ERR_SHAPE;
    }
    if (K > ((int64_t)1 << 40) / dims[n]) {
      set_error("tensor too large");
      return CP_ERR_SHAPE;
    }
    K *= dims[n];
  }
  CP_TRY(use_device(ctx));
  cp_tensor* t = new (std::nothrow) cp_tensor();
  if (!t) return CP_ERR_OOM;
  t->kind = 0;
  t->N = N;
  t->device = ctx->device;
  t->dtype = dtype;
  t->K = K;
  for (int n = 0; n < N; ++n) t->dims[n] = dims[n];
  const size_t bytes = (size_t)K * (dtype == CP_DTYPE_F64 ? 8 : 4);
  const void* src = data;
  void* tmp = nullptr;
  cp_status st = CP_OK;
  if (!on_device(data)) {
    cudaError_t e = cudaMallocAsync(&tmp, bytes, ctx->stream);
    if (e != cudaSuccess) {
      cp_tensor_destroy(t);
      return cuda_fail(e, "cudaMallocAsync(upload)", __FILE__, __LINE__);
    }
    e = cudaMemcpyAsync(tmp, data, bytes, cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) st = cuda_fail(e, "upload", __FILE__, __LINE__);
    src = tmp;
  }
  if (st == CP_OK) st = dense_build(ctx, t, src);
  if (tmp) cudaFreeAsync(tmp, ctx->stream);
  if (st != CP_OK) {
    cp_tensor_destroy(t);
    return st;
  }
  *out = t;
  return CP_OK;
}

cp_status cp_tensor_coo(cp_ctx* ctx, int N, const int64_t* dims, int64_t nnz, const int64_t* coords,
                        const float* vals, cp_tensor** out) {
  CP_NULLCHECK(ctx);
  CP_NULLCHECK(dims);
  CP_NULLCHECK(out);
  *out = nullptr;
  if (N < 2 || N > CP_MAX_N) {
    set_error("tensor order N = %d outside [2, %d]", N, CP_MAX_N);
    return CP_ERR_ARG;
  }
  if (nnz < 0 || nnz > ((int64_t)1 << 31) - 1) {
    set_error("nnz = %lld out of range", (long long)nnz);
    return CP_ERR_SHAPE;
  }
  if (nnz > 0 && (!coords || !vals)) {
    set_error("cp_tensor_coo: null coords/vals with nnz > 0");
    return CP_ERR_ARG;
  }
  for (int n = 0; n < N; ++n)
    if (dims[n] < 1 || dims[n] > ((int64_t)1 << 31) - 1) {
      set_error("dim %d = %lld out of range", n, (long long)dims[n]);
      return CP_ERR_SHAPE;
    }
  CP_TRY(use_device(ctx));
  cp_tensor* t = new (std::nothrow) cp_tensor();
  if (!t) return CP_ERR_OOM;
  t->kind = 1;
  t->N = N;
  t->device = ctx->device;
  t->dtype = CP_DTYPE_F32;
  t->nnz = nnz;
  t->K = 1;
  for (int n = 0; n < N; ++n) t->dims[n] = dims[n];
  const int64_t* dc = coords;
  const float* dv = vals;
  void* tc = nullptr;
  void* tv = nullptr;
  cp_status st = CP_OK;
  if (nnz > 0 && !on_device(coords)) {
    cudaError_t e = cudaMalloc(&tc, sizeof(int64_t) * nnz * N);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(tc, coords, sizeof(int64_t) * nnz * N, cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) st = cuda_fail(e, "upload coords", __FILE__, __LINE__);
    dc = (const int64_t*)tc;
  }
  if (st == CP_OK && nnz > 0 && !on_device(vals)) {
    cudaError_t e = cudaMalloc(&tv, sizeof(float) * nnz);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(tv, vals, sizeof(float) * nnz, cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) st = cuda_fail(e, "upload values", __FILE__, __LINE__);
    dv = (const float*)tv;
  }
  if (st == CP_OK) st = coo_build(ctx, t, dc, dv);
  cudaStreamSynchronize(ctx->stream);
  if (tc) cudaFree(tc);
  if (tv) cudaFree(tv);
  if (st != CP_OK) {
    cp_tensor_destroy(t);
    return st;
  }
  *out = t;
  return CP_OK;
}

cp_status cp_tensor_info(const cp_tensor* t, int* N, int64_t* dims, double* norm2) {
  CP_NULLCHECK(t);
  if (N) *N = t->N;
  if (dims)
    for (int n = 0; n < t->N; ++n) dims[n] = t->dims[n];
  if (norm2) *norm2 = t->norm2;
  return CP_OK;
}

cp_status cp_tensor_sorted_mode(cp_ctx* ctx, const cp_tensor* t, int mode, int64_t* perm,
                                int64_t* seg_ptr, int64_t* seg_row, int64_t* nseg) {
  CP_NULLCHECK(ctx);
  CP_NULLCHECK(t);
  if (t->kind != 1) {
    set_error("cp_tensor_sorted_mode: not a COO tensor");
    return CP_ERR_ARG;
  }
  if (mode < 0 || mode >= t->N) {
    set_error("mode %d outside [0, %d)", mode, t->N);
    return CP_ERR_ARG;
  }
  CP_TRY(use_device(ctx));
  const CooMode& md = t->modes[mode];
  if (nseg) *nseg = md.nseg;
  if (perm && t->nnz > 0)
    CP_CUDA(cudaMemcpyAsync(perm, md.perm, sizeof(int64_t) * t->nnz, cudaMemcpyDeviceToHost, ctx->stream));
  if (seg_ptr)
    CP_CUDA(cudaMemcpyAsync(seg_ptr, md.seg_ptr, sizeof(int64_t) * (md.nseg + 1), cudaMemcpyDeviceToHost,
                            ctx->stream));
  if (seg_row && md.nseg > 0) {
    std::vector<int32_t> rows((size_t)md.nseg);
    CP_CUDA(cudaMemcpyAsync(rows.data(), md.seg_row, sizeof(int32_t) * md.nseg, cudaMemcpyDeviceToHost,
                            ctx->stream));
    CP_CUDA(cudaStreamSynchronize(ctx->stream));
    for (int64_t s = 0; s < md.nseg; ++s) seg_row[s] = rows[(size_t)s];
  }
  CP_CUDA(cudaStreamSynchronize(ctx->stream));
  return CP_OK;
}

void cp_tensor_destroy(cp_tensor* t) {
  if (!t) return;
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != t->device) cudaSetDevice(t->device);
  cudaDeviceSynchronize();
  cpg::tensor_release(t, cudaStreamLegacy);
  cudaStreamSynchronize(cudaStreamLegacy);
}

// The tensor must live on the context's device: its copies are device
// arrays of the device it was created on, and a kernel on another device
// would read that device's memory.
static cp_status check_tensor_R(const cp_ctx* ctx, const cp_tensor* t, int R) {
  CP_NULLCHECK(t);
  if (ctx && t->device != ctx->device) {
    set_error("tensor on device %d, context on device %d", t->device, ctx->device);
    return CP_ERR_ARG;
  }
  return check_R(R);
}

cp_status cp_mttkrp(cp_ctx* ctx, const cp_tensor* t, int R, const double* u, int mode, double* out,
                    cp_precision prec) {
  CP_NULLCHECK(ctx);
  CP_TRY(check_tensor_R(ctx, t, R));
  CP_NULLCHECK(u);
  CP_NULLCHECK(out);
  if (mode < 0 || mode >= t->N) {
    set_error("mode %d outside [0, %d)", mode, t->N);
    return CP_ERR_ARG;
  }
  if (prec != CP_FP64 && prec != CP_MIXED_BF16X3) {
    set_error("unknown precision %d", (int)prec);
    return CP_ERR_ARG;
  }
  CP_TRY(use_device(ctx));
  Layout L;
  L.set(t->N, t->dims, R);
  return mttkrp_any(ctx, t, L, u, mode, out, prec);
}

cp_status cp_mttkrp_variants(cp_ctx* ctx, const cp_tensor* t, int R, const double* u, const double* d,
                             const int* modes, int nmodes, double* out, cp_precision prec) {
  CP_NULLCHECK(ctx);
  CP_TRY(check_tensor_R(ctx, t, R));
  CP_NULLCHECK(u);
  CP_NULLCHECK(d);
  CP_NULLCHECK(modes);
  CP_NULLCHECK(out);
  if (nmodes < 1 || nmodes > t->N) {
    set_error("cp_mttkrp_variants: nmodes = %d outside [1, %d]", nmodes, t->N);
    return CP_ERR_ARG;
  }
  for (int k = 0; k < nmodes; ++k) {
    if (modes[k] < 0 || modes[k] >= t->N) {
      set_error("cp_mttkrp_variants: mode %d outside [0, %d)", modes[k], t->N);
      return CP_ERR_ARG;
    }
    for (int q = 0; q < k; ++q)
      if (modes[q] == modes[k]) {
        set_error("cp_mttkrp_variants: mode %d listed twice", modes[k]);
        return CP_ERR_ARG;
      }
  }
  if (prec != CP_FP64 && prec != CP_MIXED_BF16X3) {
    set_error("unknown precision %d", (int)prec);
    return CP_ERR_ARG;
  }
  CP_TRY(use_device(ctx));
  Layout L;
  L.set(t->N, t->dims, R);
  return mttkrp_variants_any(ctx, t, L, u, d, modes, nmodes, out, prec);
}

cp_status cp_mttkrp_dimtree(cp_ctx* ctx, const cp_tensor* t, int R, const double* u, int contracted, double* out,
                            cp_precision prec) {
  CP_NULLCHECK(ctx);
  CP_TRY(check_tensor_R(ctx, t, R));
  CP_NULLCHECK(u);
  CP_NULLCHECK(out);
  if (t->kind != 0 || t->N != 3 || prec != CP_MIXED_BF16X3) {
    set_error("cp_mttkrp_dimtree: 3-way dense tensors in CP_MIXED_BF16X3 only");
    return CP_ERR_UNSUPPORTED;
  }
  if (contracted != 0 && contracted != 2) {
    set_error("cp_mttkrp_dimtree: contracted mode %d is not 0 or 2", contracted);
    return CP_ERR_ARG;
  }
  CP_TRY(use_device(ctx));
  Layout L;
  L.set(t->N, t->dims, R);
  cp_tensor* tt = const_cast<cp_tensor*>(t);
  int64_t acc32 = 0;
  const F32Off o32 = f32_layout(L, &acc32);
  float* u32 = nullptr;
  CP_TRY(ws_alloc(ctx, (void**)&u32, sizeof(float) * (size_t)acc32 + 64));
  CP_TRY(f32_copy(ctx, L, u, o32, acc32, u32));
  Parts W;
  CP_TRY(dimtree_w(ctx, tt, L, u32, o32, contracted, &W));
  const int a = contracted == 0 ? 1 : 0, b = contracted == 2 ? 1 : 2;
  CP_TRY(dimtree_contract(ctx, t, L, W, contracted, a, u32, o32, out));
  CP_TRY(dimtree_contract(ctx, t, L, W, contracted, b, u32, o32, out + t->dims[a] * R));
  ws_free(ctx, const_cast<void*>(W.p));
  ws_free(ctx, u32);
  return CP_OK;
}

cp_status cp_fg(cp_ctx* ctx, const cp_tensor* t, int R, const double* u, double* f, double* g,
                cp_precision prec) {
  CP_NULLCHECK(ctx);
  CP_TRY(check_tensor_R(ctx, t, R));
  CP_NULLCHECK(u);
  CP_NULLCHECK(f);
  CP_TRY(use_device(ctx));
  Layout L;
  L.set(t->N, t->dims, R);
  return fg_eval(ctx, t, L, u, f, g, prec);
}

cp_status cp_als_sweep(cp_ctx* ctx, const cp_tensor* t, int R, double* u, int normalize,
                       cp_precision prec) {
  CP_NULLCHECK(ctx);
  CP_TRY(check_tensor_R(ctx, t, R));
  CP_NULLCHECK(u);
  CP_TRY(use_device(ctx));
  Layout L;
  L.set(t->N, t->dims, R);
  double* grams = nullptr;
  CP_TRY(ws_alloc(ctx, (void**)&grams, sizeof(double) * (size_t)t->N * R * R));
  CP_TRY(als_sweep_v2(ctx, t, L, u, prec, grams, false));
  if (normalize) {
    double* tmp = nullptr;
    CP_TRY(ws_alloc(ctx, (void**)&tmp, sizeof(double) * (size_t)L.P()));
    CP_CUDA(cudaMemcpyAsync(tmp, u, sizeof(double) * L.P(), cudaMemcpyDeviceToDevice, ctx->stream));
    CP_TRY(normalize_into(ctx, L, tmp, u, nullptr, nullptr, nullptr, grams));
    ws_free(ctx, tmp);
  }
  ws_free(ctx, grams);
  return CP_OK;
}

cp_status cp_normalize(cp_ctx* ctx, int N, const int64_t* dims, int R, double* u, double* g,
                       double* lambda) {
  CP_NULLCHECK(ctx);
  CP_NULLCHECK(dims);
  CP_NULLCHECK(u);
  CP_TRY(check_R(R));
  if (N < 2 || N > CP_MAX_N) {
    set_error("order N = %d outside [2, %d]", N, CP_MAX_N);
    return CP_ERR_ARG;
  }
  for (int n = 0; n < N; ++n)
    if (dims[n] < 1) {
      set_error("dim %d < 1", n);
      return CP_ERR_SHAPE;
    }
  CP_TRY(use_device(ctx));
  Layout L;
  L.set(N, dims, R);
  const int64_t P = L.P();
  double* tmp = nullptr;
  CP_TRY(ws_alloc(ctx, (void**)&tmp, sizeof(double) * (size_t)P * 2));
  CP_CUDA(cudaMemcpyAsync(tmp, u, sizeof(double) * P, cudaMemcpyDeviceToDevice, ctx->stream));
  if (g) CP_CUDA(cudaMemcpyAsync(tmp + P, g, sizeof(double) * P, cudaMemcpyDeviceToDevice, ctx->stream));
  CP_TRY(normalize_into(ctx, L, tmp, u, g ? tmp + P : nullptr, g, lambda));
  ws_free(ctx, tmp);
  return CP_OK;
}

cp_status ngmres_step(cp_ctx* ctx, int64_t Pn, int m, const double* U, const double* G,
                      const double* ubar, const double* gbar, double eps, double* uhat,
                      double* alpha) {
  CP_NULLCHECK(ctx);
  CP_NULLCHECK(U);
  CP_NULLCHECK(G);
  CP_NULLCHECK(ubar);
  CP_NULLCHECK(gbar);
  CP_NULLCHECK(uhat);
  if (Pn < 1) {
    set_error("ngmres_step: P = %lld < 1", (long long)Pn);
    return CP_ERR_ARG;
  }
  if (m < 1 || m > CP_MAX_W) {
    set_error("ngmres_step: m = %d outside [1, %d]", m, CP_MAX_W);
    return CP_ERR_ARG;
  }
  if (!(eps >= 0.0)) {
    set_error("ngmres_step: eps must be >= 0");
    return CP_ERR_ARG;
  }
  CP_TRY(use_device(ctx));
  int* win = nullptr;
  CP_TRY(ws_alloc(ctx, (void**)&win, sizeof(int) * 2));
  ctx->h_pinned_i[8] = 0;
  ctx->h_pinned_i[9] = m;
  CP_CUDA(cudaMemcpyAsync(win, ctx->h_pinned_i + 8, sizeof(int) * 2, cudaMemcpyHostToDevice, ctx->stream));
  const cp_status st = ngmres_core(ctx, Pn, win, m, U, G, ubar, gbar, eps, uhat, alpha);
  ws_free(ctx, win);
  // the pinned staging slot must not be reused before the copy has run
  CP_CUDA(cudaStreamSynchronize(ctx->stream));
  return st;
}

void cp_ls_opts_default(cp_ls_opts* o) {
  if (!o) return;
  o->ftol = 1e-4;
  o->gtol = 1e-2;
  o->xtol = 1e-15;
  o->stpmin = 1e-15;
  o->stpmax = 1e15;
  o->stp0 = 1.0;
  o->maxfev = 20;
}

cp_status linesearch(cp_ctx* ctx, const cp_tensor* t, int R, const double* x0, double f0,
                     const double* g0, const double* d, const cp_ls_opts* opts, double* x,
                     double* f, double* g, double* stp, int* nfev, int* info, cp_precision prec) {
  CP_NULLCHECK(ctx);
  CP_TRY(check_tensor_R(ctx, t, R));
  CP_NULLCHECK(x0);
  CP_NULLCHECK(g0);
  CP_NULLCHECK(d);
  CP_NULLCHECK(x);
  CP_NULLCHECK(g);
  CP_TRY(use_device(ctx));
  cp_ls_opts o;
  if (opts)
    o = *opts;
  else
    cp_ls_opts_default(&o);
  if (o.maxfev < 1 || !(o.ftol > 0) || !(o.gtol > 0) || !(o.stpmin >= 0) || !(o.stpmax > o.stpmin)) {
    set_error("linesearch: bad options");
    return CP_ERR_ARG;
  }
  Layout L;
  L.set(t->N, t->dims, R);
  const int64_t P = L.P();
  (void)f0;
  (void)g0;
  double* sc = nullptr;
  CP_TRY(ws_alloc(ctx, (void**)&sc, sizeof(double) * 40 + sizeof(MTState) + 64));
  MTState* st = (MTState*)(((uintptr_t)(sc + 40) + 63) & ~(uintptr_t)63);
  CP_TRY(ls_poly(ctx, t, L, x0, d, prec, o, st, sc + 4, nullptr, cudaGraphConditionalHandle{}, 0));
  // the final point, evaluated directly
  CP_TRY(axpy_scalar(ctx, P, x0, d, &st->stp_eval, x));
  CP_TRY(fg_eval(ctx, t, L, x, sc, g, prec));
  MTState* hs = (MTState*)(ctx->h_pinned + 16);
  CP_CUDA(cudaMemcpyAsync(hs, st, sizeof(MTState), cudaMemcpyDeviceToHost, ctx->stream));
  CP_CUDA(cudaMemcpyAsync(ctx->h_pinned, sc, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CP_CUDA(cudaStreamSynchronize(ctx->stream));
  const MTState ms = *hs;
  const double fx = ctx->h_pinned[0];
  ws_free(ctx, sc);
  CP_TRY(read_status(ctx));
  if (ms.info == -1) {
    set_error("linesearch: phi'(0) = g0^T d = %g is not negative", ms.g0);
    return CP_ERR_LINESEARCH;
  }
  if (f) *f = fx;
  if (stp) *stp = ms.stp_eval;
  if (nfev) *nfev = ms.nfev;
  if (info) *info = ms.info;
  return CP_OK;
}

void cp_solve_opts_default(cp_solve_opts* o, int R) {
  if (!o) return;
  o->R = R;
  o->w = 20;
  o->maxit = 10000;
  o->tol = 1e-7;
  o->eps = 1e-12;
  o->prec = CP_FP64;
  o->polish = 1;
  o->mixed_tol_factor = 1.0;
  cp_ls_opts_default(&o->ls);
  o->mixed_maxfev = 0;
  o->dimtree = -1;
  o->mixed_stall = 0;
  o->mixed_min_entries = 0;
}

cp_status cp_solve(cp_ctx* ctx, const cp_tensor* t, const cp_solve_opts* opts, double* u,
                   cp_solve_report* rep) {
  CP_NULLCHECK(ctx);
  CP_NULLCHECK(opts);
  CP_TRY(check_tensor_R(ctx, t, opts->R));
  CP_NULLCHECK(u);
  if (opts->w < 1 || opts->w > CP_MAX_W) {
    set_error("cp_solve: window w = %d outside [1, %d]", opts->w, CP_MAX_W);
    return CP_ERR_ARG;
  }
  if (opts->maxit < 0 || !(opts->tol > 0) || !(opts->eps >= 0)) {
    set_error("cp_solve: bad maxit/tol/eps");
    return CP_ERR_ARG;
  }
  if (opts->prec != CP_FP64 && opts->prec != CP_MIXED_BF16X3) {
    set_error("cp_solve: unknown precision %d", (int)opts->prec);
    return CP_ERR_ARG;
  }
  CP_TRY(use_device(ctx));
  return solve_impl(ctx, t, opts, u, on_device(u), rep);
}

}  // extern "C"
