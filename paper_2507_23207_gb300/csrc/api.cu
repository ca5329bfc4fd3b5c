// C ABI edge: context management, argument validation, error translation, and
// the primitive entry points (factors, Philox words, sketches, QR, multi-TTM).
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "common.cuh"
#include "pipeline.h"

struct krp_ctx_s {
  krp::Ctx c;
};

namespace krp {

static thread_local Ctx* g_current = nullptr;

Ctx* current() { return g_current; }
cudaStream_t stream() { return g_current->stream; }

void fail(krp_status s, const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  throw Error{s, std::string(buf)};
}

void note_launch(const char*) {
  if (g_current) ++g_current->launches;
}

static cudaEvent_t trace_event(Ctx* c) {
  const size_t i = c->trace.size();
  while (c->trace_pool.size() <= i) {
    cudaEvent_t e;
    KRP_CUDA_CHECK(cudaEventCreate(&e));
    c->trace_pool.push_back(e);
  }
  return c->trace_pool[i];
}

void check_launch(const char* name) {
  note_launch(name);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) fail(KRP_ECUDA, "launch of %s failed: %s", name, cudaGetErrorString(e));
  Ctx* c = g_current;
  if (c && c->trace_on) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(c->stream, &cs);
    if (cs == cudaStreamCaptureStatusNone) {
      cudaEvent_t ev = trace_event(c);
      KRP_CUDA_CHECK(cudaEventRecord(ev, c->stream));
      c->trace.push_back({name, ev, c->stream});
    }
  }
}

void trace_marker() {
  Ctx* c = g_current;
  if (c && c->trace_on) {
    cudaEvent_t ev = trace_event(c);
    KRP_CUDA_CHECK(cudaEventRecord(ev, c->stream));
    c->trace.push_back({nullptr, ev, c->stream});
  }
}

void ensure_workspace(Ctx* c, size_t bytes) {
  bytes = (bytes + (size_t(1) << 20)) & ~((size_t(1) << 20) - 1);
  // the second stream's work of an earlier call (joined into the context's
  // stream on success; possibly still running after an error) must not see
  // its workspace handed out again
  if (c->side_stream) KRP_CUDA_CHECK(cudaStreamSynchronize(c->side_stream));
  c->ws.off = 0;
  if (c->ws.cap >= bytes) return;
  if (c->ws.base) {
    KRP_CUDA_CHECK(cudaStreamSynchronize(c->stream));
    KRP_CUDA_CHECK(cudaFree(c->ws.base));
    c->ws.base = nullptr;
    c->ws.cap = 0;
  }
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    fail(KRP_ENOMEM, "workspace allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
  }
  c->ws.base = static_cast<char*>(p);
  c->ws.cap = bytes;
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

size_t dtype_size(krp_dtype t) {
  switch (t) {
    case KRP_F32: return 4;
    case KRP_BF16: return 2;
    case KRP_F64: return 8;
    case KRP_FP8_E4M3: return 1;
    case KRP_BF16X2: return 4;
  }
  return 0;
}

int64_t checked_numel(int d, const int64_t* dims) {
  KRP_REQUIRE(dims != nullptr, "dims is NULL");
  int64_t n = 1;
  for (int j = 0; j < d; ++j) {
    KRP_REQUIRE(dims[j] >= 1, "dims[%d] = %lld must be >= 1", j, (long long)dims[j]);
    KRP_REQUIRE(n <= (int64_t(1) << 62) / dims[j], "tensor too large");
    n *= dims[j];
  }
  return n;
}

// Runs `body` with ctx as the current context and converts errors.
template <class F>
static krp_status guarded(krp_ctx ctx, F&& body) {
  if (!ctx) return KRP_EINVAL;
  Ctx* c = &ctx->c;
  Ctx* prev = g_current;
  g_current = c;
  krp_status st = KRP_OK;
  try {
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess || cur != c->device) {
      cudaGetLastError();
      KRP_CUDA_CHECK(cudaSetDevice(c->device));
    }
    body();
    c->last_error.clear();
  } catch (const Error& e) {
    c->last_error = e.msg;
    st = e.status;
  } catch (const std::bad_alloc&) {
    c->last_error = "host allocation failed";
    st = KRP_ENOMEM;
  } catch (...) {
    c->last_error = "unexpected internal error";
    st = KRP_ECUDA;
  }
  g_current = prev;
  return st;
}

}  // namespace krp

using namespace krp;

extern "C" {

krp_status krp_create(krp_ctx* out, int device, void* cuda_stream) {
  if (!out) return KRP_EINVAL;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess) {
    cudaGetLastError();
    return KRP_ECUDA;
  }
  if (device < 0 || device >= n) return KRP_EINVAL;
  krp_ctx ctx = new (std::nothrow) krp_ctx_s();
  if (!ctx) return KRP_ENOMEM;
  ctx->c.device = device;
  ctx->c.stream = static_cast<cudaStream_t>(cuda_stream);
  krp_status st = guarded(ctx, [&] {
    KRP_CUDA_CHECK(cudaDeviceGetAttribute(&ctx->c.num_sms, cudaDevAttrMultiProcessorCount, device));
    void* p = nullptr;
    KRP_CUDA_CHECK(cudaMalloc(&p, 256));
    ctx->c.d_status = static_cast<int*>(p);
    KRP_CUDA_CHECK(cudaMemset(ctx->c.d_status, 0, 256));
  });
  if (st != KRP_OK) {
    delete ctx;
    return st;
  }
  *out = ctx;
  return KRP_OK;
}

krp_status krp_destroy(krp_ctx ctx) {
  if (!ctx) return KRP_EINVAL;
  krp_status st = guarded(ctx, [&] {
    KRP_CUDA_CHECK(cudaStreamSynchronize(ctx->c.stream));
    for (cudaEvent_t e : ctx->c.trace_pool) cudaEventDestroy(e);
    ctx->c.trace_pool.clear();
    for (cudaEvent_t e : ctx->c.copy_events) cudaEventDestroy(e);
    ctx->c.copy_events.clear();
    if (ctx->c.copy_stream) cudaStreamDestroy(ctx->c.copy_stream);
    ctx->c.copy_stream = nullptr;
    for (cudaEvent_t& e : ctx->c.side_events) {
      if (e) cudaEventDestroy(e);
      e = nullptr;
    }
    if (ctx->c.side_stream) {
      cudaStreamSynchronize(ctx->c.side_stream);
      cudaStreamDestroy(ctx->c.side_stream);
    }
    ctx->c.side_stream = nullptr;
    if (ctx->c.batch_plan) ctx->c.batch_plan_free(ctx->c.batch_plan);
    ctx->c.batch_plan = nullptr;
    if (ctx->c.hankel_plan) ctx->c.hankel_plan_free(ctx->c.hankel_plan);
    ctx->c.hankel_plan = nullptr;
    if (ctx->c.ws.base) KRP_CUDA_CHECK(cudaFree(ctx->c.ws.base));
    if (ctx->c.d_status) KRP_CUDA_CHECK(cudaFree(ctx->c.d_status));
    ctx->c.ws.base = nullptr;
    ctx->c.d_status = nullptr;
  });
  delete ctx;
  return st;
}

krp_status krp_set_stream(krp_ctx ctx, void* cuda_stream) {
  return guarded(ctx, [&] { ctx->c.stream = static_cast<cudaStream_t>(cuda_stream); });
}

krp_status krp_set_wait_limit(krp_ctx ctx, uint64_t ns) {
  return guarded(ctx, [&] {
    // the limit sits beside the status word (bytes 8..15 of that block);
    // ordered with the context's later kernels by its stream
    KRP_CUDA_CHECK(cudaMemcpyAsync(ctx->c.d_status + 2, &ns, sizeof(ns), cudaMemcpyHostToDevice,
                                   ctx->c.stream));
    KRP_CUDA_CHECK(cudaStreamSynchronize(ctx->c.stream));
  });
}

const char* krp_last_error(krp_ctx ctx) { return ctx ? ctx->c.last_error.c_str() : "null context"; }

const char* krp_status_string(krp_status s) {
  switch (s) {
    case KRP_OK: return "KRP_OK";
    case KRP_EINVAL: return "KRP_EINVAL";
    case KRP_ENOMEM: return "KRP_ENOMEM";
    case KRP_ECUDA: return "KRP_ECUDA";
    case KRP_EUNSUPPORTED: return "KRP_EUNSUPPORTED";
    case KRP_ETIMEOUT: return "KRP_ETIMEOUT";
    case KRP_ENUMERIC: return "KRP_ENUMERIC";
  }
  return "KRP_UNKNOWN";
}

int krp_abi_version(void) { return KRP_ABI_VERSION; }

uint64_t krp_launch_count(krp_ctx ctx) { return ctx ? ctx->c.launches : 0; }

krp_status krp_gen_factors(krp_ctx ctx, uint64_t seed, uint32_t draw_id, uint32_t tag, int d,
                           const int64_t* rows, int ell, krp_dtype out_type, void* const* omega) {
  return guarded(ctx, [&] {
    KRP_REQUIRE(d >= 1 && d <= KRP_MAXD, "d = %d out of range 1..%d", d, KRP_MAXD);
    KRP_REQUIRE(rows && omega, "rows/omega is NULL");
    KRP_REQUIRE(ell >= 1, "ell = %d must be >= 1", ell);
    KRP_REQUIRE(out_type == KRP_F32 || out_type == KRP_BF16 || out_type == KRP_F64,
                "unsupported factor dtype %d", (int)out_type);
    FactorJob jobs[KRP_MAXD];
    int nj = 0;
    for (int j = 0; j < d; ++j) {
      KRP_REQUIRE(rows[j] >= 1, "rows[%d] must be >= 1", j);
      if (!omega[j]) continue;
      jobs[nj++] = FactorJob{omega[j], rows[j], (rows[j] * ell + 3) / 4, (uint32_t)j};
    }
    launch_gen_factors(seed, draw_id, tag, ell, out_type, jobs, nj);
  });
}

krp_status krp_philox_words(krp_ctx ctx, uint64_t seed, uint32_t c1, uint32_t c2, uint32_t c3,
                            uint64_t first_block, int64_t nblocks, uint32_t* out) {
  return guarded(ctx, [&] {
    KRP_REQUIRE(nblocks >= 0, "nblocks < 0");
    KRP_REQUIRE(nblocks == 0 || out, "out is NULL");
    launch_philox_words(seed, c1, c2, c3, first_block, nblocks, out);
  });
}

krp_status krp_sketch_mode(krp_ctx ctx, const void* X, krp_dtype xt, int d, const int64_t* dims,
                           const int64_t* ld, int n, const void* const* omega, krp_dtype omt,
                           int ell, float* Y) {
  return guarded(ctx, [&] {
    SketchArgs a = validate_sketch(X, xt, d, dims, omega, omt, ell);
    KRP_REQUIRE(n >= 0 && n < d, "mode n = %d out of range", n);
    KRP_REQUIRE(Y, "Y is NULL");
    ensure_workspace(current(), sketch_workspace_bytes(a, false) + dense_copy_bytes(d, dims, ld, xt));
    a.X = dense_copy(X, xt, d, dims, ld);
    sketch_one_mode(a, n, Y);
  });
}

krp_status krp_sketch_all_modes(krp_ctx ctx, const void* X, krp_dtype xt, int d,
                                const int64_t* dims, const int64_t* ld,
                                const void* const* omega, krp_dtype omt, int ell,
                                float* const* Y, int tree_split) {
  return guarded(ctx, [&] {
    SketchArgs a = validate_sketch(X, xt, d, dims, omega, omt, ell);
    KRP_REQUIRE(Y, "Y is NULL");
    for (int j = 0; j < d; ++j) KRP_REQUIRE(Y[j], "Y[%d] is NULL", j);
    KRP_REQUIRE(tree_split == -1 || (tree_split >= 1 && tree_split <= d - 1),
                "tree_split = %d out of range 1..%d (or -1)", tree_split, d - 1);
    ensure_workspace(current(), sketch_workspace_bytes(a, true, tree_split) +
                                    dense_copy_bytes(d, dims, ld, xt));
    a.X = dense_copy(X, xt, d, dims, ld);
    sketch_all_modes(a, Y, tree_split);
  });
}

krp_status krp_qr(krp_ctx ctx, int count, const float* const* Y, const int64_t* m, const int* l,
                  double* const* Q, double* const* R) {
  return guarded(ctx, [&] {
    KRP_REQUIRE(count >= 0 && count <= 4096, "count out of range");
    if (count == 0) return;
    KRP_REQUIRE(Y && m && l && Q, "NULL argument");
    size_t bytes = ws_bytes(count, sizeof(QrJob));
    for (int b = 0; b < count; ++b) {
      KRP_REQUIRE(Y[b] && Q[b], "Y[%d]/Q[%d] is NULL", b, b);
      KRP_REQUIRE(l[b] >= 1 && l[b] <= 256 && m[b] >= l[b], "QR %d: need m >= l, 1 <= l <= 256", b);
      bytes += ws_bytes((size_t)m[b] * l[b], sizeof(double));
    }
    Ctx* c = current();
    ensure_workspace(c, bytes);
    std::vector<QrJob> jobs(count);
    for (int b = 0; b < count; ++b)
      jobs[b] = QrJob{Y[b], Q[b], R ? R[b] : nullptr, c->ws.take<double>((size_t)m[b] * l[b]),
                      m[b], l[b]};
    KRP_CUDA_CHECK(cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream));
    qr_householder_f64(jobs.data(), count, c->d_status);
    raise_device_status(c);
  });
}

krp_status krp_multi_ttm(krp_ctx ctx, const void* X, krp_dtype xt, int d, const int64_t* dims,
                         const int64_t* ld, const double* const* Q, const int* cols, float* G) {
  return guarded(ctx, [&] {
    KRP_REQUIRE(d >= 1 && d <= KRP_MAXD, "d out of range");
    checked_numel(d, dims);
    KRP_REQUIRE(X && Q && cols && G, "NULL argument");
    KRP_REQUIRE(xt == KRP_F32 || xt == KRP_BF16 || xt == KRP_BF16X2,
                "X dtype must be F32, BF16 or BF16X2");
    for (int j = 0; j < d; ++j) {
      KRP_REQUIRE(Q[j], "Q[%d] is NULL", j);
      KRP_REQUIRE(cols[j] >= 1 && cols[j] <= 256, "cols[%d] out of range", j);
    }
    ensure_workspace(current(), multi_ttm_workspace_bytes(d, dims, cols, xt) +
                                    dense_copy_bytes(d, dims, ld, xt));
    multi_ttm(dense_copy(X, xt, d, dims, ld), xt, d, dims, Q, cols, G);
  });
}

krp_status krp_core_truncate(krp_ctx ctx, int d, const int64_t* dims, const int* ell,
                             const int* ranks, const float* core, const double* const* factors,
                             float* core_out, double* const* factors_out) {
  return guarded(ctx, [&] {
    KRP_REQUIRE(d >= 1 && d <= KRP_MAXD, "d out of range");
    KRP_REQUIRE(dims && ell && ranks && core && factors && core_out && factors_out, "NULL argument");
    for (int i = 0; i < d; ++i) {
      KRP_REQUIRE(ranks[i] >= 1 && ranks[i] <= ell[i], "need 1 <= ranks[%d] <= ell[%d]", i, i);
      KRP_REQUIRE(ell[i] <= 64 && ell[i] <= dims[i], "need ell[%d] <= min(64, dims[%d])", i, i);
      KRP_REQUIRE(factors[i] && factors_out[i], "factors[%d] / factors_out[%d] is NULL", i, i);
      KRP_REQUIRE(is_device_ptr(factors[i]) && is_device_ptr(factors_out[i]),
                  "factors must be device memory");
    }
    KRP_REQUIRE(is_device_ptr(core) && is_device_ptr(core_out), "core must be device memory");
    Ctx* c = current();
    ensure_workspace(c, core_truncate_workspace_bytes(d, ell, ranks));
    KRP_CUDA_CHECK(cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream));
    core_truncate(d, dims, ell, ranks, core, factors, core_out, factors_out);
    raise_device_status(c);
  });
}

krp_status krp_residual(krp_ctx ctx, const void* X, krp_dtype xt, int d, const int64_t* dims,
                        const int64_t* ld, const int* core_dims, const float* core,
                        const double* const* factors, double* sums) {
  return guarded(ctx, [&] {
    KRP_REQUIRE(d >= 2 && d <= KRP_MAXD, "d out of range");
    checked_numel(d, dims);
    KRP_REQUIRE(X && core_dims && core && factors && sums, "NULL argument");
    KRP_REQUIRE(xt == KRP_F32 || xt == KRP_BF16 || xt == KRP_BF16X2,
                "X dtype must be F32, BF16 or BF16X2");
    KRP_REQUIRE(is_device_ptr(X) && is_device_ptr(core), "X and core must be device memory");
    int64_t cdim[KRP_MAXD];
    for (int i = 0; i < d; ++i) {
      KRP_REQUIRE(core_dims[i] >= 1 && core_dims[i] <= 256, "core_dims[%d] out of range", i);
      KRP_REQUIRE(factors[i] && is_device_ptr(factors[i]), "factors[%d] must be device memory", i);
      cdim[i] = core_dims[i];
    }
    Ctx* c = current();
    ensure_workspace(c, residual_workspace_bytes(d, dims, cdim, xt) + ws_bytes(4, 8) +
                            dense_copy_bytes(d, dims, ld, xt));
    double* acc = c->ws.take<double>(4);
    KRP_CUDA_CHECK(cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream));
    KRP_CUDA_CHECK(cudaMemsetAsync(acc, 0, 2 * sizeof(double), c->stream));
    residual_sums(dense_copy(X, xt, d, dims, ld), xt, d, dims, core, cdim, factors, acc);
    KRP_CUDA_CHECK(cudaMemcpyAsync(sums, acc, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    raise_device_status(c);
  });
}

krp_status krp_tucker_rhosvd(krp_ctx ctx, const void* X, krp_dtype xt, int d, const int64_t* dims,
                             const int64_t* ld, const int* ranks, int oversample, uint64_t seed,
                             unsigned flags, krp_tucker_out* out) {
  return guarded(ctx, [&] {
    tucker_pipeline(false, X, xt, d, dims, ld, ranks, oversample, seed, flags, out);
  });
}

krp_status krp_tucker_sthosvd(krp_ctx ctx, const void* X, krp_dtype xt, int d,
                              const int64_t* dims, const int64_t* ld, const int* ranks,
                              int oversample, uint64_t seed, unsigned flags, krp_tucker_out* out) {
  return guarded(ctx, [&] {
    tucker_pipeline(true, X, xt, d, dims, ld, ranks, oversample, seed, flags, out);
  });
}

krp_status krp_trace_begin(krp_ctx ctx) {
  return guarded(ctx, [&] {
    Ctx* c = &ctx->c;
    c->trace.clear();
    cudaEvent_t ev = trace_event(c);
    KRP_CUDA_CHECK(cudaEventRecord(ev, c->stream));
    c->trace.push_back({nullptr, ev, c->stream});
    c->trace_on = true;
  });
}

krp_status krp_trace_end(krp_ctx ctx, char* json, size_t cap) {
  return guarded(ctx, [&] {
    Ctx* c = &ctx->c;
    c->trace_on = false;
    KRP_REQUIRE(json && cap > 2, "json buffer is NULL or too small");
    KRP_CUDA_CHECK(cudaStreamSynchronize(c->stream));
    if (c->side_stream) KRP_CUDA_CHECK(cudaStreamSynchronize(c->side_stream));
    // each launch: the time since the previous event on its own stream
    std::string out = "[";
    bool first = true;
    for (size_t i = 1; i < c->trace.size(); ++i) {
      if (!c->trace[i].name) continue;
      size_t p = i;
      while (p > 0 && c->trace[p - 1].st != c->trace[i].st) --p;
      if (p == 0) continue;  // no earlier event on this stream
      float ms = 0.f;
      KRP_CUDA_CHECK(cudaEventElapsedTime(&ms, c->trace[p - 1].ev, c->trace[i].ev));
      char item[160];
      snprintf(item, sizeof(item), "%s[\"%s\", %.6f]", first ? "" : ", ", c->trace[i].name, ms);
      first = false;
      out += item;
    }
    out += "]";
    c->trace.clear();
    KRP_REQUIRE(out.size() < cap, "trace needs %zu bytes", out.size() + 1);
    std::memcpy(json, out.c_str(), out.size() + 1);
  });
}

krp_status krp_split_bf16x2(krp_ctx ctx, const float* X, int64_t n, void* out) {
  return guarded(ctx, [&] {
    KRP_REQUIRE(X && out && n >= 0, "bad arguments");
    KRP_REQUIRE(is_device_ptr(X) && is_device_ptr(out), "X and out must be device pointers");
    KRP_REQUIRE((reinterpret_cast<uintptr_t>(out) & 15) == 0, "out must be 16-byte aligned");
    split_f32_bf16x2(X, n, static_cast<__nv_bfloat16*>(out));
  });
}

krp_status krp_tucker_rhosvd_batched(krp_ctx ctx, krp_dtype xt, int count, krp_tucker_item* items,
                                     int oversample, unsigned flags) {
  return guarded(ctx, [&] { tucker_batched(xt, count, items, oversample, flags); });
}

krp_status krp_era_realize(krp_ctx ctx, const void* blocks, krp_dtype bt, int m, int n, int s,
                           int r, const double* U, const double* S, const double* V, double* A,
                           double* eig_re, double* eig_im) {
  return guarded(ctx, [&] {
    KRP_REQUIRE(blocks && U && S && V && eig_re && eig_im, "NULL argument");
    KRP_REQUIRE(bt == KRP_F32 || bt == KRP_BF16, "blocks must be KRP_F32 or KRP_BF16");
    KRP_REQUIRE(m >= 1 && n >= 1 && s >= 2, "need m, n >= 1 and s >= 2");
    KRP_REQUIRE(r >= 1 && r <= 64 && r <= (int64_t)(s - 1) * m && r <= (int64_t)s * n,
                "need 1 <= r <= min(64, (s-1) m, s n)");
    for (const void* p : {blocks, (const void*)U, (const void*)S, (const void*)V, (const void*)eig_re,
                          (const void*)eig_im})
      KRP_REQUIRE(is_device_ptr(p), "all buffers must be device memory");
    KRP_REQUIRE(!A || is_device_ptr(A), "A must be device memory");
    Ctx* c = current();
    ensure_workspace(c, era_workspace_bytes(m, s, r));
    KRP_CUDA_CHECK(cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream));
    era_realize(blocks, bt, m, n, s, r, U, S, V, A, eig_re, eig_im);
    raise_device_status(c);
  });
}

krp_status krp_block_hankel_batched(krp_ctx ctx, krp_dtype bt, int count, krp_hankel_item* items) {
  return guarded(ctx, [&] { hankel_batched(bt, count, items); });
}

krp_status krp_tucker_batch_plan_info(krp_ctx ctx, int* slabs_per_unit, int* units, int* grid) {
  return guarded(ctx, [&] {
    KRP_REQUIRE(tucker_batched_plan_info(slabs_per_unit, units, grid), "no batch plan");
  });
}

krp_status krp_block_hankel_lowrank(krp_ctx ctx, const void* blocks, krp_dtype bt, int m, int n,
                                    int s, int r, int ell_r, int ell_l, uint64_t seed, double* U,
                                    double* S, double* V) {
  return guarded(ctx, [&] { hankel_pipeline(blocks, bt, m, n, s, r, ell_r, ell_l, seed, U, S, V); });
}

krp_status krp_block_hankel_nystrom(krp_ctx ctx, const void* blocks, krp_dtype bt, int m, int s,
                                    int r, int ell, double rcond, uint64_t seed, double* U,
                                    double* Lambda) {
  return guarded(ctx, [&] { hankel_nystrom(blocks, bt, m, s, r, ell, rcond, seed, U, Lambda); });
}

krp_status krp_tucker_hadamard(krp_ctx ctx, int d, const int64_t* dims, const int* rg,
                               const double* G, const double* const* U, const int* rh,
                               const double* H, const double* const* V, int ell, uint64_t seed,
                               double* core, double* const* factors, double* rel_error) {
  return guarded(ctx, [&] {
    KRP_REQUIRE(d >= 1 && d <= KRP_MAXD, "d out of range");
    KRP_REQUIRE(dims && rg && rh && G && U && H && V && core && factors, "NULL argument");
    KRP_REQUIRE(ell >= 1 && ell <= 64, "need 1 <= ell <= 64");
    int64_t ncore = 1;
    for (int j = 0; j < d; ++j) {
      KRP_REQUIRE(dims[j] >= ell && dims[j] <= INT32_MAX, "need ell <= dims[%d] < 2^31", j);
      KRP_REQUIRE(rg[j] >= 1 && rh[j] >= 1 && rg[j] <= 4096 && rh[j] <= 4096,
                  "ranks of mode %d out of range", j);
      ncore *= (int64_t)rg[j] * rh[j];
      KRP_REQUIRE(ncore <= (int64_t(1) << 25), "the product's core G (x) H exceeds 2^25 entries");
      KRP_REQUIRE(U[j] && V[j] && factors[j], "NULL factor for mode %d", j);
      KRP_REQUIRE(is_device_ptr(U[j]) && is_device_ptr(V[j]) && is_device_ptr(factors[j]),
                  "mode %d: factors must be device memory", j);
    }
    KRP_REQUIRE(is_device_ptr(G) && is_device_ptr(H) && is_device_ptr(core),
                "G, H and core must be device memory");
    Ctx* c = current();
    ensure_workspace(c, hadamard_workspace_bytes(d, dims, rg, rh, ell));
    KRP_CUDA_CHECK(cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream));
    hadamard_rhosvd(d, dims, rg, G, U, rh, H, V, ell, seed, core, factors, rel_error);
    raise_device_status(c);
  });
}

krp_status krp_sensor_select(krp_ctx ctx, int d, const int64_t* dims, const int* ells,
                             const double* const* Q, int* const* idx, double* const* A) {
  return guarded(ctx, [&] {
    KRP_REQUIRE(d >= 1 && d <= KRP_MAXD, "d out of range");
    KRP_REQUIRE(dims && ells && Q && idx && A, "NULL argument");
    for (int i = 0; i < d; ++i) {
      KRP_REQUIRE(dims[i] >= 1 && dims[i] <= INT32_MAX, "dims[%d] out of range", i);
      KRP_REQUIRE(ells[i] >= 1 && ells[i] <= 64 && ells[i] <= dims[i],
                  "need 1 <= ells[%d] <= min(64, dims[%d])", i, i);
      KRP_REQUIRE(Q[i] && idx[i] && A[i], "NULL pointer for mode %d", i);
      KRP_REQUIRE(is_device_ptr(Q[i]) && is_device_ptr(idx[i]) && is_device_ptr(A[i]),
                  "mode %d: buffers must be device memory", i);
    }
    Ctx* c = current();
    ensure_workspace(c, sensor_select_workspace_bytes(d, dims, ells));
    KRP_CUDA_CHECK(cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream));
    sensor_select(d, dims, ells, Q, idx, A);
    raise_device_status(c);
  });
}

krp_status krp_sensor_reconstruct(krp_ctx ctx, int d, const int64_t* dims, const int* ells,
                                  const double* const* A, const float* That, float* out) {
  return guarded(ctx, [&] {
    KRP_REQUIRE(d >= 1 && d <= KRP_MAXD, "d out of range");
    KRP_REQUIRE(dims && ells && A && That && out, "NULL argument");
    checked_numel(d, dims);
    for (int i = 0; i < d; ++i) {
      KRP_REQUIRE(ells[i] >= 1 && ells[i] <= dims[i], "need 1 <= ells[%d] <= dims[%d]", i, i);
      KRP_REQUIRE(A[i] && is_device_ptr(A[i]), "A[%d] must be device memory", i);
    }
    KRP_REQUIRE(is_device_ptr(That) && is_device_ptr(out), "T_hat and out must be device memory");
    Ctx* c = current();
    ensure_workspace(c, sensor_reconstruct_workspace_bytes(d, dims, ells));
    sensor_reconstruct(d, dims, ells, A, That, out);
  });
}

krp_status krp_block_hankel2_lowrank(krp_ctx ctx, const void* blocks, krp_dtype bt, int m, int n,
                                     int s1, int s2, int r, int ell_r, int ell_l, uint64_t seed,
                                     double* U, double* S, double* V) {
  return guarded(ctx, [&] {
    hankel2_pipeline(blocks, bt, m, n, s1, s2, r, ell_r, ell_l, seed, U, S, V);
  });
}

krp_status krp_block_hankel_sketch(krp_ctx ctx, const void* blocks, krp_dtype bt, int m, int n,
                                   int s, const void* omega1, const void* omega2, int ell_r,
                                   const void* psi1, const void* psi2, int ell_l, float* Y,
                                   float* Z) {
  return guarded(ctx, [&] {
    hankel_sketch_only(blocks, bt, m, n, s, omega1, omega2, ell_r, psi1, psi2, ell_l, Y, Z);
  });
}

}  // extern "C"
