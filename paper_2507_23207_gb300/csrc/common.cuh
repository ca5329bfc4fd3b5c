// Internal declarations shared by the library's translation units.
// Nothing here is part of the C ABI (include/krp.h is).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <map>
#include <string>
#include <vector>

#include "../../include/krp.h"

namespace krp {

// Error raised inside the library; converted to a krp_status at the ABI edge.
struct Error {
  krp_status status;
  std::string msg;
};

[[noreturn]] void fail(krp_status s, const char* fmt, ...);

#define KRP_CUDA_CHECK(expr)                                                   \
  do {                                                                         \
    cudaError_t e_ = (expr);                                                   \
    if (e_ != cudaSuccess)                                                     \
      ::krp::fail(KRP_ECUDA, "%s failed: %s (%s:%d)", #expr,                   \
                  cudaGetErrorString(e_), __FILE__, __LINE__);                 \
  } while (0)

#define KRP_REQUIRE(cond, ...)                                                 \
  do {                                                                         \
    if (!(cond)) ::krp::fail(KRP_EINVAL, __VA_ARGS__);                         \
  } while (0)

// Launch bookkeeping: every kernel launch goes through this so that the
// context can report how many of its kernels ran.
struct LaunchCounter {
  uint64_t n = 0;
};
void note_launch(const char* name);
void check_launch(const char* name);

// Simple bump allocator over one device arena owned by the context.  The
// arena is (re)allocated only between API calls, never while work is queued.
struct Workspace {
  char* base = nullptr;
  size_t cap = 0;
  size_t off = 0;
  void reset() { off = 0; }
  template <class T>
  T* take(size_t count) {
    size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
    if (off + bytes > cap) fail(KRP_ENOMEM, "workspace overflow (%zu + %zu > %zu)", off, bytes, cap);
    T* p = reinterpret_cast<T*>(base + off);
    off += bytes;
    return p;
  }
};

// Byte size rounding used to pre-size the workspace.
inline size_t ws_bytes(size_t count, size_t elem) { return (count * elem + 255) & ~size_t(255); }

struct Ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string last_error;
  Workspace ws;
  uint64_t launches = 0;
  int num_sms = 0;
  int* d_status = nullptr;  // device status word for bounded waits / numerics
  void* batch_plan = nullptr;              // cached batched-Tucker plan (batched.cu)
  void (*batch_plan_free)(void*) = nullptr;
  void* hankel_plan = nullptr;             // cached batched block-Hankel plan
  void (*hankel_plan_free)(void*) = nullptr;
  // host-to-device copies overlapped with the sketch (created on first use)
  cudaStream_t copy_stream = nullptr;
  std::vector<cudaEvent_t> copy_events;
  // FP64 QR beside the FP32 form's TF32 TTMs (created on first use); the
  // TF32 TTM leaves tc_reserve_sms SMs free while it is set
  cudaStream_t side_stream = nullptr;
  cudaEvent_t side_events[4] = {};
  int tc_reserve_sms = 0;
  // tree splits picked by timing, per (dims, l, dtype)
  std::map<std::vector<int64_t>, int> tree_split_cache;
  // launch trace (krp_trace_begin/end): an event after every launch, on the
  // stream of the launch (name null: a marker, e.g. where a second stream
  // starts after waiting on the first)
  struct TraceRec {
    const char* name;
    cudaEvent_t ev;
    cudaStream_t st;
  };
  bool trace_on = false;
  std::vector<TraceRec> trace;
  std::vector<cudaEvent_t> trace_pool;
};

// launch trace: an unnamed event on the current stream (where a second
// stream starts after waiting on the first)
void trace_marker();
Ctx* current();           // context of the API call in progress (thread-local)
cudaStream_t stream();    // its stream
void ensure_workspace(Ctx* c, size_t bytes);

// ---------------------------------------------------------------- kernels --
// Factor generation (philox.cu)
struct FactorJob {
  void* ptr;
  int64_t rows;
  int64_t blocks;  // ceil(rows*ell/4)
  uint32_t factor;
};
void launch_gen_factors(uint64_t seed, uint32_t draw, uint32_t tag, int ell,
                        krp_dtype type, const FactorJob* jobs, int njobs);
// One factor of a batch: its own key (seed), counter words (factor, draw,
// tag) as above, rows x ell FP32 column-major output.
struct BatchFactorJob {
  float* ptr;
  int64_t rows;
  uint64_t seed;
  uint32_t factor, draw, tag;
  int ell;
  int bf16_round;
};
// d_start: njobs+1 prefix sums of ceil(rows*ell/4) (device memory)
void launch_gen_factors_batch(const BatchFactorJob* d_jobs, const int64_t* d_start, int njobs,
                              int64_t total_blocks);
void launch_philox_words(uint64_t seed, uint32_t c1, uint32_t c2, uint32_t c3,
                         uint64_t first_block, int64_t nblocks, uint32_t* out);

// Mixed-radix description of the "other" modes whose factors weight a
// contraction: index s = sum_j digit_j * stride_j, digit_j < radix_j, weight
// = prod_j V_j[digit_j + ld_j * k].
struct Radix {
  int n = 0;
  int64_t radix[KRP_MAXD];
  const float* V[KRP_MAXD];  // FP32 factors, column-major, ld = radix
};

// FP32 CUDA-core kernels (f32_kernels.cu; mttkrp_first_f32 hands shapes the
// tensor cores take to the TF32 MTTKRP of tc_kernels.cu)
// out[s + ldo*k] (=|+=) sum_i A[i + lda*s] * F[i + ldf*k], s<S, k<L, i<K
void gemm_tn_f32(const float* A, int64_t lda, int64_t S, int K, const float* F,
                 int64_t ldf, int L, float* out, int64_t ldo, bool accumulate);
// Y[i + n1*k] = sum_s A[i + n1*s] * prod_j V_j[digit_j(s), k]   (Y zeroed here)
void mttkrp_first_f32(const float* A, int64_t n1, int64_t S, const Radix& rest,
                      int L, float* Y);
// workspace mttkrp_first_f32 may take (S = product of the other sides,
// n2max = largest side of the second mode)
size_t mttkrp_first_f32_workspace_bytes(int64_t S, int64_t n2max);
// Diagonal contraction of T (dims m_0..m_{D-1}, then k slowest, stride tk):
// Y[i_n + m_n*k] = sum_{others} T[...,k] prod_{j != n} V_j[i_j, k]  (Y zeroed)
void diag_contract_f32(const float* T, int D, const int64_t* m, int64_t tk,
                       int n, const float* const* V, int L, float* Y);
void cast_f64_to_f32(const double* src, float* dst, int64_t n);
void cast_f32_to_f64(const float* src, double* dst, int64_t n);
void transpose_f64_to_f32(const double* src, int64_t rows, int64_t cols, float* dst);
// move mode 0 of a dense FP32 tensor to the last position
void rotate_first_to_last_f32(const float* src, int64_t m0, int64_t rest, float* dst);
// ||X - Q1 H||^2 and ||X||^2 (FP64 accumulation), X n1 x S (F32 or BF16),
// Q1 n1 x l (FP32), H l x S (FP32); results added into acc[0], acc[1].
void residual_f32(const void* X, krp_dtype xt, int64_t n1, int64_t S,
                  const float* Q1, int l, const float* H, double* acc);

// FP64 kernels (f64_kernels.cu)
struct QrJob {
  const float* Y;
  double* Q;
  double* R;      // may be null
  double* work;   // m*l doubles
  int64_t m;
  int l;
  const double* Y64 = nullptr;  // FP64 input instead of Y when set
};
void qr_householder_f64(const QrJob* jobs, int count, int* status);
// S[a + l*b] += sum over columns of G_(mode) of G[a,col] * G[b,col] (S zeroed)
void gram_mode_f64(const double* G, int D, const int64_t* dims, int mode, double* S);
// S[n] = G_(n) G_(n)^T for every mode n < D in one launch (dims[n] <= 64)
void gram_modes_f64(const double* G, int D, const int64_t* dims, double* const* S);
// eigenvectors of symmetric S (l x l), sorted by eigenvalue descending; U gets
// the first r columns (l x r column-major)
// One symmetric eigenproblem (l x l FP64, l <= 64): the r leading
// eigenvectors into U (l x r, column-major) and, if ev is set, all l
// eigenvalues in descending order.
struct EigJob {
  const double* S;
  double* U;
  double* ev;
  int l, r;
};
// Launchers over job arrays already in device memory (no host copies, so
// they can be captured in a CUDA graph); maxl bounds every job's l.
void eig_launch(const EigJob* d_jobs, int count, int maxl, int* status);
void qr_householder_launch(const QrJob* d_jobs, int count, int* status);
// Shifted CholeskyQR3 (FP64; the Householder result for full-rank inputs) of
// many jobs with l <= 64 in one set of launches over a device job array:
// cholqr3_jobs_bytes gives the device memory the caller provides,
// cholqr3_jobs_setup fills it (one host-to-device copy, before any capture)
// and cholqr3_jobs_launch enqueues three memsets and nine kernels
// (graph-capturable) and returns the number of kernels.
struct CqrJobsPlan {
  void* d_jobs = nullptr;
  int count = 0;
  int64_t maxm = 0, total_rows = 0;
  double* g_all = nullptr;
  size_t g_count = 0;
};
size_t cholqr3_jobs_bytes(const QrJob* jobs, int count);
CqrJobsPlan cholqr3_jobs_setup(const QrJob* jobs, int count, void* dmem, cudaStream_t st);
int cholqr3_jobs_launch(const CqrJobsPlan& plan, int* status);
void sym_eig_top_f64(const double* const* S, const int* l, const int* r,
                     double* const* U, int count, int* status,
                     double* const* evals = nullptr);
// workspace sym_eig_top_f64 takes for `count` problems
size_t sym_eig_workspace_bytes(int count);
// out = G x_mode U^T for a small FP64 tensor (U is dims[mode] x r col-major)
void ttm_small_f64(const double* G, int D, const int64_t* dims, int mode,
                   const double* U, int r, double* out);
// C (m x n) = A (m x k) B (k x n), all column-major FP64
void matmul_f64(const double* A, const double* B, double* C, int64_t m, int k, int n);
double sum_squares_f64_sync(const double* x, int64_t n, double* scratch);
void check_finite_f64(const double* x, int64_t n, int* status);

// Block Hankel kernels (hankel.cu)
void hankel_sketch(const void* blocks, krp_dtype bt, int m, int n, int s,
                   const void* f1, const void* f2, int ell, bool transpose,
                   float* Y, float* Zscratch);
// The two-level form (Sec. 4.3): (2 s1 - 1)(2 s2 - 1) blocks, block (k1, k2)
// at k1 + (2 s1 - 1) k2; f1 s1 x ell, f2 s2 x ell, f3 (n or m) x ell.
void hankel2_sketch(const void* blocks, krp_dtype bt, int m, int n, int s1, int s2, const void* f1,
                    const void* f2, const void* f3, int ell, bool transpose, float* Y, float* Zs);

// BF16 tensor-core kernels (tc_kernels.cu)
bool tc_available();

}  // namespace krp
