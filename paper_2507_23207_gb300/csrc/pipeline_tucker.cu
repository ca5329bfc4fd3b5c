// Randomized Tucker pipelines over the kernels:
//   RHOSVD-KRP (Alg. 7), its memoized dimension-tree variant (Sec. 5.1),
//   RSTHOSVD-KRP (Alg. 8), the multi-TTM core, FP64 core truncation and the
//   streaming FP64-accumulated residual.
//
// Layout trick used throughout: every contraction acts on the first (fastest)
// mode of the current tensor and appends the new index as the slowest mode,
// Z(m_1, rest) -> Z'(rest, l).  After d such steps the modes are back in their
// natural order, so the core comes out as (l_1, ..., l_d), mode-1 fastest,
// and no explicit unfolding/permutation of the big tensor is ever made.
#include <algorithm>
#include <cstring>

#include "pipeline.h"

namespace krp {
namespace {

__global__ void krp_rows_kernel(int n, const int64_t* radix_unused, int64_t r0, int64_t r1,
                                int64_t r2, int64_t r3, int64_t r4, int64_t r5, int64_t r6,
                                const void* v0, const void* v1, const void* v2, const void* v3,
                                const void* v4, const void* v5, const void* v6, int bf16,
                                int64_t T, int L, float* __restrict__ w) {
  const int64_t rad[7] = {r0, r1, r2, r3, r4, r5, r6};
  const void* V[7] = {v0, v1, v2, v3, v4, v5, v6};
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < T * L;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t t = e % T;
    const int64_t k = e / T;
    float acc = 1.f;
    for (int j = 0; j < n; ++j) {
      const int64_t dg = t % rad[j];
      t /= rad[j];
      const int64_t idx = dg + rad[j] * k;
      acc *= bf16 ? __bfloat162float(static_cast<const __nv_bfloat16*>(V[j])[idx])
                  : static_cast<const float*>(V[j])[idx];
    }
    w[e] = acc;
  }
}

__global__ void split_hilo_kernel(const double* __restrict__ s, int64_t n,
                                  __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float f = static_cast<float>(s[i]);
    const __nv_bfloat16 h = __float2bfloat16_rn(f);
    hi[i] = h;
    if (lo) lo[i] = __float2bfloat16_rn(f - __bfloat162float(h));
  }
}

__global__ void split_x2_kernel(const float* __restrict__ X, int64_t n, __nv_bfloat16* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const float x = X[e];
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    out[e] = h;
    out[n + e] = __float2bfloat16_rn(x - __bfloat162float(h));
  }
}

__global__ void add_f32_kernel(float* __restrict__ dst, const float* __restrict__ src, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] += src[i];
}

__global__ void bf16_to_f32_kernel(const __nv_bfloat16* __restrict__ s, float* __restrict__ d,
                                   int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    d[i] = __bfloat162float(s[i]);
}

int grid_of(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 8192)); }

// Sides and element strides of a padded tensor (element (i_1..i_d) at
// sum_j i_j str[j]).
struct StridedDims {
  int d;
  int64_t dims[KRP_MAXD];
  int64_t str[KRP_MAXD];
};

// dense[r n1 + i] = src[offset of row r + i]: one mode-1 row (n1 contiguous
// elements of both) per CTA iteration, rows r in mixed radix over modes 2..d
template <class T>
__global__ void pack_strided_kernel(const T* __restrict__ src, T* __restrict__ dst,
                                    const StridedDims A, int64_t rows) {
  const int64_t n1 = A.dims[0];
  for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) {
    int64_t rem = r, off = 0;
    for (int j = 1; j < A.d; ++j) {
      off += (rem % A.dims[j]) * A.str[j];
      rem /= A.dims[j];
    }
    for (int64_t i = threadIdx.x; i < n1; i += blockDim.x) dst[r * n1 + i] = src[off + i];
  }
}

struct Timer {
  bool on = false;
  cudaEvent_t ev[64] = {};
  int n = 0;
  void start(bool enable) {
    on = enable;
    if (!on) return;
    for (auto& e : ev) KRP_CUDA_CHECK(cudaEventCreate(&e));
    mark();
  }
  void mark() {
    if (on) KRP_CUDA_CHECK(cudaEventRecord(ev[n++], stream()));
  }
  float between(int a, int b) {
    float ms = 0.f;
    KRP_CUDA_CHECK(cudaEventElapsedTime(&ms, ev[a], ev[b]));
    return ms;
  }
  ~Timer() {
    if (on)
      for (auto& e : ev) cudaEventDestroy(e);
  }
};

}  // namespace

void raise_device_status(Ctx* c) {
  int h = 0;
  KRP_CUDA_CHECK(cudaMemcpyAsync(&h, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  KRP_CUDA_CHECK(cudaStreamSynchronize(c->stream));
  if (h != 0) {
    KRP_CUDA_CHECK(cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream));
    fail(static_cast<krp_status>(h), "device stage reported %s", krp_status_string((krp_status)h));
  }
}

void krp_rows(const Radix& R, int64_t T, int L, bool bf16, float* w) {
  if (T * L <= 0) return;
  KRP_REQUIRE(R.n <= 7, "too many modes for krp_rows");
  int64_t r[7] = {1, 1, 1, 1, 1, 1, 1};
  const void* v[7] = {};
  for (int j = 0; j < R.n; ++j) {
    r[j] = R.radix[j];
    v[j] = R.V[j];
  }
  krp_rows_kernel<<<grid_of(T * L), 256, 0, stream()>>>(R.n, nullptr, r[0], r[1], r[2], r[3], r[4],
                                                        r[5], r[6], v[0], v[1], v[2], v[3], v[4],
                                                        v[5], v[6], bf16 ? 1 : 0, T, L, w);
  check_launch("krp_rows");
}

void split_bf16_hilo(const double* src, int64_t n, __nv_bfloat16* hi, __nv_bfloat16* lo) {
  if (n <= 0) return;
  split_hilo_kernel<<<grid_of(n), 256, 0, stream()>>>(src, n, hi, lo);
  check_launch("split_bf16_hilo");
}

void split_f32_bf16x2(const float* X, int64_t n, __nv_bfloat16* out) {
  if (n <= 0) return;
  split_x2_kernel<<<grid_of(n), 256, 0, stream()>>>(X, n, out);
  check_launch("split_bf16x2");
}

void convert_bf16_to_f32(const __nv_bfloat16* src, float* dst, int64_t n) {
  if (n <= 0) return;
  bf16_to_f32_kernel<<<grid_of(n), 256, 0, stream()>>>(src, dst, n);
  check_launch("bf16_to_f32");
}

// -------------------------------------------------- padded (ld) inputs ----
bool padded(int d, const int64_t* dims, const int64_t* ld) {
  if (!ld) return false;
  bool pad = false;
  for (int j = 0; j < d; ++j) {
    KRP_REQUIRE(ld[j] >= dims[j], "ld[%d] = %lld is smaller than dims[%d] = %lld", j,
                (long long)ld[j], j, (long long)dims[j]);
    pad = pad || ld[j] != dims[j];
  }
  return pad;
}

int64_t padded_numel(int d, const int64_t* ld) {
  int64_t n = 1;
  for (int j = 0; j < d; ++j) {
    KRP_REQUIRE(ld[j] >= 1 && n <= (int64_t(1) << 46) / ld[j], "padded tensor too large");
    n *= ld[j];
  }
  return n;
}

size_t dense_copy_bytes(int d, const int64_t* dims, const int64_t* ld, krp_dtype xt) {
  return padded(d, dims, ld) ? ws_bytes((size_t)checked_numel(d, dims), dtype_size(xt)) : 0;
}

const void* dense_copy(const void* X, krp_dtype xt, int d, const int64_t* dims, const int64_t* ld) {
  if (!padded(d, dims, ld)) return X;
  KRP_REQUIRE(is_device_ptr(X), "a padded X (ld) must be device memory");
  const int64_t N = checked_numel(d, dims);
  const int64_t NP = padded_numel(d, ld);
  StridedDims A{};
  A.d = d;
  int64_t st = 1;
  for (int j = 0; j < d; ++j) {
    A.dims[j] = dims[j];
    A.str[j] = st;
    st *= ld[j];
  }
  const int64_t rows = N / dims[0];
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(rows, 65535));
  const int planes = xt == KRP_BF16X2 ? 2 : 1;  // the lo plane follows the hi plane
  void* out = current()->ws.take<char>((size_t)N * dtype_size(xt));
  for (int p = 0; p < planes; ++p) {
    if (xt == KRP_F32) {
      pack_strided_kernel<float><<<grid, 256, 0, stream()>>>(static_cast<const float*>(X),
                                                             static_cast<float*>(out), A, rows);
    } else {
      pack_strided_kernel<__nv_bfloat16><<<grid, 256, 0, stream()>>>(
          static_cast<const __nv_bfloat16*>(X) + p * NP, static_cast<__nv_bfloat16*>(out) + p * N,
          A, rows);
    }
    check_launch("pack_strided");
  }
  return out;
}

// ------------------------------------------------------------- dispatch ----
// BF16 hi/lo input: the lo plane follows the hi plane (N elements later)
static const __nv_bfloat16* lo_plane(const void* X, krp_dtype xt, int64_t N) {
  return xt == KRP_BF16X2 ? static_cast<const __nv_bfloat16*>(X) + N : nullptr;
}
static bool bf16_family(krp_dtype t) { return t == KRP_BF16 || t == KRP_BF16X2; }
static int round_up16(int v) { return (v + 15) / 16 * 16; }
// SMs the FP32 form's TF32 TTMs leave to the FP64 QR on the second stream
constexpr int kQrSideSms = 8;

void big_gemm_tn(const void* X, krp_dtype xt, int64_t n1, int64_t S, const float* Ff,
                 const __nv_bfloat16* Fhi, const __nv_bfloat16* Flo, int L, float* out) {
  if (xt == KRP_F32) {
    // tensor cores as three TF32 products where the shape allows, else FFMA
    if (tc_gemm_tn_tf32_supported(n1, S, L, X))
      tc_gemm_tn_tf32(static_cast<const float*>(X), n1, S, Ff, n1, L, out);
    else
      gemm_tn_f32(static_cast<const float*>(X), n1, S, (int)n1, Ff, n1, L, out, S, false);
  } else {
    tc_gemm_tn_bf16(static_cast<const __nv_bfloat16*>(X), n1, S, Fhi, Flo, L, out,
                    lo_plane(X, xt, n1 * S));
  }
}

void big_mttkrp_first(const void* X, krp_dtype xt, int64_t n1, int d_rest, const int64_t* rest_dims,
                      const void* const* rest_V, int L, float* Y) {
  int64_t S = 1;
  for (int j = 0; j < d_rest; ++j) S *= rest_dims[j];
  if (xt == KRP_F32) {
    Radix R;
    R.n = d_rest;
    for (int j = 0; j < d_rest; ++j) {
      R.radix[j] = rest_dims[j];
      R.V[j] = static_cast<const float*>(rest_V[j]);
    }
    mttkrp_first_f32(static_cast<const float*>(X), n1, S, R, L, Y);
  } else {
    const int64_t n2 = d_rest >= 1 ? rest_dims[0] : 1;
    const int64_t T = S / n2;
    Radix R;
    R.n = d_rest - 1;
    for (int j = 1; j < d_rest; ++j) {
      R.radix[j - 1] = rest_dims[j];
      R.V[j - 1] = static_cast<const float*>(rest_V[j]);  // bf16 bits, typed as void below
    }
    float* w = current()->ws.take<float>((size_t)T * L);
    krp_rows(R, T, L, true, w);
    KRP_REQUIRE(d_rest >= 1, "BF16 sketch needs d >= 2");
    tc_mttkrp_first_bf16(static_cast<const __nv_bfloat16*>(X), n1, n2, T,
                         static_cast<const __nv_bfloat16*>(rest_V[0]), w, L, Y,
                         lo_plane(X, xt, n1 * S));
  }
}

// ------------------------------------------------------------ sketches -----
SketchArgs validate_sketch(const void* X, krp_dtype xt, int d, const int64_t* dims,
                           const void* const* omega, krp_dtype omt, int ell) {
  SketchArgs a{};
  KRP_REQUIRE(d >= 2 && d <= KRP_MAXD, "d = %d out of range 2..%d", d, KRP_MAXD);
  a.N = checked_numel(d, dims);
  KRP_REQUIRE(X, "X is NULL");
  KRP_REQUIRE(omega, "omega is NULL");
  KRP_REQUIRE(ell >= 1 && ell <= 256, "ell = %d out of range 1..256", ell);
  KRP_REQUIRE(xt == KRP_F32 || bf16_family(xt), "X dtype must be KRP_F32, KRP_BF16 or KRP_BF16X2");
  KRP_REQUIRE(omt == (xt == KRP_BF16X2 ? KRP_BF16 : xt),
              "factor dtype must match X (F32 with F32, BF16 with BF16 or BF16X2)");
  a.X = X;
  a.xt = xt;
  a.d = d;
  a.omt = omt;
  a.ell = ell;
  for (int j = 0; j < d; ++j) {
    a.dims[j] = dims[j];
    a.omega[j] = omega[j];
  }
  return a;
}

// Splits the autotuner tries: merged second dimensions up to 2^20 rows (and
// always the plain one, s = 1); an explicit split may merge more.
static bool tree_split_candidate(int64_t n2, int s) { return s == 1 || n2 <= (int64_t(1) << 20); }

// Workspace of the one-pass tree for a split s (the largest over the
// autotuner's candidates for s = -1): the merged dimension's factor and
// sketch (n2' x l), the slab weights and sketch (T x l), and the kernel's C
// partials.
static size_t tree_ws_bytes(int d, const int64_t* dims, int ell, int split = -1) {
  int64_t N = 1;
  for (int j = 0; j < d; ++j) N *= dims[j];
  size_t best = 0;
  int64_t n2 = 1;
  for (int s = 1; s <= d - 1; ++s) {
    n2 *= dims[s];
    if (split == -1 ? !tree_split_candidate(n2, s) : s != split) continue;
    const int64_t T = N / (dims[0] * n2);
    const size_t b = 2 * ws_bytes((size_t)n2 * ell, 4) + 2 * ws_bytes((size_t)T * ell, 4) +
                     tc_tree_workspace_bytes(dims[0], n2, T, ell);
    best = std::max(best, b);
  }
  return best;
}

size_t sketch_workspace_bytes(const SketchArgs& a, bool, int tree_split) {
  const int64_t n1 = a.dims[0];
  size_t b = ws_bytes((size_t)(a.N / n1) * a.ell, 4);               // B
  for (int j = 0; j < a.d; ++j) b += ws_bytes((size_t)a.dims[j] * a.ell, 4);  // f32 factors
  b += ws_bytes((size_t)(a.N / n1) * a.ell, 4);                     // KRP rows (upper bound)
  int64_t dmax = 1;
  for (int j = 0; j < a.d; ++j) dmax = std::max<int64_t>(dmax, a.dims[j]);
  b += mttkrp_first_f32_workspace_bytes(a.N / std::max<int64_t>(1, a.dims[0]), dmax);
  if (bf16_family(a.xt))
    b += tc_workspace_bytes(n1, a.N / n1, a.ell) + tree_ws_bytes(a.d, a.dims, a.ell, tree_split);
  else
    b += tc_gemm_tn_tf32_workspace_bytes(n1, a.ell);
  return b + (1 << 20);
}

static void f32_factor_views(const SketchArgs& a, const float** out) {
  for (int j = 0; j < a.d; ++j) {
    if (!a.omega[j]) {
      out[j] = nullptr;
      continue;
    }
    if (a.omt == KRP_F32) {
      out[j] = static_cast<const float*>(a.omega[j]);
    } else {
      float* f = current()->ws.take<float>((size_t)a.dims[j] * a.ell);
      convert_bf16_to_f32(static_cast<const __nv_bfloat16*>(a.omega[j]), f, a.dims[j] * a.ell);
      out[j] = f;
    }
  }
}

void sketch_one_mode(const SketchArgs& a, int n, float* Y) {
  for (int j = 0; j < a.d; ++j)
    if (j != n) KRP_REQUIRE(a.omega[j], "omega[%d] is NULL", j);
  const int64_t n1 = a.dims[0], S = a.N / n1;
  if (n == 0) {
    big_mttkrp_first(a.X, a.xt, n1, a.d - 1, a.dims + 1, a.omega + 1, a.ell, Y);
    return;
  }
  const float* f32v[KRP_MAXD];
  f32_factor_views(a, f32v);
  float* B = current()->ws.take<float>((size_t)S * a.ell);
  big_gemm_tn(a.X, a.xt, n1, S, f32v[0], static_cast<const __nv_bfloat16*>(a.omega[0]), nullptr,
              a.ell, B);
  diag_contract_f32(B, a.d - 1, a.dims + 1, S, n - 1, f32v + 1, a.ell, Y);
}

// One-pass tree with the modes 2..s+1 merged into its second dimension
// (n2' = prod of their sides, factor = their Khatri-Rao rows, FP32) and the
// modes s+2..d as its slabs (weights w).  Y_1 comes out whole; the merged
// dimension's sketch is contracted to Y_2..Y_{s+1}, the slabs' to the rest.
static void tree_sketch(const SketchArgs& a, float* const* Y, int s) {
  Ctx* c = current();
  // FP32 copies of the factors serve only the contractions after the tree
  const float* f32v[KRP_MAXD] = {};
  if (s > 1 || a.d - 1 - s > 1) f32_factor_views(a, f32v);
  const int64_t n1 = a.dims[0];
  int64_t n2 = 1;
  for (int j = 1; j <= s; ++j) n2 *= a.dims[j];
  const int64_t T = a.N / (n1 * n2);
  float* om2 = c->ws.take<float>((size_t)n2 * a.ell);
  if (s == 1) {
    convert_bf16_to_f32(static_cast<const __nv_bfloat16*>(a.omega[1]), om2, n2 * a.ell);
  } else {
    Radix R2;
    R2.n = s;
    for (int j = 1; j <= s; ++j) {
      R2.radix[j - 1] = a.dims[j];
      R2.V[j - 1] = static_cast<const float*>(a.omega[j]);  // bf16 bits
    }
    krp_rows(R2, n2, a.ell, true, om2);
  }
  Radix R;
  R.n = a.d - 1 - s;
  for (int j = s + 1; j < a.d; ++j) {
    R.radix[j - s - 1] = a.dims[j];
    R.V[j - s - 1] = static_cast<const float*>(a.omega[j]);  // bf16 bits
  }
  float* w = c->ws.take<float>((size_t)T * a.ell);
  krp_rows(R, T, a.ell, true, w);
  float* Y2 = (s == 1) ? Y[1] : c->ws.take<float>((size_t)n2 * a.ell);
  float* C = (a.d - 1 - s == 1) ? Y[a.d - 1] : c->ws.take<float>((size_t)T * a.ell);
  tc_tree_bf16(static_cast<const __nv_bfloat16*>(a.X), n1, n2, T,
               static_cast<const __nv_bfloat16*>(a.omega[0]), om2, w, a.ell, Y[0], Y2, C,
               lo_plane(a.X, a.xt, a.N));
  if (s > 1)
    for (int n = 1; n <= s; ++n) diag_contract_f32(Y2, s, a.dims + 1, n2, n - 1, f32v + 1, a.ell, Y[n]);
  if (a.d - 1 - s > 1)
    for (int n = s + 1; n < a.d; ++n)
      diag_contract_f32(C, a.d - 1 - s, a.dims + s + 1, T, n - s - 1, f32v + s + 1, a.ell, Y[n]);
}

static bool tree_split_ok(const SketchArgs& a, int s) {
  if (s < 1 || s > a.d - 1) return false;
  int64_t n2 = 1;
  for (int j = 1; j <= s; ++j) n2 *= a.dims[j];
  return n2 < (int64_t(1) << 31) && a.N / (a.dims[0] * n2) < (int64_t(1) << 31);
}

void sketch_all_modes(const SketchArgs& a, float* const* Y, int tree_split,
                      const std::function<void()>& after_first) {
  for (int j = 0; j < a.d; ++j) KRP_REQUIRE(a.omega[j], "omega[%d] is NULL", j);
  const int64_t n1 = a.dims[0], S = a.N / n1;
  const float* f32v[KRP_MAXD];
  if (bf16_family(a.xt) && tc_tree_supported(n1, a.ell)) {
    // one pass over X for every mode (fused dimension tree on tensor cores)
    KRP_REQUIRE(tree_split == -1 || tree_split_ok(a, tree_split),
                "tree_split = %d out of range 1..%d (or -1)", tree_split, a.d - 1);
    Ctx* c = current();
    int s = tree_split;
    if (s == -1) {
      std::vector<int64_t> key(a.dims, a.dims + a.d);
      key.push_back(a.ell);
      key.push_back(static_cast<int64_t>(a.xt));
      auto it = c->tree_split_cache.find(key);
      if (it != c->tree_split_cache.end()) {
        s = it->second;
      } else {
        // time every admissible split once (after a first run of each) and
        // keep the fastest; the workspace arena is rewound between runs
        cudaEvent_t e0, e1;
        KRP_CUDA_CHECK(cudaEventCreate(&e0));
        KRP_CUDA_CHECK(cudaEventCreate(&e1));
        float best = 0.f;
        int64_t n2c = 1;
        for (int cand = 1; cand <= a.d - 1; ++cand) {
          n2c *= a.dims[cand];
          if (!tree_split_ok(a, cand) || !tree_split_candidate(n2c, cand)) continue;
          const size_t mark = c->ws.off;
          tree_sketch(a, Y, cand);
          c->ws.off = mark;
          KRP_CUDA_CHECK(cudaEventRecord(e0, c->stream));
          tree_sketch(a, Y, cand);
          KRP_CUDA_CHECK(cudaEventRecord(e1, c->stream));
          c->ws.off = mark;
          KRP_CUDA_CHECK(cudaEventSynchronize(e1));
          float ms = 0.f;
          KRP_CUDA_CHECK(cudaEventElapsedTime(&ms, e0, e1));
          if (s == -1 || ms < best) {
            best = ms;
            s = cand;
          }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        KRP_REQUIRE(s >= 1, "no admissible tree split");
        c->tree_split_cache[key] = s;
      }
    }
    tree_sketch(a, Y, s);
    return;
  }
  f32_factor_views(a, f32v);
  big_mttkrp_first(a.X, a.xt, n1, a.d - 1, a.dims + 1, a.omega + 1, a.ell, Y[0]);
  if (after_first) after_first();
  float* B = current()->ws.take<float>((size_t)S * a.ell);
  big_gemm_tn(a.X, a.xt, n1, S, f32v[0], static_cast<const __nv_bfloat16*>(a.omega[0]), nullptr,
              a.ell, B);
  for (int n = 1; n < a.d; ++n) diag_contract_f32(B, a.d - 1, a.dims + 1, S, n - 1, f32v + 1, a.ell, Y[n]);
}

// All mode sketches of a tensor that is still on the host: X is copied to
// the device buffer a.X in chunks of its last mode on a second stream, and
// each chunk is sketched on the context's stream as soon as it has landed
// (the sketches of the modes before the last are sums over the chunks, the
// last mode's sketch is the chunks' rows; the same decomposition as the
// sharded path's).  The copy of X and the sketch overlap.
static void sketch_host_overlapped(const SketchArgs& a, const void* host, float* const* Y) {
  Ctx* c = current();
  Workspace& ws = c->ws;
  const int d = a.d;
  const int64_t nd = a.dims[d - 1];
  const int64_t slab = a.N / nd;  // elements per index of the last mode
  const size_t eb = dtype_size(a.xt), fb = dtype_size(a.omt);
  const int K = static_cast<int>(std::min<int64_t>(8, nd));
  if (!c->copy_stream)
    KRP_CUDA_CHECK(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
  while (static_cast<int>(c->copy_events.size()) < K + 1) {
    cudaEvent_t e;
    KRP_CUDA_CHECK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    c->copy_events.push_back(e);
  }
  // the copies overwrite workspace that earlier work on the context's
  // stream may still read
  KRP_CUDA_CHECK(cudaEventRecord(c->copy_events[K], c->stream));
  KRP_CUDA_CHECK(cudaStreamWaitEvent(c->copy_stream, c->copy_events[K], 0));
  char* dev = static_cast<char*>(const_cast<void*>(a.X));
  for (int k = 0; k < K; ++k) {
    const int64_t t0 = nd * k / K, t1 = nd * (k + 1) / K;
    KRP_CUDA_CHECK(cudaMemcpyAsync(dev + t0 * slab * eb, static_cast<const char*>(host) + t0 * slab * eb,
                                   (t1 - t0) * slab * eb, cudaMemcpyHostToDevice, c->copy_stream));
    KRP_CUDA_CHECK(cudaEventRecord(c->copy_events[k], c->copy_stream));
  }
  const int64_t cmax = (nd + K - 1) / K;
  float* Yt[KRP_MAXD];
  for (int n = 0; n < d - 1; ++n) {
    Yt[n] = ws.take<float>((size_t)a.dims[n] * a.ell);
    KRP_CUDA_CHECK(cudaMemsetAsync(Y[n], 0, sizeof(float) * a.dims[n] * a.ell, c->stream));
  }
  Yt[d - 1] = ws.take<float>((size_t)cmax * a.ell);
  void* omc = ws.take<char>((size_t)cmax * a.ell * fb);
  for (int k = 0; k < K; ++k) {
    const int64_t t0 = nd * k / K, t1 = nd * (k + 1) / K, m = t1 - t0;
    KRP_CUDA_CHECK(cudaStreamWaitEvent(c->stream, c->copy_events[k], 0));
    const size_t mark = ws.off;
    SketchArgs ac = a;
    ac.X = dev + t0 * slab * eb;
    ac.dims[d - 1] = m;
    ac.N = slab * m;
    // rows t0..t1-1 of the last factor (column-major, leading size nd)
    KRP_CUDA_CHECK(cudaMemcpy2DAsync(omc, m * fb, static_cast<const char*>(a.omega[d - 1]) + t0 * fb,
                                     nd * fb, m * fb, a.ell, cudaMemcpyDeviceToDevice, c->stream));
    ac.omega[d - 1] = omc;
    sketch_all_modes(ac, Yt);
    for (int n = 0; n < d - 1; ++n) {
      const int64_t cnt = a.dims[n] * a.ell;
      add_f32_kernel<<<grid_of(cnt), 256, 0, stream()>>>(Y[n], Yt[n], cnt);
      check_launch("add_f32");
    }
    KRP_CUDA_CHECK(cudaMemcpy2DAsync(Y[d - 1] + t0, nd * sizeof(float), Yt[d - 1], m * sizeof(float),
                                     m * sizeof(float), a.ell, cudaMemcpyDeviceToDevice, c->stream));
    ws.off = mark;
  }
}

// ----------------------------------------------------------- multi-TTM -----
size_t multi_ttm_workspace_bytes(int d, const int64_t* dims, const int* cols, krp_dtype xt) {
  const int64_t N = checked_numel(d, dims);
  size_t big = (size_t)(N / dims[0]) * cols[0];
  size_t b = 2 * ws_bytes(big, 4);
  for (int j = 0; j < d; ++j) b += ws_bytes((size_t)dims[j] * cols[j], 4 + 2 + 2);
  if (bf16_family(xt)) {
    b += tc_workspace_bytes(dims[0], N / dims[0], 2 * cols[0]);
    if (d >= 3) b += tc_workspace_bytes(dims[1], 1, 2 * cols[1]) + 2 * ws_bytes((size_t)dims[1] * cols[1], 2);
  } else {
    b += tc_gemm_tn_tf32_workspace_bytes(dims[0], cols[0]);
  }
  return b + (1 << 20);
}

void multi_ttm(const void* X, krp_dtype xt, int d, const int64_t* dims, const double* const* Q,
               const int* cols, float* G, cudaEvent_t q0_ready, cudaEvent_t qrest_ready) {
  Ctx* c = current();
  const int64_t N = checked_numel(d, dims);
  const int64_t n1 = dims[0];
  float* Qf[KRP_MAXD];
  __nv_bfloat16 *Qh = nullptr, *Ql = nullptr;
  if (q0_ready) KRP_CUDA_CHECK(cudaStreamWaitEvent(c->stream, q0_ready, 0));
  // the other factors are read after the first TTM when they come from
  // another stream (qrest_ready), else converted here
  const int jcast = qrest_ready ? 1 : d;
  for (int j = 0; j < d; ++j) {
    Qf[j] = c->ws.take<float>((size_t)dims[j] * cols[j]);
    if (j < jcast) cast_f64_to_f32(Q[j], Qf[j], dims[j] * cols[j]);
  }
  if (bf16_family(xt)) {
    Qh = c->ws.take<__nv_bfloat16>((size_t)n1 * cols[0]);
    Ql = c->ws.take<__nv_bfloat16>((size_t)n1 * cols[0]);
    split_bf16_hilo(Q[0], n1 * cols[0], Qh, Ql);
  }
  const size_t big = (size_t)(N / n1) * cols[0];
  float* buf[2] = {c->ws.take<float>(big), c->ws.take<float>(big)};
  int64_t size = N;
  float* cur = (d == 1) ? G : buf[0];
  int j0 = 1;
  // BF16 forms with d >= 3: the first TTM writes its result as a BF16 hi/lo
  // pair (in the same 4 bytes per element as FP32, |z - hi - lo| <= 2^-17 |z|)
  // so that the second TTM, the other contraction over a large operand, also
  // runs on tensor cores
  if (bf16_family(xt) && d >= 3 && dims[1] % 8 == 0 && ((N / n1) * cols[0]) % 8 == 0 &&
      2 * round_up16(cols[1]) <= 256) {
    __nv_bfloat16* zb = reinterpret_cast<__nv_bfloat16*>(buf[0]);
    tc_gemm_tn_bf16(static_cast<const __nv_bfloat16*>(X), n1, N / n1, Qh, Ql, cols[0], nullptr,
                    lo_plane(X, xt, N), zb);
    size = (N / n1) * cols[0];
    __nv_bfloat16* q1h = c->ws.take<__nv_bfloat16>((size_t)dims[1] * cols[1]);
    __nv_bfloat16* q1l = c->ws.take<__nv_bfloat16>((size_t)dims[1] * cols[1]);
    split_bf16_hilo(Q[1], dims[1] * cols[1], q1h, q1l);
    float* nxt = (d == 2) ? G : buf[1];
    tc_gemm_tn_bf16(zb, dims[1], size / dims[1], q1h, q1l, cols[1], nxt, zb + size);
    size = (size / dims[1]) * cols[1];
    cur = nxt;
    j0 = 2;
  } else {
    big_gemm_tn(X, xt, n1, N / n1, Qf[0], Qh, Ql, cols[0], cur);
    size = (N / n1) * cols[0];
  }
  if (qrest_ready) {
    KRP_REQUIRE(j0 == 1, "factor events need the first TTM alone before the rest");
    KRP_CUDA_CHECK(cudaStreamWaitEvent(c->stream, qrest_ready, 0));
    for (int j = 1; j < d; ++j) cast_f64_to_f32(Q[j], Qf[j], dims[j] * cols[j]);
  }
  for (int j = j0; j < d; ++j) {
    float* nxt = (j == d - 1) ? G : buf[j & 1];
    const int64_t S = size / dims[j];
    gemm_tn_f32(cur, dims[j], S, (int)dims[j], Qf[j], dims[j], cols[j], nxt, S, false);
    size = S * cols[j];
    cur = nxt;
  }
}

// ------------------------------------------------ a7 truncation, a8 residual ----
size_t core_truncate_workspace_bytes(int d, const int* ell, const int* ranks) {
  int64_t core_l = 1;
  size_t b = 0;
  for (int i = 0; i < d; ++i) {
    core_l *= ell[i];
    b += ws_bytes((size_t)ell[i] * ell[i], 8) + ws_bytes((size_t)ell[i] * ranks[i], 8);
  }
  return b + 2 * ws_bytes((size_t)core_l, 8) + sym_eig_workspace_bytes(d) + (1 << 16);
}

// Rank-r truncation of an l-core by an FP64 HOSVD of the core (Gram of every
// mode unfolding, top-r eigenvectors U_i, G <- G x {U_i^T}, Q_i <- Q_i U_i).
// G FP32 (ell, mode-1 fastest), Q[i] FP64 dims[i] x ell[i]; Gout FP32
// (ranks), Qout[i] FP64 dims[i] x ranks[i]; all device memory.
void core_truncate(int d, const int64_t* dims, const int* ell, const int* ranks, const float* G,
                   const double* const* Q, float* Gout, double* const* Qout) {
  Ctx* c = current();
  Workspace& ws = c->ws;
  int64_t core_l = 1;
  int64_t cdim[KRP_MAXD];
  for (int i = 0; i < d; ++i) {
    core_l *= ell[i];
    cdim[i] = ell[i];
  }
  double* G64 = ws.take<double>((size_t)core_l);
  double* G64b = ws.take<double>((size_t)core_l);
  cast_f32_to_f64(G, G64, core_l);
  double* Sg[KRP_MAXD];
  double* U[KRP_MAXD];
  int lv[KRP_MAXD], rv[KRP_MAXD];
  for (int i = 0; i < d; ++i) {
    Sg[i] = ws.take<double>((size_t)ell[i] * ell[i]);
    U[i] = ws.take<double>((size_t)ell[i] * ranks[i]);
    lv[i] = ell[i];
    rv[i] = ranks[i];
  }
  gram_modes_f64(G64, d, cdim, Sg);
  sym_eig_top_f64(Sg, lv, rv, U, d, c->d_status);
  double* src = G64;
  double* dst = G64b;
  for (int i = 0; i < d; ++i) {
    ttm_small_f64(src, d, cdim, i, U[i], ranks[i], dst);
    cdim[i] = ranks[i];
    std::swap(src, dst);
    matmul_f64(Q[i], U[i], Qout[i], dims[i], ell[i], ranks[i]);
  }
  int64_t rl = 1;
  for (int i = 0; i < d; ++i) rl *= ranks[i];
  cast_f64_to_f32(src, Gout, rl);
}

size_t residual_workspace_bytes(int d, const int64_t* dims, const int64_t* cdim, krp_dtype xt) {
  const int64_t N = checked_numel(d, dims);
  size_t b = 2 * ws_bytes((size_t)(N / dims[0]) * cdim[0], 4);
  int64_t cl = 1;
  for (int i = 0; i < d; ++i) {
    b += ws_bytes((size_t)dims[i] * cdim[i], 4);
    cl *= cdim[i];
  }
  b += ws_bytes((size_t)cl, 4);
  if (bf16_family(xt)) b += tc_residual_workspace_bytes(dims[0], N / dims[0]);
  if (xt == KRP_F32) b += tc_residual_tf32_workspace_bytes(dims[0], N / dims[0]);
  return b + (1 << 16);
}

// acc[0] += ||X - Gc x {Q}||_F^2, acc[1] += ||X||_F^2 (FP64, device) by
// streaming reconstruction: H = Gc x_2 Q_2 ... x_d Q_d (FP32, c_1 x N/n_1)
// is expanded once, then one pass over X compares X with Q_1 H.
void residual_sums(const void* Xd, krp_dtype xt, int d, const int64_t* dims, const float* Gc,
                   const int64_t* cdim, const double* const* Qout, double* acc) {
  Workspace& ws = current()->ws;
  const int64_t N = checked_numel(d, dims);
  int64_t out_l = 1;
  for (int i = 0; i < d; ++i) out_l *= cdim[i];
  float* QTf[KRP_MAXD];
  for (int i = 1; i < d; ++i) {
    QTf[i] = ws.take<float>((size_t)dims[i] * cdim[i]);
    transpose_f64_to_f32(Qout[i], dims[i], cdim[i], QTf[i]);
  }
  float* Q1f = ws.take<float>((size_t)dims[0] * cdim[0]);
  cast_f64_to_f32(Qout[0], Q1f, dims[0] * cdim[0]);
  const size_t hbig = (size_t)(N / dims[0]) * cdim[0];
  float* hb[2] = {ws.take<float>(hbig), ws.take<float>(hbig)};
  // rotate G (c1, c2..cd) -> (c2..cd, c1), then expand modes 2..d
  rotate_first_to_last_f32(Gc, cdim[0], out_l / cdim[0], hb[0]);
  float* curh = hb[0];
  int64_t size = out_l;
  for (int j = 1; j < d; ++j) {
    float* nx = hb[j & 1];
    if (nx == curh) nx = hb[(j + 1) & 1];
    const int64_t S = size / cdim[j];
    gemm_tn_f32(curh, cdim[j], S, (int)cdim[j], QTf[j], cdim[j], (int)dims[j], nx, S, false);
    size = S * dims[j];
    curh = nx;
  }
  if (bf16_family(xt) && tc_residual_supported(dims[0], (int)cdim[0]))
    tc_residual_bf16(static_cast<const __nv_bfloat16*>(Xd), dims[0], N / dims[0], Qout[0],
                     (int)cdim[0], curh, acc, lo_plane(Xd, xt, N));
  else if (xt == KRP_BF16X2)
    fail(KRP_EUNSUPPORTED, "BF16 hi/lo residual needs n_1 %% 8 == 0 and at most 64 columns");
  else if (xt == KRP_F32 && tc_residual_tf32_supported(dims[0], N / dims[0], (int)cdim[0], Xd))
    tc_residual_tf32(static_cast<const float*>(Xd), dims[0], N / dims[0], Qout[0], (int)cdim[0], curh,
                     acc);
  else
    residual_f32(Xd, xt, dims[0], N / dims[0], Q1f, (int)cdim[0], curh, acc);
}

// ------------------------------------------------------------ pipeline -----
void tucker_pipeline(bool sequential, const void* X, krp_dtype xt, int d, const int64_t* dims,
                     const int64_t* ld, const int* ranks, int oversample, uint64_t seed,
                     unsigned flags, krp_tucker_out* out) {
  Ctx* c = current();
  KRP_REQUIRE(d >= 2 && d <= KRP_MAXD, "d = %d out of range 2..%d", d, KRP_MAXD);
  const int64_t N = checked_numel(d, dims);
  KRP_REQUIRE(X && ranks && out, "NULL argument");
  KRP_REQUIRE(xt == KRP_F32 || bf16_family(xt), "X dtype must be KRP_F32, KRP_BF16 or KRP_BF16X2");
  KRP_REQUIRE(oversample >= 0, "oversample must be >= 0");
  KRP_REQUIRE((flags & ~0xFu) == 0, "unknown flag bits 0x%x", flags);
  const bool memo = (flags & KRP_MEMO) && !sequential;
  const bool trunc = flags & KRP_TRUNCATE;
  const bool resid = flags & KRP_RESIDUAL;
  int ell[KRP_MAXD];
  int ellmax = 0;
  for (int i = 0; i < d; ++i) {
    KRP_REQUIRE(ranks[i] >= 1, "ranks[%d] must be >= 1", i);
    ell[i] = ranks[i] + oversample;
    KRP_REQUIRE(ell[i] <= dims[i], "l_%d = %d exceeds n_%d = %lld", i, ell[i], i, (long long)dims[i]);
    KRP_REQUIRE(ell[i] <= (trunc ? 64 : 256), "l_%d = %d too large", i, ell[i]);
    ellmax = std::max(ellmax, ell[i]);
    KRP_REQUIRE(out->factors[i], "out->factors[%d] is NULL", i);
  }
  KRP_REQUIRE(out->core, "out->core is NULL");
  const size_t xb = dtype_size(xt);

  // ---------------- workspace plan (upper bound; take() checks overflow)
  const bool x_dev = is_device_ptr(X);
  int64_t maxS = 0;
  for (int i = 0; i < d; ++i) maxS = std::max<int64_t>(maxS, N / dims[i]);
  const size_t big = (size_t)(N / dims[0]) * ellmax;
  size_t need = 5 * ws_bytes(big, 4);
  need += ws_bytes((size_t)maxS * ellmax, 4);  // KRP rows for the BF16 mode-1 sketch
  {
    int64_t dmax = 1;
    for (int i = 0; i < d; ++i) dmax = std::max<int64_t>(dmax, dims[i]);
    need += mttkrp_first_f32_workspace_bytes(maxS, dmax);  // FP32 slab-MTTKRP operands
  }
  const bool x_pad = padded(d, dims, ld);
  if (!x_dev) {
    need += ws_bytes((size_t)(x_pad ? padded_numel(d, ld) : N), xb);
    // chunked copy: the chunk sketches' temporaries (at most the whole
    // tensor's) and, for BF16, the tree of a chunk's shape
    for (int i = 0; i < d; ++i) need += ws_bytes((size_t)dims[i] * ellmax, 4 + 4);
    if (xt == KRP_BF16) {
      int64_t cd[KRP_MAXD];
      for (int i = 0; i < d; ++i) cd[i] = dims[i];
      cd[d - 1] = (dims[d - 1] + 7) / 8;
      need += tree_ws_bytes(d, cd, ellmax);
    }
  }
  if (x_pad) need += ws_bytes((size_t)N, xb);
  int64_t core_l = 1;
  for (int i = 0; i < d; ++i) {
    need += (size_t)d * ws_bytes((size_t)dims[i] * ellmax, 4 + 4);  // factors (both types)
    need += ws_bytes((size_t)dims[i] * ellmax, 4);                  // Y_i
    need += 3 * ws_bytes((size_t)dims[i] * ellmax, 8);              // Q_i, QR work, Q_i U_i
    need += ws_bytes((size_t)dims[i] * ellmax, 4 + 2 + 2 + 4);      // Q casts
    need += ws_bytes((size_t)ellmax * ellmax, 8) * 2;
    core_l *= ell[i];
  }
  need += 4 * ws_bytes((size_t)core_l, 8) + 2 * ws_bytes((size_t)core_l, 4);
  need += sym_eig_workspace_bytes(d);
  if (bf16_family(xt))
    need += tc_workspace_bytes(dims[0], N / dims[0], 2 * ellmax) + tree_ws_bytes(d, dims, ellmax);
  else
    need += tc_gemm_tn_tf32_workspace_bytes(dims[0], ellmax);
  if (bf16_family(xt) && resid) need += tc_residual_workspace_bytes(dims[0], N / dims[0]);
  if (xt == KRP_F32 && resid) need += tc_residual_tf32_workspace_bytes(dims[0], N / dims[0]);
  need += 4 << 20;
  ensure_workspace(c, need);
  Workspace& ws = c->ws;

  Timer tm;
  tm.start(flags & KRP_TIMINGS);  // event 0
  KRP_CUDA_CHECK(cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream));

  // a dense host X of the memoized RHOSVD (FP32 or BF16) is copied in chunks
  // of the last mode, overlapped with the sketch; other host inputs are
  // copied whole first
  const bool overlap = !x_dev && !x_pad && memo && (xt == KRP_F32 || xt == KRP_BF16) &&
                       dims[d - 1] >= 2;
  const void* Xd = X;
  if (!x_dev) {
    // host X (padded or not) is staged as given, then packed on the device
    const size_t hb = (size_t)(x_pad ? padded_numel(d, ld) : N) * xb;
    void* p = ws.take<char>(hb);
    if (!overlap) KRP_CUDA_CHECK(cudaMemcpyAsync(p, X, hb, cudaMemcpyHostToDevice, c->stream));
    Xd = p;
  }
  Xd = dense_copy(Xd, xt, d, dims, ld);

  // ---------------- factors (a1) and sketches (a2/a3), QR (a4), core (a5/a6)
  float* Y[KRP_MAXD];
  double* Q[KRP_MAXD];
  for (int i = 0; i < d; ++i) {
    Y[i] = ws.take<float>((size_t)dims[i] * ellmax);
    Q[i] = ws.take<double>((size_t)dims[i] * ell[i]);
  }
  float* G = ws.take<float>((size_t)core_l);
  double* qr_work[KRP_MAXD];
  for (int i = 0; i < d; ++i) qr_work[i] = ws.take<double>((size_t)dims[i] * ell[i]);
  auto run_qr = [&](int i0, int cnt) {
    std::vector<QrJob> jobs(cnt);
    for (int b = 0; b < cnt; ++b) {
      const int i = i0 + b;
      jobs[b] = QrJob{Y[i], Q[i], nullptr, qr_work[i], dims[i], ell[i]};
    }
    qr_householder_f64(jobs.data(), cnt, c->d_status);
  };
  // factor dtype for contractions over X (a BF16 hi/lo X takes BF16 factors:
  // a random matrix needs no more than BF16 values, only X does)
  const krp_dtype ft = xt == KRP_BF16X2 ? KRP_BF16 : xt;
  const size_t fb = dtype_size(ft);

  if (!sequential) {
    void* fac[KRP_MAXD][KRP_MAXD] = {};
    if (memo) {
      for (int j = 0; j < d; ++j) fac[0][j] = ws.take<char>((size_t)dims[j] * ellmax * fb);
      FactorJob jobs[KRP_MAXD];
      for (int j = 0; j < d; ++j) jobs[j] = FactorJob{fac[0][j], dims[j], (dims[j] * ellmax + 3) / 4, (uint32_t)j};
      launch_gen_factors(seed, KRP_DRAW_MEMO, KRP_TAG_OMEGA, ellmax, ft, jobs, d);
    } else {
      for (int i = 0; i < d; ++i) {
        FactorJob jobs[KRP_MAXD];
        int nj = 0;
        for (int j = 0; j < d; ++j) {
          if (j == i) continue;
          fac[i][j] = ws.take<char>((size_t)dims[j] * ell[i] * fb);
          jobs[nj++] = FactorJob{fac[i][j], dims[j], (dims[j] * ell[i] + 3) / 4, (uint32_t)j};
        }
        launch_gen_factors(seed, KRP_DRAW_FRESH_BASE + i, KRP_TAG_OMEGA, ell[i], ft, jobs, nj);
      }
    }
    tm.mark();  // 1
    // FP32 form (two passes over X in the sketch): the FP64 QR of mode 1 runs
    // on a second stream beside the tree's B-part TTM, the QRs of modes 2..d
    // beside the core's first TTM (which needs Q_1 only); those TF32 TTMs
    // leave kQrSideSms SMs to it.
    const bool qr_side = memo && !overlap && xt == KRP_F32 && d >= 2;
    cudaEvent_t* sev = c->side_events;
    auto side_qr = [&](int i0, int cnt, cudaEvent_t start, cudaEvent_t done) {
      KRP_CUDA_CHECK(cudaEventRecord(start, c->stream));
      KRP_CUDA_CHECK(cudaStreamWaitEvent(c->side_stream, start, 0));
      struct Swap {
        Ctx* c;
        cudaStream_t s;
        ~Swap() { c->stream = s; }
      } swap{c, c->stream};
      c->stream = c->side_stream;
      trace_marker();
      run_qr(i0, cnt);
      KRP_CUDA_CHECK(cudaEventRecord(done, c->side_stream));
    };
    if (qr_side) {
      if (!c->side_stream)
        KRP_CUDA_CHECK(cudaStreamCreateWithFlags(&c->side_stream, cudaStreamNonBlocking));
      for (cudaEvent_t& e : c->side_events)
        if (!e) KRP_CUDA_CHECK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    if (memo) {
      SketchArgs a{};
      a.X = Xd; a.xt = xt; a.d = d; a.omt = ft; a.ell = ellmax; a.N = N;
      for (int j = 0; j < d; ++j) { a.dims[j] = dims[j]; a.omega[j] = fac[0][j]; }
      if (overlap) {
        sketch_host_overlapped(a, X, Y);
      } else if (qr_side) {
        struct Reserve {
          Ctx* c;
          ~Reserve() { c->tc_reserve_sms = 0; }
        } reserve{c};
        c->tc_reserve_sms = kQrSideSms;
        sketch_all_modes(a, Y, -1, [&] { side_qr(0, 1, sev[0], sev[1]); });
        side_qr(1, d - 1, sev[2], sev[3]);
        tm.mark();  // 2
        tm.mark();  // 3 (the QR runs beside the sketch and the core)
        multi_ttm(Xd, xt, d, dims, Q, ell, G, sev[1], sev[3]);
      } else {
        sketch_all_modes(a, Y);
      }
    } else {
      for (int i = 0; i < d; ++i) {
        SketchArgs a{};
        a.X = Xd; a.xt = xt; a.d = d; a.omt = ft; a.ell = ell[i]; a.N = N;
        for (int j = 0; j < d; ++j) { a.dims[j] = dims[j]; a.omega[j] = fac[i][j]; }
        // the sketch's temporaries are dead once Y_i is written: rewind the
        // arena so the d sketches reuse the same space (stream order keeps
        // the next sketch's writes after this one's reads)
        const size_t mark = ws.off;
        sketch_one_mode(a, i, Y[i]);
        ws.off = mark;
      }
    }
    if (!qr_side) {
      tm.mark();  // 2
      run_qr(0, d);
      tm.mark();  // 3
      multi_ttm(Xd, xt, d, dims, Q, ell, G);
    }
    tm.mark();  // 4
  } else {
    // Alg. 8: G <- X; for i: sketch G_(i), QR, G <- G x_i Q_i^T  (rotated layout)
    const void* cur = Xd;
    krp_dtype ct = xt;
    int64_t size = N;
    int order[KRP_MAXD];       // rotated mode order of `cur`
    int64_t cdims[KRP_MAXD];   // its sides
    for (int j = 0; j < d; ++j) { order[j] = j; cdims[j] = dims[j]; }
    float* pp[2] = {ws.take<float>(big), ws.take<float>(big)};
    for (int i = 0; i < d; ++i) {
      const int64_t ni = dims[i];
      const krp_dtype sft = ct == KRP_BF16X2 ? KRP_BF16 : ct;  // factors for the tensor sketched
      const size_t sfb = dtype_size(sft);
      void* fac[KRP_MAXD] = {};
      FactorJob jobs[KRP_MAXD];
      int nj = 0;
      for (int j = 0; j < d; ++j) {
        if (j == i) continue;
        const int64_t rows = (j < i) ? ell[j] : dims[j];
        fac[j] = ws.take<char>((size_t)rows * ell[i] * sfb);
        jobs[nj++] = FactorJob{fac[j], rows, (rows * ell[i] + 3) / 4, (uint32_t)j};
      }
      launch_gen_factors(seed, KRP_DRAW_STHOSVD_BASE + i, KRP_TAG_OMEGA, ell[i], sft, jobs, nj);
      tm.mark();
      // rest of the rotated order: order[1..d-1]
      int64_t rdims[KRP_MAXD];
      const void* rV[KRP_MAXD];
      for (int q = 1; q < d; ++q) {
        rdims[q - 1] = cdims[q];
        rV[q - 1] = fac[order[q]];
      }
      big_mttkrp_first(cur, ct, ni, d - 1, rdims, rV, ell[i], Y[i]);
      tm.mark();
      run_qr(i, 1);
      tm.mark();
      // G <- G x_i Q_i^T
      float* Qf = ws.take<float>((size_t)ni * ell[i]);
      cast_f64_to_f32(Q[i], Qf, ni * ell[i]);
      __nv_bfloat16 *Qh = nullptr, *Ql = nullptr;
      if (bf16_family(ct)) {
        Qh = ws.take<__nv_bfloat16>((size_t)ni * ell[i]);
        Ql = ws.take<__nv_bfloat16>((size_t)ni * ell[i]);
        split_bf16_hilo(Q[i], ni * ell[i], Qh, Ql);
      }
      float* nxt = (i == d - 1) ? G : pp[i & 1];
      big_gemm_tn(cur, ct, ni, size / ni, Qf, Qh, Ql, ell[i], nxt);
      size = size / ni * ell[i];
      for (int q = 0; q < d - 1; ++q) { order[q] = order[q + 1]; cdims[q] = cdims[q + 1]; }
      order[d - 1] = i;
      cdims[d - 1] = ell[i];
      cur = nxt;
      ct = KRP_F32;
      tm.mark();
    }
  }

  // ---------------- truncation (a7): HOSVD of the core in FP64
  float* Gout = G;
  double* Qout[KRP_MAXD];
  for (int i = 0; i < d; ++i) Qout[i] = Q[i];
  int64_t cdim[KRP_MAXD];
  for (int i = 0; i < d; ++i) cdim[i] = ell[i];
  const int tmark_trunc0 = tm.n;
  if (trunc) {
    for (int i = 0; i < d; ++i) Qout[i] = ws.take<double>((size_t)dims[i] * ranks[i]);
    int64_t rl = 1;
    for (int i = 0; i < d; ++i) rl *= ranks[i];
    Gout = ws.take<float>((size_t)rl);
    core_truncate(d, dims, ell, ranks, G, Q, Gout, Qout);
    for (int i = 0; i < d; ++i) cdim[i] = ranks[i];
  }
  tm.mark();
  int64_t out_l = 1;
  for (int i = 0; i < d; ++i) out_l *= cdim[i];

  // ---------------- residual (a8): ||X - G x {Q}||_F, FP64 accumulation
  double resid_val = -1.0, xnorm = -1.0;
  double* acc = ws.take<double>(4);
  if (resid) {
    KRP_CUDA_CHECK(cudaMemsetAsync(acc, 0, 2 * sizeof(double), c->stream));
    residual_sums(Xd, xt, d, dims, Gout, cdim, Qout, acc);
  }
  tm.mark();

  // ---------------- outputs
  const bool core_dev = is_device_ptr(out->core);
  KRP_CUDA_CHECK(cudaMemcpyAsync(out->core, Gout, sizeof(float) * out_l,
                                 core_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                 c->stream));
  for (int i = 0; i < d; ++i) {
    const bool fdev = is_device_ptr(out->factors[i]);
    KRP_CUDA_CHECK(cudaMemcpyAsync(out->factors[i], Qout[i], sizeof(double) * dims[i] * cdim[i],
                                   fdev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                   c->stream));
  }
  double* gsq = ws.take<double>(1);
  // ||G||_F in FP64 from the FP32 core
  double* g64 = ws.take<double>((size_t)out_l);
  cast_f32_to_f64(Gout, g64, out_l);
  const double gn2 = sum_squares_f64_sync(g64, out_l, gsq);  // synchronises the stream
  double hacc[2] = {0, 0};
  if (resid) {
    KRP_CUDA_CHECK(cudaMemcpy(hacc, acc, 2 * sizeof(double), cudaMemcpyDeviceToHost));
    xnorm = std::sqrt(hacc[1]);
    resid_val = hacc[1] > 0 ? std::sqrt(hacc[0] / hacc[1]) : 0.0;
  }
  tm.mark();
  raise_device_status(c);

  out->d = d;
  for (int i = 0; i < d; ++i) out->core_dims[i] = cdim[i];
  out->rel_residual = resid_val;
  out->x_norm = xnorm;
  out->core_norm = std::sqrt(gn2);
  std::memset(&out->times, 0, sizeof(out->times));
  if (tm.on) {
    KRP_CUDA_CHECK(cudaEventSynchronize(tm.ev[tm.n - 1]));
    krp_phase_times& T = out->times;
    const int last = tm.n - 1;
    if (!sequential) {
      T.rng_ms = tm.between(0, 1);
      T.sketch_ms = tm.between(1, 2);
      T.qr_ms = tm.between(2, 3);
      T.core_ms = tm.between(3, 4);
    } else {
      // per step: [gen, sketch, qr, ttm] marks after event 0
      for (int i = 0; i < d; ++i) {
        const int b = 4 * i;
        T.rng_ms += tm.between(b, b + 1);
        T.sketch_ms += tm.between(b + 1, b + 2);
        T.qr_ms += tm.between(b + 2, b + 3);
        T.core_ms += tm.between(b + 3, b + 4);
      }
    }
    T.truncate_ms = tm.between(tmark_trunc0 - 1, tmark_trunc0);
    T.residual_ms = tm.between(tmark_trunc0, tmark_trunc0 + 1);
    T.total_ms = tm.between(0, last);
  }
}

}  // namespace krp
