// Alg. 6: single-pass randomized SVD of a block Hankel matrix with KRP
// sketches.  Sketches (a9) on CUDA cores in FP32; post-processing (a10) in FP64:
//   Y = Q R (FP64 thin QR);  P = Psi^T Q computed structurally,
//   P[c, :] = sum_{i,a} Psi1[i, c] Psi2[a, c] Q[(i,a), :];
//   W = P^+ Z^T by least squares through the thin QR P = Qp Rp:
//   W = B Z^T with B = Rp^{-1} Qp^T (lr x ll, back substitution per column);
//   W = U_W S V^T through the eigen-decomposition of W W^T (Jacobi);
//   U = Q U_W, V = W^T U_W S^{-1}.
#include <cmath>

#include "pipeline.h"

namespace krp {
namespace {

template <class T>
__device__ __forceinline__ double ldd(const T* p, int64_t i);
template <>
__device__ __forceinline__ double ldd<float>(const float* p, int64_t i) { return p[i]; }
template <>
__device__ __forceinline__ double ldd<__nv_bfloat16>(const __nv_bfloat16* p, int64_t i) {
  return __bfloat162float(p[i]);
}

// P[c + ll*q] = sum_{i<s, a<m} psi1[i + s*c] psi2[a + m*c] Q[(a + m*i) + ms*q]
template <class T>
__global__ void psi_t_q_kernel(const T* __restrict__ psi1, const T* __restrict__ psi2, int s,
                               int m, int ll, const double* __restrict__ Q, int lr,
                               double* __restrict__ P) {
  const int c = blockIdx.x, q = blockIdx.y;
  const int64_t ms = (int64_t)m * s;
  double acc = 0.0;
  for (int64_t row = threadIdx.x; row < ms; row += blockDim.x) {
    const int a = (int)(row % m), i = (int)(row / m);
    acc = fma(ldd(psi1, i + (int64_t)s * c) * ldd(psi2, a + (int64_t)m * c), Q[row + ms * q], acc);
  }
  __shared__ double red[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    P[c + (int64_t)ll * q] = t;
  }
}

// B = Rp^{-1} Qp^T (lr x ll, column-major): one warp per column c of Qp^T
// (grid ll), back substitution with the lanes splitting each sum over t
// (lr <= 64: entries t = lane and lane + 32 held in registers).
__global__ void __launch_bounds__(32) ls_coef_kernel(const double* __restrict__ Qp,
                                                     const double* __restrict__ Rp, int ll, int lr,
                                                     double* __restrict__ B) {
  const int c = blockIdx.x, lane = threadIdx.x;
  double b0 = 0.0, b1 = 0.0;
  for (int q = lr - 1; q >= 0; --q) {
    double part = 0.0;
    if (lane > q && lane < lr) part = Rp[q + (int64_t)lr * lane] * b0;
    if (lane + 32 > q && lane + 32 < lr) part = fma(Rp[q + (int64_t)lr * (lane + 32)], b1, part);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    const double v = (Qp[c + (int64_t)ll * q] - part) / Rp[q + (int64_t)lr * q];
    if (lane == q) b0 = v;
    if (lane + 32 == q) b1 = v;
  }
  if (lane < lr) B[lane + (int64_t)lr * c] = b0;
  if (lane + 32 < lr) B[lane + 32 + (int64_t)lr * c] = b1;
}

// W[q + lr*col] = sum_c B[q + lr*c] Z[col + ns*c]: a CTA takes kLsCols columns,
// its Z entries converted to FP64 once in shared memory.
constexpr int kLsCols = 16;
__global__ void ls_apply_kernel(const double* __restrict__ B, const float* __restrict__ Z,
                                int64_t ns, int ll, int lr, double* __restrict__ W) {
  extern __shared__ double zs[];  // ll x kLsCols
  const int64_t c0 = (int64_t)blockIdx.x * kLsCols;
  const int nc = (int)((ns - c0) < kLsCols ? (ns - c0) : kLsCols);
  for (int e = threadIdx.x; e < ll * kLsCols; e += blockDim.x) {
    const int c = e / kLsCols, k = e % kLsCols;
    zs[e] = k < nc ? (double)Z[c0 + k + ns * c] : 0.0;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < lr * nc; e += blockDim.x) {
    const int q = e % lr, k = e / lr;
    double acc = 0.0;
    for (int c = 0; c < ll; ++c) acc = fma(B[q + (int64_t)lr * c], zs[c * kLsCols + k], acc);
    W[q + (int64_t)lr * (c0 + k)] = acc;
  }
}

// V[col + ns*j] = sum_q W[q + lr*col] Uw[q + lr*j] / sigma_j ; S[j] = sigma_j
__global__ void right_vectors_kernel(const double* __restrict__ W, int64_t ns, int lr,
                                     const double* __restrict__ Uw, const double* __restrict__ ev,
                                     int r, double* __restrict__ V, double* __restrict__ S) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ns * r;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t col = e % ns;
    const int j = (int)(e / ns);
    const double sig = sqrt(fmax(ev[j], 0.0));
    double acc = 0.0;
    for (int q = 0; q < lr; ++q) acc = fma(W[q + (int64_t)lr * col], Uw[q + (int64_t)lr * j], acc);
    V[e] = sig > 0.0 ? acc / sig : 0.0;
    if (col == 0) S[j] = sig;
  }
}

// C <- (C + C^T) / 2 for an l x l column-major matrix (one CTA).
__global__ void nys_sym_kernel(double* __restrict__ C, int l) {
  for (int e = threadIdx.x; e < l * l; e += blockDim.x) {
    const int i = e % l, j = e / l;
    if (i < j) {
      const double v = 0.5 * (C[i + (int64_t)l * j] + C[j + (int64_t)l * i]);
      C[i + (int64_t)l * j] = v;
      C[j + (int64_t)l * i] = v;
    }
  }
}

// G[:, j] *= c_j^{-1/2} for the eigenvalues kept by the pseudoinverse
// (c_j > rcond * c_0, c sorted descending, c_0 > 0), else 0 (one CTA).
__global__ void nys_scale_kernel(double* __restrict__ G, const double* __restrict__ c, int l,
                                 double rcond) {
  const double c0 = c[0];
  for (int e = threadIdx.x; e < l * l; e += blockDim.x) {
    const int j = e / l;
    const double cj = c[j];
    G[e] = (c0 > 0.0 && cj > rcond * c0) ? G[e] / sqrt(cj) : 0.0;
  }
}

// P[c + ll*q] = sum_{i1<s1, i2<s2, a<m} psi1[i1 + s1*c] psi2[i2 + s2*c] psi3[a + m*c]
//                 Q[(a + m*(i2 + s2*i1)) + ms*q]   (three-factor Khatri-Rao Psi)
template <class T>
__global__ void psi3_t_q_kernel(const T* __restrict__ psi1, const T* __restrict__ psi2,
                                const T* __restrict__ psi3, int s1, int s2, int m, int ll,
                                const double* __restrict__ Q, double* __restrict__ P) {
  const int c = blockIdx.x, q = blockIdx.y;
  const int64_t ms = (int64_t)m * s1 * s2;
  double acc = 0.0;
  for (int64_t row = threadIdx.x; row < ms; row += blockDim.x) {
    const int a = (int)(row % m);
    const int64_t blk = row / m;
    const int i2 = (int)(blk % s2), i1 = (int)(blk / s2);
    const double w = ldd(psi1, i1 + (int64_t)s1 * c) * ldd(psi2, i2 + (int64_t)s2 * c) *
                     ldd(psi3, a + (int64_t)m * c);
    acc = fma(w, Q[row + ms * q], acc);
  }
  __shared__ double red[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    P[c + (int64_t)ll * q] = t;
  }
}

int grid_for(int64_t n) {
  int64_t g = (n + 255) / 256;
  return (int)(g < 1 ? 1 : (g > 8192 ? 8192 : g));
}

void validate_hankel(const void* blocks, krp_dtype bt, int m, int n, int s) {
  KRP_REQUIRE(blocks, "blocks is NULL");
  KRP_REQUIRE(bt == KRP_F32 || bt == KRP_BF16, "blocks dtype must be KRP_F32 or KRP_BF16");
  KRP_REQUIRE(m >= 1 && n >= 1 && s >= 1, "m, n, s must be >= 1");
  KRP_REQUIRE((int64_t)m * s <= (int64_t(1) << 31) && (int64_t)n * s <= (int64_t(1) << 31),
              "block Hankel too large");
}

}  // namespace

// Steps 3-6 of Alg. 6 from the two sketches Y (ms x ell_r) and Z (ns x ell_l):
// QR of Y, P = Psi^T Q (structured, by psi_t_q), W = P^+ Z^T by least
// squares, the SVD of W through W W^T, U = Q U_W, V = W^T U_W S^{-1}.
template <class PsiTQ>
void single_pass_tail(Ctx* c, Workspace& ws, const float* Y, const float* Z, int64_t ms,
                      int64_t ns, int r, int ell_r, int ell_l, PsiTQ&& psi_t_q, double* U,
                      double* S, double* V) {
  // QR of Y
  double* Q = ws.take<double>((size_t)ms * ell_r);
  double* qw = ws.take<double>((size_t)ms * ell_r);
  QrJob jy{Y, Q, nullptr, qw, ms, ell_r};
  qr_householder_f64(&jy, 1, c->d_status);
  // P = Psi^T Q (structured)
  double* P = ws.take<double>((size_t)ell_l * ell_r);
  psi_t_q(Q, P);
  // least squares W = P^+ Z^T
  double* Qp = ws.take<double>((size_t)ell_l * ell_r);
  double* Rp = ws.take<double>((size_t)ell_r * ell_r);
  double* pw = ws.take<double>((size_t)ell_l * ell_r);
  QrJob jpq{nullptr, Qp, Rp, pw, ell_l, ell_r};
  jpq.Y64 = P;
  qr_householder_f64(&jpq, 1, c->d_status);
  double* W = ws.take<double>((size_t)ell_r * ns);
  double* Bls = ws.take<double>((size_t)ell_r * ell_l);
  ls_coef_kernel<<<ell_l, 32, 0, c->stream>>>(Qp, Rp, ell_l, ell_r, Bls);
  check_launch("hankel_ls_coef");
  {
    const size_t sm = sizeof(double) * (size_t)ell_l * kLsCols;
    KRP_CUDA_CHECK(cudaFuncSetAttribute(ls_apply_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)sm));
    ls_apply_kernel<<<(unsigned)((ns + kLsCols - 1) / kLsCols), 256, sm, c->stream>>>(Bls, Z, ns, ell_l,
                                                                                   ell_r, W);
  }
  check_launch("hankel_ls_apply");
  // SVD of W via W W^T
  double* Wg = ws.take<double>((size_t)ell_r * ell_r);
  const int64_t wd[2] = {ell_r, ns};
  gram_mode_f64(W, 2, wd, 0, Wg);
  double* Uw = ws.take<double>((size_t)ell_r * ell_r);
  double* ev = ws.take<double>((size_t)ell_r);
  const double* Sarr[1] = {Wg};
  double* Uarr[1] = {Uw};
  double* Earr[1] = {ev};
  int lv[1] = {ell_r}, rv[1] = {ell_r};
  sym_eig_top_f64(Sarr, lv, rv, Uarr, 1, c->d_status, Earr);
  double* Ud = ws.take<double>((size_t)ms * r);
  double* Vd = ws.take<double>((size_t)ns * r);
  double* Sd = ws.take<double>((size_t)r);
  matmul_f64(Q, Uw, Ud, ms, ell_r, r);
  right_vectors_kernel<<<grid_for(ns * r), 256, 0, c->stream>>>(W, ns, ell_r, Uw, ev, r, Vd, Sd);
  check_launch("hankel_right_vectors");
  auto out = [&](double* dst, const double* src, size_t count) {
    const bool dev = is_device_ptr(dst);
    KRP_CUDA_CHECK(cudaMemcpyAsync(dst, src, count * sizeof(double),
                                   dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                   c->stream));
  };
  out(U, Ud, (size_t)ms * r);
  out(V, Vd, (size_t)ns * r);
  out(S, Sd, (size_t)r);
  raise_device_status(c);
}

void hankel_sketch_only(const void* blocks, krp_dtype bt, int m, int n, int s, const void* omega1,
                        const void* omega2, int ell_r, const void* psi1, const void* psi2,
                        int ell_l, float* Y, float* Z) {
  validate_hankel(blocks, bt, m, n, s);
  KRP_REQUIRE(ell_r >= 1 && ell_l >= 0, "sketch sizes out of range");
  const int nb = 2 * s - 1;
  const int64_t zs = (int64_t)std::max(m, n) * std::max(ell_r, ell_l) * nb;
  ensure_workspace(current(), ws_bytes(zs, 4) + (1 << 20));
  float* Zs = current()->ws.take<float>(zs);
  if (Y) {
    KRP_REQUIRE(omega1 && omega2, "omega1/omega2 is NULL");
    hankel_sketch(blocks, bt, m, n, s, omega1, omega2, ell_r, false, Y, Zs);
  }
  if (Z && ell_l > 0) {
    KRP_REQUIRE(psi1 && psi2, "psi1/psi2 is NULL");
    hankel_sketch(blocks, bt, m, n, s, psi1, psi2, ell_l, true, Z, Zs);
  }
}

void hankel_pipeline(const void* blocks, krp_dtype bt, int m, int n, int s, int r, int ell_r,
                     int ell_l, uint64_t seed, double* U, double* S, double* V) {
  Ctx* c = current();
  validate_hankel(blocks, bt, m, n, s);
  if (ell_l == 0) ell_l = (int)std::ceil(1.5 * ell_r);
  const int64_t ms = (int64_t)m * s, ns = (int64_t)n * s;
  KRP_REQUIRE(r >= 1 && r <= ell_r && ell_r <= ell_l, "need 1 <= r <= ell_r <= ell_l");
  KRP_REQUIRE(ell_r <= 64 && ell_l <= 256, "need ell_r <= 64 and ell_l <= 256");
  KRP_REQUIRE(ell_r <= ms && ell_l <= ns && ell_r <= ell_l, "sketch sizes exceed the matrix");
  KRP_REQUIRE(U && S && V, "U/S/V is NULL");
  const int nb = 2 * s - 1;
  const size_t eb = dtype_size(bt);
  const bool b_dev = is_device_ptr(blocks);
  size_t need = ws_bytes((size_t)m * n * nb, eb);
  need += ws_bytes((size_t)std::max(m, n) * ell_l * nb, 4);
  need += 2 * ws_bytes((size_t)s * ell_l, eb) + 2 * ws_bytes((size_t)std::max(m, n) * ell_l, eb);
  need += ws_bytes((size_t)ms * ell_r, 4) + ws_bytes((size_t)ns * ell_l, 4);
  need += 3 * ws_bytes((size_t)ms * ell_r, 8) + 5 * ws_bytes((size_t)ell_l * ell_r, 8);
  need += ws_bytes((size_t)ell_r * ns, 8) + 4 * ws_bytes((size_t)ell_r * ell_r, 8);
  need += ws_bytes((size_t)ms * r, 8) + ws_bytes((size_t)ns * r, 8) + ws_bytes(r, 8);
  need += sym_eig_workspace_bytes(1);
  need += 1 << 20;
  ensure_workspace(c, need);
  Workspace& ws = c->ws;
  KRP_CUDA_CHECK(cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream));

  const void* Bd = blocks;
  if (!b_dev) {
    void* p = ws.take<char>((size_t)m * n * nb * eb);
    KRP_CUDA_CHECK(cudaMemcpyAsync(p, blocks, (size_t)m * n * nb * eb, cudaMemcpyHostToDevice,
                                   c->stream));
    Bd = p;
  }
  float* Zs = ws.take<float>((size_t)std::max(m, n) * ell_l * nb);
  void* o1 = ws.take<char>((size_t)s * ell_r * eb);
  void* o2 = ws.take<char>((size_t)n * ell_r * eb);
  void* p1 = ws.take<char>((size_t)s * ell_l * eb);
  void* p2 = ws.take<char>((size_t)m * ell_l * eb);
  FactorJob jo[2] = {{o1, s, ((int64_t)s * ell_r + 3) / 4, 0}, {o2, n, ((int64_t)n * ell_r + 3) / 4, 1}};
  launch_gen_factors(seed, 0, KRP_TAG_OMEGA, ell_r, bt, jo, 2);
  FactorJob jp[2] = {{p1, s, ((int64_t)s * ell_l + 3) / 4, 0}, {p2, m, ((int64_t)m * ell_l + 3) / 4, 1}};
  launch_gen_factors(seed, 0, KRP_TAG_PSI, ell_l, bt, jp, 2);

  float* Y = ws.take<float>((size_t)ms * ell_r);
  float* Z = ws.take<float>((size_t)ns * ell_l);
  hankel_sketch(Bd, bt, m, n, s, o1, o2, ell_r, false, Y, Zs);
  hankel_sketch(Bd, bt, m, n, s, p1, p2, ell_l, true, Z, Zs);

  single_pass_tail(c, ws, Y, Z, ms, ns, r, ell_r, ell_l,
                   [&](const double* Q, double* P) {
                     dim3 g(ell_l, ell_r);
                     if (bt == KRP_F32)
                       psi_t_q_kernel<float><<<g, 256, 0, c->stream>>>(
                           static_cast<const float*>(p1), static_cast<const float*>(p2), s, m,
                           ell_l, Q, ell_r, P);
                     else
                       psi_t_q_kernel<__nv_bfloat16><<<g, 256, 0, c->stream>>>(
                           static_cast<const __nv_bfloat16*>(p1),
                           static_cast<const __nv_bfloat16*>(p2), s, m, ell_l, Q, ell_r, P);
                     check_launch("hankel_psi_t_q");
                   },
                   U, S, V);
}

// Nystrom approximation of a symmetric positive semidefinite block Hankel
// matrix (the remark after Alg. 6): M_nys = Y (Omega^T Y)^+ Y^T with
// Y = M Omega the column sketch of Alg. 6 (Eq. (4.1)).  With Y = Q R:
//   C = Omega^T Y = (Omega^T Q) R (structured, as Psi^T Q above),
//   C = V diag(c) V^T, G = R V diag(c_k^{-1/2}) over the kept eigenvalues,
//   M_nys = Q (G G^T) Q^T, and the eigenpairs of M_nys are Q U_T, lambda_T
//   of T = G G^T (l x l).  All stages after the sketch in FP64.
void hankel_nystrom(const void* blocks, krp_dtype bt, int m, int s, int r, int ell, double rcond,
                    uint64_t seed, double* U, double* L) {
  Ctx* c = current();
  validate_hankel(blocks, bt, m, m, s);
  const int64_t ms = (int64_t)m * s;
  KRP_REQUIRE(r >= 1 && r <= ell && ell <= 64 && ell <= ms, "need 1 <= r <= l <= min(64, m s)");
  KRP_REQUIRE(U && L, "U/Lambda is NULL");
  KRP_REQUIRE(rcond < 1.0, "rcond must be < 1");
  if (rcond <= 0.0) rcond = 1e-5;  // ten times the FP32 sketch's relative rounding of C
  const int nb = 2 * s - 1;
  const size_t eb = dtype_size(bt);
  const bool b_dev = is_device_ptr(blocks);
  size_t need = b_dev ? 0 : ws_bytes((size_t)m * m * nb, eb);
  need += ws_bytes((size_t)m * ell * nb, 4) + ws_bytes((size_t)s * ell, eb) +
          ws_bytes((size_t)m * ell, eb) + ws_bytes((size_t)ms * ell, 4);
  need += 2 * ws_bytes((size_t)ms * ell, 8) + 6 * ws_bytes((size_t)ell * ell, 8) +
          2 * ws_bytes((size_t)ell, 8) + ws_bytes((size_t)ms * r, 8);
  need += 2 * sym_eig_workspace_bytes(1) + (1 << 20);
  ensure_workspace(c, need);
  Workspace& ws = c->ws;
  KRP_CUDA_CHECK(cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream));
  const void* Bd = blocks;
  if (!b_dev) {
    void* p = ws.take<char>((size_t)m * m * nb * eb);
    KRP_CUDA_CHECK(cudaMemcpyAsync(p, blocks, (size_t)m * m * nb * eb, cudaMemcpyHostToDevice,
                                   c->stream));
    Bd = p;
  }
  float* Zs = ws.take<float>((size_t)m * ell * nb);
  void* o1 = ws.take<char>((size_t)s * ell * eb);
  void* o2 = ws.take<char>((size_t)m * ell * eb);
  FactorJob jo[2] = {{o1, s, ((int64_t)s * ell + 3) / 4, 0}, {o2, m, ((int64_t)m * ell + 3) / 4, 1}};
  launch_gen_factors(seed, 0, KRP_TAG_OMEGA, ell, bt, jo, 2);
  float* Y = ws.take<float>((size_t)ms * ell);
  hankel_sketch(Bd, bt, m, m, s, o1, o2, ell, false, Y, Zs);
  double* Q = ws.take<double>((size_t)ms * ell);
  double* qw = ws.take<double>((size_t)ms * ell);
  double* R = ws.take<double>((size_t)ell * ell);
  QrJob jy{Y, Q, R, qw, ms, ell};
  qr_householder_f64(&jy, 1, c->d_status);
  double* P = ws.take<double>((size_t)ell * ell);
  dim3 g(ell, ell);
  if (bt == KRP_F32)
    psi_t_q_kernel<float><<<g, 256, 0, c->stream>>>(static_cast<const float*>(o1),
                                                    static_cast<const float*>(o2), s, m, ell, Q,
                                                    ell, P);
  else
    psi_t_q_kernel<__nv_bfloat16><<<g, 256, 0, c->stream>>>(
        static_cast<const __nv_bfloat16*>(o1), static_cast<const __nv_bfloat16*>(o2), s, m, ell,
        Q, ell, P);
  check_launch("nystrom_omega_t_q");
  double* C = ws.take<double>((size_t)ell * ell);
  matmul_f64(P, R, C, ell, ell, ell);
  nys_sym_kernel<<<1, 256, 0, c->stream>>>(C, ell);
  check_launch("nystrom_sym");
  double* Vc = ws.take<double>((size_t)ell * ell);
  double* cev = ws.take<double>((size_t)ell);
  {
    const double* Sa[1] = {C};
    double* Ua[1] = {Vc};
    double* Ea[1] = {cev};
    int lv[1] = {ell}, rv[1] = {ell};
    sym_eig_top_f64(Sa, lv, rv, Ua, 1, c->d_status, Ea);
  }
  double* G = ws.take<double>((size_t)ell * ell);
  matmul_f64(R, Vc, G, ell, ell, ell);
  nys_scale_kernel<<<1, 256, 0, c->stream>>>(G, cev, ell, rcond);
  check_launch("nystrom_scale");
  double* T = ws.take<double>((size_t)ell * ell);
  const int64_t gd[2] = {ell, ell};
  gram_mode_f64(G, 2, gd, 0, T);
  double* Ut = ws.take<double>((size_t)ell * ell);
  double* lam = ws.take<double>((size_t)ell);
  {
    const double* Sa[1] = {T};
    double* Ua[1] = {Ut};
    double* Ea[1] = {lam};
    int lv[1] = {ell}, rv[1] = {r};
    sym_eig_top_f64(Sa, lv, rv, Ua, 1, c->d_status, Ea);
  }
  double* Ud = ws.take<double>((size_t)ms * r);
  matmul_f64(Q, Ut, Ud, ms, ell, r);
  auto out = [&](double* dst, const double* src, size_t count) {
    const bool dev = is_device_ptr(dst);
    KRP_CUDA_CHECK(cudaMemcpyAsync(dst, src, count * sizeof(double),
                                   dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                   c->stream));
  };
  out(U, Ud, (size_t)ms * r);
  out(L, lam, (size_t)r);
  raise_device_status(c);
}

// Alg. 6 on a two-level block Hankel matrix (Sec. 4.3): (m s1 s2) x
// (n s1 s2), block (i1, j1) an s2 x s2 block Hankel matrix with blocks
// H_{i1+j1, i2+j2}; Omega = Omega1 kr Omega2 kr Omega3 (s1, s2, n rows, tag 0)
// and Psi = Psi1 kr Psi2 kr Psi3 (s1, s2, m rows, tag 1), draw 0.  The sketches
// use the two-level form of Eq. (4.1); steps 3-6 as for one level.
void hankel2_pipeline(const void* blocks, krp_dtype bt, int m, int n, int s1, int s2, int r,
                      int ell_r, int ell_l, uint64_t seed, double* U, double* S, double* V) {
  Ctx* c = current();
  KRP_REQUIRE(blocks, "blocks is NULL");
  KRP_REQUIRE(bt == KRP_F32 || bt == KRP_BF16, "blocks dtype must be KRP_F32 or KRP_BF16");
  KRP_REQUIRE(m >= 1 && n >= 1 && s1 >= 1 && s2 >= 1, "m, n, s1, s2 must be >= 1");
  const int64_t ms = (int64_t)m * s1 * s2, ns = (int64_t)n * s1 * s2;
  KRP_REQUIRE(ms <= (int64_t(1) << 31) && ns <= (int64_t(1) << 31), "block Hankel too large");
  if (ell_l == 0) ell_l = (int)std::ceil(1.5 * ell_r);
  KRP_REQUIRE(r >= 1 && r <= ell_r && ell_r <= ell_l, "need 1 <= r <= ell_r <= ell_l");
  KRP_REQUIRE(ell_r <= 64 && ell_l <= 256, "need ell_r <= 64 and ell_l <= 256");
  KRP_REQUIRE(ell_r <= ms && ell_l <= ns, "sketch sizes exceed the matrix");
  KRP_REQUIRE(U && S && V, "U/S/V is NULL");
  const int64_t nb = (int64_t)(2 * s1 - 1) * (2 * s2 - 1);
  const size_t eb = dtype_size(bt);
  const bool b_dev = is_device_ptr(blocks);
  size_t need = b_dev ? 0 : ws_bytes((size_t)m * n * nb, eb);
  need += ws_bytes((size_t)std::max(m, n) * ell_l * nb, 4);
  need += 2 * (ws_bytes((size_t)s1 * ell_l, eb) + ws_bytes((size_t)s2 * ell_l, eb) +
               ws_bytes((size_t)std::max(m, n) * ell_l, eb));
  need += ws_bytes((size_t)ms * ell_r, 4) + ws_bytes((size_t)ns * ell_l, 4);
  need += 3 * ws_bytes((size_t)ms * ell_r, 8) + 5 * ws_bytes((size_t)ell_l * ell_r, 8);
  need += ws_bytes((size_t)ell_r * ns, 8) + 4 * ws_bytes((size_t)ell_r * ell_r, 8);
  need += ws_bytes((size_t)ms * r, 8) + ws_bytes((size_t)ns * r, 8) + ws_bytes(r, 8);
  need += sym_eig_workspace_bytes(1) + (1 << 20);
  ensure_workspace(c, need);
  Workspace& ws = c->ws;
  KRP_CUDA_CHECK(cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream));
  const void* Bd = blocks;
  if (!b_dev) {
    void* p = ws.take<char>((size_t)m * n * nb * eb);
    KRP_CUDA_CHECK(cudaMemcpyAsync(p, blocks, (size_t)m * n * nb * eb, cudaMemcpyHostToDevice,
                                   c->stream));
    Bd = p;
  }
  float* Zs = ws.take<float>((size_t)std::max(m, n) * ell_l * nb);
  void* o1 = ws.take<char>((size_t)s1 * ell_r * eb);
  void* o2 = ws.take<char>((size_t)s2 * ell_r * eb);
  void* o3 = ws.take<char>((size_t)n * ell_r * eb);
  void* p1 = ws.take<char>((size_t)s1 * ell_l * eb);
  void* p2 = ws.take<char>((size_t)s2 * ell_l * eb);
  void* p3 = ws.take<char>((size_t)m * ell_l * eb);
  FactorJob jo[3] = {{o1, s1, ((int64_t)s1 * ell_r + 3) / 4, 0},
                     {o2, s2, ((int64_t)s2 * ell_r + 3) / 4, 1},
                     {o3, n, ((int64_t)n * ell_r + 3) / 4, 2}};
  launch_gen_factors(seed, 0, KRP_TAG_OMEGA, ell_r, bt, jo, 3);
  FactorJob jp[3] = {{p1, s1, ((int64_t)s1 * ell_l + 3) / 4, 0},
                     {p2, s2, ((int64_t)s2 * ell_l + 3) / 4, 1},
                     {p3, m, ((int64_t)m * ell_l + 3) / 4, 2}};
  launch_gen_factors(seed, 0, KRP_TAG_PSI, ell_l, bt, jp, 3);
  float* Y = ws.take<float>((size_t)ms * ell_r);
  float* Z = ws.take<float>((size_t)ns * ell_l);
  hankel2_sketch(Bd, bt, m, n, s1, s2, o1, o2, o3, ell_r, false, Y, Zs);
  hankel2_sketch(Bd, bt, m, n, s1, s2, p1, p2, p3, ell_l, true, Z, Zs);
  single_pass_tail(c, ws, Y, Z, ms, ns, r, ell_r, ell_l,
                   [&](const double* Q, double* P) {
                     dim3 g(ell_l, ell_r);
                     if (bt == KRP_F32)
                       psi3_t_q_kernel<float><<<g, 256, 0, c->stream>>>(
                           static_cast<const float*>(p1), static_cast<const float*>(p2),
                           static_cast<const float*>(p3), s1, s2, m, ell_l, Q, P);
                     else
                       psi3_t_q_kernel<__nv_bfloat16><<<g, 256, 0, c->stream>>>(
                           static_cast<const __nv_bfloat16*>(p1),
                           static_cast<const __nv_bfloat16*>(p2),
                           static_cast<const __nv_bfloat16*>(p3), s1, s2, m, ell_l, Q, P);
                     check_launch("hankel2_psi_t_q");
                   },
                   U, S, V);
}

}  // namespace krp
