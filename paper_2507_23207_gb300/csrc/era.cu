// Eigensystem realization from the rank-r SVD of a block Hankel matrix (the
// use Sec. 4.2 makes of Alg. 6), in FP64 on the GPU.
//
// With M ~ U S V^T (block (i, j) of M = h_{i+j-1}, 1-based, m x n blocks,
// s x s of them), the observability factor is O = U S^{1/2} and the
// controllability factor G = S^{1/2} V^T.  The block Hankel matrix shifted by
// one block, H_up (block (i, j) = h_{i+j}, i = 1..s-1, j = 1..s), equals
// O_top A G with O_top the first (s-1) m rows of O, so the state matrix is
//   A = O_top^+ H_up G^+,   G^+ = V S^{-1/2}
// (up to a similarity transform; its eigenvalues are the system's).
//   era_hg_kernel:    P = H_up G^+, (s-1) m x r, from the blocks directly
//   era_gram_kernel:  N = O_top^T O_top and B = O_top^T P (r x r each)
//   era_solve_kernel: A = N^{-1} B by Cholesky (O_top is well conditioned:
//                     its condition number is that of S^{1/2} on the orthonormal
//                     U_top, ~35 on a rank-40 block Hankel), then the
//                     eigenvalues of A by Householder reduction to Hessenberg
//                     form and the Francis double-shift QR iteration
//                     (Golub & Van Loan, Matrix Computations, Sec. 7.4-7.5).
#include "pipeline.h"

namespace krp {
namespace {

template <class BT>
__device__ __forceinline__ double ldh(const BT* p, int64_t i);
template <>
__device__ __forceinline__ double ldh<float>(const float* p, int64_t i) {
  return static_cast<double>(p[i]);
}
template <>
__device__ __forceinline__ double ldh<__nv_bfloat16>(const __nv_bfloat16* p, int64_t i) {
  return static_cast<double>(__bfloat162float(p[i]));
}

// P[(i a) + rows c] = sum_{j < s} sum_{b < n} h_{i+j+1}[a, b] V[(j n + b) + n s c] / sqrt(S[c])
// (0-based blocks: block k at blocks + k m n, column-major m x n), rows = (s-1) m
template <class BT>
__global__ void era_hg_kernel(const BT* __restrict__ blocks, int m, int n, int s, int r,
                              const double* __restrict__ V, const double* __restrict__ S,
                              double* __restrict__ P) {
  const int64_t rows = static_cast<int64_t>(s - 1) * m;
  const int64_t ns = static_cast<int64_t>(n) * s;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < rows * r;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = e % rows;
    const int c = static_cast<int>(e / rows);
    const int i = static_cast<int>(row / m), a = static_cast<int>(row % m);
    const double* vc = V + ns * c;
    double acc = 0.0;
    for (int j = 0; j < s; ++j) {
      const BT* h = blocks + static_cast<int64_t>(i + j + 1) * m * n + a;
      const double* vj = vc + static_cast<int64_t>(j) * n;
      for (int b = 0; b < n; ++b) acc = fma(ldh(h, static_cast<int64_t>(m) * b), vj[b], acc);
    }
    P[e] = acc / sqrt(S[c]);
  }
}

// N += O_top^T O_top and B += O_top^T P over the CTA's chunk of rows, with
// O_top[row, c] = U[row + ms c] sqrt(S[c]); N and B (r x r, column-major)
// are zeroed before the launch and receive FP64 atomics.
__global__ void __launch_bounds__(256) era_gram_kernel(const double* __restrict__ U, int64_t ms,
                                                       int64_t rows, int r,
                                                       const double* __restrict__ S,
                                                       const double* __restrict__ P,
                                                       int64_t rows_per, double* __restrict__ Nm,
                                                       double* __restrict__ B) {
  const int64_t r0 = blockIdx.x * rows_per;
  const int64_t r1 = min(rows, r0 + rows_per);
  if (r0 >= r1) return;
  for (int e = threadIdx.x; e < 2 * r * r; e += blockDim.x) {
    const int which = e / (r * r);
    const int c1 = (e % (r * r)) % r, c2 = (e % (r * r)) / r;
    const double* u1 = U + ms * c1;
    double acc = 0.0;
    if (which == 0) {
      if (c1 > c2) continue;  // symmetric: the upper triangle, mirrored below
      const double* u2 = U + ms * c2;
      for (int64_t row = r0; row < r1; ++row) acc = fma(u1[row], u2[row], acc);
      acc *= sqrt(S[c1]) * sqrt(S[c2]);
      atomicAdd(Nm + c1 + static_cast<int64_t>(r) * c2, acc);
      if (c1 != c2) atomicAdd(Nm + c2 + static_cast<int64_t>(r) * c1, acc);
    } else {
      const double* p2 = P + rows * c2;
      for (int64_t row = r0; row < r1; ++row) acc = fma(u1[row], p2[row], acc);
      atomicAdd(B + c1 + static_cast<int64_t>(r) * c2, acc * sqrt(S[c1]));
    }
  }
}

constexpr int kEraMaxR = 64;
constexpr int kEraEP = kEraMaxR + 1;  // row pitch of the shared matrices

// Householder vector of x (length len, in shared memory) into v, with
// beta = 2 / v^T v (0: nothing to reflect); one thread.
__device__ double house(const double* x, int len, double* v) {
  double nx = 0.0;
  for (int i = 0; i < len; ++i) nx = fma(x[i], x[i], nx);
  nx = sqrt(nx);
  for (int i = 0; i < len; ++i) v[i] = x[i];
  if (nx == 0.0) return 0.0;
  v[0] -= -copysign(nx, x[0]);
  double vv = 0.0;
  for (int i = 0; i < len; ++i) vv = fma(v[i], v[i], vv);
  return vv > 0.0 ? 2.0 / vv : 0.0;
}

// One CTA: N (r x r, SPD) and B from global memory; A = N^{-1} B by Cholesky
// (written to A_out if not null); A reduced to upper Hessenberg form by
// Householder reflections (all threads), then its eigenvalues by the Francis
// double-shift QR iteration on the active diagonal block (warp 0: the
// reflector's row and column updates spread over the lanes, its scalar work
// repeated in every lane).  Eigenvalues into wr, wi in deflation order;
// KRP_ENUMERIC in status if N is not positive definite, a value is not
// finite, or a block needs more than 100 iterations.
__global__ void __launch_bounds__(256) era_solve_kernel(const double* __restrict__ Ng,
                                                        const double* __restrict__ Bg, int r,
                                                        double* __restrict__ A_out,
                                                        double* __restrict__ wr,
                                                        double* __restrict__ wi, int* status) {
  extern __shared__ double era_smem[];  // L, then H: kEraMaxR rows of pitch kEraEP each
  double(*L)[kEraEP] = reinterpret_cast<double(*)[kEraEP]>(era_smem);
  double(*H)[kEraEP] = reinterpret_cast<double(*)[kEraEP]>(era_smem + kEraMaxR * kEraEP);
  __shared__ double v[kEraMaxR];
  __shared__ double sb;
  __shared__ int bad;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) bad = 0;
  for (int e = tid; e < r * r; e += nt) {
    L[e % r][e / r] = Ng[e];
    H[e % r][e / r] = Bg[e];
  }
  __syncthreads();
  // Cholesky N = L L^T (lower triangle of L), one column per step
  for (int j = 0; j < r; ++j) {
    if (tid == 0) {
      const double d = L[j][j];
      if (!(d > 0.0) || !isfinite(d)) bad = 1;
      L[j][j] = sqrt(fmax(d, 0.0));
    }
    __syncthreads();
    const double ljj = L[j][j];
    for (int i = j + 1 + tid; i < r; i += nt) L[i][j] = ljj > 0.0 ? L[i][j] / ljj : 0.0;
    __syncthreads();
    for (int e = tid; e < (r - j - 1) * (r - j - 1); e += nt) {
      const int i = j + 1 + e % (r - j - 1), k = j + 1 + e / (r - j - 1);
      if (k <= i) L[i][k] = fma(-L[i][j], L[k][j], L[i][k]);
    }
    __syncthreads();
  }
  // L Y = B, then L^T A = Y, column by column of B (one thread per column)
  for (int c = tid; c < r; c += nt) {
    for (int i = 0; i < r; ++i) {
      double acc = H[i][c];
      for (int k = 0; k < i; ++k) acc = fma(-L[i][k], H[k][c], acc);
      H[i][c] = L[i][i] > 0.0 ? acc / L[i][i] : 0.0;
    }
    for (int i = r - 1; i >= 0; --i) {
      double acc = H[i][c];
      for (int k = i + 1; k < r; ++k) acc = fma(-L[k][i], H[k][c], acc);
      H[i][c] = L[i][i] > 0.0 ? acc / L[i][i] : 0.0;
    }
  }
  __syncthreads();
  if (A_out)
    for (int e = tid; e < r * r; e += nt) A_out[e] = H[e % r][e / r];
  // Householder reduction to upper Hessenberg form
  for (int k = 0; k + 2 < r; ++k) {
    if (tid == 0) {
      double x[kEraMaxR];
      for (int i = k + 1; i < r; ++i) x[i - k - 1] = H[i][k];
      sb = house(x, r - k - 1, v);
    }
    __syncthreads();
    const double beta = sb;
    const int len = r - k - 1;
    if (beta != 0.0) {
      for (int j = k + tid; j < r; j += nt) {  // rows k+1..r-1 of columns j >= k
        double w = 0.0;
        for (int i = 0; i < len; ++i) w = fma(v[i], H[k + 1 + i][j], w);
        for (int i = 0; i < len; ++i) H[k + 1 + i][j] = fma(-beta * w, v[i], H[k + 1 + i][j]);
      }
      __syncthreads();
      for (int i = tid; i < r; i += nt) {  // columns k+1..r-1 of every row
        double w = 0.0;
        for (int j = 0; j < len; ++j) w = fma(H[i][k + 1 + j], v[j], w);
        for (int j = 0; j < len; ++j) H[i][k + 1 + j] = fma(-beta * w, v[j], H[i][k + 1 + j]);
      }
    }
    __syncthreads();
  }
  if (tid >= 32) return;
  // Francis double-shift QR on the active block [p, q] (warp 0)
  const int lane = tid;
  const double eps = 2.220446049250313e-16;
  int q = r - 1, it = 0;
  while (q >= 0) {
    int p = q;
    while (p > 0) {
      const double sub = fabs(H[p][p - 1]);
      const double ds = fabs(H[p][p]) + fabs(H[p - 1][p - 1]);
      if (sub <= eps * (ds > 0.0 ? ds : 1.0)) break;
      --p;
    }
    __syncwarp();
    if (p > 0 && lane == 0) H[p][p - 1] = 0.0;
    __syncwarp();
    if (p == q) {
      if (lane == 0) {
        wr[q] = H[q][q];
        wi[q] = 0.0;
      }
      --q;
      it = 0;
      continue;
    }
    if (p == q - 1) {  // a 2 x 2 block: two real or a complex pair
      const double a = H[q - 1][q - 1], b = H[q - 1][q], c = H[q][q - 1], d = H[q][q];
      const double h = 0.5 * (a - d), mid = 0.5 * (a + d), disc = h * h + b * c;
      if (lane == 0) {
        if (disc >= 0.0) {
          const double sq = sqrt(disc);
          const double l1 = mid != 0.0 ? mid + copysign(sq, mid) : mid + sq;
          wr[q - 1] = l1;
          wr[q] = l1 != 0.0 ? (a * d - b * c) / l1 : mid - sq;
          wi[q - 1] = 0.0;
          wi[q] = 0.0;
        } else {
          const double sq = sqrt(-disc);
          wr[q - 1] = mid;
          wr[q] = mid;
          wi[q - 1] = sq;
          wi[q] = -sq;
        }
      }
      q -= 2;
      it = 0;
      continue;
    }
    if (++it > 100) {
      if (lane == 0) bad = 1;
      break;
    }
    double s_, t_;
    if (it == 11 || it == 21) {  // a shift off the stagnating pair
      const double mu = H[q][q] + fabs(H[q][q - 1]) + fabs(H[q - 1][q - 2]);
      s_ = 2.0 * mu;
      t_ = mu * mu;
    } else {
      s_ = H[q - 1][q - 1] + H[q][q];
      t_ = H[q - 1][q - 1] * H[q][q] - H[q - 1][q] * H[q][q - 1];
    }
    double x = H[p][p] * H[p][p] + H[p][p + 1] * H[p + 1][p] - s_ * H[p][p] + t_;
    double y = H[p + 1][p] * (H[p][p] + H[p + 1][p + 1] - s_);
    double z = H[p + 1][p] * H[p + 2][p + 1];
    for (int k = p; k <= q - 2; ++k) {
      // 3 x 3 reflector taking (x, y, z) to a multiple of e_1
      const double nrm = sqrt(x * x + y * y + z * z);
      const double v0 = x + copysign(nrm, x), v1 = y, v2 = z;
      const double vv = v0 * v0 + v1 * v1 + v2 * v2;
      if (nrm > 0.0 && vv > 0.0) {
        const double beta = 2.0 / vv;
        for (int j = max(p, k - 1) + lane; j <= q; j += 32) {
          const double w = beta * (v0 * H[k][j] + v1 * H[k + 1][j] + v2 * H[k + 2][j]);
          H[k][j] -= w * v0;
          H[k + 1][j] -= w * v1;
          H[k + 2][j] -= w * v2;
        }
        __syncwarp();
        for (int i = p + lane; i <= min(k + 3, q); i += 32) {
          const double w = beta * (H[i][k] * v0 + H[i][k + 1] * v1 + H[i][k + 2] * v2);
          H[i][k] -= w * v0;
          H[i][k + 1] -= w * v1;
          H[i][k + 2] -= w * v2;
        }
        __syncwarp();
      }
      x = H[k + 1][k];
      y = H[k + 2][k];
      z = (k + 3 <= q) ? H[k + 3][k] : 0.0;
      __syncwarp();
    }
    {  // 2 x 2 reflector on rows / columns q-1, q
      const double nrm = sqrt(x * x + y * y);
      const double v0 = x + copysign(nrm, x), v1 = y;
      const double vv = v0 * v0 + v1 * v1;
      if (nrm > 0.0 && vv > 0.0) {
        const double beta = 2.0 / vv;
        for (int j = max(p, q - 2) + lane; j <= q; j += 32) {
          const double w = beta * (v0 * H[q - 1][j] + v1 * H[q][j]);
          H[q - 1][j] -= w * v0;
          H[q][j] -= w * v1;
        }
        __syncwarp();
        for (int i = p + lane; i <= q; i += 32) {
          const double w = beta * (H[i][q - 1] * v0 + H[i][q] * v1);
          H[i][q - 1] -= w * v0;
          H[i][q] -= w * v1;
        }
        __syncwarp();
      }
    }
  }
  __syncwarp();
  if (lane == 0) {
    for (int i = 0; i < r; ++i)
      if (!isfinite(wr[i]) || !isfinite(wi[i])) bad = 1;
    if (bad) atomicCAS(status, 0, static_cast<int>(KRP_ENUMERIC));
  }
}

}  // namespace

void era_realize(const void* blocks, krp_dtype bt, int m, int n, int s, int r, const double* U,
                 const double* S, const double* V, double* A, double* wr, double* wi) {
  Ctx* c = current();
  const int64_t rows = static_cast<int64_t>(s - 1) * m;
  double* P = c->ws.take<double>((size_t)rows * r);
  double* Nm = c->ws.take<double>((size_t)r * r);
  double* B = c->ws.take<double>((size_t)r * r);
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((rows * r + 255) / 256, 8192));
  if (bt == KRP_F32)
    era_hg_kernel<float><<<grid, 256, 0, stream()>>>(static_cast<const float*>(blocks), m, n, s, r, V,
                                                     S, P);
  else
    era_hg_kernel<__nv_bfloat16><<<grid, 256, 0, stream()>>>(
        static_cast<const __nv_bfloat16*>(blocks), m, n, s, r, V, S, P);
  check_launch("era_hg");
  KRP_CUDA_CHECK(cudaMemsetAsync(Nm, 0, sizeof(double) * r * r, stream()));
  KRP_CUDA_CHECK(cudaMemsetAsync(B, 0, sizeof(double) * r * r, stream()));
  const int gchunks = (int)std::max<int64_t>(1, std::min<int64_t>(2 * c->num_sms, (rows + 7) / 8));
  const int64_t per = (rows + gchunks - 1) / gchunks;
  era_gram_kernel<<<gchunks, 256, 0, stream()>>>(U, static_cast<int64_t>(m) * s, rows, r, S, P, per,
                                                 Nm, B);
  check_launch("era_gram");
  const size_t smem = sizeof(double) * 2 * kEraMaxR * kEraEP;
  KRP_CUDA_CHECK(cudaFuncSetAttribute(era_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      static_cast<int>(smem)));
  era_solve_kernel<<<1, 256, smem, stream()>>>(Nm, B, r, A, wr, wi, c->d_status);
  check_launch("era_solve");
}

size_t era_workspace_bytes(int m, int s, int r) {
  return ws_bytes((size_t)(s - 1) * m * r, 8) + 2 * ws_bytes((size_t)r * r, 8) + (1 << 12);
}

}  // namespace krp
