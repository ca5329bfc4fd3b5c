// Sensor placement from Tucker factors (Sec. 6), FP64 on the GPU.
//
// Training: for each spatial mode i with Q_i (N_i x l_i, orthonormal
// columns), a column-pivoted Householder QR of W = Q_i^T picks l_i grid
// indices (the pivots, in the order picked), and the interpolation factor is
// A_i = Q_i (P_i^T Q_i)^{-1} with P_i^T Q_i = Q_i[idx, :].
// Test: T ~ T_hat x_1 A_1 ... x_d A_d from the measurements T_hat on the grid
// I_1 x ... x I_d.
//
// One CTA per mode runs the pivoted QR: step k computes the norms of columns
// k..N-1 over rows k..l-1 (FP64, one column per thread), takes the largest
// (ties: the lowest position) by a block reduction, swaps it into place k,
// forms the reflector of W[k:, k] in one warp and applies it to columns
// k..N-1.  The pivot decisions are taken in FP64, as in the host reference.
// (P^T Q)^{-1} is Gauss-Jordan elimination with partial pivoting on one CTA.
#include <climits>

#include "pipeline.h"

namespace krp {
namespace {

constexpr int kSpThreads = 256;
constexpr int kSpMaxL = 64;

struct SensorJob {
  const double* Q;  // N x l, column-major
  double* W;        // l x N working copy of Q^T
  int* perm;        // N
  int* idx;         // l: the picked indices
  double* Binv;     // l x l: (Q[idx, :])^{-1}
  int64_t n;
  int l;
};

__device__ __forceinline__ void better(double& v, int& i, double v2, int i2) {
  if (v2 > v || (v2 == v && i2 < i)) {
    v = v2;
    i = i2;
  }
}

__global__ void __launch_bounds__(kSpThreads) sensor_pqr_kernel(const SensorJob* __restrict__ jobs) {
  const SensorJob J = jobs[blockIdx.x];
  const int l = J.l, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int64_t n = J.n;
  double* W = J.W;
  __shared__ double v[kSpMaxL];
  __shared__ double s_tau;
  __shared__ double red_v[kSpThreads / 32];
  __shared__ int red_i[kSpThreads / 32];
  __shared__ int s_j;
  for (int64_t e = tid; e < (int64_t)l * n; e += blockDim.x) {
    const int r = (int)(e % l);
    const int64_t c = e / l;
    W[e] = J.Q[c + n * r];
  }
  for (int64_t c = tid; c < n; c += blockDim.x) J.perm[c] = (int)c;
  __syncthreads();
  for (int k = 0; k < l; ++k) {
    // the candidate of largest norm over rows k..l-1
    double bv = -1.0;
    int bi = INT_MAX;
    for (int64_t c = k + tid; c < n; c += blockDim.x) {
      const double* col = W + (int64_t)l * c;
      double s = 0.0;
      for (int r = k; r < l; ++r) s = fma(col[r], col[r], s);
      better(bv, bi, s, (int)c);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double v2 = __shfl_xor_sync(0xffffffffu, bv, o);
      const int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
      better(bv, bi, v2, i2);
    }
    if (lane == 0) {
      red_v[wid] = bv;
      red_i[wid] = bi;
    }
    __syncthreads();
    if (tid == 0) {
      double v0 = red_v[0];
      int i0 = red_i[0];
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w) better(v0, i0, red_v[w], red_i[w]);
      s_j = i0;
    }
    __syncthreads();
    const int j = s_j;
    if (j != k) {
      for (int r = tid; r < l; r += blockDim.x) {
        const double a = W[r + (int64_t)l * k];
        W[r + (int64_t)l * k] = W[r + (int64_t)l * j];
        W[r + (int64_t)l * j] = a;
      }
      if (tid == 0) {
        const int p = J.perm[k];
        J.perm[k] = J.perm[j];
        J.perm[j] = p;
      }
    }
    __syncthreads();
    // reflector mapping W[k:, k] onto alpha e_1, alpha = -sign(W[k, k]) ||W[k:, k]||
    if (wid == 0) {
      double ss = 0.0;
      for (int r = k + lane; r < l; r += 32) {
        const double x = W[r + (int64_t)l * k];
        ss = fma(x, x, ss);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
      const double x0 = W[k + (int64_t)l * k];
      const double nx = sqrt(ss);
      const double alpha = x0 >= 0.0 ? -nx : nx;
      double vv = 0.0;
      for (int r = k + lane; r < l; r += 32) {
        const double x = W[r + (int64_t)l * k] - (r == k ? alpha : 0.0);
        v[r - k] = x;
        vv = fma(x, x, vv);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) vv += __shfl_xor_sync(0xffffffffu, vv, o);
      if (lane == 0) s_tau = vv > 0.0 ? 2.0 / vv : 0.0;
    }
    __syncthreads();
    const double tau = s_tau;
    if (tau != 0.0) {
      for (int64_t c = k + tid; c < n; c += blockDim.x) {
        double* col = W + (int64_t)l * c;
        double w = 0.0;
        for (int r = k; r < l; ++r) w = fma(v[r - k], col[r], w);
        w *= tau;
        for (int r = k; r < l; ++r) col[r] = fma(-w, v[r - k], col[r]);
      }
    }
    __syncthreads();
  }
  for (int k = tid; k < l; k += blockDim.x) J.idx[k] = J.perm[k];
}

// Binv = (Q[idx, :])^{-1} by Gauss-Jordan elimination with partial pivoting
// (largest |entry| of the column, ties: the lowest row) on [B | I] in shared
// memory; a zero pivot raises KRP_ENUMERIC.
__global__ void __launch_bounds__(kSpThreads)
    sensor_inv_kernel(const SensorJob* __restrict__ jobs, int* status) {
  const SensorJob J = jobs[blockIdx.x];
  const int l = J.l, tid = threadIdx.x, w2 = 2 * l;
  extern __shared__ double aug[];  // l x 2l, row-major
  __shared__ double fac[kSpMaxL];
  __shared__ int s_p;
  for (int e = tid; e < l * w2; e += blockDim.x) {
    const int a = e / w2, b = e % w2;
    aug[e] = b < l ? J.Q[J.idx[a] + J.n * b] : (b - l == a ? 1.0 : 0.0);
  }
  __syncthreads();
  for (int p = 0; p < l; ++p) {
    if (tid == 0) {
      int best = p;
      double bv = fabs(aug[p * w2 + p]);
      for (int r = p + 1; r < l; ++r) {
        const double x = fabs(aug[r * w2 + p]);
        if (x > bv) {
          bv = x;
          best = r;
        }
      }
      s_p = bv > 0.0 ? best : -1;
      if (bv == 0.0) atomicCAS(status, 0, static_cast<int>(KRP_ENUMERIC));
    }
    __syncthreads();
    const int pr = s_p;
    if (pr < 0) return;  // uniform: every thread read the same s_p
    if (pr != p)
      for (int b = tid; b < w2; b += blockDim.x) {
        const double t = aug[p * w2 + b];
        aug[p * w2 + b] = aug[pr * w2 + b];
        aug[pr * w2 + b] = t;
      }
    __syncthreads();
    const double piv = aug[p * w2 + p];
    __syncthreads();
    for (int b = tid; b < w2; b += blockDim.x) aug[p * w2 + b] /= piv;
    __syncthreads();
    // the multipliers of column p, read before any row is updated
    for (int a = tid; a < l; a += blockDim.x) fac[a] = aug[a * w2 + p];
    __syncthreads();
    for (int e = tid; e < l * w2; e += blockDim.x) {
      const int a = e / w2, b = e % w2;
      if (a != p) aug[e] = fma(-fac[a], aug[p * w2 + b], aug[e]);
    }
    __syncthreads();
  }
  for (int e = tid; e < l * l; e += blockDim.x) {
    const int a = e % l, b = e / l;
    J.Binv[a + (int64_t)l * b] = aug[a * w2 + l + b];
  }
}

// out[a + l * c] = A[c + n * a]: the l x N transpose of an N x l matrix.
__global__ void transpose_f64_kernel(const double* __restrict__ A, int64_t n, int l,
                                     double* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * l;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(e % l);
    const int64_t c = e / l;
    out[e] = A[c + n * a];
  }
}

__global__ void f32_to_f64_kernel(const float* __restrict__ x, int64_t n, double* __restrict__ y) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    y[e] = x[e];
}

__global__ void f64_to_f32_kernel(const double* __restrict__ x, int64_t n, float* __restrict__ y) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    y[e] = (float)x[e];
}

int sp_grid(int64_t n) {
  const int64_t g = (n + 255) / 256;
  return (int)(g < 1 ? 1 : (g > 4096 ? 4096 : g));
}

size_t expanded_max(int d, const int64_t* dims, const int* ells, size_t* first) {
  size_t cur = 1;
  for (int i = 0; i < d; ++i) cur *= (size_t)ells[i];
  if (first) *first = cur;
  size_t big = cur;
  for (int i = 0; i < d; ++i) {
    cur = cur / ells[i] * (size_t)dims[i];
    big = std::max(big, cur);
  }
  return big;
}

}  // namespace

size_t sensor_select_workspace_bytes(int d, const int64_t* dims, const int* ells) {
  size_t b = ws_bytes((size_t)d, sizeof(SensorJob)) + (1 << 16);
  for (int i = 0; i < d; ++i)
    b += ws_bytes((size_t)dims[i] * ells[i], 8) + ws_bytes((size_t)dims[i], 4) +
         ws_bytes((size_t)ells[i] * ells[i], 8);
  return b;
}

void sensor_select(int d, const int64_t* dims, const int* ells, const double* const* Q,
                   int* const* idx, double* const* A) {
  Ctx* c = current();
  Workspace& ws = c->ws;
  std::vector<SensorJob> jobs(d);
  int lmax = 1;
  for (int i = 0; i < d; ++i) {
    SensorJob& j = jobs[i];
    j.Q = Q[i];
    j.n = dims[i];
    j.l = ells[i];
    j.W = ws.take<double>((size_t)dims[i] * ells[i]);
    j.perm = ws.take<int>((size_t)dims[i]);
    j.idx = idx[i];
    j.Binv = ws.take<double>((size_t)ells[i] * ells[i]);
    lmax = std::max(lmax, ells[i]);
  }
  SensorJob* dj = ws.take<SensorJob>(d);
  KRP_CUDA_CHECK(cudaMemcpyAsync(dj, jobs.data(), sizeof(SensorJob) * d, cudaMemcpyHostToDevice,
                                 c->stream));
  sensor_pqr_kernel<<<d, kSpThreads, 0, c->stream>>>(dj);
  check_launch("sensor_pqr");
  const size_t sm = sizeof(double) * (size_t)lmax * 2 * lmax;
  KRP_CUDA_CHECK(cudaFuncSetAttribute(sensor_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)sm));
  sensor_inv_kernel<<<d, kSpThreads, sm, c->stream>>>(dj, c->d_status);
  check_launch("sensor_inv");
  for (int i = 0; i < d; ++i) matmul_f64(Q[i], jobs[i].Binv, A[i], dims[i], ells[i], ells[i]);
}

size_t sensor_reconstruct_workspace_bytes(int d, const int64_t* dims, const int* ells) {
  size_t b = 2 * ws_bytes(expanded_max(d, dims, ells, nullptr), 8) + (1 << 16);
  for (int i = 0; i < d; ++i) b += ws_bytes((size_t)dims[i] * ells[i], 8);
  return b;
}

void sensor_reconstruct(int d, const int64_t* dims, const int* ells, const double* const* A,
                        const float* That, float* out) {
  Ctx* c = current();
  Workspace& ws = c->ws;
  size_t n0 = 1;
  const size_t big = expanded_max(d, dims, ells, &n0);
  double* g0 = ws.take<double>(big);
  double* g1 = ws.take<double>(big);
  f32_to_f64_kernel<<<sp_grid((int64_t)n0), 256, 0, c->stream>>>(That, (int64_t)n0, g0);
  check_launch("sensor_widen");
  int64_t cd[KRP_MAXD];
  size_t cur = n0;
  for (int i = 0; i < d; ++i) cd[i] = ells[i];
  for (int i = 0; i < d; ++i) {
    double* At = ws.take<double>((size_t)dims[i] * ells[i]);
    transpose_f64_kernel<<<sp_grid(dims[i] * ells[i]), 256, 0, c->stream>>>(A[i], dims[i], ells[i],
                                                                              At);
    check_launch("sensor_transpose");
    ttm_small_f64(g0, d, cd, i, At, (int)dims[i], g1);
    cur = cur / ells[i] * (size_t)dims[i];
    cd[i] = dims[i];
    std::swap(g0, g1);
  }
  f64_to_f32_kernel<<<sp_grid((int64_t)cur), 256, 0, c->stream>>>(g0, (int64_t)cur, out);
  check_launch("sensor_narrow");
}

}  // namespace krp
