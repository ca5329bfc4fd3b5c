// Recompression of the Hadamard (elementwise) product of two Tucker tensors
// with KRP sketches (Sec. 5, its opening), FP64, without forming the product.
//
// With X = G x {U_j} (core r_1 x ... x r_d) and Y = H x {V_j} (core s_j), the
// product Z = X * Y is the Tucker tensor with the Kronecker core C = G (x) H
// (index c_j = a_j + r_j b_j) and the face-splitting factors
// W_j[i, c_j] = U_j[i, a_j] V_j[i, b_j].  RHOSVD-KRP-MEMO of Z (one factor set
// Omega_j, n_j x l) then needs only small objects:
//   sketch   Y_n = Z_(n) (kr_{j != n} Omega_j) = W_n MTTKRP_n(C, {P_j}),
//            P_j = W_j^T Omega_j (r_j s_j x l)   (mixed-product property)
//   QR       Y_n = Q_n R_n (FP64 Householder)
//   core     G_Z = C x_1 (Q_1^T W_1) ... x_d (Q_d^T W_d)
//   error    ||Z||^2 = <C, C x_j (W_j^T W_j)>, ||Z_hat||^2 = ||G_Z||^2 (Q_j
//            orthonormal), e = sqrt(max(0, ||Z||^2 - ||G_Z||^2)) / ||Z||
//            (exact up to cancellation, which limits it to e >~ 1e-7).
// Every step is a small FP64 contraction; the cost is dominated by the core
// MTTKRP, prod_j (r_j s_j) l d flops, against l prod_j n_j for a sketch of
// the explicit product.
#include "pipeline.h"

namespace krp {
namespace {

struct Dims8 {
  int64_t v[KRP_MAXD];
};

// out[(a + r b) + r s k] = sum_i U[i + n a] V[i + n b] F[i + n k]
__global__ void fs_contract_kernel(const double* __restrict__ U, const double* __restrict__ V,
                                   const double* __restrict__ F, int64_t n, int r, int s, int ell,
                                   double* __restrict__ out) {
  const int64_t total = (int64_t)r * s * ell;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(e % r);
    const int b = (int)((e / r) % s);
    const int k = (int)(e / ((int64_t)r * s));
    const double* u = U + n * a;
    const double* v = V + n * b;
    const double* f = F + n * k;
    double acc = 0.0;
    for (int64_t i = 0; i < n; ++i) acc = fma(u[i] * v[i], f[i], acc);
    out[e] = acc;
  }
}

// C[c] = G[a] H[b] with c_j = a_j + r_j b_j (all indices mode-1 fastest)
__global__ void kron_core_kernel(const double* __restrict__ G, const double* __restrict__ H, int d,
                                 Dims8 r, Dims8 s, int64_t total, double* __restrict__ C) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t rem = e, gi = 0, hi = 0, gs = 1, hs = 1;
    for (int j = 0; j < d; ++j) {
      const int64_t cj = rem % (r.v[j] * s.v[j]);
      rem /= r.v[j] * s.v[j];
      gi += (cj % r.v[j]) * gs;
      hi += (cj / r.v[j]) * hs;
      gs *= r.v[j];
      hs *= s.v[j];
    }
    C[e] = G[gi] * H[hi];
  }
}

struct PtrList {
  const double* p[KRP_MAXD];
};

// out[c_n + cd_n k] = sum_{c_j, j != n} C[c] prod_{j != n} P_j[c_j + cd_j k],
// one CTA per output (c_n, k): the threads split the modes other than n and
// j0 (the first mode other than n), and each runs the j0 index innermost
// (no index arithmetic in the inner loop); block sum at the end.
constexpr int kMtThreads = 128;
__global__ void __launch_bounds__(kMtThreads)
    small_mttkrp_kernel(const double* __restrict__ C, int d, Dims8 cd, int n, PtrList P, int ell,
                        double* __restrict__ out) {
  const int64_t e = blockIdx.x;
  const int64_t c_n = e % cd.v[n];
  const int k = (int)(e / cd.v[n]);
  int64_t stride[KRP_MAXD];
  int64_t st = 1;
  for (int j = 0; j < d; ++j) {
    stride[j] = st;
    st *= cd.v[j];
  }
  double acc = 0.0;
  if (d == 1) {
    acc = threadIdx.x == 0 ? C[c_n] : 0.0;
  } else {
    const int j0 = n == 0 ? 1 : 0;
    int64_t rest = 1;
    for (int j = 0; j < d; ++j)
      if (j != n && j != j0) rest *= cd.v[j];
    const int64_t r0 = cd.v[j0], s0 = stride[j0];
    const double* p0 = P.p[j0] + r0 * k;
    for (int64_t o = threadIdx.x; o < rest; o += blockDim.x) {
      int64_t rem = o, base = c_n * stride[n];
      double w = 1.0;
      for (int j = 0; j < d; ++j) {
        if (j == n || j == j0) continue;
        const int64_t cj = rem % cd.v[j];
        rem /= cd.v[j];
        base += cj * stride[j];
        w *= P.p[j][cj + cd.v[j] * k];
      }
      const double* cp = C + base;
      double part = 0.0;
      for (int64_t c0 = 0; c0 < r0; ++c0) part = fma(cp[c0 * s0], p0[c0], part);
      acc = fma(w, part, acc);
    }
  }
  __shared__ double red[kMtThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kMtThreads / 32; ++w) t += red[w];
    out[e] = t;
  }
}

// Y[i + n k] = sum_{a, b} U[i + n a] V[i + n b] M[(a + r b) + r s k]
__global__ void expand_rows_kernel(const double* __restrict__ U, const double* __restrict__ V,
                                   const double* __restrict__ M, int64_t n, int r, int s, int ell,
                                   double* __restrict__ Y) {
  const int64_t total = n * ell;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % n;
    const int k = (int)(e / n);
    const double* m = M + (int64_t)r * s * k;
    double acc = 0.0;
    for (int b = 0; b < s; ++b) {
      const double vb = V[i + n * b];
      double part = 0.0;
      for (int a = 0; a < r; ++a) part = fma(U[i + n * a], m[a + r * b], part);
      acc = fma(vb, part, acc);
    }
    Y[e] = acc;
  }
}

// W[i + n (a + r b)] = U[i + n a] V[i + n b]
__global__ void face_split_kernel(const double* __restrict__ U, const double* __restrict__ V,
                                  int64_t n, int r, int s, double* __restrict__ W) {
  const int64_t total = n * r * s;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % n;
    const int64_t c = e / n;
    W[e] = U[i + n * (c % r)] * V[i + n * (c / r)];
  }
}

__global__ void dot_kernel(const double* __restrict__ x, const double* __restrict__ y, int64_t n,
                           double* __restrict__ out) {
  double acc = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    acc = fma(x[e], y[e], acc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, acc);
}

int hd_grid(int64_t n) {
  const int64_t g = (n + 255) / 256;
  return (int)(g < 1 ? 1 : (g > 4096 ? 4096 : g));
}

// Largest intermediate of a TTM chain that maps dims from[] to to[] mode by mode.
size_t chain_max(int d, const int64_t* from, const int64_t* to) {
  size_t cur = 1;
  for (int j = 0; j < d; ++j) cur *= (size_t)from[j];
  size_t big = cur;
  for (int j = 0; j < d; ++j) {
    cur = cur / from[j] * (size_t)to[j];
    big = std::max(big, cur);
  }
  return big;
}

}  // namespace

size_t hadamard_workspace_bytes(int d, const int64_t* dims, const int* rg, const int* rh, int ell) {
  int64_t cd[KRP_MAXD], ld[KRP_MAXD];
  size_t ncore = 1, b = 1 << 20;
  for (int j = 0; j < d; ++j) {
    cd[j] = (int64_t)rg[j] * rh[j];
    ld[j] = ell;
    ncore *= (size_t)cd[j];
  }
  b += ws_bytes(ncore, 8) + 2 * ws_bytes(chain_max(d, cd, ld), 8) + 2 * ws_bytes(ncore, 8);
  for (int j = 0; j < d; ++j) {
    b += ws_bytes((size_t)dims[j] * ell, 8) * 4 + 3 * ws_bytes((size_t)cd[j] * ell, 8);
    b += ws_bytes((size_t)dims[j] * cd[j], 8) + ws_bytes((size_t)cd[j] * cd[j], 8);
  }
  return b + ws_bytes(d, sizeof(QrJob)) + ws_bytes(2, 8);
}

void hadamard_rhosvd(int d, const int64_t* dims, const int* rg, const double* G,
                     const double* const* U, const int* rh, const double* H,
                     const double* const* V, int ell, uint64_t seed, double* core,
                     double* const* factors, double* rel_error) {
  Ctx* c = current();
  Workspace& ws = c->ws;
  cudaStream_t st = c->stream;
  Dims8 r{}, s{}, cdd{};
  int64_t cd[KRP_MAXD], ld[KRP_MAXD];
  size_t ncore = 1;
  for (int j = 0; j < d; ++j) {
    r.v[j] = rg[j];
    s.v[j] = rh[j];
    cd[j] = cdd.v[j] = (int64_t)rg[j] * rh[j];
    ld[j] = ell;
    ncore *= (size_t)cd[j];
  }
  // C = G (x) H
  double* C = ws.take<double>(ncore);
  kron_core_kernel<<<hd_grid((int64_t)ncore), 256, 0, st>>>(G, H, d, r, s, (int64_t)ncore, C);
  check_launch("hadamard_kron_core");
  // one factor set Omega_j (n_j x l), FP64, draw 0 (the MEMO set)
  std::vector<double*> om(d);
  std::vector<FactorJob> fj(d);
  for (int j = 0; j < d; ++j) {
    om[j] = ws.take<double>((size_t)dims[j] * ell);
    fj[j] = FactorJob{om[j], dims[j], ((int64_t)dims[j] * ell + 3) / 4, (uint32_t)j};
  }
  launch_gen_factors(seed, KRP_DRAW_MEMO, KRP_TAG_OMEGA, ell, KRP_F64, fj.data(), d);
  // P_j = W_j^T Omega_j
  PtrList P{};
  for (int j = 0; j < d; ++j) {
    double* p = ws.take<double>((size_t)cd[j] * ell);
    fs_contract_kernel<<<hd_grid(cd[j] * ell), 256, 0, st>>>(U[j], V[j], om[j], dims[j], rg[j],
                                                            rh[j], ell, p);
    check_launch("hadamard_fs_contract");
    P.p[j] = p;
  }
  // sketches Y_n = W_n MTTKRP_n(C, {P_j}) and their QR
  std::vector<QrJob> jobs(d);
  for (int n = 0; n < d; ++n) {
    double* M = ws.take<double>((size_t)cd[n] * ell);
    small_mttkrp_kernel<<<(unsigned)(cd[n] * ell), kMtThreads, 0, st>>>(C, d, cdd, n, P, ell, M);
    check_launch("hadamard_mttkrp");
    double* Yn = ws.take<double>((size_t)dims[n] * ell);
    expand_rows_kernel<<<hd_grid(dims[n] * ell), 256, 0, st>>>(U[n], V[n], M, dims[n], rg[n],
                                                              rh[n], ell, Yn);
    check_launch("hadamard_expand_rows");
    QrJob q{nullptr, factors[n], nullptr, ws.take<double>((size_t)dims[n] * ell), dims[n], ell};
    q.Y64 = Yn;
    jobs[n] = q;
  }
  qr_householder_f64(jobs.data(), d, c->d_status);
  // core G_Z = C x_j (Q_j^T W_j): ttm_small contracts mode j with U' = W_j^T Q_j
  const size_t big = chain_max(d, cd, ld);
  double* g0 = ws.take<double>(big);
  double* g1 = ws.take<double>(big);
  KRP_CUDA_CHECK(cudaMemcpyAsync(g0, C, ncore * sizeof(double), cudaMemcpyDeviceToDevice, st));
  int64_t cur[KRP_MAXD];
  for (int j = 0; j < d; ++j) cur[j] = cd[j];
  for (int j = 0; j < d; ++j) {
    double* Uq = ws.take<double>((size_t)cd[j] * ell);
    fs_contract_kernel<<<hd_grid(cd[j] * ell), 256, 0, st>>>(U[j], V[j], factors[j], dims[j], rg[j],
                                                            rh[j], ell, Uq);
    check_launch("hadamard_fs_contract");
    ttm_small_f64(g0, d, cur, j, Uq, ell, g1);
    cur[j] = ell;
    std::swap(g0, g1);
  }
  size_t ncz = 1;
  for (int j = 0; j < d; ++j) ncz *= (size_t)ell;
  KRP_CUDA_CHECK(cudaMemcpyAsync(core, g0, ncz * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (rel_error) {
    // ||Z||^2 = <C, C x_j (W_j^T W_j)>,  ||Z_hat||^2 = ||G_Z||^2
    double* t0 = ws.take<double>(ncore);
    double* t1 = ws.take<double>(ncore);
    KRP_CUDA_CHECK(cudaMemcpyAsync(t0, C, ncore * sizeof(double), cudaMemcpyDeviceToDevice, st));
    for (int j = 0; j < d; ++j) {
      double* W = ws.take<double>((size_t)dims[j] * cd[j]);
      face_split_kernel<<<hd_grid(dims[j] * cd[j]), 256, 0, st>>>(U[j], V[j], dims[j], rg[j], rh[j],
                                                                  W);
      check_launch("hadamard_face_split");
      double* Gr = ws.take<double>((size_t)cd[j] * cd[j]);
      fs_contract_kernel<<<hd_grid(cd[j] * cd[j]), 256, 0, st>>>(U[j], V[j], W, dims[j], rg[j],
                                                                 rh[j], (int)cd[j], Gr);
      check_launch("hadamard_gram");
      int64_t same[KRP_MAXD];
      for (int i = 0; i < d; ++i) same[i] = cd[i];
      ttm_small_f64(t0, d, same, j, Gr, (int)cd[j], t1);
      std::swap(t0, t1);
    }
    double* acc = ws.take<double>(2);
    KRP_CUDA_CHECK(cudaMemsetAsync(acc, 0, 2 * sizeof(double), st));
    dot_kernel<<<hd_grid((int64_t)ncore), 256, 0, st>>>(C, t0, (int64_t)ncore, acc);
    check_launch("hadamard_dot");
    dot_kernel<<<hd_grid((int64_t)ncz), 256, 0, st>>>(g0, g0, (int64_t)ncz, acc + 1);
    check_launch("hadamard_dot");
    double h[2];
    KRP_CUDA_CHECK(cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, st));
    KRP_CUDA_CHECK(cudaStreamSynchronize(st));
    *rel_error = h[0] > 0.0 ? std::sqrt(std::max(0.0, h[0] - h[1]) / h[0]) : 0.0;
  }
}

}  // namespace krp
