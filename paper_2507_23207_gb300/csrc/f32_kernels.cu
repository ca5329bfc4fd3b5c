// FP32 CUDA-core kernels of the plain form.
//
// Every contraction over the big tensor is one of two shapes, because the
// library always works on the fastest (first) mode and rotates the new index
// to the slowest position (Z(m1, rest) -> Z'(rest, l)):
//   gemm_tn_f32:        out[s, k] = sum_i A[i, s] F[i, k]         (TTM, Sec. 2.1)
//   mttkrp_first_f32:   Y[i, k]   = sum_s A[i, s] prod_j V_j[digit_j(s), k]
//                       (mode-1 MTTKRP with the Khatri-Rao row generated on
//                        the fly from the factors, Alg. 7 MTTKRP step)
// plus the "diagonal" contractions that finish a dimension tree (Sec. 5.1,
// memoization) and the streaming FP64-accumulated residual.
#include <algorithm>

#include "common.cuh"

namespace krp {
namespace {

constexpr int TM = 128;  // rows of the output tile (s for gemm_tn, i for mttkrp)
constexpr int TK = 32;   // contraction chunk
constexpr int APITCH = TK + 4;

__device__ __forceinline__ float comp(const float4& v, int c) {
  return c == 0 ? v.x : (c == 1 ? v.y : (c == 2 ? v.z : v.w));
}

// ---- cp.async helpers --------------------------------------------------------
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool pred) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  const int n = pred ? 16 : 0;  // src-size 0 zero-fills the 16 bytes
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(s), "l"(gmem), "r"(n)
               : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem, bool pred) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  const int n = pred ? 4 : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(s), "l"(gmem), "r"(n)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// ----------------------------------------------------------------------------
// out[s + ldo*k] (=|+=) sum_{i<K} A[i + lda*s] * F[i + ldf*k]
// CTA: 128 rows s x NP columns k; thread (g, h) owns rows s0+g+16j (j<8) and
// columns k0+4h..4h+3.  Two-stage cp.async ring: A chunk staged [s][i], F chunk
// staged [k][i] (both i contiguous, rows padded to 36 floats).
constexpr int kGemmStages = 2;

template <int NP, bool VEC>
__global__ void __launch_bounds__(NP * 4, (NP <= 48) ? 3 : 2)
    gemm_tn_kernel(const float* __restrict__ A, int64_t lda, int64_t S, int K,
                   const float* __restrict__ F, int64_t ldf, int L, float* __restrict__ out,
                   int64_t ldo, int accumulate) {
  constexpr int NT = NP * 4;
  extern __shared__ __align__(16) float gsm[];
  float(*As)[TM][APITCH] = reinterpret_cast<float(*)[TM][APITCH]>(gsm);
  float(*Fs)[NP][APITCH] = reinterpret_cast<float(*)[NP][APITCH]>(gsm + kGemmStages * TM * APITCH);

  const int tid = threadIdx.x, g = tid & 15, h = tid >> 4;
  const int64_t s0 = (int64_t)blockIdx.x * TM;
  const int k0 = blockIdx.y * NP;
  float acc[8][4];
#pragma unroll
  for (int j = 0; j < 8; ++j)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[j][c] = 0.f;
  const int nchunks = (K + TK - 1) / TK;

  auto issue = [&](int chunk, int stage) {
    const int kc = chunk * TK;
    if (VEC) {
      for (int q = tid; q < TM * (TK / 4); q += NT) {
        const int sl = q >> 3, c4 = q & 7;
        const int64_t s = s0 + sl;
        const int i = kc + 4 * c4;
        const bool ok = (s < S) && (i < K);
        cp_async16(&As[stage][sl][4 * c4], ok ? (const void*)(A + i + lda * s) : (const void*)A, ok);
      }
      for (int q = tid; q < NP * (TK / 4); q += NT) {
        const int kk = q >> 3, c4 = q & 7;
        const int i = kc + 4 * c4;
        const bool ok = (k0 + kk < L) && (i < K);
        cp_async16(&Fs[stage][kk][4 * c4], ok ? (const void*)(F + i + ldf * (k0 + kk)) : (const void*)F, ok);
      }
    } else {
      for (int q = tid; q < TM * TK; q += NT) {
        const int sl = q >> 5, ii = q & 31;
        const int64_t s = s0 + sl;
        const int i = kc + ii;
        const bool ok = (s < S) && (i < K);
        cp_async4(&As[stage][sl][ii], ok ? (const void*)(A + i + lda * s) : (const void*)A, ok);
      }
      for (int q = tid; q < NP * TK; q += NT) {
        const int kk = q >> 5, ii = q & 31;
        const int i = kc + ii;
        const bool ok = (k0 + kk < L) && (i < K);
        cp_async4(&Fs[stage][kk][ii], ok ? (const void*)(F + i + ldf * (k0 + kk)) : (const void*)F, ok);
      }
    }
    cp_commit();
  };

  issue(0, 0);
  for (int c = 0; c < nchunks; ++c) {
    const int st = c % kGemmStages;
    if (c + 1 < nchunks) {
      issue(c + 1, (c + 1) % kGemmStages);
      cp_wait<1>();
    } else {
      cp_wait<0>();
    }
    __syncthreads();
#pragma unroll
    for (int ii = 0; ii < TK; ii += 4) {
      float4 a[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) a[j] = *reinterpret_cast<const float4*>(&As[st][g + 16 * j][ii]);
      float4 f[4];
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) f[cc] = *reinterpret_cast<const float4*>(&Fs[st][4 * h + cc][ii]);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const float av = comp(a[j], q);
          acc[j][0] = fmaf(av, comp(f[0], q), acc[j][0]);
          acc[j][1] = fmaf(av, comp(f[1], q), acc[j][1]);
          acc[j][2] = fmaf(av, comp(f[2], q), acc[j][2]);
          acc[j][3] = fmaf(av, comp(f[3], q), acc[j][3]);
        }
      }
    }
    __syncthreads();  // stage st is refilled by the next-but-one issue
  }
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int64_t s = s0 + g + 16 * j;
    if (s >= S) continue;
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
      const int k = k0 + 4 * h + cc;
      if (k < L) {
        float* o = out + s + ldo * k;
        *o = accumulate ? *o + acc[j][cc] : acc[j][cc];
      }
    }
  }
}

template <class Kern>
void set_dyn_smem(Kern k, size_t bytes) {
  if (bytes > 48 * 1024)
    KRP_CUDA_CHECK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
}

template <int NP>
void gemm_tn_launch(const float* A, int64_t lda, int64_t S, int K, const float* F, int64_t ldf,
                    int L, float* out, int64_t ldo, bool accumulate) {
  dim3 grid((unsigned)((S + TM - 1) / TM), (unsigned)((L + NP - 1) / NP));
  const bool vec = (lda % 4 == 0) && (ldf % 4 == 0) && (K % 4 == 0) &&
                   ((reinterpret_cast<uintptr_t>(A) & 15) == 0) &&
                   ((reinterpret_cast<uintptr_t>(F) & 15) == 0);
  const size_t smem = sizeof(float) * kGemmStages * (TM + NP) * APITCH;
  if (vec) {
    set_dyn_smem(gemm_tn_kernel<NP, true>, smem);
    gemm_tn_kernel<NP, true><<<grid, NP * 4, smem, stream()>>>(A, lda, S, K, F, ldf, L, out, ldo,
                                                               accumulate ? 1 : 0);
  } else {
    set_dyn_smem(gemm_tn_kernel<NP, false>, smem);
    gemm_tn_kernel<NP, false><<<grid, NP * 4, smem, stream()>>>(A, lda, S, K, F, ldf, L, out, ldo,
                                                                accumulate ? 1 : 0);
  }
  check_launch("gemm_tn_f32");
}

// ----------------------------------------------------------------------------
// Y[i + n1*k] += sum_{s in split} A[i + n1*s] * W(s, k),
// W(s, k) = prod_j V_j[digit_j(s) + radix_j * k]   (the Khatri-Rao row)
// Three-stage cp.async ring for A (staged [s][i]); the Khatri-Rao rows of the
// next chunk are gathered into registers while the current chunk is
// multiplied, and written to shared memory afterwards.
struct RadixDev {
  int n;
  int64_t radix[KRP_MAXD];
  const float* V[KRP_MAXD];
};

constexpr int kMttStages = 3;

// DR: upper bound on the number of Khatri-Rao factors of a row (R.n <= DR),
// so that the gathered factor values take DR registers per row value.
template <int NP, bool VEC, int DR>
__global__ void __launch_bounds__(NP * 4, (NP <= 48) ? 3 : 2)
    mttkrp_first_kernel(const float* __restrict__ A, int64_t n1, int64_t S, const RadixDev R,
                        int L, float* __restrict__ Y, int64_t s_per_split) {
  constexpr int NT = NP * 4;
  constexpr int WV = (TK * NP + NT - 1) / NT;  // = 8
  extern __shared__ __align__(16) float msm[];
  float(*As)[TK][TM] = reinterpret_cast<float(*)[TK][TM]>(msm);
  float(*Ws)[TK][NP] = reinterpret_cast<float(*)[TK][NP]>(msm + kMttStages * TK * TM);
  int(*dig)[TK][KRP_MAXD] =
      reinterpret_cast<int(*)[TK][KRP_MAXD]>(msm + kMttStages * TK * TM + 2 * TK * NP);

  const int tid = threadIdx.x, g = tid & 15, h = tid >> 4;
  const int64_t i0 = (int64_t)blockIdx.x * TM;
  const int k0 = blockIdx.y * NP;
  const int64_t sb = (int64_t)blockIdx.z * s_per_split;
  const int64_t se = min(S, sb + s_per_split);
  if (sb >= se) return;
  float acc[8][4];
#pragma unroll
  for (int j = 0; j < 8; ++j)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[j][c] = 0.f;
  const int64_t nchunks = (se - sb + TK - 1) / TK;

  auto issue = [&](int64_t chunk) {
    if (chunk < nchunks) {
      const int st = (int)(chunk % kMttStages);
      const int64_t sc = sb + chunk * TK;
      if (VEC) {
        for (int q = tid; q < TK * (TM / 4); q += NT) {
          const int sl = q >> 5, c4 = q & 31;
          const int64_t s = sc + sl, i = i0 + 4 * c4;
          const bool ok = (s < se) && (i < n1);
          cp_async16(&As[st][sl][4 * c4], ok ? (const void*)(A + i + n1 * s) : (const void*)A, ok);
        }
      } else {
        for (int q = tid; q < TK * TM; q += NT) {
          const int sl = q >> 7, ii = q & 127;
          const int64_t s = sc + sl, i = i0 + ii;
          const bool ok = (s < se) && (i < n1);
          cp_async4(&As[st][sl][ii], ok ? (const void*)(A + i + n1 * s) : (const void*)A, ok);
        }
      }
    }
    cp_commit();  // always one group per call (possibly empty)
  };
  auto decode = [&](int64_t chunk) {
    if (tid < TK && chunk < nchunks) {
      int64_t s = sb + chunk * TK + tid;
      for (int j = 0; j < R.n; ++j) {
        const int64_t r = R.radix[j];
        dig[chunk & 1][tid][j] = (int)(s % r);
        s /= r;
      }
    }
  };
  // factor values of the Khatri-Rao rows of `chunk`, gathered into registers
  float fv[WV][DR];
  auto gather = [&](int64_t chunk) {
    const int64_t sc = sb + chunk * TK;
#pragma unroll
    for (int v = 0; v < WV; ++v) {
      const int q = tid + v * NT;
      const int sl = q / NP, kk = q % NP;
      const bool ok = (chunk < nchunks) && (q < TK * NP) && (sc + sl < se) && (k0 + kk < L);
#pragma unroll
      for (int j = 0; j < DR; ++j)
        fv[v][j] = (ok && j < R.n) ? R.V[j][dig[chunk & 1][sl][j] + R.radix[j] * (k0 + kk)] : 0.f;
    }
  };
  auto scatter = [&](int64_t chunk) {
#pragma unroll
    for (int v = 0; v < WV; ++v) {
      const int q = tid + v * NT;
      if (q < TK * NP) {
        float w = (R.n > 0) ? fv[v][0] : 1.f;
#pragma unroll
        for (int j = 1; j < DR; ++j)
          if (j < R.n) w *= fv[v][j];
        const int sl = q / NP;
        const bool ok = (chunk < nchunks) && (sb + chunk * TK + sl < se) && (k0 + q % NP < L);
        Ws[chunk & 1][sl][q % NP] = ok ? w : 0.f;
      }
    }
  };

  issue(0);
  issue(1);
  decode(0);
  decode(1);
  __syncthreads();
  gather(0);
  scatter(0);
  for (int64_t c = 0; c < nchunks; ++c) {
    cp_wait<1>();  // chunk c has landed (chunk c+1 may be in flight)
    __syncthreads();
    issue(c + 2);
    gather(c + 1);  // global loads overlap the multiply below
    const int st = (int)(c % kMttStages);
    const int wb = (int)(c & 1);
#pragma unroll 8
    for (int sl = 0; sl < TK; ++sl) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[st][sl][4 * g]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[st][sl][64 + 4 * g]);
      const float4 w = *reinterpret_cast<const float4*>(&Ws[wb][sl][4 * h]);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        acc[j][0] = fmaf(av[j], w.x, acc[j][0]);
        acc[j][1] = fmaf(av[j], w.y, acc[j][1]);
        acc[j][2] = fmaf(av[j], w.z, acc[j][2]);
        acc[j][3] = fmaf(av[j], w.w, acc[j][3]);
      }
    }
    scatter(c + 1);  // Ws[(c+1)&1] was last read in the previous iteration
    __syncthreads();
    decode(c + 2);   // dig[c&1] was last read by gather(c) in the previous iteration
  }
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int64_t i = i0 + (j < 4 ? 4 * g + j : 64 + 4 * g + (j - 4));
    if (i >= n1) continue;
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
      const int k = k0 + 4 * h + cc;
      if (k < L) atomicAdd(Y + i + n1 * k, acc[j][cc]);
    }
  }
}

template <int NP>
void mttkrp_first_launch(const float* A, int64_t n1, int64_t S, const RadixDev& R, int L,
                         float* Y) {
  const int mt = (int)((n1 + TM - 1) / TM);
  const int nt = (L + NP - 1) / NP;
  const int want = 6 * current()->num_sms;  // two waves of three CTAs per SM
  int64_t splits = std::max<int64_t>(1, want / std::max(1, mt * nt));
  int64_t per = (S + splits - 1) / splits;
  per = std::max<int64_t>(per, 4 * TK);
  per = (per + TK - 1) / TK * TK;
  splits = (S + per - 1) / per;
  dim3 grid(mt, nt, (unsigned)splits);
  const bool vec = (n1 % 4 == 0) && ((reinterpret_cast<uintptr_t>(A) & 15) == 0);
  const size_t smem = sizeof(float) * (kMttStages * TK * TM + 2 * TK * NP) + sizeof(int) * 2 * TK * KRP_MAXD;
  auto go = [&](auto kern) {
    set_dyn_smem(kern, smem);
    kern<<<grid, NP * 4, smem, stream()>>>(A, n1, S, R, L, Y, per);
  };
  if (vec) {
    if (R.n <= 1) go(mttkrp_first_kernel<NP, true, 1>);
    else if (R.n == 2) go(mttkrp_first_kernel<NP, true, 2>);
    else if (R.n == 3) go(mttkrp_first_kernel<NP, true, 3>);
    else go(mttkrp_first_kernel<NP, true, KRP_MAXD - 1>);
  } else {
    if (R.n <= 2) go(mttkrp_first_kernel<NP, false, 2>);
    else go(mttkrp_first_kernel<NP, false, KRP_MAXD - 1>);
  }
  check_launch("mttkrp_first_f32");
}

// ----------------------------------------------------------------------------
// Diagonal contractions over an intermediate T (dims m_0..m_{D-1}, then the
// sketch column k slowest with stride tk).
struct DiagDev {
  int D;
  int64_t m[KRP_MAXD];
  const float* V[KRP_MAXD];  // V_j: m_j x L, column-major; V[n] unused
};

// target n = 0: Y[i + m0*k] = sum_s T[i + m0*s + tk*k] * prod_{j>=1} V_j[digit, k]
__global__ void diag_first_kernel(const float* __restrict__ T, const DiagDev P, int64_t tk,
                                  int L, float* __restrict__ Y, int64_t s_per_split) {
  __shared__ float wsh[256];
  const int k = blockIdx.y;
  const int64_t m0 = P.m[0];
  int64_t S = 1;
  for (int j = 1; j < P.D; ++j) S *= P.m[j];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t sb = (int64_t)blockIdx.z * s_per_split;
  const int64_t se = min(S, sb + s_per_split);
  float acc = 0.f;
  const float* Tk = T + tk * k;
  for (int64_t sc = sb; sc < se; sc += 256) {
    __syncthreads();
    for (int q = threadIdx.x; q < 256; q += blockDim.x) {
      int64_t s = sc + q;
      float w = 0.f;
      if (s < se) {
        w = 1.f;
        for (int j = 1; j < P.D; ++j) {
          const int64_t r = P.m[j];
          w *= P.V[j][(s % r) + r * k];
          s /= r;
        }
      }
      wsh[q] = w;
    }
    __syncthreads();
    if (i < m0) {
      const int lim = (int)((se - sc) < 256 ? (se - sc) : 256);
      for (int q = 0; q < lim; ++q) acc = fmaf(Tk[i + m0 * (sc + q)], wsh[q], acc);
    }
  }
  if (i < m0) atomicAdd(Y + i + m0 * k, acc);
}

// target n >= 1: one warp per row (i_n, s): sum over the P contiguous prefix
// entries weighted by prod_{j<n} V_j, times prod_{j>n} V_j of s.
__global__ void diag_mid_kernel(const float* __restrict__ T, const DiagDev P, int64_t tk, int n,
                                int L, float* __restrict__ Y) {
  const int k = blockIdx.y;
  int64_t Pp = 1, Sfx = 1;
  for (int j = 0; j < n; ++j) Pp *= P.m[j];
  for (int j = n + 1; j < P.D; ++j) Sfx *= P.m[j];
  const int64_t mn = P.m[n];
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const float* Tk = T + tk * k;
  for (int64_t row = warp; row < mn * Sfx; row += nwarps) {
    const int64_t in = row % mn, s = row / mn;
    const float* base = Tk + Pp * row;  // = Pp*(in + mn*s)
    float part = 0.f;
    for (int64_t p = lane; p < Pp; p += 32) {
      float w = 1.f;
      int64_t q = p;
      for (int j = 0; j < n; ++j) {
        const int64_t r = P.m[j];
        w *= P.V[j][(q % r) + r * k];
        q /= r;
      }
      part = fmaf(base[p], w, part);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if (lane == 0) {
      float w = 1.f;
      int64_t q = s;
      for (int j = n + 1; j < P.D; ++j) {
        const int64_t r = P.m[j];
        w *= P.V[j][(q % r) + r * k];
        q /= r;
      }
      atomicAdd(Y + in + mn * k, part * w);
    }
  }
}

__global__ void cast_f64_f32_kernel(const double* __restrict__ s, float* __restrict__ d, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    d[i] = static_cast<float>(s[i]);
}
__global__ void cast_f32_f64_kernel(const float* __restrict__ s, double* __restrict__ d, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    d[i] = static_cast<double>(s[i]);
}
// dst (cols x rows, col-major) = src^T (src rows x cols col-major), as FP32
__global__ void transpose_f64_f32_kernel(const double* __restrict__ s, int64_t rows, int64_t cols,
                                         float* __restrict__ d) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < rows * cols;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e % rows, c = e / rows;
    d[c + cols * r] = static_cast<float>(s[e]);
  }
}
// dst[r + rest*i] = src[i + m0*r]
__global__ void rotate_kernel(const float* __restrict__ s, int64_t m0, int64_t rest,
                              float* __restrict__ d) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m0 * rest;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % m0, r = e / m0;
    d[r + rest * i] = s[e];
  }
}

int grid_for(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, 8192));
}

// ----------------------------------------------------------------------------
// Residual: acc[0] += ||X - Q1 H||_F^2, acc[1] += ||X||_F^2 with X n1 x S
// (FP32 or BF16), Q1 n1 x l, H l x S (column-major, FP32).  A 128 x 128 tile
// of X_hat is formed in registers (thread tile 8 x 8), compared with X, and
// squared differences are summed in FP32 per thread and in FP64 across threads.
template <class XT>
__device__ __forceinline__ float ldx(const XT* p);
template <>
__device__ __forceinline__ float ldx<float>(const float* p) { return *p; }
template <>
__device__ __forceinline__ float ldx<__nv_bfloat16>(const __nv_bfloat16* p) {
  return __bfloat162float(*p);
}

// four consecutive elements (16-byte / 8-byte aligned)
template <class XT>
__device__ __forceinline__ void ld4(const XT* p, float* v);
template <>
__device__ __forceinline__ void ld4<float>(const float* p, float* v) {
  const float4 q = *reinterpret_cast<const float4*>(p);
  v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
template <>
__device__ __forceinline__ void ld4<__nv_bfloat16>(const __nv_bfloat16* p, float* v) {
  const uint2 q = *reinterpret_cast<const uint2*>(p);
  v[0] = __uint_as_float(q.x << 16);
  v[1] = __uint_as_float(q.x & 0xFFFF0000u);
  v[2] = __uint_as_float(q.y << 16);
  v[3] = __uint_as_float(q.y & 0xFFFF0000u);
}

template <class XT>
__global__ void __launch_bounds__(256)
    residual_kernel(const XT* __restrict__ X, int64_t n1, int64_t S,
                    const float* __restrict__ Q1, int l, const float* __restrict__ H,
                    double* __restrict__ acc) {
  constexpr int KC = 16;
  __shared__ __align__(16) float Qs[KC][TM];
  __shared__ __align__(16) float Hs[KC][TM + 4];
  __shared__ double red[2][8];
  const int tid = threadIdx.x, gi = tid & 15, gs = tid >> 4;
  const int64_t s0 = (int64_t)blockIdx.x * TM;
  const int64_t i0 = (int64_t)blockIdx.y * TM;
  float xh[8][8];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) xh[a][b] = 0.f;
  for (int kc = 0; kc < l; kc += KC) {
    __syncthreads();
    for (int q = tid; q < KC * TM; q += 256) {
      const int kk = q / TM, r = q % TM;
      const int64_t i = i0 + r, s = s0 + r;
      Qs[kk][r] = (kc + kk < l && i < n1) ? Q1[i + n1 * (kc + kk)] : 0.f;
    }
    for (int q = tid; q < KC * TM; q += 256) {
      const int kk = q % KC, r = q / KC;
      const int64_t s = s0 + r;
      Hs[kk][r] = (kc + kk < l && s < S) ? H[(kc + kk) + (int64_t)l * s] : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < KC; ++kk) {
      const float4 q0 = *reinterpret_cast<const float4*>(&Qs[kk][4 * gi]);
      const float4 q1 = *reinterpret_cast<const float4*>(&Qs[kk][64 + 4 * gi]);
      const float4 h0 = *reinterpret_cast<const float4*>(&Hs[kk][4 * gs]);
      const float4 h1 = *reinterpret_cast<const float4*>(&Hs[kk][64 + 4 * gs]);
      const float qa[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
      const float ha[8] = {h0.x, h0.y, h0.z, h0.w, h1.x, h1.y, h1.z, h1.w};
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) xh[a][b] = fmaf(qa[a], ha[b], xh[a][b]);
    }
  }
  float d2 = 0.f, x2 = 0.f;
  const bool vec = (n1 % 4) == 0;
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    const int64_t s = s0 + (b < 4 ? 4 * gs + b : 64 + 4 * gs + (b - 4));
    if (s >= S) continue;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int64_t ib = i0 + half * 64 + 4 * gi;
      float xv[4];
      if (vec && ib + 3 < n1) {
        ld4<XT>(X + ib + n1 * s, xv);
      } else {
#pragma unroll
        for (int a = 0; a < 4; ++a) xv[a] = (ib + a < n1) ? ldx<XT>(X + ib + a + n1 * s) : 0.f;
      }
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        if (ib + a >= n1) continue;
        const float df = xv[a] - xh[half * 4 + a][b];
        d2 = fmaf(df, df, d2);
        x2 = fmaf(xv[a], xv[a], x2);
      }
    }
  }
  double dd = d2, xx = x2;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    dd += __shfl_xor_sync(0xffffffffu, dd, o);
    xx += __shfl_xor_sync(0xffffffffu, xx, o);
  }
  if ((tid & 31) == 0) {
    red[0][tid >> 5] = dd;
    red[1][tid >> 5] = xx;
  }
  __syncthreads();
  if (tid == 0) {
    double a = 0, b = 0;
    for (int w = 0; w < 8; ++w) {
      a += red[0][w];
      b += red[1][w];
    }
    atomicAdd(acc, a);
    atomicAdd(acc + 1, b);
  }
}

}  // namespace

void gemm_tn_f32(const float* A, int64_t lda, int64_t S, int K, const float* F, int64_t ldf,
                 int L, float* out, int64_t ldo, bool accumulate) {
  if (S <= 0 || L <= 0) return;
  if (K <= 0) {
    if (!accumulate)
      for (int k = 0; k < L; ++k)
        KRP_CUDA_CHECK(cudaMemsetAsync(out + ldo * k, 0, sizeof(float) * S, stream()));
    return;
  }
  if (L <= 16)
    gemm_tn_launch<16>(A, lda, S, K, F, ldf, L, out, ldo, accumulate);
  else if (L <= 32)
    gemm_tn_launch<32>(A, lda, S, K, F, ldf, L, out, ldo, accumulate);
  else if (L <= 48)
    gemm_tn_launch<48>(A, lda, S, K, F, ldf, L, out, ldo, accumulate);
  else
    gemm_tn_launch<64>(A, lda, S, K, F, ldf, L, out, ldo, accumulate);
}

void mttkrp_first_f32(const float* A, int64_t n1, int64_t S, const Radix& rest, int L, float* Y) {
  KRP_CUDA_CHECK(cudaMemsetAsync(Y, 0, sizeof(float) * n1 * L, stream()));
  if (S <= 0) return;
  RadixDev R{};
  R.n = rest.n;
  for (int j = 0; j < rest.n; ++j) {
    R.radix[j] = rest.radix[j];
    R.V[j] = rest.V[j];
  }
  if (L <= 16)
    mttkrp_first_launch<16>(A, n1, S, R, L, Y);
  else if (L <= 32)
    mttkrp_first_launch<32>(A, n1, S, R, L, Y);
  else if (L <= 48)
    mttkrp_first_launch<48>(A, n1, S, R, L, Y);
  else
    mttkrp_first_launch<64>(A, n1, S, R, L, Y);
}

void diag_contract_f32(const float* T, int D, const int64_t* m, int64_t tk, int n,
                       const float* const* V, int L, float* Y) {
  DiagDev P{};
  P.D = D;
  int64_t total = 1;
  for (int j = 0; j < D; ++j) {
    P.m[j] = m[j];
    P.V[j] = V[j];
    total *= m[j];
  }
  KRP_CUDA_CHECK(cudaMemsetAsync(Y, 0, sizeof(float) * m[n] * L, stream()));
  if (total == 0) return;
  if (n == 0) {
    const int64_t S = total / m[0];
    const int threads = 256;
    const int bx = (int)((m[0] + threads - 1) / threads);
    const int want = 4 * current()->num_sms;
    int64_t splits = std::max<int64_t>(1, want / std::max(1, bx * L));
    int64_t per = std::max<int64_t>(256, (S + splits - 1) / splits);
    splits = (S + per - 1) / per;
    dim3 grid(bx, L, (unsigned)splits);
    diag_first_kernel<<<grid, threads, 0, stream()>>>(T, P, tk, L, Y, per);
    check_launch("diag_first_f32");
  } else {
    int64_t nrows = m[n];
    for (int j = n + 1; j < D; ++j) nrows *= m[j];
    const int threads = 256;
    const int64_t blocks = std::min<int64_t>((nrows * 32 + threads - 1) / threads, 2048);
    dim3 grid((unsigned)std::max<int64_t>(1, blocks), L);
    diag_mid_kernel<<<grid, threads, 0, stream()>>>(T, P, tk, n, L, Y);
    check_launch("diag_mid_f32");
  }
}

void cast_f64_to_f32(const double* src, float* dst, int64_t n) {
  if (n <= 0) return;
  cast_f64_f32_kernel<<<grid_for(n, 256), 256, 0, stream()>>>(src, dst, n);
  check_launch("cast_f64_f32");
}
void cast_f32_to_f64(const float* src, double* dst, int64_t n) {
  if (n <= 0) return;
  cast_f32_f64_kernel<<<grid_for(n, 256), 256, 0, stream()>>>(src, dst, n);
  check_launch("cast_f32_f64");
}
void transpose_f64_to_f32(const double* src, int64_t rows, int64_t cols, float* dst) {
  if (rows * cols <= 0) return;
  transpose_f64_f32_kernel<<<grid_for(rows * cols, 256), 256, 0, stream()>>>(src, rows, cols, dst);
  check_launch("transpose_f64_f32");
}
void rotate_first_to_last_f32(const float* src, int64_t m0, int64_t rest, float* dst) {
  if (m0 * rest <= 0) return;
  rotate_kernel<<<grid_for(m0 * rest, 256), 256, 0, stream()>>>(src, m0, rest, dst);
  check_launch("rotate_f32");
}

void residual_f32(const void* X, krp_dtype xt, int64_t n1, int64_t S, const float* Q1, int l,
                  const float* H, double* acc) {
  if (n1 <= 0 || S <= 0) return;
  dim3 grid((unsigned)((S + TM - 1) / TM), (unsigned)((n1 + TM - 1) / TM));
  if (xt == KRP_F32)
    residual_kernel<float><<<grid, 256, 0, stream()>>>(static_cast<const float*>(X), n1, S, Q1,
                                                       l, H, acc);
  else
    residual_kernel<__nv_bfloat16><<<grid, 256, 0, stream()>>>(
        static_cast<const __nv_bfloat16*>(X), n1, S, Q1, l, H, acc);
  check_launch("residual");
}

}  // namespace krp
