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
#include <type_traits>

#include "common.cuh"
#include "pipeline.h"

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

// target n >= 1: one warp per row (i_n, s): sum over the Pp contiguous prefix
// entries weighted by wpre[p + Pp k] = prod_{j<n} V_j[digit_j(p), k] (a table
// formed once, so the inner loop is two coalesced loads and an FMA), times
// prod_{j>n} V_j of s.  VEC: 16-byte loads (Pp, tk multiples of 4, T aligned).
template <bool VEC>
__global__ void diag_mid_kernel(const float* __restrict__ T, const DiagDev P, int64_t tk, int n,
                                int L, const float* __restrict__ wpre, float* __restrict__ Y) {
  const int k = blockIdx.y;
  int64_t Pp = 1, Sfx = 1;
  for (int j = 0; j < n; ++j) Pp *= P.m[j];
  for (int j = n + 1; j < P.D; ++j) Sfx *= P.m[j];
  const int64_t mn = P.m[n];
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const float* Tk = T + tk * k;
  const float* wk = wpre + Pp * k;
  for (int64_t row = warp; row < mn * Sfx; row += nwarps) {
    const int64_t in = row % mn, s = row / mn;
    const float* base = Tk + Pp * row;  // = Pp*(in + mn*s)
    float part = 0.f;
    if (VEC) {
      const float4* b4 = reinterpret_cast<const float4*>(base);
      const float4* w4 = reinterpret_cast<const float4*>(wk);
      for (int64_t p = lane; p < (Pp >> 2); p += 32) {
        const float4 x = b4[p], w = __ldg(w4 + p);
        part = fmaf(x.x, w.x, part);
        part = fmaf(x.y, w.y, part);
        part = fmaf(x.z, w.z, part);
        part = fmaf(x.w, w.w, part);
      }
    } else {
      for (int64_t p = lane; p < Pp; p += 32) part = fmaf(base[p], __ldg(wk + p), part);
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

// PRE: the CTA's 128 x 128 tile of X is copied into shared memory with
// cp.async as the CTA starts, so that its HBM latency overlaps the
// reconstruction product (needs n1 to be a multiple of 16 bytes' worth of
// elements and a 16-byte aligned X).
template <class XT, bool PRE>
__global__ void __launch_bounds__(256)
    residual_kernel(const XT* __restrict__ X, int64_t n1, int64_t S,
                    const float* __restrict__ Q1, int l, const float* __restrict__ H,
                    double* __restrict__ acc) {
  constexpr int KC = 16;
  __shared__ __align__(16) float Qs[KC][TM];
  __shared__ __align__(16) float Hs[KC][TM + 4];
  __shared__ double red[2][8];
  extern __shared__ __align__(16) unsigned char rxs[];
  XT(*Xs)[TM] = reinterpret_cast<XT(*)[TM]>(rxs);  // [s][i]
  const int tid = threadIdx.x, gi = tid & 15, gs = tid >> 4;
  const int64_t s0 = (int64_t)blockIdx.x * TM;
  const int64_t i0 = (int64_t)blockIdx.y * TM;
  if (PRE) {
    constexpr int E = 16 / sizeof(XT);  // elements per 16-byte copy
    constexpr int CPR = TM / E;         // copies per s row of the tile
    for (int q = tid; q < TM * CPR; q += 256) {
      const int sl = q / CPR, c = q % CPR;
      const int64_t s = s0 + sl, i = i0 + c * E;
      const bool ok = (s < S) && (i < n1);  // n1 % E == 0: a copy is all in or all out
      cp_async16(&Xs[sl][c * E], ok ? (const void*)(X + i + n1 * s) : (const void*)X, ok);
    }
    cp_commit();
  }
  float xh[8][8];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) xh[a][b] = 0.f;
  for (int kc = 0; kc < l; kc += KC) {
    __syncthreads();
    for (int q = tid; q < KC * TM; q += 256) {
      const int kk = q / TM, r = q % TM;
      const int64_t i = i0 + r;
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
  if (PRE) {
    cp_wait<0>();
    __syncthreads();
  }
  float d2 = 0.f, x2 = 0.f;
  const bool vec = (n1 % 4) == 0;
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    const int sl = b < 4 ? 4 * gs + b : 64 + 4 * gs + (b - 4);
    const int64_t s = s0 + sl;
    if (s >= S) continue;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int64_t ib = i0 + half * 64 + 4 * gi;
      float xv[4];
      if (PRE) {
        ld4<XT>(&Xs[sl][half * 64 + 4 * gi], xv);
      } else if (vec && ib + 3 < n1) {
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


// Persistent form of the residual for FP32 X with c % 4 == 0: a CTA keeps its
// 128-row block of Q1 (c x 128, staged [k][i]) in shared memory and walks the
// 64-column tiles s0 = 64 (blockIdx.x + j gridDim.x), with the H tile (64 x c,
// one contiguous run of H) and the X tile (64 x 128, staged [s][i]) of the
// next tile in flight by cp.async while the current one is reconstructed.
// Thread (gi = tid & 15, gs = tid >> 4) owns rows 4 gi + {0..3}, 64 + 4 gi +
// {0..3} and columns 4 gs + {0..3}; each group of four contraction indices
// costs two 16-byte Q loads per index and one 16-byte H load per column for
// 128 FMAs.  Per-tile FP32 partial sums are added into FP64 per thread.
constexpr int kRtS = 64;  // s columns per tile
constexpr int kRtStages = 2;
size_t residual_tiled_smem(int c) {
  return sizeof(float) * ((size_t)c * TM + (size_t)kRtStages * kRtS * (c + TM));
}
__global__ void __launch_bounds__(256, 2)
    residual_tiled_kernel(const float* __restrict__ X, int64_t n1, int64_t S,
                          const float* __restrict__ Q1, int c, const float* __restrict__ H,
                          double* __restrict__ acc) {
  extern __shared__ __align__(16) float rsm[];
  float* Qs = rsm;                              // [c][TM]
  float* Hs = Qs + c * TM;                      // stages x [kRtS][c]
  float* Xs = Hs + kRtStages * kRtS * c;        // stages x [kRtS][TM]
  __shared__ double red[2][8];
  const int tid = threadIdx.x, gi = tid & 15, gs = tid >> 4;
  const int64_t i0 = (int64_t)blockIdx.y * TM;
  const int64_t ntile = (S + kRtS - 1) / kRtS;
  const bool rows_full = i0 + TM <= n1;
  for (int q = tid; q < c * (TM / 4); q += 256) {
    const int k = q / (TM / 4), c4 = q % (TM / 4);
    const int64_t i = i0 + 4 * c4;
    const bool ok = i < n1;
    cp_async16(Qs + k * TM + 4 * c4, ok ? (const void*)(Q1 + i + n1 * k) : (const void*)Q1, ok);
  }
  cp_commit();
  auto issue = [&](int64_t t, int st) {
    if (t < ntile) {
      const int64_t s0 = t * kRtS;
      const bool full = s0 + kRtS <= S;
      float* hs = Hs + st * kRtS * c;
      float* xs = Xs + st * kRtS * TM;
      for (int e = 4 * tid; e < kRtS * c; e += 4 * 256) {  // a copy stays within one s (c % 4 == 0)
        const bool ok = full || s0 + e / c < S;
        cp_async16(hs + e, ok ? (const void*)(H + c * s0 + e) : (const void*)H, ok);
      }
      // X tile: thread tid copies the 4 rows at 4 (tid % 32) of columns
      // tid / 32 + 8 v (no index division per copy)
      const int c4 = tid & 31;
      const bool row_ok = rows_full || i0 + 4 * c4 < n1;
      const float* xp = X + i0 + 4 * c4 + n1 * (s0 + (tid >> 5));
#pragma unroll
      for (int v = 0; v < kRtS / 8; ++v) {
        const int sl = (tid >> 5) + 8 * v;
        const bool ok = row_ok && (full || s0 + sl < S);
        cp_async16(xs + sl * TM + 4 * c4, ok ? (const void*)(xp + n1 * 8 * v) : (const void*)X, ok);
      }
    }
    cp_commit();  // possibly empty: keeps one group per tile slot
  };
  const int64_t t0 = blockIdx.x, dt = gridDim.x;
#pragma unroll 1
  for (int st = 0; st < kRtStages - 1; ++st) issue(t0 + st * dt, st);
  double dd = 0.0, xx = 0.0;
  int st = 0;
#pragma unroll 1
  for (int64_t t = t0; t < ntile; t += dt) {
    __syncthreads();  // the stage refilled below was consumed one tile ago
    issue(t + (kRtStages - 1) * dt, (st + kRtStages - 1) % kRtStages);
    cp_wait<kRtStages - 1>();
    __syncthreads();
    const float* hs = Hs + st * kRtS * c;
    const float* xs = Xs + st * kRtS * TM;
    float xh[8][4];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) xh[a][b] = 0.f;
#pragma unroll 1
    for (int k = 0; k < c; k += 4) {
      float4 hv[4];
#pragma unroll
      for (int b = 0; b < 4; ++b) hv[b] = *reinterpret_cast<const float4*>(hs + (4 * gs + b) * c + k);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const float4 q0 = *reinterpret_cast<const float4*>(Qs + (k + kk) * TM + 4 * gi);
        const float4 q1 = *reinterpret_cast<const float4*>(Qs + (k + kk) * TM + 64 + 4 * gi);
        const float qa[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const float hb = comp(hv[b], kk);
#pragma unroll
          for (int a = 0; a < 8; ++a) xh[a][b] = fmaf(qa[a], hb, xh[a][b]);
        }
      }
    }
    const int64_t s0 = t * kRtS;
    float d2 = 0.f, x2 = 0.f;
    if (rows_full && s0 + kRtS <= S) {  // a full tile: no bounds checks
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int sl = 4 * gs + b;
#pragma unroll
        for (int half = 0; half < 2; ++half) {
          const float4 xq = *reinterpret_cast<const float4*>(xs + sl * TM + half * 64 + 4 * gi);
          const float xv[4] = {xq.x, xq.y, xq.z, xq.w};
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            const float df = xv[a] - xh[half * 4 + a][b];
            d2 = fmaf(df, df, d2);
            x2 = fmaf(xv[a], xv[a], x2);
          }
        }
      }
    } else {
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int sl = 4 * gs + b;
        if (s0 + sl >= S) continue;
#pragma unroll
        for (int half = 0; half < 2; ++half) {
          const int64_t ib = i0 + half * 64 + 4 * gi;
          const float4 xq = *reinterpret_cast<const float4*>(xs + sl * TM + half * 64 + 4 * gi);
          const float xv[4] = {xq.x, xq.y, xq.z, xq.w};
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            if (ib + a >= n1) continue;
            const float df = xv[a] - xh[half * 4 + a][b];
            d2 = fmaf(df, df, d2);
            x2 = fmaf(xv[a], xv[a], x2);
          }
        }
      }
    }
    dd += d2;
    xx += x2;
    st = (st + 1) % kRtStages;
  }
  cp_wait<0>();
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

// ----------------------------------------------------------------------------
// Tiled TTM with 128-row tiles (the main FP32 contraction):
//   out[s + ldo*k] (=|+=) sum_i A[i + lda*s] F[i + ldf*k]
// Thread (g = tid >> 3, h = tid & 7) owns rows g + (BMS/8) j (j < 8) and the
// strided columns h + 8 c (c < NP/8), so that both operand reads below are
// conflict-free 16-byte shared-memory loads.  Chunks of GK contraction indices
// (16 or 32) are staged [s][i] and [k][i] (pitch GK + 4 floats: consecutive
// rows start 16 bytes apart in the banks) by an NS-stage cp.async ring with
// one block barrier per chunk.  Each copy slot of a thread is fixed, so its
// global address is computed once and advanced by GK per chunk.
// PAIR: each accumulator is a pair of partial sums over the even and the odd
// contraction indices, updated by the paired FP32 FMA (fma.rn.f32x2): both
// operands come as natural register pairs of the 16-byte loads, and one
// instruction does two FMAs, leaving issue slots for the loads and barriers
// (the pair is summed once at the end).
template <int NP, int BMS, int NS, int MINB, bool PAIR, int GK>
__global__ void __launch_bounds__(BMS, MINB)
    gemm_tn_tile_kernel(const float* __restrict__ A, int64_t lda, int64_t S, int K,
                        const float* __restrict__ F, int64_t ldf, int L, float* __restrict__ out,
                        int64_t ldo, int accumulate) {
  constexpr int NT = BMS, RG = BMS / 8, CPT = NP / 8, GP = GK + 4, CPR = GK / 4;
  static_assert(GK == 16 || GK == 32, "chunk width");
  extern __shared__ __align__(16) float gts[];
  float(*As)[BMS][GP] = reinterpret_cast<float(*)[BMS][GP]>(gts);
  float(*Fs)[NP][GP] = reinterpret_cast<float(*)[NP][GP]>(gts + NS * BMS * GP);
  const int tid = threadIdx.x, g = tid >> 3, h = tid & 7;
  const int64_t s0 = (int64_t)blockIdx.x * BMS;
  const int k0 = blockIdx.y * NP;
  using Acc = typename std::conditional<PAIR, float2, float>::type;
  Acc acc[8][CPT];
#pragma unroll
  for (int j = 0; j < 8; ++j)
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
      if constexpr (PAIR)
        acc[j][c] = make_float2(0.f, 0.f);
      else
        acc[j][c] = 0.f;
    }
  const int nchunks = (K + GK - 1) / GK;
  constexpr int AV = BMS * CPR / NT;
  constexpr int FV = (NP * CPR + NT - 1) / NT;
  const float* pa[AV];
  bool oka[AV];
#pragma unroll
  for (int v = 0; v < AV; ++v) {
    const int q = tid + NT * v;
    const int64_t s = s0 + (q / CPR);
    oka[v] = s < S;
    pa[v] = A + 4 * (q % CPR) + lda * (oka[v] ? s : 0);
  }
  const float* pf[FV];
  bool okf[FV];
#pragma unroll
  for (int v = 0; v < FV; ++v) {
    const int q = tid + NT * v;
    okf[v] = (q < NP * CPR) && (k0 + (q / CPR) < L);
    pf[v] = F + 4 * (q % CPR) + ldf * (okf[v] ? (k0 + (q / CPR)) : 0);
  }
  auto issue = [&](int chunk) {
    if (chunk < nchunks) {
      const int stage = chunk % NS;
      const int kc = chunk * GK;
#pragma unroll
      for (int v = 0; v < AV; ++v) {
        const int q = tid + NT * v;
        const bool ok = oka[v] && (kc + 4 * (q % CPR) < K);
        cp_async16(&As[stage][q / CPR][4 * (q % CPR)], ok ? (const void*)(pa[v] + kc) : (const void*)A, ok);
      }
#pragma unroll
      for (int v = 0; v < FV; ++v) {
        const int q = tid + NT * v;
        if (q < NP * CPR) {
          const bool ok = okf[v] && (kc + 4 * (q % CPR) < K);
          cp_async16(&Fs[stage][q / CPR][4 * (q % CPR)], ok ? (const void*)(pf[v] + kc) : (const void*)F, ok);
        }
      }
    }
    cp_commit();  // one group per call, possibly empty
  };
#pragma unroll
  for (int p = 0; p < NS - 1; ++p) issue(p);
  for (int c = 0; c < nchunks; ++c) {
    cp_wait<NS - 2>();  // chunk c has landed
    __syncthreads();    // ... for every thread; stage (c-1) % NS is free again
    issue(c + NS - 1);
    const int st = c % NS;
#pragma unroll
    for (int ii = 0; ii < GK; ii += 4) {
      float4 f[CPT];
#pragma unroll
      for (int cc = 0; cc < CPT; ++cc) f[cc] = *reinterpret_cast<const float4*>(&Fs[st][h + 8 * cc][ii]);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const float4 a = *reinterpret_cast<const float4*>(&As[st][g + RG * j][ii]);
#pragma unroll
        for (int cc = 0; cc < CPT; ++cc) {
          if constexpr (PAIR) {
            acc[j][cc] = __ffma2_rn(make_float2(a.x, a.y), make_float2(f[cc].x, f[cc].y), acc[j][cc]);
            acc[j][cc] = __ffma2_rn(make_float2(a.z, a.w), make_float2(f[cc].z, f[cc].w), acc[j][cc]);
          } else {
            float v = acc[j][cc];
            v = fmaf(a.x, f[cc].x, v);
            v = fmaf(a.y, f[cc].y, v);
            v = fmaf(a.z, f[cc].z, v);
            v = fmaf(a.w, f[cc].w, v);
            acc[j][cc] = v;
          }
        }
      }
    }
  }
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int64_t s = s0 + g + RG * j;
    if (s >= S) continue;
#pragma unroll
    for (int cc = 0; cc < CPT; ++cc) {
      const int k = k0 + h + 8 * cc;
      if (k < L) {
        float* o = out + s + ldo * k;
        float v;
        if constexpr (PAIR)
          v = acc[j][cc].x + acc[j][cc].y;
        else
          v = acc[j][cc];
        *o = accumulate ? *o + v : v;
      }
    }
  }
}

// ----------------------------------------------------------------------------
// Two-stage partial-Khatri-Rao MTTKRP of the first mode (Alg. 7 MTTKRP step
// without forming the KRP):
//   Y[i + n1*k] += sum_t wT[t*NP + k] sum_{i2 < n2} X[i + n1*(i2 + n2*t)] O2T[i2*NP + k]
// Stage one is a GEMM of each slab X(:, :, t) (n1 x n2) with the mode-2
// factor; stage two weights it by the Khatri-Rao row w_t of modes 3..d and
// sums over t.  The weight is folded into the B operand as it is staged
// (B_t = O2 diag(w_t), 4 columns per thread with 16-byte loads), so the
// accumulators hold Y directly.  CTA: BM rows i x NP columns, BM threads;
// thread (g = tid >> 3, h = tid & 7) owns rows 4g..4g+3, BM/2+4g..BM/2+4g+3 and
// columns h*CPT..h*CPT+CPT-1.  A moves through an NS-stage cp.async ring, B is
// loaded one chunk ahead into registers and stored after the multiply; one
// block barrier per chunk.  Chunks are numbered c = t * cps + b (the b-th block
// of BK rows of slab t); CTA (x, z) takes rows x and chunks [z per, (z+1) per).
constexpr int MBM = 256, MBK = 16, MNS = 4;
template <int NP, int BK = MBK, int NS = MNS>
__global__ void __launch_bounds__(MBM, 2)
    krp_slab_mttkrp_kernel(const float* __restrict__ X, int64_t n1, int64_t n2, int64_t T,
                           const float* __restrict__ O2T, const float* __restrict__ wT,
                           float* __restrict__ Y, int L, int64_t per) {
  constexpr int BM = MBM, NT = MBM, CPT = NP / 8;
  static_assert(CPT % 2 == 0, "columns per thread must be even");
  extern __shared__ __align__(16) float kss[];
  float(*As)[BK][BM] = reinterpret_cast<float(*)[BK][BM]>(kss);
  float(*Bs)[BK][NP] = reinterpret_cast<float(*)[BK][NP]>(kss + NS * BK * BM);
  const int tid = threadIdx.x, g = tid >> 3, h = tid & 7;
  const int64_t i0 = (int64_t)blockIdx.x * BM;
  const int64_t cps = (n2 + BK - 1) / BK;
  const int64_t total = T * cps;
  const int64_t cb = (int64_t)blockIdx.y * per;
  const int64_t ce = min(total, cb + per);
  if (cb >= ce) return;
  float acc[8][CPT];
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < CPT; ++c) acc[r][c] = 0.f;
  // slab / row-block positions of the next A chunk to issue and of the next
  // B chunk to load, advanced one chunk at a time
  int64_t tA = cb / cps, rA = (cb % cps) * BK, tB = tA, rB = rA;
  auto advance = [&](int64_t& t, int64_t& r) {
    r += BK;
    if (r >= n2) {
      r = 0;
      ++t;
    }
  };
  constexpr int RPV = NT / (BM / 4);  // chunk rows covered per copy round
  const int arow = tid / (BM / 4), ac4 = tid % (BM / 4);
  const bool a_in = (i0 + 4 * ac4) < n1;
  auto issueA = [&](int64_t c) {
    if (c < ce) {
      const int st = (int)((c - cb) % NS);
      const float* src = X + i0 + 4 * ac4 + n1 * (rA + arow + n2 * tA);
#pragma unroll
      for (int v = 0; v < BK / RPV; ++v) {
        const int r = arow + RPV * v;
        const bool ok = a_in && (rA + r < n2);
        cp_async16(&As[st][r][4 * ac4], ok ? (const void*)(src + n1 * RPV * v) : (const void*)X, ok);
      }
      advance(tA, rA);
    }
    cp_commit();
  };
  constexpr int QPR = NP / 4;
  constexpr int NQ = (BK * QPR + NT - 1) / NT;  // quads of B per thread (1 or 2)
  static_assert(NQ <= 2, "at most two quads of B per thread");
  int brow[NQ], bq[NQ];
  bool b_act[NQ];
#pragma unroll
  for (int u = 0; u < NQ; ++u) {
    const int idx = tid + NT * u;
    brow[u] = idx / QPR;
    bq[u] = idx % QPR;
    b_act[u] = idx < BK * QPR;
  }
  float4 bv[NQ];
  auto loadB = [&](int64_t c) {
#pragma unroll
    for (int u = 0; u < NQ; ++u) {
      bv[u] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (b_act[u] && c < ce && rB + brow[u] < n2) {
        const float4 o = __ldg(reinterpret_cast<const float4*>(O2T + (rB + brow[u]) * NP) + bq[u]);
        const float4 w = __ldg(reinterpret_cast<const float4*>(wT + tB * NP) + bq[u]);
        bv[u] = make_float4(o.x * w.x, o.y * w.y, o.z * w.z, o.w * w.w);
      }
    }
    if (c < ce) advance(tB, rB);
  };
  auto storeB = [&](int64_t c) {
#pragma unroll
    for (int u = 0; u < NQ; ++u)
      if (b_act[u]) *reinterpret_cast<float4*>(&Bs[(int)((c - cb) & 1)][brow[u]][4 * bq[u]]) = bv[u];
  };
#pragma unroll
  for (int p = 0; p < NS - 1; ++p) issueA(cb + p);
  loadB(cb);
  storeB(cb);
  for (int64_t c = cb; c < ce; ++c) {
    cp_wait<NS - 2>();  // chunk c of A has landed
    __syncthreads();    // ... for all threads; B[c] stored; stage (c-1) % NS free
    issueA(c + NS - 1);
    loadB(c + 1);       // global loads overlap the multiply below
    const int st = (int)((c - cb) % NS), buf = (int)((c - cb) & 1);
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[st][k][4 * g]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[st][k][BM / 2 + 4 * g]);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      float bb[CPT];
#pragma unroll
      for (int m = 0; m < CPT / 2; ++m) {
        const float2 b = *reinterpret_cast<const float2*>(&Bs[buf][k][h * CPT + 2 * m]);
        bb[2 * m] = b.x;
        bb[2 * m + 1] = b.y;
      }
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c2 = 0; c2 < CPT; ++c2) acc[r][c2] = fmaf(av[r], bb[c2], acc[r][c2]);
    }
    storeB(c + 1);  // buffer (c+1) & 1 was last read in iteration c-1
  }
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int64_t ib = i0 + (r < 4 ? 4 * g + r : BM / 2 + 4 * g + (r - 4));
#pragma unroll
    for (int c2 = 0; c2 < CPT; ++c2) {
      const int k = h * CPT + c2;
      if (k < L && ib < n1) atomicAdd(Y + ib + n1 * k, acc[r][c2]);
    }
  }
}

// OT[i*NP + k] = O[i + n*k] for k < L, 0 for L <= k < NP
__global__ void pad_transpose_kernel(const float* __restrict__ O, int64_t n, int L, int NP,
                                     float* __restrict__ OT) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * NP;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / NP;
    const int k = (int)(e % NP);
    OT[e] = k < L ? O[i + n * k] : 0.f;
  }
}

// wT[t*NP + k] = prod_j V_j[digit_j(t) + radix_j*k] (k < L; 0 for L <= k < NP),
// digits of t in mixed radix with the first listed mode fastest; 1 if no modes
__global__ void krp_weights_padded_kernel(const RadixDev R, int64_t T, int L, int NP,
                                          float* __restrict__ wT) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < T * NP;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = e / NP;
    const int k = (int)(e % NP);
    float w = 0.f;
    if (k < L) {
      w = 1.f;
      int64_t s = t;
      for (int j = 0; j < R.n; ++j) {
        const int64_t r = R.radix[j];
        w *= R.V[j][s % r + r * k];
        s /= r;
      }
    }
    wT[e] = w;
  }
}

}  // namespace

namespace {
template <int NP, int MINB, int NS, bool PAIR, int GK>
void gemm_tn_tile_launch(const float* A, int64_t lda, int64_t S, int K, const float* F, int64_t ldf,
                         int L, float* out, int64_t ldo, bool accumulate) {
  constexpr int BMS = 128;
  dim3 grid((unsigned)((S + BMS - 1) / BMS), (unsigned)((L + NP - 1) / NP));
  const size_t smem = sizeof(float) * NS * (BMS + NP) * (GK + 4);
  set_dyn_smem(gemm_tn_tile_kernel<NP, BMS, NS, MINB, PAIR, GK>, smem);
  gemm_tn_tile_kernel<NP, BMS, NS, MINB, PAIR, GK><<<grid, BMS, smem, stream()>>>(
      A, lda, S, K, F, ldf, L, out, ldo, accumulate ? 1 : 0);
  check_launch(NP == 16 ? "gemm_tn_tile<16>" : NP == 32 ? "gemm_tn_tile<32>"
               : NP == 48 ? "gemm_tn_tile<48>" : "gemm_tn_tile<64>");
}

template <int NP, int BK = MBK, int NS = MNS>
void krp_slab_mttkrp_launch(const float* X, int64_t n1, int64_t n2, int64_t T, const float* O2,
                            const RadixDev& W, int L, float* Y) {
  float* O2T = current()->ws.take<float>((size_t)n2 * NP);
  float* wT = current()->ws.take<float>((size_t)T * NP);
  pad_transpose_kernel<<<grid_for(n2 * NP, 256), 256, 0, stream()>>>(O2, n2, L, NP, O2T);
  check_launch("pad_transpose");
  krp_weights_padded_kernel<<<grid_for(T * NP, 256), 256, 0, stream()>>>(W, T, L, NP, wT);
  check_launch("krp_weights_padded");
  const int mt = (int)((n1 + MBM - 1) / MBM);
  const int64_t cps = (n2 + BK - 1) / BK;
  const int64_t total = T * cps;
  const int64_t want = std::max<int64_t>(1, (int64_t)2 * current()->num_sms / mt);
  const int64_t per = (total + want - 1) / want;
  const int64_t splits = (total + per - 1) / per;
  const size_t smem = sizeof(float) * (NS * BK * MBM + 2 * BK * NP);
  set_dyn_smem(krp_slab_mttkrp_kernel<NP, BK, NS>, smem);
  krp_slab_mttkrp_kernel<NP, BK, NS><<<dim3(mt, (unsigned)splits), MBM, smem, stream()>>>(
      X, n1, n2, T, O2T, wT, Y, L, per);
  check_launch("krp_slab_mttkrp_f32");
}
}  // namespace

size_t mttkrp_first_f32_workspace_bytes(int64_t S, int64_t n2max) {
  // padded mode-2 factor (n2 x 64, or the TF32 hi/lo buffer of up to 128 rows
  // of n2 rounded up to 32) and Khatri-Rao weights (S / n2 x 64, n2 >= 16)
  return std::max(ws_bytes((size_t)n2max * 64, 4), tc_mttkrp_tf32_workspace_bytes(n2max, 64)) +
         ws_bytes((size_t)(S / 16 + 1) * 64, 4);
}

void gemm_tn_f32(const float* A, int64_t lda, int64_t S, int K, const float* F, int64_t ldf,
                 int L, float* out, int64_t ldo, bool accumulate) {
  if (S <= 0 || L <= 0) return;
  if (K <= 0) {
    if (!accumulate)
      for (int k = 0; k < L; ++k)
        KRP_CUDA_CHECK(cudaMemsetAsync(out + ldo * k, 0, sizeof(float) * S, stream()));
    return;
  }
  const bool vec = (lda % 4 == 0) && (ldf % 4 == 0) && (K % 4 == 0) &&
                   ((reinterpret_cast<uintptr_t>(A) & 15) == 0) &&
                   ((reinterpret_cast<uintptr_t>(F) & 15) == 0);
  if (vec) {
    // paired FMAs over 32-wide chunks in three stages up to 48 columns (1024^3
    // launch: 47.4 TFLOP/s single FMAs, 49.6 paired, 51.7 paired with 32-wide
    // chunks); 64 columns keep single FMAs (the pairs would not fit the
    // registers)
    if (L <= 16)
      gemm_tn_tile_launch<16, 2, 3, true, 32>(A, lda, S, K, F, ldf, L, out, ldo, accumulate);
    else if (L <= 32)
      gemm_tn_tile_launch<32, 2, 3, true, 32>(A, lda, S, K, F, ldf, L, out, ldo, accumulate);
    else if (L <= 48)
      gemm_tn_tile_launch<48, 2, 3, true, 32>(A, lda, S, K, F, ldf, L, out, ldo, accumulate);
    else
      gemm_tn_tile_launch<64, 2, 4, false, 16>(A, lda, S, K, F, ldf, L, out, ldo, accumulate);
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
  // two-stage slab kernel: needs 16-byte rows of X, slabs of >= 16 rows and
  // at most 64 sketch columns (one column tile)
  if (L <= 64 && rest.n >= 1 && rest.radix[0] >= MBK && n1 % 4 == 0 &&
      (reinterpret_cast<uintptr_t>(A) & 15) == 0) {
    const int64_t n2 = rest.radix[0];
    RadixDev W{};
    W.n = rest.n - 1;
    for (int j = 1; j < rest.n; ++j) {
      W.radix[j - 1] = rest.radix[j];
      W.V[j - 1] = rest.V[j];
    }
    const int64_t T = S / n2;
    if (tc_mttkrp_tf32_supported(n1, n2, T, L, A)) {
      // tensor cores, three TF32 products per multiply (FP32-level error)
      const int Lp = (L + 15) / 16 * 16;
      float* wT = current()->ws.take<float>((size_t)T * Lp);
      krp_weights_padded_kernel<<<grid_for(T * Lp, 256), 256, 0, stream()>>>(W, T, L, Lp, wT);
      check_launch("krp_weights_padded");
      tc_mttkrp_first_tf32(A, n1, n2, T, rest.V[0], wT, L, Y);
      return;
    }
    if (L <= 16)
      krp_slab_mttkrp_launch<16>(A, n1, n2, T, rest.V[0], W, L, Y);
    else if (L <= 32)
      krp_slab_mttkrp_launch<32>(A, n1, n2, T, rest.V[0], W, L, Y);
    else if (L <= 48)
      krp_slab_mttkrp_launch<48>(A, n1, n2, T, rest.V[0], W, L, Y);
    else
      krp_slab_mttkrp_launch<64>(A, n1, n2, T, rest.V[0], W, L, Y);
    return;
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

// w[t + T*k] = prod_j V_j[digit_j(t) + r_j*k] (pipeline_tucker.cu)
void krp_rows(const Radix& R, int64_t T, int L, bool bf16, float* w);

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
    // prefix weights of modes 0..n-1, one table for all rows
    int64_t Pp = 1;
    Radix R;
    R.n = n;
    for (int j = 0; j < n; ++j) {
      Pp *= m[j];
      R.radix[j] = m[j];
      R.V[j] = V[j];
    }
    float* wpre = current()->ws.take<float>((size_t)Pp * L);
    krp_rows(R, Pp, L, false, wpre);
    const int threads = 256;
    const int64_t blocks = std::min<int64_t>((nrows * 32 + threads - 1) / threads, 2048);
    dim3 grid((unsigned)std::max<int64_t>(1, blocks), L);
    const bool vec = (Pp % 4 == 0) && (tk % 4 == 0) && ((reinterpret_cast<uintptr_t>(T) & 15) == 0) &&
                     ((reinterpret_cast<uintptr_t>(wpre) & 15) == 0);
    if (vec)
      diag_mid_kernel<true><<<grid, threads, 0, stream()>>>(T, P, tk, n, L, wpre, Y);
    else
      diag_mid_kernel<false><<<grid, threads, 0, stream()>>>(T, P, tk, n, L, wpre, Y);
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
  const bool aligned = (reinterpret_cast<uintptr_t>(X) & 15) == 0;
  if (xt == KRP_F32) {
    const float* Xf = static_cast<const float*>(X);
    const bool qh_aligned = ((reinterpret_cast<uintptr_t>(Q1) | reinterpret_cast<uintptr_t>(H)) & 15) == 0;
    if (aligned && qh_aligned && n1 % 4 == 0 && l % 4 == 0 && l <= 64) {
      const size_t smem = residual_tiled_smem(l);
      set_dyn_smem(residual_tiled_kernel, smem);
      int per_sm = 0, sms = 0, dev = 0;
      KRP_CUDA_CHECK(cudaGetDevice(&dev));
      KRP_CUDA_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
      KRP_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, residual_tiled_kernel, 256, smem));
      const int64_t nib = (n1 + TM - 1) / TM, ntile = (S + kRtS - 1) / kRtS;
      const int64_t want = std::max<int64_t>(1, (int64_t)std::max(per_sm, 1) * sms / nib);
      const dim3 g2((unsigned)std::min<int64_t>(ntile, want), (unsigned)nib);
      residual_tiled_kernel<<<g2, 256, smem, stream()>>>(Xf, n1, S, Q1, l, H, acc);
    } else if (aligned && n1 % 4 == 0) {
      const size_t smem = sizeof(float) * TM * TM;
      set_dyn_smem(residual_kernel<float, true>, smem);
      residual_kernel<float, true><<<grid, 256, smem, stream()>>>(Xf, n1, S, Q1, l, H, acc);
    } else {
      residual_kernel<float, false><<<grid, 256, 0, stream()>>>(Xf, n1, S, Q1, l, H, acc);
    }
  } else {
    const __nv_bfloat16* Xb = static_cast<const __nv_bfloat16*>(X);
    if (aligned && n1 % 8 == 0) {
      const size_t smem = sizeof(__nv_bfloat16) * TM * TM;
      set_dyn_smem(residual_kernel<__nv_bfloat16, true>, smem);
      residual_kernel<__nv_bfloat16, true><<<grid, 256, smem, stream()>>>(Xb, n1, S, Q1, l, H, acc);
    } else {
      residual_kernel<__nv_bfloat16, false><<<grid, 256, 0, stream()>>>(Xb, n1, S, Q1, l, H, acc);
    }
  }
  check_launch("residual");
}

}  // namespace krp
