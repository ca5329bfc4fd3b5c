// FP64 stages: thin QR of every sketch (Alg. 1 step 3, used by Alg. 6-8), the
// HOSVD of the small core used for rank truncation, and helpers.
#include <algorithm>

#include <cooperative_groups.h>

#include "common.cuh"

namespace krp {
namespace {

constexpr int kQrThreads = 512;
constexpr int kQrMaxL = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Householder QR of one m x l matrix per CTA.  Reflector j: x = A[j:, j],
// alpha = -sign(x_0)||x||, v = x - alpha e_1 (stored over column j),
// ||v||^2 = 2||x||(||x|| + |x_0|), A[j:, k] -= (2/||v||^2) v (v^T A[j:, k]) with
// v^T A[j:, k] = x^T A[j:, k] - alpha A[j, k] (one fused reduction per step).
// Q is formed by applying the reflectors in reverse order to [I; 0]; then the
// signs are fixed so that diag(R) >= 0.
__global__ void __launch_bounds__(kQrThreads) qr_kernel(const QrJob* __restrict__ jobs,
                                                        int* status) {
  const QrJob job = jobs[blockIdx.x];
  const int64_t m = job.m;
  const int l = job.l;
  double* A = job.work;
  __shared__ double w[kQrMaxL];
  __shared__ double tau[kQrMaxL];
  __shared__ double alph[kQrMaxL];
  __shared__ int bad;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  if (tid == 0) bad = 0;
  __syncthreads();
  for (int64_t e = tid; e < m * l; e += blockDim.x) {
    const double v = job.Y64 ? job.Y64[e] : (double)job.Y[e];
    if (!isfinite(v)) bad = 1;
    A[e] = v;
  }
  __syncthreads();
  if (bad) {
    if (tid == 0) atomicCAS(status, 0, (int)KRP_ENUMERIC);
    return;
  }
  for (int j = 0; j < l; ++j) {
    const double* aj = A + m * j;
    for (int k = j + warp; k < l; k += nwarps) {
      const double* ak = A + m * k;
      double part = 0.0;
      for (int64_t r = j + lane; r < m; r += 32) part = fma(aj[r], ak[r], part);
      part = warp_sum(part);
      if (lane == 0) w[k] = part;
    }
    __syncthreads();
    if (tid == 0) {
      const double normx = sqrt(w[j]);
      const double x0 = A[j + m * j];
      if (normx == 0.0) {
        alph[j] = 0.0;
        tau[j] = 0.0;
        for (int k = j + 1; k < l; ++k) w[k] = 0.0;
        A[j + m * j] = 0.0;
      } else {
        const double alpha = (x0 >= 0.0) ? -normx : normx;
        const double vtv = 2.0 * normx * (normx + fabs(x0));
        const double t = 2.0 / vtv;
        alph[j] = alpha;
        tau[j] = t;
        for (int k = j + 1; k < l; ++k) w[k] = t * (w[k] - alpha * A[j + m * k]);
        A[j + m * j] = x0 - alpha;  // v_0
      }
    }
    __syncthreads();
    const int64_t rows = m - j;
    const int cols = l - j - 1;
    for (int64_t e = tid; e < rows * cols; e += blockDim.x) {
      const int64_t r = j + e % rows;
      const int k = j + 1 + (int)(e / rows);
      A[r + m * k] -= A[r + m * j] * w[k];
    }
    __syncthreads();
  }
  // R (upper triangle) before A's columns are reused
  if (job.R) {
    for (int e = tid; e < l * l; e += blockDim.x) {
      const int r = e % l, c = e / l;
      double v = 0.0;
      if (r < c) v = A[r + m * c];
      if (r == c) v = alph[r];
      job.R[e] = v;
    }
  }
  double* Q = job.Q;
  for (int64_t e = tid; e < m * l; e += blockDim.x) {
    const int64_t r = e % m;
    const int64_t c = e / m;
    Q[e] = (r == c) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int j = l - 1; j >= 0; --j) {
    const double* v = A + m * j;  // v_r for r >= j
    for (int c = j + warp; c < l; c += nwarps) {
      const double* qc = Q + m * c;
      double part = 0.0;
      for (int64_t r = j + lane; r < m; r += 32) part = fma(v[r], qc[r], part);
      part = warp_sum(part);
      if (lane == 0) w[c] = tau[j] * part;
    }
    __syncthreads();
    const int64_t rows = m - j;
    const int cols = l - j;
    for (int64_t e = tid; e < rows * cols; e += blockDim.x) {
      const int64_t r = j + e % rows;
      const int c = j + (int)(e / rows);
      Q[r + m * c] -= v[r] * w[c];
    }
    __syncthreads();
  }
  // diag(R) >= 0
  for (int64_t e = tid; e < m * l; e += blockDim.x) {
    const int c = (int)(e / m);
    if (alph[c] < 0.0) Q[e] = -Q[e];
  }
  if (job.R) {
    __syncthreads();
    for (int e = tid; e < l * l; e += blockDim.x) {
      const int r = e % l;
      if (alph[r] < 0.0) job.R[e] = -job.R[e];
    }
  }
}

// S[a + l*b] += sum over the CTA's columns of G_(mode)[a, col] G_(mode)[b, col]
__global__ void gram_kernel(const double* __restrict__ G, int64_t P, int64_t l, int64_t ncols,
                            int64_t cols_per_cta, double* __restrict__ S) {
  extern __shared__ double colbuf[];  // 32 columns x l
  const int64_t c0 = (int64_t)blockIdx.x * cols_per_cta;
  const int64_t c1 = min(ncols, c0 + cols_per_cta);
  const int64_t pairs = l * l;
  double acc[16];
  for (int q = 0; q < 16; ++q) acc[q] = 0.0;
  for (int64_t cc = c0; cc < c1; cc += 32) {
    const int nc = (int)((c1 - cc) < 32 ? (c1 - cc) : 32);
    __syncthreads();
    for (int64_t e = threadIdx.x; e < nc * l; e += blockDim.x) {
      const int64_t a = e % l, c = cc + e / l;
      const int64_t p = c % P, s = c / P;
      colbuf[e] = G[p + P * a + P * l * s];
    }
    __syncthreads();
    for (int q = 0; q < 16; ++q) {
      const int64_t pr = threadIdx.x + (int64_t)q * blockDim.x;
      if (pr >= pairs) break;
      const int64_t a = pr % l, b = pr / l;
      double s = acc[q];
      for (int c = 0; c < nc; ++c) s = fma(colbuf[a + l * c], colbuf[b + l * c], s);
      acc[q] = s;
    }
  }
  for (int q = 0; q < 16; ++q) {
    const int64_t pr = threadIdx.x + (int64_t)q * blockDim.x;
    if (pr >= pairs) break;
    atomicAdd(S + pr, acc[q]);
  }
}

// Gram matrices of every mode of a small FP64 tensor in one launch:
//   S_n[a, b] = sum_c G_(n)[a, c] G_(n)[b, c],  a <= b computed, mirrored
// (G_(n)[a, c] = G[p + P a + P l s], c = (p, s)).  blockIdx.y is the mode;
// the CTAs of a mode split its columns, stage 32 of them at a time and add
// their partial sums into S_n (zeroed beforehand).  The pairs a <= b are
// enumerated (an FP64 warp instruction costs the same with idle lanes).
struct GramModes {
  const double* G;
  double* S[KRP_MAXD];
  int64_t P[KRP_MAXD];
  int64_t l[KRP_MAXD];
  int64_t ncols[KRP_MAXD];
  int64_t per[KRP_MAXD];
};
__global__ void __launch_bounds__(256) gram_modes_kernel(const GramModes M) {
  const int mode = blockIdx.y;
  const int64_t P = M.P[mode], l = M.l[mode], ncols = M.ncols[mode];
  const int64_t c0 = (int64_t)blockIdx.x * M.per[mode];
  const int64_t c1 = min(ncols, c0 + M.per[mode]);
  if (c0 >= c1) return;
  __shared__ double colbuf[32 * 64];
  __shared__ unsigned short tri[64 * 65 / 2];
  const int li = (int)l;
  for (int a = threadIdx.x; a < li; a += blockDim.x) {
    const int off = a * li - a * (a - 1) / 2;
    for (int b = a; b < li; ++b) tri[off + b - a] = (unsigned short)(a | (b << 8));
  }
  const int npair = li * (li + 1) / 2;
  constexpr int kMaxPairs = (64 * 65 / 2 + 255) / 256;
  double acc[kMaxPairs];
#pragma unroll
  for (int q = 0; q < kMaxPairs; ++q) acc[q] = 0.0;
  for (int64_t cc = c0; cc < c1; cc += 32) {
    const int nc = (int)((c1 - cc) < 32 ? (c1 - cc) : 32);
    __syncthreads();
    for (int e = threadIdx.x; e < nc * li; e += blockDim.x) {
      const int64_t a = e % li, c = cc + e / li;
      const int64_t p = c % P, sfx = c / P;
      colbuf[e] = M.G[p + P * a + P * l * sfx];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kMaxPairs; ++q) {
      const int pr = threadIdx.x + q * 256;
      if (pr >= npair) break;
      const int a = tri[pr] & 0xff, b = tri[pr] >> 8;
      double s0 = acc[q], s1 = 0.0;
      int c = 0;
      for (; c + 1 < nc; c += 2) {
        s0 = fma(colbuf[a + li * c], colbuf[b + li * c], s0);
        s1 = fma(colbuf[a + li * (c + 1)], colbuf[b + li * (c + 1)], s1);
      }
      if (c < nc) s0 = fma(colbuf[a + li * c], colbuf[b + li * c], s0);
      acc[q] = s0 + s1;
    }
  }
  double* S = M.S[mode];
#pragma unroll
  for (int q = 0; q < kMaxPairs; ++q) {
    const int pr = threadIdx.x + q * 256;
    if (pr >= npair) break;
    const int a = tri[pr] & 0xff, b = tri[pr] >> 8;
    atomicAdd(S + a + l * b, acc[q]);
    if (a != b) atomicAdd(S + b + l * a, acc[q]);
  }
}

constexpr int kEigMaxL = 64;


// Symmetric eigensolver for one l x l FP64 matrix per CTA (l <= 64), in two
// stages.  GB300 issues FP32 at ~58x its FP64 rate, so
//  1. cyclic Jacobi runs in FP32 on the matrix scaled by a power of two, with
//     the parallel (round-robin) pair ordering: each round rotates n/2
//     disjoint pairs (p_k, q_k).  The two-sided update S <- J^T S J of a round
//     maps every 2 x 2 block {p_i, q_i} x {p_j, q_j} onto itself, so each
//     thread updates whole blocks in place and a round needs two barriers;
//  2. the FP32 eigenvectors are refined in FP64 by the iteration of Ogita and
//     Aishima (Japan J. Indust. Appl. Math. 35, 2018), which uses only matrix
//     products: with R = I - X^T X and S = X^T A X, lambda_i = s_ii / (1 - r_ii),
//     E_ij = (s_ij + lambda_j r_ij) / (lambda_j - lambda_i) for eigenvalues
//     further apart than delta = 2 (||S - diag(lambda)|| + ||A|| ||R||), else
//     E_ij = r_ij / 2, and X <- X + X E.  It converges quadratically, so two
//     steps take the FP32 start (error ~1e-7) to FP64 rounding; within a
//     cluster narrower than delta it only restores orthonormality.
constexpr int kEigThreads = 256;
constexpr int kEigRefine = 2;
constexpr int kEigSweeps32 = 15;

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide FP32 sum of one value per thread (all threads call it).
__device__ float block_sum_f(float v, float* red) {
  const int tid = threadIdx.x, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((tid & 31) == 0) red[tid >> 5] = v;
  __syncthreads();
  float s = 0.f;
  for (int w = 0; w < nw; ++w) s += red[w];
  return s;
}

// Block-wide sum of one value per thread (all threads call it).
__device__ double block_sum(double v, double* red) {
  const int tid = threadIdx.x, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if ((tid & 31) == 0) red[tid >> 5] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < nw; ++w) s += red[w];
  return s;
}

// The Jacobi stage of the split eigensolver runs 16 warps: its rounds are
// latency-bound, and more warps shorten each thread's share of a round.
constexpr int kJacobiThreads = 512;

// NT threads, n <= 64 so P <= 32 pairs and jstep = NT / P >= NT / 32; red
// holds 2 * NT / 32 doubles.
template <int EP, int NT>  // row pitch of the padded matrices, threads
__device__ void jacobi32(float (*Sa)[EP], float (*Sb)[EP], float (*V)[EP], int n, double* red) {
  // per-thread work bounds of a round: blocks per thread and V rows
  constexpr int kJm = (32 + NT / 32 - 1) / (NT / 32);
  constexpr int kJv = (64 + NT / 32 - 1) / (NT / 32);
  const int tid = threadIdx.x, lane = tid & 31, P = n / 2;
  // fixed work split of the round updates (no per-item integer division):
  // threads t < jstep * P own pair ib0 = t % P and rows/blocks jb0 + m jstep
  const int jstep = (int)blockDim.x / P;
  const int ib0 = tid % P;
  const int jb0 = (tid < jstep * P) ? tid / P : n;  // idle threads get an empty range
  float(*S)[EP] = Sa;    // current matrix
  float(*Sn)[EP] = Sb;   // the round writes the rotated matrix here
  for (int sweep = 0; sweep < kEigSweeps32; ++sweep) {
    // squared norms in FP32: the matrix is scaled to max |s_ij| < 1, so the
    // sums of squares are far inside FP32 range for a threshold test
    float o = 0.f, dg = 0.f;
    for (int e = tid; e < n * n; e += blockDim.x) {
      const int r = e % n, c = e / n;
      const float v = S[r][c] * S[r][c];
      if (r == c)
        dg += v;
      else
        o += v;
    }
    float* redf = reinterpret_cast<float*>(red);
    const float off = block_sum_f(o, redf);
    const float dia = block_sum_f(dg, redf + NT / 32);
    // off-diagonal norm at 1e-6 of the diagonal's: the FP64 stage does the
    // rest (stopping at 1e-4 left the refined vectors of graded spectra, such
    // as a block Hankel's, orthonormal only to ~1e-5)
    if (!(off > 1e-12f * dia) || off == 0.f) break;
    // round-robin tournament: position 0 holds player 0, position k >= 1
    // holds player ((k - 1 + round) mod (n - 1)) + 1; pairs (k, n-1-k).  Lane
    // k < P keeps (k - 1 + round) and (n - 2 - k + round) mod (n - 1) as
    // counters advanced once per round.
    int pos_p = (lane >= 1) ? lane - 1 : 0, pos_q = n - 2 - lane;
    for (int round = 0; round < n - 1; ++round) {
      // every warp forms all P rotations of the round, lane k the k-th, from
      // the matrix of the previous round (read-only during this round), and
      // hands them to the other lanes by shuffles: one barrier per round
      int p = 0, q = 0;
      float c = 1.f, s = 0.f;
      if (lane < P) {
        p = (lane == 0) ? 0 : pos_p + 1;
        q = pos_q + 1;
        pos_p = (pos_p + 1 == n - 1) ? 0 : pos_p + 1;
        pos_q = (pos_q + 1 == n - 1) ? 0 : pos_q + 1;
        if (p > q) {
          const int t = p;
          p = q;
          q = t;
        }
        const float apq = S[p][q], app = S[p][p], aqq = S[q][q];
        if (apq * apq > 1e-16f * fabsf(app * aqq)) {
          // t = tan of the angle: the root of t^2 + 2 theta t - 1 = 0 with
          // |t| <= 1, theta = (aqq - app) / (2 apq), written without theta:
          // t = 2 apq sgn(dq) / (|dq| + sqrt(dq^2 + 4 apq^2)), dq = aqq - app.
          // t only decides how far apq is reduced; c^2 + s^2 = 1 is kept to
          // FP32 rounding by one Newton step on the hardware rsqrt.
          const float dq = aqq - app;
          const float h = sqrtf(fmaf(dq, dq, 4.f * apq * apq));
          const float t = __fdividef(2.f * apq * copysignf(1.f, dq), fabsf(dq) + h);
          const float x = fmaf(t, t, 1.f);
          c = rsqrtf(x);
          c = c * fmaf(-0.5f * x * c, c, 1.5f);
          s = t * c;
        }
      }
      const int pi = __shfl_sync(0xffffffffu, p, ib0), qi = __shfl_sync(0xffffffffu, q, ib0);
      const float ci = __shfl_sync(0xffffffffu, c, ib0), si = __shfl_sync(0xffffffffu, s, ib0);
      // 2x2 blocks (i, j) of S: thread t takes i = t % P and j = t / P + m * jstep
      // (m < kJm); every load of the round is issued before any store, so the
      // shared-memory round trips overlap (S and Sn are swapped at run time,
      // which keeps the compiler from reordering them itself)
      int pj[kJm], qj[kJm];
      float cj[kJm], sj[kJm], ea[kJm], eb[kJm], ec[kJm], ed[kJm];
      bool live[kJm];
#pragma unroll
      for (int m = 0; m < kJm; ++m) {
        const int j = jb0 + m * jstep;
        live[m] = j < P;
        const int jj = live[m] ? j : 0;
        pj[m] = __shfl_sync(0xffffffffu, p, jj);
        qj[m] = __shfl_sync(0xffffffffu, q, jj);
        cj[m] = __shfl_sync(0xffffffffu, c, jj);
        sj[m] = __shfl_sync(0xffffffffu, s, jj);
      }
#pragma unroll
      for (int m = 0; m < kJm; ++m) {
        ea[m] = S[pi][pj[m]];
        eb[m] = S[pi][qj[m]];
        ec[m] = S[qi][pj[m]];
        ed[m] = S[qi][qj[m]];
      }
      float vp[kJv], vq[kJv];
#pragma unroll
      for (int m = 0; m < kJv; ++m) {
        const int r = min(jb0 + m * jstep, n - 1);
        vp[m] = V[r][pi];
        vq[m] = V[r][qi];
      }
#pragma unroll
      for (int m = 0; m < kJm; ++m) {
        if (!live[m]) continue;
        // columns (p_j, q_j), then rows (p_i, q_i)
        const float a1 = cj[m] * ea[m] - sj[m] * eb[m], b1 = sj[m] * ea[m] + cj[m] * eb[m];
        const float c1 = cj[m] * ec[m] - sj[m] * ed[m], d1 = sj[m] * ec[m] + cj[m] * ed[m];
        float a2 = ci * a1 - si * c1, c2 = si * a1 + ci * c1;
        float b2 = ci * b1 - si * d1, d2 = si * b1 + ci * d1;
        if (ib0 == jb0 + m * jstep && si != 0.f) {  // the rotated pair's coupling is zero by construction
          b2 = 0.f;
          c2 = 0.f;
        }
        Sn[pi][pj[m]] = a2;
        Sn[pi][qj[m]] = b2;
        Sn[qi][pj[m]] = c2;
        Sn[qi][qj[m]] = d2;
      }
      // rows r of V for pair k = t % P: r = t / P + m * jstep
#pragma unroll
      for (int m = 0; m < kJv; ++m) {
        const int r = jb0 + m * jstep;
        if (r >= n) continue;
        V[r][pi] = ci * vp[m] - si * vq[m];
        V[r][qi] = si * vp[m] + ci * vq[m];
      }
      __syncthreads();
      float(*t)[EP] = S;
      S = Sn;
      Sn = t;
    }
  }
}

// C = A B for l x l matrices in shared memory.
template <int EP>
__device__ void smem_gemm(const double (*A)[EP], const double (*B)[EP], double (*C)[EP], int l) {
  for (int e = threadIdx.x; e < l * l; e += blockDim.x) {
    const int i = e % l, j = e / l;
    double acc = 0.0;
    for (int k = 0; k < l; ++k) acc = fma(A[i][k], B[k][j], acc);
    C[i][j] = acc;
  }
}

// S = X^T T and G = X^T X (both symmetric when T = A X with A symmetric),
// computed together over the packed pairs i <= j and mirrored: an FP64 warp
// instruction costs the same with idle lanes, so the pairs are enumerated
// rather than masked out of a full l x l loop.
template <int EP>
__device__ void smem_sym_pair(const double (*X)[EP], const double (*T)[EP], double (*S)[EP],
                              double (*G)[EP], const unsigned short* tri, int l) {
  const int np = l * (l + 1) / 2;
  for (int p = threadIdx.x; p < np; p += blockDim.x) {
    const int i = tri[p] & 0xff, j = tri[p] >> 8;
    double s = 0.0, g = 0.0;
    for (int k = 0; k < l; ++k) {
      const double xi = X[k][i];
      s = fma(xi, T[k][j], s);
      g = fma(xi, X[k][j], g);
    }
    S[i][j] = s;
    S[j][i] = s;
    G[i][j] = g;
    G[j][i] = g;
  }
}

// ML: largest l the instance handles (shared memory 5 * 8 * ML * (ML+1) bytes)
template <int ML>
__global__ void __launch_bounds__(kEigThreads) eig_kernel(const EigJob* __restrict__ jobs, int* status) {
  constexpr int kEP = ML + 1;  // padded row pitch
  const EigJob job = jobs[blockIdx.x];
  const int l = job.l;
  const int n = (l + 1) & ~1;  // padded to even for the tournament
  extern __shared__ double eig_smem[];
  constexpr int kMat = ML * kEP;
  double(*A)[kEP] = reinterpret_cast<double(*)[kEP]>(eig_smem);
  double(*X)[kEP] = reinterpret_cast<double(*)[kEP]>(eig_smem + kMat);
  double(*T)[kEP] = reinterpret_cast<double(*)[kEP]>(eig_smem + 2 * kMat);
  double(*Sm)[kEP] = reinterpret_cast<double(*)[kEP]>(eig_smem + 3 * kMat);
  double(*Rm)[kEP] = reinterpret_cast<double(*)[kEP]>(eig_smem + 4 * kMat);
  // the FP32 stage lives in T's storage (S, V) and Sm's (the second S buffer)
  float(*S32)[kEP] = reinterpret_cast<float(*)[kEP]>(eig_smem + 2 * kMat);
  float(*V32)[kEP] = reinterpret_cast<float(*)[kEP]>(eig_smem + 2 * kMat) + ML;
  float(*S32b)[kEP] = reinterpret_cast<float(*)[kEP]>(eig_smem + 3 * kMat);
  __shared__ int order[ML];
  __shared__ double lam[ML];
  __shared__ double red[16];
  __shared__ float redf[8];
  __shared__ unsigned short tri[ML * (ML + 1) / 2];
  const int tid = threadIdx.x;
  for (int i = tid; i < l; i += blockDim.x) {  // pairs (i, j), i <= j, ordered by i
    const int off = i * l - i * (i - 1) / 2;
    for (int j = i; j < l; ++j) tri[off + j - i] = (unsigned short)(i | (j << 8));
  }

  // scale by a power of two (exact) so that max |a_ij| is in [0.5, 1)
  float amax = 0.f;
  for (int e = tid; e < l * l; e += blockDim.x) amax = fmaxf(amax, (float)fabs(job.S[e]));
  amax = warp_max(amax);
  if ((tid & 31) == 0) redf[tid >> 5] = amax;
  __syncthreads();
  amax = 0.f;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) amax = fmaxf(amax, redf[w]);
  int ex = 0;
  if (amax > 0.f && isfinite(amax)) frexpf(amax, &ex);
  const double scale = ldexp(1.0, -ex);
  bool finite_in = true;
  for (int e = tid; e < n * n; e += blockDim.x) {
    const int r = e % n, c = e / n;
    const double v = (r < l && c < l) ? job.S[r + l * c] * scale : 0.0;
    finite_in = finite_in && isfinite(v);
    A[r][c] = v;
    S32[r][c] = (float)v;
    V32[r][c] = (r == c) ? 1.f : 0.f;
  }
  if (!__syncthreads_and(finite_in)) {
    if (tid == 0) atomicCAS(status, 0, (int)KRP_ENUMERIC);
    return;
  }
  jacobi32<kEP, kEigThreads>(S32, S32b, V32, n, red);
  for (int e = tid; e < l * l; e += blockDim.x) {
    const int r = e % l, c = e / l;
    X[r][c] = (double)V32[r][c];
  }
  __syncthreads();
  double a2 = 0.0;
  for (int e = tid; e < l * l; e += blockDim.x) a2 = fma(A[e % l][e / l], A[e % l][e / l], a2);
  const double anorm = sqrt(block_sum(a2, red));
  for (int it = 0; it < kEigRefine; ++it) {
    smem_gemm<kEP>(A, X, T, l);  // T = A X
    __syncthreads();
    smem_sym_pair<kEP>(X, T, Sm, Rm, tri, l);  // S = X^T A X, X^T X (turned into R below)
    __syncthreads();
    double soff = 0.0, r2 = 0.0;
    for (int e = tid; e < l * l; e += blockDim.x) {
      const int i = e % l, j = e / l;
      const double rij = (i == j ? 1.0 : 0.0) - Rm[i][j];
      r2 = fma(rij, rij, r2);
      if (i != j) soff = fma(Sm[i][j], Sm[i][j], soff);
    }
    for (int i = tid; i < l; i += blockDim.x) lam[i] = Sm[i][i] / Rm[i][i];  // 1 - r_ii = (X^T X)_ii
    const double sn = block_sum(soff, red);  // diag(S) - lambda is second order: left out
    const double rn = block_sum(r2, red + 8);
    const double delta = 2.0 * (sqrt(sn) + anorm * sqrt(rn));
    // E (into T): built from the symmetric S and R, read before any write
    for (int e = tid; e < l * l; e += blockDim.x) {
      const int i = e % l, j = e / l;
      const double rij = (i == j ? 1.0 : 0.0) - Rm[i][j];
      double eij = 0.5 * rij;
      const double gap = lam[j] - lam[i];
      if (i != j && fabs(gap) > delta) eij = (Sm[i][j] + lam[j] * rij) / gap;
      T[i][j] = eij;
    }
    __syncthreads();
    smem_gemm<kEP>(X, T, Sm, l);  // X E
    __syncthreads();
    for (int e = tid; e < l * l; e += blockDim.x) {
      const int i = e % l, j = e / l;
      X[i][j] += Sm[i][j];
    }
    __syncthreads();
  }
  if (tid == 0) {
    for (int i = 0; i < l; ++i) order[i] = i;
    for (int i = 1; i < l; ++i) {  // insertion sort, descending eigenvalue
      const int key = order[i];
      int j = i - 1;
      while (j >= 0 && lam[order[j]] < lam[key]) {
        order[j + 1] = order[j];
        --j;
      }
      order[j + 1] = key;
    }
    bool ok = true;
    for (int i = 0; i < l; ++i) ok = ok && isfinite(lam[i]);
    if (!ok) atomicCAS(status, 0, (int)KRP_ENUMERIC);
  }
  __syncthreads();
  for (int e = tid; e < l * job.r; e += blockDim.x) {
    const int r = e % l, c = e / l;
    job.U[e] = X[r][order[c]];
  }
  if (job.ev)
    for (int i = tid; i < l; i += blockDim.x) job.ev[i] = lam[order[i]] / scale;
}

// Split form of the eigensolver for a few problems (a d-mode truncation): the
// FP32 Jacobi stage runs one CTA per problem and leaves its eigenvectors X0
// and the power-of-two scale in a scratch block; the FP64 refinement then runs
// on a cluster of kEigCluster CTAs per problem, so that its O(l^3) FP64 work
// (GB300: 0.5 FMA per clock per SM sub-partition) spreads over as many SMs.
constexpr int kEigCluster = 8;
constexpr int kEigScratch = kEigMaxL * kEigMaxL + 8;  // doubles per problem

template <int ML>
__global__ void __launch_bounds__(kJacobiThreads)
    eig_jacobi_kernel(const EigJob* __restrict__ jobs, double* __restrict__ scratch, int* status) {
  constexpr int kEP = ML + 1;
  const EigJob job = jobs[blockIdx.x];
  const int l = job.l;
  const int n = (l + 1) & ~1;
  extern __shared__ float ej_smem[];
  float(*S32)[kEP] = reinterpret_cast<float(*)[kEP]>(ej_smem);
  float(*S32b)[kEP] = reinterpret_cast<float(*)[kEP]>(ej_smem + ML * kEP);
  float(*V32)[kEP] = reinterpret_cast<float(*)[kEP]>(ej_smem + 2 * ML * kEP);
  __shared__ double red[2 * kJacobiThreads / 32];
  __shared__ float redf[kJacobiThreads / 32];
  const int tid = threadIdx.x;
  // scale by a power of two (exact) so that max |a_ij| is in [0.5, 1)
  float amax = 0.f;
  for (int e = tid; e < l * l; e += blockDim.x) amax = fmaxf(amax, (float)fabs(job.S[e]));
  amax = warp_max(amax);
  if ((tid & 31) == 0) redf[tid >> 5] = amax;
  __syncthreads();
  amax = 0.f;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) amax = fmaxf(amax, redf[w]);
  int ex = 0;
  if (amax > 0.f && isfinite(amax)) frexpf(amax, &ex);
  const double scale = ldexp(1.0, -ex);
  bool finite_in = true;
  for (int e = tid; e < n * n; e += blockDim.x) {
    const int r = e % n, c = e / n;
    const double v = (r < l && c < l) ? job.S[r + l * c] * scale : 0.0;
    finite_in = finite_in && isfinite(v);
    S32[r][c] = (float)v;
    V32[r][c] = (r == c) ? 1.f : 0.f;
  }
  double* out = scratch + (size_t)blockIdx.x * kEigScratch;
  if (!__syncthreads_and(finite_in)) {
    if (tid == 0) {
      atomicCAS(status, 0, (int)KRP_ENUMERIC);
      out[kEigMaxL * kEigMaxL] = 0.0;  // marks the problem as failed for the refinement
    }
    return;
  }
  jacobi32<kEP, kJacobiThreads>(S32, S32b, V32, n, red);
  for (int e = tid; e < l * l; e += blockDim.x) out[e] = (double)V32[e % l][e / l];
  if (tid == 0) out[kEigMaxL * kEigMaxL] = scale;
}

// Ogita-Aishima refinement of X0 (see the fused kernel above) on a cluster:
// CTA `rank` owns the columns [c0, c0 + w) of T = A X, S = X^T T, G = X^T X,
// E and X + X E; each CTA holds all of A and X.  Per step the CTAs exchange
// their eigenvalue estimates and partial norms, then their new X columns,
// through distributed shared memory, with one cluster barrier after each.
template <int ML>
__global__ void __cluster_dims__(kEigCluster, 1, 1) __launch_bounds__(kEigThreads)
    eig_refine_kernel(const EigJob* __restrict__ jobs, const double* __restrict__ scratch,
                      int* status) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  constexpr int kEP = ML + 1;
  constexpr int CW = (ML + kEigCluster - 1) / kEigCluster;
  const int rank = (int)cluster.block_rank();
  const EigJob job = jobs[blockIdx.y];
  const int l = job.l;
  const int cw = (l + kEigCluster - 1) / kEigCluster;
  const int c0 = rank * cw;
  const int w = max(0, min(l, c0 + cw) - c0);
  extern __shared__ double er_smem[];
  double(*A)[kEP] = reinterpret_cast<double(*)[kEP]>(er_smem);
  double(*Xa)[kEP] = reinterpret_cast<double(*)[kEP]>(er_smem + ML * kEP);
  double(*Xb)[kEP] = reinterpret_cast<double(*)[kEP]>(er_smem + 2 * ML * kEP);
  __shared__ double Tc[ML][CW + 1], Sc[ML][CW + 1], Gc[ML][CW + 1];
  __shared__ double lam[ML];
  __shared__ double part[kEigCluster][2];
  __shared__ double red[16];
  __shared__ int order[ML];
  const int tid = threadIdx.x;
  const double* src = scratch + (size_t)blockIdx.y * kEigScratch;
  const double scale = src[kEigMaxL * kEigMaxL];
  const bool failed = !(scale > 0.0);  // uniform over the cluster
  double a2 = 0.0;
  for (int e = tid; e < l * l; e += blockDim.x) {
    const int r = e % l, c = e / l;
    const double v = failed ? 0.0 : job.S[e] * scale;
    A[r][c] = v;
    Xa[r][c] = failed ? 0.0 : src[e];
    a2 = fma(v, v, a2);
  }
  const double anorm = sqrt(block_sum(a2, red));  // its barriers publish A and X
  double(*X)[kEP] = Xa;
  double(*Xn)[kEP] = Xb;
  for (int it = 0; it < kEigRefine && !failed; ++it) {
    for (int e = tid; e < l * w; e += blockDim.x) {  // T = A X(:, own)
      const int i = e % l, cc = e / l;
      double acc = 0.0;
      for (int k = 0; k < l; ++k) acc = fma(A[i][k], X[k][c0 + cc], acc);
      Tc[i][cc] = acc;
    }
    __syncthreads();
    for (int e = tid; e < l * w; e += blockDim.x) {  // S, G (own columns)
      const int i = e % l, cc = e / l;
      double sacc = 0.0, gacc = 0.0;
      for (int k = 0; k < l; ++k) {
        const double xi = X[k][i];
        sacc = fma(xi, Tc[k][cc], sacc);
        gacc = fma(xi, X[k][c0 + cc], gacc);
      }
      Sc[i][cc] = sacc;
      Gc[i][cc] = gacc;
    }
    __syncthreads();
    double soff = 0.0, r2 = 0.0;
    for (int e = tid; e < l * w; e += blockDim.x) {
      const int i = e % l, cc = e / l, j = c0 + cc;
      const double rij = (i == j ? 1.0 : 0.0) - Gc[i][cc];
      r2 = fma(rij, rij, r2);
      if (i != j) soff = fma(Sc[i][cc], Sc[i][cc], soff);
    }
    const double sn_part = block_sum(soff, red);
    const double rn_part = block_sum(r2, red + 8);
    // own eigenvalue estimates and partial norms to every CTA of the cluster
    for (int e = tid; e < w * kEigCluster; e += blockDim.x) {
      const int cc = e % w, q = e / w, j = c0 + cc;
      double* rl = cluster.map_shared_rank(lam, q);
      rl[j] = Sc[j][cc] / Gc[j][cc];  // 1 - r_jj = (X^T X)_jj
    }
    if (tid < kEigCluster) {
      double* rp = cluster.map_shared_rank(&part[0][0], tid);
      rp[2 * rank] = sn_part;
      rp[2 * rank + 1] = rn_part;
    }
    cluster.sync();
    double sn = 0.0, rn = 0.0;
    for (int q = 0; q < kEigCluster; ++q) {
      sn += part[q][0];
      rn += part[q][1];
    }
    const double delta = 2.0 * (sqrt(sn) + anorm * sqrt(rn));
    for (int e = tid; e < l * w; e += blockDim.x) {  // E (own columns) into Tc
      const int i = e % l, cc = e / l, j = c0 + cc;
      const double rij = (i == j ? 1.0 : 0.0) - Gc[i][cc];
      double eij = 0.5 * rij;
      const double gap = lam[j] - lam[i];
      if (i != j && fabs(gap) > delta) eij = (Sc[i][cc] + lam[j] * rij) / gap;
      Tc[i][cc] = eij;
    }
    __syncthreads();
    for (int e = tid; e < l * w; e += blockDim.x) {  // X + X E (own columns) to every CTA
      const int k = e % l, cc = e / l, j = c0 + cc;
      double acc = X[k][j];
      for (int i = 0; i < l; ++i) acc = fma(X[k][i], Tc[i][cc], acc);
      for (int q = 0; q < kEigCluster; ++q) {
        double* rx = cluster.map_shared_rank(&Xn[0][0], q);
        rx[k * kEP + j] = acc;
      }
    }
    cluster.sync();
    double(*t)[kEP] = X;
    X = Xn;
    Xn = t;
  }
  if (rank != 0 || failed) return;
  if (tid == 0) {
    for (int i = 0; i < l; ++i) order[i] = i;
    for (int i = 1; i < l; ++i) {  // insertion sort, descending eigenvalue
      const int key = order[i];
      int j = i - 1;
      while (j >= 0 && lam[order[j]] < lam[key]) {
        order[j + 1] = order[j];
        --j;
      }
      order[j + 1] = key;
    }
    bool ok = true;
    for (int i = 0; i < l; ++i) ok = ok && isfinite(lam[i]);
    if (!ok) atomicCAS(status, 0, (int)KRP_ENUMERIC);
  }
  __syncthreads();
  for (int e = tid; e < l * job.r; e += blockDim.x) {
    const int r = e % l, c = e / l;
    job.U[e] = X[r][order[c]];
  }
  if (job.ev)
    for (int i = tid; i < l; i += blockDim.x) job.ev[i] = lam[order[i]] / scale;
}

// out = G x_mode U^T: out[p + P*a + P*r*s] = sum_i G[p + P*i + P*n*s] U[i + n*a]
__global__ void ttm_small_kernel(const double* __restrict__ G, int64_t P, int64_t n, int64_t Sfx,
                                 const double* __restrict__ U, int r, double* __restrict__ out) {
  const int64_t total = P * r * Sfx;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = e % P;
    const int64_t a = (e / P) % r;
    const int64_t s = e / (P * r);
    double acc = 0.0;
    const double* g = G + p + P * n * s;
    for (int64_t i = 0; i < n; ++i) acc = fma(g[P * i], U[i + n * a], acc);
    out[e] = acc;
  }
}

__global__ void matmul_kernel(const double* __restrict__ A, const double* __restrict__ B,
                              double* __restrict__ C, int64_t m, int k, int n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % m, j = e / m;
    double acc = 0.0;
    for (int t = 0; t < k; ++t) acc = fma(A[i + m * t], B[t + (int64_t)k * j], acc);
    C[e] = acc;
  }
}

__global__ void sumsq_kernel(const double* __restrict__ x, int64_t n, double* out) {
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    acc = fma(x[i], x[i], acc);
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, acc);
}

__global__ void finite_kernel(const double* __restrict__ x, int64_t n, int* status) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    if (!isfinite(x[i])) atomicCAS(status, 0, (int)KRP_ENUMERIC);
}

// ---------------------------------------------------------------------------
// Shifted CholeskyQR3 in FP64 (Fukaya, Kannan, Nakatsukasa, Zhang, Yamamoto,
// SIAM J. Sci. Comput. 2020): three passes of  G = W^T W (+ s I on the first),
// G = R^T R (Cholesky), W <- W R^{-1}.  The thin QR it returns is the unique one
// with diag(R) > 0 whenever Y has full column rank (then it equals the
// Householder result), and the first-pass shift keeps it defined for rank-
// deficient sketches.  All three kinds of step spread over many SMs.
constexpr int kCqrMaxL = 64;
constexpr int kCqrRows = 32;  // rows per CTA in the Gram / solve kernels

struct CqrJob {
  const float* Y;      // FP32 input (pass 1) or null
  const double* Y64;   // FP64 input (pass 1) or null
  double* W;           // m x l FP64 working matrix (passes 2, 3 read it)
  double* Q;           // final output
  double* G;           // l x l Gram accumulator
  double* Rk;          // 3 x l x l upper factors of the passes
  double* R;           // optional product R3 R2 R1
  unsigned long long* defmask;  // columns refilled in the current pass (bit j)
  int64_t m;
  int l;
};

// Deterministic pseudo-random entry used to refill a column whose pivot
// collapsed (exactly dependent or zero column): the next pass orthonormalises
// it against the others, completing the basis as Householder QR would.
__device__ __forceinline__ double refill_value(int64_t r, int j) {
  uint32_t h = static_cast<uint32_t>(r) * 0x9E3779B1u ^ static_cast<uint32_t>(j) * 0x85EBCA77u;
  h ^= h >> 15;
  h *= 0x2C1B3C6Du;
  h ^= h >> 12;
  h *= 0x297A2D39u;
  h ^= h >> 15;
  return (static_cast<double>(h) + 0.5) * 0x1p-32 - 0.5;
}

// Up to kCqrMaxBatch problems passed to the kernels by value, or any number
// as a job array in device memory.
constexpr int kCqrMaxBatch = 8;
struct CqrBatch {
  CqrJob job[kCqrMaxBatch];
};
struct CqrJobArray {
  const CqrJob* job;
};
__device__ __forceinline__ CqrJob job_at(const CqrBatch& b, int i) { return b.job[i]; }
__device__ __forceinline__ CqrJob job_at(const CqrJobArray& b, int i) { return b.job[i]; }

template <bool FROM_INPUT, class JOBS>
__global__ void __launch_bounds__(256) cqr_gram_kernel(const JOBS jobs, int* status) {
  const CqrJob job = job_at(jobs, blockIdx.y);
  const int64_t r0 = (int64_t)blockIdx.x * kCqrRows;
  if (r0 >= job.m) return;
  const int l = job.l;
  const int rows = (int)((job.m - r0) < kCqrRows ? (job.m - r0) : kCqrRows);
  __shared__ double blk[kCqrRows][kCqrMaxL + 1];
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int e = threadIdx.x; e < rows * l; e += blockDim.x) {
    const int r = e % rows, c = e / rows;
    const int64_t idx = r0 + r + job.m * c;
    double v;
    if (FROM_INPUT)
      v = job.Y64 ? job.Y64[idx] : (double)job.Y[idx];
    else
      v = job.W[idx];
    if (!isfinite(v)) bad = 1;
    blk[r][c] = v;
  }
  __syncthreads();
  if (bad) {
    if (threadIdx.x == 0) atomicCAS(status, 0, (int)KRP_ENUMERIC);
    return;
  }
  // upper triangle (a <= b) of the partial Gram
  const int pairs = l * (l + 1) / 2;
  for (int p = threadIdx.x; p < pairs; p += blockDim.x) {
    int a = 0, rem = p;
    while (rem >= l - a) {
      rem -= l - a;
      ++a;
    }
    const int b = a + rem;
    double s = 0.0;
    for (int r = 0; r < rows; ++r) s = fma(blk[r][a], blk[r][b], s);
    atomicAdd(job.G + a + l * b, s);
  }
}

// Cholesky G (+ shift) = R^T R of one l x l matrix per CTA; R stored in Rk[pass].
// GB300 runs FP64 at 0.5 FMA per clock in each of an SM's four sub-partitions,
// so the CTA is four warps (one per sub-partition) and a column step is one
// barrier: every thread takes d_j = A[j, j] and its reciprocal itself, then
// updates its share of the trailing upper triangle,
//   A[a, b] -= (A[j, a] / d_j) A[j, b]   (j < a <= b),
// over a packed pair list, four pairs per pass with all loads ahead of the
// stores.  Row j is not touched after step j, so the unscaled rows give
// R[j, i] = A[j, i] / sqrt(d_j) in one parallel pass at the end (sqrt off the
// dependent chain).
constexpr int kCholThreads = 128;
template <class JOBS>
__global__ void __launch_bounds__(kCholThreads) cqr_chol_kernel(const JOBS jobs, int pass) {
  const CqrJob job = job_at(jobs, blockIdx.x);
  const int l = job.l;
  __shared__ double A[kCqrMaxL][kCqrMaxL + 1];
  __shared__ double diag0[kCqrMaxL], rsq[kCqrMaxL], sq[kCqrMaxL];
  __shared__ unsigned short tri[kCqrMaxL * (kCqrMaxL + 1) / 2];
  __shared__ double tol;
  __shared__ unsigned long long mask;
  const int tid = threadIdx.x;
  for (int e = tid; e < l * l; e += blockDim.x) {
    const int a = e % l, b = e / l;
    if (a <= b) A[a][b] = job.G[a + l * b];
  }
  // pairs (a, b), a <= b, ordered by a: those with a > j start at
  // off(j + 1) = sum_{a <= j} (l - a)
  for (int a = tid; a < l; a += blockDim.x) {
    const int off = a * l - a * (a - 1) / 2;
    for (int b = a; b < l; ++b) tri[off + b - a] = (unsigned short)(a | (b << 8));
  }
  __syncthreads();
  if (tid == 0) {
    double tr = 0.0, dmax = 0.0;
    for (int j = 0; j < l; ++j) {
      diag0[j] = A[j][j];
      tr += A[j][j];
      dmax = fmax(dmax, A[j][j]);
    }
    if (pass == 0) {
      // s = 11 (m l + l (l + 1)) u ||Y||^2 with ||Y||_F^2 >= ||Y||_2^2
      const double s = 11.0 * ((double)job.m * l + (double)l * (l + 1)) * 0x1p-53 * tr;
      for (int j = 0; j < l; ++j) A[j][j] += s;
    }
    // pass 0: only exactly zero columns are refilled (the shift handles the
    // rest); later passes: pivots lost to cancellation
    tol = (pass == 0) ? 0.0 : 64.0 * l * 0x1p-53 * dmax;
  }
  __syncthreads();
  const int npair = l * (l + 1) / 2;
  const double tl = tol;
  unsigned long long msk = 0ull;
  int off = 0;
  for (int j = 0; j < l; ++j) {
    off += l - j;  // first pair with a > j
    const double d = A[j][j];
    const bool deficient = (pass == 0) ? !(diag0[j] > 0.0) : !(d > tl);
    // a refilled column gets R[j, j] = 1 and a zero row: no update
    const double nid = deficient ? 0.0 : -__drcp_rn(d);
    msk |= (unsigned long long)deficient << j;
    for (int e0 = off; e0 < npair; e0 += 4 * kCholThreads) {
      int ia[4], ib[4];
      bool ok[4];
      double ja[4], jb[4], ab[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int e = e0 + tid + kCholThreads * q;
        ok[q] = e < npair;
        const unsigned t = ok[q] ? tri[e] : 0u;
        ia[q] = t & 0xff;
        ib[q] = t >> 8;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        ja[q] = A[j][ia[q]];
        jb[q] = A[j][ib[q]];
        ab[q] = A[ia[q]][ib[q]];
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (ok[q]) A[ia[q]][ib[q]] = fma(ja[q] * nid, jb[q], ab[q]);
    }
    __syncthreads();
  }
  if (tid == 0) mask = msk;
  __syncthreads();
  msk = mask;
  for (int j = tid; j < l; j += blockDim.x) {
    const bool deficient = (msk >> j) & 1ull;
    const double r = deficient ? 1.0 : sqrt(A[j][j]);
    sq[j] = r;
    rsq[j] = deficient ? 0.0 : 1.0 / r;
  }
  __syncthreads();
  double* R = job.Rk + (size_t)pass * l * l;
  for (int e = tid; e < l * l; e += blockDim.x) {
    const int a = e % l, b = e / l;
    R[e] = (a < b) ? A[a][b] * rsq[a] : (a == b ? sq[a] : 0.0);
  }
  if (tid == 0) *job.defmask = msk;
  if (job.R && pass == 2) {
    __syncthreads();  // R3 (global) written by this block
    // R = R3 (R2 R1): T = R2 R1 into the lower triangle of A (T[a, b] at
    // A[b][a]), then R3 T; both upper triangular products cost l^3 / 6
    const double* R1 = job.Rk;
    const double* R2 = job.Rk + (size_t)l * l;
    const double* R3 = job.Rk + 2 * (size_t)l * l;
    for (int p = tid; p < npair; p += blockDim.x) {
      const int a = tri[p] & 0xff, b = tri[p] >> 8;
      double t = 0.0;
      for (int q = a; q <= b; ++q) t = fma(R2[a + l * q], R1[q + l * b], t);
      A[b][a] = t;
    }
    __syncthreads();
    for (int e = tid; e < l * l; e += blockDim.x) {
      const int a = e % l, b = e / l;
      double acc = 0.0;
      for (int k = a; k <= b; ++k) acc = fma(R3[a + l * k], A[b][k], acc);
      job.R[e] = (a <= b) ? acc : 0.0;
    }
  }
}

// W_out[r, :] = W_in[r, :] R^{-1} by forward substitution.  GB300 runs FP64
// at 0.5 FMA per clock in each of an SM's four sub-partitions, so one warp
// instruction occupies its sub-partition's FP64 unit for ~64 clocks: the
// rows are spread so that as many warps as possible, each on its own
// sub-partition, share the work.  A CTA of 4 warps takes 32 / TPR rows per
// warp; the TPR lanes of a row split the dot product sum_{k<j} x_k R[k, j]
// (k = lane mod TPR, TPR apart) and combine it with log2(TPR) shuffles.  R is
// copied to shared memory column-major (column j contiguous in k).
constexpr int kSolveThreads = 128;
constexpr int kSolveRowPitch = kCqrMaxL + 1;
template <int TPR>
__host__ __device__ constexpr int solve_rows() { return kSolveThreads / TPR; }
template <int TPR>
constexpr size_t solve_smem() {
  return sizeof(double) * ((size_t)kCqrMaxL * kCqrMaxL + (size_t)solve_rows<TPR>() * kSolveRowPitch + kCqrMaxL);
}
template <bool FROM_INPUT, bool TO_Q, int TPR, class JOBS>
__global__ void __launch_bounds__(kSolveThreads) cqr_solve_kernel(const JOBS jobs, int pass) {
  constexpr int ROWS = solve_rows<TPR>();
  const CqrJob job = job_at(jobs, blockIdx.y);
  const int l = job.l;
  const int64_t r0 = (int64_t)blockIdx.x * ROWS;
  if (r0 >= job.m) return;
  extern __shared__ double csm[];
  double* Rs = csm;
  double(*X)[kSolveRowPitch] = reinterpret_cast<double(*)[kSolveRowPitch]>(csm + kCqrMaxL * kCqrMaxL);
  double* invd = csm + kCqrMaxL * kCqrMaxL + ROWS * kSolveRowPitch;
  const int tid = threadIdx.x;
  const double* Rg = job.Rk + (size_t)pass * l * l;
  const int ll = l * l;
  for (int e = tid; e < ll; e += 4 * kSolveThreads) {
    double v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = (e + kSolveThreads * q < ll) ? Rg[e + kSolveThreads * q] : 0.0;
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (e + kSolveThreads * q < ll) Rs[e + kSolveThreads * q] = v[q];
  }
  const int rows = (int)((job.m - r0) < ROWS ? (job.m - r0) : ROWS);
  for (int e = tid; e < ROWS * l; e += kSolveThreads) {
    const int rr = e % ROWS, j = e / ROWS;
    double v = 0.0;
    if (rr < rows) {
      const int64_t idx = r0 + rr + job.m * j;
      if (FROM_INPUT)
        v = job.Y64 ? job.Y64[idx] : (double)job.Y[idx];
      else
        v = job.W[idx];
    }
    X[rr][j] = v;
  }
  __syncthreads();
  for (int j = tid; j < l; j += kSolveThreads) invd[j] = 1.0 / Rs[j + l * j];
  __syncthreads();
  const unsigned long long refill = *job.defmask;
  const int row = tid / TPR, sub = tid % TPR;
  double* x = X[row];
  for (int j = 0; j < l; ++j) {
    const double* rc = Rs + (size_t)l * j;
    double a0 = 0.0, a1 = 0.0;
    int k = sub;
    for (; k + TPR < j; k += 2 * TPR) {
      a0 = fma(x[k], rc[k], a0);
      a1 = fma(x[k + TPR], rc[k + TPR], a1);
    }
    if (k < j) a0 = fma(x[k], rc[k], a0);
    double acc = a0 + a1;
#pragma unroll
    for (int o = 1; o < TPR; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (sub == 0)
      x[j] = ((refill >> j) & 1ull) ? refill_value(r0 + row, j) : (x[j] - acc) * invd[j];
    __syncwarp();
  }
  __syncthreads();
  double* out = TO_Q ? job.Q : job.W;
  for (int e = tid; e < ROWS * l; e += kSolveThreads) {
    const int rr = e % ROWS, j = e / ROWS;
    if (rr < rows) out[r0 + rr + job.m * j] = X[rr][j];
  }
}

// Lanes per row: as many as keep the warps within one per sub-partition.
int solve_tpr(int64_t total_rows) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    sms = 1;
  const int64_t parts = 4 * (int64_t)std::max(1, sms);
  return (total_rows * 8 / 32 <= parts) ? 8 : 4;
}

template <int TPR, class JOBS>
void cqr_solve_launch(const JOBS& batch, int nq, int64_t maxm, int pass, cudaStream_t st) {
  const dim3 gs((unsigned)((maxm + solve_rows<TPR>() - 1) / solve_rows<TPR>()), (unsigned)nq);
  const size_t sm = solve_smem<TPR>();
  auto run = [&](auto kern) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    kern<<<gs, kSolveThreads, sm, st>>>(batch, pass);
  };
  if (pass == 0)
    run(cqr_solve_kernel<true, false, TPR, JOBS>);
  else if (pass == 1)
    run(cqr_solve_kernel<false, false, TPR, JOBS>);
  else
    run(cqr_solve_kernel<false, true, TPR, JOBS>);
}
template <class JOBS>
void cqr_solve_any(const JOBS& batch, int nq, int64_t maxm, int64_t total_rows, int pass,
                   cudaStream_t st) {
  if (solve_tpr(total_rows) == 8)
    cqr_solve_launch<8>(batch, nq, maxm, pass, st);
  else
    cqr_solve_launch<4>(batch, nq, maxm, pass, st);
}

int grid_for(int64_t n, int threads, int cap = 8192) {
  int64_t g = (n + threads - 1) / threads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, cap));
}

}  // namespace

void cholqr3_launch(const CqrBatch& batch, int nq, int64_t maxm, int* status);

// Shifted CholeskyQR3 of one m x l FP32 matrix on an explicit stream, with
// every scratch buffer taken from `scratch` (m*l + 4*l*l + 2 doubles): the
// working matrix, the Gram accumulator, the three pass factors, the refill
// mask and a status word.  Allocates nothing and copies nothing from the host.
cudaError_t cholqr3_single_on_stream(const float* Y, int64_t m, int l, double* Q, double* R,
                                     double* scratch, cudaStream_t st) {
  CqrBatch batch{};
  CqrJob& q = batch.job[0];
  q.Y = Y;
  q.Y64 = nullptr;
  q.Q = Q;
  q.R = R;
  q.m = m;
  q.l = l;
  q.W = scratch;
  q.G = scratch + (size_t)m * l;
  q.Rk = q.G + (size_t)l * l;
  q.defmask = reinterpret_cast<unsigned long long*>(q.Rk + (size_t)3 * l * l);
  int* status = reinterpret_cast<int*>(q.Rk + (size_t)3 * l * l + 1);
  const dim3 g((unsigned)((m + kCqrRows - 1) / kCqrRows), 1u);
  for (int pass = 0; pass < 3; ++pass) {
    cudaError_t e = cudaMemsetAsync(q.G, 0, sizeof(double) * l * l, st);
    if (e != cudaSuccess) return e;
    if (pass == 0)
      cqr_gram_kernel<true><<<g, 256, 0, st>>>(batch, status);
    else
      cqr_gram_kernel<false><<<g, 256, 0, st>>>(batch, status);
    cqr_chol_kernel<<<1, kCholThreads, 0, st>>>(batch, pass);
    cqr_solve_any(batch, 1, m, m, pass, st);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

void qr_householder_f64(const QrJob* jobs, int count, int* status) {
  if (count <= 0) return;
  for (int b = 0; b < count; ++b) {
    KRP_REQUIRE(jobs[b].m >= jobs[b].l && jobs[b].l >= 1, "QR needs m >= l >= 1 (m=%lld l=%d)",
                (long long)jobs[b].m, jobs[b].l);
    KRP_REQUIRE(jobs[b].l <= kQrMaxL, "QR supports l <= %d", kQrMaxL);
  }
  Ctx* c = current();
  // narrow sketches (l <= 64): shifted CholeskyQR3 over many SMs; wider ones:
  // one-CTA Householder
  std::vector<QrJob> hh;
  std::vector<CqrJob> cq;
  int64_t maxm = 0;
  for (int b = 0; b < count; ++b) {
    const QrJob& j = jobs[b];
    if (j.l > kCqrMaxL) {
      hh.push_back(j);
      continue;
    }
    CqrJob q{};
    q.Y = j.Y;
    q.Y64 = j.Y64;
    q.W = j.work;
    q.Q = j.Q;
    q.R = j.R;
    q.m = j.m;
    q.l = j.l;
    q.G = c->ws.take<double>((size_t)j.l * j.l);
    q.Rk = c->ws.take<double>((size_t)3 * j.l * j.l);
    q.defmask = c->ws.take<unsigned long long>(1);
    cq.push_back(q);
    maxm = std::max<int64_t>(maxm, j.m);
  }
  if (!hh.empty()) {
    QrJob* d_jobs = c->ws.take<QrJob>(hh.size());
    KRP_CUDA_CHECK(cudaMemcpyAsync(d_jobs, hh.data(), sizeof(QrJob) * hh.size(),
                                   cudaMemcpyHostToDevice, stream()));
    qr_kernel<<<(int)hh.size(), kQrThreads, 0, stream()>>>(d_jobs, status);
    check_launch("qr_householder_f64");
  }
  for (size_t b0 = 0; b0 < cq.size(); b0 += kCqrMaxBatch) {
    const int nq = (int)std::min<size_t>(kCqrMaxBatch, cq.size() - b0);
    CqrBatch batch{};
    int64_t bm = 0;
    for (int q = 0; q < nq; ++q) {
      batch.job[q] = cq[b0 + q];
      bm = std::max<int64_t>(bm, cq[b0 + q].m);
    }
    cholqr3_launch(batch, nq, bm, status);
  }
  (void)maxm;
}

void cholqr3_launch(const CqrBatch& batch, int nq, int64_t maxm, int* status) {
  const dim3 g((unsigned)((maxm + kCqrRows - 1) / kCqrRows), (unsigned)nq);
  int64_t total_rows = 0;
  for (int q = 0; q < nq; ++q) total_rows += batch.job[q].m;
  for (int pass = 0; pass < 3; ++pass) {
    for (int q = 0; q < nq; ++q)
      KRP_CUDA_CHECK(cudaMemsetAsync(batch.job[q].G, 0, sizeof(double) * batch.job[q].l * batch.job[q].l,
                                     stream()));
    if (pass == 0)
      cqr_gram_kernel<true><<<g, 256, 0, stream()>>>(batch, status);
    else
      cqr_gram_kernel<false><<<g, 256, 0, stream()>>>(batch, status);
    check_launch("cholqr_gram_f64");
    cqr_chol_kernel<<<nq, kCholThreads, 0, stream()>>>(batch, pass);
    check_launch("cholqr_chol_f64");
    cqr_solve_any(batch, nq, maxm, total_rows, pass, stream());
    check_launch("cholqr_solve_f64");
  }
}

// Shifted CholeskyQR3 of many small jobs in one set of launches (device job
// array): layout of the caller's device block is [CqrJob x count][G: sum l^2]
// [Rk: sum 3 l^2][defmask x count]; every job has l <= 64.
size_t cholqr3_jobs_bytes(const QrJob* jobs, int count) {
  size_t d = 0;
  for (int b = 0; b < count; ++b) d += 4 * (size_t)jobs[b].l * jobs[b].l;
  return ((sizeof(CqrJob) * count + 255) & ~size_t(255)) + sizeof(double) * d +
         sizeof(unsigned long long) * count + 256;
}

CqrJobsPlan cholqr3_jobs_setup(const QrJob* jobs, int count, void* dmem, cudaStream_t st) {
  CqrJobsPlan pl{};
  pl.count = count;
  pl.d_jobs = dmem;
  char* p = static_cast<char*>(dmem) + ((sizeof(CqrJob) * count + 255) & ~size_t(255));
  double* g = reinterpret_cast<double*>(p);
  size_t gsum = 0;
  for (int b = 0; b < count; ++b) gsum += (size_t)jobs[b].l * jobs[b].l;
  double* rk = g + gsum;
  size_t rsum = 0;
  for (int b = 0; b < count; ++b) rsum += 3 * (size_t)jobs[b].l * jobs[b].l;
  unsigned long long* mask = reinterpret_cast<unsigned long long*>(rk + rsum);
  std::vector<CqrJob> h(count);
  size_t go = 0, ro = 0;
  for (int b = 0; b < count; ++b) {
    const QrJob& j = jobs[b];
    KRP_REQUIRE(j.m >= j.l && j.l >= 1 && j.l <= kCqrMaxL, "CholeskyQR3 job needs m >= l, 1 <= l <= %d",
                kCqrMaxL);
    CqrJob& q = h[b];
    q.Y = j.Y;
    q.Y64 = j.Y64;
    q.W = j.work;
    q.Q = j.Q;
    q.R = j.R;
    q.m = j.m;
    q.l = j.l;
    q.G = g + go;
    q.Rk = rk + ro;
    q.defmask = mask + b;
    go += (size_t)j.l * j.l;
    ro += 3 * (size_t)j.l * j.l;
    pl.maxm = std::max<int64_t>(pl.maxm, j.m);
    pl.total_rows += j.m;
  }
  pl.g_all = g;
  pl.g_count = gsum;
  KRP_CUDA_CHECK(cudaMemcpyAsync(dmem, h.data(), sizeof(CqrJob) * count, cudaMemcpyHostToDevice, st));
  return pl;
}

int cholqr3_jobs_launch(const CqrJobsPlan& pl, int* status) {
  const CqrJobArray jobs{static_cast<const CqrJob*>(pl.d_jobs)};
  const dim3 g((unsigned)((pl.maxm + kCqrRows - 1) / kCqrRows), (unsigned)pl.count);
  for (int pass = 0; pass < 3; ++pass) {
    KRP_CUDA_CHECK(cudaMemsetAsync(pl.g_all, 0, sizeof(double) * pl.g_count, stream()));
    if (pass == 0)
      cqr_gram_kernel<true><<<g, 256, 0, stream()>>>(jobs, status);
    else
      cqr_gram_kernel<false><<<g, 256, 0, stream()>>>(jobs, status);
    check_launch("cholqr_jobs_gram_f64");
    cqr_chol_kernel<<<pl.count, kCholThreads, 0, stream()>>>(jobs, pass);
    check_launch("cholqr_jobs_chol_f64");
    cqr_solve_any(jobs, pl.count, pl.maxm, pl.total_rows, pass, stream());
    check_launch("cholqr_jobs_solve_f64");
  }
  return 9;
}

void gram_modes_f64(const double* G, int D, const int64_t* dims, double* const* S) {
  GramModes M{};
  M.G = G;
  int64_t total = 1;
  for (int j = 0; j < D; ++j) total *= dims[j];
  const int want = std::max(1, current()->num_sms / D);  // CTAs per mode
  int64_t maxblocks = 1;
  for (int n = 0; n < D; ++n) {
    KRP_REQUIRE(dims[n] <= kEigMaxL, "core truncation supports ranks l <= %d", kEigMaxL);
    int64_t P = 1;
    for (int j = 0; j < n; ++j) P *= dims[j];
    M.S[n] = S[n];
    M.P[n] = P;
    M.l[n] = dims[n];
    M.ncols[n] = total / dims[n];
    M.per[n] = std::max<int64_t>(8, (M.ncols[n] + want - 1) / want);
    maxblocks = std::max<int64_t>(maxblocks, (M.ncols[n] + M.per[n] - 1) / M.per[n]);
    KRP_CUDA_CHECK(cudaMemsetAsync(S[n], 0, sizeof(double) * dims[n] * dims[n], stream()));
  }
  gram_modes_kernel<<<dim3((unsigned)maxblocks, (unsigned)D), 256, 0, stream()>>>(M);
  check_launch("gram_modes_f64");
}

void gram_mode_f64(const double* G, int D, const int64_t* dims, int mode, double* S) {
  int64_t P = 1, Sfx = 1;
  for (int j = 0; j < mode; ++j) P *= dims[j];
  for (int j = mode + 1; j < D; ++j) Sfx *= dims[j];
  const int64_t l = dims[mode];
  const int64_t ncols = P * Sfx;
  KRP_REQUIRE(l <= kEigMaxL, "core truncation supports ranks l <= %d", kEigMaxL);
  KRP_CUDA_CHECK(cudaMemsetAsync(S, 0, sizeof(double) * l * l, stream()));
  const int threads = 256;
  const int want = 2 * current()->num_sms;
  int64_t per = std::max<int64_t>(32, (ncols + want - 1) / want);
  const int blocks = (int)((ncols + per - 1) / per);
  gram_kernel<<<blocks, threads, sizeof(double) * 32 * l, stream()>>>(G, P, l, ncols, per, S);
  check_launch("gram_f64");
}

template <int ML>
void eig_split_launch_t(const EigJob* d_jobs, int count, double* scratch, int* status) {
  const size_t js = 3 * sizeof(float) * ML * (ML + 1);
  KRP_CUDA_CHECK(cudaFuncSetAttribute(eig_jacobi_kernel<ML>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)js));
  eig_jacobi_kernel<ML><<<count, kJacobiThreads, js, stream()>>>(d_jobs, scratch, status);
  check_launch("jacobi32_eig");
  const size_t rs = 3 * sizeof(double) * ML * (ML + 1);
  KRP_CUDA_CHECK(cudaFuncSetAttribute(eig_refine_kernel<ML>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)rs));
  eig_refine_kernel<ML><<<dim3(kEigCluster, count), kEigThreads, rs, stream()>>>(d_jobs, scratch, status);
  check_launch("eig_refine_f64");
}

void eig_launch(const EigJob* d_jobs, int count, int maxl, int* status) {
  if (count <= 0) return;
  KRP_REQUIRE(maxl >= 1 && maxl <= kEigMaxL, "eigensolver needs l <= %d", kEigMaxL);
  if (maxl <= 32) {
    const size_t smem = 5 * sizeof(double) * 32 * 33;
    KRP_CUDA_CHECK(cudaFuncSetAttribute(eig_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem));
    eig_kernel<32><<<count, kEigThreads, smem, stream()>>>(d_jobs, status);
  } else {
    const size_t smem = 5 * sizeof(double) * kEigMaxL * (kEigMaxL + 1);
    KRP_CUDA_CHECK(cudaFuncSetAttribute(eig_kernel<kEigMaxL>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    eig_kernel<kEigMaxL><<<count, kEigThreads, smem, stream()>>>(d_jobs, status);
  }
  check_launch("jacobi_eig_f64");
}

void qr_householder_launch(const QrJob* d_jobs, int count, int* status) {
  if (count <= 0) return;
  qr_kernel<<<count, kQrThreads, 0, stream()>>>(d_jobs, status);
  check_launch("qr_householder_f64");
}

void sym_eig_top_f64(const double* const* S, const int* l, const int* r, double* const* U,
                     int count, int* status, double* const* evals) {
  if (count <= 0) return;
  std::vector<EigJob> jobs(count);
  for (int b = 0; b < count; ++b) {
    KRP_REQUIRE(l[b] >= 1 && l[b] <= kEigMaxL && r[b] >= 1 && r[b] <= l[b],
                "eigensolver needs 1 <= r <= l <= %d", kEigMaxL);
    jobs[b] = EigJob{S[b], U[b], evals ? evals[b] : nullptr, l[b], r[b]};
  }
  EigJob* d_jobs = current()->ws.take<EigJob>(count);
  KRP_CUDA_CHECK(cudaMemcpyAsync(d_jobs, jobs.data(), sizeof(EigJob) * count,
                                 cudaMemcpyHostToDevice, stream()));
  int maxl = 1;
  for (int b = 0; b < count; ++b) maxl = std::max(maxl, l[b]);
  // a few problems: Jacobi per CTA, refinement spread over a cluster each
  if ((int64_t)count * kEigCluster <= current()->num_sms && maxl > 16) {
    double* scratch = current()->ws.take<double>((size_t)count * kEigScratch);
    if (maxl <= 32)
      eig_split_launch_t<32>(d_jobs, count, scratch, status);
    else
      eig_split_launch_t<kEigMaxL>(d_jobs, count, scratch, status);
    return;
  }
  eig_launch(d_jobs, count, maxl, status);
}

size_t sym_eig_workspace_bytes(int count) {
  return ws_bytes((size_t)count, sizeof(EigJob)) + ws_bytes((size_t)count * kEigScratch, 8);
}

void ttm_small_f64(const double* G, int D, const int64_t* dims, int mode, const double* U, int r,
                   double* out) {
  int64_t P = 1, Sfx = 1;
  for (int j = 0; j < mode; ++j) P *= dims[j];
  for (int j = mode + 1; j < D; ++j) Sfx *= dims[j];
  const int64_t total = P * r * Sfx;
  if (total <= 0) return;
  ttm_small_kernel<<<grid_for(total, 256), 256, 0, stream()>>>(G, P, dims[mode], Sfx, U, r, out);
  check_launch("ttm_small_f64");
}

void matmul_f64(const double* A, const double* B, double* C, int64_t m, int k, int n) {
  if (m * n <= 0) return;
  matmul_kernel<<<grid_for(m * n, 256), 256, 0, stream()>>>(A, B, C, m, k, n);
  check_launch("matmul_f64");
}

double sum_squares_f64_sync(const double* x, int64_t n, double* scratch) {
  KRP_CUDA_CHECK(cudaMemsetAsync(scratch, 0, sizeof(double), stream()));
  if (n > 0) {
    sumsq_kernel<<<grid_for(n, 256, 1024), 256, 0, stream()>>>(x, n, scratch);
    check_launch("sumsq_f64");
  }
  double h = 0.0;
  KRP_CUDA_CHECK(cudaMemcpyAsync(&h, scratch, sizeof(double), cudaMemcpyDeviceToHost, stream()));
  KRP_CUDA_CHECK(cudaStreamSynchronize(stream()));
  return h;
}

void check_finite_f64(const double* x, int64_t n, int* status) {
  if (n <= 0) return;
  finite_kernel<<<grid_for(n, 256, 1024), 256, 0, stream()>>>(x, n, status);
  check_launch("finite_f64");
}

}  // namespace krp
