// a11: many small, uneven 3-way tensors in one launch per phase.
//
// RHOSVD-KRP-MEMO (Alg. 7 with one factor set, Sec. 5.1) of every tensor of a
// batch.  Each phase is one kernel launch over the whole batch:
//   factors     one Philox launch over all (tensor, mode) factors, then
//               row-major FP32 (and, for BF16, k-major BF16) copies
//   sketch      persistent kernel whose warps take work units from an atomic
//               counter: a row unit (32 rows i, a range of mode-3 slabs X_t)
//               forms A_t = X_t Om2 and accumulates Y1 += A_t diag(Om3[t,:])
//               and Y3[t,:] = colsum(Om1 * A_t); a column unit (32 columns j)
//               forms B_t = X_t^T Om1 and accumulates Y2 += B_t diag(Om3[t,:])
//               (the dimension tree of Sec. 5.1, 4 N l flops)
//   QR          one CTA per (tensor, mode), FP64 Householder
//   core        persistent kernel, one slab per warp unit: C_t = Q1^T X_t Q2,
//               then G(:,:,c) = sum_t C_t Q3[t,c] in a per-tensor kernel
//   truncation  FP64 Gram matrices of the core unfoldings, the eigensolver
//               on all 3 x count of them, then G x {U_i^T}, Q_i U_i
//   residual    persistent kernel over (tensor, slab range) tiles, one warp per
//               (slab, 32 rows): ||X_t - F1 M_t F2^T||^2 with FP64 sums per tensor
// Units and tiles are ordered by work (largest first).  The slabs per sketch
// unit are picked once per batch by timing the sketch phase for a few
// candidates.  The whole sequence is captured in a CUDA graph when the batch
// is first seen; a repeated call with the same descriptors replays the graph.
// FP32 X: products on CUDA cores (FFMA).  BF16 X: the sketch and core
// contractions on warp-level tensor-core MMAs (m16n8k16, FP32 accumulators);
// the residual stays on CUDA cores.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "pipeline.h"

namespace krp {
namespace {

constexpr int kBT = 256;              // threads of the slab kernels
constexpr int kMaxSide = 256;         // n_i
constexpr int kMaxEll = 32;           // l_i

struct TbItem {
  const void* X;
  int n[3];
  int l[3];
  int lm;            // memo factor width: max l_i
  int r[3];          // output sizes (r_i with truncation, l_i without)
  float* om[3];      // n_i x lm
  float* orow[3];    // n_i x 4 ceil(lm / 4), row-major FP32 copy of om
  float* qrow[3];    // n_i x 4 ceil(l_i / 4), row-major FP32 copy of Q
  // BF16 form only (null otherwise): k-major BF16 tables for the warp MMAs,
  // ot[m][k * np16[m] + i] = Omega_m[i, k] (m < 2; k < 8 ceil(lm / 8)), and
  // q2t[p][k * np16[1] + j], p = 0, 1, 2: Q2 = hi + mid + lo (k < 8 ceil(l2 / 8));
  // zero outside the matrix.
  __nv_bfloat16* ot[2];
  __nv_bfloat16* q2t;
  __nv_bfloat16* q1t;  // q1t[p][a * np16[0] + i] = part p of Q1[i, a], a < 32
  int np16[2];       // n1, n2 rounded up to 16
  float* Y[3];       // n_i x lm
  double* Q[3];      // n_i x l_i
  float* C;          // n3 slab cores, l1 x l2 each
  float* G;          // l1 l2 l3
  double* T1;        // r1 l2 l3 (truncation scratch)
  double* T2;        // r1 r2 l3
  double* S[3];      // l_i x l_i
  double* U[3];      // l_i x r_i
  float* core_out;   // r1 r2 r3
  double* fac_out[3];
  double* acc;       // ||X - X_hat||^2, ||X||^2
  float* M;          // n3 x (r1 r2): the slab matrices of the residual
};

struct TbTile {
  int item, t0, t1, pad;
};

template <class XT>
__device__ __forceinline__ float ldx(const XT* p, int64_t i);
template <>
__device__ __forceinline__ float ldx<float>(const float* p, int64_t i) { return p[i]; }
template <>
__device__ __forceinline__ float ldx<__nv_bfloat16>(const __nv_bfloat16* p, int64_t i) {
  return __bfloat162float(p[i]);
}

__device__ int next_tile(int* counter, int* s_tile) {
  __syncthreads();  // everyone is done with the previous tile's shared memory
  if (threadIdx.x == 0) *s_tile = atomicAdd(counter, 1);
  __syncthreads();
  return *s_tile;
}

// Warp-level work units of the sketch and core kernels, handed out by an
// atomic counter (one per warp, no barrier across the CTA).
struct SkUnit {
  int item;
  int kb;      // kind << 16 | block: kind 0 = rows (block of 32 i), 1 = columns (block of 32 j)
  int t0, t1;  // slabs t0 .. t1-1
};
constexpr int kUnitCols = 1 << 16;

__device__ __forceinline__ int warp_next(int* counter, int lane) {
  int u = 0;
  if (lane == 0) u = atomicAdd(counter, 1);
  return __shfl_sync(0xffffffffu, u, 0);
}

// Reduce-scatter of CNT (a power of two <= 32) per-lane values: returns the
// warp's total of value (lane % CNT).  Each halving step exchanges half of
// the values with the lane h apart and keeps the half selected by that lane
// bit (CNT - 1 shuffles), then lanes that share lane % CNT are summed.
template <int CNT>
__device__ __forceinline__ float reduce_scatter(float (&v)[CNT], int lane) {
#pragma unroll
  for (int h = CNT / 2; h >= 1; h >>= 1) {
    const bool upper = lane & h;
#pragma unroll
    for (int q = 0; q < h; ++q) {
      const float send = upper ? v[q] : v[q + h];
      const float keep = upper ? v[q + h] : v[q];
      v[q] = keep + __shfl_xor_sync(0xffffffffu, send, h);
    }
  }
  float r = v[0];
#pragma unroll
  for (int o = CNT; o < 32; o <<= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
  return r;
}

__device__ __forceinline__ void fma4(float* acc, float x, const float4& w) {
  acc[0] = fmaf(x, w.x, acc[0]);
  acc[1] = fmaf(x, w.y, acc[1]);
  acc[2] = fmaf(x, w.z, acc[2]);
  acc[3] = fmaf(x, w.w, acc[3]);
}

// ---------------------------------------------------------------- sketch ----
// All three mode sketches of the memoized tree (Sec. 5.1) from the slabs
// X_t = X[:, :, t] (n1 x n2, i fastest), FP32 on CUDA cores, as two kinds of
// warp units over the same slabs (one launch; a tensor's row and column
// units are adjacent in the unit list, so the second read of a slab is
// served by L2):
//   row unit (32 rows i, lane = row; slabs t0..t1-1):
//     A_t[i, :] = sum_j X[i, j, t] Om2[j, :]   (X straight from global memory,
//                 coalesced over the lanes, 16 columns in flight; Om2 rows broadcast)
//     Y1[i, :] += A_t[i, :] * Om3[t, :]        (registers across the unit's slabs)
//     Y3[t, :] += sum_i Om1[i, :] * A_t[i, :]  (warp reduce-scatter, then atomics)
//   column unit (32 columns j, lane = column):
//     B_t[j, :] = sum_i X[i, j, t] Om1[i, :]   (32 x 32 blocks of X transposed
//                 through the warp's shared buffer; Om1 rows broadcast)
//     Y2[j, :] += B_t[j, :] * Om3[t, :]        (registers across the unit's slabs)
// Factor rows come from the row-major FP32 tables orow[m] (LP = 4 LQ columns,
// zero beyond l).  Every Y_n is zeroed before the launch and receives atomics.
template <class XT, int LQ>
__device__ void sketch_rows_unit(const TbItem& it, const SkUnit& u, int lane) {
  constexpr int LP = 4 * LQ;
  constexpr int CNT = LP <= 16 ? 16 : 32;
  constexpr int NC = LQ <= 4 ? 16 : 8;
  const int n1 = it.n[0], n2 = it.n[1], n3 = it.n[2], lm = it.lm;
  const int i = 32 * (u.kb & (kUnitCols - 1)) + lane;
  const bool valid = i < n1;
  const float4* o2 = reinterpret_cast<const float4*>(it.orow[1]);
  const float4* o3 = reinterpret_cast<const float4*>(it.orow[2]);
  const float4* o1 = reinterpret_cast<const float4*>(it.orow[0] + (size_t)(valid ? i : 0) * LP);
  const XT* X = static_cast<const XT*>(it.X);
  float y1[LP];
#pragma unroll
  for (int k = 0; k < LP; ++k) y1[k] = 0.f;
  for (int t = u.t0; t < u.t1; ++t) {
    float a[LP];
#pragma unroll
    for (int k = 0; k < LP; ++k) a[k] = 0.f;
    const XT* xp = X + (int64_t)n1 * n2 * t + (valid ? i : 0);
    int j = 0;
    for (; j + NC <= n2; j += NC) {
      float xv[NC];
      const XT* xj = xp + (int64_t)n1 * j;
#pragma unroll
      for (int c = 0; c < NC; ++c) xv[c] = valid ? ldx(xj, n1 * c) : 0.f;
#pragma unroll
      for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int q = 0; q < LQ; ++q) fma4(&a[4 * q], xv[c], __ldg(o2 + (j + c) * LQ + q));
    }
    for (; j < n2; ++j) {
      const float x = valid ? ldx(xp, (int64_t)n1 * j) : 0.f;
#pragma unroll
      for (int q = 0; q < LQ; ++q) fma4(&a[4 * q], x, __ldg(o2 + j * LQ + q));
    }
    float v[CNT];
#pragma unroll
    for (int q = 0; q < LQ; ++q) {
      const float4 w3 = __ldg(o3 + t * LQ + q);
      const float4 w1 = valid ? __ldg(o1 + q) : make_float4(0.f, 0.f, 0.f, 0.f);
      y1[4 * q + 0] = fmaf(a[4 * q + 0], w3.x, y1[4 * q + 0]);
      y1[4 * q + 1] = fmaf(a[4 * q + 1], w3.y, y1[4 * q + 1]);
      y1[4 * q + 2] = fmaf(a[4 * q + 2], w3.z, y1[4 * q + 2]);
      y1[4 * q + 3] = fmaf(a[4 * q + 3], w3.w, y1[4 * q + 3]);
      v[4 * q + 0] = a[4 * q + 0] * w1.x;
      v[4 * q + 1] = a[4 * q + 1] * w1.y;
      v[4 * q + 2] = a[4 * q + 2] * w1.z;
      v[4 * q + 3] = a[4 * q + 3] * w1.w;
    }
#pragma unroll
    for (int k = LP; k < CNT; ++k) v[k] = 0.f;
    const float s3 = reduce_scatter<CNT>(v, lane);
    if (lane < CNT && lane < lm) atomicAdd(&it.Y[2][t + (int64_t)n3 * lane], s3);
  }
  if (valid) {
#pragma unroll
    for (int k = 0; k < LP; ++k)
      if (k < lm) atomicAdd(&it.Y[0][i + (int64_t)n1 * k], y1[k]);
  }
}

template <class XT, int LQ>
__device__ void sketch_cols_unit(const TbItem& it, const SkUnit& u, int lane, float* Xw) {
  constexpr int LP = 4 * LQ;
  constexpr int NC = LQ <= 4 ? 16 : 8;  // columns loaded per group
  const int n1 = it.n[0], n2 = it.n[1], lm = it.lm;
  const int j0 = 32 * (u.kb & (kUnitCols - 1));
  const int jn = min(32, n2 - j0);
  const int j = j0 + lane;
  const int RB = (n1 + 31) >> 5;
  const float4* o1 = reinterpret_cast<const float4*>(it.orow[0]);
  const float4* o3 = reinterpret_cast<const float4*>(it.orow[2]);
  const XT* X = static_cast<const XT*>(it.X);
  float y2[LP];
#pragma unroll
  for (int k = 0; k < LP; ++k) y2[k] = 0.f;
  for (int t = u.t0; t < u.t1; ++t) {
    float b[LP];
#pragma unroll
    for (int k = 0; k < LP; ++k) b[k] = 0.f;
    for (int rb = 0; rb < RB; ++rb) {
      const int i = 32 * rb + lane;
      const bool vi = i < n1;
      const XT* xp = X + (int64_t)n1 * ((int64_t)n2 * t + j0) + (vi ? i : 0);
      __syncwarp();  // the previous block has been read
#pragma unroll 1
      for (int h = 0; h < 32; h += NC) {
        float xv[NC];
        const XT* xh = xp + (int64_t)n1 * h;
#pragma unroll
        for (int c = 0; c < NC; ++c) xv[c] = (vi && h + c < jn) ? ldx(xh, n1 * c) : 0.f;
#pragma unroll
        for (int c = 0; c < NC; ++c) Xw[lane * 33 + h + c] = xv[c];  // [i][j], pitch 33
      }
      __syncwarp();
      const int ni = min(32, n1 - 32 * rb);
      const float4* w = o1 + (size_t)(32 * rb) * LQ;
      for (int ii = 0; ii < ni; ++ii) {
        const float x = Xw[ii * 33 + lane];
#pragma unroll
        for (int q = 0; q < LQ; ++q) fma4(&b[4 * q], x, __ldg(w + ii * LQ + q));
      }
    }
#pragma unroll
    for (int q = 0; q < LQ; ++q) {
      const float4 w3 = __ldg(o3 + t * LQ + q);
      y2[4 * q + 0] = fmaf(b[4 * q + 0], w3.x, y2[4 * q + 0]);
      y2[4 * q + 1] = fmaf(b[4 * q + 1], w3.y, y2[4 * q + 1]);
      y2[4 * q + 2] = fmaf(b[4 * q + 2], w3.z, y2[4 * q + 2]);
      y2[4 * q + 3] = fmaf(b[4 * q + 3], w3.w, y2[4 * q + 3]);
    }
  }
  if (lane < jn) {
#pragma unroll
    for (int k = 0; k < LP; ++k)
      if (k < lm) atomicAdd(&it.Y[1][j + (int64_t)n2 * k], y2[k]);
  }
}

// ------------------------------------------------ BF16 form: warp MMAs ----
// For BF16 X the two contractions of the sketch and the first one of the core
// run on the tensor cores as warp-level mma.sync m16n8k16 (BF16 operands,
// FP32 accumulators): the products of BF16 X with the BF16 factors (and with
// the three BF16 parts of Q2) are exact, so the sums are the CUDA-core sums
// up to order.  The units are the same as above (32 rows or columns, slabs
// t0..t1-1); A fragments are gathered straight from global memory (two 16-bit
// loads per register, zero outside the slab), B fragments are 32-bit loads
// from the k-major tables ot / q2t.
// Fragment layout (g = lane / 4, q = lane % 4; lower half of a register =
// lower k): A regs {A[g][2q..2q+1]}, {A[g+8][2q..]}, {A[g][2q+8..]},
// {A[g+8][2q+8..]}; B regs {B[2q..2q+1][g]}, {B[2q+8..2q+9][g]}; D
// {D[g][2q]}, {D[g][2q+1]}, {D[g+8][2q]}, {D[g+8][2q+1]}.
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t ldb16(const __nv_bfloat16* p, bool ok) {
  return ok ? (uint32_t)__ldg(reinterpret_cast<const unsigned short*>(p)) : 0u;
}

// rows unit of the sketch (see sketch_rows_unit), NT = ceil(lm / 8) n-tiles:
// D = A_t for the unit's 32 rows (two m-tiles) x 8 NT columns
template <int NT>
__device__ void sketch_rows_tc(const TbItem& it, const SkUnit& u, int lane) {
  const int g = lane >> 2, q = lane & 3;
  const int n1 = it.n[0], n2 = it.n[1], n3 = it.n[2], lm = it.lm;
  const int lp = 4 * ((lm + 3) / 4);
  const int i0 = 32 * (u.kb & (kUnitCols - 1));
  const int n2p = it.np16[1];
  const uint32_t* o2t = reinterpret_cast<const uint32_t*>(it.ot[1]);
  const __nv_bfloat16* X = static_cast<const __nv_bfloat16*>(it.X);
  int rr[2][2];
  bool rv[2][2];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      rr[mt][h] = i0 + 16 * mt + g + 8 * h;
      rv[mt][h] = rr[mt][h] < n1;
    }
  float w1[2][NT][4], y1[2][NT][4];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < NT; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int col = nt * 8 + 2 * q + (e & 1);
        const bool ok = rv[mt][e >> 1] && col < lm;
        w1[mt][nt][e] = ok ? it.orow[0][(size_t)rr[mt][e >> 1] * lp + col] : 0.f;
        y1[mt][nt][e] = 0.f;
      }
  for (int t = u.t0; t < u.t1; ++t) {
    float d[2][NT][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) d[mt][nt][0] = d[mt][nt][1] = d[mt][nt][2] = d[mt][nt][3] = 0.f;
    const __nv_bfloat16* xt = X + (int64_t)n1 * n2 * t;
    for (int j0 = 0; j0 < n2; j0 += 16) {
      uint32_t a[2][4];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int h = r & 1, j = j0 + 2 * q + 8 * (r >> 1);
          const bool ok = rv[mt][h];
          const __nv_bfloat16* p = xt + (ok ? rr[mt][h] : 0) + (int64_t)n1 * j;
          a[mt][r] = ldb16(p, ok && j < n2) | (ldb16(p + n1, ok && j + 1 < n2) << 16);
        }
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) {
        const uint32_t* bp = o2t + (((nt * 8 + g) * n2p + j0 + 2 * q) >> 1);
        const uint32_t b0 = __ldg(bp), b1 = __ldg(bp + 4);
        mma16816(d[0][nt], a[0], b0, b1);
        mma16816(d[1][nt], a[1], b0, b1);
      }
    }
    const float* o3r = it.orow[2] + (size_t)t * lp;
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
      float s[2];
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int col = nt * 8 + 2 * q + c;
        const float o3v = col < lm ? o3r[col] : 0.f;
        float acc = 0.f;
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int e = 2 * h + c;
            y1[mt][nt][e] = fmaf(d[mt][nt][e], o3v, y1[mt][nt][e]);
            acc = fmaf(d[mt][nt][e], w1[mt][nt][e], acc);
          }
        acc += __shfl_xor_sync(0xffffffffu, acc, 4);
        acc += __shfl_xor_sync(0xffffffffu, acc, 8);
        acc += __shfl_xor_sync(0xffffffffu, acc, 16);
        s[c] = acc;
      }
      if (g == 0) {
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const int col = nt * 8 + 2 * q + c;
          if (col < lm) atomicAdd(&it.Y[2][t + (int64_t)n3 * col], s[c]);
        }
      }
    }
  }
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < NT; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int col = nt * 8 + 2 * q + (e & 1);
        if (rv[mt][e >> 1] && col < lm)
          atomicAdd(&it.Y[0][rr[mt][e >> 1] + (int64_t)n1 * col], y1[mt][nt][e]);
      }
}

// columns unit of the sketch (see sketch_cols_unit): D = B_t for the unit's
// 32 columns j (two m-tiles; A = X_t^T, K = i) x 8 NT columns
template <int NT>
__device__ void sketch_cols_tc(const TbItem& it, const SkUnit& u, int lane) {
  const int g = lane >> 2, q = lane & 3;
  const int n1 = it.n[0], n2 = it.n[1], lm = it.lm;
  const int lp = 4 * ((lm + 3) / 4);
  const int j0 = 32 * (u.kb & (kUnitCols - 1));
  const int n1p = it.np16[0];
  const uint32_t* o1t = reinterpret_cast<const uint32_t*>(it.ot[0]);
  const __nv_bfloat16* X = static_cast<const __nv_bfloat16*>(it.X);
  int cc[2][2];
  bool cv[2][2];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      cc[mt][h] = j0 + 16 * mt + g + 8 * h;
      cv[mt][h] = cc[mt][h] < n2;
    }
  float y2[2][NT][4];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) y2[mt][nt][0] = y2[mt][nt][1] = y2[mt][nt][2] = y2[mt][nt][3] = 0.f;
  for (int t = u.t0; t < u.t1; ++t) {
    float d[2][NT][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) d[mt][nt][0] = d[mt][nt][1] = d[mt][nt][2] = d[mt][nt][3] = 0.f;
    const __nv_bfloat16* xt = X + (int64_t)n1 * n2 * t;
    for (int i0 = 0; i0 < n1; i0 += 16) {
      uint32_t a[2][4];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int h = r & 1, i = i0 + 2 * q + 8 * (r >> 1);
          const bool ok = cv[mt][h];
          const __nv_bfloat16* p = xt + (int64_t)n1 * (ok ? cc[mt][h] : 0) + i;
          a[mt][r] = ldb16(p, ok && i < n1) | (ldb16(p + 1, ok && i + 1 < n1) << 16);
        }
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) {
        const uint32_t* bp = o1t + (((nt * 8 + g) * n1p + i0 + 2 * q) >> 1);
        const uint32_t b0 = __ldg(bp), b1 = __ldg(bp + 4);
        mma16816(d[0][nt], a[0], b0, b1);
        mma16816(d[1][nt], a[1], b0, b1);
      }
    }
    const float* o3r = it.orow[2] + (size_t)t * lp;
#pragma unroll
    for (int nt = 0; nt < NT; ++nt)
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int col = nt * 8 + 2 * q + c;
        const float o3v = col < lm ? o3r[col] : 0.f;
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
          for (int h = 0; h < 2; ++h)
            y2[mt][nt][2 * h + c] = fmaf(d[mt][nt][2 * h + c], o3v, y2[mt][nt][2 * h + c]);
      }
  }
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < NT; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int col = nt * 8 + 2 * q + (e & 1);
        if (cv[mt][e >> 1] && col < lm)
          atomicAdd(&it.Y[1][cc[mt][e >> 1] + (int64_t)n2 * col], y2[mt][nt][e]);
      }
}

// T[i, :] = X_t[i, :] Q2 for the 32 rows of block rb (two m-tiles) into the
// warp's buffer Tw[32][ldt] (columns < ldt), Q2 = hi + mid + lo (three MMAs)
template <int NT>
__device__ void core_rows_tc(const TbItem& it, int t, int rb, int lane, float* Tw, int ldt) {
  const int g = lane >> 2, q = lane & 3;
  const int n1 = it.n[0], n2 = it.n[1], l2 = it.l[1];
  const int n2p = it.np16[1];
  const size_t plane = (size_t)8 * NT * n2p / 2;  // uint32 per plane
  const uint32_t* q2t = reinterpret_cast<const uint32_t*>(it.q2t);
  const __nv_bfloat16* xt = static_cast<const __nv_bfloat16*>(it.X) + (int64_t)n1 * n2 * t;
  int rr[2][2];
  bool rv[2][2];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      rr[mt][h] = 32 * rb + 16 * mt + g + 8 * h;
      rv[mt][h] = rr[mt][h] < n1;
    }
  float d[2][NT][4];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) d[mt][nt][0] = d[mt][nt][1] = d[mt][nt][2] = d[mt][nt][3] = 0.f;
  for (int j0 = 0; j0 < n2; j0 += 16) {
    uint32_t a[2][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int h = r & 1, j = j0 + 2 * q + 8 * (r >> 1);
        const bool ok = rv[mt][h];
        const __nv_bfloat16* p = xt + (ok ? rr[mt][h] : 0) + (int64_t)n1 * j;
        a[mt][r] = ldb16(p, ok && j < n2) | (ldb16(p + n1, ok && j + 1 < n2) << 16);
      }
#pragma unroll
    for (int nt = 0; nt < NT; ++nt)
#pragma unroll
      for (int pl = 0; pl < 3; ++pl) {
        const uint32_t* bp = q2t + pl * plane + (((nt * 8 + g) * n2p + j0 + 2 * q) >> 1);
        const uint32_t b0 = __ldg(bp), b1 = __ldg(bp + 4);
        mma16816(d[0][nt], a[0], b0, b1);
        mma16816(d[1][nt], a[1], b0, b1);
      }
  }
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < NT; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int col = nt * 8 + 2 * q + (e & 1);
        if (col < ldt) Tw[(16 * mt + g + 8 * (e >> 1)) * ldt + col] = col < l2 ? d[mt][nt][e] : 0.f;
      }
}

__device__ __forceinline__ void split3(float x, uint32_t& h, uint32_t& m, uint32_t& l) {
  const __nv_bfloat16 bh = __float2bfloat16_rn(x);
  const float r = x - __bfloat162float(bh);
  const __nv_bfloat16 bm = __float2bfloat16_rn(r);
  const __nv_bfloat16 bl = __float2bfloat16_rn(r - __bfloat162float(bm));
  h = __bfloat16_as_ushort(bh);
  m = __bfloat16_as_ushort(bm);
  l = __bfloat16_as_ushort(bl);
}

// Core unit of the BF16 form: C_t = Q1^T X_t Q2 for one slab, both
// contractions on the tensor cores.  Per block of 32 rows i, T = X_t Q2
// (core_rows_tc) goes to the warp's buffer; then C_t += Q1[block]^T T with
// M = a (two m-tiles), K = i, N = b, Q1 and T each split into BF16 hi + mid +
// lo and the six products above 2^-24 accumulated (FP32 accuracy).  NT =
// ceil(l2 / 8).
template <int NT>
__device__ void core_unit_tc(const TbItem& it, int t, int lane, float* Tw) {
  constexpr int LDT = 8 * NT;
  const int g = lane >> 2, q = lane & 3;
  const int n1 = it.n[0], l1 = it.l[0], l2 = it.l[1];
  const int n1p = it.np16[0];
  const size_t plane = (size_t)32 * n1p / 2;  // uint32 per part of q1t
  const uint32_t* q1t = reinterpret_cast<const uint32_t*>(it.q1t);
  float c[2][NT][4];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) c[mt][nt][0] = c[mt][nt][1] = c[mt][nt][2] = c[mt][nt][3] = 0.f;
  const int RB = (n1 + 31) >> 5;
  for (int rb = 0; rb < RB; ++rb) {
    __syncwarp();  // the previous block's T has been read
    core_rows_tc<NT>(it, t, rb, lane, Tw, LDT);
    __syncwarp();
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
      const int ib = 32 * rb + 16 * ks;  // first row i of this K step
      if (ib >= n1) break;
      uint32_t a[3][2][4];
#pragma unroll
      for (int pl = 0; pl < 3; ++pl)
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const int row = 16 * mt + g + 8 * (r & 1), k = ib + 2 * q + 8 * (r >> 1);
            a[pl][mt][r] = __ldg(q1t + pl * plane + (((size_t)row * n1p + k) >> 1));
          }
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) {
        uint32_t bh[2], bm[2], bl[2];
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
          uint32_t h0, m0, l0, h1, m1, l1_;
          const float* tp = Tw + (16 * ks + 2 * q + 8 * kk) * LDT + nt * 8 + g;
          split3(tp[0], h0, m0, l0);
          split3(tp[LDT], h1, m1, l1_);
          bh[kk] = h0 | (h1 << 16);
          bm[kk] = m0 | (m1 << 16);
          bl[kk] = l0 | (l1_ << 16);
        }
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
          mma16816(c[mt][nt], a[0][mt], bh[0], bh[1]);
          mma16816(c[mt][nt], a[0][mt], bm[0], bm[1]);
          mma16816(c[mt][nt], a[1][mt], bh[0], bh[1]);
          mma16816(c[mt][nt], a[0][mt], bl[0], bl[1]);
          mma16816(c[mt][nt], a[2][mt], bh[0], bh[1]);
          mma16816(c[mt][nt], a[1][mt], bm[0], bm[1]);
        }
      }
    }
  }
  float* Ct = it.C + (int64_t)t * l1 * l2;
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < NT; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int a = 16 * mt + g + 8 * (e >> 1), b = nt * 8 + 2 * q + (e & 1);
        if (a < l1 && b < l2) Ct[a + l1 * b] = c[mt][nt][e];
      }
}

template <class XT, int LQ>
__device__ __forceinline__ void sketch_unit(const TbItem& it, const SkUnit& u, int lane, float* Xw) {
  if (u.kb >= kUnitCols)
    sketch_cols_unit<XT, LQ>(it, u, lane, Xw);
  else
    sketch_rows_unit<XT, LQ>(it, u, lane);
}

template <int NT>
__device__ __forceinline__ void sketch_unit_tc(const TbItem& it, const SkUnit& u, int lane) {
  if (u.kb >= kUnitCols)
    sketch_cols_tc<NT>(it, u, lane);
  else
    sketch_rows_tc<NT>(it, u, lane);
}

template <class XT>
__global__ void __launch_bounds__(kBT, 2)
    batch_sketch_kernel(const TbItem* __restrict__ items, const SkUnit* __restrict__ units,
                        int nunits, int* counter) {
  __shared__ float xw[kBT / 32][32 * 33];
  const int lane = threadIdx.x & 31;
  float* Xw = xw[threadIdx.x >> 5];
  for (;;) {
    const int ui = warp_next(counter, lane);
    if (ui >= nunits) break;
    const SkUnit u = units[ui];
    const TbItem& it = items[u.item];
    if constexpr (std::is_same<XT, __nv_bfloat16>::value) {
      switch ((it.lm + 7) >> 3) {  // uniform over the warp
        case 1: sketch_unit_tc<1>(it, u, lane); break;
        case 2: sketch_unit_tc<2>(it, u, lane); break;
        case 3: sketch_unit_tc<3>(it, u, lane); break;
        default: sketch_unit_tc<4>(it, u, lane); break;
      }
    } else {
      switch ((it.lm + 3) >> 2) {  // uniform over the warp
      case 1: sketch_unit<XT, 1>(it, u, lane, Xw); break;
      case 2: sketch_unit<XT, 2>(it, u, lane, Xw); break;
      case 3: sketch_unit<XT, 3>(it, u, lane, Xw); break;
      case 4: sketch_unit<XT, 4>(it, u, lane, Xw); break;
      case 5: sketch_unit<XT, 5>(it, u, lane, Xw); break;
      case 6: sketch_unit<XT, 6>(it, u, lane, Xw); break;
      case 7: sketch_unit<XT, 7>(it, u, lane, Xw); break;
      default: sketch_unit<XT, 8>(it, u, lane, Xw); break;
      }
    }
  }
}

// Row-major FP32 tables of the factors (which = 0: Omega_m from om[m], LP =
// 4 ceil(lm / 4) columns; which = 1: Q_m from the FP64 Q[m], 4 ceil(l_m / 4)
// columns), zero beyond the last column; grid (count, 3).
__global__ void batch_rows_kernel(const TbItem* __restrict__ items, int which) {
  const TbItem& it = items[blockIdx.x];
  const int m = blockIdx.y, n = it.n[m];
  const int l = which ? it.l[m] : it.lm;
  const int lp = 4 * ((l + 3) / 4);
  float* dst = which ? it.qrow[m] : it.orow[m];
  for (int e = threadIdx.x; e < n * lp; e += blockDim.x) {
    const int i = e % n, k = e / n;
    float v = 0.f;
    if (k < l) v = which ? (float)it.Q[m][i + (int64_t)n * k] : it.om[m][i + (int64_t)n * k];
    dst[(size_t)i * lp + k] = v;
  }
  if (which == 0 && m < 2 && it.ot[m]) {  // BF16 factors (exact: the BF16 form draws them rounded)
    const int np = it.np16[m], l8 = 8 * ((l + 7) / 8);
    for (int e = threadIdx.x; e < l8 * np; e += blockDim.x) {
      const int k = e / np, i = e % np;
      it.ot[m][e] = __float2bfloat16_rn(k < l && i < n ? it.om[m][i + (int64_t)n * k] : 0.f);
    }
  }
  if (which == 1 && m == 0 && it.q1t) {  // Q1 = hi + mid + lo in BF16, a-major, 32 rows of a
    const int np = it.np16[0];
    const size_t plane = (size_t)32 * np;
    for (int e = threadIdx.x; e < 32 * np; e += blockDim.x) {
      const int k = e / np, i = e % np;
      const double v = k < l && i < n ? it.Q[0][i + (int64_t)n * k] : 0.0;
      const __nv_bfloat16 h = __double2bfloat16(v);
      const double r1 = v - (double)__bfloat162float(h);
      const __nv_bfloat16 md = __double2bfloat16(r1);
      const __nv_bfloat16 lo = __double2bfloat16(r1 - (double)__bfloat162float(md));
      it.q1t[e] = h;
      it.q1t[plane + e] = md;
      it.q1t[2 * plane + e] = lo;
    }
  }
  if (which == 1 && m == 1 && it.q2t) {  // Q2 = hi + mid + lo in BF16
    const int np = it.np16[1], l8 = 8 * ((l + 7) / 8);
    const size_t plane = (size_t)l8 * np;
    for (int e = threadIdx.x; e < l8 * np; e += blockDim.x) {
      const int k = e / np, j = e % np;
      const double v = k < l && j < n ? it.Q[1][j + (int64_t)n * k] : 0.0;
      const __nv_bfloat16 h = __double2bfloat16(v);
      const double r1 = v - (double)__bfloat162float(h);
      const __nv_bfloat16 md = __double2bfloat16(r1);
      const __nv_bfloat16 lo = __double2bfloat16(r1 - (double)__bfloat162float(md));
      it.q2t[e] = h;
      it.q2t[plane + e] = md;
      it.q2t[2 * plane + e] = lo;
    }
  }
}

// ------------------------------------------------------------------ core ----
// C_t = Q1^T X_t Q2 (l1 x l2) for one slab t per warp unit.  For each block
// of 32 rows i (lane = row): T[i, :] = sum_j X[i, j, t] Q2[j, :] (X straight
// from global memory, Q2 rows broadcast), staged in the warp's shared buffer,
// then C_t[a, 4bq .. 4bq+3] += sum_i Q1[i, a] T[i, 4bq .. 4bq+3] for the
// lane's pairs (a, bq) (pair p = lane + 32 m, a = p / LQ, bq = p % LQ).  C_t
// is stored whole at the end (no atomics).  LQ = ceil(l2 / 4).
template <class XT, int LQ>
__device__ void core_unit(const TbItem& it, int t, int lane, float* Tw) {
  constexpr int LP = 4 * LQ;
  constexpr int NC = LQ <= 4 ? 16 : 8;
  const int n1 = it.n[0], n2 = it.n[1], l1 = it.l[0], l2 = it.l[1];
  const int l1p = 4 * ((l1 + 3) / 4);
  const int npairs = l1 * LQ;  // <= 32 LQ
  const float4* q2 = reinterpret_cast<const float4*>(it.qrow[1]);
  const float* q1 = it.qrow[0];
  const XT* X = static_cast<const XT*>(it.X);
  float c[LQ][4];
#pragma unroll
  for (int m = 0; m < LQ; ++m) c[m][0] = c[m][1] = c[m][2] = c[m][3] = 0.f;
  const int RB = (n1 + 31) >> 5;
  for (int rb = 0; rb < RB; ++rb) {
    if constexpr (std::is_same<XT, __nv_bfloat16>::value) {
      __syncwarp();  // the previous block's T has been read
      core_rows_tc<(LQ + 1) / 2>(it, t, rb, lane, Tw, LP);
      __syncwarp();
    } else {
    const int i = 32 * rb + lane;
    const bool valid = i < n1;
    const XT* xp = X + (int64_t)n1 * n2 * t + (valid ? i : 0);
    float tr[LP];
#pragma unroll
    for (int k = 0; k < LP; ++k) tr[k] = 0.f;
    int j = 0;
    for (; j + NC <= n2; j += NC) {
      float xv[NC];
      const XT* xj = xp + (int64_t)n1 * j;
#pragma unroll
      for (int cc = 0; cc < NC; ++cc) xv[cc] = valid ? ldx(xj, n1 * cc) : 0.f;
#pragma unroll
      for (int cc = 0; cc < NC; ++cc)
#pragma unroll
        for (int q = 0; q < LQ; ++q) fma4(&tr[4 * q], xv[cc], __ldg(q2 + (j + cc) * LQ + q));
    }
    for (; j < n2; ++j) {
      const float x = valid ? ldx(xp, (int64_t)n1 * j) : 0.f;
#pragma unroll
      for (int q = 0; q < LQ; ++q) fma4(&tr[4 * q], x, __ldg(q2 + j * LQ + q));
    }
    __syncwarp();  // the previous block's T has been read
#pragma unroll
    for (int q = 0; q < LQ; ++q)
      *reinterpret_cast<float4*>(&Tw[lane * LP + 4 * q]) =
          make_float4(tr[4 * q], tr[4 * q + 1], tr[4 * q + 2], tr[4 * q + 3]);
    __syncwarp();
    }
    const int ni = min(32, n1 - 32 * rb);
    for (int ii = 0; ii < ni; ++ii) {
      const float* q1r = q1 + (size_t)(32 * rb + ii) * l1p;
      const float4* trow = reinterpret_cast<const float4*>(Tw + ii * LP);
#pragma unroll
      for (int m = 0; m < LQ; ++m) {
        const int p = lane + 32 * m;
        if (p < npairs) fma4(c[m], __ldg(q1r + p / LQ), trow[p % LQ]);
      }
    }
  }
  float* Ct = it.C + (int64_t)t * l1 * l2;
#pragma unroll
  for (int m = 0; m < LQ; ++m) {
    const int p = lane + 32 * m;
    if (p < npairs) {
      const int a = p / LQ, b0 = 4 * (p % LQ);
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (b0 + e < l2) Ct[a + l1 * (b0 + e)] = c[m][e];
    }
  }
}

template <class XT>
__global__ void __launch_bounds__(kBT, 2)
    batch_core_kernel(const TbItem* __restrict__ items, const SkUnit* __restrict__ units,
                      int nunits, int* counter) {
  __shared__ __align__(16) float tw[kBT / 32][32 * 4 * 8];
  const int lane = threadIdx.x & 31;
  float* Tw = tw[threadIdx.x >> 5];
  for (;;) {
    const int ui = warp_next(counter, lane);
    if (ui >= nunits) break;
    const SkUnit u = units[ui];
    const TbItem& it = items[u.item];
    if constexpr (std::is_same<XT, __nv_bfloat16>::value) {
      switch ((it.l[1] + 7) >> 3) {
        case 1: core_unit_tc<1>(it, u.t0, lane, Tw); break;
        case 2: core_unit_tc<2>(it, u.t0, lane, Tw); break;
        case 3: core_unit_tc<3>(it, u.t0, lane, Tw); break;
        default: core_unit_tc<4>(it, u.t0, lane, Tw); break;
      }
    } else {
    switch ((it.l[1] + 3) >> 2) {
      case 1: core_unit<XT, 1>(it, u.t0, lane, Tw); break;
      case 2: core_unit<XT, 2>(it, u.t0, lane, Tw); break;
      case 3: core_unit<XT, 3>(it, u.t0, lane, Tw); break;
      case 4: core_unit<XT, 4>(it, u.t0, lane, Tw); break;
      case 5: core_unit<XT, 5>(it, u.t0, lane, Tw); break;
      case 6: core_unit<XT, 6>(it, u.t0, lane, Tw); break;
      case 7: core_unit<XT, 7>(it, u.t0, lane, Tw); break;
      default: core_unit<XT, 8>(it, u.t0, lane, Tw); break;
    }
    }
  }
}

// G[ab + l1 l2 c] = sum_t C_t[ab] Q3[t, c]; one CTA per tensor.  Q3 goes to
// shared memory in FP32 once (rows of kMaxEll, zero-padded); a thread owns
// one ab and all l3 outputs, so every C_t[ab] is loaded once (coalesced over
// ab) and multiplied by a broadcast row of Q3.
__global__ void batch_core_finish_kernel(const TbItem* __restrict__ items) {
  extern __shared__ __align__(16) float q3s[];  // n3 x kMaxEll
  const TbItem& it = items[blockIdx.x];
  const int l12 = it.l[0] * it.l[1], l3 = it.l[2], n3 = it.n[2];
  for (int e = threadIdx.x; e < n3 * kMaxEll; e += blockDim.x) {
    const int t = e / kMaxEll, c = e % kMaxEll;
    q3s[e] = c < l3 ? (float)it.Q[2][t + (int64_t)n3 * c] : 0.f;
  }
  __syncthreads();
  for (int ab = threadIdx.x; ab < l12; ab += blockDim.x) {
    float acc[kMaxEll];
#pragma unroll
    for (int c = 0; c < kMaxEll; ++c) acc[c] = 0.f;
    const float* cp = it.C + ab;
    for (int t = 0; t < n3; ++t) {
      const float cv = cp[(int64_t)t * l12];
      const float* q = q3s + t * kMaxEll;
#pragma unroll
      for (int cq = 0; cq < kMaxEll / 4; ++cq) {
        if (4 * cq < l3) {
          const float4 v = *reinterpret_cast<const float4*>(&q[4 * cq]);
          acc[4 * cq + 0] = fmaf(cv, v.x, acc[4 * cq + 0]);
          acc[4 * cq + 1] = fmaf(cv, v.y, acc[4 * cq + 1]);
          acc[4 * cq + 2] = fmaf(cv, v.z, acc[4 * cq + 2]);
          acc[4 * cq + 3] = fmaf(cv, v.w, acc[4 * cq + 3]);
        }
      }
    }
#pragma unroll
    for (int c = 0; c < kMaxEll; ++c)
      if (c < l3) it.G[ab + (int64_t)l12 * c] = acc[c];
  }
}

// ------------------------------------------------------------ truncation ----
// Gram of unfolding `mode` of the FP32 core, FP64 accumulation; grid (count, 3).
// The core is converted to ST once in shared memory (ST = double when it
// fits, so no per-term conversion runs on the FP64 pipe); a thread owns one
// pair p <= q and walks the unfolding's columns as two nested loops over the
// other two modes (no index division).
template <class ST>
__global__ void batch_gram_kernel(const TbItem* __restrict__ items) {
  extern __shared__ __align__(16) unsigned char gram_raw[];
  ST* gsh = reinterpret_cast<ST*>(gram_raw);
  const TbItem& it = items[blockIdx.x];
  const int mode = blockIdx.y;
  const int l0 = it.l[0], l1 = it.l[1], l2 = it.l[2];
  const int L = l0 * l1 * l2;
  for (int e = threadIdx.x; e < L; e += blockDim.x) gsh[e] = (ST)it.G[e];
  __syncthreads();
  const int lm = it.l[mode];
  // element (x0, x1, x2) at x0 + l0 x1 + l0 l1 x2; the unfolding's column
  // index runs over the other two modes, the first one fastest
  const int stride = mode == 0 ? 1 : (mode == 1 ? l0 : l0 * l1);
  const int na = mode == 0 ? l1 : l0, sa = mode == 0 ? l0 : 1;
  const int nb = mode == 2 ? l1 : l2, sb = mode == 2 ? l0 : l0 * l1;
  const int npairs = lm * (lm + 1) / 2;
  for (int pq = threadIdx.x; pq < npairs; pq += blockDim.x) {
    // pq = q (q + 1) / 2 + p with p <= q
    int q = (int)((sqrtf(8.f * pq + 1.f) - 1.f) * 0.5f);
    while (q * (q + 1) / 2 > pq) --q;
    while ((q + 1) * (q + 2) / 2 <= pq) ++q;
    const int p = pq - q * (q + 1) / 2;
    const ST* gp = gsh + p * stride;
    const ST* gq = gsh + q * stride;
    double s = 0.0;
    for (int y = 0; y < nb; ++y) {
      const int base = y * sb;
      for (int x = 0; x < na; ++x) {
        const int off = base + x * sa;
        s = fma((double)gp[off], (double)gq[off], s);
      }
    }
    it.S[mode][p + lm * q] = s;
    it.S[mode][q + lm * p] = s;
  }
}

// Truncated core and factors (one CTA per tensor): G' = G x_1 U1^T x_2 U2^T
// x_3 U3^T through two global scratch tensors, Q_i U_i; without truncation
// the core and factors are copied out.  The core is stored in FP32, so its
// three contractions run in FP32 (U_i rounded to FP32: relative 2^-24 per
// entry, ~1e-7 on the core, against the 1e-5 bounds of the reconstruction);
// GB300 issues FP64 at 1/64 of the FP32 rate, and these products were two
// thirds of the kernel's FP64 work.  The factors Q_i U_i stay FP64.
__global__ void batch_trunc_apply_kernel(const TbItem* __restrict__ items, int trunc) {
  const TbItem& it = items[blockIdx.x];
  const int l0 = it.l[0], l1 = it.l[1], l2 = it.l[2];
  const int r0 = it.r[0], r1 = it.r[1], r2 = it.r[2];
  const int tid = threadIdx.x, nt = blockDim.x;
  if (!trunc) {
    for (int e = tid; e < l0 * l1 * l2; e += nt) it.core_out[e] = it.G[e];
    for (int m = 0; m < 3; ++m)
      for (int e = tid; e < it.n[m] * it.l[m]; e += nt) it.fac_out[m][e] = it.Q[m][e];
    return;
  }
  float* T1 = reinterpret_cast<float*>(it.T1);  // FP32 views of the FP64 scratch
  float* T2 = reinterpret_cast<float*>(it.T2);
  // T1[a', x1, x2] = sum_a U0[a, a'] G[a, x1, x2]
  for (int e = tid; e < r0 * l1 * l2; e += nt) {
    const int ap = e % r0, rest = e / r0;
    float s = 0.f;
    for (int a = 0; a < l0; ++a) s = fmaf((float)it.U[0][a + l0 * ap], it.G[a + l0 * rest], s);
    T1[e] = s;
  }
  __syncthreads();
  // T2[a', b', x2] = sum_b U1[b, b'] T1[a', b, x2]
  for (int e = tid; e < r0 * r1 * l2; e += nt) {
    const int ap = e % r0, bp = (e / r0) % r1, c = e / (r0 * r1);
    float s = 0.f;
    for (int b = 0; b < l1; ++b) s = fmaf((float)it.U[1][b + l1 * bp], T1[ap + r0 * (b + l1 * c)], s);
    T2[e] = s;
  }
  __syncthreads();
  for (int e = tid; e < r0 * r1 * r2; e += nt) {
    const int ab = e % (r0 * r1), cp = e / (r0 * r1);
    float s = 0.f;
    for (int c = 0; c < l2; ++c) s = fmaf((float)it.U[2][c + l2 * cp], T2[ab + r0 * r1 * c], s);
    it.core_out[e] = s;
  }
  for (int m = 0; m < 3; ++m) {
    const int n = it.n[m], l = it.l[m], r = it.r[m];
    for (int e = tid; e < n * r; e += nt) {
      const int i = e % n, k = e / n;
      double s = 0.0;
      for (int a = 0; a < l; ++a) s = fma(it.Q[m][i + (int64_t)n * a], it.U[m][a + l * k], s);
      it.fac_out[m][e] = s;
    }
  }
}

// -------------------------------------------------------------- residual ----
// M_t[a + r0 b] = sum_c Gt[a + r0 b + r0 r1 c] F3[t, c] for every slab t of a
// tensor (one CTA per tensor), so the residual kernel reads each M_t as one
// contiguous block.  F3 is converted to FP32 once, in shared memory.
__global__ void batch_resid_prep_kernel(const TbItem* __restrict__ items) {
  extern __shared__ float f3s[];  // n3 x r2, row-major
  const TbItem& it = items[blockIdx.x];
  const int r01 = it.r[0] * it.r[1], r2 = it.r[2], n3 = it.n[2];
  for (int e = threadIdx.x; e < n3 * r2; e += blockDim.x) {
    const int t = e % n3, c = e / n3;
    f3s[t * r2 + c] = (float)it.fac_out[2][e];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n3 * r01; e += blockDim.x) {
    const int t = e / r01, ab = e % r01;
    float s = 0.f;
    for (int c = 0; c < r2; ++c) s = fmaf(it.core_out[ab + r01 * c], f3s[t * r2 + c], s);
    it.M[e] = s;
  }
}

// ||X_t - F1 M_t F2^T||^2 and ||X_t||^2 over the slabs of a tile.  A warp
// owns one unit (slab t, block of 32 rows i; lane = row): it forms
// P[i, :] = F1[i, :] M_t in registers (r1 values, padded to 4 RQ), then walks
// the slab's columns j reading X[i, j, t] straight from global memory
// (coalesced over the lanes, 16 columns in flight, 8 for r1 > 16) with
// x_hat[i, j] = P[i, :] . F2[j, :], the F2 rows broadcast from shared memory.
// The warps of a CTA share the tile's F1, F2 and M_t in shared memory and
// meet at no barrier inside the tile.  Per-unit sums are FP32 (at most n2
// terms per lane), then FP64.
// Shared memory (floats): F1s[r0][32 RB] (zero for i >= n1), F2s[n2][4 RQ],
// Ms[slabs][r0][4 RQ] (zero for b >= r1).
constexpr int kResidUnits = 16;  // target units (slab x row block) per tile

template <class XT, int RQ>
__device__ void resid_tile(const TbItem& it, const TbTile& tile, float* sm, double& dd,
                           double& xx) {
  constexpr int R1P = 4 * RQ;
  constexpr int kRCols = RQ <= 4 ? 16 : 8;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n1 = it.n[0], n2 = it.n[1], r0 = it.r[0], r1 = it.r[1];
  const int RB = (n1 + 31) >> 5, pitch = 32 * RB;
  const int nt = tile.t1 - tile.t0;
  float* F1s = sm;
  float* F2s = F1s + r0 * pitch;
  float* Ms = F2s + n2 * R1P;
  const double* f1 = it.fac_out[0];
  const double* f2 = it.fac_out[1];
  for (int e = tid; e < r0 * pitch; e += kBT) {
    const int a = e / pitch, i = e - a * pitch;
    F1s[e] = i < n1 ? (float)f1[i + (int64_t)n1 * a] : 0.f;
  }
  for (int e = tid; e < n2 * R1P; e += kBT) {
    const int j = e % n2, b = e / n2;
    F2s[j * R1P + b] = b < r1 ? (float)f2[j + (int64_t)n2 * b] : 0.f;
  }
  for (int e = tid; e < nt * r0 * R1P; e += kBT) {
    const int b = e % R1P, rest = e / R1P, a = rest % r0, tt = rest / r0;
    Ms[e] = b < r1 ? it.M[(int64_t)(tile.t0 + tt) * r0 * r1 + a + r0 * b] : 0.f;
  }
  __syncthreads();
  const XT* X = static_cast<const XT*>(it.X);
  for (int u = warp; u < nt * RB; u += kBT / 32) {
    const int tt = u / RB, rb = u - tt * RB;
    const int i = 32 * rb + lane;
    const bool valid = i < n1;
    float P[R1P];
#pragma unroll
    for (int b = 0; b < R1P; ++b) P[b] = 0.f;
    const float* mt = Ms + tt * r0 * R1P;
    for (int a = 0; a < r0; ++a) {
      const float f = F1s[a * pitch + i];
#pragma unroll
      for (int q = 0; q < RQ; ++q) {
        const float4 m = *reinterpret_cast<const float4*>(&mt[a * R1P + 4 * q]);
        P[4 * q + 0] = fmaf(f, m.x, P[4 * q + 0]);
        P[4 * q + 1] = fmaf(f, m.y, P[4 * q + 1]);
        P[4 * q + 2] = fmaf(f, m.z, P[4 * q + 2]);
        P[4 * q + 3] = fmaf(f, m.w, P[4 * q + 3]);
      }
    }
    const XT* xp = X + (int64_t)n1 * n2 * (tile.t0 + tt) + (valid ? i : 0);
    float d0 = 0.f, d1 = 0.f, s0 = 0.f, s1 = 0.f;
    auto column = [&](float xv, int j, float& d, float& s) {
      const float* w = F2s + j * R1P;
      float h0 = 0.f, h1 = 0.f;
#pragma unroll
      for (int q = 0; q < RQ; ++q) {
        const float4 v = *reinterpret_cast<const float4*>(&w[4 * q]);
        h0 = fmaf(P[4 * q + 0], v.x, h0);
        h1 = fmaf(P[4 * q + 1], v.y, h1);
        h0 = fmaf(P[4 * q + 2], v.z, h0);
        h1 = fmaf(P[4 * q + 3], v.w, h1);
      }
      const float df = xv - (h0 + h1);
      d = fmaf(df, df, d);
      s = fmaf(xv, xv, s);
    };
    int j = 0;
    for (; j + kRCols <= n2; j += kRCols) {
      float xv[kRCols];
#pragma unroll
      for (int c = 0; c < kRCols; ++c) xv[c] = valid ? ldx(xp, (int64_t)n1 * (j + c)) : 0.f;
#pragma unroll
      for (int c = 0; c < kRCols; c += 2) {
        column(xv[c], j + c, d0, s0);
        column(xv[c + 1], j + c + 1, d1, s1);
      }
    }
    for (; j < n2; ++j) column(valid ? ldx(xp, (int64_t)n1 * j) : 0.f, j, d0, s0);
    dd += (double)(d0 + d1);
    xx += (double)(s0 + s1);
  }
}

// WIDE: r1 up to 32 (two CTAs per SM); otherwise r1 <= 16 (three CTAs per SM).
template <class XT, bool WIDE>
__global__ void __launch_bounds__(kBT, WIDE ? 2 : 3)
    batch_resid_kernel(const TbItem* __restrict__ items, const TbTile* __restrict__ tiles,
                       int ntiles, int* counter) {
  extern __shared__ __align__(16) float bsm[];
  __shared__ int s_tile;
  __shared__ double red[2][kBT / 32];
  const int tid = threadIdx.x;
  for (;;) {
    const int ti = next_tile(counter, &s_tile);
    if (ti >= ntiles) break;
    const TbTile tile = tiles[ti];
    const TbItem& it = items[tile.item];
    double dd = 0.0, xx = 0.0;
    switch ((it.r[1] + 3) >> 2) {  // uniform over the CTA
      case 1: resid_tile<XT, 1>(it, tile, bsm, dd, xx); break;
      case 2: resid_tile<XT, 2>(it, tile, bsm, dd, xx); break;
      case 3: resid_tile<XT, 3>(it, tile, bsm, dd, xx); break;
      case 4: resid_tile<XT, 4>(it, tile, bsm, dd, xx); break;
      default:
        if constexpr (WIDE) {
          switch ((it.r[1] + 3) >> 2) {
            case 5: resid_tile<XT, 5>(it, tile, bsm, dd, xx); break;
            case 6: resid_tile<XT, 6>(it, tile, bsm, dd, xx); break;
            case 7: resid_tile<XT, 7>(it, tile, bsm, dd, xx); break;
            default: resid_tile<XT, 8>(it, tile, bsm, dd, xx); break;
          }
        }
        break;
    }
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
      double a = 0.0, b = 0.0;
      for (int w = 0; w < kBT / 32; ++w) {
        a += red[0][w];
        b += red[1][w];
      }
      atomicAdd(it.acc, a);
      atomicAdd(it.acc + 1, b);
    }
  }
}

__global__ void batch_resid_finish_kernel(const TbItem* __restrict__ items, int count,
                                          double* __restrict__ rel) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < count; b += gridDim.x * blockDim.x) {
    const double* a = items[b].acc;
    rel[b] = a[1] > 0.0 ? sqrt(a[0] / a[1]) : 0.0;
  }
}

// ------------------------------------------------------------------ plan ----
template <class T>
T* carve(char*& p, size_t count) {
  T* r = reinterpret_cast<T*>(p);
  p += (count * sizeof(T) + 255) & ~size_t(255);
  return r;
}

struct TbPlan {
  // signature
  krp_dtype xt{};
  int count = 0, oversample = 0;
  unsigned flags = 0;
  std::vector<krp_tucker_item> sig;
  // device state
  char* arena = nullptr;
  TbItem* d_items = nullptr;
  SkUnit* d_sunits = nullptr;  // sketch units (rows and columns)
  int nsunits = 0;
  SkUnit* d_cunits = nullptr;  // core units (one slab each)
  int ncunits = 0;
  TbTile* d_rtiles = nullptr;  // residual tiles: about kResidUnits warp units each
  int nrtiles = 0;
  int* d_counters = nullptr;  // 3
  BatchFactorJob* d_fjobs = nullptr;
  int64_t* d_fstart = nullptr;
  int64_t fblocks = 0;
  QrJob* d_qjobs = nullptr;
  EigJob* d_ejobs = nullptr;
  double* d_rel = nullptr;
  double* h_rel = nullptr;  // pinned
  float* y_begin = nullptr;
  size_t y_bytes = 0;
  double* acc_begin = nullptr;
  int n1max = 0, n2max = 0, lmax = 0;
  size_t sm_resid = 0, sm_gram = 0, sm_prep = 0, sm_finish = 0;
  bool gram_f64 = true;
  bool resid_wide = false;  // some r_2 > 16
  int grid_sketch = 0, grid_core = 0, grid_resid = 0;
  int slabs_per_unit = 0;
  std::vector<TbItem> h_items;
  cudaGraphExec_t exec = nullptr;
  int kernels_per_run = 0;
  // the graph is captured and replayed on a stream of the plan (the caller's
  // stream may be the legacy default stream, which cannot be captured),
  // ordered after and before the caller's work with two events
  cudaStream_t cs = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;

  ~TbPlan() {
    if (exec) cudaGraphExecDestroy(exec);
    if (ev_in) cudaEventDestroy(ev_in);
    if (ev_out) cudaEventDestroy(ev_out);
    if (cs) cudaStreamDestroy(cs);
    if (arena) cudaFree(arena);
    if (h_rel) cudaFreeHost(h_rel);
  }
};

bool same_signature(const TbPlan& p, krp_dtype xt, int count, const krp_tucker_item* items,
                    int oversample, unsigned flags) {
  if (p.xt != xt || p.count != count || p.oversample != oversample || p.flags != flags) return false;
  for (int b = 0; b < count; ++b) {
    const krp_tucker_item& a = p.sig[b];
    const krp_tucker_item& c = items[b];
    if (a.X != c.X || a.seed != c.seed || a.core != c.core) return false;
    for (int m = 0; m < 3; ++m)
      if (a.dims[m] != c.dims[m] || a.ranks[m] != c.ranks[m] || a.factors[m] != c.factors[m])
        return false;
  }
  return true;
}

// Sketch units with `spu` slabs each: for every tensor and slab group, its
// row units then its column units (adjacent, so the column units find the
// slabs in L2); groups ordered by work, largest first.
void build_sketch_units(const std::vector<TbItem>& items, int spu, std::vector<SkUnit>& units) {
  struct Group { int item, t0, t1; int64_t work; };
  std::vector<Group> groups;
  for (int b = 0; b < (int)items.size(); ++b) {
    const TbItem& it = items[b];
    for (int t0 = 0; t0 < it.n[2]; t0 += spu) {
      const int t1 = std::min(it.n[2], t0 + spu);
      groups.push_back(Group{b, t0, t1, (int64_t)it.n[0] * it.n[1] * (t1 - t0)});
    }
  }
  std::stable_sort(groups.begin(), groups.end(),
                   [](const Group& x, const Group& y) { return x.work > y.work; });
  units.clear();
  for (const Group& g : groups) {
    const TbItem& it = items[g.item];
    for (int rb = 0; rb < (it.n[0] + 31) / 32; ++rb) units.push_back(SkUnit{g.item, rb, g.t0, g.t1});
    for (int jb = 0; jb < (it.n[1] + 31) / 32; ++jb)
      units.push_back(SkUnit{g.item, kUnitCols | jb, g.t0, g.t1});
  }
}

void launch_sketch(const TbPlan& P) {
  if (P.xt == KRP_F32)
    batch_sketch_kernel<float><<<P.grid_sketch, kBT, 0, stream()>>>(P.d_items, P.d_sunits,
                                                                     P.nsunits, P.d_counters + 0);
  else
    batch_sketch_kernel<__nv_bfloat16><<<P.grid_sketch, kBT, 0, stream()>>>(
        P.d_items, P.d_sunits, P.nsunits, P.d_counters + 0);
  check_launch("batch_sketch");
}

template <class XT>
void launch_resid(const TbPlan& P) {
  if (P.resid_wide)
    batch_resid_kernel<XT, true><<<P.grid_resid, kBT, P.sm_resid, stream()>>>(
        P.d_items, P.d_rtiles, P.nrtiles, P.d_counters + 2);
  else
    batch_resid_kernel<XT, false><<<P.grid_resid, kBT, P.sm_resid, stream()>>>(
        P.d_items, P.d_rtiles, P.nrtiles, P.d_counters + 2);
}

// The whole batch, enqueued on the context stream (captured once into a graph).
void enqueue_all(TbPlan& P, int* status) {
  const bool trunc = P.flags & KRP_TRUNCATE;
  const bool resid = P.flags & KRP_RESIDUAL;
  int nk = 0;
  KRP_CUDA_CHECK(cudaMemsetAsync(P.d_counters, 0, 3 * sizeof(int), stream()));
  KRP_CUDA_CHECK(cudaMemsetAsync(P.y_begin, 0, P.y_bytes, stream()));
  KRP_CUDA_CHECK(cudaMemsetAsync(P.acc_begin, 0, sizeof(double) * 2 * P.count, stream()));
  launch_gen_factors_batch(P.d_fjobs, P.d_fstart, 3 * P.count, P.fblocks);
  batch_rows_kernel<<<dim3(P.count, 3), 256, 0, stream()>>>(P.d_items, 0);
  check_launch("batch_rows");
  nk += 2;
  launch_sketch(P);
  ++nk;
  // the sketches are short (n <= 256 rows): one CTA per Householder QR keeps
  // the 3 x count problems in one launch (measured faster than CholeskyQR3
  // over row blocks, whose nine launches each see tiny problems)
  qr_householder_launch(P.d_qjobs, 3 * P.count, status);
  batch_rows_kernel<<<dim3(P.count, 3), 256, 0, stream()>>>(P.d_items, 1);
  check_launch("batch_rows");
  nk += 2;
  if (P.xt == KRP_F32)
    batch_core_kernel<float><<<P.grid_core, kBT, 0, stream()>>>(P.d_items, P.d_cunits, P.ncunits,
                                                                P.d_counters + 1);
  else
    batch_core_kernel<__nv_bfloat16><<<P.grid_core, kBT, 0, stream()>>>(
        P.d_items, P.d_cunits, P.ncunits, P.d_counters + 1);
  check_launch("batch_core");
  batch_core_finish_kernel<<<P.count, 256, P.sm_finish, stream()>>>(P.d_items);
  check_launch("batch_core_finish");
  nk += 2;
  if (trunc) {
    if (P.gram_f64)
      batch_gram_kernel<double><<<dim3(P.count, 3), 256, P.sm_gram, stream()>>>(P.d_items);
    else
      batch_gram_kernel<float><<<dim3(P.count, 3), 256, P.sm_gram, stream()>>>(P.d_items);
    check_launch("batch_gram");
    eig_launch(P.d_ejobs, 3 * P.count, P.lmax, status);
    nk += 2;
  }
  batch_trunc_apply_kernel<<<P.count, 256, 0, stream()>>>(P.d_items, trunc ? 1 : 0);
  check_launch("batch_trunc_apply");
  ++nk;
  if (resid) {
    batch_resid_prep_kernel<<<P.count, 256, P.sm_prep, stream()>>>(P.d_items);
    check_launch("batch_resid_prep");
    ++nk;
    if (P.xt == KRP_F32)
      launch_resid<float>(P);
    else
      launch_resid<__nv_bfloat16>(P);
    check_launch("batch_resid");
    batch_resid_finish_kernel<<<(P.count + 255) / 256, 256, 0, stream()>>>(P.d_items, P.count,
                                                                          P.d_rel);
    check_launch("batch_resid_finish");
    nk += 2;
    KRP_CUDA_CHECK(cudaMemcpyAsync(P.h_rel, P.d_rel, sizeof(double) * P.count,
                                   cudaMemcpyDeviceToHost, stream()));
  }
  P.kernels_per_run = nk;
}

template <class K>
void allow_smem(K k, size_t bytes) {
  KRP_CUDA_CHECK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
}

std::unique_ptr<TbPlan> build_plan(Ctx* c, krp_dtype xt, int count, const krp_tucker_item* items,
                                   int oversample, unsigned flags) {
  auto P = std::make_unique<TbPlan>();
  P->xt = xt;
  P->count = count;
  P->oversample = oversample;
  P->flags = flags;
  P->sig.assign(items, items + count);
  const bool trunc = flags & KRP_TRUNCATE;
  // sizes
  size_t bytes = 0;
  auto add = [&](size_t n, size_t e) { bytes += (n * e + 255) & ~size_t(255); };
  std::vector<int> lm(count);
  for (int b = 0; b < count; ++b) {
    const krp_tucker_item& it = items[b];
    int l[3], r[3];
    int lmx = 0;
    for (int m = 0; m < 3; ++m) {
      l[m] = it.ranks[m] + oversample;
      r[m] = trunc ? it.ranks[m] : l[m];
      lmx = std::max(lmx, l[m]);
    }
    lm[b] = lmx;
    for (int m = 0; m < 3; ++m) {
      add((size_t)it.dims[m] * lmx, 4);       // om
      add((size_t)it.dims[m] * (lmx + 3), 4);     // orow
      add((size_t)it.dims[m] * (l[m] + 3), 4);    // qrow
      if (xt == KRP_BF16) {
        const size_t np = (size_t)((it.dims[m] + 15) / 16) * 16;
        if (m < 2) add(np * 8 * ((lmx + 7) / 8), 2);   // ot
        if (m == 1) add(3 * np * 8 * ((l[m] + 7) / 8), 2);  // q2t
        if (m == 0) add(3 * np * 32, 2);                     // q1t
      }
      add((size_t)it.dims[m] * lmx, 4);       // Y (added separately below too)
      add((size_t)it.dims[m] * l[m], 8);      // Q
      add((size_t)it.dims[m] * l[m], 8);      // QR work
      add((size_t)l[m] * l[m], 8);            // S
      add((size_t)l[m] * r[m], 8);            // U
    }
    add((size_t)it.dims[2] * l[0] * l[1], 4);       // C
    add((size_t)l[0] * l[1] * l[2], 4);             // G
    add((size_t)r[0] * l[1] * l[2], 8);             // T1
    add((size_t)r[0] * r[1] * l[2], 8);             // T2
    add((size_t)it.dims[2] * r[0] * r[1], 4);       // M
  }
  add((size_t)2 * count, 8);  // acc
  add((size_t)count, sizeof(TbItem));
  add((size_t)3 * count, sizeof(BatchFactorJob));
  add((size_t)3 * count + 1, 8);
  add((size_t)3 * count, sizeof(QrJob));
  add((size_t)3 * count, sizeof(EigJob));
  add((size_t)count, 8);  // rel
  add(3, 4);              // counters
  int64_t total_slabs = 0, max_sunits = 0;
  for (int b = 0; b < count; ++b) {
    total_slabs += items[b].dims[2];
    max_sunits += (int64_t)items[b].dims[2] * ((items[b].dims[0] + 31) / 32 + (items[b].dims[1] + 31) / 32);
  }
  add((size_t)max_sunits, sizeof(SkUnit));
  add((size_t)total_slabs, sizeof(SkUnit));
  add((size_t)total_slabs, sizeof(TbTile));
  KRP_CUDA_CHECK(cudaStreamCreateWithFlags(&P->cs, cudaStreamNonBlocking));
  KRP_CUDA_CHECK(cudaEventCreateWithFlags(&P->ev_in, cudaEventDisableTiming));
  KRP_CUDA_CHECK(cudaEventCreateWithFlags(&P->ev_out, cudaEventDisableTiming));
  KRP_CUDA_CHECK(cudaMalloc(&P->arena, bytes));
  KRP_CUDA_CHECK(cudaMallocHost(&P->h_rel, sizeof(double) * count));
  char* p = P->arena;
  // Y arrays first and contiguous (one memset per run), then the rest
  P->h_items.resize(count);
  char* y0 = p;
  for (int b = 0; b < count; ++b)
    for (int m = 0; m < 3; ++m)
      P->h_items[b].Y[m] = carve<float>(p, (size_t)items[b].dims[m] * lm[b]);
  P->y_begin = reinterpret_cast<float*>(y0);
  P->y_bytes = (size_t)(p - y0);
  P->acc_begin = carve<double>(p, (size_t)2 * count);
  std::vector<BatchFactorJob> fj;
  std::vector<int64_t> fstart(1, 0);
  std::vector<QrJob> qj;
  std::vector<EigJob> ej;
  P->n1max = P->n2max = P->lmax = 0;
  int rmax = 0;
  for (int b = 0; b < count; ++b) {
    const krp_tucker_item& src = items[b];
    TbItem& it = P->h_items[b];
    it.X = src.X;
    it.lm = lm[b];
    for (int m = 0; m < 3; ++m) {
      it.n[m] = (int)src.dims[m];
      it.l[m] = src.ranks[m] + oversample;
      it.r[m] = trunc ? src.ranks[m] : it.l[m];
      it.om[m] = carve<float>(p, (size_t)it.n[m] * it.lm);
      it.orow[m] = carve<float>(p, (size_t)it.n[m] * (4 * ((it.lm + 3) / 4)));
      it.qrow[m] = carve<float>(p, (size_t)it.n[m] * (4 * ((it.l[m] + 3) / 4)));
      if (m < 2) {
        it.np16[m] = (it.n[m] + 15) / 16 * 16;
        it.ot[m] = xt == KRP_BF16 ? carve<__nv_bfloat16>(p, (size_t)it.np16[m] * 8 * ((it.lm + 7) / 8))
                                  : nullptr;
      }
      if (m == 0)
        it.q1t = xt == KRP_BF16 ? carve<__nv_bfloat16>(p, (size_t)3 * it.np16[0] * 32) : nullptr;
      if (m == 1)
        it.q2t = xt == KRP_BF16 ? carve<__nv_bfloat16>(p, (size_t)3 * it.np16[1] * 8 * ((it.l[1] + 7) / 8))
                                : nullptr;
      it.Q[m] = carve<double>(p, (size_t)it.n[m] * it.l[m]);
      double* work = carve<double>(p, (size_t)it.n[m] * it.l[m]);
      it.S[m] = carve<double>(p, (size_t)it.l[m] * it.l[m]);
      it.U[m] = carve<double>(p, (size_t)it.l[m] * it.r[m]);
      it.fac_out[m] = src.factors[m];
      BatchFactorJob f{};
      f.ptr = it.om[m];
      f.rows = it.n[m];
      f.seed = src.seed;
      f.factor = (uint32_t)m;
      f.draw = KRP_DRAW_MEMO;
      f.tag = KRP_TAG_OMEGA;
      f.ell = it.lm;
      f.bf16_round = xt == KRP_BF16 ? 1 : 0;
      fj.push_back(f);
      fstart.push_back(fstart.back() + ((int64_t)it.n[m] * it.lm + 3) / 4);
      QrJob q{};
      q.Y = it.Y[m];
      q.Q = it.Q[m];
      q.R = nullptr;
      q.work = work;
      q.m = it.n[m];
      q.l = it.l[m];
      qj.push_back(q);
      ej.push_back(EigJob{it.S[m], it.U[m], nullptr, it.l[m], it.r[m]});
      P->lmax = std::max(P->lmax, it.l[m]);
      rmax = std::max(rmax, it.r[m]);
    }
    it.C = carve<float>(p, (size_t)it.n[2] * it.l[0] * it.l[1]);
    it.G = carve<float>(p, (size_t)it.l[0] * it.l[1] * it.l[2]);
    it.T1 = carve<double>(p, (size_t)it.r[0] * it.l[1] * it.l[2]);
    it.T2 = carve<double>(p, (size_t)it.r[0] * it.r[1] * it.l[2]);
    it.M = carve<float>(p, (size_t)it.n[2] * it.r[0] * it.r[1]);
    it.core_out = src.core;
    it.acc = P->acc_begin + 2 * b;
    P->n1max = std::max(P->n1max, it.n[0]);
    P->n2max = std::max(P->n2max, it.n[1]);
  }
  P->d_items = carve<TbItem>(p, count);
  P->d_fjobs = carve<BatchFactorJob>(p, (size_t)3 * count);
  P->d_fstart = carve<int64_t>(p, (size_t)3 * count + 1);
  P->d_qjobs = carve<QrJob>(p, (size_t)3 * count);
  P->d_ejobs = carve<EigJob>(p, (size_t)3 * count);
  P->d_rel = carve<double>(p, count);
  P->d_counters = carve<int>(p, 3);
  P->d_sunits = carve<SkUnit>(p, (size_t)max_sunits);
  P->d_cunits = carve<SkUnit>(p, (size_t)total_slabs);
  P->d_rtiles = carve<TbTile>(p, (size_t)total_slabs);
  KRP_REQUIRE((size_t)(p - P->arena) <= bytes, "batch plan arena overflow");
  P->fblocks = fstart.back();
  cudaStream_t s = c->stream;
  KRP_CUDA_CHECK(cudaMemcpyAsync(P->d_items, P->h_items.data(), sizeof(TbItem) * count,
                                 cudaMemcpyHostToDevice, s));
  KRP_CUDA_CHECK(cudaMemcpyAsync(P->d_fjobs, fj.data(), sizeof(BatchFactorJob) * fj.size(),
                                 cudaMemcpyHostToDevice, s));
  KRP_CUDA_CHECK(cudaMemcpyAsync(P->d_fstart, fstart.data(), sizeof(int64_t) * fstart.size(),
                                 cudaMemcpyHostToDevice, s));
  KRP_CUDA_CHECK(cudaMemcpyAsync(P->d_qjobs, qj.data(), sizeof(QrJob) * qj.size(),
                                 cudaMemcpyHostToDevice, s));
  KRP_CUDA_CHECK(cudaMemcpyAsync(P->d_ejobs, ej.data(), sizeof(EigJob) * ej.size(),
                                 cudaMemcpyHostToDevice, s));
  // core units: one slab each, largest slabs first
  {
    std::vector<SkUnit> cu;
    cu.reserve((size_t)total_slabs);
    for (int b = 0; b < count; ++b)
      for (int t = 0; t < P->h_items[b].n[2]; ++t) cu.push_back(SkUnit{b, 0, t, t + 1});
    std::stable_sort(cu.begin(), cu.end(), [&](const SkUnit& x, const SkUnit& y) {
      const TbItem& a = P->h_items[x.item];
      const TbItem& c = P->h_items[y.item];
      return (int64_t)a.n[0] * a.n[1] > (int64_t)c.n[0] * c.n[1];
    });
    P->ncunits = (int)cu.size();
    KRP_CUDA_CHECK(cudaMemcpyAsync(P->d_cunits, cu.data(), sizeof(SkUnit) * cu.size(),
                                   cudaMemcpyHostToDevice, s));
    KRP_CUDA_CHECK(cudaStreamSynchronize(s));
  }
  // residual tiles: per tensor, enough slabs for about kResidUnits warp units
  {
    std::vector<TbTile> rt;
    size_t smr = 0, smp = 0;
    for (int b = 0; b < count; ++b) {
      const TbItem& it = P->h_items[b];
      const int RB = (it.n[0] + 31) / 32, R1P = 4 * ((it.r[1] + 3) / 4);
      const int spt = std::max(1, std::min(it.n[2], (kResidUnits + RB - 1) / RB));
      for (int t0 = 0; t0 < it.n[2]; t0 += spt) rt.push_back(TbTile{b, t0, std::min(it.n[2], t0 + spt), 0});
      smr = std::max(smr, (size_t)it.r[0] * 32 * RB + (size_t)it.n[1] * R1P + (size_t)spt * it.r[0] * R1P);
      smp = std::max(smp, (size_t)it.n[2] * it.r[2]);
      if (it.r[1] > 16) P->resid_wide = true;
    }
    std::stable_sort(rt.begin(), rt.end(), [&](const TbTile& x, const TbTile& y) {
      const TbItem& a = P->h_items[x.item];
      const TbItem& c = P->h_items[y.item];
      return (int64_t)a.n[0] * a.n[1] * (x.t1 - x.t0) > (int64_t)c.n[0] * c.n[1] * (y.t1 - y.t0);
    });
    P->nrtiles = (int)rt.size();
    KRP_CUDA_CHECK(cudaMemcpyAsync(P->d_rtiles, rt.data(), sizeof(TbTile) * rt.size(),
                                   cudaMemcpyHostToDevice, s));
    KRP_CUDA_CHECK(cudaStreamSynchronize(s));
    P->sm_resid = sizeof(float) * smr;
    P->sm_prep = sizeof(float) * smp;
  }
  {
    size_t lcube = 0;
    int n3max = 0;
    for (const TbItem& it : P->h_items) {
      lcube = std::max(lcube, (size_t)it.l[0] * it.l[1] * it.l[2]);
      n3max = std::max(n3max, it.n[2]);
    }
    P->gram_f64 = lcube * sizeof(double) <= 160 * 1024;
    P->sm_gram = lcube * (P->gram_f64 ? sizeof(double) : sizeof(float));
    P->sm_finish = sizeof(float) * (size_t)n3max * kMaxEll;
  }
  allow_smem(batch_resid_kernel<float, false>, P->sm_resid);
  allow_smem(batch_resid_kernel<__nv_bfloat16, false>, P->sm_resid);
  allow_smem(batch_resid_kernel<float, true>, P->sm_resid);
  allow_smem(batch_resid_kernel<__nv_bfloat16, true>, P->sm_resid);
  allow_smem(batch_gram_kernel<double>, P->sm_gram);
  allow_smem(batch_gram_kernel<float>, P->sm_gram);
  allow_smem(batch_core_finish_kernel, P->sm_finish);
  allow_smem(batch_resid_prep_kernel, P->sm_prep);
  auto grid_of = [&](auto k0, auto k1) {
    int o0 = 1, o1 = 1;
    KRP_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o0, k0, kBT, 0));
    KRP_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o1, k1, kBT, 0));
    return std::max(1, std::min(o0, o1)) * c->num_sms;
  };
  P->grid_sketch = grid_of(batch_sketch_kernel<float>, batch_sketch_kernel<__nv_bfloat16>);
  P->grid_core = grid_of(batch_core_kernel<float>, batch_core_kernel<__nv_bfloat16>);
  int occ_r = 1, occ_rb = 1;
  if (P->resid_wide) {
    KRP_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &occ_r, batch_resid_kernel<float, true>, kBT, P->sm_resid));
    KRP_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &occ_rb, batch_resid_kernel<__nv_bfloat16, true>, kBT, P->sm_resid));
  } else {
    KRP_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &occ_r, batch_resid_kernel<float, false>, kBT, P->sm_resid));
    KRP_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &occ_rb, batch_resid_kernel<__nv_bfloat16, false>, kBT, P->sm_resid));
  }
  P->grid_resid = std::max(1, std::min(occ_r, occ_rb)) * c->num_sms;
  return P;
}

// Slabs per sketch unit: time the sketch phase for a few granularities
// (fewer slabs per unit balance better, more slabs issue fewer atomics).
void autotune(TbPlan& P) {
  const int cand[] = {2, 4, 8, 16};
  std::vector<SkUnit> units;
  float best_ms = 1e30f;
  int best = cand[0];
  cudaEvent_t e0, e1;
  KRP_CUDA_CHECK(cudaEventCreate(&e0));
  KRP_CUDA_CHECK(cudaEventCreate(&e1));
  // factors and their row tables for the sketch
  launch_gen_factors_batch(P.d_fjobs, P.d_fstart, 3 * P.count, P.fblocks);
  batch_rows_kernel<<<dim3(P.count, 3), 256, 0, stream()>>>(P.d_items, 0);
  check_launch("batch_rows");
  for (int spu : cand) {
    build_sketch_units(P.h_items, spu, units);
    P.nsunits = (int)units.size();
    KRP_CUDA_CHECK(cudaMemcpyAsync(P.d_sunits, units.data(), sizeof(SkUnit) * units.size(),
                                   cudaMemcpyHostToDevice, stream()));
    float ms_sum = 0.f;
    for (int rep = 0; rep < 2; ++rep) {
      KRP_CUDA_CHECK(cudaMemsetAsync(P.d_counters, 0, 3 * sizeof(int), stream()));
      KRP_CUDA_CHECK(cudaMemsetAsync(P.y_begin, 0, P.y_bytes, stream()));
      KRP_CUDA_CHECK(cudaEventRecord(e0, stream()));
      launch_sketch(P);
      KRP_CUDA_CHECK(cudaEventRecord(e1, stream()));
      KRP_CUDA_CHECK(cudaEventSynchronize(e1));
      float ms = 0.f;
      KRP_CUDA_CHECK(cudaEventElapsedTime(&ms, e0, e1));
      if (rep) ms_sum += ms;
    }
    if (ms_sum < best_ms) {
      best_ms = ms_sum;
      best = spu;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  P.slabs_per_unit = best;
  build_sketch_units(P.h_items, best, units);
  P.nsunits = (int)units.size();
  KRP_CUDA_CHECK(cudaMemcpyAsync(P.d_sunits, units.data(), sizeof(SkUnit) * units.size(),
                                 cudaMemcpyHostToDevice, stream()));
  KRP_CUDA_CHECK(cudaStreamSynchronize(stream()));
}

// Temporarily direct the context's launches to another stream.
struct StreamSwap {
  Ctx* c;
  cudaStream_t saved;
  StreamSwap(Ctx* ctx, cudaStream_t s) : c(ctx), saved(ctx->stream) { c->stream = s; }
  ~StreamSwap() { c->stream = saved; }
};

void capture(TbPlan& P, Ctx* c) {
  cudaGraph_t g = nullptr;
  const uint64_t launches = c->launches;  // captured kernels do not run here
  StreamSwap sw(c, P.cs);
  KRP_CUDA_CHECK(cudaStreamBeginCapture(P.cs, cudaStreamCaptureModeRelaxed));
  try {
    enqueue_all(P, c->d_status);
  } catch (...) {
    cudaStreamEndCapture(P.cs, &g);
    if (g) cudaGraphDestroy(g);
    throw;
  }
  KRP_CUDA_CHECK(cudaStreamEndCapture(P.cs, &g));
  c->launches = launches;
  const cudaError_t e = cudaGraphInstantiate(&P.exec, g, 0);
  cudaGraphDestroy(g);
  KRP_CUDA_CHECK(e);
}

void plan_free(void* p) { delete static_cast<TbPlan*>(p); }

// ======================================================= block Hankel ======
// Alg. 6 for many block Hankel matrices, one launch per phase over the batch
// (same arithmetic as the single-matrix pipeline: structured sketches in
// FP32, FP64 Householder QR, structured Psi^T Q, least squares, Gram + FP64
// eigensolver, output vectors).
struct HbItem {
  const void* blocks;  // 2s-1 column-major m x n blocks
  int m, n, s, r, lr, ll;
  float* o1;           // s x lr   (tag Omega, factor 0)
  float* o2;           // n x lr   (tag Omega, factor 1)
  float* p1;           // s x ll   (tag Psi, factor 0)
  float* p2;           // m x ll   (tag Psi, factor 1)
  float* Zy;           // (2s-1) blocks of m x lr:  H_k Omega2
  float* Zz;           // (2s-1) blocks of n x ll:  H_k^T Psi2
  float* Y;            // ms x lr
  float* Z;            // ns x ll
  double* Q;           // ms x lr
  double* P;           // ll x lr
  double* Qp;          // ll x lr
  double* Rp;          // lr x lr
  double* W;           // lr x ns
  double* Sg;          // lr x lr
  double* Uw;          // lr x lr
  double* ev;          // lr
  double* U;           // out: ms x r
  double* S;           // out: r
  double* V;           // out: ns x r
};

template <class BT>
__device__ __forceinline__ float ldb(const BT* p, int64_t i);
template <>
__device__ __forceinline__ float ldb<float>(const float* p, int64_t i) { return p[i]; }
template <>
__device__ __forceinline__ float ldb<__nv_bfloat16>(const __nv_bfloat16* p, int64_t i) {
  return __bfloat162float(p[i]);
}

// Z-blocks of both sketches: grid (x: element chunks, y: item, z: 0 = Y, 1 = Z)
//   Zy[a + m (c + lr k)] = sum_b H_k[a, b] Omega2[b, c]
//   Zz[b + n (c + ll k)] = sum_a H_k[a, b] Psi2[a, c]
template <class BT>
__global__ void hb_blockmul_kernel(const HbItem* __restrict__ items) {
  const HbItem& it = items[blockIdx.y];
  const bool tz = blockIdx.z == 1;
  const int m = it.m, n = it.n, nb = 2 * it.s - 1;
  const int mo = tz ? n : m, ki = tz ? m : n, ell = tz ? it.ll : it.lr;
  const float* F2 = tz ? it.p2 : it.o2;
  float* Zs = tz ? it.Zz : it.Zy;
  const BT* B = static_cast<const BT*>(it.blocks);
  const int64_t total = (int64_t)mo * ell * nb;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(e % mo);
    const int c = (int)((e / mo) % ell);
    const int k = (int)(e / ((int64_t)mo * ell));
    const BT* H = B + (int64_t)m * n * k;
    float acc = 0.f;
    for (int b = 0; b < ki; ++b) {
      const float h = tz ? ldb(H, b + (int64_t)m * a) : ldb(H, a + (int64_t)m * b);
      acc = fmaf(h, F2[b + (int64_t)ki * c], acc);
    }
    Zs[e] = acc;
  }
}

// Y[(a + mo i) + mo s c] = sum_{j<s} F1[j + s c] Zs[a + mo (c + ell (i + j))]
__global__ void hb_corr_kernel(const HbItem* __restrict__ items) {
  const HbItem& it = items[blockIdx.y];
  const bool tz = blockIdx.z == 1;
  const int s = it.s, mo = tz ? it.n : it.m, ell = tz ? it.ll : it.lr;
  const float* F1 = tz ? it.p1 : it.o1;
  const float* Zs = tz ? it.Zz : it.Zy;
  float* out = tz ? it.Z : it.Y;
  const int64_t total = (int64_t)mo * s * ell;
  const int64_t zstride = (int64_t)mo * ell;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(e % mo);
    const int i = (int)((e / mo) % s);
    const int c = (int)(e / ((int64_t)mo * s));
    const float* z = Zs + a + (int64_t)mo * c;
    float acc = 0.f;
    for (int j = 0; j < s; ++j) acc = fmaf(F1[j + (int64_t)s * c], z[zstride * (i + j)], acc);
    out[e] = acc;
  }
}

// P[c + ll q] = sum_{i, a} Psi1[i, c] Psi2[a, c] Q[(a + m i) + ms q]; grid (ll_max, count).
// The weights w[row] = Psi1[i, c] Psi2[a, c] are formed once per chunk of
// kHbRows rows in shared memory (FP64), so each term is one FP64 FMA; warp w
// keeps the sums of columns q = w, w + 8, ... (lr <= 64) in registers.
constexpr int kHbRows = 2048;
__global__ void __launch_bounds__(256) hb_psitq_kernel(const HbItem* __restrict__ items) {
  __shared__ double wsh[kHbRows];
  const HbItem& it = items[blockIdx.y];
  const int c = blockIdx.x;
  if (c >= it.ll) return;
  const int m = it.m, s = it.s, lr = it.lr;
  const int64_t ms = (int64_t)m * s;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double acc[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) acc[k] = 0.0;
  for (int64_t r0 = 0; r0 < ms; r0 += kHbRows) {
    const int nr = (int)((ms - r0) < kHbRows ? (ms - r0) : kHbRows);
    __syncthreads();  // the previous chunk has been read
    for (int rr = threadIdx.x; rr < nr; rr += blockDim.x) {
      const int64_t row = r0 + rr;
      const int a = (int)(row % m), i = (int)(row / m);
      wsh[rr] = (double)it.p1[i + (int64_t)s * c] * (double)it.p2[a + (int64_t)m * c];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int q = warp + 8 * k;
      if (q < lr) {
        const double* qc = it.Q + ms * q + r0;
        for (int rr = lane; rr < nr; rr += 32) acc[k] = fma(wsh[rr], qc[rr], acc[k]);
      }
    }
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int q = warp + 8 * k;
    double v = acc[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0 && q < lr) it.P[c + (int64_t)it.ll * q] = v;
  }
}

// W[q + lr col] = (Rp^{-1} Qp^T Z^T)[q, col]: grid (x: column chunks, y: item);
// a CTA's 64 columns of Z are converted to FP64 once, in shared memory.
constexpr int kHbLsCols = 64;
__global__ void __launch_bounds__(kHbLsCols) hb_ls_kernel(const HbItem* __restrict__ items) {
  extern __shared__ double zsh[];  // ll x kHbLsCols
  const HbItem& it = items[blockIdx.y];
  const int ll = it.ll, lr = it.lr;
  const int64_t ns = (int64_t)it.n * it.s;
  for (int64_t c0 = blockIdx.x * (int64_t)kHbLsCols; c0 < ns; c0 += (int64_t)gridDim.x * kHbLsCols) {
    __syncthreads();  // the previous chunk's columns have been read
    for (int c = 0; c < ll; ++c) {
      const int64_t col = c0 + threadIdx.x;
      zsh[c * kHbLsCols + threadIdx.x] = col < ns ? (double)it.Z[col + ns * c] : 0.0;
    }
    __syncthreads();
    const int64_t col = c0 + threadIdx.x;
    if (col >= ns) continue;
    double* w = it.W + (int64_t)lr * col;
    for (int q = 0; q < lr; ++q) {
      double acc = 0.0;
      const double* qp = it.Qp + (int64_t)ll * q;
      for (int c = 0; c < ll; ++c) acc = fma(qp[c], zsh[c * kHbLsCols + threadIdx.x], acc);
      w[q] = acc;
    }
    for (int q = lr - 1; q >= 0; --q) {
      double acc = w[q];
      for (int t = q + 1; t < lr; ++t) acc -= it.Rp[q + (int64_t)lr * t] * w[t];
      w[q] = acc / it.Rp[q + (int64_t)lr * q];
    }
  }
}

// Sg = W W^T (lr x lr, FP64) over column chunks: grid (x: chunks of
// kHbGramCols columns, y: item); a CTA stages its W columns in shared memory
// and adds its partial Gram (pairs p <= q) atomically into Sg, which
// hb_zero_kernel has cleared.
constexpr int kHbGramCols = 64;
__global__ void hb_zero_kernel(const HbItem* __restrict__ items) {
  const HbItem& it = items[blockIdx.x];
  for (int e = threadIdx.x; e < it.lr * it.lr; e += blockDim.x) it.Sg[e] = 0.0;
}
__global__ void hb_gram_kernel(const HbItem* __restrict__ items) {
  extern __shared__ double wt[];  // lr x kHbGramCols
  const HbItem& it = items[blockIdx.y];
  const int lr = it.lr;
  const int64_t ns = (int64_t)it.n * it.s;
  const int64_t c0 = (int64_t)blockIdx.x * kHbGramCols;
  if (c0 >= ns) return;
  const int nc = (int)((ns - c0) < kHbGramCols ? (ns - c0) : kHbGramCols);
  for (int e = threadIdx.x; e < lr * nc; e += blockDim.x) wt[e] = it.W[e + (int64_t)lr * c0];
  __syncthreads();
  const int npairs = lr * (lr + 1) / 2;
  for (int pq = threadIdx.x; pq < npairs; pq += blockDim.x) {
    int q = (int)((sqrtf(8.f * pq + 1.f) - 1.f) * 0.5f);
    while (q * (q + 1) / 2 > pq) --q;
    while ((q + 1) * (q + 2) / 2 <= pq) ++q;
    const int p = pq - q * (q + 1) / 2;
    double acc = 0.0;
    for (int col = 0; col < nc; ++col) acc = fma(wt[p + lr * col], wt[q + lr * col], acc);
    atomicAdd(&it.Sg[p + lr * q], acc);
    if (p != q) atomicAdd(&it.Sg[q + lr * p], acc);
  }
}

// U = Q Uw[:, :r], V = W^T Uw[:, :r] / sigma, S = sigma; grid (x: chunks, y: item)
__global__ void hb_out_kernel(const HbItem* __restrict__ items) {
  const HbItem& it = items[blockIdx.y];
  const int lr = it.lr, r = it.r;
  const int64_t ms = (int64_t)it.m * it.s, ns = (int64_t)it.n * it.s;
  const int64_t nu = ms * r, total = nu + ns * r;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (e < nu) {
      const int64_t row = e % ms;
      const int j = (int)(e / ms);
      double acc = 0.0;
      for (int q = 0; q < lr; ++q) acc = fma(it.Q[row + ms * q], it.Uw[q + (int64_t)lr * j], acc);
      it.U[e] = acc;
    } else {
      const int64_t f = e - nu;
      const int64_t col = f % ns;
      const int j = (int)(f / ns);
      const double sig = sqrt(fmax(it.ev[j], 0.0));
      double acc = 0.0;
      for (int q = 0; q < lr; ++q) acc = fma(it.W[q + (int64_t)lr * col], it.Uw[q + (int64_t)lr * j], acc);
      it.V[f] = sig > 0.0 ? acc / sig : 0.0;
      if (col == 0) it.S[j] = sig;
    }
  }
}

struct HbPlan {
  krp_dtype bt{};
  int count = 0;
  std::vector<krp_hankel_item> sig;
  char* arena = nullptr;
  HbItem* d_items = nullptr;
  BatchFactorJob* d_fjobs = nullptr;
  int64_t* d_fstart = nullptr;
  int64_t fblocks = 0;
  QrJob* d_qy = nullptr;
  QrJob* d_qp = nullptr;
  void* cqr_mem[2] = {nullptr, nullptr};
  CqrJobsPlan cqr_y, cqr_p;
  EigJob* d_ej = nullptr;
  int gx_blockmul = 1, gx_corr = 1, gx_ls = 1, gx_out = 1, gx_gram = 1, llmax = 1, lrmax = 1;
  size_t sm_ls = 0, sm_gram = 0;
  int kernels_per_run = 0;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cs = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  ~HbPlan() {
    for (void* m : cqr_mem)
      if (m) cudaFree(m);
    if (exec) cudaGraphExecDestroy(exec);
    if (ev_in) cudaEventDestroy(ev_in);
    if (ev_out) cudaEventDestroy(ev_out);
    if (cs) cudaStreamDestroy(cs);
    if (arena) cudaFree(arena);
  }
};

bool hb_same(const HbPlan& p, krp_dtype bt, int count, const krp_hankel_item* items) {
  if (p.bt != bt || p.count != count) return false;
  return std::memcmp(p.sig.data(), items, sizeof(krp_hankel_item) * count) == 0;
}

int chunks_for(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 1024)); }

void hb_enqueue(HbPlan& P, int* status) {
  int nk = 0;
  launch_gen_factors_batch(P.d_fjobs, P.d_fstart, 4 * P.count, P.fblocks);
  ++nk;
  if (P.bt == KRP_F32)
    hb_blockmul_kernel<float><<<dim3(P.gx_blockmul, P.count, 2), 256, 0, stream()>>>(P.d_items);
  else
    hb_blockmul_kernel<__nv_bfloat16><<<dim3(P.gx_blockmul, P.count, 2), 256, 0, stream()>>>(
        P.d_items);
  check_launch("hb_blockmul");
  hb_corr_kernel<<<dim3(P.gx_corr, P.count, 2), 256, 0, stream()>>>(P.d_items);
  check_launch("hb_corr");
  nk += cholqr3_jobs_launch(P.cqr_y, status);
  hb_psitq_kernel<<<dim3(P.llmax, P.count), 256, 0, stream()>>>(P.d_items);
  check_launch("hb_psitq");
  nk += cholqr3_jobs_launch(P.cqr_p, status);
  hb_ls_kernel<<<dim3(P.gx_ls, P.count), kHbLsCols, P.sm_ls, stream()>>>(P.d_items);
  check_launch("hb_ls");
  hb_zero_kernel<<<P.count, 256, 0, stream()>>>(P.d_items);
  check_launch("hb_zero");
  hb_gram_kernel<<<dim3(P.gx_gram, P.count), 256, P.sm_gram, stream()>>>(P.d_items);
  check_launch("hb_gram");
  eig_launch(P.d_ej, P.count, P.lrmax, status);
  hb_out_kernel<<<dim3(P.gx_out, P.count), 256, 0, stream()>>>(P.d_items);
  check_launch("hb_out");
  nk += 8;
  P.kernels_per_run = nk;
}

std::unique_ptr<HbPlan> hb_build(Ctx* c, krp_dtype bt, int count, const krp_hankel_item* items) {
  auto P = std::make_unique<HbPlan>();
  P->bt = bt;
  P->count = count;
  P->sig.assign(items, items + count);
  size_t bytes = 0;
  auto add = [&](size_t n, size_t e) { bytes += (n * e + 255) & ~size_t(255); };
  for (int b = 0; b < count; ++b) {
    const krp_hankel_item& h = items[b];
    const size_t ms = (size_t)h.m * h.s, ns = (size_t)h.n * h.s, nb = 2 * (size_t)h.s - 1;
    const size_t lr = h.ell_r, ll = h.ell_l;
    add((size_t)h.s * lr, 4); add((size_t)h.n * lr, 4); add((size_t)h.s * ll, 4); add((size_t)h.m * ll, 4);
    add(nb * h.m * lr, 4); add(nb * h.n * ll, 4);
    add(ms * lr, 4); add(ns * ll, 4);
    add(ms * lr, 8); add(ms * lr, 8);          // Q, QR work
    add(ll * lr, 8); add(ll * lr, 8); add(ll * lr, 8); add(lr * lr, 8);  // P, Qp, QR work, Rp
    add(lr * ns, 8); add(lr * lr, 8); add(lr * lr, 8); add(lr, 8);        // W, Sg, Uw, ev
  }
  add(count, sizeof(HbItem));
  add((size_t)4 * count, sizeof(BatchFactorJob));
  add((size_t)4 * count + 1, 8);
  add(count, sizeof(QrJob));
  add(count, sizeof(QrJob));
  add(count, sizeof(EigJob));
  KRP_CUDA_CHECK(cudaStreamCreateWithFlags(&P->cs, cudaStreamNonBlocking));
  KRP_CUDA_CHECK(cudaEventCreateWithFlags(&P->ev_in, cudaEventDisableTiming));
  KRP_CUDA_CHECK(cudaEventCreateWithFlags(&P->ev_out, cudaEventDisableTiming));
  KRP_CUDA_CHECK(cudaMalloc(&P->arena, bytes));
  char* p = P->arena;
  std::vector<HbItem> hi(count);
  std::vector<BatchFactorJob> fj;
  std::vector<int64_t> fstart(1, 0);
  std::vector<QrJob> qy, qp;
  std::vector<EigJob> ej;
  int64_t maxbm = 1, maxcorr = 1, maxns = 1, maxout = 1;
  for (int b = 0; b < count; ++b) {
    const krp_hankel_item& h = items[b];
    HbItem& it = hi[b];
    it.blocks = h.blocks;
    it.m = h.m; it.n = h.n; it.s = h.s; it.r = h.r; it.lr = h.ell_r; it.ll = h.ell_l;
    const int64_t ms = (int64_t)h.m * h.s, ns = (int64_t)h.n * h.s, nb = 2 * (int64_t)h.s - 1;
    it.o1 = carve<float>(p, (size_t)h.s * it.lr);
    it.o2 = carve<float>(p, (size_t)h.n * it.lr);
    it.p1 = carve<float>(p, (size_t)h.s * it.ll);
    it.p2 = carve<float>(p, (size_t)h.m * it.ll);
    it.Zy = carve<float>(p, (size_t)nb * h.m * it.lr);
    it.Zz = carve<float>(p, (size_t)nb * h.n * it.ll);
    it.Y = carve<float>(p, (size_t)ms * it.lr);
    it.Z = carve<float>(p, (size_t)ns * it.ll);
    it.Q = carve<double>(p, (size_t)ms * it.lr);
    double* qwork = carve<double>(p, (size_t)ms * it.lr);
    it.P = carve<double>(p, (size_t)it.ll * it.lr);
    it.Qp = carve<double>(p, (size_t)it.ll * it.lr);
    double* pwork = carve<double>(p, (size_t)it.ll * it.lr);
    it.Rp = carve<double>(p, (size_t)it.lr * it.lr);
    it.W = carve<double>(p, (size_t)it.lr * ns);
    it.Sg = carve<double>(p, (size_t)it.lr * it.lr);
    it.Uw = carve<double>(p, (size_t)it.lr * it.lr);
    it.ev = carve<double>(p, (size_t)it.lr);
    it.U = h.U; it.S = h.S; it.V = h.V;
    // factors: Omega1 (s x lr, factor 0), Omega2 (n x lr, factor 1) with tag
    // Omega; Psi1 (s x ll), Psi2 (m x ll) with tag Psi; draw 0, key = seed
    struct F { float* ptr; int64_t rows; uint32_t factor, tag; int ell; };
    const F fs[4] = {{it.o1, h.s, 0, KRP_TAG_OMEGA, it.lr}, {it.o2, h.n, 1, KRP_TAG_OMEGA, it.lr},
                     {it.p1, h.s, 0, KRP_TAG_PSI, it.ll}, {it.p2, h.m, 1, KRP_TAG_PSI, it.ll}};
    for (const F& f : fs) {
      BatchFactorJob j{};
      j.ptr = f.ptr; j.rows = f.rows; j.seed = h.seed; j.factor = f.factor; j.draw = 0;
      j.tag = f.tag; j.ell = f.ell; j.bf16_round = bt == KRP_BF16 ? 1 : 0;
      fj.push_back(j);
      fstart.push_back(fstart.back() + (f.rows * f.ell + 3) / 4);
    }
    QrJob a{};
    a.Y = it.Y; a.Q = it.Q; a.R = nullptr; a.work = qwork; a.m = ms; a.l = it.lr;
    qy.push_back(a);
    QrJob pq{};
    pq.Y = nullptr; pq.Y64 = it.P; pq.Q = it.Qp; pq.R = it.Rp; pq.work = pwork; pq.m = it.ll; pq.l = it.lr;
    qp.push_back(pq);
    ej.push_back(EigJob{it.Sg, it.Uw, it.ev, it.lr, it.lr});
    maxbm = std::max<int64_t>(maxbm, std::max<int64_t>(nb * h.m * it.lr, nb * h.n * it.ll));
    maxcorr = std::max<int64_t>(maxcorr, std::max<int64_t>(ms * it.lr, ns * it.ll));
    maxns = std::max<int64_t>(maxns, ns);
    maxout = std::max<int64_t>(maxout, (ms + ns) * h.r);
    P->llmax = std::max(P->llmax, it.ll);
    P->lrmax = std::max(P->lrmax, it.lr);
  }
  P->d_items = carve<HbItem>(p, count);
  P->d_fjobs = carve<BatchFactorJob>(p, (size_t)4 * count);
  P->d_fstart = carve<int64_t>(p, (size_t)4 * count + 1);
  P->d_qy = carve<QrJob>(p, count);
  P->d_qp = carve<QrJob>(p, count);
  P->d_ej = carve<EigJob>(p, count);
  KRP_REQUIRE((size_t)(p - P->arena) <= bytes, "Hankel batch arena overflow");
  P->fblocks = fstart.back();
  P->gx_blockmul = chunks_for(maxbm);
  P->gx_corr = chunks_for(maxcorr);
  P->gx_ls = (int)std::min<int64_t>((maxns + kHbLsCols - 1) / kHbLsCols, 1024);
  P->gx_out = chunks_for(maxout);
  P->gx_gram = (int)((maxns + kHbGramCols - 1) / kHbGramCols);
  {
    P->sm_ls = sizeof(double) * (size_t)P->llmax * kHbLsCols;
    P->sm_gram = sizeof(double) * (size_t)P->lrmax * kHbGramCols;
    KRP_CUDA_CHECK(cudaFuncSetAttribute(hb_ls_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)P->sm_ls));
    KRP_CUDA_CHECK(cudaFuncSetAttribute(hb_gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)P->sm_gram));
  }
  cudaStream_t s = c->stream;
  KRP_CUDA_CHECK(cudaMemcpyAsync(P->d_items, hi.data(), sizeof(HbItem) * count, cudaMemcpyHostToDevice, s));
  KRP_CUDA_CHECK(cudaMemcpyAsync(P->d_fjobs, fj.data(), sizeof(BatchFactorJob) * fj.size(), cudaMemcpyHostToDevice, s));
  KRP_CUDA_CHECK(cudaMemcpyAsync(P->d_fstart, fstart.data(), sizeof(int64_t) * fstart.size(), cudaMemcpyHostToDevice, s));
  KRP_CUDA_CHECK(cudaMemcpyAsync(P->d_qy, qy.data(), sizeof(QrJob) * count, cudaMemcpyHostToDevice, s));
  KRP_CUDA_CHECK(cudaMemcpyAsync(P->d_qp, qp.data(), sizeof(QrJob) * count, cudaMemcpyHostToDevice, s));
  KRP_CUDA_CHECK(cudaMalloc(&P->cqr_mem[0], cholqr3_jobs_bytes(qy.data(), count)));
  KRP_CUDA_CHECK(cudaMalloc(&P->cqr_mem[1], cholqr3_jobs_bytes(qp.data(), count)));
  P->cqr_y = cholqr3_jobs_setup(qy.data(), count, P->cqr_mem[0], s);
  P->cqr_p = cholqr3_jobs_setup(qp.data(), count, P->cqr_mem[1], s);
  KRP_CUDA_CHECK(cudaMemcpyAsync(P->d_ej, ej.data(), sizeof(EigJob) * count, cudaMemcpyHostToDevice, s));
  KRP_CUDA_CHECK(cudaStreamSynchronize(s));
  return P;
}

void hb_plan_free(void* p) { delete static_cast<HbPlan*>(p); }

}  // namespace

void tucker_batched(krp_dtype xt, int count, krp_tucker_item* items, int oversample,
                    unsigned flags) {
  Ctx* c = current();
  KRP_REQUIRE(count >= 1, "count must be >= 1");
  KRP_REQUIRE(items, "items is NULL");
  KRP_REQUIRE(xt == KRP_F32 || xt == KRP_BF16, "X dtype must be KRP_F32 or KRP_BF16");
  KRP_REQUIRE(oversample >= 0, "oversample must be >= 0");
  KRP_REQUIRE(!(flags & ~(unsigned)(KRP_MEMO | KRP_TRUNCATE | KRP_RESIDUAL)),
              "batched flags: KRP_MEMO, KRP_TRUNCATE, KRP_RESIDUAL");
  for (int b = 0; b < count; ++b) {
    const krp_tucker_item& it = items[b];
    KRP_REQUIRE(it.X && is_device_ptr(it.X), "item %d: X must be a device pointer", b);
    KRP_REQUIRE(it.core && is_device_ptr(it.core), "item %d: core must be a device pointer", b);
    for (int m = 0; m < 3; ++m) {
      KRP_REQUIRE(it.dims[m] >= 1 && it.dims[m] <= kMaxSide, "item %d: n_%d = %lld out of 1..%d",
                  b, m, (long long)it.dims[m], kMaxSide);
      const int l = it.ranks[m] + oversample;
      KRP_REQUIRE(it.ranks[m] >= 1 && l <= kMaxEll && l <= it.dims[m],
                  "item %d: l_%d = %d must be <= min(%d, n_%d)", b, m, l, kMaxEll, m);
      KRP_REQUIRE(it.factors[m] && is_device_ptr(it.factors[m]),
                  "item %d: factors[%d] must be a device pointer", b, m);
    }
    if (xt == KRP_BF16)
      KRP_REQUIRE((reinterpret_cast<uintptr_t>(it.X) & 1) == 0, "item %d: X misaligned", b);
  }
  flags |= KRP_MEMO;  // the batched path draws one factor set per tensor
  TbPlan* P = static_cast<TbPlan*>(c->batch_plan);
  if (!P || !same_signature(*P, xt, count, items, oversample, flags)) {
    if (c->batch_plan) c->batch_plan_free(c->batch_plan);
    c->batch_plan = nullptr;
    std::unique_ptr<TbPlan> np = build_plan(c, xt, count, items, oversample, flags);
    autotune(*np);
    // one eager run (validates the sequence), then the graph
    enqueue_all(*np, c->d_status);
    KRP_CUDA_CHECK(cudaStreamSynchronize(c->stream));
    raise_device_status(c);
    capture(*np, c);
    P = np.release();
    c->batch_plan = P;
    c->batch_plan_free = plan_free;
  }
  KRP_CUDA_CHECK(cudaEventRecord(P->ev_in, c->stream));
  KRP_CUDA_CHECK(cudaStreamWaitEvent(P->cs, P->ev_in, 0));
  KRP_CUDA_CHECK(cudaGraphLaunch(P->exec, P->cs));
  KRP_CUDA_CHECK(cudaEventRecord(P->ev_out, P->cs));
  KRP_CUDA_CHECK(cudaStreamWaitEvent(c->stream, P->ev_out, 0));
  c->launches += P->kernels_per_run;
  KRP_CUDA_CHECK(cudaStreamSynchronize(P->cs));
  raise_device_status(c);
  for (int b = 0; b < count; ++b)
    items[b].rel_residual = (flags & KRP_RESIDUAL) ? P->h_rel[b] : -1.0;
}

int tucker_batched_plan_info(int* slabs_per_unit, int* units, int* grid) {
  TbPlan* P = static_cast<TbPlan*>(current()->batch_plan);
  if (!P) return 0;
  if (slabs_per_unit) *slabs_per_unit = P->slabs_per_unit;
  if (units) *units = P->nsunits;
  if (grid) *grid = P->grid_sketch;
  return 1;
}

void hankel_batched(krp_dtype bt, int count, krp_hankel_item* items) {
  Ctx* c = current();
  KRP_REQUIRE(count >= 1, "count must be >= 1");
  KRP_REQUIRE(items, "items is NULL");
  KRP_REQUIRE(bt == KRP_F32 || bt == KRP_BF16, "blocks dtype must be KRP_F32 or KRP_BF16");
  for (int b = 0; b < count; ++b) {
    krp_hankel_item& h = items[b];
    if (h.ell_l == 0) h.ell_l = (int)std::ceil(1.5 * h.ell_r);
    KRP_REQUIRE(h.blocks && is_device_ptr(h.blocks), "item %d: blocks must be a device pointer", b);
    KRP_REQUIRE(h.m >= 1 && h.n >= 1 && h.s >= 1, "item %d: m, n, s must be >= 1", b);
    KRP_REQUIRE(h.r >= 1 && h.r <= h.ell_r && h.ell_r <= h.ell_l && h.ell_r <= 64 &&
                    h.ell_l <= 256,
                "item %d: need 1 <= r <= ell_r <= ell_l, ell_r <= 64, ell_l <= 256", b);
    KRP_REQUIRE((int64_t)h.ell_r <= (int64_t)h.m * h.s && (int64_t)h.ell_l <= (int64_t)h.n * h.s,
                "item %d: sketch sizes exceed the matrix", b);
    KRP_REQUIRE(h.U && h.S && h.V && is_device_ptr(h.U) && is_device_ptr(h.S) && is_device_ptr(h.V),
                "item %d: U, S, V must be device pointers", b);
  }
  HbPlan* P = static_cast<HbPlan*>(c->hankel_plan);
  if (!P || !hb_same(*P, bt, count, items)) {
    if (c->hankel_plan) c->hankel_plan_free(c->hankel_plan);
    c->hankel_plan = nullptr;
    std::unique_ptr<HbPlan> np = hb_build(c, bt, count, items);
    KRP_CUDA_CHECK(cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream));
    hb_enqueue(*np, c->d_status);  // eager run: validates the sequence
    raise_device_status(c);
    cudaGraph_t g = nullptr;
    const uint64_t launches = c->launches;
    {
      StreamSwap sw(c, np->cs);
      KRP_CUDA_CHECK(cudaStreamBeginCapture(np->cs, cudaStreamCaptureModeRelaxed));
      try {
        hb_enqueue(*np, c->d_status);
      } catch (...) {
        cudaStreamEndCapture(np->cs, &g);
        if (g) cudaGraphDestroy(g);
        throw;
      }
      KRP_CUDA_CHECK(cudaStreamEndCapture(np->cs, &g));
    }
    c->launches = launches;
    const cudaError_t e = cudaGraphInstantiate(&np->exec, g, 0);
    cudaGraphDestroy(g);
    KRP_CUDA_CHECK(e);
    P = np.release();
    c->hankel_plan = P;
    c->hankel_plan_free = hb_plan_free;
  }
  KRP_CUDA_CHECK(cudaEventRecord(P->ev_in, c->stream));
  KRP_CUDA_CHECK(cudaStreamWaitEvent(P->cs, P->ev_in, 0));
  KRP_CUDA_CHECK(cudaGraphLaunch(P->exec, P->cs));
  KRP_CUDA_CHECK(cudaEventRecord(P->ev_out, P->cs));
  KRP_CUDA_CHECK(cudaStreamWaitEvent(c->stream, P->ev_out, 0));
  c->launches += P->kernels_per_run;
  raise_device_status(c);
}

}  // namespace krp
