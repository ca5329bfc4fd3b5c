// a11: many small, uneven 3-way tensors in one launch per phase.
//
// RHOSVD-KRP-MEMO (Alg. 7 with one factor set, Sec. 5.1) of every tensor of a
// batch.  Each phase is one kernel launch over the whole batch:
//   factors     one Philox launch over all (tensor, mode) factors
//   sketch      persistent kernel over (tensor, slab range) work tiles: for a
//               mode-3 slab X_t (n1 x n2) it forms A_t = X_t Om2 and
//               B_t = X_t^T Om1 and accumulates Y1 += A_t diag(Om3[t,:]),
//               Y2 += B_t diag(Om3[t,:]), Y3[t,:] = colsum(Om1 * A_t): all
//               three mode sketches from one pass over X (the dimension tree
//               of Sec. 5.1, 4 N l flops)
//   QR          one CTA per (tensor, mode), FP64 Householder
//   core        persistent kernel over the same tiles: C_t = Q1^T X_t Q2,
//               then G(:,:,c) = sum_t C_t Q3[t,c] in a per-tensor kernel
//   truncation  FP64 Gram matrices of the core unfoldings, the eigensolver
//               on all 3 x count of them, then G x {U_i^T}, Q_i U_i
//   residual    persistent kernel: ||X_t - Q1 (sum_c G(:,:,c) Q3[t,c]) Q2^T||^2
//               with FP64 sums per tensor
// The tiles are sorted by work (largest first) and handed out by an atomic
// counter.  The slabs-per-tile granularity is picked once per batch by timing
// the sketch phase for a few candidates.  The whole sequence is captured in a
// CUDA graph when the batch is first seen; a repeated call with the same
// descriptors replays the graph.  Products run on CUDA cores in FP32 with
// FP32 accumulation (the slabs are too small and too unevenly shaped for
// 128-row tensor-core tiles); X may be FP32 or BF16.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <vector>

#include "common.cuh"
#include "pipeline.h"

namespace krp {
namespace {

constexpr int kBT = 256;              // threads of the slab kernels
constexpr int kMaxSide = 256;         // n_i
constexpr int kMaxEll = 32;           // l_i
constexpr int kJB = 32;               // slab columns per staged chunk
constexpr int kRPT = kMaxSide / 32;   // rows per thread in the row mappings

struct TbItem {
  const void* X;
  int n[3];
  int l[3];
  int lm;            // memo factor width: max l_i
  int r[3];          // output sizes (r_i with truncation, l_i without)
  float* om[3];      // n_i x lm
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

// A chunk of columns j0 .. j0+kJB-1 of slab t, moved through registers so
// that all of a thread's loads are in flight together (and the next chunk's
// while the current one is multiplied): warp w holds rows jl = w + 8p of the
// chunk, lane l holds entries i = l + 32u (u < R = ceil(n1 / 32)); zero
// outside the slab.
template <int R>
struct ChunkRegs {
  float v[kJB / 8][R];
};

template <class XT, int R>
__device__ __forceinline__ void chunk_load(ChunkRegs<R>& r, const XT* X, int n1, int n2, int t,
                                           int j0) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int p = 0; p < kJB / 8; ++p) {
    const int j = j0 + warp + 8 * p;
    const bool jok = j < n2;
    const int64_t base = (int64_t)n1 * (j + (int64_t)n2 * t);
#pragma unroll
    for (int u = 0; u < R; ++u) {
      const int i = lane + 32 * u;
      r.v[p][u] = (jok && i < n1) ? ldx(X, base + i) : 0.f;
    }
  }
}

template <int R>
__device__ __forceinline__ void chunk_store(const ChunkRegs<R>& r, float* Xs, int pitch) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int p = 0; p < kJB / 8; ++p)
#pragma unroll
    for (int u = 0; u < R; ++u) Xs[(warp + 8 * p) * pitch + lane + 32 * u] = r.v[p][u];
}

// sum_i Xs[row][i] W[i][4kg..4kg+3] over i < n1p8, with two partial sums per
// output (even and odd groups of four i) for instruction-level parallelism;
// W rows n1..n1p8-1 and Xs entries beyond n1 are zero.
__device__ __forceinline__ float4 row_dot4(const float* Xrow, const float* W, int Lp, int kg,
                                           int n1p8) {
  float e0 = 0.f, e1 = 0.f, e2 = 0.f, e3 = 0.f, o0 = 0.f, o1 = 0.f, o2 = 0.f, o3 = 0.f;
  for (int i = 0; i < n1p8; i += 8) {
    const float4 xa = *reinterpret_cast<const float4*>(&Xrow[i]);
    const float4 xb = *reinterpret_cast<const float4*>(&Xrow[i + 4]);
    const float xva[4] = {xa.x, xa.y, xa.z, xa.w};
    const float xvb[4] = {xb.x, xb.y, xb.z, xb.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float4 wa = *reinterpret_cast<const float4*>(&W[(i + q) * Lp + 4 * kg]);
      const float4 wb = *reinterpret_cast<const float4*>(&W[(i + 4 + q) * Lp + 4 * kg]);
      e0 = fmaf(xva[q], wa.x, e0);
      e1 = fmaf(xva[q], wa.y, e1);
      e2 = fmaf(xva[q], wa.z, e2);
      e3 = fmaf(xva[q], wa.w, e3);
      o0 = fmaf(xvb[q], wb.x, o0);
      o1 = fmaf(xvb[q], wb.y, o1);
      o2 = fmaf(xvb[q], wb.z, o2);
      o3 = fmaf(xvb[q], wb.w, o3);
    }
  }
  return make_float4(e0 + o0, e1 + o1, e2 + o2, e3 + o3);
}

__device__ int next_tile(int* counter, int* s_tile) {
  __syncthreads();  // everyone is done with the previous tile's shared memory
  if (threadIdx.x == 0) *s_tile = atomicAdd(counter, 1);
  __syncthreads();
  return *s_tile;
}

// ---------------------------------------------------------------- sketch ----
// Shared memory (floats): Xs[kJB][pitch], O1s[n1max8][Lp], O2s[n2max][Lp],
// Y2p[n2max][Lp], o3s[Lp], y3s[Lp].
struct SketchSmem {
  float *Xs, *O1s, *O2s, *Y2p, *o3s, *y3s;
  int pitch, Lp;
};

template <class XT, int R>
__device__ void sketch_tile(const TbItem& it, const TbTile& tile, const SketchSmem& S) {
  const int tid = threadIdx.x, ig = tid >> 3, kg = tid & 7;
  const int n1 = it.n[0], n2 = it.n[1], n3 = it.n[2], lm = it.lm;
  const int pitch = S.pitch, Lp = S.Lp;
  const int n1p8 = (n1 + 7) & ~7;
  const XT* X = static_cast<const XT*>(it.X);
  // factors are column-major: consecutive threads read consecutive rows
  for (int e = tid; e < n1p8 * Lp; e += kBT) {
    const int i = e % n1p8, k = e / n1p8;
    S.O1s[i * Lp + k] = (i < n1 && k < lm) ? it.om[0][i + (int64_t)n1 * k] : 0.f;
  }
  for (int e = tid; e < n2 * Lp; e += kBT) {
    const int j = e % n2, k = e / n2;
    S.O2s[j * Lp + k] = k < lm ? it.om[1][j + (int64_t)n2 * k] : 0.f;
    S.Y2p[j * Lp + k] = 0.f;
  }
  float y1[R][4];
#pragma unroll
  for (int u = 0; u < R; ++u)
#pragma unroll
    for (int c = 0; c < 4; ++c) y1[u][c] = 0.f;
  const bool kact = 4 * kg < Lp;
  const int nch = (n2 + kJB - 1) / kJB;
  const int nq = (tile.t1 - tile.t0) * nch;
  ChunkRegs<R> cr;
  chunk_load<XT, R>(cr, X, n1, n2, tile.t0, 0);
  float a[R][4];
  for (int q = 0; q < nq; ++q) {
    const int t = tile.t0 + q / nch, ch = q % nch, j0 = ch * kJB;
    __syncthreads();  // previous chunk and slab epilogue consumed
    if (ch == 0) {
      if (tid < Lp) {
        S.o3s[tid] = tid < lm ? it.om[2][t + (int64_t)n3 * tid] : 0.f;
        S.y3s[tid] = 0.f;
      }
#pragma unroll
      for (int u = 0; u < R; ++u)
#pragma unroll
        for (int c = 0; c < 4; ++c) a[u][c] = 0.f;
    }
    chunk_store<R>(cr, S.Xs, pitch);
    __syncthreads();
    if (q + 1 < nq) chunk_load<XT, R>(cr, X, n1, n2, tile.t0 + (q + 1) / nch, ((q + 1) % nch) * kJB);
    const int jn = min(kJB, n2 - j0);
    if (kact) {
      // A_t rows ig + 32u, columns 4kg..4kg+3
      for (int jl = 0; jl < jn; ++jl) {
        const float4 w = *reinterpret_cast<const float4*>(&S.O2s[(j0 + jl) * Lp + 4 * kg]);
#pragma unroll
        for (int u = 0; u < R; ++u) {
          const float x = S.Xs[jl * pitch + ig + 32 * u];
          a[u][0] = fmaf(x, w.x, a[u][0]);
          a[u][1] = fmaf(x, w.y, a[u][1]);
          a[u][2] = fmaf(x, w.z, a[u][2]);
          a[u][3] = fmaf(x, w.w, a[u][3]);
        }
      }
      // B_t row j0 + ig (ig doubles as the chunk column here)
      if (ig < jn) {
        const float4 bb = row_dot4(&S.Xs[ig * pitch], S.O1s, Lp, kg, n1p8);
        float* yp = &S.Y2p[(j0 + ig) * Lp + 4 * kg];
        yp[0] = fmaf(bb.x, S.o3s[4 * kg + 0], yp[0]);
        yp[1] = fmaf(bb.y, S.o3s[4 * kg + 1], yp[1]);
        yp[2] = fmaf(bb.z, S.o3s[4 * kg + 2], yp[2]);
        yp[3] = fmaf(bb.w, S.o3s[4 * kg + 3], yp[3]);
      }
    }
    if (ch == nch - 1) {
      // slab t done: Y1 partial and Y3[t, :]
      float p[4] = {0.f, 0.f, 0.f, 0.f};
      if (kact) {
#pragma unroll
        for (int u = 0; u < R; ++u) {
          const int i = ig + 32 * u;
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            y1[u][c] = fmaf(a[u][c], S.o3s[4 * kg + c], y1[u][c]);
            if (i < n1) p[c] = fmaf(S.O1s[i * Lp + 4 * kg + c], a[u][c], p[c]);
          }
        }
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        p[c] += __shfl_xor_sync(0xffffffffu, p[c], 8);
        p[c] += __shfl_xor_sync(0xffffffffu, p[c], 16);
      }
      if ((tid & 31) < 8 && kact) {
#pragma unroll
        for (int c = 0; c < 4; ++c) atomicAdd(&S.y3s[4 * kg + c], p[c]);
      }
      __syncthreads();
      if (tid < lm) it.Y[2][t + (int64_t)n3 * tid] = S.y3s[tid];
    }
  }
  // flush the tile's partial Y2 and Y1 with row-contiguous (coalesced) atomics;
  // Y1 goes through shared memory (the Xs staging area, free by now)
  __syncthreads();
  for (int e = tid; e < n2 * lm; e += kBT) {
    const int j = e % n2, k = e / n2;
    atomicAdd(&it.Y[1][j + (int64_t)n2 * k], S.Y2p[j * Lp + k]);
  }
  float* Y1p = S.Xs;  // [k][i], n1 x Lp <= kJB * pitch floats
  if (kact) {
#pragma unroll
    for (int u = 0; u < R; ++u) {
      const int i = ig + 32 * u;
      if (i < n1) {
#pragma unroll
        for (int c = 0; c < 4; ++c) Y1p[(4 * kg + c) * n1 + i] = y1[u][c];
      }
    }
  }
  __syncthreads();
  for (int e = tid; e < n1 * lm; e += kBT) atomicAdd(&it.Y[0][e], Y1p[e]);
}

template <class XT>
__global__ void __launch_bounds__(kBT, 2)
    batch_sketch_kernel(const TbItem* __restrict__ items, const TbTile* __restrict__ tiles,
                        int ntiles, int* counter, int pitch, int Lp, int n1max8, int n2max) {
  extern __shared__ __align__(16) float bsm[];
  SketchSmem S;
  S.Xs = bsm;
  S.O1s = S.Xs + kJB * pitch;
  S.O2s = S.O1s + n1max8 * Lp;
  S.Y2p = S.O2s + n2max * Lp;
  S.o3s = S.Y2p + n2max * Lp;
  S.y3s = S.o3s + Lp;
  S.pitch = pitch;
  S.Lp = Lp;
  __shared__ int s_tile;
  for (;;) {
    const int ti = next_tile(counter, &s_tile);
    if (ti >= ntiles) break;
    const TbTile tile = tiles[ti];
    const TbItem& it = items[tile.item];
    switch ((it.n[0] + 31) >> 5) {  // uniform over the CTA
      case 1: sketch_tile<XT, 1>(it, tile, S); break;
      case 2: sketch_tile<XT, 2>(it, tile, S); break;
      case 3: sketch_tile<XT, 3>(it, tile, S); break;
      case 4: sketch_tile<XT, 4>(it, tile, S); break;
      case 5: sketch_tile<XT, 5>(it, tile, S); break;
      case 6: sketch_tile<XT, 6>(it, tile, S); break;
      case 7: sketch_tile<XT, 7>(it, tile, S); break;
      default: sketch_tile<XT, 8>(it, tile, S); break;
    }
  }
}

// ------------------------------------------------------------------ core ----
// C_t = Q1^T X_t Q2 (l1 x l2) for every slab of the tile.  Shared memory
// (floats): Xs[kJB][pitch], Q1s[n1max8][Lp], Q2s[n2max][Lp], Ts[kJB][Lp].
template <class XT, int R>
__device__ void core_tile(const TbItem& it, const TbTile& tile, float* Xs, float* Q1s, float* Q2s,
                          float* Ts, int pitch, int Lp) {
  const int tid = threadIdx.x, hi = tid >> 3, kg = tid & 7;
  const int n1 = it.n[0], n2 = it.n[1], l1 = it.l[0], l2 = it.l[1];
  const int n1p8 = (n1 + 7) & ~7;
  const XT* X = static_cast<const XT*>(it.X);
  for (int e = tid; e < n1p8 * Lp; e += kBT) {
    const int i = e % n1p8, a = e / n1p8;
    Q1s[i * Lp + a] = (i < n1 && a < l1) ? (float)it.Q[0][i + (int64_t)n1 * a] : 0.f;
  }
  for (int e = tid; e < n2 * Lp; e += kBT) {
    const int j = e % n2, b = e / n2;
    Q2s[j * Lp + b] = b < l2 ? (float)it.Q[1][j + (int64_t)n2 * b] : 0.f;
  }
  const bool kact = 4 * kg < Lp;
  const int nch = (n2 + kJB - 1) / kJB;
  const int nq = (tile.t1 - tile.t0) * nch;
  ChunkRegs<R> cr;
  chunk_load<XT, R>(cr, X, n1, n2, tile.t0, 0);
  // thread (a = hi, b = 4kg..4kg+3) of C_t
  float cacc[4];
  for (int q = 0; q < nq; ++q) {
    const int t = tile.t0 + q / nch, ch = q % nch, j0 = ch * kJB;
    if (ch == 0) cacc[0] = cacc[1] = cacc[2] = cacc[3] = 0.f;
    __syncthreads();
    chunk_store<R>(cr, Xs, pitch);
    __syncthreads();
    if (q + 1 < nq) chunk_load<XT, R>(cr, X, n1, n2, tile.t0 + (q + 1) / nch, ((q + 1) % nch) * kJB);
    const int jn = min(kJB, n2 - j0);
    // Ts[jl][a] = sum_i Xs[jl][i] Q1s[i][a]: thread (jl = hi, a = 4kg..)
    if (kact) {
      const float4 tv = hi < jn ? row_dot4(&Xs[hi * pitch], Q1s, Lp, kg, n1p8)
                                : make_float4(0.f, 0.f, 0.f, 0.f);
      *reinterpret_cast<float4*>(&Ts[hi * Lp + 4 * kg]) = tv;
    }
    __syncthreads();
    if (kact && hi < Lp) {
      for (int jl = 0; jl < jn; ++jl) {
        const float ta = Ts[jl * Lp + hi];
        const float4 w = *reinterpret_cast<const float4*>(&Q2s[(j0 + jl) * Lp + 4 * kg]);
        cacc[0] = fmaf(ta, w.x, cacc[0]);
        cacc[1] = fmaf(ta, w.y, cacc[1]);
        cacc[2] = fmaf(ta, w.z, cacc[2]);
        cacc[3] = fmaf(ta, w.w, cacc[3]);
      }
    }
    if (ch == nch - 1 && kact && hi < l1) {
      float* Ct = it.C + (int64_t)t * l1 * l2;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int b = 4 * kg + c;
        if (b < l2) Ct[hi + l1 * b] = cacc[c];
      }
    }
  }
}

template <class XT>
__global__ void __launch_bounds__(kBT, 2)
    batch_core_kernel(const TbItem* __restrict__ items, const TbTile* __restrict__ tiles,
                      int ntiles, int* counter, int pitch, int Lp, int n1max8, int n2max) {
  extern __shared__ __align__(16) float bsm[];
  float* Xs = bsm;
  float* Q1s = Xs + kJB * pitch;
  float* Q2s = Q1s + n1max8 * Lp;
  float* Ts = Q2s + n2max * Lp;
  __shared__ int s_tile;
  for (;;) {
    const int ti = next_tile(counter, &s_tile);
    if (ti >= ntiles) break;
    const TbTile tile = tiles[ti];
    const TbItem& it = items[tile.item];
    switch ((it.n[0] + 31) >> 5) {
      case 1: core_tile<XT, 1>(it, tile, Xs, Q1s, Q2s, Ts, pitch, Lp); break;
      case 2: core_tile<XT, 2>(it, tile, Xs, Q1s, Q2s, Ts, pitch, Lp); break;
      case 3: core_tile<XT, 3>(it, tile, Xs, Q1s, Q2s, Ts, pitch, Lp); break;
      case 4: core_tile<XT, 4>(it, tile, Xs, Q1s, Q2s, Ts, pitch, Lp); break;
      case 5: core_tile<XT, 5>(it, tile, Xs, Q1s, Q2s, Ts, pitch, Lp); break;
      case 6: core_tile<XT, 6>(it, tile, Xs, Q1s, Q2s, Ts, pitch, Lp); break;
      case 7: core_tile<XT, 7>(it, tile, Xs, Q1s, Q2s, Ts, pitch, Lp); break;
      default: core_tile<XT, 8>(it, tile, Xs, Q1s, Q2s, Ts, pitch, Lp); break;
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
// x_3 U3^T in FP64 through two global scratch tensors, Q_i U_i; without
// truncation the core and factors are copied out.
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
  // T1[a', x1, x2] = sum_a U0[a, a'] G[a, x1, x2]
  for (int e = tid; e < r0 * l1 * l2; e += nt) {
    const int ap = e % r0, rest = e / r0;
    double s = 0.0;
    for (int a = 0; a < l0; ++a) s = fma(it.U[0][a + l0 * ap], (double)it.G[a + l0 * rest], s);
    it.T1[e] = s;
  }
  __syncthreads();
  // T2[a', b', x2] = sum_b U1[b, b'] T1[a', b, x2]
  for (int e = tid; e < r0 * r1 * l2; e += nt) {
    const int ap = e % r0, bp = (e / r0) % r1, c = e / (r0 * r1);
    double s = 0.0;
    for (int b = 0; b < l1; ++b) s = fma(it.U[1][b + l1 * bp], it.T1[ap + r0 * (b + l1 * c)], s);
    it.T2[e] = s;
  }
  __syncthreads();
  for (int e = tid; e < r0 * r1 * r2; e += nt) {
    const int ab = e % (r0 * r1), cp = e / (r0 * r1);
    double s = 0.0;
    for (int c = 0; c < l2; ++c) s = fma(it.U[2][c + l2 * cp], it.T2[ab + r0 * r1 * c], s);
    it.core_out[e] = (float)s;
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
  TbTile* d_tiles = nullptr;
  int ntiles = 0;
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
  int pitch = 0, Lp = 0, Rp = 0, n1max = 0, n1max8 = 0, n2max = 0, lmax = 0;
  size_t sm_sketch = 0, sm_core = 0, sm_resid = 0, sm_gram = 0, sm_prep = 0, sm_finish = 0;
  bool gram_f64 = true;
  bool resid_wide = false;  // some r_2 > 16
  int grid_persist = 0, grid_resid = 0;
  int slabs_per_tile = 0;
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

void build_tiles(const std::vector<TbItem>& items, int spt, std::vector<TbTile>& tiles) {
  tiles.clear();
  for (int b = 0; b < (int)items.size(); ++b) {
    const int n3 = items[b].n[2];
    for (int t0 = 0; t0 < n3; t0 += spt) tiles.push_back(TbTile{b, t0, std::min(n3, t0 + spt), 0});
  }
  // largest work first: n1 * n2 * slabs
  std::stable_sort(tiles.begin(), tiles.end(), [&](const TbTile& a, const TbTile& c) {
    const int64_t wa = (int64_t)items[a.item].n[0] * items[a.item].n[1] * (a.t1 - a.t0);
    const int64_t wc = (int64_t)items[c.item].n[0] * items[c.item].n[1] * (c.t1 - c.t0);
    return wa > wc;
  });
}

void launch_sketch(const TbPlan& P) {
  if (P.xt == KRP_F32)
    batch_sketch_kernel<float><<<P.grid_persist, kBT, P.sm_sketch, stream()>>>(
        P.d_items, P.d_tiles, P.ntiles, P.d_counters + 0, P.pitch, P.Lp, P.n1max8, P.n2max);
  else
    batch_sketch_kernel<__nv_bfloat16><<<P.grid_persist, kBT, P.sm_sketch, stream()>>>(
        P.d_items, P.d_tiles, P.ntiles, P.d_counters + 0, P.pitch, P.Lp, P.n1max8, P.n2max);
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
  ++nk;
  launch_sketch(P);
  ++nk;
  qr_householder_launch(P.d_qjobs, 3 * P.count, status);
  ++nk;
  if (P.xt == KRP_F32)
    batch_core_kernel<float><<<P.grid_persist, kBT, P.sm_core, stream()>>>(
        P.d_items, P.d_tiles, P.ntiles, P.d_counters + 1, P.pitch, P.Lp, P.n1max8, P.n2max);
  else
    batch_core_kernel<__nv_bfloat16><<<P.grid_persist, kBT, P.sm_core, stream()>>>(
        P.d_items, P.d_tiles, P.ntiles, P.d_counters + 1, P.pitch, P.Lp, P.n1max8, P.n2max);
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
  int64_t total_slabs = 0;
  for (int b = 0; b < count; ++b) total_slabs += items[b].dims[2];
  add((size_t)total_slabs, sizeof(TbTile));
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
  P->d_tiles = carve<TbTile>(p, (size_t)total_slabs);
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
  // shared-memory shapes
  P->n1max8 = (P->n1max + 7) & ~7;
  P->pitch = ((P->n1max + 31) & ~31) + 4;
  P->Lp = (P->lmax + 3) & ~3;
  P->Rp = std::max(1, rmax);
  P->sm_sketch = sizeof(float) * ((size_t)kJB * P->pitch + (size_t)P->n1max8 * P->Lp +
                                  2 * (size_t)P->n2max * P->Lp + 2 * P->Lp);
  P->sm_core = sizeof(float) * ((size_t)kJB * P->pitch + (size_t)P->n1max8 * P->Lp +
                                (size_t)P->n2max * P->Lp + (size_t)kJB * P->Lp);
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
  allow_smem(batch_sketch_kernel<float>, P->sm_sketch);
  allow_smem(batch_sketch_kernel<__nv_bfloat16>, P->sm_sketch);
  allow_smem(batch_core_kernel<float>, P->sm_core);
  allow_smem(batch_core_kernel<__nv_bfloat16>, P->sm_core);
  allow_smem(batch_resid_kernel<float, false>, P->sm_resid);
  allow_smem(batch_resid_kernel<__nv_bfloat16, false>, P->sm_resid);
  allow_smem(batch_resid_kernel<float, true>, P->sm_resid);
  allow_smem(batch_resid_kernel<__nv_bfloat16, true>, P->sm_resid);
  allow_smem(batch_gram_kernel<double>, P->sm_gram);
  allow_smem(batch_gram_kernel<float>, P->sm_gram);
  allow_smem(batch_core_finish_kernel, P->sm_finish);
  allow_smem(batch_resid_prep_kernel, P->sm_prep);
  int occ = 1;
  KRP_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &occ, batch_sketch_kernel<float>, kBT, P->sm_sketch));
  P->grid_persist = std::max(1, occ) * c->num_sms;
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

// Slabs per work tile: time the sketch phase for a few granularities.
void autotune(TbPlan& P) {
  const int cand[] = {1, 2, 4, 8};
  std::vector<TbTile> tiles;
  float best_ms = 1e30f;
  int best = 1;
  cudaEvent_t e0, e1;
  KRP_CUDA_CHECK(cudaEventCreate(&e0));
  KRP_CUDA_CHECK(cudaEventCreate(&e1));
  // factors for the sketch
  launch_gen_factors_batch(P.d_fjobs, P.d_fstart, 3 * P.count, P.fblocks);
  for (int spt : cand) {
    build_tiles(P.h_items, spt, tiles);
    P.ntiles = (int)tiles.size();
    KRP_CUDA_CHECK(cudaMemcpyAsync(P.d_tiles, tiles.data(), sizeof(TbTile) * tiles.size(),
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
      best = spt;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  P.slabs_per_tile = best;
  build_tiles(P.h_items, best, tiles);
  P.ntiles = (int)tiles.size();
  KRP_CUDA_CHECK(cudaMemcpyAsync(P.d_tiles, tiles.data(), sizeof(TbTile) * tiles.size(),
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

// P[c + ll q] = sum_{i, a} Psi1[i, c] Psi2[a, c] Q[(a + m i) + ms q]; grid (ll_max, count)
__global__ void hb_psitq_kernel(const HbItem* __restrict__ items) {
  const HbItem& it = items[blockIdx.y];
  const int c = blockIdx.x;
  if (c >= it.ll) return;
  const int m = it.m, s = it.s, lr = it.lr;
  const int64_t ms = (int64_t)m * s;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int q = warp; q < lr; q += nw) {
    double acc = 0.0;
    for (int64_t row = lane; row < ms; row += 32) {
      const int a = (int)(row % m), i = (int)(row / m);
      const double w = (double)it.p1[i + (int64_t)s * c] * (double)it.p2[a + (int64_t)m * c];
      acc = fma(w, it.Q[row + ms * q], acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) it.P[c + (int64_t)it.ll * q] = acc;
  }
}

// W[q + lr col] = (Rp^{-1} Qp^T Z^T)[q, col]: grid (x: column chunks, y: item)
__global__ void hb_ls_kernel(const HbItem* __restrict__ items) {
  const HbItem& it = items[blockIdx.y];
  const int ll = it.ll, lr = it.lr;
  const int64_t ns = (int64_t)it.n * it.s;
  for (int64_t col = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; col < ns;
       col += (int64_t)gridDim.x * blockDim.x) {
    double* w = it.W + (int64_t)lr * col;
    for (int q = 0; q < lr; ++q) {
      double acc = 0.0;
      for (int c = 0; c < ll; ++c) acc = fma(it.Qp[c + (int64_t)ll * q], (double)it.Z[col + ns * c], acc);
      w[q] = acc;
    }
    for (int q = lr - 1; q >= 0; --q) {
      double acc = w[q];
      for (int t = q + 1; t < lr; ++t) acc -= it.Rp[q + (int64_t)lr * t] * w[t];
      w[q] = acc / it.Rp[q + (int64_t)lr * q];
    }
  }
}

// Sg = W W^T (lr x lr, FP64); one CTA per item
__global__ void hb_gram_kernel(const HbItem* __restrict__ items) {
  const HbItem& it = items[blockIdx.x];
  const int lr = it.lr;
  const int64_t ns = (int64_t)it.n * it.s;
  for (int pq = threadIdx.x; pq < lr * lr; pq += blockDim.x) {
    const int p = pq % lr, q = pq / lr;
    if (p > q) continue;
    double acc = 0.0;
    for (int64_t col = 0; col < ns; ++col)
      acc = fma(it.W[p + (int64_t)lr * col], it.W[q + (int64_t)lr * col], acc);
    it.Sg[p + lr * q] = acc;
    it.Sg[q + lr * p] = acc;
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
  EigJob* d_ej = nullptr;
  int gx_blockmul = 1, gx_corr = 1, gx_ls = 1, gx_out = 1, llmax = 1, lrmax = 1;
  int kernels_per_run = 0;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cs = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  ~HbPlan() {
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
  qr_householder_launch(P.d_qy, P.count, status);
  hb_psitq_kernel<<<dim3(P.llmax, P.count), 256, 0, stream()>>>(P.d_items);
  check_launch("hb_psitq");
  qr_householder_launch(P.d_qp, P.count, status);
  hb_ls_kernel<<<dim3(P.gx_ls, P.count), 256, 0, stream()>>>(P.d_items);
  check_launch("hb_ls");
  hb_gram_kernel<<<P.count, 256, 0, stream()>>>(P.d_items);
  check_launch("hb_gram");
  eig_launch(P.d_ej, P.count, P.lrmax, status);
  hb_out_kernel<<<dim3(P.gx_out, P.count), 256, 0, stream()>>>(P.d_items);
  check_launch("hb_out");
  nk += 9;
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
  P->gx_ls = chunks_for(maxns);
  P->gx_out = chunks_for(maxout);
  cudaStream_t s = c->stream;
  KRP_CUDA_CHECK(cudaMemcpyAsync(P->d_items, hi.data(), sizeof(HbItem) * count, cudaMemcpyHostToDevice, s));
  KRP_CUDA_CHECK(cudaMemcpyAsync(P->d_fjobs, fj.data(), sizeof(BatchFactorJob) * fj.size(), cudaMemcpyHostToDevice, s));
  KRP_CUDA_CHECK(cudaMemcpyAsync(P->d_fstart, fstart.data(), sizeof(int64_t) * fstart.size(), cudaMemcpyHostToDevice, s));
  KRP_CUDA_CHECK(cudaMemcpyAsync(P->d_qy, qy.data(), sizeof(QrJob) * count, cudaMemcpyHostToDevice, s));
  KRP_CUDA_CHECK(cudaMemcpyAsync(P->d_qp, qp.data(), sizeof(QrJob) * count, cudaMemcpyHostToDevice, s));
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

int tucker_batched_plan_info(int* slabs_per_tile, int* tiles, int* grid) {
  TbPlan* P = static_cast<TbPlan*>(current()->batch_plan);
  if (!P) return 0;
  if (slabs_per_tile) *slabs_per_tile = P->slabs_per_tile;
  if (tiles) *tiles = P->ntiles;
  if (grid) *grid = P->grid_persist;
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
