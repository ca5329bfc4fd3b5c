// Tensor-core contractions over the big tensor on sm_103a: tcgen05.mma
// (kind::f16 with BF16 operands; kind::tf32 for FP32 data as three TF32
// products of exact hi/lo splits; FP32 accumulators in TMEM) fed by TMA
// (cp.async.bulk.tensor, 128-byte swizzle) through mbarrier pipelines.
//
//   tc_gemm_tn_tf32, tc_mttkrp_first_tf32, tc_residual_tf32: the same three
//       contractions for FP32 X (the MTTKRP's converter warps transpose each
//       X tile into K-major rows, since these MMAs take K-major operands)
//
//   tc_gemm_tn_bf16:       out[s, k] = sum_i X[i, s] F[i, k]
//       (TTM of the fastest mode, Sec. 2.1; A = X is K-major: i contiguous)
//   tc_mttkrp_first_bf16:  Y[i, k] = sum_t w[t, k] sum_{i2} X[i, i2, t] Om2[i2, k]
//       (mode-1 MTTKRP, Alg. 7: the contraction against one factor is the MMA,
//        A = X is MN-major: i contiguous; the remaining Khatri-Rao factors enter
//        as the per-slab weights w[t, :] applied to the TMEM result)
//
// Both kernels are persistent (one CTA per SM) and warp-specialised:
//   warp 0: TMA producer (one elected lane), warp 1: TMEM allocator + MMA
//   issuer (one elected lane), warps 2-5: epilogue (TMEM -> registers -> HBM).
// Accumulators are double-buffered in TMEM so the epilogue of one tile
// overlaps the MMAs of the next.  Every mbarrier wait is bounded (1 s of
// %globaltimer); on expiry the kernel raises KRP_ETIMEOUT in the status word,
// drains its own TMA loads and MMAs (bounded again), frees TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "pipeline.h"

namespace krp {
namespace {

constexpr uint64_t kWaitNs = 1000000000ull;  // 1 s per wait
constexpr int kThreads = 192;                // 6 warps
constexpr int kBM = 128;                     // rows per tile (TMEM lanes)
constexpr int kBK = 64;                      // K elements per stage (128 B of BF16)

// ------------------------------------------------------------ PTX helpers ---
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t gtime() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase with the given parity; false on timeout/abort.
// lim: the wait's limit in ns (the context's setting for the pipeline's
// waits; the drains after an abort keep the full kWaitNs).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                          uint64_t lim = kWaitNs) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = gtime();
  for (;;) {
    if (mbar_try(bar, parity)) return true;
    if (*abort_flag) return false;
    if (gtime() - t0 > lim) return false;
  }
}
// The context's limit of the pipeline's waits: a uint64 in ns beside the
// status word (0: kWaitNs).
__device__ __forceinline__ uint64_t wait_limit(const int* status) {
  const uint64_t v = *reinterpret_cast<const volatile uint64_t*>(status + 2);
  return v ? v : kWaitNs;
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar,
                                            int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(c0), "r"(c1)
      : "memory");
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, uint32_t bar,
                                            int c0, int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   bar)
               : "memory");
}
// 32 lanes x 16 consecutive 32-bit columns per warp.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// The same load without the wait: the registers are valid after tmem_ld_wait().
__device__ __forceinline__ void tmem_ld16_issue(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld_wait() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor, 128-byte swizzle (sm_100 layout):
// start>>4 [0,14), leading-byte-offset>>4 [16,30), stride-byte-offset>>4
// [32,46), version 1 at [46,48), layout SWIZZLE_128B (=2) at [61,64).
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((addr & 0x3FFFFu) >> 4);
  d |= static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16;
  d |= static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32;
  d |= static_cast<uint64_t>(1) << 46;
  d |= static_cast<uint64_t>(2) << 61;
  return d;
}
// Instruction descriptor of kind::f16: D FP32, A/B BF16, M x N, majorness.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N, bool a_mn, bool b_mn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((a_mn ? 1u : 0u) << 15) | ((b_mn ? 1u : 0u) << 16) |
         (static_cast<uint32_t>(N >> 3) << 17) | (static_cast<uint32_t>(M >> 4) << 24);
}

struct Bars {
  uint64_t full[8];
  uint64_t empty[8];
  uint64_t tfull[2];
  uint64_t tempty[2];
  uint64_t drain;
  uint32_t tmem_base;
  int abort_flag;
  int issued;    // TMA loads issued (producer)
  int consumed;  // stages consumed by the MMA warp
};

__device__ __forceinline__ void raise_timeout(Bars* b, int* status) {
  b->abort_flag = 1;
  atomicCAS(status, 0, static_cast<int>(KRP_ETIMEOUT));  // the first error is kept
}

// Producer-side drain after an abort: wait (bounded) for every TMA load that
// was issued but not consumed, so no copy lands in shared memory after exit.
template <int NS>
__device__ void drain_loads(Bars* b) {
  int dummy = 0;
  for (int j = b->consumed; j < b->issued; ++j) {
    const int st = j % NS;
    const uint32_t ph = (j / NS) & 1;
    mbar_wait(smem_u32(&b->full[st]), ph, reinterpret_cast<volatile int*>(&dummy));
  }
}

// ----------------------------------------------------------------------------
// out[s + S*k] = sum_i X[i + n1*s] F[i, k] (+ lo part at column Lp + k)
// A tile: 128 rows (s) x 64 K (i), box of mapA = {64, 128}.  B: mapB over the
// combined factor buffer (K = n1p contiguous, rows = N columns of F).
// XLO: X is given as a BF16 hi/lo pair (second map mapAlo over the lo
// plane); its lo tile is multiplied by the hi columns of F into the same
// accumulator (X F ~ Xh [Fh|Fl] + Xl Fh, dropping Xl Fl, below 2^-16).
template <int N, int NS, bool XLO>
__global__ void __launch_bounds__(kThreads, 1)
    tc_gemm_tn_kernel(const __grid_constant__ CUtensorMap mapA,
                      const __grid_constant__ CUtensorMap mapAlo,
                      const __grid_constant__ CUtensorMap mapB, int64_t S, int kchunks, int L,
                      int Lp, int has_lo, float* __restrict__ out,
                      __nv_bfloat16* __restrict__ outb, int* status) {
  constexpr uint32_t kABytes = kBM * kBK * 2;  // 16 KB
  constexpr uint32_t kANum = XLO ? 2 : 1;
  constexpr uint32_t kBBytes = N * kBK * 2;
  constexpr uint32_t kStage = kANum * kABytes + kBBytes;
  constexpr uint32_t kTmemCols = (2 * N <= 32) ? 32 : (2 * N <= 64) ? 64 : (2 * N <= 128) ? 128 : (2 * N <= 256) ? 256 : 512;
  constexpr uint32_t kIdesc = idesc_bf16(kBM, N, false, false);
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  Bars* bars = reinterpret_cast<Bars*>(smem + NS * kStage);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t tiles = (S + kBM - 1) / kBM;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(smem_u32(&bars->full[s]), 1);
      mbar_init(smem_u32(&bars->empty[s]), 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(smem_u32(&bars->tfull[a]), 1);
      mbar_init(smem_u32(&bars->tempty[a]), 4);
    }
    mbar_init(smem_u32(&bars->drain), 1);
    bars->abort_flag = 0;
    bars->issued = 0;
    bars->consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(smem_u32(&bars->tmem_base), kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = bars->tmem_base;
  volatile int* abort_flag = &bars->abort_flag;
  const uint64_t lim = wait_limit(status);
  const uint32_t idesc_lo = idesc_bf16(kBM, Lp, false, false);

  if (warp == 0) {
    if (lane == 0) {
      int it = 0;
      for (int64_t tile = blockIdx.x; tile < tiles && !*abort_flag; tile += gridDim.x) {
        for (int kc = 0; kc < kchunks; ++kc, ++it) {
          const int st = it % NS;
          const uint32_t ph = (it / NS) & 1;
          if (!mbar_wait(smem_u32(&bars->empty[st]), ph ^ 1, abort_flag, lim)) {
            raise_timeout(bars, status);
            break;
          }
          const uint32_t a = smem_u32(smem + st * kStage);
          const uint32_t fb = smem_u32(&bars->full[st]);
          mbar_expect_tx(fb, kStage);
          tma_load_2d(a, &mapA, fb, kc * kBK, static_cast<int>(tile * kBM));
          if (XLO) tma_load_2d(a + kABytes, &mapAlo, fb, kc * kBK, static_cast<int>(tile * kBM));
          tma_load_2d(a + kANum * kABytes, &mapB, fb, kc * kBK, 0);
          bars->issued = it + 1;
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int it = 0, tl = 0;
      for (int64_t tile = blockIdx.x; tile < tiles && !*abort_flag; tile += gridDim.x, ++tl) {
        const int acc = tl & 1;
        const uint32_t aph = (tl >> 1) & 1;
        if (!mbar_wait(smem_u32(&bars->tempty[acc]), aph ^ 1, abort_flag, lim)) {
          raise_timeout(bars, status);
          break;
        }
        tc_fence_after();
        const uint32_t dt = tmem + acc * N;
        bool ok = true;
        for (int kc = 0; kc < kchunks; ++kc, ++it) {
          const int st = it % NS;
          const uint32_t ph = (it / NS) & 1;
          if (!mbar_wait(smem_u32(&bars->full[st]), ph, abort_flag, lim)) {
            raise_timeout(bars, status);
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a = smem_u32(smem + st * kStage);
          const uint32_t b = a + kANum * kABytes;
#pragma unroll
          for (int k = 0; k < kBK / 16; ++k) {
            mma_bf16(dt, sdesc(a + 32 * k, 16, 1024), sdesc(b + 32 * k, 16, 1024), kIdesc,
                     (kc | k) != 0);
            if (XLO)  // Xl times the hi columns of F (the first Lp rows of B)
              mma_bf16(dt, sdesc(a + kABytes + 32 * k, 16, 1024), sdesc(b + 32 * k, 16, 1024),
                       idesc_lo, 1);
          }
          mma_commit(smem_u32(&bars->empty[st]));
          bars->consumed = it + 1;
        }
        if (!ok) break;
        mma_commit(smem_u32(&bars->tfull[acc]));
      }
      // all MMAs issued by this thread have completed once this commit fires
      mma_commit(smem_u32(&bars->drain));
      int dummy = 0;
      mbar_wait(smem_u32(&bars->drain), 0, reinterpret_cast<volatile int*>(&dummy));
    }
  } else {
    const int q = warp & 3;  // TMEM lane quarter of this warp
    int tl = 0;
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x, ++tl) {
      const int acc = tl & 1;
      const uint32_t ph = (tl >> 1) & 1;
      if (!mbar_wait(smem_u32(&bars->tfull[acc]), ph, abort_flag, lim)) {
        if (lane == 0) raise_timeout(bars, status);
        break;
      }
      tc_fence_after();
      const int row = q * 32 + lane;
      const int64_t s = tile * kBM + row;
      const uint32_t base = tmem + (static_cast<uint32_t>(q * 32) << 16) + acc * N;
      for (int c0 = 0; c0 < Lp; c0 += 16) {
        float v[16];
        tmem_ld16(base + c0, v);
        if (has_lo) {
          float w[16];
          tmem_ld16(base + Lp + c0, w);
#pragma unroll
          for (int j = 0; j < 16; ++j) v[j] += w[j];
        }
        if (s < S) {
          if (outb) {  // BF16 hi/lo pair: hi plane, then the lo plane S*L later
#pragma unroll
            for (int j = 0; j < 16; ++j)
              if (c0 + j < L) {
                const __nv_bfloat16 h = __float2bfloat16_rn(v[j]);
                outb[s + S * (c0 + j)] = h;
                outb[S * L + s + S * (c0 + j)] = __float2bfloat16_rn(v[j] - __bfloat162float(h));
              }
          } else {
#pragma unroll
            for (int j = 0; j < 16; ++j)
              if (c0 + j < L) out[s + S * (c0 + j)] = v[j];
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&bars->tempty[acc]));
    }
  }
  __syncthreads();
  if (warp == 0 && lane == 0 && bars->abort_flag) drain_loads<NS>(bars);
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

// ----------------------------------------------------------------------------
// FP32 TTM on the tensor cores as three TF32 products (kind::tf32):
//   out[s + S*k] = sum_i X[i + n1*s] F[i, k]   (FP32 X, FP32 F, FP32 out)
// Each FP32 value splits exactly as x = x_h + x_l, x_h = x with its low 13
// mantissa bits cleared (the TF32 value an MMA reads from the FP32 word) and
// x_l = x - x_h; then X F ~ X_h [F_h | F_l] + X_l F_h, dropping X_l F_l and
// the truncation of the lo parts (each below 2^-20 |x| |f|), which is the
// size of FP32 rounding over these sums.  A tile: 128 rows (s) x 32 K (i),
// 128-byte FP32 rows by TMA; four converter warps write X_l beside it
// (elementwise, so in the same swizzled layout) and release it to the MMA
// warp through an mbarrier after a proxy fence.  B: the combined factor
// buffer [F_h rows 0..L-1 | F_l rows Lp..Lp+L-1] (FP32, K = n1p contiguous).
// Warps: 0 TMA producer, 1 TMEM + MMA issuer, 2-5 epilogue, 6-9 converters.
constexpr int kBK32 = 32;                 // K elements per stage (128 B of FP32)
constexpr int kTf32Threads = 320;

__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  // D FP32 (bit 4), A and B TF32 (format 2 at bits 7-9 and 10-12), K-major
  return (1u << 4) | (2u << 7) | (2u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
         (static_cast<uint32_t>(M >> 4) << 24);
}
__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

struct BarsT : Bars {
  uint64_t lofull[8];
};

template <int N, int NS>
__global__ void __launch_bounds__(kTf32Threads, 1)
    tc_gemm_tn_tf32_kernel(const __grid_constant__ CUtensorMap mapA,
                           const __grid_constant__ CUtensorMap mapB, int64_t S, int kchunks, int L,
                           int Lp, float* __restrict__ out, int* status) {
  constexpr uint32_t kABytes = kBM * kBK32 * 4;  // 16 KB
  constexpr uint32_t kBBytes = N * kBK32 * 4;
  constexpr uint32_t kStage = 2 * kABytes + kBBytes;
  constexpr uint32_t kTmemCols = (2 * N <= 32) ? 32 : (2 * N <= 64) ? 64 : (2 * N <= 128) ? 128 : (2 * N <= 256) ? 256 : 512;
  constexpr uint32_t kIdesc = idesc_tf32(kBM, N);
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  BarsT* bars = reinterpret_cast<BarsT*>(smem + NS * kStage);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t tiles = (S + kBM - 1) / kBM;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(smem_u32(&bars->full[s]), 1);
      mbar_init(smem_u32(&bars->empty[s]), 1);
      mbar_init(smem_u32(&bars->lofull[s]), 4);  // the four converter warps
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(smem_u32(&bars->tfull[a]), 1);
      mbar_init(smem_u32(&bars->tempty[a]), 4);
    }
    mbar_init(smem_u32(&bars->drain), 1);
    bars->abort_flag = 0;
    bars->issued = 0;
    bars->consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(smem_u32(&bars->tmem_base), kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = bars->tmem_base;
  volatile int* abort_flag = &bars->abort_flag;
  const uint64_t lim = wait_limit(status);
  const uint32_t idesc_lo = idesc_tf32(kBM, Lp);

  if (warp == 0) {
    if (lane == 0) {
      int it = 0;
      for (int64_t tile = blockIdx.x; tile < tiles && !*abort_flag; tile += gridDim.x) {
        for (int kc = 0; kc < kchunks; ++kc, ++it) {
          const int st = it % NS;
          const uint32_t ph = (it / NS) & 1;
          if (!mbar_wait(smem_u32(&bars->empty[st]), ph ^ 1, abort_flag, lim)) {
            raise_timeout(bars, status);
            break;
          }
          const uint32_t a = smem_u32(smem + st * kStage);
          const uint32_t fb = smem_u32(&bars->full[st]);
          mbar_expect_tx(fb, kABytes + kBBytes);
          tma_load_2d(a, &mapA, fb, kc * kBK32, static_cast<int>(tile * kBM));
          tma_load_2d(a + 2 * kABytes, &mapB, fb, kc * kBK32, 0);
          bars->issued = it + 1;
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int it = 0, tl = 0;
      for (int64_t tile = blockIdx.x; tile < tiles && !*abort_flag; tile += gridDim.x, ++tl) {
        const int acc = tl & 1;
        const uint32_t aph = (tl >> 1) & 1;
        if (!mbar_wait(smem_u32(&bars->tempty[acc]), aph ^ 1, abort_flag, lim)) {
          raise_timeout(bars, status);
          break;
        }
        tc_fence_after();
        const uint32_t dt = tmem + acc * N;
        bool ok = true;
        for (int kc = 0; kc < kchunks; ++kc, ++it) {
          const int st = it % NS;
          const uint32_t ph = (it / NS) & 1;
          if (!mbar_wait(smem_u32(&bars->full[st]), ph, abort_flag, lim) ||
              !mbar_wait(smem_u32(&bars->lofull[st]), ph, abort_flag, lim)) {
            raise_timeout(bars, status);
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a = smem_u32(smem + st * kStage);
          const uint32_t b = a + 2 * kABytes;
#pragma unroll
          for (int k = 0; k < kBK32 / 8; ++k) {
            mma_tf32(dt, sdesc(a + 32 * k, 16, 1024), sdesc(b + 32 * k, 16, 1024), kIdesc,
                     (kc | k) != 0);
            // X_l times the hi columns of F (the first Lp rows of B)
            mma_tf32(dt, sdesc(a + kABytes + 32 * k, 16, 1024), sdesc(b + 32 * k, 16, 1024),
                     idesc_lo, 1);
          }
          mma_commit(smem_u32(&bars->empty[st]));
          bars->consumed = it + 1;
        }
        if (!ok) break;
        mma_commit(smem_u32(&bars->tfull[acc]));
      }
      // all MMAs issued by this thread have completed once this commit fires
      mma_commit(smem_u32(&bars->drain));
      int dummy = 0;
      mbar_wait(smem_u32(&bars->drain), 0, reinterpret_cast<volatile int*>(&dummy));
    }
  } else if (warp < 6) {
    const int q = warp & 3;  // TMEM lane quarter of this warp
    int tl = 0;
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x, ++tl) {
      const int acc = tl & 1;
      const uint32_t ph = (tl >> 1) & 1;
      if (!mbar_wait(smem_u32(&bars->tfull[acc]), ph, abort_flag, lim)) {
        if (lane == 0) raise_timeout(bars, status);
        break;
      }
      tc_fence_after();
      const int row = q * 32 + lane;
      const int64_t s = tile * kBM + row;
      const uint32_t base = tmem + (static_cast<uint32_t>(q * 32) << 16) + acc * N;
      for (int c0 = 0; c0 < Lp; c0 += 16) {
        float v[16], w[16];
        tmem_ld16(base + c0, v);
        tmem_ld16(base + Lp + c0, w);
        if (s < S) {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (c0 + j < L) out[s + S * (c0 + j)] = v[j] + w[j];
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&bars->tempty[acc]));
    }
  } else {
    // converters: X_l = X - X_h of each landed A tile, written beside it
    const int ct = threadIdx.x - 6 * 32;  // 0..127
    int it = 0;
    bool ok = true;
    for (int64_t tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x) {
      for (int kc = 0; kc < kchunks; ++kc, ++it) {
        const int st = it % NS;
        const uint32_t ph = (it / NS) & 1;
        if (!mbar_wait(smem_u32(&bars->full[st]), ph, abort_flag, lim)) {
          raise_timeout(bars, status);
          ok = false;
          break;
        }
        const float4* src = reinterpret_cast<const float4*>(smem + st * kStage);
        float4* dst = reinterpret_cast<float4*>(smem + st * kStage + kABytes);
#pragma unroll
        for (int j = 0; j < (int)(kABytes / 16 / 128); ++j) {
          const float4 x = src[ct + 128 * j];
          float4 l;
          l.x = x.x - __uint_as_float(__float_as_uint(x.x) & 0xFFFFE000u);
          l.y = x.y - __uint_as_float(__float_as_uint(x.y) & 0xFFFFE000u);
          l.z = x.z - __uint_as_float(__float_as_uint(x.z) & 0xFFFFE000u);
          l.w = x.w - __uint_as_float(__float_as_uint(x.w) & 0xFFFFE000u);
          dst[ct + 128 * j] = l;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&bars->lofull[st]));
      }
    }
  }
  __syncthreads();
  if (warp == 0 && lane == 0 && bars->abort_flag) drain_loads<NS>(bars);
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

// ----------------------------------------------------------------------------
// FP32 mode-1 MTTKRP on the tensor cores, three TF32 products as in the TF32
// TTM (Alg. 7's MTTKRP step without forming the Khatri-Rao product):
//   Y[i + n1*k] += sum_{t in range} wT[t*Lp + k] D_t[i, k],
//   D_t[i, k] = sum_{i2} X[i, i2, t] Om2[i2, k].
// The contraction runs over i2, which is not X's contiguous index, and these
// MMAs take K-major operands only, so four converter warps turn each landed
// X tile (four TMA boxes of 32 i x 32 i2, rows i2) into K-major rows i of 32
// i2, once as X (the MMA reads its TF32 part X_h) and once as X_l = X - X_h,
// both in the 128-byte swizzle of the descriptors.  D_t = X_h [Om2_h | Om2_l]
// + X_l Om2_h accumulates in TMEM over the i2 chunks of slab t (two buffers of
// width N = 2 Lp; one MMA of width N reads the X_h tile once); the epilogue
// adds the two column halves, weights them by w_t and keeps Y's partial sums
// in registers, one FP32 atomic add per output at the end.  CTA (mb, z) takes rows mb*128.. and slabs [z t_per_cta, ...).
// Two rings: NR raw X tiles (TMA, released by the converters as soon as they
// hold the values in registers, so that many tiles are in flight from HBM)
// and NC operand stages (X_h^T, X_l^T written by the converters, the Om2
// chunk loaded by TMA from converter thread 0; released by the MMA commit).
// Two groups of four converter warps take the even and the odd chunks (so
// that one group converts while the other waits on its loads), each with its
// own operand stage.  Warps: 0 TMA producer of X, 1 TMEM + MMA issuer, 2-5
// epilogue, 6-9 and 10-13 the converter groups.
constexpr int kMtThreads = 448;
struct BarsM : Bars {
  uint64_t rempty[8];  // raw X stage read by one group of four converter warps
  uint64_t bfull[8];   // the Om2 chunk of an operand stage has landed
  uint64_t lofull[8];  // X_h^T, X_l^T of an operand stage are written
  int r_consumed[2];   // chunks (of group g's parity) group g's thread 0 saw land
  int b_issued[2];     // Om2 chunk loads group g's thread 0 issued
  int b_consumed;      // Om2 chunk loads the MMA warp saw land
};

template <int N, int NR, int NC>
__global__ void __launch_bounds__(kMtThreads, 1)
    tc_mttkrp_tf32_kernel(const __grid_constant__ CUtensorMap mapX,
                          const __grid_constant__ CUtensorMap mapB, int64_t n1, int64_t T,
                          int kchunks, int mblocks, int64_t t_per_cta,
                          const float* __restrict__ wT, int L, float* __restrict__ Y,
                          int* status) {
  constexpr int Lp = N / 2;
  constexpr uint32_t kBox = 32 * kBK32 * 4;    // 32 (i) x 32 (i2) FP32 = 4 KB
  constexpr uint32_t kRaw = 4 * kBox;          // one landed X tile (16 KB)
  constexpr uint32_t kA = kBM * kBK32 * 4;     // one K-major operand tile (16 KB)
  constexpr uint32_t kBBytes = N * kBK32 * 4;
  constexpr uint32_t kOp = 2 * kA + kBBytes;   // [X_h^T | X_l^T | Om2 chunk]
  static_assert(kOp % 1024 == 0, "operand stages must keep the 1 KB swizzle alignment");
  constexpr uint32_t kTmemCols = (2 * N <= 64) ? 64 : (2 * N <= 128) ? 128 : 256;
  constexpr uint32_t kIdesc = idesc_tf32(kBM, N);
  constexpr uint32_t kIdescLo = idesc_tf32(kBM, Lp);
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* ops = smem;
  uint8_t* raws = smem + NC * kOp;
  BarsM* bars = reinterpret_cast<BarsM*>(raws + NR * kRaw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int mb = blockIdx.x % mblocks;
  const int64_t t0 = static_cast<int64_t>(blockIdx.x / mblocks) * t_per_cta;
  const int64_t t1 = min(T, t0 + t_per_cta);

  if (threadIdx.x == 0) {
    for (int s = 0; s < NR; ++s) {
      mbar_init(smem_u32(&bars->full[s]), 1);
      mbar_init(smem_u32(&bars->rempty[s]), 4);
    }
    for (int c = 0; c < NC; ++c) {
      mbar_init(smem_u32(&bars->empty[c]), 1);
      mbar_init(smem_u32(&bars->bfull[c]), 1);
      mbar_init(smem_u32(&bars->lofull[c]), 4);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(smem_u32(&bars->tfull[a]), 1);
      mbar_init(smem_u32(&bars->tempty[a]), 4);
    }
    mbar_init(smem_u32(&bars->drain), 1);
    bars->abort_flag = 0;
    bars->issued = 0;
    bars->consumed = 0;
    bars->r_consumed[0] = bars->r_consumed[1] = 0;
    bars->b_issued[0] = bars->b_issued[1] = 0;
    bars->b_consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(smem_u32(&bars->tmem_base), kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = bars->tmem_base;
  volatile int* abort_flag = &bars->abort_flag;
  const uint64_t lim = wait_limit(status);

  if (warp == 0) {
    if (lane == 0) {
      int it = 0;
      for (int64_t t = t0; t < t1 && !*abort_flag; ++t) {
        for (int kc = 0; kc < kchunks; ++kc, ++it) {
          const int r = it % NR;
          const uint32_t ph = (it / NR) & 1;
          if (!mbar_wait(smem_u32(&bars->rempty[r]), ph ^ 1, abort_flag, lim)) {
            raise_timeout(bars, status);
            break;
          }
          const uint32_t a = smem_u32(raws + r * kRaw);
          const uint32_t fb = smem_u32(&bars->full[r]);
          mbar_expect_tx(fb, kRaw);
#pragma unroll
          for (int b = 0; b < 4; ++b)
            tma_load_3d(a + b * kBox, &mapX, fb, mb * kBM + 32 * b, kc * kBK32, static_cast<int>(t));
          bars->issued = it + 1;
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int it = 0, tl = 0;
      for (int64_t t = t0; t < t1 && !*abort_flag; ++t, ++tl) {
        const int acc = tl & 1;
        const uint32_t aph = (tl >> 1) & 1;
        if (!mbar_wait(smem_u32(&bars->tempty[acc]), aph ^ 1, abort_flag, lim)) {
          raise_timeout(bars, status);
          break;
        }
        tc_fence_after();
        const uint32_t dt = tmem + acc * N;
        bool ok = true;
        for (int kc = 0; kc < kchunks; ++kc, ++it) {
          const int c = it % NC;
          const uint32_t ph = (it / NC) & 1;
          if (!mbar_wait(smem_u32(&bars->bfull[c]), ph, abort_flag, lim) ||
              !mbar_wait(smem_u32(&bars->lofull[c]), ph, abort_flag, lim)) {
            raise_timeout(bars, status);
            ok = false;
            break;
          }
          bars->b_consumed = it + 1;
          tc_fence_after();
          const uint32_t ah = smem_u32(ops + c * kOp);
          const uint32_t al = ah + kA;
          const uint32_t b = ah + 2 * kA;
#pragma unroll
          for (int k = 0; k < kBK32 / 8; ++k) {
            mma_tf32(dt, sdesc(ah + 32 * k, 16, 1024), sdesc(b + 32 * k, 16, 1024), kIdesc,
                     (kc | k) != 0);
            // X_l times the hi columns of Om2 (the first Lp rows of B)
            mma_tf32(dt, sdesc(al + 32 * k, 16, 1024), sdesc(b + 32 * k, 16, 1024), kIdescLo, 1);
          }
          mma_commit(smem_u32(&bars->empty[c]));
        }
        if (!ok) break;
        mma_commit(smem_u32(&bars->tfull[acc]));
      }
      mma_commit(smem_u32(&bars->drain));
      int dummy = 0;
      mbar_wait(smem_u32(&bars->drain), 0, reinterpret_cast<volatile int*>(&dummy));
    }
  } else if (warp < 6) {
    const int q = warp & 3;
    const int row = q * 32 + lane;
    const int64_t i = static_cast<int64_t>(mb) * kBM + row;
    float accum[Lp];
#pragma unroll
    for (int k = 0; k < Lp; ++k) accum[k] = 0.f;
    int tl = 0;
    for (int64_t t = t0; t < t1; ++t, ++tl) {
      const int acc = tl & 1;
      const uint32_t ph = (tl >> 1) & 1;
      if (!mbar_wait(smem_u32(&bars->tfull[acc]), ph, abort_flag, lim)) {
        if (lane == 0) raise_timeout(bars, status);
        break;
      }
      tc_fence_after();
      const uint32_t base = tmem + (static_cast<uint32_t>(q * 32) << 16) + acc * N;
      const float* wt = wT + t * Lp;
#pragma unroll
      for (int c0 = 0; c0 < Lp; c0 += 16) {
        float v[16], u[16];
        tmem_ld16(base + c0, v);
        tmem_ld16(base + Lp + c0, u);
#pragma unroll
        for (int j = 0; j < 16; ++j) accum[c0 + j] = fmaf(__ldg(wt + c0 + j), v[j] + u[j], accum[c0 + j]);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&bars->tempty[acc]));
    }
    if (i < n1) {
#pragma unroll
      for (int k = 0; k < Lp; ++k)
        if (k < L) atomicAdd(Y + i + n1 * k, accum[k]);
    }
  } else {
    // converters: group g takes the chunks it with it % 2 == g (operand
    // stage g); thread ct owns row i = ct of the K-major tiles and reads its
    // 32 values of i2 from box ct / 32 (a warp reads one 128-byte row per load)
    const int g = (warp - 6) >> 2;
    const int ct = (threadIdx.x - 6 * 32) & 127;
    const int bx = ct >> 5, il = ct & 31;
    const uint32_t sw = static_cast<uint32_t>(ct & 7);
    int it = 0;
    bool ok = true;
    for (int64_t t = t0; t < t1 && ok; ++t) {
      for (int kc = 0; kc < kchunks; ++kc, ++it) {
        if ((it & 1) != g) continue;
        const int r = it % NR, c = it % NC;
        const uint32_t rph = (it / NR) & 1, cph = (it / NC) & 1;
        // the operand stage is free once the MMAs of its previous use are done
        if (!mbar_wait(smem_u32(&bars->empty[c]), cph ^ 1, abort_flag, lim)) {
          raise_timeout(bars, status);
          ok = false;
          break;
        }
        uint8_t* og = ops + c * kOp;
        if (ct == 0) {
          const uint32_t bb = smem_u32(&bars->bfull[c]);
          mbar_expect_tx(bb, kBBytes);
          tma_load_2d(smem_u32(og + 2 * kA), &mapB, bb, kc * kBK32, 0);
          bars->b_issued[g] = it + 1;
        }
        if (!mbar_wait(smem_u32(&bars->full[r]), rph, abort_flag, lim)) {
          raise_timeout(bars, status);
          ok = false;
          break;
        }
        if (ct == 0) bars->r_consumed[g] = it + 1;
        const uint8_t* raw = raws + r * kRaw + bx * kBox + ((il & 3) << 2);
        float x[kBK32];
#pragma unroll
        for (int rr = 0; rr < kBK32; ++rr)
          x[rr] = *reinterpret_cast<const float*>(raw + rr * 128 + ((((il >> 2) ^ (rr & 7))) << 4));
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&bars->rempty[r]));
        uint8_t* hrow = og + ct * 128;
        uint8_t* lrow = og + kA + ct * 128;
#pragma unroll
        for (int q4 = 0; q4 < kBK32 / 4; ++q4) {
          const float4 h = make_float4(x[4 * q4], x[4 * q4 + 1], x[4 * q4 + 2], x[4 * q4 + 3]);
          float4 l;
          l.x = h.x - __uint_as_float(__float_as_uint(h.x) & 0xFFFFE000u);
          l.y = h.y - __uint_as_float(__float_as_uint(h.y) & 0xFFFFE000u);
          l.z = h.z - __uint_as_float(__float_as_uint(h.z) & 0xFFFFE000u);
          l.w = h.w - __uint_as_float(__float_as_uint(h.w) & 0xFFFFE000u);
          const uint32_t off = (static_cast<uint32_t>(q4) ^ sw) << 4;
          *reinterpret_cast<float4*>(hrow + off) = h;
          *reinterpret_cast<float4*>(lrow + off) = l;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&bars->lofull[c]));
      }
    }
  }
  __syncthreads();
  if (warp == 0 && lane == 0 && bars->abort_flag) {
    // every TMA write into shared memory must land before the CTA exits:
    // the X tiles issued but not seen by their group, the Om2 chunks issued
    // but not seen by the MMA warp (neither stage can have been reused)
    int dummy = 0;
    const int rc[2] = {bars->r_consumed[0], bars->r_consumed[1]};
    const int bi[2] = {bars->b_issued[0], bars->b_issued[1]};
    for (int j = min(rc[0], rc[1]); j < bars->issued; ++j)
      if (j >= rc[j & 1])
        mbar_wait(smem_u32(&bars->full[j % NR]), (j / NR) & 1, reinterpret_cast<volatile int*>(&dummy));
    for (int j = bars->b_consumed; j < max(bi[0], bi[1]); ++j)
      if (j < bi[j & 1])
        mbar_wait(smem_u32(&bars->bfull[j % NC]), (j / NC) & 1, reinterpret_cast<volatile int*>(&dummy));
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

// Residual of the FP32 form on the tensor cores: acc[0] += ||X - Q1 H||_F^2,
// acc[1] += ||X||_F^2 for FP32 X (n1 x S) and c <= 32.  Same orientation as
// the BF16 residual (the tile is X_hat^T[s, i], A = H with M = s, B = Q1 with
// N = i), with FP32 operands split into TF32 hi and lo parts (rows of
// [hi 32 | lo 32], 256 bytes) and X_hat^T = Hh Qh^T + Hl Qh^T + Hh Ql^T
// (kind::tf32; the dropped Hl Ql^T and the truncation of the lo parts are
// below 2^-20 relative).  A stage holds Hh, Hl (128 x 32 FP32 each) and the X
// tile as four TMA boxes of 32 (i) x 128 (s) FP32; an epilogue thread owns
// one s and compares 16 consecutive i per TMEM load, four 16-byte chunks of
// one box row (chunks swizzled by s mod 8).  A CTA keeps the 128-row block of
// Q1 (hi and lo, 32 KB) resident; release of a stage as in the BF16 form.
__global__ void __launch_bounds__(kThreads, 1)
    tc_residual_tf32_kernel(const __grid_constant__ CUtensorMap mapX,
                            const __grid_constant__ CUtensorMap mapQ,
                            const __grid_constant__ CUtensorMap mapH, int64_t n1, int64_t S,
                            int mblocks, int cpm, double* __restrict__ acc, int* status) {
  constexpr int NS = 2;
  constexpr uint32_t kOp = 128 * 32 * 4;    // one 128-row x 32-element FP32 operand tile (16 KB)
  constexpr uint32_t kXBox = 32 * 128 * 4;  // 32 (i) x 128 (s) FP32 (16 KB)
  constexpr uint32_t kStage = 2 * kOp + 4 * kXBox;  // Hh Hl + X boxes (96 KB)
  constexpr uint32_t kTmemCols = 256;
  constexpr uint32_t kIdesc = idesc_tf32(kBM, 128);
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* qres = smem + NS * kStage;  // Qh, Ql of this CTA's row block
  Bars* bars = reinterpret_cast<Bars*>(qres + 2 * kOp);
  __shared__ uint64_t qbar;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t sblocks = (S + 127) / 128;
  const int mb = static_cast<int>(blockIdx.x % mblocks);
  const int64_t sb0 = blockIdx.x / mblocks;  // this CTA's tiles: sb0, sb0 + cpm, ...

  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(smem_u32(&bars->full[s]), 1);
      mbar_init(smem_u32(&bars->empty[s]), 1 + 4);  // MMA commit + four epilogue warps
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(smem_u32(&bars->tfull[a]), 1);
      mbar_init(smem_u32(&bars->tempty[a]), 4);
    }
    mbar_init(smem_u32(&bars->drain), 1);
    mbar_init(smem_u32(&qbar), 1);
    bars->abort_flag = 0;
    bars->issued = 0;
    bars->consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(smem_u32(&bars->tmem_base), kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = bars->tmem_base;
  volatile int* abort_flag = &bars->abort_flag;
  const uint64_t lim = wait_limit(status);

  if (warp == 0) {
    if (lane == 0) {
      const uint32_t qb = smem_u32(&qbar);
      mbar_expect_tx(qb, 2 * kOp);
      tma_load_2d(smem_u32(qres), &mapQ, qb, 0, mb * kBM);          // Qh
      tma_load_2d(smem_u32(qres + kOp), &mapQ, qb, 32, mb * kBM);   // Ql
      int it = 0;
      for (int64_t sb = sb0; sb < sblocks && !*abort_flag; sb += cpm, ++it) {
        const int st = it % NS;
        const uint32_t ph = (it / NS) & 1;
        if (!mbar_wait(smem_u32(&bars->empty[st]), ph ^ 1, abort_flag, lim)) {
          raise_timeout(bars, status);
          break;
        }
        const uint32_t a = smem_u32(smem + st * kStage);
        const uint32_t fb = smem_u32(&bars->full[st]);
        mbar_expect_tx(fb, kStage);
        const int s0 = static_cast<int>(sb * 128);
        tma_load_2d(a, &mapH, fb, 0, s0);                             // Hh
        tma_load_2d(a + kOp, &mapH, fb, 32, s0);                      // Hl
#pragma unroll
        for (int j = 0; j < 4; ++j)                                   // X, i 32 j .. 32 j + 31
          tma_load_2d(a + 2 * kOp + j * kXBox, &mapX, fb, mb * kBM + 32 * j, s0);
        bars->issued = it + 1;
      }
      // the resident Q load must land before the CTA can exit
      int dummy = 0;
      mbar_wait(qb, 0, reinterpret_cast<volatile int*>(&dummy));
    }
  } else if (warp == 1) {
    if (lane == 0) {
      bool ok = mbar_wait(smem_u32(&qbar), 0, abort_flag, lim);
      if (!ok) raise_timeout(bars, status);
      int it = 0;
      for (int64_t sb = sb0; ok && sb < sblocks && !*abort_flag; sb += cpm, ++it) {
        const int st = it % NS;
        const uint32_t ph = (it / NS) & 1;
        const int accb = it & 1;
        const uint32_t aph = (it >> 1) & 1;
        if (!mbar_wait(smem_u32(&bars->tempty[accb]), aph ^ 1, abort_flag, lim) ||
            !mbar_wait(smem_u32(&bars->full[st]), ph, abort_flag, lim)) {
          raise_timeout(bars, status);
          break;
        }
        tc_fence_after();
        const uint32_t a = smem_u32(smem + st * kStage);
        const uint32_t dt = tmem + accb * 128;
        const uint32_t hh = a, hl = a + kOp, qh = smem_u32(qres), ql = qh + kOp;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          mma_tf32(dt, sdesc(hh + 32 * k, 16, 1024), sdesc(qh + 32 * k, 16, 1024), kIdesc, k != 0);
          mma_tf32(dt, sdesc(hl + 32 * k, 16, 1024), sdesc(qh + 32 * k, 16, 1024), kIdesc, 1);
          mma_tf32(dt, sdesc(hh + 32 * k, 16, 1024), sdesc(ql + 32 * k, 16, 1024), kIdesc, 1);
        }
        mma_commit(smem_u32(&bars->empty[st]));
        mma_commit(smem_u32(&bars->tfull[accb]));
        bars->consumed = it + 1;
      }
      mma_commit(smem_u32(&bars->drain));
      int dummy = 0;
      mbar_wait(smem_u32(&bars->drain), 0, reinterpret_cast<volatile int*>(&dummy));
    }
  } else {
    const int q = warp & 3;
    const int srow = q * 32 + lane;  // s within the tile (TMEM lane)
    const uint32_t sw = static_cast<uint32_t>(srow & 7);
    double dsum = 0.0, xsum = 0.0;
    int it = 0;
    for (int64_t sb = sb0; sb < sblocks; sb += cpm, ++it) {
      const int st = it % NS;
      const int accb = it & 1;
      const uint32_t aph = (it >> 1) & 1;
      if (!mbar_wait(smem_u32(&bars->tfull[accb]), aph, abort_flag, lim)) {
        if (lane == 0) raise_timeout(bars, status);
        break;
      }
      tc_fence_after();
      const uint8_t* xrow = smem + st * kStage + 2 * kOp + srow * 128;
      const uint32_t base = tmem + (static_cast<uint32_t>(q * 32) << 16) + accb * 128;
      float d2 = 0.f, x2 = 0.f;
#pragma unroll 1
      for (int c0 = 0; c0 < 128; c0 += 16) {
        float v[16];
        tmem_ld16(base + c0, v);
        const uint8_t* bx = xrow + (c0 >> 5) * kXBox;
        const uint32_t j0 = static_cast<uint32_t>((c0 & 31) >> 2);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float4 xv = *reinterpret_cast<const float4*>(bx + (((j0 + u) ^ sw) << 4));
          const float xs[4] = {xv.x, xv.y, xv.z, xv.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const float df = xs[e] - v[4 * u + e];
            d2 = fmaf(df, df, d2);
            x2 = fmaf(xs[e], xs[e], x2);
          }
        }
      }
      dsum += d2;
      xsum += x2;
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(smem_u32(&bars->tempty[accb]));
        mbar_arrive(smem_u32(&bars->empty[st]));
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
      xsum += __shfl_xor_sync(0xffffffffu, xsum, o);
    }
    if (lane == 0) {
      atomicAdd(acc, dsum);
      atomicAdd(acc + 1, xsum);
    }
  }
  __syncthreads();
  if (warp == 0 && lane == 0 && bars->abort_flag) drain_loads<NS>(bars);
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

// rows of a K-major TF32 hi/lo pair: out[r * 64 + k] = v, out[r * 64 + 32 + k]
// = v - (v with the low 13 mantissa bits cleared), for k < c (zero for
// c <= k < 32), v = (float) src[k * ld_k + r * ld_r]
template <class T>
__global__ void pack_rows_tf32_kernel(const T* __restrict__ src, int64_t rows, int c, int64_t ld_k,
                                      int64_t ld_r, float* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < rows * 32;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int k = static_cast<int>(e & 31);
    const int64_t r = e >> 5;
    float v = 0.f;
    if (k < c) v = static_cast<float>(src[k * ld_k + r * ld_r]);
    out[r * 64 + k] = v;
    out[r * 64 + 32 + k] = v - __uint_as_float(__float_as_uint(v) & 0xFFFFE000u);
  }
}

// Combined FP32 factor buffer for the TF32 TTM: Fc[r * n1p + i], r < N:
// rows 0..L-1 the F_h part, rows Lp..Lp+L-1 the F_l part of F[i + ldf*r],
// zeros elsewhere and for i >= n1.
__global__ void pack_factor_tf32_kernel(const float* __restrict__ F, int64_t ldf, int64_t n1,
                                        int64_t n1p, int L, int Lp, int N,
                                        float* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n1p * N;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % n1p;
    const int r = static_cast<int>(e / n1p);
    float v = 0.f;
    if (i < n1) {
      if (r < L) {
        v = F[i + ldf * r];
      } else if (r >= Lp && r - Lp < L) {
        const float f = F[i + ldf * (r - Lp)];
        v = f - __uint_as_float(__float_as_uint(f) & 0xFFFFE000u);
      }
    }
    out[e] = v;
  }
}

// ----------------------------------------------------------------------------
// Y[i + n1*k] += sum_{t in range} w[t + T*k] * D_t[i, k],
// D_t[i, k] = sum_{i2} X[i, i2, t] Om2[i2, k]   (MN-major A, two 64-row boxes)
// XLO: X as a BF16 hi/lo pair; the lo boxes (map mapXlo) are multiplied by
// the same B into the same accumulator.
template <int N, int NS, bool XLO>
__global__ void __launch_bounds__(kThreads, 1)
    tc_mttkrp_kernel(const __grid_constant__ CUtensorMap mapX,
                     const __grid_constant__ CUtensorMap mapXlo,
                     const __grid_constant__ CUtensorMap mapB, int64_t n1, int64_t T, int kchunks,
                     int mblocks, int64_t t_per_cta, const float* __restrict__ w, int L,
                     float* __restrict__ Y, int* status) {
  constexpr uint32_t kBox = 64 * kBK * 2;  // 64 (i) x 64 (i2) BF16 = 8 KB
  constexpr uint32_t kAHi = 2 * kBox;
  constexpr uint32_t kABytes = (XLO ? 2 : 1) * kAHi;
  constexpr uint32_t kBBytes = N * kBK * 2;
  constexpr uint32_t kStage = kABytes + kBBytes;
  constexpr uint32_t kTmemCols = (2 * N <= 32) ? 32 : (2 * N <= 64) ? 64 : (2 * N <= 128) ? 128 : (2 * N <= 256) ? 256 : 512;
  constexpr uint32_t kIdesc = idesc_bf16(kBM, N, true, false);
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  Bars* bars = reinterpret_cast<Bars*>(smem + NS * kStage);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int mb = blockIdx.x % mblocks;
  const int64_t t0 = static_cast<int64_t>(blockIdx.x / mblocks) * t_per_cta;
  const int64_t t1 = min(T, t0 + t_per_cta);

  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(smem_u32(&bars->full[s]), 1);
      mbar_init(smem_u32(&bars->empty[s]), 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(smem_u32(&bars->tfull[a]), 1);
      mbar_init(smem_u32(&bars->tempty[a]), 4);
    }
    mbar_init(smem_u32(&bars->drain), 1);
    bars->abort_flag = 0;
    bars->issued = 0;
    bars->consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(smem_u32(&bars->tmem_base), kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = bars->tmem_base;
  volatile int* abort_flag = &bars->abort_flag;
  const uint64_t lim = wait_limit(status);

  if (warp == 0) {
    if (lane == 0) {
      int it = 0;
      for (int64_t t = t0; t < t1 && !*abort_flag; ++t) {
        for (int kc = 0; kc < kchunks; ++kc, ++it) {
          const int st = it % NS;
          const uint32_t ph = (it / NS) & 1;
          if (!mbar_wait(smem_u32(&bars->empty[st]), ph ^ 1, abort_flag, lim)) {
            raise_timeout(bars, status);
            break;
          }
          const uint32_t a = smem_u32(smem + st * kStage);
          const uint32_t fb = smem_u32(&bars->full[st]);
          mbar_expect_tx(fb, kStage);
          tma_load_3d(a, &mapX, fb, mb * kBM, kc * kBK, static_cast<int>(t));
          tma_load_3d(a + kBox, &mapX, fb, mb * kBM + 64, kc * kBK, static_cast<int>(t));
          if (XLO) {
            tma_load_3d(a + kAHi, &mapXlo, fb, mb * kBM, kc * kBK, static_cast<int>(t));
            tma_load_3d(a + kAHi + kBox, &mapXlo, fb, mb * kBM + 64, kc * kBK, static_cast<int>(t));
          }
          tma_load_2d(a + kABytes, &mapB, fb, kc * kBK, 0);
          bars->issued = it + 1;
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int it = 0, tl = 0;
      for (int64_t t = t0; t < t1 && !*abort_flag; ++t, ++tl) {
        const int acc = tl & 1;
        const uint32_t aph = (tl >> 1) & 1;
        if (!mbar_wait(smem_u32(&bars->tempty[acc]), aph ^ 1, abort_flag, lim)) {
          raise_timeout(bars, status);
          break;
        }
        tc_fence_after();
        const uint32_t dt = tmem + acc * N;
        bool ok = true;
        for (int kc = 0; kc < kchunks; ++kc, ++it) {
          const int st = it % NS;
          const uint32_t ph = (it / NS) & 1;
          if (!mbar_wait(smem_u32(&bars->full[st]), ph, abort_flag, lim)) {
            raise_timeout(bars, status);
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a = smem_u32(smem + st * kStage);
          const uint32_t b = a + kABytes;
          // A (MN-major): 8-row K groups 1024 B apart, the two 64-wide M atoms
          // kBox apart; each MMA (K = 16) spans two K groups.
#pragma unroll
          for (int k = 0; k < kBK / 16; ++k) {
            mma_bf16(dt, sdesc(a + 2048 * k, kBox, 1024), sdesc(b + 32 * k, 16, 1024), kIdesc,
                     (kc | k) != 0);
            if (XLO)
              mma_bf16(dt, sdesc(a + kAHi + 2048 * k, kBox, 1024), sdesc(b + 32 * k, 16, 1024),
                       kIdesc, 1);
          }
          mma_commit(smem_u32(&bars->empty[st]));
          bars->consumed = it + 1;
        }
        if (!ok) break;
        mma_commit(smem_u32(&bars->tfull[acc]));
      }
      mma_commit(smem_u32(&bars->drain));
      int dummy = 0;
      mbar_wait(smem_u32(&bars->drain), 0, reinterpret_cast<volatile int*>(&dummy));
    }
  } else {
    const int q = warp & 3;
    const int row = q * 32 + lane;
    const int64_t i = static_cast<int64_t>(mb) * kBM + row;
    float accum[N];
#pragma unroll
    for (int k = 0; k < N; ++k) accum[k] = 0.f;
    int tl = 0;
    for (int64_t t = t0; t < t1; ++t, ++tl) {
      const int acc = tl & 1;
      const uint32_t ph = (tl >> 1) & 1;
      if (!mbar_wait(smem_u32(&bars->tfull[acc]), ph, abort_flag, lim)) {
        if (lane == 0) raise_timeout(bars, status);
        break;
      }
      tc_fence_after();
      const uint32_t base = tmem + (static_cast<uint32_t>(q * 32) << 16) + acc * N;
#pragma unroll
      for (int c0 = 0; c0 < N; c0 += 16) {
        float v[16];
        tmem_ld16(base + c0, v);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int k = c0 + j;
          const float wk = (k < L) ? __ldg(w + t + T * k) : 0.f;
          accum[k] = fmaf(wk, v[j], accum[k]);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&bars->tempty[acc]));
    }
    if (i < n1) {
#pragma unroll
      for (int k = 0; k < N; ++k)
        if (k < L) atomicAdd(Y + i + n1 * k, accum[k]);
    }
  }
  __syncthreads();
  if (warp == 0 && lane == 0 && bars->abort_flag) drain_loads<NS>(bars);
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

// ----------------------------------------------------------------------------
// Dimension tree in one pass over X (Sec. 5.1, memoization): X viewed as
// (n1, n2, T), T = prod_{j>=3} n_j, w[t, k] = prod_{j>=3} Omega_j[i_j(t), k].
// Work items are (i2 block b of 128 rows, slab t).  The i1 range is cut into
// segments of kseg chunks of 128 rows, so that a segment's accumulators fit
// in TMEM; a CTA owns one segment and a contiguous range of items (b-major).
// It keeps the segment's rows of Omega1 resident in shared memory (loaded
// once by TMA) and streams the tiles X[128 i1, 128 i2, t] (two 64-wide
// boxes; with XLO also the lo plane's two boxes) through an NS-stage ring.
// Each tile is read twice by the tensor core:
//   MMA1 (K-major, rows i2, K = i1): D1[i2, k] = sum_i1 X Omega1, per item
//        (a partial over the segment's i1);
//   MMA2 (MN-major, M = i1, K = i2): D2[i1, :] += X [B2hi_t | B2lo_t], one
//        MMA of width 2N per K step.  B2_t[i2, k] = Omega2[i2, k] w[t, k] is
//        exact as a BF16 hi/lo pair (hi in operand rows 0..N-1, lo in rows
//        N..2N-1), written to shared memory per item by a producer
//        warpgroup; D2 accumulates over a group of items, and its two column
//        halves are summed when it is stored.
// XLO adds Xlo Omega1 to D1 and Xlo B2hi_t to D2's hi half (the dropped
// Xlo B2lo_t is below 2^-16 relative).
// Long accumulation chains in TMEM lose accuracy (the error of a chain of m
// MMA accumulations grows about linearly in m), so with drain > 0 the CTA's
// items are cut into groups of `drain` items (chains of 8 drain K steps per
// accumulator); after each group the epilogue adds D2 into the CTA's FP32
// partials of Y1.  With nd2 = 2 buffers the MMAs fill one while the other is
// stored; with one buffer the next group waits for the store.  Without
// draining D2 holds all of the CTA's items and is stored once at the end.
// Epilogue per item: Y2[i2, k] += D1 w[t, k] (registers, flushed when the
// block b changes) and C[t, k] = sum_i2 Omega2[i2, k] D1[i2, k]: each warp
// reduces its 32 rows (warp reduce-scatter) and adds them into a shared
// slot with shared-memory atomics; the last of the four warps to finish the
// item stores the slot into the item's entry of the C partials and clears
// it (no barrier among the warps, so an aborted CTA cannot deadlock).
// Second kernels sum the Y1 and C partials in a fixed order (no global
// atomics on the contended C rows).  For d = 3, C is Y3 itself.
// Warp reduce-scatter of CNT per-lane values: on return the warp's sums over
// its 32 lanes have been handed to sink(kbase + j, sum) by one lane each
// (j < CNT).  Each halving step exchanges half of the values with the lane
// BIT apart (CNT/2 shuffles) and keeps the half selected by that lane bit;
// the bits left when CNT is odd are summed by a plain butterfly.  For 16
// values: 8 + 4 + 2 + 1 + 1 = 16 shuffles instead of 16 x 5.
template <int CNT, int BIT>
struct WarpReduceScatter {
  template <class Sink>
  __device__ __forceinline__ static void run(float* v, int lane, int kbase, Sink&& sink) {
    if constexpr (BIT > 0 && CNT % 2 == 0) {
      constexpr int H = CNT / 2;
      const bool hb = (lane & BIT) != 0;
#pragma unroll
      for (int j = 0; j < H; ++j) {
        const float keep = hb ? v[H + j] : v[j];
        const float send = hb ? v[j] : v[H + j];
        v[j] = keep + __shfl_xor_sync(0xffffffffu, send, BIT);
      }
      WarpReduceScatter<H, BIT / 2>::run(v, lane, kbase + (hb ? H : 0), sink);
    } else {
#pragma unroll
      for (int j = 0; j < CNT; ++j) {
        float x = v[j];
#pragma unroll
        for (int b = BIT; b > 0; b >>= 1) x += __shfl_xor_sync(0xffffffffu, x, b);
        v[j] = x;
      }
      constexpr int kMask = BIT > 0 ? 2 * BIT - 1 : 0;  // the lane bits still shared
      if ((lane & kMask) == 0) {
#pragma unroll
        for (int j = 0; j < CNT; ++j) sink(kbase + j, v[j]);
      }
    }
  }
};

struct TreeArgs {
  const float* w;            // T x L
  const float* om2;          // n2 x L (column-major): the second operand's factor
  float* Y2;                 // n2 x L
  float* Cw;                 // C partials: [seg nb + b][t][k < N]
  float* Yw;                 // Y1 partials: [cta][k < N][kseg * 128 rows of its segment]
  int64_t n2, T, items;      // items = nb * T
  int L, nb, kch, kseg, cps; // kch = ceil(n1 / 128); cps = CTAs per segment
  int drain, nd2;            // items per D2 accumulation chain (0: all), D2 buffers
};

// TMEM columns of the tree: D1 double buffer (2N) + nd2 buffers of the
// segment's D2 (2N per chunk)
__host__ __device__ constexpr int tree_kseg_max(int N, int nd2) {
  return (512 - 2 * N) / (nd2 * 2 * N);
}

template <int N, int NS, bool XLO>
__global__ void __launch_bounds__(320, 1)
    tc_tree_kernel(const __grid_constant__ CUtensorMap mapX,
                   const __grid_constant__ CUtensorMap mapXlo,
                   const __grid_constant__ CUtensorMap mapF, const TreeArgs P, int* status) {
  constexpr uint32_t kXBox = 64 * 128 * 2;            // 64 i1 x 128 i2
  constexpr uint32_t kStage = (XLO ? 4 : 2) * kXBox;  // hi boxes, then lo boxes
  constexpr uint32_t kFBox = N * 128;                 // N rows (k) x 64 i1
  constexpr uint32_t kB2Atom = 2 * N * 128;           // 2N rows (hi, lo) x 64 i2
  constexpr uint32_t kB2Buf = 2 * kB2Atom;            // i2 0..63 and 64..127
  constexpr uint32_t kIdesc1 = idesc_bf16(kBM, N, false, false);
  constexpr uint32_t kIdesc2 = idesc_bf16(kBM, 2 * N, true, false);
  constexpr uint32_t kIdesc2h = idesc_bf16(kBM, N, true, false);
  static_assert(N % 16 == 0 && N <= 64, "tree width");
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* fres = smem;                           // 2 kseg boxes of Omega1 (resident)
  uint8_t* xst = fres + 2 * P.kseg * kFBox;       // X ring
  uint8_t* b2 = xst + NS * kStage;                // two B2 buffers
  Bars* bars = reinterpret_cast<Bars*>(b2 + 2 * kB2Buf);
  __shared__ uint64_t b2full[2], b2empty[2], fbar, d2full[2], d2empty[2];
  __shared__ float wsm[2][N];  // w[t, :] beside B2_t, same double buffering
  __shared__ float csm[2][N];  // C[t, :] of the item, summed over the four epilogue warps
  __shared__ int cdone[2];     // warps done with the item's csm slot
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int seg = blockIdx.x / P.cps;
  const int rk = blockIdx.x % P.cps;
  const int64_t j0 = P.items * rk / P.cps, j1 = P.items * (rk + 1) / P.cps;
  const int c0 = seg * P.kseg;                        // first 128-row chunk of i1
  const int kc = min(P.kseg, P.kch - c0);             // chunks in this segment
  const uint32_t tmem_cols = 512;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(smem_u32(&bars->full[s]), 1);
      mbar_init(smem_u32(&bars->empty[s]), 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(smem_u32(&bars->tfull[a]), 1);
      mbar_init(smem_u32(&bars->tempty[a]), 4);
      mbar_init(smem_u32(&b2full[a]), 4);
      mbar_init(smem_u32(&b2empty[a]), 1 + 4);  // MMA commit + four epilogue warps (wsm)
      mbar_init(smem_u32(&d2full[a]), 1);
      mbar_init(smem_u32(&d2empty[a]), 4);
      cdone[a] = 0;
    }
    for (int k = 0; k < 2 * N; ++k) (&csm[0][0])[k] = 0.f;
    mbar_init(smem_u32(&fbar), 1);
    mbar_init(smem_u32(&bars->drain), 1);
    bars->abort_flag = 0;
    bars->issued = 0;
    bars->consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(smem_u32(&bars->tmem_base), tmem_cols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  // D1 buffers at columns 0 and N; chunk c of D2 buffer u at (2 + 2 (u kseg + c)) N
  const uint32_t tmem = bars->tmem_base;
  volatile int* abort_flag = &bars->abort_flag;
  const uint64_t lim = wait_limit(status);

  if (warp == 0) {
    if (lane == 0) {
      // the segment's rows of Omega1, once
      mbar_expect_tx(smem_u32(&fbar), static_cast<uint32_t>(2 * kc) * kFBox);
      for (int c = 0; c < kc; ++c)
        for (int h = 0; h < 2; ++h)
          tma_load_2d(smem_u32(fres + (2 * c + h) * kFBox), &mapF, smem_u32(&fbar),
                      (c0 + c) * 128 + h * 64, 0);
      int it = 0;
      for (int64_t j = j0; j < j1 && !*abort_flag; ++j) {
        const int b = static_cast<int>(j / P.T);
        const int t = static_cast<int>(j % P.T);
        for (int c = 0; c < kc; ++c, ++it) {
          const int st = it % NS;
          const uint32_t ph = (it / NS) & 1;
          if (!mbar_wait(smem_u32(&bars->empty[st]), ph ^ 1, abort_flag, lim)) {
            raise_timeout(bars, status);
            break;
          }
          const uint32_t a = smem_u32(xst + st * kStage);
          const uint32_t fb = smem_u32(&bars->full[st]);
          const int x0 = (c0 + c) * 128;
          mbar_expect_tx(fb, kStage);
          tma_load_3d(a, &mapX, fb, x0, b * 128, t);
          tma_load_3d(a + kXBox, &mapX, fb, x0 + 64, b * 128, t);
          if (XLO) {
            tma_load_3d(a + 2 * kXBox, &mapXlo, fb, x0, b * 128, t);
            tma_load_3d(a + 3 * kXBox, &mapXlo, fb, x0 + 64, b * 128, t);
          }
          bars->issued = it + 1;
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // Omega1 must have landed before the first MMA (and before exit)
      const bool f_ok = mbar_wait(smem_u32(&fbar), 0, abort_flag, lim);
      if (!f_ok) raise_timeout(bars, status);
      tc_fence_after();
      const uint64_t fdesc = sdesc(smem_u32(fres), 16, 1024);
      int it = 0, tl = 0;
      for (int64_t j = j0; f_ok && j < j1 && !*abort_flag; ++j, ++tl) {
        const int acc = tl & 1;
        const uint32_t aph = (tl >> 1) & 1;
        if (!mbar_wait(smem_u32(&bars->tempty[acc]), aph ^ 1, abort_flag, lim) ||
            !mbar_wait(smem_u32(&b2full[acc]), aph, abort_flag, lim)) {
          raise_timeout(bars, status);
          break;
        }
        // the D2 buffer of this item's group; the group's first item starts
        // its chains, once the buffer's previous group has been stored
        const int grp = P.drain ? tl / P.drain : 0;
        const int u = grp % P.nd2;
        const bool first = P.drain ? (tl % P.drain == 0) : (tl == 0);
        const bool last = P.drain && (tl % P.drain == P.drain - 1 || j == j1 - 1);
        if (P.drain && first &&
            !mbar_wait(smem_u32(&d2empty[u]), ((grp / P.nd2) & 1) ^ 1, abort_flag, lim)) {
          raise_timeout(bars, status);
          break;
        }
        tc_fence_after();
        const uint32_t d1 = tmem + acc * N;
        const uint32_t d2b = tmem + (2 + 2 * u * P.kseg) * N;
        const uint64_t bdesc = sdesc(smem_u32(b2 + acc * kB2Buf), 16, 1024);
        bool ok = true;
        for (int c = 0; c < kc; ++c, ++it) {
          const int st = it % NS;
          const uint32_t ph = (it / NS) & 1;
          if (!mbar_wait(smem_u32(&bars->full[st]), ph, abort_flag, lim)) {
            raise_timeout(bars, status);
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a = smem_u32(xst + st * kStage);
          // descriptors differ only in their start address (field in 16-byte
          // units, no carry: shared addresses are below 2^18)
          const uint64_t ak = sdesc(a, 16, 1024);       // K-major view (MMA1)
          const uint64_t am = sdesc(a, kXBox, 1024);    // MN-major view (MMA2)
          // MMA1: rows i2, K = i1 (two 64-wide boxes, 4 K-steps each)
#pragma unroll
          for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const uint64_t fo = ((2 * c + h) * kFBox + 32 * k) >> 4;
              mma_bf16(d1, ak + ((h * kXBox + 32 * k) >> 4), fdesc + fo, kIdesc1, (c | h | k) != 0);
              if (XLO)
                mma_bf16(d1, ak + (((2 + h) * kXBox + 32 * k) >> 4), fdesc + fo, kIdesc1, 1u);
            }
          // MMA2: M = i1 (the two boxes kXBox apart), K = i2 (128 rows, 8 K-steps),
          // B = [B2hi | B2lo] (2N rows per 64-wide K atom); the lo plane of X
          // takes the hi rows only
          const uint32_t d2 = d2b + 2 * c * N;
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const uint64_t bo = ((k >> 2) * kB2Atom + 32 * (k & 3)) >> 4;
            mma_bf16(d2, am + ((2048 * k) >> 4), bdesc + bo, kIdesc2, (!first || k != 0) ? 1u : 0u);
            if (XLO) mma_bf16(d2, am + ((2 * kXBox + 2048 * k) >> 4), bdesc + bo, kIdesc2h, 1u);
          }
          mma_commit(smem_u32(&bars->empty[st]));
          bars->consumed = it + 1;
        }
        if (!ok) break;
        mma_commit(smem_u32(&bars->tfull[acc]));
        mma_commit(smem_u32(&b2empty[acc]));
        if (last) mma_commit(smem_u32(&d2full[u]));
      }
      mma_commit(smem_u32(&bars->drain));
      int dummy = 0;
      mbar_wait(smem_u32(&bars->drain), 0, reinterpret_cast<volatile int*>(&dummy));
    }
  } else if (warp >= 6) {
    // B2 producer warpgroup: B2_t[i2, k] = Omega2[i2, k] w[t, k] in the K-major
    // 128-byte swizzled layout (rows k, 64 i2 per atom): hi in row k, lo in
    // row N + k (the same swizzle phase, N being a multiple of 8).
    const int tid = threadIdx.x - 192;  // 0..127, one i2 row each
    const int col = tid & 63;
    float om[N];
    int cur_b = -1;
    int tl = 0;
    // w[t, :]: two loads per lane, shared within the warp by shuffles (no
    // barrier across the producer warps), loaded one item ahead; the first
    // warp also stages it in shared memory for the epilogue (published by
    // the b2full arrival)
    auto load_w = [&](int64_t jj, float& a0, float& a1) {
      const int64_t tt = jj % P.T;
      a0 = (jj < j1 && lane < P.L) ? __ldg(P.w + tt + P.T * lane) : 0.f;
      a1 = (jj < j1 && lane + 32 < P.L) ? __ldg(P.w + tt + P.T * (lane + 32)) : 0.f;
    };
    float nw0, nw1;
    load_w(j0, nw0, nw1);
    for (int64_t j = j0; j < j1; ++j, ++tl) {
      const int b = static_cast<int>(j / P.T);
      if (b != cur_b) {
        cur_b = b;
        const int64_t i2 = static_cast<int64_t>(b) * 128 + tid;
#pragma unroll
        for (int k = 0; k < N; ++k)
          om[k] = (k < P.L && i2 < P.n2) ? P.om2[i2 + P.n2 * k] : 0.f;
      }
      const float wl0 = nw0, wl1 = nw1;
      load_w(j + 1, nw0, nw1);
      const int buf = tl & 1;
      const uint32_t ph = (tl >> 1) & 1;
      if (!mbar_wait(smem_u32(&b2empty[buf]), ph ^ 1, abort_flag, lim)) {
        if (lane == 0) raise_timeout(bars, status);
        break;
      }
      uint8_t* base = b2 + buf * kB2Buf + (tid >> 6) * kB2Atom;
      if (tid < 32) {
        if (lane < N) wsm[buf][lane] = wl0;
        if (lane + 32 < N) wsm[buf][lane + 32] = wl1;
      }
#pragma unroll
      for (int k = 0; k < N; ++k) {
        const float v = om[k] * __shfl_sync(0xffffffffu, k < 32 ? wl0 : wl1, k & 31);
        const __nv_bfloat16 hi = __float2bfloat16_rn(v);
        const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
        const uint32_t off = k * 128 + ((((col >> 3) ^ (k & 7)) << 4)) + (col & 7) * 2;
        *reinterpret_cast<__nv_bfloat16*>(base + off) = hi;
        *reinterpret_cast<__nv_bfloat16*>(base + N * 128 + off) = lo;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&b2full[buf]));
    }
  } else {
    const int q = warp & 3;
    const int row = q * 32 + lane;  // i2 within the block; i1 within a chunk
    float y2[N];
    float o2[N];
    int cur_b = -1;
    int64_t i2 = 0;
    bool valid = false;
    auto flush_y2 = [&]() {
      if (valid) {
#pragma unroll
        for (int k = 0; k < N; ++k)
          if (k < P.L) atomicAdd(P.Y2 + i2 + P.n2 * k, y2[k]);
      }
    };
    // D2 buffer u -> the CTA's partials of Y1 for its segment (hi and lo
    // halves summed), coalesced over i1; `init` stores, otherwise adds; a
    // buffer that holds nothing (`have` false) contributes zeros
    const int64_t segrows = static_cast<int64_t>(P.kseg) * 128;
    float* yw = P.Yw + static_cast<size_t>(blockIdx.x) * N * segrows;
    auto store_d2 = [&](int u, bool init, bool have) {
      for (int c = 0; c < P.kseg; ++c) {
        const uint32_t base =
            tmem + (static_cast<uint32_t>(q * 32) << 16) + (2 + 2 * (u * P.kseg + c)) * N;
#pragma unroll
        for (int cc = 0; cc < N; cc += 16) {
          float vh[16], vl[16];
          if (have && c < kc) {
            tmem_ld16(base + cc, vh);
            tmem_ld16(base + N + cc, vl);
          } else {
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) vh[jj] = vl[jj] = 0.f;
          }
          float* dst = yw + static_cast<size_t>(cc) * segrows + c * 128 + row;
          // the 16 old values are loaded before any store (one L2 round trip)
          float prev[16];
#pragma unroll
          for (int jj = 0; jj < 16; ++jj)
            prev[jj] = init ? 0.f : __ldcg(dst + static_cast<size_t>(jj) * segrows);
#pragma unroll
          for (int jj = 0; jj < 16; ++jj)
            __stcg(dst + static_cast<size_t>(jj) * segrows, prev[jj] + (vh[jj] + vl[jj]));
        }
      }
    };
    int tl = 0;
    for (int64_t j = j0; j < j1; ++j, ++tl) {
      const int b = static_cast<int>(j / P.T);
      const int64_t t = j % P.T;
      if (b != cur_b) {
        if (cur_b >= 0) flush_y2();
        cur_b = b;
        i2 = static_cast<int64_t>(b) * 128 + row;
        valid = i2 < P.n2;
#pragma unroll
        for (int k = 0; k < N; ++k) {
          y2[k] = 0.f;
          o2[k] = (valid && k < P.L) ? P.om2[i2 + P.n2 * k] : 0.f;
        }
      }
      const int acc = tl & 1;
      const uint32_t ph = (tl >> 1) & 1;
      if (!mbar_wait(smem_u32(&bars->tfull[acc]), ph, abort_flag, lim)) {
        if (lane == 0) raise_timeout(bars, status);
        break;
      }
      // w[t, :] was staged with B2_t (that phase is complete once tfull is)
      if (!mbar_wait(smem_u32(&b2full[acc]), ph, abort_flag, lim)) {
        if (lane == 0) raise_timeout(bars, status);
        break;
      }
      tc_fence_after();
      const uint32_t base = tmem + (static_cast<uint32_t>(q * 32) << 16) + acc * N;
      // the item's entry of the C partials
      float* cw = P.Cw + (static_cast<size_t>(seg) * P.nb + b) * P.T * N +
                  static_cast<size_t>(t) * N;
      // all of D1's columns in flight at once, one wait
      float v[N];
#pragma unroll
      for (int cc = 0; cc < N; cc += 16) tmem_ld16_issue(base + cc, v + cc);
      tmem_ld_wait();
#pragma unroll
      for (int cc = 0; cc < N; cc += 16) {
        float cp[16];
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) {
          const int k = cc + jj;
          y2[k] = fmaf(v[k], wsm[acc][k], y2[k]);
          cp[jj] = v[k] * o2[k];
        }
        WarpReduceScatter<16, 16>::run(cp, lane, cc,
                                       [&](int k, float x) { atomicAdd(&csm[acc][k], x); });
      }
      // the last warp stores the slot and clears it; it is reused two items
      // later, which the MMAs reach only after all four warps have released
      // D1 buffer acc below
      __syncwarp();
      int last_w = 0;
      if (lane == 0) {
        __threadfence_block();
        last_w = atomicAdd(&cdone[acc], 1) == 3;
      }
      last_w = __shfl_sync(0xffffffffu, last_w, 0);
      if (last_w) {
        __threadfence_block();
        for (int k = lane; k < N; k += 32) {
          cw[k] = csm[acc][k];
          csm[acc][k] = 0.f;
        }
        if (lane == 0) cdone[acc] = 0;
        __threadfence_block();
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(smem_u32(&bars->tempty[acc]));
        mbar_arrive(smem_u32(&b2empty[acc]));
      }
      if (P.drain && (tl % P.drain == P.drain - 1 || j == j1 - 1)) {
        const int grp = tl / P.drain;
        const int u = grp % P.nd2;
        if (!mbar_wait(smem_u32(&d2full[u]), (grp / P.nd2) & 1, abort_flag, lim)) {
          if (lane == 0) raise_timeout(bars, status);
          break;
        }
        tc_fence_after();
        store_d2(u, grp == 0, true);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&d2empty[u]));
      }
    }
    if (cur_b >= 0) flush_y2();
    // Without draining, D2 (complete once the last tfull has been observed)
    // is stored once; a CTA without items stores zeros
    const bool have = j1 > j0 && !*abort_flag;
    if (!P.drain || !have) {
      if (have) tc_fence_after();
      store_d2(0, true, have);
    }
  }
  __syncthreads();
  if (warp == 0 && lane == 0 && bars->abort_flag) {
    drain_loads<NS>(bars);
    int dummy = 0;  // the resident Omega1 load too (bounded)
    mbar_wait(smem_u32(&fbar), 0, reinterpret_cast<volatile int*>(&dummy));
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, tmem_cols);
  }
}

// ----------------------------------------------------------------------------
// Residual of the BF16 form: acc[0] += ||X - Q1 H||_F^2, acc[1] += ||X||_F^2,
// X n1 x S (BF16), Q1 n1 x c (K-major rows, BF16 hi/lo), H c x S (K-major rows
// per s, BF16 hi/lo), c <= 64 padded to 64.  The tile is the transpose,
// X_hat^T[s, i] for 128 columns s (TMEM lanes) x 128 rows i (TMEM columns):
// A = H (M = s), B = Q1 (N = i), X_hat^T = Hh Qh^T + Hl Qh^T + Hh Ql^T (the
// dropped Hl Ql^T term is below 2^-16 relative).  In that orientation an
// epilogue thread owns one s and 16 consecutive i per TMEM load, which are
// two 16-byte chunks of the X tile as TMA placed it ([s][64 i] rows of 128 B,
// chunks swizzled by s mod 8), so X is read with 16-byte shared loads.
// A CTA keeps one 128-row block of Q1 (hi and lo, 32 KB) resident and walks
// the column tiles of that block; the CTAs of one column tile run together,
// so each H tile comes from HBM once and from L2 for the other blocks.  A
// stage (H hi/lo + X boxes) is released when both the MMAs (tcgen05.commit)
// and the four epilogue warps are done with it.  XLO: X is a BF16 hi/lo pair
// (two more boxes per stage); the epilogue compares with hi + lo.
template <bool XLO>
__global__ void __launch_bounds__(kThreads, 1)
    tc_residual_kernel(const __grid_constant__ CUtensorMap mapX,
                       const __grid_constant__ CUtensorMap mapXlo,
                       const __grid_constant__ CUtensorMap mapQ,
                       const __grid_constant__ CUtensorMap mapH, int64_t n1, int64_t S,
                       int mblocks, int cpm, double* __restrict__ acc, int* status) {
  constexpr int NS = XLO ? 2 : 3;
  constexpr uint32_t kOp = 128 * 128;            // one 128-row x 64-element BF16 operand tile
  constexpr uint32_t kXBox = 64 * 128 * 2;       // 64 (i) x 128 (s) BF16
  constexpr uint32_t kXNum = XLO ? 4 : 2;
  constexpr uint32_t kStage = 2 * kOp + kXNum * kXBox;  // Hh Hl + X boxes
  constexpr uint32_t kTmemCols = 256;
  constexpr uint32_t kIdesc = idesc_bf16(kBM, 128, false, false);
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* qres = smem + NS * kStage;  // Qh, Ql of this CTA's row block
  Bars* bars = reinterpret_cast<Bars*>(qres + 2 * kOp);
  __shared__ uint64_t qbar;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t sblocks = (S + 127) / 128;
  const int mb = static_cast<int>(blockIdx.x % mblocks);
  const int64_t sb0 = blockIdx.x / mblocks;  // this CTA's tiles: sb0, sb0 + cpm, ...

  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(smem_u32(&bars->full[s]), 1);
      mbar_init(smem_u32(&bars->empty[s]), 1 + 4);  // MMA commit + four epilogue warps
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(smem_u32(&bars->tfull[a]), 1);
      mbar_init(smem_u32(&bars->tempty[a]), 4);
    }
    mbar_init(smem_u32(&bars->drain), 1);
    mbar_init(smem_u32(&qbar), 1);
    bars->abort_flag = 0;
    bars->issued = 0;
    bars->consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(smem_u32(&bars->tmem_base), kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = bars->tmem_base;
  volatile int* abort_flag = &bars->abort_flag;
  const uint64_t lim = wait_limit(status);

  if (warp == 0) {
    if (lane == 0) {
      const uint32_t qb = smem_u32(&qbar);
      mbar_expect_tx(qb, 2 * kOp);
      tma_load_2d(smem_u32(qres), &mapQ, qb, 0, mb * kBM);          // Qh
      tma_load_2d(smem_u32(qres + kOp), &mapQ, qb, 64, mb * kBM);   // Ql
      int it = 0;
      for (int64_t sb = sb0; sb < sblocks && !*abort_flag; sb += cpm, ++it) {
        const int st = it % NS;
        const uint32_t ph = (it / NS) & 1;
        if (!mbar_wait(smem_u32(&bars->empty[st]), ph ^ 1, abort_flag, lim)) {
          raise_timeout(bars, status);
          break;
        }
        const uint32_t a = smem_u32(smem + st * kStage);
        const uint32_t fb = smem_u32(&bars->full[st]);
        mbar_expect_tx(fb, kStage);
        const int s0 = static_cast<int>(sb * 128);
        tma_load_2d(a, &mapH, fb, 0, s0);                             // Hh
        tma_load_2d(a + kOp, &mapH, fb, 64, s0);                      // Hl
        tma_load_2d(a + 2 * kOp, &mapX, fb, mb * kBM, s0);            // X, i 0..63
        tma_load_2d(a + 2 * kOp + kXBox, &mapX, fb, mb * kBM + 64, s0);  // i 64..127
        if (XLO) {
          tma_load_2d(a + 2 * kOp + 2 * kXBox, &mapXlo, fb, mb * kBM, s0);
          tma_load_2d(a + 2 * kOp + 3 * kXBox, &mapXlo, fb, mb * kBM + 64, s0);
        }
        bars->issued = it + 1;
      }
      // the resident Q load must land before the CTA can exit
      int dummy = 0;
      mbar_wait(qb, 0, reinterpret_cast<volatile int*>(&dummy));
    }
  } else if (warp == 1) {
    if (lane == 0) {
      bool ok = mbar_wait(smem_u32(&qbar), 0, abort_flag, lim);
      if (!ok) raise_timeout(bars, status);
      int it = 0;
      for (int64_t sb = sb0; ok && sb < sblocks && !*abort_flag; sb += cpm, ++it) {
        const int st = it % NS;
        const uint32_t ph = (it / NS) & 1;
        const int accb = it & 1;
        const uint32_t aph = (it >> 1) & 1;
        if (!mbar_wait(smem_u32(&bars->tempty[accb]), aph ^ 1, abort_flag, lim) ||
            !mbar_wait(smem_u32(&bars->full[st]), ph, abort_flag, lim)) {
          raise_timeout(bars, status);
          break;
        }
        tc_fence_after();
        const uint32_t a = smem_u32(smem + st * kStage);
        const uint32_t dt = tmem + accb * 128;
        const uint32_t hh = a, hl = a + kOp, qh = smem_u32(qres), ql = qh + kOp;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          mma_bf16(dt, sdesc(hh + 32 * k, 16, 1024), sdesc(qh + 32 * k, 16, 1024), kIdesc, k != 0);
          mma_bf16(dt, sdesc(hl + 32 * k, 16, 1024), sdesc(qh + 32 * k, 16, 1024), kIdesc, 1);
          mma_bf16(dt, sdesc(hh + 32 * k, 16, 1024), sdesc(ql + 32 * k, 16, 1024), kIdesc, 1);
        }
        mma_commit(smem_u32(&bars->empty[st]));
        mma_commit(smem_u32(&bars->tfull[accb]));
        bars->consumed = it + 1;
      }
      mma_commit(smem_u32(&bars->drain));
      int dummy = 0;
      mbar_wait(smem_u32(&bars->drain), 0, reinterpret_cast<volatile int*>(&dummy));
    }
  } else {
    const int q = warp & 3;
    const int srow = q * 32 + lane;  // s within the tile (TMEM lane)
    const uint32_t sw = static_cast<uint32_t>(srow & 7);
    double dsum = 0.0, xsum = 0.0;
    int it = 0;
    for (int64_t sb = sb0; sb < sblocks; sb += cpm, ++it) {
      const int st = it % NS;
      const int accb = it & 1;
      const uint32_t aph = (it >> 1) & 1;
      if (!mbar_wait(smem_u32(&bars->tfull[accb]), aph, abort_flag, lim)) {
        if (lane == 0) raise_timeout(bars, status);
        break;
      }
      tc_fence_after();
      const uint8_t* xrow = smem + st * kStage + 2 * kOp + srow * 128;
      const uint32_t base = tmem + (static_cast<uint32_t>(q * 32) << 16) + accb * 128;
      float d2 = 0.f, x2 = 0.f;
#pragma unroll 1
      for (int c0 = 0; c0 < 128; c0 += 16) {
        float v[16];
        tmem_ld16(base + c0, v);
        const uint8_t* bx = xrow + (c0 >> 6) * kXBox;
        const uint32_t j0 = static_cast<uint32_t>((c0 & 63) >> 3);
        uint4 w[2];
        w[0] = *reinterpret_cast<const uint4*>(bx + (((j0) ^ sw) << 4));
        w[1] = *reinterpret_cast<const uint4*>(bx + (((j0 + 1) ^ sw) << 4));
        uint4 wl[2];
        if (XLO) {
          wl[0] = *reinterpret_cast<const uint4*>(bx + 2 * kXBox + (((j0) ^ sw) << 4));
          wl[1] = *reinterpret_cast<const uint4*>(bx + 2 * kXBox + (((j0 + 1) ^ sw) << 4));
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const uint32_t u[4] = {w[h].x, w[h].y, w[h].z, w[h].w};
          uint32_t ul[4] = {0u, 0u, 0u, 0u};
          if (XLO) {
            ul[0] = wl[h].x;
            ul[1] = wl[h].y;
            ul[2] = wl[h].z;
            ul[3] = wl[h].w;
          }
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            float xa = __uint_as_float(u[e] << 16);          // element 2e (low half)
            float xb = __uint_as_float(u[e] & 0xFFFF0000u);  // element 2e + 1
            if (XLO) {
              xa += __uint_as_float(ul[e] << 16);
              xb += __uint_as_float(ul[e] & 0xFFFF0000u);
            }
            const float da = xa - v[h * 8 + 2 * e], db = xb - v[h * 8 + 2 * e + 1];
            d2 = fmaf(da, da, d2);
            d2 = fmaf(db, db, d2);
            x2 = fmaf(xa, xa, x2);
            x2 = fmaf(xb, xb, x2);
          }
        }
      }
      dsum += d2;
      xsum += x2;
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(smem_u32(&bars->tempty[accb]));
        mbar_arrive(smem_u32(&bars->empty[st]));
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
      xsum += __shfl_xor_sync(0xffffffffu, xsum, o);
    }
    if (lane == 0) {
      atomicAdd(acc, dsum);
      atomicAdd(acc + 1, xsum);
    }
  }
  __syncthreads();
  if (warp == 0 && lane == 0 && bars->abort_flag) drain_loads<NS>(bars);
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

// Y1[i + n1 k] = sum over the cps CTAs of i's segment (in order) of their
// partials Yw[cta][k][i - first row of the segment]
__global__ void tree_reduce_kernel(const float* __restrict__ Yw, int cps, int64_t segrows,
                                   int64_t n1, int L, int N, float* __restrict__ Y1) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n1 * L;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % n1;
    const int k = static_cast<int>(e / n1);
    const int64_t seg = i / segrows;
    const size_t step = static_cast<size_t>(N) * segrows;
    const float* src = Yw + seg * cps * step + static_cast<size_t>(k) * segrows + (i - seg * segrows);
    float acc = 0.f;
    for (int c = 0; c < cps; ++c) acc += src[c * step];
    Y1[e] = acc;
  }
}

// C[t + T k] = sum over the `parts` partial slots p of Cw[(p T + t) N + k]:
// one CTA per slab t, 256 threads as 8 slices x 32 lanes over k; lane k' of
// slice q sums the slots p = q, q + 8, ..., the slices then add up in a
// fixed order in shared memory
__global__ void __launch_bounds__(256) tree_c_reduce_kernel(const float* __restrict__ Cw,
                                                            int64_t parts, int64_t T, int L, int N,
                                                            float* __restrict__ C) {
  __shared__ float part[8][64];
  const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const size_t step = static_cast<size_t>(T) * N;
  for (int64_t t = blockIdx.x; t < T; t += gridDim.x) {
    for (int k0 = 0; k0 < L; k0 += 32) {
      const int k = k0 + lane;
      float acc = 0.f;
      if (k < L) {
        const float* src = Cw + static_cast<size_t>(t) * N + k;
        for (int64_t p = q; p < parts; p += 8) acc += src[p * step];
      }
      part[q][lane] = acc;
      __syncthreads();
      if (q == 0 && k < L) {
        float s = 0.f;
        for (int r = 0; r < 8; ++r) s += part[r][lane];
        C[t + T * k] = s;
      }
      __syncthreads();
    }
  }
}

// rows of a K-major hi/lo pair: out[r * 128 + k] = hi(v), out[r * 128 + 64 + k]
// = lo(v) for k < c (zero for c <= k < 64), v = src[k * ld_k + r * ld_r]
template <class T>
__global__ void pack_rows_hilo_kernel(const T* __restrict__ src, int64_t rows, int c, int64_t ld_k,
                                      int64_t ld_r, __nv_bfloat16* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < rows * 64;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int k = static_cast<int>(e & 63);
    const int64_t r = e >> 6;
    float v = 0.f;
    if (k < c) v = static_cast<float>(src[k * ld_k + r * ld_r]);
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    out[r * 128 + k] = h;
    out[r * 128 + 64 + k] = __float2bfloat16_rn(v - __bfloat162float(h));
  }
}

// combined factor buffer Fc[r * n1p + i], r < N: hi rows 0..L-1, lo rows
// Lp..Lp+L-1, zeros elsewhere and for i >= n1.
__global__ void pack_factor_kernel(const __nv_bfloat16* __restrict__ hi,
                                   const __nv_bfloat16* __restrict__ lo, int64_t n1, int64_t n1p,
                                   int L, int Lp, int N, __nv_bfloat16* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n1p * N;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % n1p;
    const int r = static_cast<int>(e / n1p);
    __nv_bfloat16 v = __float2bfloat16_rn(0.f);
    if (i < n1) {
      if (r < L)
        v = hi[i + n1 * r];
      else if (lo && r >= Lp && r - Lp < L)
        v = lo[i + n1 * (r - Lp)];
    }
    out[e] = v;
  }
}

// ------------------------------------------------------------- host side ----
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    cudaGetLastError();
  });
  if (!fn) fail(KRP_ECUDA, "cuTensorMapEncodeTiled is unavailable");
  return fn;
}

CUtensorMap make_map(const void* base, int rank, const uint64_t* dims, const uint64_t* strides_bytes,
                     const uint32_t* box,
                     CUtensorMapDataType dtype = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16) {
  CUtensorMap m;
  uint32_t estr[3] = {1, 1, 1};
  const CUresult r = encode_fn()(&m, dtype, rank, const_cast<void*>(base),
                                 dims, strides_bytes, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                 CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) fail(KRP_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return m;
}

int round_up(int64_t v, int64_t m) { return static_cast<int>((v + m - 1) / m * m); }

template <class K>
void set_smem(K kernel, size_t bytes) {
  KRP_CUDA_CHECK(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      static_cast<int>(bytes)));
}

template <int N>
void launch_gemm_tn(const CUtensorMap& ma, const CUtensorMap* malo, const CUtensorMap& mb, int64_t S,
                    int kchunks, int L, int Lp, int has_lo, float* out, __nv_bfloat16* outb) {
  const int64_t tiles = (S + kBM - 1) / kBM;
  const int grid = static_cast<int>(std::min<int64_t>(tiles, current()->num_sms));
  if (!malo) {
    constexpr int NS = (N <= 64) ? 8 : (N <= 128 ? 6 : 4);
    const size_t smem = 1024 + NS * (size_t)(kBM * kBK * 2 + N * kBK * 2) + sizeof(Bars) + 64;
    set_smem(tc_gemm_tn_kernel<N, NS, false>, smem);
    tc_gemm_tn_kernel<N, NS, false><<<grid, kThreads, smem, stream()>>>(
        ma, ma, mb, S, kchunks, L, Lp, has_lo, out, outb, current()->d_status);
  } else {
    constexpr int NS = (N <= 64) ? 5 : (N <= 128 ? 4 : 3);
    const size_t smem = 1024 + NS * (size_t)(2 * kBM * kBK * 2 + N * kBK * 2) + sizeof(Bars) + 64;
    set_smem(tc_gemm_tn_kernel<N, NS, true>, smem);
    tc_gemm_tn_kernel<N, NS, true><<<grid, kThreads, smem, stream()>>>(
        ma, *malo, mb, S, kchunks, L, Lp, has_lo, out, outb, current()->d_status);
  }
  check_launch("tc_gemm_tn_bf16");
}

template <int N>
void launch_mttkrp(const CUtensorMap& mx, const CUtensorMap* mxlo, const CUtensorMap& mb, int64_t n1,
                   int64_t T, int kchunks, const float* w, int L, float* Y) {
  const int mblocks = static_cast<int>((n1 + kBM - 1) / kBM);
  const int sms = current()->num_sms;
  int64_t chunks = std::max<int64_t>(1, sms / mblocks);
  chunks = std::min<int64_t>(chunks, T);
  const int64_t per = (T + chunks - 1) / chunks;
  chunks = (T + per - 1) / per;
  const int grid = static_cast<int>(mblocks * chunks);
  if (!mxlo) {
    constexpr int NS = (N <= 64) ? 8 : 6;
    const size_t smem = 1024 + NS * (size_t)(2 * 64 * kBK * 2 + N * kBK * 2) + sizeof(Bars) + 64;
    set_smem(tc_mttkrp_kernel<N, NS, false>, smem);
    tc_mttkrp_kernel<N, NS, false><<<grid, kThreads, smem, stream()>>>(
        mx, mx, mb, n1, T, kchunks, mblocks, per, w, L, Y, current()->d_status);
  } else {
    constexpr int NS = (N <= 64) ? 5 : 4;
    const size_t smem = 1024 + NS * (size_t)(4 * 64 * kBK * 2 + N * kBK * 2) + sizeof(Bars) + 64;
    set_smem(tc_mttkrp_kernel<N, NS, true>, smem);
    tc_mttkrp_kernel<N, NS, true><<<grid, kThreads, smem, stream()>>>(
        mx, *mxlo, mb, n1, T, kchunks, mblocks, per, w, L, Y, current()->d_status);
  }
  check_launch("tc_mttkrp_bf16");
}

}  // namespace

bool tc_available() { return true; }

size_t tc_tree_workspace_bytes(int64_t n1, int64_t n2, int64_t T, int L) {
  const int64_t N = round_up(L, 16);
  const int64_t nseg = (n1 + 127) / 128;  // at most one segment per chunk
  return ws_bytes((size_t)nseg * ((n2 + 127) / 128) * T * N, 4) + (1 << 16);
}

size_t tc_workspace_bytes(int64_t n1, int64_t S, int L) {
  (void)S;
  const int64_t n1p = (n1 + 63) / 64 * 64;
  const int64_t Lp = (L + 15) / 16 * 16;
  const int64_t n1t = (n1 + 127) / 128 * 128;
  const int sms = std::max(1, current()->num_sms);
  return ws_bytes((size_t)n1p * 2 * Lp, 2) + ws_bytes((size_t)(n1p + 64) * Lp * 2, 2) +
         ws_bytes((size_t)sms * Lp * n1t, 4) + (1 << 16);  // + tree partials of Y1
}

void tc_gemm_tn_bf16(const __nv_bfloat16* X, int64_t n1, int64_t S, const __nv_bfloat16* Fhi,
                     const __nv_bfloat16* Flo, int L, float* out, const __nv_bfloat16* Xlo,
                     __nv_bfloat16* outb) {
  KRP_REQUIRE(n1 % 8 == 0, "BF16 tensor-core path needs n_1 %% 8 == 0 (n_1 = %lld)", (long long)n1);
  KRP_REQUIRE((reinterpret_cast<uintptr_t>(X) & 15) == 0, "X must be 16-byte aligned");
  KRP_REQUIRE(S < (int64_t(1) << 31), "too many rows for the TMA coordinates");
  const int Lp = round_up(L, 16);
  const int N = Flo ? 2 * Lp : Lp;
  KRP_REQUIRE(N <= 256, "sketch width too large for one MMA (L = %d)", L);
  const int64_t n1p = round_up(n1, 64);
  Ctx* c = current();
  __nv_bfloat16* Fc = c->ws.take<__nv_bfloat16>((size_t)n1p * N);
  const int64_t tot = n1p * N;
  pack_factor_kernel<<<(int)std::min<int64_t>((tot + 255) / 256, 4096), 256, 0, stream()>>>(
      Fhi, Flo, n1, n1p, L, Lp, N, Fc);
  check_launch("pack_factor");
  const uint64_t adims[2] = {(uint64_t)n1, (uint64_t)S};
  const uint64_t astr[1] = {(uint64_t)n1 * 2};
  const uint32_t abox[2] = {kBK, kBM};
  const CUtensorMap ma = make_map(X, 2, adims, astr, abox);
  CUtensorMap malo_v;
  const CUtensorMap* malo = nullptr;
  if (Xlo) {
    KRP_REQUIRE((reinterpret_cast<uintptr_t>(Xlo) & 15) == 0, "X lo plane must be 16-byte aligned");
    malo_v = make_map(Xlo, 2, adims, astr, abox);
    malo = &malo_v;
  }
  const uint64_t bdims[2] = {(uint64_t)n1p, (uint64_t)N};
  const uint64_t bstr[1] = {(uint64_t)n1p * 2};
  const uint32_t bbox[2] = {kBK, (uint32_t)N};
  const CUtensorMap mb = make_map(Fc, 2, bdims, bstr, bbox);
  const int kchunks = static_cast<int>((n1 + kBK - 1) / kBK);
  const int has_lo = Flo ? 1 : 0;
  switch (N) {
    case 16: launch_gemm_tn<16>(ma, malo, mb, S, kchunks, L, Lp, has_lo, out, outb); break;
    case 32: launch_gemm_tn<32>(ma, malo, mb, S, kchunks, L, Lp, has_lo, out, outb); break;
    case 48: launch_gemm_tn<48>(ma, malo, mb, S, kchunks, L, Lp, has_lo, out, outb); break;
    case 64: launch_gemm_tn<64>(ma, malo, mb, S, kchunks, L, Lp, has_lo, out, outb); break;
    case 96: launch_gemm_tn<96>(ma, malo, mb, S, kchunks, L, Lp, has_lo, out, outb); break;
    case 128: launch_gemm_tn<128>(ma, malo, mb, S, kchunks, L, Lp, has_lo, out, outb); break;
    case 160: launch_gemm_tn<160>(ma, malo, mb, S, kchunks, L, Lp, has_lo, out, outb); break;
    case 192: launch_gemm_tn<192>(ma, malo, mb, S, kchunks, L, Lp, has_lo, out, outb); break;
    case 224: launch_gemm_tn<224>(ma, malo, mb, S, kchunks, L, Lp, has_lo, out, outb); break;
    case 256: launch_gemm_tn<256>(ma, malo, mb, S, kchunks, L, Lp, has_lo, out, outb); break;
    default:
      if (N == 80) launch_gemm_tn<80>(ma, malo, mb, S, kchunks, L, Lp, has_lo, out, outb);
      else if (N == 112) launch_gemm_tn<112>(ma, malo, mb, S, kchunks, L, Lp, has_lo, out, outb);
      else if (N == 144) launch_gemm_tn<144>(ma, malo, mb, S, kchunks, L, Lp, has_lo, out, outb);
      else if (N == 176) launch_gemm_tn<176>(ma, malo, mb, S, kchunks, L, Lp, has_lo, out, outb);
      else if (N == 208) launch_gemm_tn<208>(ma, malo, mb, S, kchunks, L, Lp, has_lo, out, outb);
      else if (N == 240) launch_gemm_tn<240>(ma, malo, mb, S, kchunks, L, Lp, has_lo, out, outb);
      else fail(KRP_EUNSUPPORTED, "unsupported MMA width %d", N);
  }
}

namespace {
template <int N>
void launch_gemm_tf32(const CUtensorMap& ma, const CUtensorMap& mb, int64_t S, int kchunks, int L,
                      int Lp, float* out) {
  const int64_t tiles = (S + kBM - 1) / kBM;
  // SMs left to work on another stream (the FP64 QR beside the TTM)
  const int sms = std::max(1, current()->num_sms - current()->tc_reserve_sms);
  const int grid = static_cast<int>(std::min<int64_t>(tiles, sms));
  constexpr int NS = (N <= 96) ? 5 : 4;
  const size_t smem = 1024 + NS * (size_t)(2 * kBM * kBK32 * 4 + N * kBK32 * 4) + sizeof(BarsT) + 64;
  set_smem(tc_gemm_tn_tf32_kernel<N, NS>, smem);
  tc_gemm_tn_tf32_kernel<N, NS><<<grid, kTf32Threads, smem, stream()>>>(ma, mb, S, kchunks, L, Lp,
                                                                          out, current()->d_status);
  check_launch("tc_gemm_tn_tf32");
}
}  // namespace

bool tc_gemm_tn_tf32_supported(int64_t n1, int64_t S, int L, const void* X) {
  return n1 % 4 == 0 && n1 <= (int64_t(1) << 30) && S < (int64_t(1) << 31) && L >= 1 && L <= 64 &&
         (reinterpret_cast<uintptr_t>(X) & 15) == 0;
}

size_t tc_gemm_tn_tf32_workspace_bytes(int64_t n1, int L) {
  const int64_t n1p = (n1 + kBK32 - 1) / kBK32 * kBK32;
  const int64_t Lp = (L + 15) / 16 * 16;
  return ws_bytes((size_t)n1p * 2 * Lp, 4) + (1 << 12);
}

void tc_gemm_tn_tf32(const float* X, int64_t n1, int64_t S, const float* F, int64_t ldf, int L,
                     float* out) {
  KRP_REQUIRE(tc_gemm_tn_tf32_supported(n1, S, L, X), "TF32 TTM: unsupported shape or alignment");
  const int Lp = round_up(L, 16);
  const int N = 2 * Lp;
  const int64_t n1p = round_up(n1, kBK32);
  float* Fc = current()->ws.take<float>((size_t)n1p * N);
  const int64_t tot = n1p * N;
  pack_factor_tf32_kernel<<<(int)std::min<int64_t>((tot + 255) / 256, 4096), 256, 0, stream()>>>(
      F, ldf, n1, n1p, L, Lp, N, Fc);
  check_launch("pack_factor_tf32");
  const uint64_t adims[2] = {(uint64_t)n1, (uint64_t)S};
  const uint64_t astr[1] = {(uint64_t)n1 * 4};
  const uint32_t abox[2] = {kBK32, kBM};
  const CUtensorMap ma = make_map(X, 2, adims, astr, abox, CU_TENSOR_MAP_DATA_TYPE_FLOAT32);
  const uint64_t bdims[2] = {(uint64_t)n1p, (uint64_t)N};
  const uint64_t bstr[1] = {(uint64_t)n1p * 4};
  const uint32_t bbox[2] = {kBK32, (uint32_t)N};
  const CUtensorMap mb = make_map(Fc, 2, bdims, bstr, bbox, CU_TENSOR_MAP_DATA_TYPE_FLOAT32);
  const int kchunks = static_cast<int>((n1 + kBK32 - 1) / kBK32);
  switch (N) {
    case 32: launch_gemm_tf32<32>(ma, mb, S, kchunks, L, Lp, out); break;
    case 64: launch_gemm_tf32<64>(ma, mb, S, kchunks, L, Lp, out); break;
    case 96: launch_gemm_tf32<96>(ma, mb, S, kchunks, L, Lp, out); break;
    case 128: launch_gemm_tf32<128>(ma, mb, S, kchunks, L, Lp, out); break;
    default: fail(KRP_EUNSUPPORTED, "unsupported TF32 MMA width %d", N);
  }
}

namespace {
template <int N>
void launch_mttkrp_tf32(const CUtensorMap& mx, const CUtensorMap& mb, int64_t n1, int64_t T,
                        int kchunks, const float* wT, int L, float* Y) {
  const int mblocks = static_cast<int>((n1 + kBM - 1) / kBM);
  int64_t chunks = std::max<int64_t>(1, current()->num_sms / mblocks);
  chunks = std::min<int64_t>(chunks, T);
  const int64_t per = (T + chunks - 1) / chunks;
  chunks = (T + per - 1) / per;
  const int grid = static_cast<int>(mblocks * chunks);
  // 8 raw X tiles in flight (7 for the widest operand stages), one operand
  // stage per converter group
  constexpr int NR = (N <= 96) ? 8 : 7, NC = 2;
  const size_t smem = 1024 + NC * (size_t)(2 * kBM * kBK32 * 4 + N * kBK32 * 4) +
                      NR * (size_t)(4 * 32 * kBK32 * 4) + sizeof(BarsM) + 64;
  set_smem(tc_mttkrp_tf32_kernel<N, NR, NC>, smem);
  tc_mttkrp_tf32_kernel<N, NR, NC><<<grid, kMtThreads, smem, stream()>>>(
      mx, mb, n1, T, kchunks, mblocks, per, wT, L, Y, current()->d_status);
  check_launch("tc_mttkrp_tf32");
}
}  // namespace

bool tc_mttkrp_tf32_supported(int64_t n1, int64_t n2, int64_t T, int L, const void* X) {
  return n1 % 4 == 0 && n1 < (int64_t(1) << 31) && n2 < (int64_t(1) << 31) &&
         T < (int64_t(1) << 31) && L >= 1 && L <= 64 && (reinterpret_cast<uintptr_t>(X) & 15) == 0;
}

size_t tc_mttkrp_tf32_workspace_bytes(int64_t n2, int L) {
  const int64_t n2p = (n2 + kBK32 - 1) / kBK32 * kBK32;
  const int64_t Lp = (L + 15) / 16 * 16;
  return ws_bytes((size_t)n2p * 2 * Lp, 4) + (1 << 12);
}

void tc_mttkrp_first_tf32(const float* X, int64_t n1, int64_t n2, int64_t T, const float* Om2,
                          const float* wT, int L, float* Y) {
  KRP_REQUIRE(tc_mttkrp_tf32_supported(n1, n2, T, L, X), "TF32 MTTKRP: unsupported shape or alignment");
  const int Lp = round_up(L, 16);
  const int N = 2 * Lp;
  const int64_t n2p = round_up(n2, kBK32);
  float* Bc = current()->ws.take<float>((size_t)n2p * N);
  const int64_t tot = n2p * N;
  pack_factor_tf32_kernel<<<(int)std::min<int64_t>((tot + 255) / 256, 4096), 256, 0, stream()>>>(
      Om2, n2, n2, n2p, L, Lp, N, Bc);
  check_launch("pack_factor_tf32");
  const uint64_t xdims[3] = {(uint64_t)n1, (uint64_t)n2, (uint64_t)T};
  const uint64_t xstr[2] = {(uint64_t)n1 * 4, (uint64_t)n1 * n2 * 4};
  const uint32_t xbox[3] = {32, kBK32, 1};
  const CUtensorMap mx = make_map(X, 3, xdims, xstr, xbox, CU_TENSOR_MAP_DATA_TYPE_FLOAT32);
  const uint64_t bdims[2] = {(uint64_t)n2p, (uint64_t)N};
  const uint64_t bstr[1] = {(uint64_t)n2p * 4};
  const uint32_t bbox[2] = {kBK32, (uint32_t)N};
  const CUtensorMap mb = make_map(Bc, 2, bdims, bstr, bbox, CU_TENSOR_MAP_DATA_TYPE_FLOAT32);
  const int kchunks = static_cast<int>((n2 + kBK32 - 1) / kBK32);
  switch (N) {
    case 32: launch_mttkrp_tf32<32>(mx, mb, n1, T, kchunks, wT, L, Y); break;
    case 64: launch_mttkrp_tf32<64>(mx, mb, n1, T, kchunks, wT, L, Y); break;
    case 96: launch_mttkrp_tf32<96>(mx, mb, n1, T, kchunks, wT, L, Y); break;
    case 128: launch_mttkrp_tf32<128>(mx, mb, n1, T, kchunks, wT, L, Y); break;
    default: fail(KRP_EUNSUPPORTED, "unsupported TF32 MMA width %d", N);
  }
}

bool tc_tree_supported(int64_t n1, int L) {
  const int N = round_up(L, 16);
  return n1 % 8 == 0 && N <= 64;
}

namespace {
// dynamic shared memory of the tree kernel with NS stages and kseg resident
// Omega1 chunks (1 KB alignment slack, the barriers)
size_t tree_smem(int N, bool xlo, int kseg, int ns) {
  return 1024 + (size_t)2 * kseg * N * 128 + (size_t)ns * (xlo ? 4 : 2) * 16384 +
         (size_t)2 * 2 * (2 * N * 128) + sizeof(Bars) + 64;
}
constexpr size_t kTreeSmemMax = 232448 - 1024;  // 227 KB less the static shared arrays

template <int N, int NS, bool XLO>
void launch_tree(const CUtensorMap& mx, const CUtensorMap& mxlo, const CUtensorMap& mf,
                 const TreeArgs& P, int grid, size_t smem) {
  set_smem(tc_tree_kernel<N, NS, XLO>, smem);
  tc_tree_kernel<N, NS, XLO><<<grid, 320, smem, stream()>>>(mx, mxlo, mf, P, current()->d_status);
}

template <int N, bool XLO>
void launch_tree_ns(const CUtensorMap& mx, const CUtensorMap& mxlo, const CUtensorMap& mf,
                    const TreeArgs& P, int grid, int ns) {
  const size_t smem = tree_smem(N, XLO, P.kseg, ns);
  if (ns >= 4) launch_tree<N, 4, XLO>(mx, mxlo, mf, P, grid, smem);
  else if (ns == 3) launch_tree<N, 3, XLO>(mx, mxlo, mf, P, grid, smem);
  else launch_tree<N, 2, XLO>(mx, mxlo, mf, P, grid, smem);
}

template <int N>
void launch_tree_n(const CUtensorMap& mx, const CUtensorMap& mxlo, const CUtensorMap& mf,
                   const TreeArgs& P, int grid, bool xlo, int ns) {
  if (xlo) launch_tree_ns<N, true>(mx, mxlo, mf, P, grid, ns);
  else launch_tree_ns<N, false>(mx, mxlo, mf, P, grid, ns);
}
}  // namespace

void tc_tree_bf16(const __nv_bfloat16* X, int64_t n1, int64_t n2, int64_t T,
                  const __nv_bfloat16* Om1, const float* Om2, const float* w, int L,
                  float* Y1, float* Y2, float* C, const __nv_bfloat16* Xlo) {
  KRP_REQUIRE(tc_tree_supported(n1, L), "fused tree needs n_1 %% 8 == 0 and l <= 64");
  KRP_REQUIRE((reinterpret_cast<uintptr_t>(X) & 15) == 0, "X must be 16-byte aligned");
  KRP_REQUIRE(!Xlo || (reinterpret_cast<uintptr_t>(Xlo) & 15) == 0,
              "X lo plane must be 16-byte aligned");
  KRP_REQUIRE(T < (int64_t(1) << 31) && n2 < (int64_t(1) << 31), "tensor too large for TMA");
  const bool xlo = Xlo != nullptr;
  const int N = round_up(L, 16);
  const int64_t n1p = round_up(n1, 128);
  Ctx* ctx = current();
  TreeArgs P{};
  P.kch = static_cast<int>(n1p / 128);
  // the hi/lo form drains D2 every 16 items (chains of 128 MMA steps: Y1 to
  // ~5e-6, against ~3.5e-5 for one chain per CTA at 1024^3) from one buffer;
  // the BF16 form, whose input carries 2^-9 rounding, keeps one chain per CTA
  P.drain = xlo ? 16 : 0;
  P.nd2 = 1;
  // the segment as long as TMEM allows, shortened while the ring would hold
  // fewer than two stages
  P.kseg = std::min(P.kch, tree_kseg_max(N, P.nd2));
  auto stages = [&](int kseg) {
    int ns = 4;
    while (ns > 1 && tree_smem(N, xlo, kseg, ns) > kTreeSmemMax) --ns;
    return ns;
  };
  while (P.kseg > 1 && stages(P.kseg) < 2) --P.kseg;
  const int ns = stages(P.kseg);
  KRP_REQUIRE(ns >= 2, "fused tree: shared memory too small (l = %d)", L);
  const int nseg = (P.kch + P.kseg - 1) / P.kseg;
  __nv_bfloat16* Fc = ctx->ws.take<__nv_bfloat16>((size_t)n1p * N);
  pack_factor_kernel<<<(int)std::min<int64_t>((n1p * N + 255) / 256, 4096), 256, 0, stream()>>>(
      Om1, nullptr, n1, n1p, L, N, N, Fc);
  check_launch("pack_factor");
  KRP_CUDA_CHECK(cudaMemsetAsync(Y2, 0, sizeof(float) * n2 * L, stream()));
  const uint64_t xd[3] = {(uint64_t)n1, (uint64_t)n2, (uint64_t)T};
  const uint64_t xs[2] = {(uint64_t)n1 * 2, (uint64_t)n1 * n2 * 2};
  const uint32_t xbox[3] = {64, 128, 1};
  const CUtensorMap mx = make_map(X, 3, xd, xs, xbox);
  const CUtensorMap mxlo = xlo ? make_map(Xlo, 3, xd, xs, xbox) : mx;
  const uint64_t fd[2] = {(uint64_t)n1p, (uint64_t)N};
  const uint64_t fs[1] = {(uint64_t)n1p * 2};
  const uint32_t fbox[2] = {64, (uint32_t)N};
  const CUtensorMap mf = make_map(Fc, 2, fd, fs, fbox);
  P.w = w;
  P.om2 = Om2;
  P.Y2 = Y2;
  P.n2 = n2;
  P.T = T;
  P.L = L;
  const int64_t nb = (n2 + 127) / 128;
  P.nb = static_cast<int>(nb);
  P.items = nb * T;
  P.Cw = ctx->ws.take<float>((size_t)nseg * nb * T * N);
  P.cps = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(ctx->num_sms / nseg, P.items)));
  const int grid = nseg * P.cps;
  const int64_t segrows = static_cast<int64_t>(P.kseg) * 128;
  P.Yw = ctx->ws.take<float>((size_t)grid * N * segrows);
  switch (N) {
    case 16: launch_tree_n<16>(mx, mxlo, mf, P, grid, xlo, ns); break;
    case 32: launch_tree_n<32>(mx, mxlo, mf, P, grid, xlo, ns); break;
    case 48: launch_tree_n<48>(mx, mxlo, mf, P, grid, xlo, ns); break;
    case 64: launch_tree_n<64>(mx, mxlo, mf, P, grid, xlo, ns); break;
    default: fail(KRP_EUNSUPPORTED, "fused tree width %d", N);
  }
  check_launch("tc_tree_bf16");
  tree_reduce_kernel<<<(int)std::min<int64_t>((n1 * L + 255) / 256, 4096), 256, 0, stream()>>>(
      P.Yw, P.cps, segrows, n1, L, N, Y1);
  check_launch("tree_reduce");
  tree_c_reduce_kernel<<<(int)std::min<int64_t>(T, 65535), 256, 0, stream()>>>(
      P.Cw, (int64_t)nseg * nb, T, L, N, C);
  check_launch("tree_c_reduce");
}

size_t tc_residual_workspace_bytes(int64_t n1, int64_t S) {
  return ws_bytes((size_t)S * 128, 2) + ws_bytes((size_t)n1 * 128, 2) + (1 << 16);
}

bool tc_residual_supported(int64_t n1, int c) { return n1 % 8 == 0 && c >= 1 && c <= 64; }

template <bool XLO>
void launch_residual(const CUtensorMap& mx, const CUtensorMap& mxlo, const CUtensorMap& mq,
                     const __nv_bfloat16* Hp, int64_t n1, int64_t S, double* acc) {
  Ctx* ctx = current();
  const uint64_t hd[2] = {128, (uint64_t)S};
  const uint64_t hs[1] = {256};
  const uint32_t hbox[2] = {64, 128};
  const CUtensorMap mh = make_map(Hp, 2, hd, hs, hbox);
  const int mblocks = static_cast<int>((n1 + kBM - 1) / kBM);
  const int64_t sblocks = (S + 127) / 128;
  // CTAs per row block: fill the SMs, but no more than there are column tiles
  const int cpm = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(sblocks, ctx->num_sms / mblocks)));
  const int ns = XLO ? 2 : 3;
  const size_t stage = 2 * (size_t)128 * 128 + (XLO ? 4 : 2) * (size_t)64 * 128 * 2;
  const size_t smem = 1024 + ns * stage + 2 * (size_t)128 * 128 + sizeof(Bars) + 64;
  set_smem(tc_residual_kernel<XLO>, smem);
  const int grid = cpm * mblocks;
  tc_residual_kernel<XLO><<<grid, kThreads, smem, stream()>>>(mx, mxlo, mq, mh, n1, S, mblocks,
                                                              cpm, acc, ctx->d_status);
  check_launch("tc_residual_bf16");
}

void tc_residual_bf16(const __nv_bfloat16* X, int64_t n1, int64_t S, const double* Q1, int c,
                      const float* H, double* acc, const __nv_bfloat16* Xlo) {
  KRP_REQUIRE(tc_residual_supported(n1, c), "tensor-core residual needs n_1 %% 8 == 0 and c <= 64");
  KRP_REQUIRE((reinterpret_cast<uintptr_t>(X) & 15) == 0, "X must be 16-byte aligned");
  KRP_REQUIRE(!Xlo || (reinterpret_cast<uintptr_t>(Xlo) & 15) == 0, "X lo plane must be 16-byte aligned");
  KRP_REQUIRE(S < (int64_t(1) << 31) && n1 < (int64_t(1) << 31), "tensor too large for TMA");
  Ctx* ctx = current();
  __nv_bfloat16* Qp = ctx->ws.take<__nv_bfloat16>((size_t)n1 * 128);
  __nv_bfloat16* Hp = ctx->ws.take<__nv_bfloat16>((size_t)S * 128);
  pack_rows_hilo_kernel<double><<<(int)std::min<int64_t>((n1 * 64 + 255) / 256, 4096), 256, 0, stream()>>>(
      Q1, n1, c, n1, 1, Qp);
  check_launch("pack_rows_hilo");
  pack_rows_hilo_kernel<float><<<(int)std::min<int64_t>((S * 64 + 255) / 256, 8192), 256, 0, stream()>>>(
      H, S, c, 1, c, Hp);
  check_launch("pack_rows_hilo");
  const uint64_t xd[2] = {(uint64_t)n1, (uint64_t)S};
  const uint64_t xs[1] = {(uint64_t)n1 * 2};
  const uint64_t qd[2] = {128, (uint64_t)n1};
  const uint64_t qs[1] = {256};
  const uint32_t qbox[2] = {64, kBM};
  const CUtensorMap mq = make_map(Qp, 2, qd, qs, qbox);
  const uint32_t xbox[2] = {64, 128};
  const CUtensorMap mx = make_map(X, 2, xd, xs, xbox);
  if (!Xlo) {
    launch_residual<false>(mx, mx, mq, Hp, n1, S, acc);
  } else {
    const CUtensorMap mxlo = make_map(Xlo, 2, xd, xs, xbox);
    launch_residual<true>(mx, mxlo, mq, Hp, n1, S, acc);
  }
}

size_t tc_residual_tf32_workspace_bytes(int64_t n1, int64_t S) {
  return ws_bytes((size_t)S * 64, 4) + ws_bytes((size_t)n1 * 64, 4) + (1 << 16);
}

bool tc_residual_tf32_supported(int64_t n1, int64_t S, int c, const void* X) {
  return n1 % 4 == 0 && c >= 1 && c <= 32 && S < (int64_t(1) << 31) && n1 < (int64_t(1) << 31) &&
         (reinterpret_cast<uintptr_t>(X) & 15) == 0;
}

void tc_residual_tf32(const float* X, int64_t n1, int64_t S, const double* Q1, int c, const float* H,
                      double* acc) {
  KRP_REQUIRE(tc_residual_tf32_supported(n1, S, c, X), "TF32 residual: unsupported shape or alignment");
  Ctx* ctx = current();
  float* Qp = ctx->ws.take<float>((size_t)n1 * 64);
  float* Hp = ctx->ws.take<float>((size_t)S * 64);
  pack_rows_tf32_kernel<double><<<(int)std::min<int64_t>((n1 * 32 + 255) / 256, 4096), 256, 0, stream()>>>(
      Q1, n1, c, n1, 1, Qp);
  check_launch("pack_rows_tf32");
  pack_rows_tf32_kernel<float><<<(int)std::min<int64_t>((S * 32 + 255) / 256, 8192), 256, 0, stream()>>>(
      H, S, c, 1, c, Hp);
  check_launch("pack_rows_tf32");
  const uint64_t xd[2] = {(uint64_t)n1, (uint64_t)S};
  const uint64_t xs[1] = {(uint64_t)n1 * 4};
  const uint32_t xbox[2] = {32, 128};
  const CUtensorMap mx = make_map(X, 2, xd, xs, xbox, CU_TENSOR_MAP_DATA_TYPE_FLOAT32);
  const uint64_t qd[2] = {64, (uint64_t)n1};
  const uint64_t qs[1] = {256};
  const uint32_t qbox[2] = {32, kBM};
  const CUtensorMap mq = make_map(Qp, 2, qd, qs, qbox, CU_TENSOR_MAP_DATA_TYPE_FLOAT32);
  const uint64_t hd[2] = {64, (uint64_t)S};
  const uint64_t hs[1] = {256};
  const uint32_t hbox[2] = {32, 128};
  const CUtensorMap mh = make_map(Hp, 2, hd, hs, hbox, CU_TENSOR_MAP_DATA_TYPE_FLOAT32);
  const int mblocks = static_cast<int>((n1 + kBM - 1) / kBM);
  const int64_t sblocks = (S + 127) / 128;
  const int cpm = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(sblocks, ctx->num_sms / mblocks)));
  const size_t stage = 2 * (size_t)128 * 32 * 4 + 4 * (size_t)32 * 128 * 4;
  const size_t smem = 1024 + 2 * stage + 2 * (size_t)128 * 32 * 4 + sizeof(Bars) + 64;
  set_smem(tc_residual_tf32_kernel, smem);
  tc_residual_tf32_kernel<<<cpm * mblocks, kThreads, smem, stream()>>>(mx, mq, mh, n1, S, mblocks, cpm,
                                                                       acc, ctx->d_status);
  check_launch("tc_residual_tf32");
}

void tc_mttkrp_first_bf16(const __nv_bfloat16* X, int64_t n1, int64_t n2, int64_t T,
                          const __nv_bfloat16* Om2, const float* w, int L, float* Y,
                          const __nv_bfloat16* Xlo) {
  KRP_REQUIRE(n1 % 8 == 0, "BF16 tensor-core path needs n_1 %% 8 == 0 (n_1 = %lld)", (long long)n1);
  KRP_REQUIRE((reinterpret_cast<uintptr_t>(X) & 15) == 0, "X must be 16-byte aligned");
  KRP_REQUIRE(T < (int64_t(1) << 31) && n2 < (int64_t(1) << 31), "tensor too large for TMA");
  const int Lp = round_up(L, 16);
  KRP_REQUIRE(Lp <= 128, "sketch width too large (L = %d)", L);
  const int64_t n2p = round_up(n2, 64);
  Ctx* c = current();
  __nv_bfloat16* Bc = c->ws.take<__nv_bfloat16>((size_t)n2p * Lp);
  const int64_t tot = n2p * Lp;
  pack_factor_kernel<<<(int)std::min<int64_t>((tot + 255) / 256, 4096), 256, 0, stream()>>>(
      Om2, nullptr, n2, n2p, L, Lp, Lp, Bc);
  check_launch("pack_factor");
  KRP_CUDA_CHECK(cudaMemsetAsync(Y, 0, sizeof(float) * n1 * L, stream()));
  const uint64_t xdims[3] = {(uint64_t)n1, (uint64_t)n2, (uint64_t)T};
  const uint64_t xstr[2] = {(uint64_t)n1 * 2, (uint64_t)n1 * n2 * 2};
  const uint32_t xbox[3] = {64, kBK, 1};
  const CUtensorMap mx = make_map(X, 3, xdims, xstr, xbox);
  CUtensorMap mxlo_v;
  const CUtensorMap* mxlo = nullptr;
  if (Xlo) {
    KRP_REQUIRE((reinterpret_cast<uintptr_t>(Xlo) & 15) == 0, "X lo plane must be 16-byte aligned");
    mxlo_v = make_map(Xlo, 3, xdims, xstr, xbox);
    mxlo = &mxlo_v;
  }
  const uint64_t bdims[2] = {(uint64_t)n2p, (uint64_t)Lp};
  const uint64_t bstr[1] = {(uint64_t)n2p * 2};
  const uint32_t bbox[2] = {kBK, (uint32_t)Lp};
  const CUtensorMap mb = make_map(Bc, 2, bdims, bstr, bbox);
  const int kchunks = static_cast<int>((n2 + kBK - 1) / kBK);
  switch (Lp) {
    case 16: launch_mttkrp<16>(mx, mxlo, mb, n1, T, kchunks, w, L, Y); break;
    case 32: launch_mttkrp<32>(mx, mxlo, mb, n1, T, kchunks, w, L, Y); break;
    case 48: launch_mttkrp<48>(mx, mxlo, mb, n1, T, kchunks, w, L, Y); break;
    case 64: launch_mttkrp<64>(mx, mxlo, mb, n1, T, kchunks, w, L, Y); break;
    case 80: launch_mttkrp<80>(mx, mxlo, mb, n1, T, kchunks, w, L, Y); break;
    case 96: launch_mttkrp<96>(mx, mxlo, mb, n1, T, kchunks, w, L, Y); break;
    case 112: launch_mttkrp<112>(mx, mxlo, mb, n1, T, kchunks, w, L, Y); break;
    case 128: launch_mttkrp<128>(mx, mxlo, mb, n1, T, kchunks, w, L, Y); break;
    default: fail(KRP_EUNSUPPORTED, "unsupported sketch width %d", L);
  }
}

}  // namespace krp
