// a1: on-device Gaussian sketching factors from Philox4x32-10 + Box-Muller.
//
// Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, SC'11):
//   round: (c0,c1,c2,c3) -> (hi(M1 c2)^c1^k0, lo(M1 c2), hi(M0 c0)^c3^k1, lo(M0 c0))
//   key bump between rounds: k0 += W0, k1 += W1.
// Counter of factor entry e = i + rows*k of factor j: (e>>2, j, draw, tag);
// key = (seed lo32, seed hi32).  Box-Muller in FP64 (Def. of KRP, Sec. 2.5
// only asks for i.i.d. mean-zero unit-variance sub-Gaussian entries).
#include "common.cuh"

namespace krp {
namespace {

constexpr uint32_t kM0 = 0xD2511F53u;
constexpr uint32_t kM1 = 0xCD9E8D57u;
constexpr uint32_t kW0 = 0x9E3779B9u;
constexpr uint32_t kW1 = 0xBB67AE85u;

__device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += kW0;
      k1 += kW1;
    }
    const uint32_t hi0 = __umulhi(kM0, c.x), lo0 = kM0 * c.x;
    const uint32_t hi1 = __umulhi(kM1, c.z), lo1 = kM1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

__device__ __forceinline__ double uopen(uint32_t w) {
  return (static_cast<double>(w) + 0.5) * 0x1p-32;
}

struct GenParams {
  FactorJob jobs[KRP_MAXD + 4];
  int64_t start[KRP_MAXD + 5];  // prefix sums of blocks
  int njobs;
  int ell;
  uint32_t k0, k1, draw, tag;
  int type;
};

template <class T>
__device__ __forceinline__ void store_val(void* p, int64_t e, double z);
template <>
__device__ __forceinline__ void store_val<float>(void* p, int64_t e, double z) {
  static_cast<float*>(p)[e] = static_cast<float>(z);
}
template <>
__device__ __forceinline__ void store_val<__nv_bfloat16>(void* p, int64_t e, double z) {
  static_cast<__nv_bfloat16*>(p)[e] = __float2bfloat16_rn(static_cast<float>(z));
}
template <>
__device__ __forceinline__ void store_val<double>(void* p, int64_t e, double z) {
  static_cast<double*>(p)[e] = z;
}

template <class T>
__global__ void gen_factors_kernel(const GenParams P) {
  const int64_t total = P.start[P.njobs];
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total;
       g += (int64_t)gridDim.x * blockDim.x) {
    int j = 0;
    while (j + 1 < P.njobs && g >= P.start[j + 1]) ++j;
    const FactorJob& job = P.jobs[j];
    const int64_t b = g - P.start[j];
    const uint4 w = philox10(
        make_uint4(static_cast<uint32_t>(b), job.factor, P.draw, P.tag), P.k0, P.k1);
    const int64_t n = job.rows * P.ell;
    const double ra = sqrt(-2.0 * log(uopen(w.x)));
    const double rb = sqrt(-2.0 * log(uopen(w.z)));
    double sa, ca, sb, cb;
    sincospi(2.0 * uopen(w.y), &sa, &ca);
    sincospi(2.0 * uopen(w.w), &sb, &cb);
    const double z[4] = {ra * ca, ra * sa, rb * cb, rb * sb};
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const int64_t e = 4 * b + l;
      if (e < n) store_val<T>(job.ptr, e, z[l]);
    }
  }
}

// Many factors with their own keys: job j covers blocks [start[j], start[j+1])
// of the flattened launch; values are stored as FP32 (bf16_round: rounded to
// BF16 first, the values a BF16 factor would hold).
__global__ void gen_factors_batch_kernel(const BatchFactorJob* __restrict__ jobs,
                                         const int64_t* __restrict__ start, int njobs) {
  const int64_t total = start[njobs];
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total;
       g += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = njobs - 1;  // last job with start <= g
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (start[mid] <= g) lo = mid; else hi = mid - 1;
    }
    const BatchFactorJob& job = jobs[lo];
    const int64_t b = g - start[lo];
    const uint4 w = philox10(make_uint4(static_cast<uint32_t>(b), job.factor, job.draw, job.tag),
                             static_cast<uint32_t>(job.seed & 0xFFFFFFFFu),
                             static_cast<uint32_t>(job.seed >> 32));
    const int64_t n = job.rows * job.ell;
    const double ra = sqrt(-2.0 * log(uopen(w.x)));
    const double rb = sqrt(-2.0 * log(uopen(w.z)));
    double sa, ca, sb, cb;
    sincospi(2.0 * uopen(w.y), &sa, &ca);
    sincospi(2.0 * uopen(w.w), &sb, &cb);
    const double z[4] = {ra * ca, ra * sa, rb * cb, rb * sb};
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const int64_t e = 4 * b + l;
      if (e < n) {
        float v = static_cast<float>(z[l]);
        if (job.bf16_round) v = __bfloat162float(__float2bfloat16_rn(v));
        job.ptr[e] = v;
      }
    }
  }
}

__global__ void philox_words_kernel(uint32_t k0, uint32_t k1, uint32_t c1, uint32_t c2,
                                    uint32_t c3, uint64_t first, int64_t n, uint32_t* out) {
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < n;
       b += (int64_t)gridDim.x * blockDim.x) {
    const uint4 w = philox10(make_uint4(static_cast<uint32_t>(first + b), c1, c2, c3), k0, k1);
    reinterpret_cast<uint4*>(out)[b] = w;
  }
}

}  // namespace

void launch_gen_factors(uint64_t seed, uint32_t draw, uint32_t tag, int ell, krp_dtype type,
                        const FactorJob* jobs, int njobs) {
  if (njobs == 0) return;
  GenParams P{};
  KRP_REQUIRE(njobs <= KRP_MAXD + 4, "too many factors in one draw (%d)", njobs);
  P.njobs = njobs;
  P.ell = ell;
  P.k0 = static_cast<uint32_t>(seed & 0xFFFFFFFFu);
  P.k1 = static_cast<uint32_t>(seed >> 32);
  P.draw = draw;
  P.tag = tag;
  P.start[0] = 0;
  for (int j = 0; j < njobs; ++j) {
    P.jobs[j] = jobs[j];
    P.start[j + 1] = P.start[j] + jobs[j].blocks;
    KRP_REQUIRE(jobs[j].blocks <= (int64_t(1) << 32), "factor too large for a 32-bit counter");
  }
  const int64_t total = P.start[njobs];
  const int threads = 256;
  const int64_t want = (total + threads - 1) / threads;
  const int grid = static_cast<int>(want < 4096 ? want : 4096);
  switch (type) {
    case KRP_F32: gen_factors_kernel<float><<<grid, threads, 0, stream()>>>(P); break;
    case KRP_BF16: gen_factors_kernel<__nv_bfloat16><<<grid, threads, 0, stream()>>>(P); break;
    case KRP_F64: gen_factors_kernel<double><<<grid, threads, 0, stream()>>>(P); break;
    default: fail(KRP_EINVAL, "unsupported factor dtype %d", (int)type);
  }
  check_launch("gen_factors");
}

void launch_gen_factors_batch(const BatchFactorJob* d_jobs, const int64_t* d_start, int njobs,
                              int64_t total_blocks) {
  if (njobs <= 0 || total_blocks <= 0) return;
  const int threads = 256;
  const int64_t want = (total_blocks + threads - 1) / threads;
  const int grid = static_cast<int>(want < 4096 ? want : 4096);
  gen_factors_batch_kernel<<<grid, threads, 0, stream()>>>(d_jobs, d_start, njobs);
  check_launch("gen_factors_batch");
}

void launch_philox_words(uint64_t seed, uint32_t c1, uint32_t c2, uint32_t c3, uint64_t first,
                         int64_t n, uint32_t* out) {
  if (n <= 0) return;
  const int threads = 256;
  const int64_t want = (n + threads - 1) / threads;
  const int grid = static_cast<int>(want < 4096 ? want : 4096);
  philox_words_kernel<<<grid, threads, 0, stream()>>>(static_cast<uint32_t>(seed & 0xFFFFFFFFu),
                                                      static_cast<uint32_t>(seed >> 32), c1, c2,
                                                      c3, first, n, out);
  check_launch("philox_words");
}

}  // namespace krp
