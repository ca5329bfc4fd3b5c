// a9: column / row sketches of a block Hankel matrix without forming it or the
// Khatri-Rao product, by the identity of Eq. (4.1):
//   M (Omega1 kr Omega2) = sum_k (E_k Omega1) kr (H_k Omega2).
// With Z_k = H_k Omega2 (m x l), block row i of the sketch is a correlation
// along the block index:  Y[(i,a), c] = sum_j Omega1[j, c] Z_{i+j}[a, c]
// (0-based, block (i, j) of M is H_{i+j}).  The row sketch M^T (Psi1 kr Psi2)
// is the same with H_k^T.  The two-level form (Sec. 4.3: block Hankel
// matrices whose blocks are block Hankel) correlates along both block indices,
// with a three-factor Khatri-Rao sketch.
#include "common.cuh"

namespace krp {
namespace {

template <class T>
__device__ __forceinline__ float ld(const T* p, int64_t i);
template <>
__device__ __forceinline__ float ld<float>(const float* p, int64_t i) { return p[i]; }
template <>
__device__ __forceinline__ float ld<__nv_bfloat16>(const __nv_bfloat16* p, int64_t i) {
  return __bfloat162float(p[i]);
}

// Zs[a + mo*(c + ell*k)] = sum_b H_k[a,b] F2[b,c]  (or H_k^T when transpose)
template <class T>
__global__ void blockmul_kernel(const T* __restrict__ blocks, int m, int n, int nb,
                                const T* __restrict__ F2, int ell, int transpose,
                                float* __restrict__ Zs) {
  const int mo = transpose ? n : m;
  const int ki = transpose ? m : n;
  const int64_t total = (int64_t)mo * ell * nb;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(e % mo);
    const int c = (int)((e / mo) % ell);
    const int k = (int)(e / ((int64_t)mo * ell));
    const T* H = blocks + (int64_t)m * n * k;
    float acc = 0.f;
    for (int b = 0; b < ki; ++b) {
      const float h = transpose ? ld(H, b + (int64_t)m * a) : ld(H, a + (int64_t)m * b);
      acc = fmaf(h, ld(F2, b + (int64_t)ki * c), acc);
    }
    Zs[e] = acc;
  }
}

// Y[(a + mo*i) + mo*s*c] = sum_{j<s} F1[j + s*c] Zs[a + mo*(c + ell*(i+j))]
template <class T>
__global__ void corr_kernel(const float* __restrict__ Zs, int mo, int s, int ell,
                            const T* __restrict__ F1, float* __restrict__ Y) {
  const int64_t total = (int64_t)mo * s * ell;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(e % mo);
    const int i = (int)((e / mo) % s);
    const int c = (int)(e / ((int64_t)mo * s));
    float acc = 0.f;
    const float* z = Zs + a + (int64_t)mo * c;
    const int64_t zstride = (int64_t)mo * ell;
    for (int j = 0; j < s; ++j) acc = fmaf(ld(F1, j + (int64_t)s * c), z[zstride * (i + j)], acc);
    Y[e] = acc;
  }
}

// Two levels (Sec. 4.3): block (k1, k2) of Zs is H_{k1,k2} F3 (index
// k1 + nb1 k2, from blockmul over all nb1 nb2 blocks), and
// Y[(a + mo (i2 + s2 i1)) + mo s1 s2 c] =
//   sum_{j1 < s1, j2 < s2} F1[j1 + s1 c] F2[j2 + s2 c] Zs[a + mo (c + ell ((i1+j1) + nb1 (i2+j2)))]
template <class T>
__global__ void corr2_kernel(const float* __restrict__ Zs, int mo, int s1, int s2, int ell,
                             const T* __restrict__ F1, const T* __restrict__ F2,
                             float* __restrict__ Y) {
  const int nb1 = 2 * s1 - 1;
  const int64_t total = (int64_t)mo * s1 * s2 * ell;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(e % mo);
    const int64_t rb = (e / mo) % ((int64_t)s1 * s2);
    const int i2 = (int)(rb % s2), i1 = (int)(rb / s2);
    const int c = (int)(e / ((int64_t)mo * s1 * s2));
    const float* z = Zs + a + (int64_t)mo * c;
    const int64_t zstride = (int64_t)mo * ell;
    float acc = 0.f;
    for (int j2 = 0; j2 < s2; ++j2) {
      const float* zr = z + zstride * (int64_t)nb1 * (i2 + j2);
      float part = 0.f;
      for (int j1 = 0; j1 < s1; ++j1) part = fmaf(ld(F1, j1 + (int64_t)s1 * c), zr[zstride * (i1 + j1)], part);
      acc = fmaf(ld(F2, j2 + (int64_t)s2 * c), part, acc);
    }
    Y[e] = acc;
  }
}

int grid_for(int64_t n) {
  int64_t g = (n + 255) / 256;
  return (int)(g < 1 ? 1 : (g > 8192 ? 8192 : g));
}

}  // namespace

void hankel_sketch(const void* blocks, krp_dtype bt, int m, int n, int s, const void* f1,
                   const void* f2, int ell, bool transpose, float* Y, float* Zs) {
  const int nb = 2 * s - 1;
  const int mo = transpose ? n : m;
  const int64_t zt = (int64_t)mo * ell * nb;
  const int64_t yt = (int64_t)mo * s * ell;
  if (bt == KRP_F32) {
    blockmul_kernel<float><<<grid_for(zt), 256, 0, stream()>>>(
        static_cast<const float*>(blocks), m, n, nb, static_cast<const float*>(f2), ell,
        transpose ? 1 : 0, Zs);
    check_launch("hankel_blockmul");
    corr_kernel<float><<<grid_for(yt), 256, 0, stream()>>>(Zs, mo, s, ell,
                                                           static_cast<const float*>(f1), Y);
    check_launch("hankel_corr");
  } else {
    blockmul_kernel<__nv_bfloat16><<<grid_for(zt), 256, 0, stream()>>>(
        static_cast<const __nv_bfloat16*>(blocks), m, n, nb,
        static_cast<const __nv_bfloat16*>(f2), ell, transpose ? 1 : 0, Zs);
    check_launch("hankel_blockmul");
    corr_kernel<__nv_bfloat16><<<grid_for(yt), 256, 0, stream()>>>(
        Zs, mo, s, ell, static_cast<const __nv_bfloat16*>(f1), Y);
    check_launch("hankel_corr");
  }
}


void hankel2_sketch(const void* blocks, krp_dtype bt, int m, int n, int s1, int s2, const void* f1,
                    const void* f2, const void* f3, int ell, bool transpose, float* Y, float* Zs) {
  const int nb = (2 * s1 - 1) * (2 * s2 - 1);
  const int mo = transpose ? n : m;
  const int64_t zt = (int64_t)mo * ell * nb;
  const int64_t yt = (int64_t)mo * s1 * s2 * ell;
  if (bt == KRP_F32) {
    blockmul_kernel<float><<<grid_for(zt), 256, 0, stream()>>>(
        static_cast<const float*>(blocks), m, n, nb, static_cast<const float*>(f3), ell,
        transpose ? 1 : 0, Zs);
    check_launch("hankel2_blockmul");
    corr2_kernel<float><<<grid_for(yt), 256, 0, stream()>>>(
        Zs, mo, s1, s2, ell, static_cast<const float*>(f1), static_cast<const float*>(f2), Y);
    check_launch("hankel2_corr");
  } else {
    blockmul_kernel<__nv_bfloat16><<<grid_for(zt), 256, 0, stream()>>>(
        static_cast<const __nv_bfloat16*>(blocks), m, n, nb,
        static_cast<const __nv_bfloat16*>(f3), ell, transpose ? 1 : 0, Zs);
    check_launch("hankel2_blockmul");
    corr2_kernel<__nv_bfloat16><<<grid_for(yt), 256, 0, stream()>>>(
        Zs, mo, s1, s2, ell, static_cast<const __nv_bfloat16*>(f1),
        static_cast<const __nv_bfloat16*>(f2), Y);
    check_launch("hankel2_corr");
  }
}

}  // namespace krp
