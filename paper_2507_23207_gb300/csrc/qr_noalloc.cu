// krp_qr_noalloc: the FP64 thin QR of one FP32 sketch without any device
// allocation.
//
// Who needs this: callers that are not allowed to call cudaMalloc once they
// are running -- code that lives inside a framework whose caching allocator
// owns all device memory (a raw cudaMalloc would bypass its accounting and can
// fail or fragment the pool), latency-critical loops in which the implicit
// device synchronisation of cudaMalloc/cudaFree is unacceptable, and programs
// that reserve their whole device memory budget up front.  krp_qr grows the
// context's workspace with cudaMalloc when it is too small; this entry point
// instead uses one fixed scratch array that lives in the library image.
//
// The scratch is a file-scope __device__ array (KRP_QR_NOALLOC_MAX_DOUBLES
// doubles, 4 MiB), present on every GPU that loads the library until the
// process exits.  Its host-side name is only a stand-in, so every call looks
// the device address up with cudaGetSymbolAddress on the current device (no
// cached pointer that a device reset or a new primary context could make
// stale; the lookup costs microseconds).
#include "common.cuh"

namespace krp {
cudaError_t cholqr3_single_on_stream(const float* Y, int64_t m, int l, double* Q, double* R,
                                     double* scratch, cudaStream_t st);
}

namespace {

__device__ __align__(256) double g_qr_noalloc_scratch[KRP_QR_NOALLOC_MAX_DOUBLES];

// Device address of the scratch array in the current device's context.
cudaError_t scratch_on_current_device(double** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_qr_noalloc_scratch);
  if (e != cudaSuccess) return e;
  *out = static_cast<double*>(p);
  return cudaSuccess;
}

}  // namespace

extern "C" krp_status krp_qr_noalloc(const float* Y, int64_t m, int l, double* Q, double* R,
                                     void* cuda_stream) {
  if (!Y || !Q) return KRP_EINVAL;
  if (l < 1 || l > 64 || m < l) return KRP_EINVAL;
  // working matrix + Gram + three pass factors + refill mask + status word
  const int64_t need = m * l + 4 * (int64_t)l * l + 2;
  if (m > (int64_t(1) << 40) || need > KRP_QR_NOALLOC_MAX_DOUBLES) return KRP_EINVAL;
  double* scratch = nullptr;
  if (scratch_on_current_device(&scratch) != cudaSuccess) {
    cudaGetLastError();
    return KRP_ECUDA;
  }
  const cudaError_t e = krp::cholqr3_single_on_stream(Y, m, l, Q, R, scratch,
                                                      static_cast<cudaStream_t>(cuda_stream));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return KRP_ECUDA;
  }
  return KRP_OK;
}
