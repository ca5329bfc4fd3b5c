// BF16 tensor-core (tcgen05) kernels: placeholder until the sm_103a kernels land.
#include "pipeline.h"

namespace krp {

bool tc_available() { return false; }

size_t tc_workspace_bytes(int64_t, int64_t, int) { return 0; }

void tc_gemm_tn_bf16(const __nv_bfloat16*, int64_t, int64_t, const __nv_bfloat16*,
                     const __nv_bfloat16*, int, float*) {
  fail(KRP_EUNSUPPORTED, "BF16 tensor-core contraction not built yet");
}

void tc_mttkrp_first_bf16(const __nv_bfloat16*, int64_t, int64_t, int64_t, const __nv_bfloat16*,
                          const float*, int, float*) {
  fail(KRP_EUNSUPPORTED, "BF16 tensor-core MTTKRP not built yet");
}

}  // namespace krp
