// Internal: pipelines built from the kernels (not part of the C ABI).
#pragma once

#include <functional>

#include "common.cuh"

namespace krp {

bool is_device_ptr(const void* p);
size_t dtype_size(krp_dtype t);
int64_t checked_numel(int d, const int64_t* dims);
// Synchronise the stream, read and clear the device status word; fail on error.
void raise_device_status(Ctx* c);

struct SketchArgs {
  const void* X;
  krp_dtype xt;
  int d;
  int64_t dims[KRP_MAXD];
  const void* omega[KRP_MAXD];
  krp_dtype omt;
  int ell;
  int64_t N;
};
SketchArgs validate_sketch(const void* X, krp_dtype xt, int d, const int64_t* dims,
                           const void* const* omega, krp_dtype omt, int ell);
size_t sketch_workspace_bytes(const SketchArgs& a, bool all_modes, int tree_split = -1);
void sketch_one_mode(const SketchArgs& a, int n, float* Y);
// tree_split: the dimension tree of the tensor-core forms contracts mode 1
// and the merged modes 2..tree_split+1 in one pass (1 <= tree_split <= d-1);
// -1 picks it by timing each candidate on the first call for a shape
// (cached in the context).  The FP32 form ignores it.
// after_first: called (if set) once Y[0] is enqueued and before the rest of
// the FP32 form's tree, so that work on Y[0] can start beside it
void sketch_all_modes(const SketchArgs& a, float* const* Y, int tree_split = -1,
                      const std::function<void()>& after_first = {});

size_t multi_ttm_workspace_bytes(int d, const int64_t* dims, const int* cols, krp_dtype xt);
// q0_ready / qrest_ready (optional): events after which Q[0] / Q[1..d-1]
// are written (by work on another stream); the context's stream waits on
// each before it first reads that factor
void multi_ttm(const void* X, krp_dtype xt, int d, const int64_t* dims, const double* const* Q,
               const int* cols, float* G, cudaEvent_t q0_ready = nullptr,
               cudaEvent_t qrest_ready = nullptr);

size_t core_truncate_workspace_bytes(int d, const int* ell, const int* ranks);
void core_truncate(int d, const int64_t* dims, const int* ell, const int* ranks, const float* G,
                   const double* const* Q, float* Gout, double* const* Qout);
size_t residual_workspace_bytes(int d, const int64_t* dims, const int64_t* cdim, krp_dtype xt);
void residual_sums(const void* Xd, krp_dtype xt, int d, const int64_t* dims, const float* Gc,
                   const int64_t* cdim, const double* const* Q, double* acc);

void tucker_pipeline(bool sequential, const void* X, krp_dtype xt, int d, const int64_t* dims,
                     const int64_t* ld, const int* ranks, int oversample, uint64_t seed,
                     unsigned flags, krp_tucker_out* out);

// Padded tensors (ld: per-mode leading sizes, ld[j] >= dims[j]; element
// (i_1..i_d) at sum_j i_j prod_{m<j} ld[m]): padded() checks ld and tells
// whether it differs from dims; dense_copy() packs a padded device X (both
// planes of a BF16 hi/lo pair, the lo plane prod(ld) elements after the hi
// plane) into a dense workspace copy and returns it, or returns X itself.
bool padded(int d, const int64_t* dims, const int64_t* ld);
int64_t padded_numel(int d, const int64_t* ld);
size_t dense_copy_bytes(int d, const int64_t* dims, const int64_t* ld, krp_dtype xt);
const void* dense_copy(const void* X, krp_dtype xt, int d, const int64_t* dims, const int64_t* ld);

void tucker_batched(krp_dtype xt, int count, krp_tucker_item* items, int oversample,
                    unsigned flags);
int tucker_batched_plan_info(int* slabs_per_unit, int* units, int* grid);
void hankel_batched(krp_dtype bt, int count, krp_hankel_item* items);

void hankel_pipeline(const void* blocks, krp_dtype bt, int m, int n, int s, int r, int ell_r,
                     int ell_l, uint64_t seed, double* U, double* S, double* V);
// Alg. 6 on a two-level block Hankel matrix (Sec. 4.3; blocks (k1, k2) at
// k1 + (2 s1 - 1) k2, each m x n column-major).
void hankel2_pipeline(const void* blocks, krp_dtype bt, int m, int n, int s1, int s2, int r,
                      int ell_r, int ell_l, uint64_t seed, double* U, double* S, double* V);
// Nystrom approximation of an SPSD block Hankel matrix (square m x m blocks):
// its top r eigenpairs, U (m s x r) and L (r), FP64 (device or host).
void hankel_nystrom(const void* blocks, krp_dtype bt, int m, int s, int r, int ell, double rcond,
                    uint64_t seed, double* U, double* L);
// Recompression of the Hadamard product of two Tucker tensors (hadamard.cu):
// RHOSVD-KRP-MEMO of (G x {U_j}) * (H x {V_j}) without forming it, FP64.
size_t hadamard_workspace_bytes(int d, const int64_t* dims, const int* rg, const int* rh, int ell);
void hadamard_rhosvd(int d, const int64_t* dims, const int* rg, const double* G,
                     const double* const* U, const int* rh, const double* H,
                     const double* const* V, int ell, uint64_t seed, double* core,
                     double* const* factors, double* rel_error);
// Sensor placement (sensor.cu, Sec. 6): pivoted-QR indices and interpolation
// factors of d orthonormal factors Q_i (N_i x l_i, FP64, device), and the
// reconstruction T_hat x {A_i} of measurements on the sensor grid.
size_t sensor_select_workspace_bytes(int d, const int64_t* dims, const int* ells);
void sensor_select(int d, const int64_t* dims, const int* ells, const double* const* Q,
                   int* const* idx, double* const* A);
size_t sensor_reconstruct_workspace_bytes(int d, const int64_t* dims, const int* ells);
void sensor_reconstruct(int d, const int64_t* dims, const int* ells, const double* const* A,
                        const float* That, float* out);
// Eigensystem realization (era.cu): A (r x r, nullable) and its eigenvalues
// (wr, wi) from the blocks and the rank-r factors U (m s x r), S, V (n s x r),
// all device memory, FP64; r <= 64.
void era_realize(const void* blocks, krp_dtype bt, int m, int n, int s, int r, const double* U,
                 const double* S, const double* V, double* A, double* wr, double* wi);
size_t era_workspace_bytes(int m, int s, int r);
void hankel_sketch_only(const void* blocks, krp_dtype bt, int m, int n, int s,
                        const void* omega1, const void* omega2, int ell_r, const void* psi1,
                        const void* psi2, int ell_l, float* Y, float* Z);

// Contractions over the big tensor, dispatched on its element type:
// FP32 -> tcgen05 as three TF32 products where the shape allows (else FP32
// CUDA-core kernels), BF16 -> tcgen05 tensor-core kernels.
//   out[s + S*k] = sum_{i < n1} X[i + n1*s] F[i + n1*k],  S = N / n1
// F is given in FP32 (Ff) and, for BF16 X, as a bf16 hi/lo pair (Fhi, Flo;
// Flo may be null).
void big_gemm_tn(const void* X, krp_dtype xt, int64_t n1, int64_t S, const float* Ff,
                 const __nv_bfloat16* Fhi, const __nv_bfloat16* Flo, int L, float* out);
//   Y[i + n1*k] = sum_s X[i + n1*s] prod_j V_j[digit_j(s), k] over the modes
//   2..d (rest), with V_j FP32 (F32 X) or BF16 (BF16 X).
void big_mttkrp_first(const void* X, krp_dtype xt, int64_t n1, int d_rest,
                      const int64_t* rest_dims, const void* const* rest_V, int L, float* Y);

// tcgen05 kernels (tc_kernels.cu)
// Xlo (optional): lo plane of X given as a BF16 hi/lo pair (X ~ X + Xlo)
// outb (optional): the result as a BF16 hi/lo pair instead of FP32 (hi plane
// of S*L values at outb, lo plane at outb + S*L; `out` is not written)
void tc_gemm_tn_bf16(const __nv_bfloat16* X, int64_t n1, int64_t S, const __nv_bfloat16* Fhi,
                     const __nv_bfloat16* Flo, int L, float* out,
                     const __nv_bfloat16* Xlo = nullptr, __nv_bfloat16* outb = nullptr);
// Y[i + n1*k] = sum_t w[t + T*k] sum_{i2} X[i + n1*(i2 + n2*t)] Om2[i2 + n2*k]
void tc_mttkrp_first_bf16(const __nv_bfloat16* X, int64_t n1, int64_t n2, int64_t T,
                          const __nv_bfloat16* Om2, const float* w, int L, float* Y,
                          const __nv_bfloat16* Xlo = nullptr);
size_t tc_workspace_bytes(int64_t n1, int64_t S, int L);
// acc[0] += ||X - Q1 H||^2, acc[1] += ||X||^2 for BF16 X (n1 x S), Q1 FP64
// n1 x c, H FP32 c x S, on tensor cores (c <= 64, n1 % 8 == 0)
// One pass over BF16 X viewed as (n1, n2, T) for the dimension tree: Y1
// (n1 x L), Y2 (n2 x L) and C (T x L, the contraction of the first two
// dimensions weighted by their factors); Om1 is the BF16 factor of mode 1,
// Om2 the FP32 factor of the second dimension (one mode, or the Khatri-Rao
// rows of several merged modes), w the T x L table of Khatri-Rao weights of
// the rest.  Xlo (optional): the lo plane of a BF16 hi/lo X.
bool tc_tree_supported(int64_t n1, int L);
// FP32 TTM out[s + S*k] = sum_i X[i + n1*s] F[i + ldf*k] on the tensor cores
// as three TF32 products (FP32-level error); needs n1 % 4 == 0, 16-byte X,
// L <= 64.
bool tc_gemm_tn_tf32_supported(int64_t n1, int64_t S, int L, const void* X);
// FP32 residual on the tensor cores (TF32 hi/lo products of H and Q1, FP32
// comparison with X): needs n1 % 4 == 0, 16-byte X, c <= 32.
bool tc_residual_tf32_supported(int64_t n1, int64_t S, int c, const void* X);
// FP32 mode-1 MTTKRP on the tensor cores (TF32 hi/lo products):
// Y[i + n1*k] += sum_t wT[t*Lp + k] sum_{i2} X[i, i2, t] Om2[i2 + n2*k],
// Lp = L rounded up to 16 (wT zero for L <= k < Lp); Y is added to, not set.
// Needs n1 % 4 == 0, 16-byte X, L <= 64.
bool tc_mttkrp_tf32_supported(int64_t n1, int64_t n2, int64_t T, int L, const void* X);
size_t tc_mttkrp_tf32_workspace_bytes(int64_t n2, int L);
void tc_mttkrp_first_tf32(const float* X, int64_t n1, int64_t n2, int64_t T, const float* Om2,
                          const float* wT, int L, float* Y);
size_t tc_residual_tf32_workspace_bytes(int64_t n1, int64_t S);
void tc_residual_tf32(const float* X, int64_t n1, int64_t S, const double* Q1, int c, const float* H,
                      double* acc);
size_t tc_gemm_tn_tf32_workspace_bytes(int64_t n1, int L);
void tc_gemm_tn_tf32(const float* X, int64_t n1, int64_t S, const float* F, int64_t ldf, int L,
                     float* out);
// workspace of the tree's C partials (beyond tc_workspace_bytes)
size_t tc_tree_workspace_bytes(int64_t n1, int64_t n2, int64_t T, int L);
void tc_tree_bf16(const __nv_bfloat16* X, int64_t n1, int64_t n2, int64_t T,
                  const __nv_bfloat16* Om1, const float* Om2, const float* w, int L,
                  float* Y1, float* Y2, float* C, const __nv_bfloat16* Xlo = nullptr);
bool tc_residual_supported(int64_t n1, int c);
size_t tc_residual_workspace_bytes(int64_t n1, int64_t S);
void tc_residual_bf16(const __nv_bfloat16* X, int64_t n1, int64_t S, const double* Q1, int c,
                      const float* H, double* acc, const __nv_bfloat16* Xlo = nullptr);

// weights w[t + T*k] = prod_j V_j[digit_j(t) + r_j*k] (bf16 or f32 factors)
void krp_rows(const Radix& R, int64_t T, int L, bool bf16, float* w);
void split_bf16_hilo(const double* src, int64_t n, __nv_bfloat16* hi, __nv_bfloat16* lo);
void convert_bf16_to_f32(const __nv_bfloat16* src, float* dst, int64_t n);
// out[e] = bf16(x), out[n + e] = bf16(x - bf16(x))
void split_f32_bf16x2(const float* X, int64_t n, __nv_bfloat16* out);

}  // namespace krp
