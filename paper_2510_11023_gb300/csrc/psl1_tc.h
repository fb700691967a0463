// psl1_tc.h -- dense stiffness assembly on the tensor cores (tcgen05) and by the
// Toeplitz+Hankel moments (see psl1_tc.cu).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace psl1 {

constexpr int TC_KMAX = 256;   // largest K of the tensor-core assembly (N <= 256 of one MMA)

size_t assemble_tc_smem(int Npad);
cudaError_t launch_tc_tables(const double* Dt, const double* C, const double* wh, int K, int Qh, int Kpad, int Qpad,
                             __nv_bfloat16* phiT, float* cosT, float* w, cudaStream_t s);
cudaError_t launch_assemble_tc(const __nv_bfloat16* phiT, const float* wD, int units, int K, int Npad, int Kpad,
                               int Qpad, float* A, int* status, cudaStream_t s);
// C = beta C + A B^T (+ bias; act = SiLU(C)), FP32 results on tcgen05 kind::tf32 with split
// operands; B is BF16 (B16) or FP32 (B32); A, B K-major with row strides lda, ldb.
cudaError_t launch_gemm_tc(int M, int N, int K, const float* A, long long lda, const __nv_bfloat16* B16,
                           const float* B32, long long ldb, float* C, long long ldc, float beta, const float* bias,
                           float* act, int* status, cudaStream_t s);
cudaError_t launch_transpose(const float* in, int rows, int cols, float* out, cudaStream_t s);
cudaError_t launch_assemble_th(const float* cosT, const float* wD, int units, int K, int Qpad, int Q, float cA,
                               float* A, cudaStream_t s);

}  // namespace psl1
