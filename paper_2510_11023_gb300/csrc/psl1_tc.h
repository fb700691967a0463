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
cudaError_t launch_assemble_th(const float* cosT, const float* wD, int units, int K, int Qpad, int Q, float cA,
                               float* A, cudaStream_t s);

}  // namespace psl1
