// psl1_mlp.h -- internal interface of the learned coarse correction (MLP):
// parameters, training state and the kernels that train it and run it.
//
//   G_theta(U_{0:n}) = G_n(U_{0:n}) + s o MLP(z_n)
//   z_n = [k^2 U_n(k), k < nU ; k^2 eta_n(k), k < nH ; alpha ; T_n]
//   eta_n = sum_{j<n} b_{n-j} (U_{j+1} - U_j)   (the coarse L1 history)
//   MLP: Linear(nin, W) - SiLU - Linear(W, W) - SiLU - Linear(W, W) - SiLU - Linear(W, nout)
//
// Flat parameter layout (shared with the CPU oracle): W1[W][nin], b1[W],
// W2[W][W], b2[W], W3[W][W], b3[W], W4[nout][W], b4[nout].  FP32 master
// weights and Adam moments; BF16 copies feed every product, on the tensor
// cores with FP32 accumulation.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <string>

namespace psl1 {

constexpr int MLP_MAX_IN = 320;
constexpr int MLP_MAX_WIDTH = 512;
constexpr int MLP_MAX_OUT = 512;

struct MlpDev {                    // what the coarse-sweep kernel needs for inference
    const __nv_bfloat16* wT;       // per layer, transposed [in][out] BF16 weights
    const float* bias;             // FP32 biases, concatenated b1 b2 b3 b4
    const float* oscale;           // nout output scales
    long long oT[4];               // offsets of the transposed layers in wT
    long long ob[4];               // offsets of the biases in bias
    int nU, nH, nin, width, nout;
    int on;                        // 0: plain L1 coarse propagator
};

struct MlpLayout {
    long long oW[4], ob[4];        // offsets in the flat parameter vector
    int din[4], dout[4];
    long long nparam;
};

MlpLayout mlp_layout(int nin, int width, int nout);

// kernels (launchers)
cudaError_t mlp_init_params(float* master, const MlpLayout& L, unsigned long long seed, cudaStream_t s);
cudaError_t mlp_refresh_bf16(const float* master, __nv_bfloat16* w16, __nv_bfloat16* wT, float* bias,
                             const MlpLayout& L, cudaStream_t s);
// what the tensor-core products of the network need besides the weights:
// the transposed BF16 weights, two transpose buffers (>= B x max(width, nin,
// nout) floats each) and a device status word (set if a bounded wait gave up)
struct MlpTc {
    const __nv_bfloat16* wT;
    float *tA, *tB;
    int* status;
};
cudaError_t mlp_forward(const float* X0, int B, const __nv_bfloat16* w16, const float* master, const MlpLayout& L,
                        float* const* pre, float* const* act, float* Y, const MlpTc& tc, cudaStream_t s);
// loss = mean (Y - T)^2, dY = 2 (Y - T) / (B nout); gradients of every parameter
cudaError_t mlp_backward(const float* X0, int B, const float* T, const __nv_bfloat16* w16, const MlpLayout& L,
                         float* const* pre, float* const* act, const float* Y, float* dY, float* dH, float* dH2,
                         float* grad, float* loss_acc, const MlpTc& tc, cudaStream_t s);
cudaError_t mlp_adam(float* master, const float* grad, float* m, float* v, long long n, int t, float lr, float b1,
                     float b2, float eps, cudaStream_t s);
cudaError_t mlp_gather(const float* Z, const float* T, const int* valid, int S, int nin, int nout, int B, long long a,
                       long long c, long long start, float* Xb, float* Tb, cudaStream_t s);
cudaError_t mlp_scale_targets(float* R, int S, int nvalid, int nout, float* oscale, cudaStream_t s);

}  // namespace psl1
