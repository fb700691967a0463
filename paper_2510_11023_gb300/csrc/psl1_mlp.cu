// psl1_mlp.cu -- training and inference kernels of the learned coarse correction.
#include "psl1_mlp.h"
#include "psl1_tc.h"

namespace psl1 {

MlpLayout mlp_layout(int nin, int width, int nout)
{
    MlpLayout L;
    int din[4] = {nin, width, width, width}, dout[4] = {width, width, width, nout};
    long long o = 0;
    for (int l = 0; l < 4; ++l) {
        L.din[l] = din[l];
        L.dout[l] = dout[l];
        L.oW[l] = o;
        o += (long long)din[l] * dout[l];
        L.ob[l] = o;
        o += dout[l];
    }
    L.nparam = o;
    return L;
}

// splitmix64 of (seed, index) -> uniform in [-1, 1)
__device__ __forceinline__ float hash_uniform(unsigned long long seed, unsigned long long i)
{
    unsigned long long z = seed + 0x9E3779B97F4A7C15ULL * (i + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z ^= z >> 31;
    return (float)((double)(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0);
}

// Linear-layer default: U(-1/sqrt(fan_in), 1/sqrt(fan_in)) for weights and biases;
// the output layer starts at zero, so an untrained correction is exactly zero.
__global__ void k_mlp_init(float* p, MlpLayout L, unsigned long long seed)
{
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= L.nparam) return;
    int l = 0;
    while (l < 3 && e >= L.oW[l + 1]) ++l;
    float a = rsqrtf((float)L.din[l]);
    p[e] = (l == 3) ? 0.f : a * hash_uniform(seed, (unsigned long long)e);
}

cudaError_t mlp_init_params(float* master, const MlpLayout& L, unsigned long long seed, cudaStream_t s)
{
    k_mlp_init<<<(unsigned)((L.nparam + 255) / 256), 256, 0, s>>>(master, L, seed);
    return cudaGetLastError();
}

// BF16 copy in the flat layout, and transposed [in][out] BF16 weights per layer
__global__ void k_mlp_refresh(const float* master, __nv_bfloat16* w16, __nv_bfloat16* wT, MlpLayout L)
{
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= L.nparam) return;
    w16[e] = __float2bfloat16_rn(master[e]);
    int l = 0;
    while (l < 3 && e >= L.oW[l + 1]) ++l;
    long long r = e - L.oW[l];
    long long nw = (long long)L.din[l] * L.dout[l];
    if (r < nw) {   // weight W[o][i] -> wT[i][o]
        long long o = r / L.din[l], i = r % L.din[l];
        long long oT = 0;
        for (int q = 0; q < l; ++q) oT += (long long)L.din[q] * L.dout[q];
        wT[oT + i * L.dout[l] + o] = w16[e];
    }
}

cudaError_t mlp_refresh_bf16(const float* master, __nv_bfloat16* w16, __nv_bfloat16* wT, float* /*bias*/,
                             const MlpLayout& L, cudaStream_t s)
{
    k_mlp_refresh<<<(unsigned)((L.nparam + 255) / 256), 256, 0, s>>>(master, w16, wT, L);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ GEMMs
// Every product of the network runs on the tensor cores (psl1_tc.cu,
// launch_gemm_tc: tcgen05 kind::tf32 with the FP32 operands split into TF32
// hi + lo parts, FP32 accumulation in tensor memory; BF16 weights are exact in
// TF32), so the forward pass, the gradients and the training keep FP32-level
// accuracy.  Offsets of the transposed BF16 weights [in][out] of layer l.
static long long wT_offset(const MlpLayout& L, int l)
{
    long long o = 0;
    for (int q = 0; q < l; ++q) o += (long long)L.din[q] * L.dout[q];
    return o;
}

// pre[l] = act[l-1] W_l^T + b_l, act[l] = SiLU(pre[l]) for l < 3; Y = pre[3].
cudaError_t mlp_forward(const float* X0, int B, const __nv_bfloat16* w16, const float* master, const MlpLayout& L,
                        float* const* pre, float* const* act, float* Y, const MlpTc& tc, cudaStream_t s)
{
    const float* in = X0;
    for (int l = 0; l < 4; ++l) {
        int din = L.din[l], dout = L.dout[l];
        float* out = (l < 3) ? pre[l] : Y;
        // out[b][o] = sum_i in[b][i] W[o][i] + b[o]  (W rows are K-major: the flat layout)
        cudaError_t e = launch_gemm_tc(B, dout, din, in, din, w16 + L.oW[l], nullptr, din, out, dout, 0.f,
                                       master + L.ob[l], l < 3 ? act[l] : nullptr, tc.status, s);
        if (e != cudaSuccess) return e;
        in = (l < 3) ? act[l] : nullptr;
    }
    return cudaSuccess;
}

__global__ void k_loss_grad(const float* Y, const float* T, int n, float inv, float* dY, float* loss_acc)
{
    __shared__ float red[8];
    float s = 0.f;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        float d = Y[e] - T[e];
        dY[e] = 2.f * d * inv;
        s += d * d * inv;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) t += red[w];
        atomicAdd(loss_acc, t);
    }
}

// dA = dH * SiLU'(A) in place
__global__ void k_silu_back(float* dH, const float* A, long long n)
{
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    float a = A[e], sg = 1.0f / (1.0f + expf(-a));
    dH[e] *= sg * (1.0f + a * (1.0f - sg));
}

// db[n] = sum_b D[b][n]
__global__ void k_colsum(const float* D, int B, int N, float* db)
{
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float s = 0.f;
    for (int b = 0; b < B; ++b) s += D[(long long)b * N + n];
    db[n] = s;
}

cudaError_t mlp_backward(const float* X0, int B, const float* T, const __nv_bfloat16* w16, const MlpLayout& L,
                         float* const* pre, float* const* act, const float* Y, float* dY, float* dH, float* dH2,
                         float* grad, float* loss_acc, const MlpTc& tc, cudaStream_t s)
{
    const int nout = L.dout[3];
    const int n = B * nout;
    k_loss_grad<<<std::min(1024, (n + 255) / 256), 256, 0, s>>>(Y, T, n, 1.0f / (float)n, dY, loss_acc);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const float* d = dY;   // gradient w.r.t. the layer output (pre-activation for l < 3 after SiLU')
    float* bufs[2] = {dH, dH2};
    for (int l = 3; l >= 0; --l) {
        int din = L.din[l], dout = L.dout[l];
        const float* xin = (l > 0) ? act[l - 1] : X0;
        // dW_l = d^T xin : C[o][i] = sum_b d[b][o] xin[b][i], both operands transposed to K(=b)-major
        e = launch_transpose(d, B, dout, tc.tA, s);
        if (e == cudaSuccess) e = launch_transpose(xin, B, din, tc.tB, s);
        if (e == cudaSuccess)
            e = launch_gemm_tc(dout, din, B, tc.tA, B, nullptr, tc.tB, B, grad + L.oW[l], din, 0.f, nullptr, nullptr,
                               tc.status, s);
        if (e != cudaSuccess) return e;
        k_colsum<<<(dout + 255) / 256, 256, 0, s>>>(d, B, dout, grad + L.ob[l]);
        if (l == 0) break;
        // dX = d W_l : C[b][i] = sum_o d[b][o] W[o][i] = sum_o d[b][o] W^T[i][o]
        float* dx = bufs[l & 1];
        e = launch_gemm_tc(B, din, dout, d, dout, tc.wT + wT_offset(L, l), nullptr, dout, dx, din, 0.f, nullptr,
                           nullptr, tc.status, s);
        if (e != cudaSuccess) return e;
        long long nn = (long long)B * din;
        k_silu_back<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(dx, pre[l - 1], nn);
        d = dx;
    }
    return cudaGetLastError();
}

__global__ void k_adam(float* p, const float* g, float* m, float* v, long long n, float c1, float c2, float lr,
                       float b1, float b2, float eps)
{
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    float gi = g[e];
    float mi = b1 * m[e] + (1.f - b1) * gi;
    float vi = b2 * v[e] + (1.f - b2) * gi * gi;
    m[e] = mi;
    v[e] = vi;
    p[e] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

cudaError_t mlp_adam(float* master, const float* grad, float* m, float* v, long long n, int t, float lr, float b1,
                     float b2, float eps, cudaStream_t s)
{
    float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
    k_adam<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(master, grad, m, v, n, c1, c2, lr, b1, b2, eps);
    return cudaGetLastError();
}

// minibatch j <- sample valid[(a (start + j) + c) mod S]  (an affine permutation of
// the S valid sample slots when gcd(a, S) = 1)
__global__ void k_gather(const float* Z, const float* T, const int* valid, int S, int nin, int nout, int B,
                         long long a, long long c, long long start, float* Xb, float* Tb)
{
    int j = blockIdx.x;
    if (j >= B) return;
    long long idx = valid[(a * (start + j) + c) % S];
    for (int i = threadIdx.x; i < nin; i += blockDim.x) Xb[(long long)j * nin + i] = Z[idx * nin + i];
    for (int i = threadIdx.x; i < nout; i += blockDim.x) Tb[(long long)j * nout + i] = T[idx * nout + i];
}

cudaError_t mlp_gather(const float* Z, const float* T, const int* valid, int S, int nin, int nout, int B, long long a,
                       long long c, long long start, float* Xb, float* Tb, cudaStream_t s)
{
    k_gather<<<B, 128, 0, s>>>(Z, T, valid, S, nin, nout, B, a, c, start, Xb, Tb);
    return cudaGetLastError();
}

// oscale[k] = RMS over the nvalid samples of R[:,k] (rows that are not samples hold
// zeros); 1 where it vanishes; R[:,k] /= oscale[k]
__global__ void k_scale_targets(float* R, int S, int nvalid, int nout, float* oscale)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nout) return;
    double s = 0.0;
    for (int i = 0; i < S; ++i) {
        double r = R[(long long)i * nout + k];
        s += r * r;
    }
    double rms = sqrt(s / (nvalid > 0 ? nvalid : 1));
    float sc = rms > 0.0 ? (float)rms : 1.0f;
    oscale[k] = sc;
    for (int i = 0; i < S; ++i) R[(long long)i * nout + k] /= sc;
}

cudaError_t mlp_scale_targets(float* R, int S, int nvalid, int nout, float* oscale, cudaStream_t s)
{
    k_scale_targets<<<(nout + 127) / 128, 128, 0, s>>>(R, S, nvalid, nout, oscale);
    return cudaGetLastError();
}

}  // namespace psl1
