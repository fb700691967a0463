// psl1_tc.cu -- dense stiffness assembly on the 5th-generation tensor cores
// (tcgen05) and, for comparison, by the Toeplitz+Hankel moments.
//
// The stiffness of the 1D sine-Galerkin step is a quadrature contraction
// (Eq. AForm):   A_kl = sum_q phi_k'(x_q) w_q D_q phi_l'(x_q),
// i.e. A = Phi'^T diag(w D) Phi' with Phi' the Q x K table of derivatives.
// k_assemble_tc computes it as a GEMM for one (unit, 128-row block): the A
// operand is rows of Phi'^T (BF16, built once per table set), the B operand is
// Phi'^T scaled column-wise by w D of the unit (BF16, formed in shared memory),
// accumulation in FP32 in tensor memory, 64 nodes per stage in two shared-memory
// buffers, one elected thread issuing tcgen05.mma.cta_group::1.kind::f16 with
// M = 128, N = K rounded up to 16, K-step 16.
//
// k_assemble_th computes the same matrix from the 2K+1 moments
// g_s = sum_q w_q D_q cos(s pi th_q), A_kl = cA k l (g_|k-l| + g_{k+l})
// (the product-to-sum identity of the sine derivatives), in FP32 on the CUDA
// cores: O(QK) work instead of O(QK^2).  The solver uses the moments; these two
// kernels exist to measure that choice.
//
// Shared-memory operand layout (no swizzle, K-major): 8-row x 16-byte core
// matrices stored as 128 contiguous bytes; cores adjacent along K are 128 bytes
// apart (the descriptor's leading byte offset) and 8-row groups are 1024 bytes
// apart (its stride byte offset), so a 64-node stage of R rows takes R * 128
// bytes.  Every address the descriptors can form stays inside its tile even if
// the two offsets were read the other way round.
#include <cuda_bf16.h>

#include "psl1_kernels.h"
#include "psl1_tc.h"

namespace psl1 {

namespace {

constexpr int TM = 128;        // accumulator rows of one MMA (tensor-memory lanes)
constexpr int TKC = 64;        // nodes per stage: 64 BF16 = 128 bytes per row
constexpr int TNT = 128;       // threads: 4 warps, one per tensor-memory lane quarter
constexpr int LBO = 128;       // bytes between K-adjacent core matrices
constexpr int SBO = 1024;      // bytes between 8-row groups (8 cores of 128 bytes)
constexpr long long WAIT_LIMIT = 1LL << 26;   // bounded mbarrier polls (~ seconds)

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr)
{
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((LBO >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((SBO >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;   // descriptor version of sm_100-class tensor cores; no swizzle, base offset 0
    return d;
}

// kind::f16 instruction descriptor: D FP32, A and B BF16, both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(1));
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait; false if the limit was reached
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity)
{
    for (long long i = 0; i < WAIT_LIMIT; ++i)
        if (mbar_try(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, int acc)
{
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// byte offset of element (row r, node c) in a K-major 64-node stage
__device__ __forceinline__ int tile_off(int r, int c)
{
    return (r >> 3) * SBO + (c >> 3) * LBO + (r & 7) * 16 + (c & 7) * 2;
}

}  // namespace

// One unit's stiffness rows [128 mt, 128 mt + 128) (blockIdx.y = mt, blockIdx.x = unit).
//   phiT : Kpad x Qpad BF16, row k = phi_{k+1}'(x_q) over the nodes in ascending order
//          (zero rows k >= K and zero columns q >= Q)
//   wD   : units x Qpad FP32, w_q D_q of each unit (zero for q >= Q)
//   A    : units x K x K FP32 (row-major)
// Dynamic shared memory: 2 stages x (128 + Npad) x 128 bytes, then the
// barriers and the tensor-memory address.
__global__ void __launch_bounds__(TNT) k_assemble_tc(const __nv_bfloat16* __restrict__ phiT,
                                                     const float* __restrict__ wD, int K, int Npad, int Qpad,
                                                     int ncols, float* __restrict__ A, int* status)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int unit = blockIdx.x, mt = blockIdx.y;
    const int abytes = TM * TKC * 2, bbytes = Npad * TKC * 2, stage = abytes + bbytes;
    unsigned char* st[2] = {sm, sm + stage};
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + 2 * stage);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 2);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        mbar_init(&bar[0]);
        mbar_init(&bar[1]);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    const uint32_t idesc = idesc_bf16(TM, Npad);
    const float* w = wD + (size_t)unit * Qpad;
    const int nchunks = Qpad / TKC;
    bool ok = true;
    for (int c = 0; c < nchunks && ok; ++c) {
        const int b = c & 1;
        if (c >= 2) ok = mbar_wait(&bar[b], (uint32_t)(((c - 2) >> 1) & 1));   // stage b free again
        if (!ok) break;
        unsigned char* ta = st[b];
        unsigned char* tb = st[b] + abytes;
        const int q0 = c * TKC;
        // A: rows 128 mt + r of phiT, 8 nodes (16 bytes) per piece
        for (int e = tid; e < TM * (TKC / 8); e += TNT) {
            const int r = e >> 3, cc = (e & 7) * 8;
            const uint4 v = *reinterpret_cast<const uint4*>(phiT + (size_t)(mt * TM + r) * Qpad + q0 + cc);
            *reinterpret_cast<uint4*>(ta + tile_off(r, cc)) = v;
        }
        // B: rows l of phiT scaled by w D at the stage's nodes, rounded to BF16
        for (int e = tid; e < Npad * (TKC / 8); e += TNT) {
            const int r = e >> 3, cc = (e & 7) * 8;
            const uint4 v = *reinterpret_cast<const uint4*>(phiT + (size_t)r * Qpad + q0 + cc);
            const __nv_bfloat16* pv = reinterpret_cast<const __nv_bfloat16*>(&v);
            const float4 w0 = *reinterpret_cast<const float4*>(w + q0 + cc);
            const float4 w1 = *reinterpret_cast<const float4*>(w + q0 + cc + 4);
            const float ws[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
            __align__(16) __nv_bfloat16 o[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) o[i] = __float2bfloat16_rn(__bfloat162float(pv[i]) * ws[i]);
            *reinterpret_cast<uint4*>(tb + tile_off(r, cc)) = *reinterpret_cast<const uint4*>(o);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic writes -> tensor-core reads
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int kk = 0; kk < TKC / 16; ++kk) {   // K-step 16 = two K-adjacent cores
                const uint64_t ad = smem_desc(smem_u32(ta + kk * 2 * LBO));
                const uint64_t bd = smem_desc(smem_u32(tb + kk * 2 * LBO));
                mma_bf16(tmem, ad, bd, idesc, (c > 0 || kk > 0) ? 1 : 0);
            }
            mma_commit(&bar[b]);
        }
        __syncthreads();
    }
    // the last commit covers every earlier MMA of this thread
    if (ok && nchunks > 0) ok = mbar_wait(&bar[(nchunks - 1) & 1], (uint32_t)(((nchunks - 1) >> 1) & 1));
    if (!ok && tid == 0) atomicCAS(status, 0, 1);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
        // warp w reads lanes 32 w .. 32 w + 31 = rows of the block
        const int row = mt * TM + warp * 32 + lane;
        for (int c0 = 0; c0 < Npad; c0 += 16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            if (row < K) {
                float* out = A + ((size_t)unit * K + row) * K;
#pragma unroll
                for (int i = 0; i < 16; ++i)
                    if (c0 + i < K) out[c0 + i] = v[i];
            }
        }
    } else {
        // give the tensor cores time to finish (or fail) before the memory is released
        mbar_wait(&bar[0], 0);
        mbar_wait(&bar[1], 0);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
}

// The same matrices from the moments: g_s = sum_q wD_q cos(s pi th_q), s = 0..2K,
// A_kl = cA k l (g_|k-l| + g_{k+l}), FP32.  cosT: Qpad x (2K+1) FP32 (row = node).
__global__ void __launch_bounds__(256) k_assemble_th(const float* __restrict__ cosT, const float* __restrict__ wD,
                                                     int K, int Qpad, int Q, float cA, float* __restrict__ A)
{
    extern __shared__ float g[];   // 2K + 1 moments
    const int unit = blockIdx.x, ns = 2 * K + 1;
    const float* w = wD + (size_t)unit * Qpad;
    for (int s = threadIdx.x; s < ns; s += blockDim.x) {
        float a0 = 0.f, a1 = 0.f;
        int q = 0;
        for (; q + 1 < Q; q += 2) {
            a0 = fmaf(w[q], cosT[(size_t)q * ns + s], a0);
            a1 = fmaf(w[q + 1], cosT[(size_t)(q + 1) * ns + s], a1);
        }
        if (q < Q) a0 = fmaf(w[q], cosT[(size_t)q * ns + s], a0);
        g[s] = a0 + a1;
    }
    __syncthreads();
    float* out = A + (size_t)unit * K * K;
    for (int e = threadIdx.x; e < K * K; e += blockDim.x) {
        const int k = e / K, l = e - k * K;
        const int d = k > l ? k - l : l - k;
        out[e] = cA * (float)(k + 1) * (float)(l + 1) * (g[d] + g[k + l + 2]);
    }
}

// Unfolded tables of one (K, Q, box): phiT[k][q] = phi_{k+1}'(x_q) in BF16 and
// cosT[q][s] = cos(s pi th_q), w[q] (ascending nodes), from the folded FP64
// tables (node q < Q/2 and its mirror Q-1-q: phi_k'(x') = (-1)^k phi_k'(x),
// cos(s pi (1 - th)) = (-1)^s cos(s pi th)).
__global__ void k_tc_tables(const double* Dt, const double* C, const double* wh, int K, int Qh, int Kpad, int Qpad,
                            __nv_bfloat16* phiT, float* cosT, float* w)
{
    const int Q = 2 * Qh, ns = 2 * K + 1;
    const long long n1 = (long long)Kpad * Qpad;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n1; e += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(e / Qpad), q = (int)(e % Qpad);
        double v = 0.0;
        if (k < K && q < Q) {
            const bool mir = q >= Qh;
            const int qq = mir ? Q - 1 - q : q;
            v = Dt[(size_t)k * Qh + qq];
            if (mir && ((k + 1) & 1)) v = -v;
        }
        phiT[e] = __float2bfloat16_rn((float)v);
    }
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < (long long)Q * ns;
         e += (long long)gridDim.x * blockDim.x) {
        const int q = (int)(e / ns), s = (int)(e % ns);
        const bool mir = q >= Qh;
        const int qq = mir ? Q - 1 - q : q;
        double v = C[(size_t)qq * ns + s];
        if (mir && (s & 1)) v = -v;
        cosT[e] = (float)v;
    }
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < Q; q += gridDim.x * blockDim.x)
        w[q] = (float)wh[q < Qh ? q : Q - 1 - q];
}

// ------------------------------------------------------------------ GEMM for the MLP
// C[m][n] = beta C[m][n] + sum_k A[m][k] B[n][k] (+ bias[n]); act[m][n] = SiLU(C[m][n])
// when act is given.  A (FP32) and B (BF16 weights, or FP32 data when SPLIT_B)
// are K-major with row strides lda, ldb.  tcgen05.mma kind::tf32: every FP32
// operand is split into TF32 parts, x = hi + lo with hi = x truncated to TF32
// (the bits the tensor cores read) and lo = x - hi (exact in FP32), and the
// products hi*hi + lo*hi (+ hi*lo) are accumulated in FP32 in tensor memory,
// so the result has FP32-level accuracy (BF16 weights are exact in TF32).
// One CTA per 128 x 128 output tile, 32 K-elements (128 bytes per row) per
// stage in two shared-memory buffers, the same core-matrix geometry as above.
constexpr int GN = 128;                     // output columns per CTA (tensor-memory columns)
constexpr int GKC = 32;                     // K elements (FP32) per stage

__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, int acc)
{
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
}

// byte offset of FP32 element (row r, k c) in a K-major 32-element stage
__device__ __forceinline__ int tile_off4(int r, int c)
{
    return (r >> 3) * SBO + (c >> 2) * LBO + (r & 7) * 16 + (c & 3) * 4;
}

__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

template <bool SPLIT_B>
__global__ void __launch_bounds__(TNT) k_gemm_tc(int M, int N, int K, const float* __restrict__ A, long long lda,
                                                 const __nv_bfloat16* __restrict__ B16, const float* __restrict__ B32,
                                                 long long ldb, float* C, long long ldc, float beta,
                                                 const float* __restrict__ bias, float* act, int* status)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n0 = blockIdx.x * GN, m0 = blockIdx.y * TM;
    constexpr int tbytes = TM * GKC * 4;              // one 128-row operand tile (16 KB)
    constexpr int stage = (SPLIT_B ? 4 : 3) * tbytes;  // A hi, A lo, B hi [, B lo]
    unsigned char* st[2] = {sm, sm + stage};
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + 2 * stage);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 2);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(GN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        mbar_init(&bar[0]);
        mbar_init(&bar[1]);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    const uint32_t idesc = idesc_tf32(TM, GN);
    const int nchunks = (K + GKC - 1) / GKC;
    bool ok = true;
    for (int c = 0; c < nchunks && ok; ++c) {
        const int b = c & 1;
        if (c >= 2) ok = mbar_wait(&bar[b], (uint32_t)(((c - 2) >> 1) & 1));
        if (!ok) break;
        unsigned char* ah = st[b];
        unsigned char* al = ah + tbytes;
        unsigned char* bh = al + tbytes;
        unsigned char* bl = bh + tbytes;
        const int k0 = c * GKC;
        for (int e = tid; e < TM * GKC; e += TNT) {   // A: split into TF32 hi + lo, zero outside
            const int r = e / GKC, kk = e % GKC, m = m0 + r, k = k0 + kk;
            const float x = (m < M && k < K) ? A[(long long)m * lda + k] : 0.f;
            const float h = tf32_hi(x);
            *reinterpret_cast<float*>(ah + tile_off4(r, kk)) = h;
            *reinterpret_cast<float*>(al + tile_off4(r, kk)) = x - h;
        }
        for (int e = tid; e < GN * GKC; e += TNT) {   // B rows n0 + r
            const int r = e / GKC, kk = e % GKC, n = n0 + r, k = k0 + kk;
            float x = 0.f;
            if (n < N && k < K) x = SPLIT_B ? B32[(long long)n * ldb + k] : __bfloat162float(B16[(long long)n * ldb + k]);
            const float h = SPLIT_B ? tf32_hi(x) : x;
            *reinterpret_cast<float*>(bh + tile_off4(r, kk)) = h;
            if (SPLIT_B) *reinterpret_cast<float*>(bl + tile_off4(r, kk)) = x - h;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int kk = 0; kk < GKC / 8; ++kk) {   // K-step 8 = two K-adjacent cores of 4 FP32
                const uint32_t off = kk * 2 * LBO;
                const uint64_t dah = smem_desc(smem_u32(ah + off)), dal = smem_desc(smem_u32(al + off));
                const uint64_t dbh = smem_desc(smem_u32(bh + off));
                mma_tf32(tmem, dah, dbh, idesc, (c > 0 || kk > 0) ? 1 : 0);
                mma_tf32(tmem, dal, dbh, idesc, 1);
                if (SPLIT_B) mma_tf32(tmem, dah, smem_desc(smem_u32(bl + off)), idesc, 1);
            }
            mma_commit(&bar[b]);
        }
        __syncthreads();
    }
    if (ok && nchunks > 0) ok = mbar_wait(&bar[(nchunks - 1) & 1], (uint32_t)(((nchunks - 1) >> 1) & 1));
    if (!ok && tid == 0) atomicCAS(status, 0, 1);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
        const int m = m0 + warp * 32 + lane;
        for (int c0 = 0; c0 < GN; c0 += 16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            if (m < M) {
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int n = n0 + c0 + i;
                    if (n >= N) continue;
                    const long long ci = (long long)m * ldc + n;
                    float y = v[i];
                    if (beta != 0.f) y += beta * C[ci];
                    if (bias) y += bias[n];
                    C[ci] = y;
                    if (act) act[ci] = y / (1.0f + expf(-y));
                }
            }
        }
    } else {
        mbar_wait(&bar[0], 0);
        mbar_wait(&bar[1], 0);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(GN));
}

cudaError_t launch_gemm_tc(int M, int N, int K, const float* A, long long lda, const __nv_bfloat16* B16,
                           const float* B32, long long ldb, float* C, long long ldc, float beta, const float* bias,
                           float* act, int* status, cudaStream_t s)
{
    if (M <= 0 || N <= 0) return cudaSuccess;
    dim3 grid((N + GN - 1) / GN, (M + TM - 1) / TM);
    const bool split = B32 != nullptr;
    const size_t sm = 2 * (size_t)(split ? 4 : 3) * TM * GKC * 4 + 64;
    if (split) {
        cudaError_t e = cudaFuncSetAttribute(k_gemm_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        k_gemm_tc<true><<<grid, TNT, sm, s>>>(M, N, K, A, lda, B16, B32, ldb, C, ldc, beta, bias, act, status);
    } else {
        cudaError_t e = cudaFuncSetAttribute(k_gemm_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        k_gemm_tc<false><<<grid, TNT, sm, s>>>(M, N, K, A, lda, B16, B32, ldb, C, ldc, beta, bias, act, status);
    }
    return cudaGetLastError();
}

// out[c][r] = in[r][c] (rows x cols FP32), 32 x 32 tiles through shared memory
__global__ void k_transpose(const float* __restrict__ in, int rows, int cols, float* __restrict__ out)
{
    __shared__ float t[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int r = r0 + i, c = c0 + threadIdx.x;
        if (r < rows && c < cols) t[i][threadIdx.x] = in[(long long)r * cols + c];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int c = c0 + i, r = r0 + threadIdx.x;
        if (r < rows && c < cols) out[(long long)c * rows + r] = t[threadIdx.x][i];
    }
}

cudaError_t launch_transpose(const float* in, int rows, int cols, float* out, cudaStream_t s)
{
    dim3 grid((cols + 31) / 32, (rows + 31) / 32), block(32, 8);
    k_transpose<<<grid, block, 0, s>>>(in, rows, cols, out);
    return cudaGetLastError();
}

size_t assemble_tc_smem(int Npad) { return 2 * (size_t)(TM + Npad) * TKC * 2 + 64; }

cudaError_t launch_tc_tables(const double* Dt, const double* C, const double* wh, int K, int Qh, int Kpad, int Qpad,
                             __nv_bfloat16* phiT, float* cosT, float* w, cudaStream_t s)
{
    k_tc_tables<<<256, 256, 0, s>>>(Dt, C, wh, K, Qh, Kpad, Qpad, phiT, cosT, w);
    return cudaGetLastError();
}

cudaError_t launch_assemble_tc(const __nv_bfloat16* phiT, const float* wD, int units, int K, int Npad, int Kpad,
                               int Qpad, float* A, int* status, cudaStream_t s)
{
    int ncols = 32;
    while (ncols < Npad) ncols <<= 1;
    const size_t sm = assemble_tc_smem(Npad);
    cudaError_t e = cudaFuncSetAttribute(k_assemble_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    dim3 grid(units, Kpad / TM);
    k_assemble_tc<<<grid, TNT, sm, s>>>(phiT, wD, K, Npad, Qpad, ncols, A, status);
    return cudaGetLastError();
}

cudaError_t launch_assemble_th(const float* cosT, const float* wD, int units, int K, int Qpad, int Q, float cA,
                               float* A, cudaStream_t s)
{
    k_assemble_th<<<units, 256, (2 * K + 1) * sizeof(float), s>>>(cosT, wD, K, Qpad, Q, cA, A);
    return cudaGetLastError();
}

}  // namespace psl1
