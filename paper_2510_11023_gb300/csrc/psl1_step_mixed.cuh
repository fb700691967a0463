// psl1_step_mixed.cuh -- the linearised step on the FP32 pipes.
//
// GB300 runs FP64 at 1/62 of its FP32 rate, so the FP64-accurate step is
// rebuilt from FP32 arithmetic:
//   * mode -> node transform, quadrature moments g_s and the load vector are
//     accumulated in double-float (unevaluated FP32 pairs, ~48-bit
//     significand) from double-float tables;
//   * D and f are evaluated in FP64 at the nodes (Q evaluations per step);
//   * the SPD matrix I + mu cA k l (g_|k-l| + g_{k+l}) is factored in FP32
//     (block-packed lower storage in shared memory when it fits);
//   * iterative refinement: r = rhs - M x with M applied in double-float
//     through the Toeplitz+Hankel form, z = M32^{-1} r in FP32, x += z, until
//     max|z| <= 1e-11 max|x| (at most 6 sweeps).  The FP32 factor is only a
//     preconditioner; the fixed point is the solution of the FP64-accurate
//     system.
// PSL1_PREC_FP32 runs the same kernel with D and f evaluated in FP32 and a
// single FP32 solve (no refinement).  Its transforms stay double-float: a
// plain FP32 moment loop was found to produce wrong moments under ptxas -O3
// whenever one thread accumulates more than one moment (correct at -O1 and
// in double-float), so that loop form is not used.
#pragma once
#include "psl1_step.cuh"

namespace psl1 {



struct MixSmem {
    df* cdf;      // K   : c as double-float
    df* wpd;      // Qh  : w (D_q + D_q')  (double-float)
    df* wmd;      // Qh
    df* fpd;      // Qh  : w (f_q + f_q')
    df* fmd;      // Qh
    df* gdf;      // 2K+1 moments
    df* ydf;      // K   : l x_l
    double* x;    // Kp  solution
    double* rhs;  // Kp
    float* z;     // Kp  FP32 correction
    float* red;   // NT/32 reduction scratch
    int* flag;
};

__device__ __forceinline__ float block_max(float v, float* red)
{
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    float m = 0.f;
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) m = fmaxf(m, red[w]);
    return m;
}

// nodes + moments + load.  fp32_only: D and f in FP32.
__device__ void nodes_moments_mixed(const InstDev& I, const TabDev& Tb, const double* tp, const double* c,
                                    double te, MixSmem& ms, double* F, bool fp32_only)
{
    const int tid = threadIdx.x, K = I.K, Qh = Tb.Qh;
    const df* Std = reinterpret_cast<const df*>(tp + Tb.oStd);
    const double* xh = tp + Tb.oX;
    const double* wh = tp + Tb.oWq;
    const double* aux = tp + Tb.oAux;
    const double mid2 = I.lo0 + I.hi0;
    for (int k = tid; k < K; k += NT) ms.cdf[k] = df_from_double(c[k]);
    __syncthreads();
    for (int q = tid; q < Qh; q += NT) {
        double ua, ub;
        {
            dfacc O{0.f, 0.f}, E{0.f, 0.f};
            int k = 0;
            for (; k + 1 < K; k += 2) {
                dfacc_fma(O, Std[(size_t)k * Qh + q], ms.cdf[k]);
                dfacc_fma(E, Std[(size_t)(k + 1) * Qh + q], ms.cdf[k + 1]);
            }
            if (k < K) dfacc_fma(O, Std[(size_t)k * Qh + q], ms.cdf[k]);
            double o = df_to_double(dfacc_result(O)), e = df_to_double(dfacc_result(E));
            ua = o + e;
            ub = o - e;
        }
        double xa = xh[q], xb = mid2 - xa, w = wh[q];
        double Da, Db, fa, fb;
        if (!fp32_only) {
            Da = D_eval(I, aux[4 * q], aux[4 * q + 1], ua);
            Db = D_eval(I, aux[4 * q + 2], aux[4 * q + 3], ub);
            fa = f_eval(I, xa, aux[4 * q], te, ua);
            fb = f_eval(I, xb, aux[4 * q + 2], te, ub);
        } else {
            Da = D_eval32(I, (float)aux[4 * q], (float)aux[4 * q + 1], (float)ua);
            Db = D_eval32(I, (float)aux[4 * q + 2], (float)aux[4 * q + 3], (float)ub);
            fa = f_eval(I, xa, aux[4 * q], te, ua);   // sources keep FP64 (rarely used)
            fb = f_eval(I, xb, aux[4 * q + 2], te, ub);
            if (I.fpar[4] == 0.0 && I.fpar[5] == 0.0) {
                fa = f_eval32(I, (float)aux[4 * q], (float)te, (float)ua);
                fb = f_eval32(I, (float)aux[4 * q + 2], (float)te, (float)ub);
            }
        }
        ms.wpd[q] = df_from_double(w * (Da + Db));
        ms.wmd[q] = df_from_double(w * (Da - Db));
        ms.fpd[q] = df_from_double(w * (fa + fb));
        ms.fmd[q] = df_from_double(w * (fa - fb));
    }
    __syncthreads();
    const df* Cd = reinterpret_cast<const df*>(tp + Tb.oCd);
    const df* Sd = reinterpret_cast<const df*>(tp + Tb.oSd);
    const int ns = 2 * K + 1;
    for (int sI = tid; sI < ns; sI += NT) {
        const df* wv = (sI & 1) ? ms.wmd : ms.wpd;
        dfacc acc{0.f, 0.f};
        for (int q = 0; q < Qh; ++q) dfacc_fma(acc, Cd[(size_t)q * ns + sI], wv[q]);
        ms.gdf[sI] = dfacc_result(acc);
    }
    for (int k = tid; k < K; k += NT) {
        const df* fv = (k & 1) ? ms.fmd : ms.fpd;
        dfacc acc{0.f, 0.f};
        for (int q = 0; q < Qh; ++q) dfacc_fma(acc, Sd[(size_t)q * K + k], fv[q]);
        F[k] = df_to_double(dfacc_result(acc));
    }
    __syncthreads();
}

// FP32 matrix from the moments (hi parts), identity padding.
__device__ void fill_matrix32(const InstDev& I, const df* g, double mu, BPack<float, MIX_LDB> A)
{
    const int nb = I.nb, K = I.K;
    const int total = nb * (nb + 1) / 2 * TILE * TILE;
    const float sc = (float)(mu * I.cA);
    for (int e = threadIdx.x; e < total; e += NT) {
        int bidx = e >> 10, w = e & 1023, i = w >> 5, j = w & 31;
        int a = (int)((sqrtf(8.0f * bidx + 1.0f) - 1.0f) * 0.5f);
        while ((a + 1) * (a + 2) / 2 <= bidx) ++a;
        while (a * (a + 1) / 2 > bidx) --a;
        int Jb = bidx - a * (a + 1) / 2;
        int k = TILE * a + i, l = TILE * Jb + j;
        float val;
        if (k < K && l < K) {
            int d = k > l ? k - l : l - k;
            val = (k == l ? 1.0f : 0.0f) + sc * (float)((k + 1) * (l + 1)) * (g[d].hi + g[k + l + 2].hi);
        } else {
            val = (k == l) ? 1.0f : 0.0f;
        }
        A.blk(a, Jb)[i * MIX_LDB + j] = val;
    }
    __syncthreads();
}

// r = rhs - (I + mu cA k l T+H(g)) x, matrix applied in double-float.
__device__ void residual_df(const InstDev& I, double mu, MixSmem& ms)
{
    const int K = I.K, tid = threadIdx.x;
    for (int l = tid; l < K; l += NT) ms.ydf[l] = df_from_double((double)(l + 1) * ms.x[l]);
    __syncthreads();
    const double sc = mu * I.cA;
    for (int k = tid; k < K; k += NT) {
        dfacc a1{0.f, 0.f}, a2{0.f, 0.f};
        for (int l = 0; l < K; ++l) {
            int d = k > l ? k - l : l - k;
            dfacc_fma(a1, ms.gdf[d], ms.ydf[l]);
            dfacc_fma(a2, ms.gdf[k + l + 2], ms.ydf[l]);
        }
        double s = df_to_double(dfacc_result(a1)) + df_to_double(dfacc_result(a2));
        ms.z[k] = (float)(ms.rhs[k] - ms.x[k] - sc * (double)(k + 1) * s);   // residual, FP32 for the solve
    }
    for (int k = K + tid; k < I.Kp; k += NT) ms.z[k] = 0.f;
    __syncthreads();
}

// The step: c (K, shared) -> out (K, shared).  Returns the first bad pivot or -1.
__device__ int step_mixed(const InstDev& I, const TabDev& Tb, const double* tp, const double* c,
                          const double* hist, double te, double mu, double* out, double* F,
                          BPack<float, MIX_LDB> A, StepSmem& s, MixSmem& ms, bool fp32_only)
{
    const int tid = threadIdx.x;
    nodes_moments_mixed(I, Tb, tp, c, te, ms, F, fp32_only);
    fill_matrix32(I, ms.gdf, mu, A);
    for (int k = tid; k < I.Kp; k += NT) {
        double r = k < I.K ? hist[k] + mu * F[k] : 0.0;
        ms.rhs[k] = r;
        ms.x[k] = 0.0;
        ms.z[k] = (float)r;
    }
    if (tid == 0) *s.bad = -1;
    __syncthreads();
    chol_factor<float, MIX_LDB>(A, I.nb, s.bad);
    chol_solve<float, MIX_LDB, float>(A, I.nb, ms.z);
    for (int sweep = 0;; ++sweep) {
        float zmax = 0.f, xmax = 0.f;
        for (int k = tid; k < I.K; k += NT) {
            double xn = ms.x[k] + (double)ms.z[k];
            ms.x[k] = xn;
            zmax = fmaxf(zmax, fabsf(ms.z[k]));
            xmax = fmaxf(xmax, (float)fabs(xn));
        }
        zmax = block_max(zmax, ms.red);
        __syncthreads();
        xmax = block_max(xmax, ms.red);
        if (fp32_only || zmax <= 1e-11f * xmax || sweep >= 6) break;
        residual_df(I, mu, ms);
        chol_solve<float, MIX_LDB, float>(A, I.nb, ms.z);
    }
    for (int k = tid; k < I.K; k += NT) out[k] = ms.x[k];
    __syncthreads();
    return *s.bad;
}

}  // namespace psl1
