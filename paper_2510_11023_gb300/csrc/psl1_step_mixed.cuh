// psl1_step_mixed.cuh -- the linearised step on the FP32 pipes.
//
// GB300 runs FP64 at 1/62 of its FP32 rate, so the FP64-accurate step is
// rebuilt from FP32 arithmetic:
//   * mode -> node transform, quadrature moments g_s and the load vector are
//     accumulated in double-float (unevaluated FP32 pairs, ~48-bit
//     significand) from double-float tables;
//   * D and f are evaluated in double-float at the nodes (psl1_dfmath.cuh; the
//     manufactured sources in FP64);
//   * the inner solver is Jacobi-preconditioned CG on the FP32 operator
//     I + mu cA k l (g_|k-l| + g_{k+l}) (an FP32 blocked Cholesky factor was
//     measured 3.7x slower at K = 256 and is not used);
//   * iterative refinement: r = rhs - M x with M applied in double-float
//     through the Toeplitz+Hankel form, z = M32^{-1} r in FP32, x += z, until
//     max|z| <= 1e-11 max|x|, or until the contraction of the last two
//     corrections puts the next one below 1e-13 max|x| (at most 6 sweeps).
//     The FP32 solver is only a preconditioner; the fixed point is the
//     solution of the FP64-accurate system.
// PSL1_PREC_FP32 runs the same kernel as an FP32 step: the three transforms
// from FP32 table copies with FP32 accumulation (f32_transform), D and f in
// FP32, and a single FP32 solve (no refinement).  The inexact early fine steps
// of parareal (psl1_set_inexact_fine) are this FP32 step.
#pragma once
#include "psl1_step.cuh"
#include "psl1_dfmath.cuh"

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
    int* flag;    // [0] first bad pivot, [1] PCG iterations, [2] refinement residuals of the step
    df* part;     // 2 NT: partial sums of the split transforms
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

// acc += v (double-float), used to add split partial sums
__device__ __forceinline__ void dfacc_add(dfacc& acc, df v)
{
    float s, e;
    two_sum(acc.hi, v.hi, s, e);
    acc.hi = s;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(e, v.lo));
}

// Double-float transform of a table in global memory (L2-resident), one of
//   TWO:  y0[o] = sum_{i even} A[i lda + o] x0[i],   y1[o] = sum_{i odd} A[i lda + o] x0[i]
//   else: y0[o] = sum_i A[i lda + o] (o odd ? x1[i] : x0[i])
// for o < nout, i < n; x in shared memory.  A thread owns output columns
// (loads coalesced across the warp) and issues its table loads D rows at a
// time ahead of the multiply-adds; R columns are walked together so that R D
// L2 requests per thread are in flight.  Outputs are dealt out in full rounds
// of NT (two columns per thread per pass); the columns of a last, partial
// round split their rows over several threads, whose partial sums meet in
// `part` (2 NT double-float entries).
template <bool TWO, int R, int D>
__device__ __forceinline__ void df_columns(const df* A, int lda, int i0, int i1, const int (&o)[R], int nout,
                                           const df* x0, const df* x1, dfacc (&a0)[R], dfacc (&a1)[R])
{
    const df* col[R];
    const df* xo[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        col[r] = A + (o[r] < nout ? o[r] : 0);
        xo[r] = TWO ? x0 : ((o[r] & 1) ? x1 : x0);
    }
    int i = i0;
    for (; i + D <= i1; i += D) {
        df tv[R][D];
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int j = 0; j < D; ++j) {   // read-only path: the tables are never written by the kernel
                const float2 v = __ldg(reinterpret_cast<const float2*>(col[r] + (size_t)(i + j) * lda));
                tv[r][j] = df{v.x, v.y};
            }
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int j = 0; j < D; ++j) dfacc_fma((TWO && (j & 1)) ? a1[r] : a0[r], tv[r][j], xo[r][i + j]);
    }
    for (; i < i1; ++i)
#pragma unroll
        for (int r = 0; r < R; ++r) dfacc_fma((TWO && (i & 1)) ? a1[r] : a0[r], col[r][(size_t)i * lda], xo[r][i]);
}

template <bool TWO>
__device__ void df_transform(const df* A, int lda, int n, int nout, const df* x0, const df* x1, df* y0, df* y1,
                             df* part)
{
    const int t = threadIdx.x;
    const int full = nout / NT, rem = nout - full * NT;
    for (int g = 0; g < full;) {
        if (full - g >= 2) {
            const int o[2] = {t + g * NT, t + (g + 1) * NT};
            dfacc a0[2] = {{0.f, 0.f}, {0.f, 0.f}}, a1[2] = {{0.f, 0.f}, {0.f, 0.f}};
            df_columns<TWO, 2, 8>(A, lda, 0, n, o, nout, x0, x1, a0, a1);
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                y0[o[r]] = dfacc_result(a0[r]);
                if (TWO) y1[o[r]] = dfacc_result(a1[r]);
            }
            g += 2;
        } else {
            const int o[1] = {t + g * NT};
            dfacc a0[1] = {{0.f, 0.f}}, a1[1] = {{0.f, 0.f}};
            df_columns<TWO, 1, 16>(A, lda, 0, n, o, nout, x0, x1, a0, a1);
            y0[o[0]] = dfacc_result(a0[0]);
            if (TWO) y1[o[0]] = dfacc_result(a1[0]);
            g += 1;
        }
    }
    if (rem == 0) return;
    // last round: rem columns starting at base, rows split S ways
    const int base = full * NT;
    const int S = NT / rem < 8 ? NT / rem : 8;
    if (S == 1) {   // rem >= NT/2: one thread per column
        if (t < rem) {
            const int o[1] = {base + t};
            dfacc a0[1] = {{0.f, 0.f}}, a1[1] = {{0.f, 0.f}};
            df_columns<TWO, 1, 16>(A, lda, 0, n, o, nout, x0, x1, a0, a1);
            y0[o[0]] = dfacc_result(a0[0]);
            if (TWO) y1[o[0]] = dfacc_result(a1[0]);
        }
        return;
    }
    const int L = ((n + S - 1) / S + 1) & ~1;   // even, so that row blocks start on even i
    const int c = t % rem, sp = t / rem;
    if (sp < S) {
        const int o[1] = {base + c};
        dfacc a0[1] = {{0.f, 0.f}}, a1[1] = {{0.f, 0.f}};
        const int i0 = sp * L, i1 = i0 + L < n ? i0 + L : n;
        if (i0 < i1) df_columns<TWO, 1, 8>(A, lda, i0, i1, o, nout, x0, x1, a0, a1);
        part[2 * (sp * rem + c)] = dfacc_result(a0[0]);
        part[2 * (sp * rem + c) + 1] = dfacc_result(a1[0]);
    }
    __syncthreads();
    if (t < rem) {
        dfacc a0{0.f, 0.f}, a1{0.f, 0.f};
        for (int q = 0; q < S; ++q) {
            dfacc_add(a0, part[2 * (q * rem + t)]);
            dfacc_add(a1, part[2 * (q * rem + t) + 1]);
        }
        y0[base + t] = dfacc_result(a0);
        if (TWO) y1[base + t] = dfacc_result(a1);
    }
    __syncthreads();
}

// FP32 rows i0..i1-1 of one output column: a0 (+)= sum A[i][o] x[i].hi, with
// odd rows into a1 when TWO; i0 is even, so a row's parity is that of j.
template <bool TWO>
__device__ __forceinline__ void f32_rows(const float* col, int lda, int i0, int i1, const df* x, float& a0,
                                         float& a1)
{
    int i = i0;
    for (; i + 8 <= i1; i += 8) {
        float v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = __ldg(col + (size_t)(i + j) * lda);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (TWO && (j & 1))
                a1 = fmaf(v[j], x[i + j].hi, a1);
            else
                a0 = fmaf(v[j], x[i + j].hi, a0);
        }
    }
    for (; i < i1; ++i) {
        const float v = __ldg(col + (size_t)i * lda);
        if (TWO && (i & 1))
            a1 = fmaf(v, x[i].hi, a1);
        else
            a0 = fmaf(v, x[i].hi, a0);
    }
}

// FP32 transform of an FP32 table (the FP32 step: the FP32 precision mode and the
// inexact early fine steps), with the index conventions of df_transform.  The
// inputs are the hi parts of x; the outputs are written as double-float with a
// zero lo part.  A thread owns one output column at a time (one accumulator,
// reset per column); with fewer than NT/2 outputs the rows are split over up to
// 8 threads per column, whose partial sums meet in `part` (2 NT floats).
template <bool TWO>
__device__ void f32_transform(const float* A, int lda, int n, int nout, const df* x0, const df* x1, df* y0, df* y1,
                              float* part)
{
    const int t = threadIdx.x;
    int S = nout >= NT / 2 ? 1 : NT / nout;
    S = S > 8 ? 8 : S;
    if (S == 1) {
        for (int o = t; o < nout; o += NT) {
            const df* x = TWO ? x0 : ((o & 1) ? x1 : x0);
            float a0 = 0.f, a1 = 0.f;
            f32_rows<TWO>(A + o, lda, 0, n, x, a0, a1);
            y0[o] = df{a0, 0.f};
            if (TWO) y1[o] = df{a1, 0.f};
        }
        __syncthreads();
        return;
    }
    const int L = ((n + S - 1) / S + 1) & ~1;   // even, so that row blocks start on even i
    const int c = t % nout, sp = t / nout;      // S * nout <= NT
    if (sp < S) {
        const df* x = TWO ? x0 : ((c & 1) ? x1 : x0);
        float a0 = 0.f, a1 = 0.f;
        const int i0 = sp * L, i1 = i0 + L < n ? i0 + L : n;
        if (i0 < i1) f32_rows<TWO>(A + c, lda, i0, i1, x, a0, a1);
        part[2 * (sp * nout + c)] = a0;
        part[2 * (sp * nout + c) + 1] = a1;
    }
    __syncthreads();
    if (t < nout) {
        float a0 = 0.f, a1 = 0.f;
        for (int q = 0; q < S; ++q) {
            a0 += part[2 * (q * nout + t)];
            a1 += part[2 * (q * nout + t) + 1];
        }
        y0[t] = df{a0, 0.f};
        if (TWO) y1[t] = df{a1, 0.f};
    }
    __syncthreads();
}

// nodes + moments + load.  fp32_only: D, f and the three transforms in FP32
// (FP32 tables); otherwise double-float throughout.
__device__ void nodes_moments_mixed(const InstDev& I, const TabDev& Tb, const double* tp, const double* c,
                                    double te, MixSmem& ms, double* F, bool fp32_only)
{
    const int tid = threadIdx.x, K = I.K, Qh = Tb.Qh;
    const df* Std = reinterpret_cast<const df*>(tp + Tb.oStd);
    const double* xh = tp + Tb.oX;
    const double* aux = tp + Tb.oAux;
    const double mid2 = I.lo0 + I.hi0;
    float* part32 = reinterpret_cast<float*>(ms.part);
    for (int k = tid; k < K; k += NT) ms.cdf[k] = df_from_double(c[k]);
    __syncthreads();
    // u at the node pairs: the odd-mode sum O (k even) into wpd, the even-mode sum E into wmd
    if (fp32_only)
        f32_transform<true>(reinterpret_cast<const float*>(tp + Tb.oSt32), Qh, K, Qh, ms.cdf, nullptr, ms.wpd,
                            ms.wmd, part32);
    else
        df_transform<true>(Std, Qh, K, Qh, ms.cdf, nullptr, ms.wpd, ms.wmd, ms.part);
    __syncthreads();
    const df* wd = reinterpret_cast<const df*>(tp + Tb.oWd);
    const df* auxd = reinterpret_cast<const df*>(tp + Tb.oAuxd);
    const df emt = (I.fpar[3] != 0.0 && !fp32_only) ? df_from_double(exp(-te)) : df{0.f, 0.f};
    for (int q = tid; q < Qh && !fp32_only; q += NT) {
        // D and f in double-float on the FP32 pipes (manufactured sources in FP64)
        const df o = ms.wpd[q], e = ms.wmd[q];
        const df ua = df_addn(o, e), ub = df_addn(o, df_neg(e));
        const df zero{0.f, 0.f};
        const df Da = D_eval_df(I, auxd[4 * q], auxd[4 * q + 1], zero, ua);
        const df Db = D_eval_df(I, auxd[4 * q + 2], auxd[4 * q + 3], zero, ub);
        df fs, fd;
        if (I.f_df) {
            const df fa = f_eval_df(I, auxd[4 * q], emt, ua), fb = f_eval_df(I, auxd[4 * q + 2], emt, ub);
            fs = df_addn(fa, fb);
            fd = df_addn(fa, df_neg(fb));
        } else {
            const double xa = xh[q], xb = mid2 - xa;
            const double fa = f_eval(I, xa, aux[4 * q], te, df_to_double(ua));
            const double fb = f_eval(I, xb, aux[4 * q + 2], te, df_to_double(ub));
            fs = df_from_double(fa + fb);
            fd = df_from_double(fa - fb);
        }
        const df w = wd[q];
        ms.wpd[q] = df_mul(w, df_addn(Da, Db));
        ms.wmd[q] = df_mul(w, df_addn(Da, df_neg(Db)));
        ms.fpd[q] = df_mul(w, fs);
        ms.fmd[q] = df_mul(w, fd);
    }
    // the FP32 step: every node quantity in FP32 (float copies of the weights and node
    // functions); only the manufactured sources, when present, are evaluated in FP64
    const bool src = I.fpar[4] != 0.0 || I.fpar[5] != 0.0;
    for (int q = tid; q < Qh && fp32_only; q += NT) {
        const float o = ms.wpd[q].hi, e = ms.wmd[q].hi;   // FP32 transform outputs (lo = 0)
        const float ua = o + e, ub = o - e, w = wd[q].hi;
        const float sa1 = auxd[4 * q].hi, sa2 = auxd[4 * q + 1].hi, sb1 = auxd[4 * q + 2].hi, sb2 = auxd[4 * q + 3].hi;
        const float Da = D_eval32(I, sa1, sa2, ua), Db = D_eval32(I, sb1, sb2, ub);
        float fa, fb;
        if (src) {
            const double xa = xh[q], xb = mid2 - xa;
            fa = (float)f_eval(I, xa, aux[4 * q], te, (double)ua);
            fb = (float)f_eval(I, xb, aux[4 * q + 2], te, (double)ub);
        } else {
            fa = f_eval32(I, sa1, (float)te, ua);
            fb = f_eval32(I, sb1, (float)te, ub);
        }
        ms.wpd[q] = df{w * (Da + Db), 0.f};
        ms.wmd[q] = df{w * (Da - Db), 0.f};
        ms.fpd[q] = df{w * (fa + fb), 0.f};
        ms.fmd[q] = df{w * (fa - fb), 0.f};
    }
    __syncthreads();
    // moments g_s (even s: w (D_q + D_q'), odd s: w (D_q - D_q')) and the load (even k: f_q + f_q')
    const int ns = 2 * K + 1;
    if (fp32_only) {
        f32_transform<false>(reinterpret_cast<const float*>(tp + Tb.oC32), ns, Qh, ns, ms.wpd, ms.wmd, ms.gdf,
                             nullptr, part32);
        f32_transform<false>(reinterpret_cast<const float*>(tp + Tb.oS32), K, Qh, K, ms.fpd, ms.fmd, ms.ydf,
                             nullptr, part32);
    } else {
        df_transform<false>(reinterpret_cast<const df*>(tp + Tb.oCd), ns, Qh, ns, ms.wpd, ms.wmd, ms.gdf, nullptr,
                            ms.part);
        __syncthreads();
        df_transform<false>(reinterpret_cast<const df*>(tp + Tb.oSd), K, Qh, K, ms.fpd, ms.fmd, ms.ydf, nullptr,
                            ms.part);
    }
    __syncthreads();
    for (int k = tid; k < K; k += NT) F[k] = df_to_double(ms.ydf[k]);
    __syncthreads();
}

// ------------------------------------------------------------------ FP32 PCG inner solver
// z = M^{-1} r approximately, M = I + mu cA k l (g_|k-l| + g_{k+l}) applied in
// FP32 from the moments' hi parts, Jacobi preconditioner.  For
// 0 < D_- <= D <= D_+ (the paper's Eq. Assumptions) the Jacobi-scaled operator
// has condition number about D_+/D_-, so a few iterations reduce the residual
// by FP32's resolution.  r: ms.z on entry; result in ms.z.
constexpr int PCG_MAXIT = 40;
constexpr float PCG_RTOL = INNER_RTOL_DEFAULT;
// Refinement stops when the last correction is below REFINE_TOL of the
// iterate, or when the contraction it shows (rho = |z_k| / |z_{k-1}|) puts the
// next correction, rho |z_k|, below REFINE_EST of the iterate.
constexpr float REFINE_TOL = 1e-11f;
constexpr float REFINE_EST = 1e-13f;

struct PcgSmem {
    float *x, *r, *p, *q, *pl, *dinv;   // Kp each
    float* red2;                         // 2 x (2 * NT/32): two reduction buffers, used in turn
    float *gs, *gh;                      // 2 Kmax + 8 each: moment windows
    float* part;                         // 4 NT: partial sums of the blocked product
};

// q_k = p_k + sc (k+1) acc_k with acc_k = sum_l (g_|k-l| + g_{k+l+2}) pl_l,
// k < K, into cg.q; returns this thread's share of p.q (threads own the k of
// the loop k = tid, tid + NT, ...).  Each thread first computes four
// consecutive acc_k over a chunk of the columns l: the Toeplitz and Hankel
// windows slide through registers (one new shared-memory load each per column
// instead of eight); the chunks are summed after one barrier.  No barrier
// follows: the caller's reduction publishes q.
__device__ float th_product32(int K, float sc, PcgSmem& cg)
{
    const int ng = (K + 3) / 4;
    int S = NT / ng;
    S = S < 1 ? 1 : (S > 16 ? 16 : S);
    // odd chunk length: the S chunks of a warp start in different shared-memory
    // banks (a multiple of 32 would put every chunk's loads in the same bank)
    const int L = ((K + S - 1) / S) | 1;
    const int t = threadIdx.x;
    for (int task = t; task < ng * S; task += NT) {
        const int grp = task / S, c = task % S;
        const int k0 = 4 * grp;
        const int l0 = c * L, l1 = (l0 + L < K) ? l0 + L : K;
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
        if (l0 < l1) {
            const float* gs = cg.gs + K + k0;   // T_r(l) = gs[r - l]
            const float* gh = cg.gh + k0 + 2;   // H_r(l) = gh[r + l]
            float T0 = gs[-l0], T1 = gs[1 - l0], T2 = gs[2 - l0], T3 = gs[3 - l0];
            float H0 = gh[l0], H1 = gh[l0 + 1], H2 = gh[l0 + 2], H3 = gh[l0 + 3];
            for (int l = l0; l < l1; ++l) {
                const float p = cg.pl[l];
                a0 = fmaf(T0 + H0, p, a0);
                a1 = fmaf(T1 + H1, p, a1);
                a2 = fmaf(T2 + H2, p, a2);
                a3 = fmaf(T3 + H3, p, a3);
                T3 = T2;
                T2 = T1;
                T1 = T0;
                T0 = gs[-(l + 1)];
                H0 = H1;
                H1 = H2;
                H2 = H3;
                H3 = gh[l + 4];
            }
        }
        float* out = cg.part + c * (4 * ng) + k0;
        out[0] = a0;
        out[1] = a1;
        out[2] = a2;
        out[3] = a3;
    }
    __syncthreads();
    float pq = 0.f;
    for (int k = t; k < K; k += NT) {
        float s = 0.f;
        for (int c = 0; c < S; ++c) s += cg.part[c * (4 * ng) + k];
        const float q = cg.p[k] + sc * (float)(k + 1) * s;
        cg.q[k] = q;
        pq += cg.p[k] * q;
    }
    return pq;
}

// Block sums of a and b with one barrier: the partial sums of consecutive calls
// go to the two halves of red2 in turn (buf toggles), so a call never
// overwrites the half that threads may still be reading from the call before;
// the barrier of the call in between orders them.  Every thread gets the same
// sums (same order of addition).
__device__ __forceinline__ float2 block_sum2(float a, float b, float* red2, int& buf)
{
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    float* r = red2 + buf * (2 * (NT / 32));
    buf ^= 1;
    if ((threadIdx.x & 31) == 0) {
        r[threadIdx.x >> 5] = a;
        r[NT / 32 + (threadIdx.x >> 5)] = b;
    }
    __syncthreads();
    float sa = 0.f, sb = 0.f;
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) {
        sa += r[w];
        sb += r[NT / 32 + w];
    }
    return make_float2(sa, sb);
}

__device__ void pcg32(const InstDev& I, double mu, MixSmem& ms, PcgSmem& cg, int maxit, float rtol)
{
    const int K = I.K, tid = threadIdx.x;
    const float sc = (float)(mu * I.cA);
    const df* g = ms.gdf;
    // normalise the right-hand side (refinement residuals can be ~1e-15 of the
    // solution; unscaled, the FP32 inner products would underflow)
    float rmax = 0.f;
    for (int k = tid; k < K; k += NT) rmax = fmaxf(rmax, fabsf(ms.z[k]));
    rmax = block_max(rmax, ms.red);
    if (!(rmax > 0.f) || !isfinite(rmax)) {
        __syncthreads();
        for (int k = tid; k < I.Kp; k += NT) ms.z[k] = 0.f;
        __syncthreads();
        return;
    }
    const float rs = 1.0f / rmax;
    // FP32 windows of the moments for the register-blocked product:
    // gs[j] = g_|j-K| (Toeplitz part), gh[s] = g_s (Hankel part), zero padded
    for (int j = tid; j < 2 * K + 8; j += NT) {
        int d = j > K ? j - K : K - j;
        cg.gs[j] = j <= 2 * K ? g[d].hi : 0.f;
        cg.gh[j] = j <= 2 * K ? g[j].hi : 0.f;
    }
    // the reductions below alternate between the two halves of red2 (the
    // barriers of block_max above order this call's first one after any earlier use)
    int buf = 0;
    float rz = 0.f, rr = 0.f;
    for (int k = tid; k < K; k += NT) {
        float d = 1.0f + sc * (float)((k + 1) * (k + 1)) * (g[0].hi + g[2 * k + 2].hi);
        float di = 1.0f / d;
        float r = ms.z[k] * rs, z = di * r;
        cg.dinv[k] = di;
        cg.x[k] = 0.f;
        cg.r[k] = r;
        cg.p[k] = z;
        cg.pl[k] = (float)(k + 1) * z;
        rz += r * z;
        rr += r * r;
    }
    float2 s0 = block_sum2(rz, rr, cg.red2, buf);   // its barrier also publishes the windows and p
    rz = s0.x;
    const float stop = rtol * rtol * s0.y;
    for (int it = 0; it < maxit && s0.y > 0.f; ++it) {
        if (tid == 0) ms.flag[1] += 1;
        // q = M p, and p.q (this reduction's barrier also publishes q)
        const float pq = th_product32(K, sc, cg);
        float2 s1 = block_sum2(pq, 0.f, cg.red2, buf);
        if (!(s1.x > 0.f)) {   // M p . p <= 0: not SPD (D <= 0 somewhere)
            if (tid == 0 && *ms.flag < 0) *ms.flag = 0;
            break;
        }
        float alpha = rz / s1.x;
        float rzn = 0.f, rrn = 0.f;
        for (int k = tid; k < K; k += NT) {
            cg.x[k] = fmaf(alpha, cg.p[k], cg.x[k]);
            float r = fmaf(-alpha, cg.q[k], cg.r[k]);
            cg.r[k] = r;
            float z = cg.dinv[k] * r;
            cg.q[k] = z;                      // q holds z until the p update
            rzn += r * z;
            rrn += r * r;
        }
        float2 s2 = block_sum2(rzn, rrn, cg.red2, buf);
        if (s2.y <= stop) break;
        float beta = rz > 0.f ? s2.x / rz : 0.f;
        rz = s2.x;
        for (int k = tid; k < K; k += NT) {
            float p = fmaf(beta, cg.p[k], cg.q[k]);
            cg.p[k] = p;
            cg.pl[k] = (float)(k + 1) * p;
        }
        __syncthreads();
    }
    for (int k = tid; k < I.Kp; k += NT) ms.z[k] = k < K ? cg.x[k] * rmax : 0.f;
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
        // (g_|k-l| + g_{k+l+2}) y_l: the Toeplitz and Hankel entries are added first
        // (one double-float multiply-add per entry), in two independent partial sums
        dfacc a0{0.f, 0.f}, a1{0.f, 0.f};
        int l = 0;
        for (; l + 1 < K; l += 2) {
            const int d0 = k > l ? k - l : l - k, d1 = k > l + 1 ? k - l - 1 : l + 1 - k;
            dfacc_fma(a0, df_add(ms.gdf[d0], ms.gdf[k + l + 2]), ms.ydf[l]);
            dfacc_fma(a1, df_add(ms.gdf[d1], ms.gdf[k + l + 3]), ms.ydf[l + 1]);
        }
        if (l < K) {
            const int d0 = k > l ? k - l : l - k;
            dfacc_fma(a0, df_add(ms.gdf[d0], ms.gdf[k + l + 2]), ms.ydf[l]);
        }
        dfacc_add(a0, dfacc_result(a1));
        const double s = df_to_double(dfacc_result(a0));
        ms.z[k] = (float)(ms.rhs[k] - ms.x[k] - sc * (double)(k + 1) * s);   // residual, FP32 for the solve
    }
    for (int k = K + tid; k < I.Kp; k += NT) ms.z[k] = 0.f;
    __syncthreads();
}

// The step: c (K, shared) -> out (K, shared).  Returns the first bad pivot or -1.
// one_solve: run the FP32 step (FP32 transforms, D and f, one FP32 solve, no
// refinement) -- the inexact fine steps of early parareal iterations.
// ftol > 0: the refinement may stop once the (measured or predicted) correction
// is below ftol of the iterate instead of REFINE_TOL / REFINE_EST (a looser
// refined step while parareal's increment is still large); the FP32 step solves
// to a relative residual of max(PCG_RTOL, ftol).
__device__ int step_mixed(const InstDev& I, const TabDev& Tb, const double* tp, const double* c,
                          const double* hist, double te, double mu, double* out, double* F, StepSmem& s,
                          MixSmem& ms, PcgSmem& cg, bool fp32_only, bool one_solve = false, float ftol = 0.f)
{
    const int tid = threadIdx.x;
    fp32_only = fp32_only || one_solve;   // the inexact step is the FP32 step
    nodes_moments_mixed(I, Tb, tp, c, te, ms, F, fp32_only);
    // refinement from x = 0: the first correction is the FP32 solve of rhs
    for (int k = tid; k < I.Kp; k += NT) {
        double r = k < I.K ? hist[k] + mu * F[k] : 0.0;
        ms.rhs[k] = r;
        ms.x[k] = 0.0;
        ms.z[k] = (float)r;
    }
    if (tid == 0) *s.bad = -1;
    __syncthreads();
    // inner tolerance: the FP32 step's own; the refined step's is tunable per instance
    const float rtol = fp32_only ? fmaxf(PCG_RTOL, ftol) : I.inner_rtol;
    pcg32(I, mu, ms, cg, PCG_MAXIT, rtol);
    float zprev = 0.f;
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
        const bool small = zmax <= fmaxf(REFINE_TOL, ftol) * xmax;
        const bool predicted =
            sweep >= 1 && zmax < zprev && zmax * zmax <= fmaxf(REFINE_EST, ftol) * xmax * zprev;
        if (fp32_only || small || predicted || sweep >= 6 || *s.bad >= 0) break;
        zprev = zmax;
        if (tid == 0) ms.flag[2] += 1;
        residual_df(I, mu, ms);
        pcg32(I, mu, ms, cg, PCG_MAXIT, rtol);
    }
    for (int k = tid; k < I.K; k += NT) out[k] = ms.x[k];
    __syncthreads();
    return *s.bad;
}

}  // namespace psl1
