// psl1_kernels.cu -- the parareal / serial solver kernels (1D and 2D instantiations).
//
//   k_fstage        F stage: every active (instance, slice) unit runs its m
//                   fine steps (Eq. NumericalSchemeFine); persistent CTAs pull
//                   units from an atomic counter (units pre-sorted by cost).
//   k_coarse_sweep  sequential coarse sweep with the parareal correction
//                   U^{k+1}_{n+1} = G_n(U^{k+1}_{0:n}) + (F_old(n) - G_old(n))
//                   (Eq. Parareal, G_old stored as in Fig. parareal), and the
//                   increment e_k of the stopping test.
//   k_serial_hyb    S_hyb: the sequential sweep U_{n+1} = F_n(U_{0:n}).
//   k_uni_hist/step S_uni: full-history uniform L1 -- an HBM-streaming history
//                   kernel over all instances plus one step CTA per instance.
#include "psl1_kernels.h"
#include "psl1_step.cuh"
#include "psl1_step_mixed.cuh"
#include "psl1_step2d.cuh"
#include "psl1_step_cheb.cuh"

namespace psl1 {

struct Carve {
    double *cur, *hist, *nxt, *F;
    StepSmem s;
    MixSmem ms;
    PcgSmem cg;
    df *mz, *mh0, *mh1;      // learned-correction features and hidden activations (double-float)
    Step2D s2;               // 2D working arrays
    Split sp;                // 2D: this CTA's share of a cluster-split step (size 1: the whole step)
    ChebSmem ch;             // collocation step
};

template <typename T>
__device__ __forceinline__ T* at(char* base, int off)
{
    return off >= 0 ? reinterpret_cast<T*>(base + off) : nullptr;
}

__device__ __forceinline__ Carve carve2d(const PathArgs& a, char* base)
{
    const Layout2D& L = a.L2;
    char* gbase = reinterpret_cast<char*>(a.work + (size_t)blockIdx.x * a.work_stride);
    auto at2 = [&](int r) -> void* {
        if (L.off[r] < 0) return nullptr;
        return (L.glob[r] ? gbase : base) + L.off[r];
    };
    Carve c{};
    c.cur = static_cast<double*>(at2(R2_CUR));
    c.hist = static_cast<double*>(at2(R2_HIST));
    c.nxt = static_cast<double*>(at2(R2_NXT));
    c.F = static_cast<double*>(at2(R2_F));
    c.s.bad = static_cast<int*>(at2(R2_BAD));
    c.ms.flag = c.s.bad;
    c.s2.cdf = static_cast<df*>(at2(R2_CDF));
    c.s2.T1 = at2(R2_T1);
    c.s2.T2 = at2(R2_T2);
    c.s2.N1 = at2(R2_N1);
    c.s2.N2 = at2(R2_N2);
    c.s2.wd = at2(R2_WD);
    c.s2.wd32 = static_cast<float*>(at2(R2_WD32));
    c.s2.dinv = at2(R2_DINV);
    c.s2.x = at2(R2_PX);
    c.s2.r = at2(R2_PR);
    c.s2.p = at2(R2_PP);
    c.s2.q = at2(R2_PQ);
    c.s2.xr = static_cast<double*>(at2(R2_XR));
    c.s2.rhs = static_cast<double*>(at2(R2_RHS));
    c.s2.z = static_cast<float*>(at2(R2_Z));
    c.s2.tab32 = static_cast<float*>(at2(R2_TAB32));
    c.s2.red = at2(R2_RED);
    if (L.off[R2_SPLIT] >= 0) {   // rank and size are set by the kernel that splits the step
        c.sp.pb = reinterpret_cast<double*>(static_cast<char*>(at2(R2_SPLIT)) + 16);
        c.sp.stride = a.Kmax + 8;   // >= K + size - 1 (size <= 8)
    }
    return c;
}

// D2: the kernel is the 2D instantiation (1D and 2D code are compiled into
// separate kernels so that neither inflates the other's register allocation)
template <bool D2>
__device__ __forceinline__ Carve carve(const PathArgs& a, char* base)
{
    if constexpr (D2) return carve2d(a, base);
    const SmemLayout& L = a.L;
    Carve c;
    c.cur = at<double>(base, L.cur);
    c.hist = at<double>(base, L.hist);
    c.nxt = at<double>(base, L.nxt);
    c.F = at<double>(base, L.F);
    c.s.v = at<double>(base, L.v);
    c.s.wp = at<double>(base, L.wp);
    c.s.wm = at<double>(base, L.wm);
    c.s.fp = at<double>(base, L.fp);
    c.s.fm = at<double>(base, L.fm);
    c.s.g = at<double>(base, L.g);
    c.s.bad = at<int>(base, L.bad);
    c.ms.cdf = at<df>(base, L.cdf);
    c.ms.wpd = at<df>(base, L.wpd);
    c.ms.wmd = at<df>(base, L.wmd);
    c.ms.fpd = at<df>(base, L.fpd);
    c.ms.fmd = at<df>(base, L.fmd);
    c.ms.gdf = at<df>(base, L.gdf);
    c.ms.ydf = at<df>(base, L.ydf);
    c.ms.x = at<double>(base, L.x);
    c.ms.rhs = at<double>(base, L.rhs);
    c.ms.z = at<float>(base, L.z);
    c.ms.red = at<float>(base, L.red);
    c.ms.flag = c.s.bad;
    c.ms.part = at<df>(base, L.mpart);
    c.cg.x = at<float>(base, L.cgx);
    c.cg.r = at<float>(base, L.cgr);
    c.cg.p = at<float>(base, L.cgp);
    c.cg.q = at<float>(base, L.cgq);
    c.cg.pl = at<float>(base, L.cgpl);
    c.cg.dinv = at<float>(base, L.cgdinv);
    c.cg.red2 = at<float>(base, L.cgred);
    c.cg.gs = at<float>(base, L.cggs);
    c.cg.gh = at<float>(base, L.cggh);
    c.cg.part = at<float>(base, L.cgpart);
    c.mz = at<df>(base, L.mz);
    c.mh0 = at<df>(base, L.mh0);
    c.mh1 = at<df>(base, L.mh1);
    c.ch.M = at<double>(base, L.cm);
    c.ch.u = at<double>(base, L.cu);
    c.ch.Dc = at<double>(base, L.cdc);
    c.ch.r = at<double>(base, L.cr);
    c.ch.l = at<double>(base, L.cl);
    c.ch.piv = at<int>(base, L.cpiv);
    return c;
}

// Shared-memory layout of the 1D step kernels.  Regions are 16-byte aligned.
SmemLayout make_layout(int prec, int Kmax, int Kpmax, int Qhmax, int Kc)
{
    SmemLayout L;
    int off = 0;
    auto take = [&](size_t bytes) {
        int o = off;
        off += (int)((bytes + 15) / 16 * 16);
        return o;
    };
    const bool f64 = prec == 0;
    L.cur = take(8 * (size_t)Kmax);
    L.hist = take(8 * (size_t)Kmax);
    L.nxt = take(8 * (size_t)Kmax);
    L.F = take(8 * (size_t)Kmax);
    L.v = f64 ? take(8 * (size_t)Kpmax) : -1;
    L.wp = f64 ? take(8 * (size_t)Qhmax) : -1;
    L.wm = f64 ? take(8 * (size_t)Qhmax) : -1;
    L.fp = f64 ? take(8 * (size_t)Qhmax) : -1;
    L.fm = f64 ? take(8 * (size_t)Qhmax) : -1;
    L.g = f64 ? take(8 * (size_t)(2 * Kmax + 1)) : -1;
    L.bad = take(16);
    L.cdf = f64 ? -1 : take(8 * (size_t)Kmax);
    L.wpd = f64 ? -1 : take(8 * (size_t)Qhmax);
    L.wmd = f64 ? -1 : take(8 * (size_t)Qhmax);
    L.fpd = f64 ? -1 : take(8 * (size_t)Qhmax);
    L.fmd = f64 ? -1 : take(8 * (size_t)Qhmax);
    L.gdf = f64 ? -1 : take(8 * (size_t)(2 * Kmax + 1));
    L.ydf = f64 ? -1 : take(8 * (size_t)Kmax);
    L.x = f64 ? -1 : take(8 * (size_t)Kpmax);
    L.rhs = f64 ? -1 : take(8 * (size_t)Kpmax);
    L.z = f64 ? -1 : take(4 * (size_t)Kpmax);
    L.red = f64 ? -1 : take(4 * (NT / 32));
    const bool pcg = !f64;   // CG inner solver of the FP32-pipe paths
    L.cgx = pcg ? take(4 * (size_t)Kpmax) : -1;
    L.cgr = pcg ? take(4 * (size_t)Kpmax) : -1;
    L.cgp = pcg ? take(4 * (size_t)Kpmax) : -1;
    L.cgq = pcg ? take(4 * (size_t)Kpmax) : -1;
    L.cgpl = pcg ? take(4 * (size_t)Kpmax) : -1;
    L.cgdinv = pcg ? take(4 * (size_t)Kpmax) : -1;
    L.cgred = pcg ? take(4 * 4 * (NT / 32)) : -1;
    L.cggs = pcg ? take(4 * (size_t)(2 * Kmax + 8)) : -1;
    L.cggh = pcg ? take(4 * (size_t)(2 * Kmax + 8)) : -1;
    L.cgpart = pcg ? take(4 * (size_t)(4 * NT)) : -1;
    L.mpart = f64 ? -1 : take(8 * 2 * (size_t)NT);
    const bool ch = Kc > 0;   // collocation: dense K x K system, nodal vectors of n + 1 = K + 2
    L.cm = ch ? take(8 * (size_t)Kc * Kc) : -1;
    L.cu = ch ? take(8 * (size_t)(Kc + 2)) : -1;
    L.cdc = ch ? take(8 * (size_t)(Kc + 2)) : -1;
    L.cr = ch ? take(8 * (size_t)Kc) : -1;
    L.cl = ch ? take(8 * (size_t)Kc) : -1;
    L.cpiv = ch ? take(16) : -1;
    // the learned correction's buffers come last, so that kernels which never run it
    // (the F stage, the serial fine sweep) launch with less shared memory: at K = 256 the
    // F stage then fits four CTAs per SM
    L.fine = off;
    L.mz = take(8 * (size_t)MLP_MAX_IN);
    L.mh0 = take(8 * (size_t)MLP_MAX_WIDTH);
    L.mh1 = take(8 * (size_t)MLP_MAX_WIDTH);
    L.total = off;
    return L;
}

size_t step_smem_bytes(const PathArgs& a) { return (size_t)a.L.total; }
size_t fine_smem_bytes(const PathArgs& a) { return (size_t)(a.dim2 ? a.L.total : a.L.fine); }

Layout2D make_layout2d(int prec, int Kmax, long long nT, long long nN, long long ntab, int max_smem, int split)
{
    Layout2D L;
    const bool f64 = prec == 0;
    const long long e = f64 ? 8 : 4;   // CG vector element
    long long bytes[R2_COUNT];
    bytes[R2_BAD] = 16;
    bytes[R2_RED] = 8 * 4 * (NT / 32);   // two buffers of two sums (8-byte elements)
    bytes[R2_SPLIT] = split > 1 ? 16 + 8LL * 2 * (Kmax + 8) : 0;   // receive and gather buffers
    bytes[R2_DINV] = e * Kmax;
    bytes[R2_PX] = e * Kmax;
    bytes[R2_PR] = e * Kmax;
    bytes[R2_PP] = e * Kmax;
    bytes[R2_PQ] = e * Kmax;
    bytes[R2_TAB32] = f64 ? 0 : 4 * 2 * ntab;
    bytes[R2_T1] = 8 * nT;
    bytes[R2_T2] = 8 * nT;
    bytes[R2_Z] = f64 ? 0 : 4LL * Kmax;
    bytes[R2_WD32] = f64 ? 0 : 4 * nN;
    bytes[R2_N1] = 8 * nN;
    bytes[R2_N2] = 8 * nN;
    bytes[R2_CDF] = f64 ? 0 : 8LL * Kmax;
    bytes[R2_XR] = f64 ? 0 : 8LL * Kmax;
    bytes[R2_RHS] = f64 ? 0 : 8LL * Kmax;
    bytes[R2_CUR] = 8LL * Kmax;
    bytes[R2_HIST] = 8LL * Kmax;
    bytes[R2_NXT] = 8LL * Kmax;
    bytes[R2_F] = 8LL * Kmax;
    bytes[R2_WD] = 8 * nN;
    long long soff = 0, goff = 0;
    for (int r = 0; r < R2_COUNT; ++r) {
        L.off[r] = -1;
        L.glob[r] = 0;
        if (bytes[r] <= 0) continue;
        const long long b = (bytes[r] + 15) / 16 * 16;
        // the flag and reduction words and the cluster's partial sums always sit in shared memory
        if (soff + b <= max_smem || r == R2_BAD || r == R2_RED || r == R2_SPLIT) {
            L.off[r] = (int)soff;
            soff += b;
        } else {
            L.off[r] = (int)goff;
            L.glob[r] = 1;
            goff += b;
        }
    }
    L.smem = (int)soff;
    L.gbytes = goff;
    return L;
}

enum { WHERE_FINE = 1, WHERE_COARSE = 2, WHERE_UNI = 3, WHERE_ONE = 4 };

template <bool D2>
__device__ __forceinline__ int do_step(const PathArgs& a, const InstDev& I, const double* c,
                                       const double* hist, double te, double mu, double* out, Carve& cv,
                                       bool one_solve = false, float ftol = 0.f)
{
    const TabDev& Tb = a.tab[I.tab];
    int bad;
    if (threadIdx.x == 0) {
        cv.s.bad[1] = 0;
        cv.s.bad[2] = 0;
    }
    if constexpr (D2) {
        const TabDev& TY = a.tab[I.tabY];
        if (a.prec == 0)
            bad = step2d_fp64(I, Tb, TY, a.tp, c, hist, te, mu, out, cv.F, cv.s2, cv.s.bad, cv.sp);
        else
            bad = step2d_mixed(I, Tb, TY, a.tp, c, hist, te, mu, out, cv.F, cv.s2, cv.s.bad, a.prec == 2 || one_solve,
                               cv.sp, ftol);
        // algorithmic FLOPs: each operator application is four folded one-axis
        // transforms, 4 (Mx My Qy/2 + Mx Qy Qx/2) multiply-adds; the set-up
        // (node values, load, diagonal) costs one application, the coefficient
        // evaluation ~30 per node.
        if (threadIdx.x == 0 && a.flops && cv.sp.rank == 0) {   // once per (split) step
            const double ap = 8.0 * ((double)I.Mx * I.My * I.Qhy + (double)I.Mx * I.Qy * I.Qh);
            const double f = ap * (1.0 + cv.s.bad[1] + cv.s.bad[2]) + 30.0 * I.Q * I.Qy;
            atomicAdd(a.flops + a.flop_slot, f);
        }
        return bad;
    } else {
        if (I.basis == 1) {   // Chebyshev-Lobatto collocation (FP64 handles only)
            bad = step_cheb(I, a.cheb, c, hist, te, mu, out, cv.ch, cv.s.bad);
            if (threadIdx.x == 0 && a.flops) {
                const double K = I.K;
                atomicAdd(a.flops + a.flop_slot, 2.0 * K * K * (K + 2) + 2.0 * K * K * K / 3.0 + 2.0 * K * K);
            }
            return bad;
        }
        if (a.prec == 0) {
            BPack<double, TILE> A{a.work + (size_t)blockIdx.x * a.work_stride};
            bad = step_fp64(I, Tb, a.tp, c, hist, te, mu, out, cv.F, A, cv.s);
        } else {
            bad = step_mixed(I, Tb, a.tp, c, hist, te, mu, out, cv.F, cv.s, cv.ms, cv.cg, a.prec == 2, one_solve,
                             ftol);
        }
        // algorithmic FLOPs of the step: transforms (u, moments, load: 4 K^2 multiply-adds with
        // Q = 2K nodes), coefficient evaluation (~30 per node), and the solve -- FP64: Cholesky
        // K^3/3 + two triangular solves 2 K^2; FP32 pipes: 4 K^2 per Toeplitz+Hankel product
        // (refinement residuals and PCG iterations).
        if (threadIdx.x == 0 && a.flops) {
            const double K = I.K, K2 = K * K;
            double f = 8.0 * K2 + 30.0 * I.Q;
            if (a.prec == 0)
                f += K * K2 / 3.0 + 2.0 * K2;
            else
                f += 4.0 * K2 * (cv.s.bad[1] + cv.s.bad[2]);
            atomicAdd(a.flops + a.flop_slot, f);
        }
        return bad;
    }
}

__device__ __forceinline__ void check_finite(const PathArgs& a, const double* v, int K, int ii, int where,
                                             int info)
{
    for (int k = threadIdx.x; k < K; k += NT)
        if (!isfinite(v[k])) report(a.status, -3, ii, where, info);
}

// The grid a slice is propagated on: its steps, step size, mu and the
// coarse-history weights m^-a b(d + r/m) (row d < P, column r - 1 < m).
struct SliceGrid {
    int m;
    double dt, mu;
    const double* bC;
    const df* bCd;
};

// the fine grid of Eq. FineGrid (m = N/P steps per slice)
__device__ __forceinline__ SliceGrid fine_grid(const PathArgs& a, const InstDev& I)
{
    return {I.m, I.dt, I.mu, a.bp + I.oB + I.Nb + 1, a.bpd + I.oB + I.Nb + 1};
}

// the coarse propagator's substep grid (mc steps per slice)
__device__ __forceinline__ SliceGrid substep_grid(const PathArgs& a, const InstDev& I)
{
    return {I.mc, I.dtc, I.muc, a.bcc + I.oBc, a.bccd + I.oBc};
}

// F_n of instance ii on coarse states U (rows 0..n, global): g.m steps with
// the local fine history kept in the CTA's ring and the coarse history
// m^-a sum_{i=1}^n b(n-i+r/m) (U_i - U_{i-1})  (Eq. L1Fine, difference form).
// Fine steps of one slice served by one pass over the coarse differences when
// the coarse-history terms are formed ahead of the steps.
constexpr int HC_R = 8;

// dud_ready: the caller has already stored the coarse differences of rows
// 0..n-1 in the CTA's slot (a sweep appends one row per step).
// ftol: the refined 1D step's looser refinement target (0: the full one).
template <bool D2>
__device__ void fine_slice(const PathArgs& a, int ii, int n, const double* U, double* Vout, double* out,
                           Carve& cv, double* ring, bool one_solve, const SliceGrid& g, bool dud_ready = false,
                           float ftol = 0.f)
{
    const InstDev& I = a.inst[ii];
    const int K = I.K, m = g.m, tid = threadIdx.x;
    const double* bF = a.bp + I.oB;
    const double* bC = g.bC;
    // FP32-pipe paths: the history sums accumulate in double-float, the coarse
    // differences U_i - U_{i-1} are formed once per slice, and the ring holds
    // the fine differences as double-float pairs
    const bool dfh = a.prec != 0;
    const df* bFd = a.bpd + I.oB;
    const df* bCd = g.bCd;
    df* dud = a.dud + (size_t)blockIdx.x * a.dud_stride;
    df* ringd = reinterpret_cast<df*>(ring);
    for (int k = tid; k < K; k += NT) {
        cv.cur[k] = U[(size_t)n * K + k];
        if (Vout) Vout[k] = cv.cur[k];
    }
    if (dfh && !dud_ready)
        for (int e = tid; e < n * K; e += NT) dud[e] = df_from_double(U[e + K] - U[e]);
    __syncthreads();
    // The coarse-history terms of all m steps, m^-a sum_i b(n-i+r/m) (U_i - U_{i-1}),
    // formed ahead of the steps, HC_R steps per pass over the differences: the
    // differences are read m / HC_R times per slice instead of once per step.  Each
    // thread later reads the entries it wrote (the same k), so no barrier is needed.
    df* hc = (dfh && a.hc) ? a.hc + (size_t)blockIdx.x * a.hc_stride : nullptr;
    if (hc && n > 0) {
        for (int r0 = 0; r0 < m; r0 += HC_R) {
            const int nr = m - r0 < HC_R ? m - r0 : HC_R;
            for (int k = tid; k < K; k += NT) {
                dfacc acc[HC_R];
#pragma unroll
                for (int q = 0; q < HC_R; ++q) acc[q] = dfacc{0.f, 0.f};
                for (int i = 1; i <= n; ++i) {
                    const df d = dud[(size_t)(i - 1) * K + k];
                    const df* bc = bCd + (size_t)(n - i) * m + r0;
#pragma unroll
                    for (int q = 0; q < HC_R; ++q)
                        if (q < nr) dfacc_fma(acc[q], bc[q], d);
                }
#pragma unroll
                for (int q = 0; q < HC_R; ++q)
                    if (q < nr) hc[(size_t)(r0 + q) * K + k] = dfacc_result(acc[q]);
            }
        }
    }
    for (int r = 1; r <= m; ++r) {
        for (int k = tid; k < K && dfh; k += NT) {
            // four independent partial sums (the loads of a term do not wait on the previous one)
            dfacc a0{0.f, 0.f}, a1{0.f, 0.f}, a2{0.f, 0.f}, a3{0.f, 0.f};
            int j = 1;
            for (; j + 3 <= r - 1; j += 4) {
                dfacc_fma(a0, bFd[r - j], ringd[(size_t)(j - 1) * K + k]);
                dfacc_fma(a1, bFd[r - j - 1], ringd[(size_t)j * K + k]);
                dfacc_fma(a2, bFd[r - j - 2], ringd[(size_t)(j + 1) * K + k]);
                dfacc_fma(a3, bFd[r - j - 3], ringd[(size_t)(j + 2) * K + k]);
            }
            for (; j <= r - 1; ++j) dfacc_fma(a0, bFd[r - j], ringd[(size_t)(j - 1) * K + k]);
            if (hc) {
                if (n > 0) dfacc_add(a0, hc[(size_t)(r - 1) * K + k]);
            } else {
                const df* bc = bCd + (r - 1);
                int i = 1;
                for (; i + 3 <= n; i += 4) {
                    dfacc_fma(a0, bc[(size_t)(n - i) * m], dud[(size_t)(i - 1) * K + k]);
                    dfacc_fma(a1, bc[(size_t)(n - i - 1) * m], dud[(size_t)i * K + k]);
                    dfacc_fma(a2, bc[(size_t)(n - i - 2) * m], dud[(size_t)(i + 1) * K + k]);
                    dfacc_fma(a3, bc[(size_t)(n - i - 3) * m], dud[(size_t)(i + 2) * K + k]);
                }
                for (; i <= n; ++i) dfacc_fma(a0, bc[(size_t)(n - i) * m], dud[(size_t)(i - 1) * K + k]);
            }
            dfacc_add(a0, dfacc_result(a1));
            dfacc_add(a2, dfacc_result(a3));
            dfacc_add(a0, dfacc_result(a2));
            cv.hist[k] = cv.cur[k] - df_to_double(dfacc_result(a0));
        }
        for (int k = tid; k < K && !dfh; k += NT) {
            double h = cv.cur[k];
            for (int j = 1; j <= r - 1; ++j) h -= bF[r - j] * ring[(size_t)(j - 1) * K + k];
            const double* bc = bC + (r - 1);
            for (int i = 1; i <= n; ++i)
                h -= bc[(size_t)(n - i) * m] * (U[(size_t)i * K + k] - U[(size_t)(i - 1) * K + k]);
            cv.hist[k] = h;
        }
        if (tid == 0 && a.flops && cv.sp.rank == 0) atomicAdd(a.flops + a.flop_slot, 2.0 * K * (r - 1 + n));
        __syncthreads();
        int bad = do_step<D2>(a, I, cv.cur, cv.hist, I.dT * n + g.dt * (r - 1), g.mu, cv.nxt, cv, one_solve, ftol);
        if (bad >= 0 && threadIdx.x == 0) report(a.status, -2, ii, WHERE_FINE, n * m + r);
        check_finite(a, cv.nxt, K, ii, WHERE_FINE, n * m + r);
        for (int k = tid; k < K; k += NT) {
            if (dfh)
                ringd[(size_t)(r - 1) * K + k] = df_from_double(cv.nxt[k] - cv.cur[k]);
            else
                ring[(size_t)(r - 1) * K + k] = cv.nxt[k] - cv.cur[k];
            cv.cur[k] = cv.nxt[k];
            if (Vout) Vout[(size_t)r * K + k] = cv.nxt[k];
        }
        __syncthreads();
    }
    for (int k = tid; k < K; k += NT) out[k] = cv.cur[k];
    __syncthreads();
}

// Features of the learned correction at coarse node n (cv.cur = U_n,
// cv.hist = U_n - eta_n after coarse_step), zero for modes beyond K.
__device__ __forceinline__ double learned_feature(const MlpDev& M, const InstDev& I, int n, const Carve& cv, int i)
{
    if (i < M.nU) return i < I.K ? (double)(i + 1) * (i + 1) * cv.cur[i] : 0.0;
    if (i < M.nU + M.nH) {
        int k = i - M.nU;
        return k < I.K ? (double)(k + 1) * (k + 1) * (cv.cur[k] - cv.hist[k]) : 0.0;
    }
    return (i == M.nU + M.nH) ? I.alpha : I.dT * n;
}

// FP32 features (training samples)
__device__ void learned_features(const MlpDev& M, const InstDev& I, int n, const Carve& cv, float* z)
{
    for (int i = threadIdx.x; i < M.nin; i += NT) z[i] = (float)learned_feature(M, I, n, cv, i);
}

// One dense layer of the single-sample forward inside a coarse step: transposed
// BF16 weights (exact in FP32), double-float inputs and accumulation, SiLU in
// FP64.  Parareal stops on the increment of its iterates, so G has to be a
// smooth function of U far below the tolerance; FP32 inference leaves a
// rounding floor near 1e-8 in the increments.
__device__ __forceinline__ void mlp_layer_df(const MlpDev& M, int l, const df* in, df* out, bool silu)
{
    const int din = l == 0 ? M.nin : M.width, dout = l == 3 ? M.nout : M.width;
    const __nv_bfloat16* w = M.wT + M.oT[l];
    const float* b = M.bias + M.ob[l];
    for (int o = threadIdx.x; o < dout; o += NT) {
        dfacc acc{b[o], 0.f};
        for (int i = 0; i < din; ++i) dfacc_fma(acc, df{__bfloat162float(w[(size_t)i * dout + o]), 0.f}, in[i]);
        double a = df_to_double(dfacc_result(acc));
        out[o] = df_from_double(silu ? a / (1.0 + exp(-a)) : a);
    }
    __syncthreads();
}

// G_theta = G_n + s o MLP(z): adds the learned correction to cv.nxt
__device__ void learned_correction(const PathArgs& a, const InstDev& I, int n, Carve& cv)
{
    const MlpDev& M = a.mlp;
    for (int i = threadIdx.x; i < M.nin; i += NT) cv.mz[i] = df_from_double(learned_feature(M, I, n, cv, i));
    __syncthreads();
    mlp_layer_df(M, 0, cv.mz, cv.mh0, true);
    mlp_layer_df(M, 1, cv.mh0, cv.mh1, true);
    mlp_layer_df(M, 2, cv.mh1, cv.mh0, true);
    mlp_layer_df(M, 3, cv.mh0, cv.mh1, false);
    const int kk = I.K < M.nout ? I.K : M.nout;
    for (int k = threadIdx.x; k < kk; k += NT) cv.nxt[k] += (double)M.oscale[k] * df_to_double(cv.mh1[k]);
    __syncthreads();
}

// G_n of instance ii on U (rows 0..n, global) -> cv.nxt.  History in the
// difference form U_n - sum_{j=0}^{n-1} b_{n-j} (U_{j+1} - U_j) of Eq. L1Scheme.
// one_solve: the FP32 step (inexact early iterations; MIXED handles).
// dud_ready: the coarse differences of rows 0..n-1 are already in the CTA's
// slot (FP32-pipe paths; the sweep appends one row per step).
template <bool D2>
__device__ void coarse_step(const PathArgs& a, int ii, int n, const double* U, Carve& cv, bool one_solve = false,
                            bool dud_ready = false)
{
    const InstDev& I = a.inst[ii];
    const int K = I.K, tid = threadIdx.x;
    if (I.mc > 1) {
        // G with mc L1 substeps per slice: the fine propagator on the substep grid
        // (the CTA's ring slot holds its local history); result in cv.nxt
        double* ring = a.ring + (size_t)blockIdx.x * a.ring_stride;
        fine_slice<D2>(a, ii, n, U, nullptr, cv.nxt, cv, ring, one_solve, substep_grid(a, I), dud_ready);
        return;
    }
    if (a.prec != 0) {
        // FP32-pipe paths: the history sum in double-float over the stored differences
        // (on GB300 an FP64 operation costs 64 FP32 lanes; this sum is n K terms per step)
        df* dud = a.dud + (size_t)blockIdx.x * a.dud_stride;
        const df* bFd = a.bpd + I.oB;
        if (!dud_ready) {
            for (int e = tid; e < n * K; e += NT) dud[e] = df_from_double(U[e + K] - U[e]);
            __syncthreads();
        }
        for (int k = tid; k < K; k += NT) {
            dfacc a0{0.f, 0.f}, a1{0.f, 0.f};
            int j = 0;
            for (; j + 1 < n; j += 2) {
                dfacc_fma(a0, bFd[n - j], dud[(size_t)j * K + k]);
                dfacc_fma(a1, bFd[n - j - 1], dud[(size_t)(j + 1) * K + k]);
            }
            if (j < n) dfacc_fma(a0, bFd[n - j], dud[(size_t)j * K + k]);
            dfacc_add(a0, dfacc_result(a1));
            const double c = U[(size_t)n * K + k];
            cv.cur[k] = c;
            cv.hist[k] = c - df_to_double(dfacc_result(a0));
        }
    } else {
        const double* bF = a.bp + I.oB;
        for (int k = tid; k < K; k += NT) {
            double c = U[(size_t)n * K + k], h = c;
            for (int j = 0; j < n; ++j) h -= bF[n - j] * (U[(size_t)(j + 1) * K + k] - U[(size_t)j * K + k]);
            cv.cur[k] = c;
            cv.hist[k] = h;
        }
    }
    if (tid == 0 && a.flops && cv.sp.rank == 0) atomicAdd(a.flops + a.flop_slot, 2.0 * K * n);
    __syncthreads();
    int bad = do_step<D2>(a, I, cv.cur, cv.hist, I.dT * n, I.muT, cv.nxt, cv, one_solve);
    if (bad >= 0 && threadIdx.x == 0) report(a.status, -2, ii, WHERE_COARSE, n);
    check_finite(a, cv.nxt, K, ii, WHERE_COARSE, n);
    if constexpr (!D2)   // the learned correction is defined for 1D instances
        if (a.mlp.on) learned_correction(a, I, n, cv);
}

// Training samples from a parareal iterate: for every (instance, n >= nfirst):
// features of U^k_{0:n} and the correction parareal applies there,
// F_old(n) - G_old(n) = F_n(U^k_{0:n}) - G_n(U^k_{0:n}).  Sample slot:
// base + ii * P + n (slots n < nfirst are left untouched and not used).
__global__ void __launch_bounds__(NT) k_iterate_dataset(PathArgs a, const double* Uk, const double* Fv,
                                                        const double* Gold, const int* nfirst, float* Z, float* R,
                                                        long long base)
{
    extern __shared__ __align__(16) char smem_raw[];
    Carve cv = carve<false>(a, smem_raw);
    const MlpDev& M = a.mlp;
    const int ii = blockIdx.y, n = blockIdx.x;
    const InstDev& I = a.inst[ii];
    if (n >= I.P || n < nfirst[ii]) return;
    const double* U = Uk + I.oU;
    const double* bF = a.bp + I.oB;
    for (int k = threadIdx.x; k < I.K; k += NT) {
        double c = U[(size_t)n * I.K + k], h = c;
        for (int j = 0; j < n; ++j) h -= bF[n - j] * (U[(size_t)(j + 1) * I.K + k] - U[(size_t)j * I.K + k]);
        cv.cur[k] = c;
        cv.hist[k] = h;
    }
    __syncthreads();
    const long long s = base + (long long)ii * I.P + n;
    learned_features(M, I, n, cv, Z + s * M.nin);
    for (int k = threadIdx.x; k < M.nout; k += NT) {
        size_t e = (size_t)I.oPK + (size_t)n * I.K + k;
        R[s * M.nout + k] = k < I.K ? (float)(Fv[e] - Gold[e]) : 0.f;
    }
}

cudaError_t launch_iterate_dataset(const PathArgs& a, int B, int P, const double* Uk, const double* Fv,
                                   const double* Gold, const int* nfirst, float* Z, float* R, long long base,
                                   cudaStream_t s)
{
    size_t sm = step_smem_bytes(a);
    cudaError_t e = cudaFuncSetAttribute(k_iterate_dataset, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    dim3 grid(P, B);
    k_iterate_dataset<<<grid, NT, sm, s>>>(a, Uk, Fv, Gold, nfirst, Z, R, base);
    return cudaGetLastError();
}

// Training samples of the learned correction from a serial S_hyb solution Us:
// for sample s = (instance ii, node n < P): features z_n and the residual
// U_{n+1} - G_n(U_{0:n}) of the plain L1 coarse propagator (first nout modes).
__global__ void __launch_bounds__(NT) k_coarse_dataset(PathArgs a, const double* Us, const int2* units, int nunits,
                                                       int* counter, float* Z, float* R)
{
    extern __shared__ __align__(16) char smem_raw[];
    Carve cv = carve<false>(a, smem_raw);
    __shared__ int s_u;
    const MlpDev& M = a.mlp;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_u = atomicAdd(counter, 1);
        __syncthreads();
        const int u = s_u;
        if (u >= nunits) break;
        const int ii = units[u].x, n = units[u].y;
        const InstDev& I = a.inst[ii];
        const double* U = Us + I.oU;
        PathArgs plain = a;
        plain.mlp.on = 0;
        coarse_step<false>(plain, ii, n, U, cv);
        const long long s = (long long)ii * I.P + n;
        learned_features(M, I, n, cv, Z + s * M.nin);
        for (int k = threadIdx.x; k < M.nout; k += NT)
            R[s * M.nout + k] = k < I.K ? (float)(U[(size_t)(n + 1) * I.K + k] - cv.nxt[k]) : 0.f;
    }
}

// Inexact early iterations (opt-in, MIXED handles: prec 1): while an instance's last increment
// is above a.loose_above (and in its first iteration, k = nfirst = 0, when no
// increment exists yet), its F stage runs the slices n > nfirst with the FP32
// step and its coarse sweep evaluates G with the FP32 step.
__device__ __forceinline__ bool inexact_iteration(const PathArgs& a, int ii, int nfirst)
{
    return a.prec == 1 && a.loose_above > 0.0 && (nfirst == 0 || a.incr[ii] > a.loose_above);
}

// MINB: CTAs per SM the register allocation is bounded for (1D: 2, or 3 or 4
// with some spilling; the autotuner picks the fastest; 2D: 1)
template <bool D2, int MINB>
__global__ void __launch_bounds__(NT, MINB)
k_fstage(PathArgs a, const double* Uold, double* Fv, const int2* units, int nunits, int* counter,
         const int* nfirst, const int* active)
{
    extern __shared__ __align__(16) char smem_raw[];
    Carve cv = carve<D2>(a, smem_raw);
    __shared__ int s_u;
    double* ring = a.ring + (size_t)blockIdx.x * a.ring_stride;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_u = atomicAdd(counter, 1);
        __syncthreads();
        const int u = s_u;
        if (u >= nunits) break;
        const int ii = units[u].x, n = units[u].y;
        if (!active[ii] || n < nfirst[ii]) continue;
        const InstDev& I = a.inst[ii];
        // Inexact early iterations: the slices after the first one still in error
        // take the FP32 step.  Slice n = nfirst starts from exact states and stays
        // exact, so U^{k+1}_{k+1} and the fixed point are unchanged.
        const bool one_solve = n > nfirst[ii] && inexact_iteration(a, ii, nfirst[ii]);
        // Looser refined steps (opt-in, MIXED): the refined F of slices n > nfirst stops
        // refining at refine_factor e_{k-1} of the iterate (at most 1e-6, at least the
        // full target; e_{-1} is taken as 1).  F is evaluated afresh in every
        // iteration, so the iteration needs no consistency between them; slice nfirst
        // keeps the full target and with it the exact prefix, and as e_k falls the
        // target returns to the full one, so the fixed point is S_hyb.
        // The FP32 steps of those slices likewise solve to a relative residual of
        // factor e_{k-1} (at most 1e-4, at least the FP32 step's own 1e-7).
        float ftol = 0.f;
        if (a.prec == 1 && a.refine_factor > 0.0 && n > nfirst[ii])
            ftol = (float)fmin(one_solve ? 1e-4 : 1e-6, a.refine_factor * (nfirst[ii] > 0 ? a.incr[ii] : 1.0));
        fine_slice<D2>(a, ii, n, Uold + I.oU, nullptr, Fv + I.oPK + (size_t)n * I.K, cv, ring, one_solve,
                       fine_grid(a, I), false, ftol);
    }
}

// G_old(n) = G_n(U_{0:n}) of every (instance, slice) unit at given states U (a
// parareal iteration resumed from a checkpoint); persistent CTAs over the units
template <bool D2>
__global__ void __launch_bounds__(NT, D2 ? 1 : 2)
k_coarse_at(PathArgs a, const double* Uk, double* Gold, const int2* units, int nunits, int* counter)
{
    extern __shared__ __align__(16) char smem_raw[];
    Carve cv = carve<D2>(a, smem_raw);
    __shared__ int s_u;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_u = atomicAdd(counter, 1);
        __syncthreads();
        const int u = s_u;
        if (u >= nunits) break;
        const int ii = units[u].x, n = units[u].y;
        const InstDev& I = a.inst[ii];
        coarse_step<D2>(a, ii, n, Uk + I.oU, cv);
        for (int k = threadIdx.x; k < I.K; k += NT) Gold[I.oPK + (size_t)n * I.K + k] = cv.nxt[k];
    }
}

// G_old(n), n >= nfirst, recomputed in the coarse-step mode of this iteration for
// every active instance whose stored values were taken in the other mode (the
// iteration switches between the FP32 and the refined G).  Each iteration of
// Eq. Parareal then uses one G at both of its call sites, G_n(U^{k+1}_{0:n})
// and G_n(U^k_{0:n}); the convergence result holds for any G, so the fixed
// point is the same.  Grid-stride over the units: iterations without a switch
// (nearly all) only read the flags.
template <bool D2>
__global__ void __launch_bounds__(NT, D2 ? 1 : 2)
k_coarse_regold(PathArgs a, const double* Uk, double* Gold, const int2* units, int nunits, const int* nfirst,
                const int* active)
{
    extern __shared__ __align__(16) char smem_raw[];
    Carve cv = carve<D2>(a, smem_raw);
    for (int u = blockIdx.x; u < nunits; u += gridDim.x) {
        const int ii = units[u].x, n = units[u].y;
        if (!active[ii] || n < nfirst[ii]) continue;
        const bool want = inexact_iteration(a, ii, nfirst[ii]);
        if ((a.gmode[ii] != 0) == want) continue;
        const InstDev& I = a.inst[ii];
        coarse_step<D2>(a, ii, n, Uk + I.oU, cv, want);
        for (int k = threadIdx.x; k < I.K; k += NT) Gold[I.oPK + (size_t)n * I.K + k] = cv.nxt[k];
        __syncthreads();
    }
}

// One CTA per instance; 2D with a.split2d > 1: one cluster of a.split2d CTAs
// per instance, which share every step (Split) and run everything else
// redundantly -- each writes the same values to U, G_old and the increment.
template <bool D2>
__global__ void __launch_bounds__(NT, D2 ? 1 : 2)
k_coarse_sweep(PathArgs a, const double* u0, const double* Uold, double* Unew, const double* Fv, double* Gold,
               int init, const int* nfirst, const int* active, double* incr)
{
    extern __shared__ __align__(16) char smem_raw[];
    Carve cv = carve<D2>(a, smem_raw);
    __shared__ double red[NT / 32];
    __shared__ double s_num, s_den;
    const int csize = (D2 && a.split2d > 1) ? a.split2d : 1;
    // the longest chains first: the first CTAs to start get an SM each, the rest share
    const int ii = a.sweep_order ? a.sweep_order[blockIdx.x / csize] : blockIdx.x / csize, tid = threadIdx.x;
    if (csize > 1) {
        cv.sp.size = csize;
        cv.sp.rank = (int)cooperative_groups::this_cluster().block_rank();
        // every CTA of the cluster is running before any writes into another's
        // shared memory
        cooperative_groups::this_cluster().sync();
    }
    const InstDev& I = a.inst[ii];
    const int K = I.K, P = I.P;
    double* U = Unew + I.oU;
    if (!init && !active[ii]) {   // converged: carry the iterate into the other buffer
        for (int e = tid; e < (P + 1) * K; e += NT) U[e] = Uold[I.oU + e];
        return;
    }
    int n0 = 0;
    if (init) {
        for (int k = tid; k < K; k += NT) U[k] = u0[I.oK + k];
    } else {
        n0 = nfirst[ii];
        for (int e = tid; e < (n0 + 1) * K; e += NT) U[e] = Uold[I.oU + e];
    }
    // the coarse-step mode of this sweep; G_old is stored in it (k_coarse_regold
    // has brought the values this sweep reads into the same mode)
    const bool g32 = inexact_iteration(a, ii, n0);
    if (tid == 0 && a.gmode) a.gmode[ii] = g32;
    __syncthreads();
    double* Go = Gold + I.oPK;
    const double* Fo = Fv + I.oPK;
    // the correction F_old(n) - G_old(n) is read before the coarse step and G_old(n)
    // written after it: in a cluster-split sweep every CTA writes G_old(n), and the
    // cluster barriers inside the step order all reads of the old value before any
    // write of the new one (each thread keeps its own k, so no block barrier is needed)
    double* corr = a.corr + (size_t)blockIdx.x * a.Kmax;
    // FP32-pipe paths: the coarse differences U_{i+1} - U_i as double-float rows in the
    // CTA's slot, rows < n0 now and one more row per step (not n rows per step)
    df* dud = a.prec != 0 ? a.dud + (size_t)blockIdx.x * a.dud_stride : nullptr;
    if (dud) {
        for (int e = tid; e < n0 * K; e += NT) dud[e] = df_from_double(U[e + K] - U[e]);
        __syncthreads();
    }
    for (int n = n0; n < P; ++n) {
        if (dud && n > n0) {
            for (int k = tid; k < K; k += NT)
                dud[(size_t)(n - 1) * K + k] = df_from_double(U[(size_t)n * K + k] - U[(size_t)(n - 1) * K + k]);
            __syncthreads();
        }
        if (!init)
            for (int k = tid; k < K; k += NT) corr[k] = Fo[(size_t)n * K + k] - Go[(size_t)n * K + k];
        coarse_step<D2>(a, ii, n, U, cv, g32, dud != nullptr);
        for (int k = tid; k < K; k += NT) {
            double g = cv.nxt[k];
            size_t e = (size_t)n * K + k;
            U[(size_t)(n + 1) * K + k] = init ? g : g + corr[k];
            Go[e] = g;
        }
        __syncthreads();
    }
    if (init) {
        if (csize > 1) cooperative_groups::this_cluster().sync();   // see the end of the kernel
        return;
    }
    // e_k = max_n ||U^{k+1}_n - U^k_n|| / max_n ||U^{k+1}_n||
    if (tid == 0) {
        s_num = 0.0;
        s_den = 0.0;
    }
    const double* Uo = Uold + I.oU;
    for (int n = 0; n <= P; ++n) {
        double sd = 0.0, sn = 0.0;
        for (int k = tid; k < K; k += NT) {
            double x = U[(size_t)n * K + k], d = x - Uo[(size_t)n * K + k];
            sd += d * d;
            sn += x * x;
        }
        for (int o = 16; o > 0; o >>= 1) {
            sd += __shfl_xor_sync(0xffffffffu, sd, o);
            sn += __shfl_xor_sync(0xffffffffu, sn, o);
        }
        __syncthreads();
        if ((tid & 31) == 0) red[tid >> 5] = sd;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < NT / 32; ++w) t += red[w];
            s_num = fmax(s_num, sqrt(t));
        }
        __syncthreads();
        if ((tid & 31) == 0) red[tid >> 5] = sn;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < NT / 32; ++w) t += red[w];
            s_den = fmax(s_den, sqrt(t));
        }
    }
    __syncthreads();
    if (tid == 0) incr[ii] = s_den > 0.0 ? s_num / s_den : s_num;
    // no CTA leaves while another may still read its shared memory
    if (csize > 1) cooperative_groups::this_cluster().sync();
}

template <bool D2>
__global__ void __launch_bounds__(NT, D2 ? 1 : 2)
k_serial_hyb(PathArgs a, const double* u0, double* Us)
{
    extern __shared__ __align__(16) char smem_raw[];
    Carve cv = carve<D2>(a, smem_raw);
    const int ii = a.serial_order ? a.serial_order[blockIdx.x] : blockIdx.x;   // the longest chains first
    const InstDev& I = a.inst[ii];
    double* U = Us + I.oU;
    double* ring = a.ring + (size_t)blockIdx.x * a.ring_stride;
    for (int k = threadIdx.x; k < I.K; k += NT) U[k] = u0[I.oK + k];
    __syncthreads();
    // FP32-pipe paths: one more row of coarse differences per slice (not n rows)
    df* dud = a.prec != 0 ? a.dud + (size_t)blockIdx.x * a.dud_stride : nullptr;
    for (int n = 0; n < I.P; ++n) {
        if (dud && n > 0) {
            for (int k = threadIdx.x; k < I.K; k += NT)
                dud[(size_t)(n - 1) * I.K + k] =
                    df_from_double(U[(size_t)n * I.K + k] - U[(size_t)(n - 1) * I.K + k]);
            __syncthreads();
        }
        fine_slice<D2>(a, ii, n, U, nullptr, U + (size_t)(n + 1) * I.K, cv, ring, false, fine_grid(a, I),
                       dud != nullptr);
    }
}

__global__ void k_uni_init(const InstDev* inst, const double* u0, double* Wcur, double* Us)
{
    const InstDev& I = inst[blockIdx.x];
    for (int k = threadIdx.x; k < I.K; k += blockDim.x) {
        Wcur[I.oK + k] = u0[I.oK + k];
        Us[I.oU + k] = u0[I.oK + k];
    }
}

// Partial history sums of the uniform scheme at step j (computing W_{j+1}):
//   part[c][k] = sum_{l in chunk c} b_{j-l} dW_l[k],  dW_l = W_{l+1} - W_l.
// Reads each history row once per step; coalesced along modes.
// DF: the FP32-pipe paths store the fine differences as double-float and sum
// them in double-float (the FP64 pipe would bound the stream); FP64 path in FP64.
// Each thread keeps eight rows in flight (four partial sums) so that the stream
// is bound by HBM, not by one load at a time.
template <bool DF>
__global__ void __launch_bounds__(NT) k_uni_hist(const InstDev* inst, const double* bp, const df* bpd,
                                                 const double* dW, int j, double* part, int chunk, int maxchunks,
                                                 int Kmax)
{
    const int ii = blockIdx.y, c = blockIdx.x;
    const InstDev& I = inst[ii];
    if (j >= I.N) return;
    const int l0 = c * chunk;
    if (l0 >= j) return;
    const int l1 = min(j, l0 + chunk);
    const size_t K = I.K;
    double* out = part + ((size_t)ii * maxchunks + c) * Kmax;
    for (int k = threadIdx.x; k < I.K; k += NT) {
        if constexpr (DF) {
            const df* w = bpd + I.oB;
            const df* h = reinterpret_cast<const df*>(dW + I.oW) + k;
            dfacc a0{0.f, 0.f}, a1{0.f, 0.f}, a2{0.f, 0.f}, a3{0.f, 0.f};
            int l = l0;
            for (; l + 8 <= l1; l += 8) {
                df v[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) v[q] = h[(size_t)(l + q) * K];
                dfacc_fma(a0, w[j - l], v[0]);
                dfacc_fma(a1, w[j - l - 1], v[1]);
                dfacc_fma(a2, w[j - l - 2], v[2]);
                dfacc_fma(a3, w[j - l - 3], v[3]);
                dfacc_fma(a0, w[j - l - 4], v[4]);
                dfacc_fma(a1, w[j - l - 5], v[5]);
                dfacc_fma(a2, w[j - l - 6], v[6]);
                dfacc_fma(a3, w[j - l - 7], v[7]);
            }
            for (; l < l1; ++l) dfacc_fma(a0, w[j - l], h[(size_t)l * K]);
            dfacc_add(a0, dfacc_result(a1));
            dfacc_add(a2, dfacc_result(a3));
            dfacc_add(a0, dfacc_result(a2));
            out[k] = df_to_double(dfacc_result(a0));
        } else {
            const double* bF = bp + I.oB;
            const double* h = dW + I.oW + k;
            double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
            int l = l0;
            for (; l + 8 <= l1; l += 8) {
                double v[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) v[q] = h[(size_t)(l + q) * K];
                a0 = fma(bF[j - l], v[0], a0);
                a1 = fma(bF[j - l - 1], v[1], a1);
                a2 = fma(bF[j - l - 2], v[2], a2);
                a3 = fma(bF[j - l - 3], v[3], a3);
                a0 = fma(bF[j - l - 4], v[4], a0);
                a1 = fma(bF[j - l - 5], v[5], a1);
                a2 = fma(bF[j - l - 6], v[6], a2);
                a3 = fma(bF[j - l - 7], v[7], a3);
            }
            for (; l < l1; ++l) a0 = fma(bF[j - l], h[(size_t)l * K], a0);
            out[k] = (a0 + a1) + (a2 + a3);
        }
    }
}

template <bool D2>
__global__ void __launch_bounds__(NT, D2 ? 1 : 2)
k_uni_step(PathArgs a, double* Wcur, double* dW, double* Us, int j, const double* part, int chunk, int maxchunks)
{
    extern __shared__ __align__(16) char smem_raw[];
    Carve cv = carve<D2>(a, smem_raw);
    const int ii = blockIdx.x, tid = threadIdx.x;
    const InstDev& I = a.inst[ii];
    if (j >= I.N) return;
    const int K = I.K;
    const int nch = (j + chunk - 1) / chunk;
    for (int k = tid; k < K; k += NT) {
        double c = Wcur[I.oK + k], h = c;
        for (int q = 0; q < nch; ++q) h -= part[((size_t)ii * maxchunks + q) * a.Kmax + k];
        cv.cur[k] = c;
        cv.hist[k] = h;
    }
    __syncthreads();
    int bad = do_step<D2>(a, I, cv.cur, cv.hist, I.dt * j, I.mu, cv.nxt, cv);
    if (bad >= 0 && tid == 0) report(a.status, -2, ii, WHERE_UNI, j);
    check_finite(a, cv.nxt, K, ii, WHERE_UNI, j);
    const bool node = ((j + 1) % I.m) == 0;
    for (int k = tid; k < K; k += NT) {
        double x = cv.nxt[k];
        if (a.prec == 0)
            dW[I.oW + (size_t)j * K + k] = x - cv.cur[k];
        else   // double-float differences for the FP32-pipe history sums
            reinterpret_cast<df*>(dW + I.oW)[(size_t)j * K + k] = df_from_double(x - cv.cur[k]);
        Wcur[I.oK + k] = x;
        if (node) Us[I.oU + (size_t)((j + 1) / I.m) * K + k] = x;
    }
}

// One step j of the uniform scheme with the fast history (psl1_soe.cu): the
// weights b(j - l) of the last nloc - 1 differences are exact, the older ones
// are sums of exponentials, carried as the state
//   Y_i(j) = sum_{l <= j - nloc} exp(-s_i (j - l)) dW_l,
//   Y_i(j) = exp(-s_i) Y_i(j-1) + exp(-s_i nloc) dW_{j - nloc}   (updated here),
// so that hist = W_j - sum_{j-l < nloc} b(j-l) dW_l - sum_i w_i Y_i(j).  The state
// and its update are FP64 (L x K per instance, L2-resident); each step costs
// O((nloc + L) K) instead of O(j K).
template <bool D2>
__global__ void __launch_bounds__(NT, D2 ? 1 : 2)
k_uni_soe_step(PathArgs a, double* Wcur, double* dW, double* Us, int j, const double* soe, double* Y, int nloc)
{
    extern __shared__ __align__(16) char smem_raw[];
    Carve cv = carve<D2>(a, smem_raw);
    const int ii = blockIdx.x, tid = threadIdx.x;
    const InstDev& I = a.inst[ii];
    if (j >= I.N) return;
    const int K = I.K, L = I.soeL;
    const double* bF = a.bp + I.oB;
    const double* dec = soe + I.oS;
    const double* inj = dec + L;
    const double* w = inj + L;
    double* Yb = Y + I.oY;
    const bool dfh = a.prec != 0;   // FP32-pipe paths store the differences as double-float pairs
    const double* dWb = dW + I.oW;
    auto diff = [&](int l, int k) -> double {
        return dfh ? df_to_double(reinterpret_cast<const df*>(dWb)[(size_t)l * K + k]) : dWb[(size_t)l * K + k];
    };
    const int l0 = j - nloc + 1 > 0 ? j - nloc + 1 : 0;
    for (int k = tid; k < K; k += NT) {
        const double c = Wcur[I.oK + k];
        double h = c;
        for (int l = l0; l < j; ++l) h -= bF[j - l] * diff(l, k);
        if (j >= nloc && L > 0) {
            const double d = diff(j - nloc, k);
            double acc0 = 0.0, acc1 = 0.0;
            int i = 0;
            for (; i + 1 < L; i += 2) {
                const double y0 = fma(dec[i], Yb[(size_t)i * K + k], inj[i] * d);
                const double y1 = fma(dec[i + 1], Yb[(size_t)(i + 1) * K + k], inj[i + 1] * d);
                Yb[(size_t)i * K + k] = y0;
                Yb[(size_t)(i + 1) * K + k] = y1;
                acc0 = fma(w[i], y0, acc0);
                acc1 = fma(w[i + 1], y1, acc1);
            }
            if (i < L) {
                const double y0 = fma(dec[i], Yb[(size_t)i * K + k], inj[i] * d);
                Yb[(size_t)i * K + k] = y0;
                acc0 = fma(w[i], y0, acc0);
            }
            h -= acc0 + acc1;
        }
        cv.cur[k] = c;
        cv.hist[k] = h;
    }
    if (tid == 0 && a.flops) atomicAdd(a.flops + a.flop_slot, 2.0 * K * ((j - l0) + (j >= nloc ? 2.0 * L : 0.0)));
    __syncthreads();
    int bad = do_step<D2>(a, I, cv.cur, cv.hist, I.dt * j, I.mu, cv.nxt, cv);
    if (bad >= 0 && tid == 0) report(a.status, -2, ii, WHERE_UNI, j);
    check_finite(a, cv.nxt, K, ii, WHERE_UNI, j);
    const bool node = ((j + 1) % I.m) == 0;
    for (int k = tid; k < K; k += NT) {
        const double x = cv.nxt[k];
        if (dfh)
            reinterpret_cast<df*>(dW + I.oW)[(size_t)j * K + k] = df_from_double(x - cv.cur[k]);
        else
            dW[I.oW + (size_t)j * K + k] = x - cv.cur[k];
        Wcur[I.oK + k] = x;
        if (node) Us[I.oU + (size_t)((j + 1) / I.m) * K + k] = x;
    }
}

template <bool D2>
__global__ void __launch_bounds__(NT, D2 ? 1 : 2)
k_one_step(PathArgs a, int ii, const double* c, const double* hist, double te, double mu, double* out)
{
    extern __shared__ __align__(16) char smem_raw[];
    Carve cv = carve<D2>(a, smem_raw);
    const InstDev& I = a.inst[ii];
    for (int k = threadIdx.x; k < I.K; k += NT) {
        cv.cur[k] = c[k];
        cv.hist[k] = hist[k];
    }
    __syncthreads();
    int bad = do_step<D2>(a, I, cv.cur, cv.hist, te, mu, cv.nxt, cv);
    if (bad >= 0 && threadIdx.x == 0) report(a.status, -2, ii, WHERE_ONE, bad);
    check_finite(a, cv.nxt, I.K, ii, WHERE_ONE, 0);
    for (int k = threadIdx.x; k < I.K; k += NT) out[k] = cv.nxt[k];
}

template <bool D2>
__global__ void __launch_bounds__(NT, D2 ? 1 : 2)
k_one_slice(PathArgs a, int ii, int n, const double* U, double* V)
{
    extern __shared__ __align__(16) char smem_raw[];
    Carve cv = carve<D2>(a, smem_raw);
    const InstDev& I = a.inst[ii];
    fine_slice<D2>(a, ii, n, U, V, V + (size_t)I.m * I.K, cv, a.ring, false, fine_grid(a, I));
}

template <bool D2>
__global__ void __launch_bounds__(NT, D2 ? 1 : 2)
k_one_coarse(PathArgs a, int ii, int n, const double* U, double* out)
{
    extern __shared__ __align__(16) char smem_raw[];
    Carve cv = carve<D2>(a, smem_raw);
    const InstDev& I = a.inst[ii];
    coarse_step<D2>(a, ii, n, U, cv);
    for (int k = threadIdx.x; k < I.K; k += NT) out[k] = cv.nxt[k];
}

__global__ void k_pr_update(const double* incr, int* active, int* nfirst, int* iters, double* errlog, int* counter,
                            int* kstate, const double* tol, cudaGraphConditionalHandle cond, int B, int P)
{
    __shared__ int s_act;
    if (threadIdx.x == 0) s_act = 0;
    __syncthreads();
    const int k = kstate[0];
    for (int b = threadIdx.x; b < B; b += blockDim.x) {
        if (active[b]) {
            errlog[(size_t)b * P + k] = incr[b];
            iters[b] = k + 1;
            if (incr[b] <= *tol)
                active[b] = 0;
            else
                atomicAdd(&s_act, 1);
        }
        nfirst[b] = k + 1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        kstate[0] = k + 1;
        *counter = 0;
        cudaGraphSetConditional(cond, (s_act > 0 && k + 1 < kstate[1]) ? 1u : 0u);
    }
}

cudaError_t launch_pr_update(const double* incr, int* active, int* nfirst, int* iters, double* errlog, int* counter,
                             int* kstate, const double* tol, cudaGraphConditionalHandle cond, int B, int P,
                             cudaStream_t s)
{
    k_pr_update<<<1, 256, 0, s>>>(incr, active, nfirst, iters, errlog, counter, kstate, tol, cond, B, P);
    return cudaGetLastError();
}

static PathArgs slot(const PathArgs& a, int s)
{
    PathArgs b = a;
    b.flop_slot = s;
    return b;
}

template <typename... KA, typename... Args>
static cudaError_t launch_k(void (*k)(KA...), dim3 grid, size_t smem, cudaStream_t s, Args... args)
{
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, NT, smem, s>>>(args...);
    return cudaGetLastError();
}

// the 1D or the 2D instantiation of a step kernel
#define LAUNCH_STEP_KERNEL(kern, grid, smem, s, ...)                              \
    (a.dim2 ? launch_k(kern<true>, grid, smem, s, __VA_ARGS__)                    \
            : launch_k(kern<false>, grid, smem, s, __VA_ARGS__))

// ------------------------------------------------------------------ allocation-free slice
// For callers that must not allocate device memory while they run (a real-time
// loop whose memory was planned up front, or code running under an allocator
// that forbids new device allocations): the single-slice fine propagator with
// its scratch taken from this fixed array instead of the handle's per-slot
// pools.  The scratch is the fine-history ring (m K doubles), then the
// FP64 1D factor or the 2D working arrays that do not fit in shared memory,
// then the coarse differences of the FP32-pipe paths ((n+1) K double-float
// pairs); each region starts on a 256-byte boundary.  Every element of the
// scratch is written before it is read, so nothing has to be cleared between
// calls; all calls share the array, so calls that overlap on the GPU race.
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_SCRATCH_DOUBLES];

template <bool D2>
__global__ void __launch_bounds__(NT, D2 ? 1 : 2)
k_one_slice_noalloc(PathArgs a, int ii, int n, const double* U, double* V)
{
    extern __shared__ __align__(16) char smem_raw[];
    Carve cv = carve<D2>(a, smem_raw);
    const InstDev& I = a.inst[ii];
    fine_slice<D2>(a, ii, n, U, V, V + (size_t)I.m * I.K, cv, a.ring, false, fine_grid(a, I));
}

// Device address of the fixed array on the current device.  Host code cannot
// use the array's name as a device pointer (it names a host-side stand-in), so
// the address is looked up here, with the device current, and kept by the
// caller (psl1_create keeps it in the handle).  The lookup also loads this
// file's kernel module on the device, which is when the array is placed.
cudaError_t noalloc_scratch_address(double** p)
{
    void* q = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&q, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    *p = static_cast<double*>(q);
    return cudaSuccess;
}

cudaError_t launch_one_slice_noalloc(const PathArgs& a, double* scratch, int b, int n, const double* U, double* V,
                                     long long ring_doubles, long long work_doubles, long long dud_doubles,
                                     cudaStream_t s)
{
    if (!scratch) return cudaErrorInvalidDevicePointer;
    const long long ring_r = noalloc_round(ring_doubles), work_r = noalloc_round(work_doubles);
    if (ring_r + work_r + dud_doubles > NOALLOC_SCRATCH_DOUBLES) return cudaErrorInvalidValue;
    PathArgs a2 = a;
    a2.ring = scratch;
    a2.ring_stride = ring_r;
    a2.work = scratch + ring_r;
    a2.work_stride = work_r;
    a2.dud = reinterpret_cast<df*>(scratch + ring_r + work_r);
    a2.dud_stride = dud_doubles;
    a2.hc = nullptr;   // the per-step coarse-history sums: no scratch beyond the fixed array
    a2.nslots = 1;
    size_t sm = step_smem_bytes(a2);
    return a.dim2 ? launch_k(k_one_slice_noalloc<true>, 1, sm, s, a2, b, n, U, V)
                  : launch_k(k_one_slice_noalloc<false>, 1, sm, s, a2, b, n, U, V);
}

// ------------------------------------------------------------------ launchers
cudaError_t launch_fstage(const PathArgs& a, const double* Uold, double* Fv, const int2* units, int nunits,
                          int* counter, const int* nfirst, const int* active, int grid, cudaStream_t s)
{
    size_t sm = fine_smem_bytes(a);
    if (grid > a.nslots) grid = a.nslots;
    if (a.dim2)
        return launch_k(k_fstage<true, 1>, grid, sm, s, slot(a, 0), Uold, Fv, units, nunits, counter, nfirst, active);
    if (a.fstage_minb == 4)
        return launch_k(k_fstage<false, 4>, grid, sm, s, slot(a, 0), Uold, Fv, units, nunits, counter, nfirst, active);
    if (a.fstage_minb == 3)
        return launch_k(k_fstage<false, 3>, grid, sm, s, slot(a, 0), Uold, Fv, units, nunits, counter, nfirst, active);
    return launch_k(k_fstage<false, 2>, grid, sm, s, slot(a, 0), Uold, Fv, units, nunits, counter, nfirst, active);
}

// launch configuration of the cluster-split 2D sweep (B clusters of `split` CTAs)
static cudaLaunchConfig_t split_config(const PathArgs& a, int B, int split, cudaStream_t s,
                                       cudaLaunchAttribute* attr)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(B * split));
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = (size_t)a.L2s.smem;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)split;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

int coarse_sweep_clusters(const PathArgs& a, int split)
{
    if (!a.dim2 || split < 2) return 0;
    if (cudaFuncSetAttribute(k_coarse_sweep<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, a.L2s.smem) !=
        cudaSuccess)
        return 0;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = split_config(a, 1, split, nullptr, attr);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_coarse_sweep<true>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

cudaError_t launch_coarse_sweep(const PathArgs& a, int B, const double* u0, const double* Uold, double* Unew,
                                const double* Fv, double* Gold, int init, const int* nfirst,
                                const int* active, double* incr, cudaStream_t s)
{
    if (a.dim2 && a.split2d > 1) {
        PathArgs as = slot(a, 1);
        as.L2 = a.L2s;
        cudaError_t e =
            cudaFuncSetAttribute(k_coarse_sweep<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, a.L2s.smem);
        if (e != cudaSuccess) return e;
        cudaLaunchAttribute attr[1];
        cudaLaunchConfig_t cfg = split_config(a, B, a.split2d, s, attr);
        return cudaLaunchKernelEx(&cfg, k_coarse_sweep<true>, as, u0, Uold, Unew, Fv, Gold, init, nfirst, active,
                                  incr);
    }
    size_t sm = step_smem_bytes(a);
    return LAUNCH_STEP_KERNEL(k_coarse_sweep, B, sm, s, slot(a, 1), u0, Uold, Unew, Fv, Gold, init, nfirst,
                              active, incr);
}

cudaError_t launch_coarse_at(const PathArgs& a, const double* Uk, double* Gold, const int2* units, int nunits,
                             int* counter, int grid, cudaStream_t s)
{
    size_t sm = step_smem_bytes(a);
    if (grid > a.nslots) grid = a.nslots;
    return LAUNCH_STEP_KERNEL(k_coarse_at, grid, sm, s, slot(a, 1), Uk, Gold, units, nunits, counter);
}

cudaError_t launch_coarse_regold(const PathArgs& a, const double* Uk, double* Gold, const int2* units, int nunits,
                                 const int* nfirst, const int* active, int grid, cudaStream_t s)
{
    if (!a.gmode) return cudaErrorInvalidValue;
    size_t sm = step_smem_bytes(a);
    if (grid > a.nslots) grid = a.nslots;
    return LAUNCH_STEP_KERNEL(k_coarse_regold, grid, sm, s, slot(a, 1), Uk, Gold, units, nunits, nfirst, active);
}

cudaError_t launch_serial_hyb(const PathArgs& a, int B, const double* u0, double* Us, cudaStream_t s)
{
    size_t sm = fine_smem_bytes(a);
    return LAUNCH_STEP_KERNEL(k_serial_hyb, B, sm, s, slot(a, 2), u0, Us);
}

cudaError_t launch_uni_init(const PathArgs& a, int B, const double* u0, double* Wcur, double* Us, cudaStream_t s)
{
    k_uni_init<<<B, 256, 0, s>>>(a.inst, u0, Wcur, Us);
    return cudaGetLastError();
}

cudaError_t launch_uni_hist(const PathArgs& a, int B, const double* dW, int j, double* part, int chunk,
                            int maxchunks, cudaStream_t s)
{
    int nch = (j + chunk - 1) / chunk;
    if (nch <= 0) return cudaSuccess;
    dim3 grid(nch, B);
    if (a.prec == 0)
        k_uni_hist<false><<<grid, NT, 0, s>>>(a.inst, a.bp, a.bpd, dW, j, part, chunk, maxchunks, a.Kmax);
    else
        k_uni_hist<true><<<grid, NT, 0, s>>>(a.inst, a.bp, a.bpd, dW, j, part, chunk, maxchunks, a.Kmax);
    return cudaGetLastError();
}

cudaError_t launch_uni_step(const PathArgs& a, int B, double* Wcur, double* dW, double* Us, int j,
                            const double* part, int chunk, int maxchunks, cudaStream_t s)
{
    size_t sm = step_smem_bytes(a);
    return LAUNCH_STEP_KERNEL(k_uni_step, B, sm, s, slot(a, 2), Wcur, dW, Us, j, part, chunk, maxchunks);
}

cudaError_t launch_uni_soe_step(const PathArgs& a, int B, double* Wcur, double* dW, double* Us, int j,
                                const double* soe, double* Y, int nloc, cudaStream_t s)
{
    size_t sm = step_smem_bytes(a);
    return LAUNCH_STEP_KERNEL(k_uni_soe_step, B, sm, s, slot(a, 2), Wcur, dW, Us, j, soe, Y, nloc);
}

cudaError_t launch_one_step(const PathArgs& a, int b, const double* c, const double* hist, double te, double mu,
                            double* out, cudaStream_t s)
{
    size_t sm = step_smem_bytes(a);
    return LAUNCH_STEP_KERNEL(k_one_step, 1, sm, s, slot(a, 3), b, c, hist, te, mu, out);
}

cudaError_t launch_one_slice(const PathArgs& a, int b, int n, const double* U, double* V, cudaStream_t s)
{
    size_t sm = step_smem_bytes(a);
    return LAUNCH_STEP_KERNEL(k_one_slice, 1, sm, s, slot(a, 3), b, n, U, V);
}

cudaError_t launch_coarse_dataset(const PathArgs& a, const double* Us, const int2* units, int nunits, int* counter,
                                  float* Z, float* R, int grid, cudaStream_t s)
{
    size_t sm = step_smem_bytes(a);
    if (grid > a.nslots) grid = a.nslots;
    return launch_k(k_coarse_dataset, grid, sm, s, slot(a, 3), Us, units, nunits, counter, Z, R);
}

cudaError_t launch_one_coarse(const PathArgs& a, int b, int n, const double* U, double* out, cudaStream_t s)
{
    size_t sm = step_smem_bytes(a);
    return LAUNCH_STEP_KERNEL(k_one_coarse, 1, sm, s, slot(a, 3), b, n, U, out);
}

}  // namespace psl1
