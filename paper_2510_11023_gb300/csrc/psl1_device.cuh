// psl1_device.cuh -- device-side descriptors and helpers of the GB300 solver.
//
// Layout in HBM (all pools are flat device arrays; every instance owns a
// contiguous range given by the offsets in InstDev):
//   u0, iterates U^k and U^{k+1}, serial result : (P+1) x K per instance
//   F_old (slice-end fine states), G_old       : P x K per instance
//   L1 weight table                            : b(j), j = 0..Nb, then
//                                                m^-a b(d + r/m), d < P, 1 <= r <= m
//   quadrature / basis tables (shared by instances with the same Mx, Qx, box)
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace psl1 {

constexpr int NT = 256;          // threads per CTA of the step kernels
constexpr int KMAX_1D = 512;     // largest 1D mode count handled by one CTA
constexpr int MMAX_2D = 64;      // largest 2D mode count per axis (K = Mx My <= 4096)
constexpr int TILE = 32;         // Cholesky block size (one warp per panel)
constexpr int CHEB_NMAX = 64;    // most collocation intervals (the step's shared-memory LU system)
constexpr float INNER_RTOL_DEFAULT = 1e-7f;   // FP32 inner CG tolerance of the refined mixed step (tunable)

// elements of a block-packed lower triangle of nb x nb blocks with row stride ldb
__host__ __device__ constexpr int bp_elems(int nb, int ldb) { return nb * (nb + 1) / 2 * TILE * ldb; }

struct InstDev {
    int dim, K, Kp, nb;          // modes, padded to a multiple of TILE, blocks
    int Mx, My, Q, Qh;           // x axis: Q nodes, Qh = Q/2 mirror pairs
    int N, m, P, tab;            // tab: x-axis table set
    double alpha, T, dT, dt;
    double mu, muT, ma;          // dt^a G(2-a), dT^a G(2-a), m^-a
    double cA;                   // pi^2 / L^3 : A_kl = cA k l (g_|k-l| + g_k+l)
    double lo0, hi0, lo1, hi1;
    double g1a, g3a;             // Gamma(1+a), Gamma(3-a) (manufactured sources)
    double dpar[8], fpar[8];
    long long oK;                // offset in K-vectors (u0)
    long long oU;                // offset in (P+1)K node arrays
    long long oPK;               // offset in P*K arrays
    long long oB;                // offset in the weight pool
    long long oW;                // offset in N*K fine-history pools (uniform solver)
    int Nb;                      // b(j) table length - 1 (max of N, P, m)
    int Qy, Qhy, tabY;           // y axis (2D): nodes, mirror pairs, table set
    int f_df;                    // f has no manufactured source term (double-float evaluation)
    float dpf[16], fpf[16];      // dpar, fpar as double-float pairs (hi, lo)
    int soeL;                    // exponentials of the fast uniform history (0: none)
    long long oS;                // offset in the exponential pool: exp(-s) [L], exp(-s nloc) [L], w [L]
    long long oY;                // offset in the exponential-state pool (L x K)
    int basis;                   // 0 sine Galerkin, 1 Chebyshev-Lobatto collocation (Mx intervals, K = Mx - 1)
    long long oC;                // collocation: offset in the collocation pool (nodes, sines, Dm)
    float inner_rtol;            // relative residual of the FP32 inner CG in the refined mixed step
    int mc;                      // coarse propagator substeps (1: the one-step L1 G)
    double dtc, muc;             // substep size dT/mc and its mu
    long long oBc;               // offset of mc^-a b(d + r/mc), d < P, r <= mc, in the substep weight pool
};

struct TabDev {
    int Mx, Qx, Qh, pad_;
    long long oX;    // Qh half-node abscissae x_q (x_q < midpoint)
    long long oWq;   // Qh weights
    long long oAux;  // 4*Qh: sin(pi x), sin(2 pi x) at x_q and at the mirror node
    long long oSt;   // Mx x Qh : phi_k(x_q)      (row k, coalesced over q)
    long long oS;    // Qh x Mx : phi_k(x_q)      (row q, coalesced over k)
    long long oC;    // Qh x (2Mx+1) : cos(s pi (x_q - lo)/L)
    long long oStd, oSd, oCd;   // the same three tables as double-float pairs
    long long oDt;   // Mx x Qh : phi_k'(x_q)    (row k)
    long long oDtd;  // the same as double-float pairs
    long long oSt32, oDt32;   // Mx x Qh FP32 copies of St and Dt (two floats per slot)
    long long oAux2; // 2*Qh: cos(2 pi x) at x_q and at the mirror node
    long long oWd, oAuxd, oAux2d;   // Qh weights, 4*Qh aux, 2*Qh aux2 as double-float pairs
    long long oS32, oC32;   // FP32 copies of S (Qh x Mx) and C (Qh x (2Mx+1)), packed floats
};

// Device error word: the first failure wins.  code < 0 is a psl1_status.
struct DevStatus {
    int code;
    int inst;
    int where;
    int info;
};

__device__ __forceinline__ void report(DevStatus* st, int code, int inst, int where, int info)
{
    if (atomicCAS(&st->code, 0, code) == 0) {
        st->inst = inst;
        st->where = where;
        st->info = info;
    }
}

// ------------------------------------------------------------------------
// Double-float (unevaluated FP32 pair) arithmetic.  Knuth's TwoSum and the
// FMA-based exact product give ~48-bit significands on the FP32 pipes,
// which GB300 runs 62x faster than FP64 (1.2 vs 74.7 TFLOP/s measured).
// ------------------------------------------------------------------------
struct df {
    float hi, lo;
};

__device__ __forceinline__ df df_from_double(double x)
{
    float h = __double2float_rn(x);
    float l = __double2float_rn(x - (double)h);
    return {h, l};
}

__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

// s + e = a + b exactly
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// accumulator (hi, lo) += a * b, a and b double-float; lo is renormalised lazily
struct dfacc {
    float hi, lo;
};

__device__ __forceinline__ void dfacc_fma(dfacc& acc, df a, df b)
{
    float p = __fmul_rn(a.hi, b.hi);
    float pe = __fmaf_rn(a.hi, b.hi, -p);                       // exact product error
    float cross = __fmaf_rn(a.hi, b.lo, __fmul_rn(a.lo, b.hi));
    float s, e;
    two_sum(acc.hi, p, s, e);
    acc.hi = s;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(e, __fadd_rn(pe, cross)));
}

__device__ __forceinline__ df dfacc_result(dfacc acc)
{
    float s = __fadd_rn(acc.hi, acc.lo);
    float e = __fsub_rn(acc.lo, __fsub_rn(s, acc.hi));
    return {s, e};
}

}  // namespace psl1
