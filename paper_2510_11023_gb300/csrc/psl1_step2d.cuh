// psl1_step2d.cuh -- one linearised L1 step of the 2D tensor-product
// sine-Galerkin scheme on a box, executed by one CTA of NT threads:
//
//   (I + mu A(D(t_e, c))) c_new = hist + mu F(f(t_e, c))      (Eq. NumericalSchemeFine /
//                                                              NumericalSchemeSequential)
//
// Basis phi_kl(x, y) = phi_k(x) phi_l(y) (orthonormal: identity mass),
// coefficients c[k][l] row-major with the y mode fastest, tensor Gauss-Legendre
// nodes (x_i, y_j) with weights w_ij = wx_i wy_j.  No matrix is assembled: with
// W = w o D at the nodes,
//   (A v)_kl = sum_ij W_ij [ phi_k'(x_i) phi_l(y_j) (dx v)_ij + phi_k(x_i) phi_l'(y_j) (dy v)_ij ]
//   (dx v)_ij = sum_kl v_kl phi_k'(x_i) phi_l(y_j),   (dy v)_ij = sum_kl v_kl phi_k(x_i) phi_l'(y_j)
// (Eq. AForm with the quadrature of the weak form), which is four one-axis
// transforms (modes -> nodes along y, then x; back along x, then y): O(M^2 Q)
// operations per application instead of O(M^4 Q^2) for the assembled matrix.
// Gauss nodes are symmetric about the midpoint and, for mode k = 1..M,
// phi_k(x') = (-1)^(k+1) phi_k(x), phi_k'(x') = (-1)^k phi_k'(x), so every
// one-axis transform runs over Q/2 mirror pairs with even/odd mode splitting.
//
// Solve: conjugate gradients on I + mu A, preconditioned by its exact diagonal
// (two squared-table transforms of W).  FP64 path: CG in FP64 to a relative
// residual of 1e-14.  Mixed path: CG in FP32 as the inner solver of an iterative
// refinement whose residual rhs - (I + mu A) x is evaluated in double-float.
#pragma once
#include <cooperative_groups.h>
#include "psl1_step.cuh"
#include "psl1_step_mixed.cuh"
#include "psl1_dfmath.cuh"

namespace psl1 {

// ------------------------------------------------------------------ number policies
struct NumF {
    using V = float;
    using A = float;
    __device__ static A zero() { return 0.f; }
    __device__ static void mac(A& a, V x, V y) { a = fmaf(x, y, a); }
    __device__ static V res(A a) { return a; }
    __device__ static V add(V a, V b) { return a + b; }
    __device__ static V sub(V a, V b) { return a - b; }
    __device__ static V mul(V a, V b) { return a * b; }
    __device__ static V neg(V a) { return -a; }
};

struct NumD {
    using V = double;
    using A = double;
    __device__ static A zero() { return 0.0; }
    __device__ static void mac(A& a, V x, V y) { a = fma(x, y, a); }
    __device__ static V res(A a) { return a; }
    __device__ static V add(V a, V b) { return a + b; }
    __device__ static V sub(V a, V b) { return a - b; }
    __device__ static V mul(V a, V b) { return a * b; }
    __device__ static V neg(V a) { return -a; }
};

struct NumDF {
    using V = df;
    using A = dfacc;
    __device__ static A zero() { return {0.f, 0.f}; }
    __device__ static void mac(A& a, V x, V y) { dfacc_fma(a, x, y); }
    __device__ static V res(A a) { return dfacc_result(a); }
    __device__ static V add(V a, V b) { return df_add(a, b); }
    __device__ static V sub(V a, V b) { return df_add(a, df_neg(b)); }
    __device__ static V mul(V a, V b) { return df_mul(a, b); }
    __device__ static V neg(V a) { return df_neg(a); }
};

// Table kinds of a one-axis transform: basis values or derivatives (mirror
// signs differ), or their squares (backward only: Jacobi diagonal).
enum { TV = 0, TD = 1, TV2 = 2, TD2 = 3 };

template <class Nm>
struct AxisOp {
    const typename Nm::V* in;
    const typename Nm::V* tab;   // M x Qh, row = mode, contiguous over node pairs
    typename Nm::V* out;
    int kind;
};

// Modes -> nodes along one axis for `rows` independent rows and up to two
// components:  out(r, q) = E + O,  out(r, Q-1-q) = +-(E - O),  q < Qh, with
// E, O the even- and odd-mode partial sums of in(r, c) tab(c, q).  The table
// rows are ts apart (ts = the axis' node-pair count; Qh may cover a sub-range
// of its pairs, with tab pointing at the first of them and Q = 2 Qh the local
// width of the output rows).
//   in(r, c)  = in[r * irs + c * ics],  out(r, j) = out[r * ors + j * ojs]
// and, if w is given, the result is multiplied by w(r, j) (strides of out).
// RFAST: consecutive threads take consecutive rows (else consecutive pairs).
template <class Nm, int RT, int QT, bool RFAST>
__device__ void axis_fwd(int ncomp, AxisOp<Nm> o0, AxisOp<Nm> o1, int rows, int M, int Qh, int ts, int irs,
                         int ics, int ors, int ojs, const typename Nm::V* w)
{
    using V = typename Nm::V;
    using A = typename Nm::A;
    const int nr = (rows + RT - 1) / RT, nq = (Qh + QT - 1) / QT, tiles = nr * nq, Q = 2 * Qh;
    for (int it = threadIdx.x; it < ncomp * tiles; it += NT) {
        const int comp = it / tiles, t = it - comp * tiles;
        const AxisOp<Nm> o = comp ? o1 : o0;
        const int tr = RFAST ? t % nr : t / nq, tq = RFAST ? t / nr : t % nq;
        int r[RT], q[QT];
#pragma unroll
        for (int c = 0; c < RT; ++c) r[c] = RFAST ? tr + c * nr : tr * RT + c;
#pragma unroll
        for (int d = 0; d < QT; ++d) q[d] = RFAST ? tq * QT + d : tq + d * nq;
        const V* ip[RT];
        const V* tp[QT];
#pragma unroll
        for (int c = 0; c < RT; ++c) ip[c] = o.in + (size_t)(r[c] < rows ? r[c] : rows - 1) * irs;
#pragma unroll
        for (int d = 0; d < QT; ++d) tp[d] = o.tab + (q[d] < Qh ? q[d] : Qh - 1);
        A E[RT][QT], O[RT][QT];
#pragma unroll
        for (int c = 0; c < RT; ++c)
#pragma unroll
            for (int d = 0; d < QT; ++d) {
                E[c][d] = Nm::zero();
                O[c][d] = Nm::zero();
            }
        int k = 0;
        for (; k + 1 < M; k += 2) {
            V a[RT], b[QT];
#pragma unroll
            for (int c = 0; c < RT; ++c) a[c] = ip[c][(size_t)k * ics];
#pragma unroll
            for (int d = 0; d < QT; ++d) b[d] = tp[d][(size_t)k * ts];
#pragma unroll
            for (int c = 0; c < RT; ++c)
#pragma unroll
                for (int d = 0; d < QT; ++d) Nm::mac(E[c][d], a[c], b[d]);
#pragma unroll
            for (int c = 0; c < RT; ++c) a[c] = ip[c][(size_t)(k + 1) * ics];
#pragma unroll
            for (int d = 0; d < QT; ++d) b[d] = tp[d][(size_t)(k + 1) * ts];
#pragma unroll
            for (int c = 0; c < RT; ++c)
#pragma unroll
                for (int d = 0; d < QT; ++d) Nm::mac(O[c][d], a[c], b[d]);
        }
        if (k < M) {
            V a[RT], b[QT];
#pragma unroll
            for (int c = 0; c < RT; ++c) a[c] = ip[c][(size_t)k * ics];
#pragma unroll
            for (int d = 0; d < QT; ++d) b[d] = tp[d][(size_t)k * ts];
#pragma unroll
            for (int c = 0; c < RT; ++c)
#pragma unroll
                for (int d = 0; d < QT; ++d) Nm::mac(E[c][d], a[c], b[d]);
        }
#pragma unroll
        for (int c = 0; c < RT; ++c)
#pragma unroll
            for (int d = 0; d < QT; ++d) {
                if (r[c] >= rows || q[d] >= Qh) continue;
                V e = Nm::res(E[c][d]), od = Nm::res(O[c][d]);
                V v1 = Nm::add(e, od), v2 = Nm::sub(e, od);
                if (o.kind == TD) v2 = Nm::neg(v2);
                const size_t i1 = (size_t)r[c] * ors + (size_t)q[d] * ojs;
                const size_t i2 = (size_t)r[c] * ors + (size_t)(Q - 1 - q[d]) * ojs;
                if (w) {
                    v1 = Nm::mul(v1, w[i1]);
                    v2 = Nm::mul(v2, w[i2]);
                }
                o.out[i1] = v1;
                o.out[i2] = v2;
            }
    }
}

// Nodes -> modes along one axis:  out(r, c) = sum_{q < Qh} tab(c, q) (in(r, q) + s_c in(r, Q-1-q))
// with s_c = (-1)^c for values, -(-1)^c for derivatives (c = 0-based mode),
// +1 for squared tables (whose entries are squared on the fly).  Table rows
// are ts apart; Qh may be a sub-range of the pairs (a partial sum), as in axis_fwd.
//   in(r, j) = in[r * irs + j * ijs],  out(r, c) = out[r * ors + c * ocs].
// sum = true: both components accumulate into o0.out; else each into its own.
// Consecutive threads take consecutive rows; a thread owns CT consecutive
// modes (CT even, so the parity of a mode is known at compile time).
template <class Nm, int RT, int CT>
__device__ void axis_bwd(int ncomp, bool sum, AxisOp<Nm> o0, AxisOp<Nm> o1, int rows, int M, int Qh, int ts,
                         int irs, int ijs, int ors, int ocs)
{
    static_assert(CT % 2 == 0, "CT must be even");
    using V = typename Nm::V;
    using A = typename Nm::A;
    const int nr = (rows + RT - 1) / RT, nc = (M + CT - 1) / CT, tiles = nr * nc, Q = 2 * Qh;
    const int nitems = sum ? tiles : ncomp * tiles;
    for (int it = threadIdx.x; it < nitems; it += NT) {
        const int comp0 = sum ? 0 : it / tiles, t = sum ? it : it - comp0 * tiles;
        const int tr = t % nr, tc = t / nr;
        int r[RT];
#pragma unroll
        for (int c = 0; c < RT; ++c) r[c] = tr + c * nr;
        const int c0 = tc * CT;
        A acc[RT][CT];
#pragma unroll
        for (int c = 0; c < RT; ++c)
#pragma unroll
            for (int e = 0; e < CT; ++e) acc[c][e] = Nm::zero();
        const int cend = sum ? ncomp : comp0 + 1;
        for (int comp = comp0; comp < cend; ++comp) {
            const AxisOp<Nm> o = comp ? o1 : o0;
            const V* ip[RT];
#pragma unroll
            for (int c = 0; c < RT; ++c) ip[c] = o.in + (size_t)(r[c] < rows ? r[c] : rows - 1) * irs;
            const V* tp[CT];
#pragma unroll
            for (int e = 0; e < CT; ++e) tp[e] = o.tab + (size_t)(c0 + e < M ? c0 + e : M - 1) * ts;
            // which fold each mode uses: s (sum) or d (difference)
            const bool sq = o.kind >= TV2;
            const bool even_sum = o.kind == TV;   // values: even c sums; derivatives: odd c sums
            for (int q = 0; q < Qh; ++q) {
                V s[RT], d[RT];
#pragma unroll
                for (int c = 0; c < RT; ++c) {
                    V a = ip[c][(size_t)q * ijs], b = ip[c][(size_t)(Q - 1 - q) * ijs];
                    s[c] = Nm::add(a, b);
                    d[c] = sq ? s[c] : Nm::sub(a, b);
                }
#pragma unroll
                for (int e = 0; e < CT; ++e) {
                    V tv = tp[e][q];
                    if (sq) tv = Nm::mul(tv, tv);
                    const bool use_s = sq || (((e & 1) == 0) == even_sum);
#pragma unroll
                    for (int c = 0; c < RT; ++c) Nm::mac(acc[c][e], use_s ? s[c] : d[c], tv);
                }
            }
        }
        typename Nm::V* out = sum ? o0.out : (comp0 ? o1.out : o0.out);
#pragma unroll
        for (int c = 0; c < RT; ++c)
#pragma unroll
            for (int e = 0; e < CT; ++e)
                if (r[c] < rows && c0 + e < M) out[(size_t)r[c] * ors + (size_t)(c0 + e) * ocs] = Nm::res(acc[c][e]);
    }
}

// ------------------------------------------------------------------ geometry and buffers
// A step split over the CTAs of a thread-block cluster (the 2D coarse sweep):
// CTA `rank` of `size` owns the y node pairs [q0, q0 + nq) of the instance and
// their mirrors, i.e. Qyl = 2 nq node columns.  Mode-space vectors are kept
// whole in every CTA; every node-to-mode result (load, diagonal, operator
// application) is a partial sum over the CTA's columns, added up across the
// cluster through distributed shared memory (split_allreduce).  size = 1 is
// the one-CTA step.
struct Split {
    int rank = 0, size = 1;
    double* pb = nullptr;   // this CTA's receive and gather buffers in shared memory: 2 x stride 8-byte slots
    int stride = 0;         // >= K + size - 1
};

struct Dims2 {
    int Mx, My, Qx, Qy, Qhx, Qhy, K;
    int q0, nq;   // this CTA's y node pairs
    int Qyl;      // its node columns (2 nq; Qy for a one-CTA step)
    int Qyp;      // Qyl + 1: padded row of the Mx x Qyl intermediates
};

__device__ __forceinline__ Dims2 dims2(const InstDev& I, const Split& sp = Split{})
{
    Dims2 g;
    g.Mx = I.Mx;
    g.My = I.My;
    g.Qx = I.Q;
    g.Qy = I.Qy;
    g.Qhx = I.Qh;
    g.Qhy = I.Qhy;
    g.K = I.K;
    const int nqb = (I.Qhy + sp.size - 1) / sp.size;
    g.q0 = min(I.Qhy, sp.rank * nqb);
    g.nq = min(nqb, I.Qhy - g.q0);
    g.Qyl = 2 * g.nq;
    g.Qyp = g.Qyl + 1;
    return g;
}

// global y node of local column jl (columns jl < nq are pairs q0 + jl, the rest their mirrors)
__device__ __forceinline__ int col_global(const Dims2& g, int jl)
{
    return jl < g.nq ? g.q0 + jl : g.Qy - g.Qyl - g.q0 + jl;
}

// Sum of the CTAs' partial vectors v (K, this CTA's partial on entry, the
// cluster's sum on return, the same in every CTA), as a reduce-scatter and an
// all-gather that move data only by stores into other CTAs' shared memory:
//   1. entry k of every partial goes to the receive buffer of the CTA that owns
//      k (slices of S = ceil(K / size) entries), at the row of the sender;
//   2. each CTA adds the rows of its slice in rank order and stores the sums
//      into the gather buffer of every CTA;
//   3. each CTA copies its gather buffer into v.
// Two cluster barriers.  A buffer is written again only after the next call's
// first barrier, which every CTA reaches after it has read this call's data.
template <class Nm>
__device__ void split_allreduce(const Split& sp, typename Nm::V* v, int K)
{
    if (sp.size <= 1) return;
    using V = typename Nm::V;
    namespace cgx = cooperative_groups;
    cgx::cluster_group cl = cgx::this_cluster();
    const int C = sp.size, S = (K + C - 1) / C;
    V* recv = reinterpret_cast<V*>(sp.pb);               // C x S: row r = rank r's entries of my slice
    V* gat = reinterpret_cast<V*>(sp.pb + sp.stride);    // K: the sums
    for (int k = threadIdx.x; k < K; k += NT) {
        const int owner = k / S;
        *cl.map_shared_rank(recv + (size_t)sp.rank * S + (k - owner * S), owner) = v[k];
    }
    cl.sync();
    const int k0 = sp.rank * S;
    for (int j = threadIdx.x; j < S && k0 + j < K; j += NT) {
        V acc = recv[j];
        for (int r = 1; r < C; ++r) acc = Nm::add(acc, recv[(size_t)r * S + j]);
        for (int r = 0; r < C; ++r) *cl.map_shared_rank(gat + k0 + j, r) = acc;
    }
    cl.sync();
    for (int k = threadIdx.x; k < K; k += NT) v[k] = gat[k];
    __syncthreads();
}

template <class Nm>
struct Tabs2 {
    const typename Nm::V *Sx, *Dx, *Sy, *Dy;   // M x Qh each (value, derivative) per axis
};

// Per-CTA working arrays of the 2D step (shared memory or the CTA slot's global
// workspace; generic pointers either way).
struct Step2D {
    df* cdf;                      // K: double-float vector being transformed
    void *T1, *T2;                // Mx x Qyp intermediates (8-byte elements)
    void *N1, *N2;                // Qx x Qy node arrays (8-byte elements)
    void* wd;                     // Qx x Qy: W = w D (double-float, or FP64)
    float* wd32;                  // Qx x Qy: W in FP32 (mixed)
    void *dinv, *x, *r, *p, *q;   // K: CG vectors (FP32 mixed, FP64 path)
    double *xr, *rhs;             // K: refinement iterate, right-hand side (mixed)
    float* z;                     // K: FP32 correction (mixed)
    float* tab32;                 // FP32 tables Sx, Dx, Sy, Dy (M x Qh each)
    void* red;                    // reduction scratch (4 NT/32 doubles)
};

// A v -> out (K): the four folded one-axis transforms.
// Node arrays hold the CTA's columns: N(i, jl) at i * Qyl + jl; the Mx x Qyl
// intermediates have rows Qyp apart.  Transforms along y use the y tables from
// the CTA's first pair on (row stride Qhy).
template <class Nm, int RT, int QT, int CT>
__device__ void op_apply(const Dims2& g, const Tabs2<Nm>& tb, const typename Nm::V* v, const typename Nm::V* W,
                         typename Nm::V* T1, typename Nm::V* T2, typename Nm::V* N1, typename Nm::V* N2,
                         typename Nm::V* out, const Split& sp = Split{})
{
    const typename Nm::V *Sy = tb.Sy + g.q0, *Dy = tb.Dy + g.q0;
    // along y: T1 = v . Sy (values), T2 = v . Dy (derivatives);  rows k < Mx
    axis_fwd<Nm, RT, QT, false>(2, {v, Sy, T1, TV}, {v, Dy, T2, TD}, g.Mx, g.My, g.nq, g.Qhy, g.My, 1, g.Qyp, 1,
                                nullptr);
    __syncthreads();
    // along x, times W: N1 = W o (Dx . T1) = W o dx v,  N2 = W o (Sx . T2) = W o dy v;  rows: the CTA's columns
    axis_fwd<Nm, RT, QT, true>(2, {T1, tb.Dx, N1, TD}, {T2, tb.Sx, N2, TV}, g.Qyl, g.Mx, g.Qhx, g.Qhx, 1, g.Qyp,
                               1, g.Qyl, W);
    __syncthreads();
    // back along x: T1 = Dx^T N1, T2 = Sx^T N2
    axis_bwd<Nm, RT, CT>(2, false, {N1, tb.Dx, T1, TD}, {N2, tb.Sx, T2, TV}, g.Qyl, g.Mx, g.Qhx, g.Qhx, 1, g.Qyl,
                         1, g.Qyp);
    __syncthreads();
    // back along y, summed: out = T1 . Sy^T + T2 . Dy^T (over the CTA's columns)
    axis_bwd<Nm, 1, CT>(2, true, {T1, Sy, out, TV}, {T2, Dy, nullptr, TD}, g.Mx, g.My, g.nq, g.Qhy, g.Qyp, 1, g.My,
                        1);
    __syncthreads();
    split_allreduce<Nm>(sp, out, g.K);
}

// values at the CTA's nodes: N = Sx . (v . Sy)
template <class Nm, int RT, int QT>
__device__ void to_nodes(const Dims2& g, const Tabs2<Nm>& tb, const typename Nm::V* v, typename Nm::V* T1,
                         typename Nm::V* N)
{
    axis_fwd<Nm, RT, QT, false>(1, {v, tb.Sy + g.q0, T1, TV}, {}, g.Mx, g.My, g.nq, g.Qhy, g.My, 1, g.Qyp, 1,
                                nullptr);
    __syncthreads();
    axis_fwd<Nm, RT, QT, true>(1, {T1, tb.Sx, N, TV}, {}, g.Qyl, g.Mx, g.Qhx, g.Qhx, 1, g.Qyp, 1, g.Qyl, nullptr);
    __syncthreads();
}

// Galerkin projection of node values: out_kl = sum_ij phi_k(x_i) phi_l(y_j) N_ij
template <class Nm, int RT, int CT>
__device__ void from_nodes(const Dims2& g, const Tabs2<Nm>& tb, const typename Nm::V* N, typename Nm::V* T1,
                           typename Nm::V* out, const Split& sp = Split{})
{
    axis_bwd<Nm, RT, CT>(1, false, {N, tb.Sx, T1, TV}, {}, g.Qyl, g.Mx, g.Qhx, g.Qhx, 1, g.Qyl, 1, g.Qyp);
    __syncthreads();
    axis_bwd<Nm, 1, CT>(1, false, {T1, tb.Sy + g.q0, out, TV}, {}, g.Mx, g.My, g.nq, g.Qhy, g.Qyp, 1, g.My, 1);
    __syncthreads();
    split_allreduce<Nm>(sp, out, g.K);
}

// diag(A)_kl = sum_ij W_ij (phi_k'(x_i)^2 phi_l(y_j)^2 + phi_k(x_i)^2 phi_l'(y_j)^2) -> out
template <class Nm, int RT, int CT>
__device__ void op_diag(const Dims2& g, const Tabs2<Nm>& tb, const typename Nm::V* W, typename Nm::V* T1,
                        typename Nm::V* T2, typename Nm::V* out, const Split& sp = Split{})
{
    axis_bwd<Nm, RT, CT>(2, false, {W, tb.Dx, T1, TD2}, {W, tb.Sx, T2, TV2}, g.Qyl, g.Mx, g.Qhx, g.Qhx, 1, g.Qyl,
                         1, g.Qyp);
    __syncthreads();
    axis_bwd<Nm, 1, CT>(2, true, {T1, tb.Sy + g.q0, out, TV2}, {T2, tb.Dy + g.q0, nullptr, TD2}, g.Mx, g.My, g.nq,
                        g.Qhy, g.Qyp, 1, g.My, 1);
    __syncthreads();
    split_allreduce<Nm>(sp, out, g.K);
}

// ------------------------------------------------------------------ families at a 2D node
__device__ __forceinline__ double D_eval2(const InstDev& I, double sx1, double sx2, double cy2, double u)
{
    const double* c = I.dpar;
    double X0 = 1.0 + c[4] * sx2 + c[5] * cy2;
    double X1 = 1.0 + c[6] * sx2 + c[7] * cy2;
    double v = c[0] + c[3] * sx1;
    if (c[1] != 0.0) v += c[1] / (1.0 + u * u) * X1;
    if (c[2] != 0.0) v += c[2] * u;
    return v * X0;
}

__device__ __forceinline__ float D_eval2_32(const InstDev& I, float sx1, float sx2, float cy2, float u)
{
    const double* c = I.dpar;
    float X0 = 1.0f + (float)c[4] * sx2 + (float)c[5] * cy2;
    float X1 = 1.0f + (float)c[6] * sx2 + (float)c[7] * cy2;
    float v = (float)c[0] + (float)c[3] * sx1;
    if (c[1] != 0.0) v += (float)c[1] / (1.0f + u * u) * X1;
    if (c[2] != 0.0) v += (float)c[2] * u;
    return v * X0;
}

// Node (i, j) geometry: abscissa, weight and the family's node functions
struct Node2 {
    double x, w, sx1, sx2, cy2;
};

__device__ __forceinline__ Node2 node2(const InstDev& I, const TabDev& TX, const TabDev& TY, const double* tp,
                                       int i, int j)
{
    Node2 n;
    const bool mx = i >= I.Qh, my = j >= I.Qhy;
    const int qi = mx ? I.Q - 1 - i : i, qj = my ? I.Qy - 1 - j : j;
    const double xh = tp[TX.oX + qi];
    n.x = mx ? I.lo0 + I.hi0 - xh : xh;
    n.w = tp[TX.oWq + qi] * tp[TY.oWq + qj];
    n.sx1 = tp[TX.oAux + 4 * qi + (mx ? 2 : 0)];
    n.sx2 = tp[TX.oAux + 4 * qi + (mx ? 3 : 1)];
    n.cy2 = tp[TY.oAux2 + 2 * qj + (my ? 1 : 0)];
    return n;
}

// The same node data as double-float, from the double-float tables
struct Node2df {
    df w, sx1, sx2, cy2;
};

__device__ __forceinline__ Node2df node2_df(const InstDev& I, const TabDev& TX, const TabDev& TY, const double* tp,
                                            int i, int j)
{
    Node2df n;
    const bool mx = i >= I.Qh, my = j >= I.Qhy;
    const int qi = mx ? I.Q - 1 - i : i, qj = my ? I.Qy - 1 - j : j;
    const df* wx = reinterpret_cast<const df*>(tp + TX.oWd);
    const df* wy = reinterpret_cast<const df*>(tp + TY.oWd);
    const df* ax = reinterpret_cast<const df*>(tp + TX.oAuxd);
    const df* ay = reinterpret_cast<const df*>(tp + TY.oAux2d);
    n.w = df_mul(wx[qi], wy[qj]);
    n.sx1 = ax[4 * qi + (mx ? 2 : 0)];
    n.sx2 = ax[4 * qi + (mx ? 3 : 1)];
    n.cy2 = ay[2 * qj + (my ? 1 : 0)];
    return n;
}

// ------------------------------------------------------------------ block reductions
// Block sums of a and b (every thread gets them, the same order of addition)
// with one barrier: consecutive calls use the two halves of red
// in turn (buf toggles), so a call never overwrites the half that threads may
// still read from the call before; the barrier of the call in between orders
// them.  red holds 2 x (2 NT/32) elements.
template <typename T>
__device__ __forceinline__ void block_sum2T_db(T& a, T& b, T* red, int& buf)
{
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    T* r = red + buf * (2 * (NT / 32));
    buf ^= 1;
    if ((threadIdx.x & 31) == 0) {
        r[threadIdx.x >> 5] = a;
        r[NT / 32 + (threadIdx.x >> 5)] = b;
    }
    __syncthreads();
    T sa = 0, sb = 0;
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) {
        sa += r[w];
        sb += r[NT / 32 + w];
    }
    a = sa;
    b = sb;
}

template <typename T>
__device__ __forceinline__ T block_maxT(T v, T* red)
{
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    T m = 0;
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) m = fmax(m, red[w]);
    __syncthreads();
    return m;
}

// ------------------------------------------------------------------ preconditioned CG
// Solves (I + mu A) x = b for the right-hand side in `b` (K, overwritten by the
// solution).  The right-hand side is scaled to unit max norm first: refinement
// residuals can be ~1e-15 of the solution, whose FP32 inner products would
// underflow unscaled.  flag[0]: set to 0 when p . (I + mu A) p <= 0 (not SPD);
// flag[1] counts operator applications.
// With a split step every CTA of the cluster runs the whole iteration on the
// whole vectors (identical values, so identical control flow); only the
// operator application is shared (op_apply's all-reduction).
template <class Nm, int RT, int QT, int CT>
__device__ void pcg2d(const Dims2& g, const Tabs2<Nm>& tb, typename Nm::V mu, const typename Nm::V* W,
                      typename Nm::V* b, const Step2D& S, int* flag, int maxit, typename Nm::V rtol,
                      const Split& sp = Split{})
{
    using T = typename Nm::V;
    const int K = g.K, tid = threadIdx.x;
    T* x = static_cast<T*>(S.x);
    T* r = static_cast<T*>(S.r);
    T* p = static_cast<T*>(S.p);
    T* q = static_cast<T*>(S.q);
    T* dinv = static_cast<T*>(S.dinv);
    T* red = static_cast<T*>(S.red);
    T* T1 = static_cast<T*>(S.T1);
    T* T2 = static_cast<T*>(S.T2);
    T* N1 = static_cast<T*>(S.N1);
    T* N2 = static_cast<T*>(S.N2);
    T bmax = 0;
    for (int k = tid; k < K; k += NT) bmax = fmax(bmax, fabs(b[k]));
    bmax = block_maxT(bmax, red);
    if (!(bmax > T(0)) || !isfinite(bmax)) {
        for (int k = tid; k < K; k += NT) b[k] = T(0);
        __syncthreads();
        return;
    }
    const T bs = T(1) / bmax;
    T rz = 0, rr = 0;
    for (int k = tid; k < K; k += NT) {
        T rk = b[k] * bs, zk = dinv[k] * rk;
        x[k] = T(0);
        r[k] = rk;
        p[k] = zk;
        rz += rk * zk;
        rr += rk * rk;
    }
    // the sums below alternate between the two halves of red (block_maxT's last
    // barrier orders the first one after its reads)
    int buf = 0;
    block_sum2T_db(rz, rr, red, buf);   // its barrier also publishes x, r and p
    const T stop = rtol * rtol * rr;
    for (int it = 0; it < maxit && rr > T(0); ++it) {
        if (tid == 0) flag[1] += 1;
        op_apply<Nm, RT, QT, CT>(g, tb, p, W, T1, T2, N1, N2, q, sp);
        T pq = 0, zero = 0;
        for (int k = tid; k < K; k += NT) {
            T qk = p[k] + mu * q[k];
            q[k] = qk;
            pq += p[k] * qk;
        }
        block_sum2T_db(pq, zero, red, buf);
        if (!(pq > T(0))) {   // (I + mu A) not positive definite (D <= 0 somewhere)
            if (tid == 0 && flag[0] < 0) flag[0] = 0;
            break;
        }
        const T al = rz / pq;
        T rzn = 0, rrn = 0;
        for (int k = tid; k < K; k += NT) {
            x[k] = fma(al, p[k], x[k]);
            T rk = fma(-al, q[k], r[k]);
            r[k] = rk;
            T zk = dinv[k] * rk;
            q[k] = zk;   // q holds z until the p update
            rzn += rk * zk;
            rrn += rk * rk;
        }
        block_sum2T_db(rzn, rrn, red, buf);
        if (rrn <= stop) break;
        const T be = rz > T(0) ? rzn / rz : T(0);
        rz = rzn;
        for (int k = tid; k < K; k += NT) p[k] = fma(be, p[k], q[k]);
        __syncthreads();
    }
    for (int k = tid; k < K; k += NT) b[k] = x[k] * bmax;
    __syncthreads();
}

constexpr int PCG2_MAXIT32 = 60;
constexpr float PCG2_RTOL32 = INNER_RTOL_DEFAULT;
constexpr int PCG2_MAXIT64 = 1000;
constexpr double PCG2_RTOL64 = 1e-14;

// FP32 tables of both axes into the CTA's copy: Sx, Dx, Sy, Dy (M x Qh each)
__device__ __forceinline__ Tabs2<NumF> stage_tab32(const InstDev& I, const TabDev& TX, const TabDev& TY,
                                                   const double* tp, float* t32)
{
    const int nx = I.Mx * I.Qh, ny = I.My * I.Qhy;
    const float* sx = reinterpret_cast<const float*>(tp + TX.oSt32);
    const float* dx = reinterpret_cast<const float*>(tp + TX.oDt32);
    const float* sy = reinterpret_cast<const float*>(tp + TY.oSt32);
    const float* dy = reinterpret_cast<const float*>(tp + TY.oDt32);
    for (int e = threadIdx.x; e < nx; e += NT) {
        t32[e] = sx[e];
        t32[nx + e] = dx[e];
    }
    for (int e = threadIdx.x; e < ny; e += NT) {
        t32[2 * nx + e] = sy[e];
        t32[2 * nx + ny + e] = dy[e];
    }
    return {t32, t32 + nx, t32 + 2 * nx, t32 + 2 * nx + ny};
}

// ------------------------------------------------------------------ the steps
// FP64 path.  c, hist: K (any memory); out, F: K.  Returns the first bad index or -1.
__device__ int step2d_fp64(const InstDev& I, const TabDev& TX, const TabDev& TY, const double* tp,
                           const double* c, const double* hist, double te, double mu, double* out, double* F,
                           const Step2D& S, int* flag, const Split& sp = Split{})
{
    const Dims2 g = dims2(I, sp);
    const int tid = threadIdx.x, QQ = g.Qx * g.Qyl;
    const Tabs2<NumD> tb{tp + TX.oSt, tp + TX.oDt, tp + TY.oSt, tp + TY.oDt};
    double* T1 = static_cast<double*>(S.T1);
    double* T2 = static_cast<double*>(S.T2);
    double* N1 = static_cast<double*>(S.N1);
    double* N2 = static_cast<double*>(S.N2);
    double* W = static_cast<double*>(S.wd);
    double* dinv = static_cast<double*>(S.dinv);
    if (tid == 0) flag[0] = -1;
    to_nodes<NumD, 2, 2>(g, tb, c, T1, N1);
    for (int e = tid; e < QQ; e += NT) {
        const int i = e / g.Qyl, j = col_global(g, e - i * g.Qyl);
        const Node2 nd = node2(I, TX, TY, tp, i, j);
        const double u = N1[e];
        W[e] = nd.w * D_eval2(I, nd.sx1, nd.sx2, nd.cy2, u);
        N2[e] = nd.w * f_eval(I, nd.x, nd.sx1, te, u);
    }
    __syncthreads();
    from_nodes<NumD, 2, 2>(g, tb, N2, T2, F, sp);
    op_diag<NumD, 2, 2>(g, tb, W, T1, T2, dinv, sp);
    for (int k = tid; k < g.K; k += NT) {
        dinv[k] = 1.0 / (1.0 + mu * dinv[k]);
        out[k] = hist[k] + mu * F[k];
    }
    __syncthreads();
    pcg2d<NumD, 2, 2, 2>(g, tb, mu, W, out, S, flag, PCG2_MAXIT64, PCG2_RTOL64, sp);
    return flag[0];
}

// Mixed path (fp32_only: FP32 coefficients and a single FP32 solve; ftol > 0:
// the refinement may stop at that fraction of the iterate, as in the 1D step).
__device__ int step2d_mixed(const InstDev& I, const TabDev& TX, const TabDev& TY, const double* tp,
                            const double* c, const double* hist, double te, double mu, double* out, double* F,
                            const Step2D& S, int* flag, bool fp32_only, const Split& sp = Split{},
                            float ftol = 0.f)
{
    const Dims2 g = dims2(I, sp);
    const int tid = threadIdx.x, QQ = g.Qx * g.Qyl, K = g.K;
    const Tabs2<NumDF> td{reinterpret_cast<const df*>(tp + TX.oStd), reinterpret_cast<const df*>(tp + TX.oDtd),
                          reinterpret_cast<const df*>(tp + TY.oStd), reinterpret_cast<const df*>(tp + TY.oDtd)};
    df* T1 = static_cast<df*>(S.T1);
    df* T2 = static_cast<df*>(S.T2);
    df* N1 = static_cast<df*>(S.N1);
    df* N2 = static_cast<df*>(S.N2);
    df* W = static_cast<df*>(S.wd);
    float* red = static_cast<float*>(S.red);
    if (tid == 0) flag[0] = -1;
    const Tabs2<NumF> tf = stage_tab32(I, TX, TY, tp, S.tab32);
    for (int k = tid; k < K; k += NT) S.cdf[k] = df_from_double(c[k]);
    __syncthreads();
    to_nodes<NumDF, 2, 2>(g, td, S.cdf, T1, N1);
    const df emt = (I.fpar[3] != 0.0 && !fp32_only) ? df_from_double(exp(-te)) : df{0.f, 0.f};
    for (int e = tid; e < QQ; e += NT) {
        const int i = e / g.Qyl, j = col_global(g, e - i * g.Qyl);
        if (fp32_only) {
            const Node2 nd = node2(I, TX, TY, tp, i, j);
            const double u = df_to_double(N1[e]);
            const double wD = nd.w * (double)D_eval2_32(I, (float)nd.sx1, (float)nd.sx2, (float)nd.cy2, (float)u);
            const double wf = nd.w * (double)f_eval32(I, (float)nd.sx1, (float)te, (float)u);
            W[e] = df_from_double(wD);
            S.wd32[e] = (float)wD;
            N2[e] = df_from_double(wf);
            continue;
        }
        // D and f in double-float on the FP32 pipes (manufactured sources in FP64)
        const Node2df nd = node2_df(I, TX, TY, tp, i, j);
        const df u = N1[e];
        const df wD = df_mul(nd.w, D_eval_df(I, nd.sx1, nd.sx2, nd.cy2, u));
        df wf;
        if (I.f_df) {
            wf = df_mul(nd.w, f_eval_df(I, nd.sx1, emt, u));
        } else {
            const Node2 n64 = node2(I, TX, TY, tp, i, j);
            wf = df_from_double(n64.w * f_eval(I, n64.x, n64.sx1, te, df_to_double(u)));
        }
        W[e] = wD;
        S.wd32[e] = wD.hi;
        N2[e] = wf;
    }
    __syncthreads();
    from_nodes<NumDF, 2, 2>(g, td, N2, T2, S.cdf, sp);
    // FP32 Jacobi diagonal (into the CG's dinv)
    float* dinv = static_cast<float*>(S.dinv);
    op_diag<NumF, 2, 4>(g, tf, S.wd32, static_cast<float*>(S.T1), static_cast<float*>(S.T2), dinv, sp);
    for (int k = tid; k < K; k += NT) {
        F[k] = df_to_double(S.cdf[k]);
        dinv[k] = 1.0f / (1.0f + (float)mu * dinv[k]);
        const double rk = hist[k] + mu * F[k];
        S.rhs[k] = rk;
        S.xr[k] = 0.0;
        S.z[k] = (float)rk;
    }
    __syncthreads();
    const float rtol = fp32_only ? fmaxf(PCG2_RTOL32, ftol) : I.inner_rtol;   // tunable in the refined step
    pcg2d<NumF, 2, 4, 4>(g, tf, (float)mu, S.wd32, S.z, S, flag, PCG2_MAXIT32, rtol, sp);
    float zprev = 0.f;
    for (int sweep = 0;; ++sweep) {
        float zmax = 0.f, xmax = 0.f;
        for (int k = tid; k < K; k += NT) {
            const double xn = S.xr[k] + (double)S.z[k];
            S.xr[k] = xn;
            zmax = fmaxf(zmax, fabsf(S.z[k]));
            xmax = fmaxf(xmax, (float)fabs(xn));
        }
        zmax = block_maxT(zmax, red);
        xmax = block_maxT(xmax, red);
        // stop on a small correction, or when the observed contraction predicts one (as in 1D)
        const bool small = zmax <= fmaxf(REFINE_TOL, ftol) * xmax;
        const bool predicted =
            sweep >= 1 && zmax < zprev && zmax * zmax <= fmaxf(REFINE_EST, ftol) * xmax * zprev;
        if (fp32_only || small || predicted || sweep >= 6 || flag[0] >= 0) break;
        zprev = zmax;
        if (tid == 0) flag[2] += 1;
        // residual rhs - (I + mu A) x with A applied in double-float
        for (int k = tid; k < K; k += NT) S.cdf[k] = df_from_double(S.xr[k]);
        __syncthreads();
        op_apply<NumDF, 2, 2, 2>(g, td, S.cdf, W, T1, T2, N1, N2, S.cdf, sp);
        for (int k = tid; k < K; k += NT)
            S.z[k] = (float)(S.rhs[k] - S.xr[k] - mu * df_to_double(S.cdf[k]));
        __syncthreads();
        pcg2d<NumF, 2, 4, 4>(g, tf, (float)mu, S.wd32, S.z, S, flag, PCG2_MAXIT32, rtol, sp);
    }
    for (int k = tid; k < K; k += NT) out[k] = S.xr[k];
    __syncthreads();
    return flag[0];
}

}  // namespace psl1
