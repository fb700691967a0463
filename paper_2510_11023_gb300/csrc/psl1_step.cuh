// psl1_step.cuh -- one linearised L1 step of the 1D sine-Galerkin scheme,
// executed by one CTA of NT threads:
//
//   (I + mu A(D(t_e, c))) c_new = hist + mu F(f(t_e, c))      (Eq. NumericalSchemeFine /
//                                                              NumericalSchemeSequential)
//
//   u_q   = sum_k c_k phi_k(x_q)                    (mode -> node, mirror-folded)
//   A_kl  = sum_q w_q D_q phi_k'(x_q) phi_l'(x_q)   (Eq. AForm with Gauss quadrature)
//         = cA k l (g_|k-l| + g_{k+l}),  g_s = sum_q w_q D_q cos(s pi th_q)
//   F_k   = sum_q w_q f_q phi_k(x_q)
//
// The second form of A_kl is the same quadrature sum rearranged with
// 2 cos a cos b = cos(a-b) + cos(a+b): 2K+1 moments instead of a K x K x Q
// contraction.  Mirror folding: Gauss nodes are symmetric, x_q' = lo+hi-x_q,
// phi_k(x_q') = (-1)^{k+1} phi_k(x_q), cos(s pi th_q') = (-1)^s cos(s pi th_q),
// so every transform runs over Q/2 node pairs.
//
// The SPD system is solved by a right-looking blocked Cholesky on 32x32
// blocks ("block-packed" lower storage): one warp factors the diagonal
// panel with intra-warp synchronisation only, all warps do the triangular
// panel solve and the register-tiled trailing update.
#pragma once
#include "psl1_device.cuh"

namespace psl1 {

// ------------------------------------------------------------------ families
__device__ __forceinline__ double D_eval(const InstDev& I, double sx1, double sx2, double u)
{
    const double* c = I.dpar;
    double X0 = 1.0 + c[4] * sx2;
    double X1 = 1.0 + c[6] * sx2;
    double v = c[0] + c[3] * sx1;
    if (c[1] != 0.0) v += c[1] / (1.0 + u * u) * X1;
    if (c[2] != 0.0) v += c[2] * u;
    return v * X0;
}

// FP32 versions (PSL1_PREC_FP32)
__device__ __forceinline__ float D_eval32(const InstDev& I, float sx1, float sx2, float u)
{
    const double* c = I.dpar;
    float X0 = 1.0f + (float)c[4] * sx2;
    float X1 = 1.0f + (float)c[6] * sx2;
    float v = (float)c[0] + (float)c[3] * sx1;
    if (c[1] != 0.0) v += (float)c[1] / (1.0f + u * u) * X1;
    if (c[2] != 0.0) v += (float)c[2] * u;
    return v * X0;
}

__device__ __forceinline__ float f_eval32(const InstDev& I, float sx1, float t, float u)
{
    const double* c = I.fpar;
    float v = 0.0f;
    if (c[0] != 0.0) v += (float)c[0] * cosf(u);
    if (c[1] != 0.0) v += (float)c[1] * sinf(u);
    if (c[2] != 0.0) v += (float)c[2] * u * (1.0f - u);
    if (c[3] != 0.0) v += (float)c[3] * sx1 * expf(-t);
    return v;
}

// manufactured source for u = (1 + t^a) sin(pi x), D = d0 + d1/(1+u^2)
__device__ double src1_eval(const InstDev& I, double x, double sx1, double t)
{
    double a = 1.0 + pow(t, I.alpha);
    double cx = cospi(x);
    const double pi = 3.141592653589793;
    double u = a * sx1, ux = a * pi * cx, uxx = -a * pi * pi * sx1;
    double d0 = I.dpar[0], d1 = I.dpar[1];
    double w = 1.0 + u * u;
    return I.g1a * sx1 - ((d0 + d1 / w) * uxx - 2.0 * d1 * u / (w * w) * ux * ux);
}

// manufactured source for u = (1 + t^2) sin(pi x)/(2 - cos(pi x)), D = d0 + d3 sin(pi x)
__device__ double src2_eval(const InstDev& I, double x, double sx1, double t)
{
    const double pi = 3.141592653589793;
    double cx = cospi(x), den = 2.0 - cx;
    double s0 = sx1 / den;
    double s1 = pi * (2.0 * cx - 1.0) / (den * den);
    double s2 = -2.0 * pi * pi * sx1 * (1.0 + cx) / (den * den * den);
    double Dx = I.dpar[0] + I.dpar[3] * sx1, Dxx = I.dpar[3] * pi * cx;
    double ca = t > 0.0 ? 2.0 * pow(t, 2.0 - I.alpha) / I.g3a : 0.0;
    return ca * s0 - (1.0 + t * t) * (Dx * s2 + Dxx * s1);
}

__device__ __forceinline__ double f_eval(const InstDev& I, double x, double sx1, double t, double u)
{
    const double* c = I.fpar;
    double v = 0.0;
    if (c[0] != 0.0) v += c[0] * cos(u);
    if (c[1] != 0.0) v += c[1] * sin(u);
    if (c[2] != 0.0) v += c[2] * u * (1.0 - u);
    if (c[3] != 0.0) v += c[3] * sx1 * exp(-t);
    if (c[4] != 0.0) v += c[4] * src1_eval(I, x, sx1, t);
    if (c[5] != 0.0) v += c[5] * src2_eval(I, x, sx1, t);
    return v;
}

// ------------------------------------------------------------------ block-packed storage
template <typename T, int LDB>
struct BPack {
    T* base;
    __device__ __forceinline__ T* blk(int I, int J) const
    {
        return base + (size_t)(I * (I + 1) / 2 + J) * (TILE * LDB);
    }
};


// ------------------------------------------------------------------ Cholesky
// Factor in place.  *bad receives the first non-positive pivot (global
// index) or stays -1; a bad pivot is replaced by 1 so that the solve stays
// finite and the caller reports PSL1_ERR_NOT_SPD.
template <typename T, int LDB>
__device__ void chol_factor(BPack<T, LDB> A, int nb, int* bad)
{
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int J = 0; J < nb; ++J) {
        if (warp == 0) {
            T* D = A.blk(J, J);
            for (int j = 0; j < TILE; ++j) {
                __syncwarp();
                T ajj = D[j * LDB + j];
                if (!(ajj > T(0))) {
                    if (lane == 0 && *bad < 0) *bad = TILE * J + j;
                    ajj = T(1);
                }
                T d = sqrt(ajj);
                __syncwarp();
                if (lane == j) D[j * LDB + j] = d;
                if (lane > j) D[lane * LDB + j] = D[lane * LDB + j] / d;
                __syncwarp();
                if (lane > j) {
                    T lij = D[lane * LDB + j];
                    for (int k = j + 1; k <= lane; ++k) D[lane * LDB + k] -= lij * D[k * LDB + j];
                }
            }
            __syncwarp();
        }
        __syncthreads();
        // panel: L_IJ = A_IJ L_JJ^{-T}, one row per thread
        const T* Ljj = A.blk(J, J);
        const int nrows = (nb - J - 1) * TILE;
        for (int rr = tid; rr < nrows; rr += NT) {
            int I = J + 1 + rr / TILE, i = rr % TILE;
            T* row = A.blk(I, J) + i * LDB;
            for (int j = 0; j < TILE; ++j) {
                T s = row[j];
                for (int p = 0; p < j; ++p) s -= row[p] * Ljj[j * LDB + p];
                row[j] = s / Ljj[j * LDB + j];
            }
        }
        __syncthreads();
        // trailing update A_{I,I2} -= L_IJ L_{I2,J}^T, J < I2 <= I, 4x4 register tiles
        const int nrem = nb - J - 1;
        const int ntiles = nrem * (nrem + 1) / 2 * 64;
        for (int t = tid; t < ntiles; t += NT) {
            int pr = t >> 6, tt = t & 63;
            int a = (int)((sqrtf(8.0f * pr + 1.0f) - 1.0f) * 0.5f);
            while ((a + 1) * (a + 2) / 2 <= pr) ++a;
            while (a * (a + 1) / 2 > pr) --a;
            int b = pr - a * (a + 1) / 2;
            int I = J + 1 + a, I2 = J + 1 + b;
            int ti = tt >> 3, tj = tt & 7;
            if (I == I2 && tj > ti) continue;
            const T* Li = A.blk(I, J) + (4 * ti) * LDB;
            const T* Lj = A.blk(I2, J) + (4 * tj) * LDB;
            T acc[4][4];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = T(0);
#pragma unroll 4
            for (int p = 0; p < TILE; ++p) {
                T x[4], y[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    x[r] = Li[r * LDB + p];
                    y[r] = Lj[r * LDB + p];
                }
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[r][c] += x[r] * y[c];
            }
            T* C = A.blk(I, I2) + (4 * ti) * LDB + 4 * tj;
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) C[r * LDB + c] -= acc[r][c];
        }
        __syncthreads();
    }
}

// Solve L L^T x = v in place (v: Kp entries, shared memory).
template <typename T, int LDB, typename V>
__device__ void chol_solve(BPack<T, LDB> A, int nb, V* v)
{
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int J = 0; J < nb; ++J) {
        if (warp == 0) {
            const T* D = A.blk(J, J);
            V bi = v[TILE * J + lane];
            for (int j = 0; j < TILE; ++j) {
                V yj = __shfl_sync(0xffffffffu, bi, j) / (V)D[j * LDB + j];
                if (lane == j) bi = yj;
                if (lane > j) bi -= (V)D[lane * LDB + j] * yj;
            }
            v[TILE * J + lane] = bi;
        }
        __syncthreads();
        const int nrows = (nb - J - 1) * TILE;
        for (int rr = tid; rr < nrows; rr += NT) {
            int I = J + 1 + rr / TILE, i = rr % TILE;
            const T* row = A.blk(I, J) + i * LDB;
            V s = 0;
            for (int p = 0; p < TILE; ++p) s += (V)row[p] * v[TILE * J + p];
            v[TILE * I + i] -= s;
        }
        __syncthreads();
    }
    for (int J = nb - 1; J >= 0; --J) {
        if (warp == 0) {
            const T* D = A.blk(J, J);
            V xi = v[TILE * J + lane];
            for (int j = TILE - 1; j >= 0; --j) {
                V xj = __shfl_sync(0xffffffffu, xi, j) / (V)D[j * LDB + j];
                if (lane == j) xi = xj;
                if (lane < j) xi -= (V)D[j * LDB + lane] * xj;
            }
            v[TILE * J + lane] = xi;
        }
        __syncthreads();
        const int nrows = J * TILE;
        for (int rr = tid; rr < nrows; rr += NT) {
            int I = rr / TILE, c = rr % TILE;
            const T* blk = A.blk(J, I);
            V s = 0;
            for (int r = 0; r < TILE; ++r) s += (V)blk[r * LDB + c] * v[TILE * J + r];
            v[TILE * I + c] -= s;
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ FP64 step
// Shared-memory work vectors of one CTA (sizes for the largest instance).
struct StepSmem {
    double* wp;   // Qh : w (D_q + D_q')
    double* wm;   // Qh : w (D_q - D_q')
    double* fp;   // Qh : w (f_q + f_q')
    double* fm;   // Qh : w (f_q - f_q')
    double* g;    // 2K+1 moments
    double* v;    // Kp : right-hand side / solution
    int* bad;     // first bad pivot
};

// Nodes, D, f, moments and load vector.  c: K coefficients (shared).
__device__ void nodes_moments_fp64(const InstDev& I, const TabDev& Tb, const double* tp, const double* c,
                                   double te, StepSmem& s, double* F)
{
    const int tid = threadIdx.x, K = I.K, Qh = Tb.Qh;
    const double* St = tp + Tb.oSt;
    const double* xh = tp + Tb.oX;
    const double* wh = tp + Tb.oWq;
    const double* aux = tp + Tb.oAux;
    const double mid2 = I.lo0 + I.hi0;
    for (int q = tid; q < Qh; q += NT) {
        double O = 0.0, E = 0.0;
        int k = 0;
        for (; k + 1 < K; k += 2) {
            O = fma(St[(size_t)k * Qh + q], c[k], O);
            E = fma(St[(size_t)(k + 1) * Qh + q], c[k + 1], E);
        }
        if (k < K) O = fma(St[(size_t)k * Qh + q], c[k], O);
        double ua = O + E, ub = O - E;
        double xa = xh[q], xb = mid2 - xa, w = wh[q];
        double Da = D_eval(I, aux[4 * q], aux[4 * q + 1], ua);
        double Db = D_eval(I, aux[4 * q + 2], aux[4 * q + 3], ub);
        double fa = f_eval(I, xa, aux[4 * q], te, ua);
        double fb = f_eval(I, xb, aux[4 * q + 2], te, ub);
        s.wp[q] = w * (Da + Db);
        s.wm[q] = w * (Da - Db);
        s.fp[q] = w * (fa + fb);
        s.fm[q] = w * (fa - fb);
    }
    __syncthreads();
    const double* C = tp + Tb.oC;
    const double* S = tp + Tb.oS;
    const int ns = 2 * K + 1;
    for (int sI = tid; sI < ns; sI += NT) {
        const double* wv = (sI & 1) ? s.wm : s.wp;
        double acc = 0.0;
        for (int q = 0; q < Qh; ++q) acc = fma(C[(size_t)q * ns + sI], wv[q], acc);
        s.g[sI] = acc;
    }
    for (int k = tid; k < K; k += NT) {
        const double* fv = (k & 1) ? s.fm : s.fp;   // mode k+1 odd <=> index k even
        double acc = 0.0;
        for (int q = 0; q < Qh; ++q) acc = fma(S[(size_t)q * K + k], fv[q], acc);
        F[k] = acc;
    }
    __syncthreads();
}

// M = I + mu cA k l (g_|k-l| + g_{k+l}) on the lower blocks; identity padding.
template <typename T, int LDB>
__device__ void fill_matrix(const InstDev& I, const double* g, double mu, BPack<T, LDB> A)
{
    const int nb = I.nb, K = I.K;
    const int total = nb * (nb + 1) / 2 * TILE * TILE;
    const double sc = mu * I.cA;
    for (int e = threadIdx.x; e < total; e += NT) {
        int bidx = e >> 10, w = e & 1023, i = w >> 5, j = w & 31;
        int a = (int)((sqrtf(8.0f * bidx + 1.0f) - 1.0f) * 0.5f);
        while ((a + 1) * (a + 2) / 2 <= bidx) ++a;
        while (a * (a + 1) / 2 > bidx) --a;
        int Jb = bidx - a * (a + 1) / 2;
        int k = TILE * a + i, l = TILE * Jb + j;
        double val;
        if (k < K && l < K) {
            int d = k > l ? k - l : l - k;
            val = (k == l ? 1.0 : 0.0) + sc * (double)(k + 1) * (double)(l + 1) * (g[d] + g[k + l + 2]);
        } else {
            val = (k == l) ? 1.0 : 0.0;
        }
        A.blk(a, Jb)[i * LDB + j] = (T)val;
    }
    __syncthreads();
}

// Full FP64 step: c (K, shared) -> out (K, shared).  F scratch: K doubles.
// Returns the first bad pivot or -1.
__device__ int step_fp64(const InstDev& I, const TabDev& Tb, const double* tp, const double* c,
                         const double* hist, double te, double mu, double* out, double* F,
                         BPack<double, TILE> A, StepSmem& s)
{
    const int tid = threadIdx.x;
    nodes_moments_fp64(I, Tb, tp, c, te, s, F);
    fill_matrix<double, TILE>(I, s.g, mu, A);
    for (int k = tid; k < I.Kp; k += NT) s.v[k] = k < I.K ? hist[k] + mu * F[k] : 0.0;
    if (tid == 0) *s.bad = -1;
    __syncthreads();
    chol_factor<double, TILE>(A, I.nb, s.bad);
    chol_solve<double, TILE, double>(A, I.nb, s.v);
    for (int k = tid; k < I.K; k += NT) out[k] = s.v[k];
    __syncthreads();
    return *s.bad;
}

}  // namespace psl1
