// psl1_step_cheb.cuh -- one linearised L1 step of the Chebyshev-Lobatto
// collocation scheme, the paper's own spatial discretisation (Sec. 4.1,
// Eq. NumericalSchemeMainSystem), executed by one CTA in FP64:
//
//   (I - mu N(u_prev, t_e)) u_new = hist + mu f(x_I, t_e, u_prev),
//   N_ik = sum_j Dm_ij D(x_j, t_e, u_j) Dm_jk      (i, k interior; j all nodes),
//
// with u the values at the n - 1 interior nodes x_j = (a+b)/2 + (b-a)/2
// cos(j pi / n) (u = 0 at j = 0, n), Dm the first-derivative matrix scaled to
// the interval, and N the discrete div(D grad .) restricted to the interior.
// The system is not symmetric: it is solved by LU factorisation with partial
// pivoting in shared memory (n <= 64: at most 63 x 63).
#pragma once
#include "psl1_step.cuh"

namespace psl1 {

struct ChebSmem {
    double* M;     // Kc x Kc system matrix, factored in place
    double* u;     // n + 1 nodal values (boundary zeros), then the solution
    double* Dc;    // n + 1 diffusivities D(x_j, t_e, u_j)
    double* r;     // Kc right-hand side / multipliers
    double* l;     // Kc multipliers of the current column
    int* piv;      // [0] pivot row of the current column
};

// Per-instance collocation data at I.oC in the collocation pool: x (n+1),
// sin(pi x) (n+1), sin(2 pi x) (n+1), Dm ((n+1) x (n+1), row-major).
__device__ int step_cheb(const InstDev& I, const double* cpool, const double* c, const double* hist, double te,
                         double mu, double* out, ChebSmem& cs, int* bad)
{
    const int n = I.Mx, Qn = n + 1, K = n - 1, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const double* x = cpool + I.oC;
    const double* s1 = x + Qn;
    const double* s2 = s1 + Qn;
    const double* Dm = s2 + Qn;
    if (tid == 0) *bad = -1;
    for (int j = tid; j < Qn; j += NT) cs.u[j] = (j == 0 || j == n) ? 0.0 : c[j - 1];
    __syncthreads();
    for (int j = tid; j < Qn; j += NT) cs.Dc[j] = D_eval(I, s1[j], s2[j], cs.u[j]);
    for (int i = tid; i < K; i += NT) cs.r[i] = hist[i] + mu * f_eval(I, x[i + 1], s1[i + 1], te, cs.u[i + 1]);
    __syncthreads();
    for (int e = tid; e < K * K; e += NT) {
        const int i = e / K, k = e - i * K;
        const double* Di = Dm + (size_t)(i + 1) * Qn;
        double s = 0.0;
        for (int j = 0; j < Qn; ++j) s = fma(Di[j] * cs.Dc[j], Dm[(size_t)j * Qn + k + 1], s);
        cs.M[e] = (i == k ? 1.0 : 0.0) - mu * s;
    }
    __syncthreads();
    // LU with partial pivoting (rows of M and r swapped together)
    for (int j = 0; j < K; ++j) {
        if (warp == 0) {
            double best = -1.0;
            int row = j;
            for (int i = j + lane; i < K; i += 32) {
                const double v = fabs(cs.M[(size_t)i * K + j]);
                if (v > best) {
                    best = v;
                    row = i;
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const double bo = __shfl_xor_sync(0xffffffffu, best, o);
                const int ro = __shfl_xor_sync(0xffffffffu, row, o);
                if (bo > best || (bo == best && ro < row)) {
                    best = bo;
                    row = ro;
                }
            }
            if (lane == 0) cs.piv[0] = best > 0.0 ? row : -1;
        }
        __syncthreads();
        const int p = cs.piv[0];
        if (p < 0) {   // singular: no nonzero pivot in this column
            if (tid == 0) *bad = j;
            __syncthreads();
            break;
        }
        if (p != j) {
            for (int k = tid; k < K; k += NT) {
                const double t = cs.M[(size_t)j * K + k];
                cs.M[(size_t)j * K + k] = cs.M[(size_t)p * K + k];
                cs.M[(size_t)p * K + k] = t;
            }
            if (tid == 0) {
                const double t = cs.r[j];
                cs.r[j] = cs.r[p];
                cs.r[p] = t;
            }
        }
        __syncthreads();
        const double dj = cs.M[(size_t)j * K + j];
        for (int i = j + 1 + tid; i < K; i += NT) cs.l[i] = cs.M[(size_t)i * K + j] / dj;
        __syncthreads();
        const int rows = K - j - 1, cols = K - j;
        for (int e = tid; e < rows * cols; e += NT) {
            const int i = j + 1 + e / cols, k = j + e % cols;
            cs.M[(size_t)i * K + k] -= cs.l[i] * cs.M[(size_t)j * K + k];
        }
        for (int i = j + 1 + tid; i < K; i += NT) cs.r[i] -= cs.l[i] * cs.r[j];
        __syncthreads();
    }
    // back substitution by one warp (u reused for the solution)
    if (*bad < 0 && warp == 0) {
        for (int i = K - 1; i >= 0; --i) {
            double s = 0.0;
            for (int k = i + 1 + lane; k < K; k += 32) s = fma(cs.M[(size_t)i * K + k], cs.u[k], s);
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) cs.u[i] = (cs.r[i] - s) / cs.M[(size_t)i * K + i];
            __syncwarp();
        }
    }
    __syncthreads();
    for (int i = tid; i < K; i += NT) out[i] = *bad < 0 ? cs.u[i] : 0.0;
    __syncthreads();
    return *bad;
}

}  // namespace psl1
