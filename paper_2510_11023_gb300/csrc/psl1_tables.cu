// psl1_tables.cu -- set-up kernels: Gauss-Legendre quadrature, sine/cosine
// tables of the 1D sine basis, per-instance constants and L1 weight tables.
#include "psl1_device.cuh"
#include "psl1_kernels.h"

namespace psl1 {

// Gauss-Legendre on (lo, hi): Newton's method on P_Q (three-term recurrence)
// from the Tricomi-type start cos(pi (i + 3/4) / (Q + 1/2)); only the Qh
// nodes left of the midpoint are stored (their mirrors are lo + hi - x).
__global__ void k_gauss_legendre_half(int Q, double lo, double hi, double* xh, double* wh)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;   // descending-root index
    if (i >= Q) return;
    int p = Q - 1 - i;                                // ascending position
    int Qh = Q / 2;
    if (p >= Qh) return;
    double xi = cospi((i + 0.75) / (Q + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
        double p0 = 1.0, p1 = xi;
        for (int k = 2; k <= Q; ++k) {
            double p2 = ((2.0 * k - 1.0) * xi * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = Q * (xi * p1 - p0) / (xi * xi - 1.0);
        double dx = p1 / dp;
        xi -= dx;
        if (fabs(dx) < 1e-16) break;
    }
    {
        double p0 = 1.0, p1 = xi;
        for (int k = 2; k <= Q; ++k) {
            double p2 = ((2.0 * k - 1.0) * xi * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = Q * (xi * p1 - p0) / (xi * xi - 1.0);
    }
    double L = hi - lo;
    xh[p] = lo + 0.5 * L * (1.0 + xi);
    wh[p] = 0.5 * L * 2.0 / ((1.0 - xi * xi) * dp * dp);
}

// Basis tables for one (Mx, Qx, box): St[k][q], S[q][k] = sqrt(2/L) sin(k pi th_q),
// C[q][s] = cos(s pi th_q), Dt[k][q] = sqrt(2/L) (k pi/L) cos(k pi th_q) (the
// derivative), th_q = (x_q - lo)/L, and the node functions of the coefficient
// families at x_q and its mirror.
__global__ void k_basis_tables(int Mx, int Qh, double lo, double hi, const double* xh, double* St,
                               double* S, double* C, double* aux, df* Std, df* Sd, df* Cd, double* Dt,
                               df* Dtd, float* St32, float* Dt32, double* aux2, const double* wh, df* Wd,
                               df* auxd, df* aux2d, float* S32, float* C32)
{
    int q = blockIdx.x;
    if (q >= Qh) return;
    double L = hi - lo;
    double th = (xh[q] - lo) / L;
    double sc = sqrt(2.0 / L);
    for (int k = threadIdx.x + 1; k <= Mx; k += blockDim.x) {
        double v = sc * sinpi(k * th);
        double dv = sc * (k * 3.141592653589793 / L) * cospi(k * th);   // phi_k'(x_q)
        St[(size_t)(k - 1) * Qh + q] = v;
        S[(size_t)q * Mx + (k - 1)] = v;
        Std[(size_t)(k - 1) * Qh + q] = df_from_double(v);
        Sd[(size_t)q * Mx + (k - 1)] = df_from_double(v);
        Dt[(size_t)(k - 1) * Qh + q] = dv;
        Dtd[(size_t)(k - 1) * Qh + q] = df_from_double(dv);
        St32[(size_t)(k - 1) * Qh + q] = (float)v;
        Dt32[(size_t)(k - 1) * Qh + q] = (float)dv;
        S32[(size_t)q * Mx + (k - 1)] = (float)v;
    }
    for (int s = threadIdx.x; s <= 2 * Mx; s += blockDim.x) {
        double v = cospi(s * th);
        C[(size_t)q * (2 * Mx + 1) + s] = v;
        Cd[(size_t)q * (2 * Mx + 1) + s] = df_from_double(v);
        C32[(size_t)q * (2 * Mx + 1) + s] = (float)v;
    }
    if (threadIdx.x == 0) {
        double xa = xh[q], xb = lo + hi - xh[q];
        aux[4 * q + 0] = sinpi(xa);
        aux[4 * q + 1] = sinpi(2.0 * xa);
        aux[4 * q + 2] = sinpi(xb);
        aux[4 * q + 3] = sinpi(2.0 * xb);
        aux2[2 * q + 0] = cospi(2.0 * xa);
        aux2[2 * q + 1] = cospi(2.0 * xb);
        for (int i = 0; i < 4; ++i) auxd[4 * q + i] = df_from_double(aux[4 * q + i]);
        aux2d[2 * q + 0] = df_from_double(aux2[2 * q + 0]);
        aux2d[2 * q + 1] = df_from_double(aux2[2 * q + 1]);
        Wd[q] = df_from_double(wh[q]);
    }
}

// b(x) = (x+1)^{1-a} - x^{1-a}, b(0) = 1  (Eq. L1Scheme; real index as in Eq. L1Fine)
__device__ __forceinline__ double l1w(double a, double x)
{
    if (x == 0.0) return 1.0;
    return pow(x + 1.0, 1.0 - a) - pow(x, 1.0 - a);
}

// Per-instance constants and weight tables.  One CTA per instance.
__global__ void k_weights(InstDev* inst, double* bpool, df* bpool_df)
{
    InstDev& I = inst[blockIdx.x];
    double a = I.alpha;
    if (threadIdx.x == 0) {
        double g2 = tgamma(2.0 - a);
        I.mu = pow(I.dt, a) * g2;
        I.muT = pow(I.dT, a) * g2;
        I.ma = pow((double)I.m, -a);
        I.g1a = tgamma(1.0 + a);
        I.g3a = tgamma(3.0 - a);
    }
    double ma = pow((double)I.m, -a);
    double* bF = bpool + I.oB;
    double* bC = bF + I.Nb + 1;
    df* bFd = bpool_df + I.oB;
    df* bCd = bFd + I.Nb + 1;
    for (int j = threadIdx.x; j <= I.Nb; j += blockDim.x) {
        bF[j] = l1w(a, (double)j);
        bFd[j] = df_from_double(bF[j]);
    }
    // bC[d*m + (r-1)] = m^-a b(d + r/m)
    for (int e = threadIdx.x; e < I.P * I.m; e += blockDim.x) {
        int d = e / I.m, r = e % I.m + 1;
        bC[e] = ma * l1w(a, (double)d + (double)r / I.m);
        bCd[e] = df_from_double(bC[e]);
    }
}

cudaError_t launch_tables(const TableJob& job, cudaStream_t s)
{
    int Q = 2 * job.Qh;
    k_gauss_legendre_half<<<(Q + 127) / 128, 128, 0, s>>>(Q, job.lo, job.hi, job.xh, job.wh);
    k_basis_tables<<<job.Qh, 128, 0, s>>>(job.Mx, job.Qh, job.lo, job.hi, job.xh, job.St, job.S, job.C,
                                          job.aux, reinterpret_cast<df*>(job.Std), reinterpret_cast<df*>(job.Sd),
                                          reinterpret_cast<df*>(job.Cd), job.Dt, reinterpret_cast<df*>(job.Dtd),
                                          reinterpret_cast<float*>(job.St32), reinterpret_cast<float*>(job.Dt32),
                                          job.aux2, job.wh, reinterpret_cast<df*>(job.Wd),
                                          reinterpret_cast<df*>(job.auxd), reinterpret_cast<df*>(job.aux2d),
                                          reinterpret_cast<float*>(job.S32), reinterpret_cast<float*>(job.C32));
    return cudaGetLastError();
}

cudaError_t launch_weights(InstDev* inst, int B, double* bpool, double* bpool_df, cudaStream_t s)
{
    k_weights<<<B, 256, 0, s>>>(inst, bpool, reinterpret_cast<df*>(bpool_df));
    return cudaGetLastError();
}

}  // namespace psl1
