// psl1_api.cu -- C ABI (include/psl1.h): problem set-up, device pools, and
// the host drivers of the serial solvers and of the parareal iteration.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "psl1.h"
#include "psl1_kernels.h"
#include "psl1_soe.h"
#include "psl1_tc.h"

using namespace psl1;

namespace {

thread_local std::string g_create_error;

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

// w_q D_q (FP32, padded to Qpad) from nodal D (FP64) and the unfolded weights
__global__ void k_tc_weights(const double* D, const float* w, int units, int Q, int Qpad, float* wD)
{
    const long long n = (long long)units * Qpad;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int u = (int)(e / Qpad), q = (int)(e % Qpad);
        wD[e] = q < Q ? (float)((double)w[q] * D[(size_t)u * Q + q]) : 0.f;
    }
}

}  // namespace

struct psl1_problem {
    int B = 0, P = 0, prec = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<psl1_instance> desc;
    std::vector<InstDev> inst;
    std::vector<TabDev> tabs;
    std::string err;
    int nsm = 0;
    int max_smem = 0;        // opt-in shared memory per CTA
    // sizes
    long long sumK = 0, sumU = 0, sumPK = 0, sumB = 0, sumNK = 0, tabElems = 0;
    int Kmax = 0, Kpmax = 0, Qhmax = 0, mmax = 0, Nmax = 0;
    // device pools
    std::vector<void*> allocs;
    InstDev* d_inst = nullptr;
    TabDev* d_tab = nullptr;
    double *d_tp = nullptr, *d_bp = nullptr, *d_bpd = nullptr, *d_dud = nullptr, *d_u0 = nullptr, *d_hc = nullptr;
    double *d_Ua = nullptr, *d_Ub = nullptr, *d_Us = nullptr, *d_Fv = nullptr, *d_Gold = nullptr;
    double *d_incr = nullptr, *d_work = nullptr, *d_ring = nullptr, *d_corr = nullptr;
    int *d_nfirst = nullptr, *d_active = nullptr, *d_counter = nullptr;
    int* d_gmode = nullptr;
    int* d_order = nullptr;   // instance order of the coarse sweep (B) and of the serial solver (B)   // per instance: the stored G_old values are FP32-step values
    int2* d_units = nullptr;
    int nunits = 0;
    DevStatus* d_status = nullptr;
    double* d_flops = nullptr;   // algorithmic FLOP accumulators: F stage, coarse, serial, pieces
    double* d_noalloc = nullptr;  // device address of the library's fixed scratch array (not owned)
    double* d_cheb = nullptr;     // collocation pool: per instance nodes, sines and derivative matrix
    int fgrid = 0;                // F-stage CTAs chosen by psl1_autotune (0: one per slot)
    double *d_bcc = nullptr, *d_bccd = nullptr;   // coarse-substep weights (FP64, double-float)
    size_t bcc_cap = 0;
    // uniform solver pools (lazy)
    double *d_Wcur = nullptr, *d_dW = nullptr, *d_part = nullptr;
    int uni_chunk = 32, uni_maxchunks = 0;   // history rows per CTA of k_uni_hist (autotuned)
    cudaGraphExec_t uni_graph = nullptr;   // the uniform solver's N-step launch sequence
    // fast (sum-of-exponentials) uniform history (lazy)
    double *d_soe = nullptr, *d_Y = nullptr;
    long long sumY = 0;
    cudaGraphExec_t soe_graph = nullptr;
    std::vector<std::vector<double>> soe_s, soe_w;
    // graph-mode parareal (device-driven while loop)
    bool graph_mode = false;
    cudaGraphExec_t par_graph = nullptr;
    int *d_iters = nullptr, *d_kstate = nullptr;
    double *d_errlog = nullptr, *d_tol = nullptr;
    PathArgs pa{};
    // state
    bool u0_set = false, par_done = false, ser_done = false;
    int ser_kind = -1;           // kind of the last serial solve
    double* d_Ucur = nullptr;   // buffer holding the current parareal iterate
    std::vector<int> iters;
    std::vector<std::vector<double>> errlog;
    bool keep_iterates = false;
    std::vector<std::vector<double>> iterates;
    psl1_stats stats{};
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
};

static psl1_status fail(psl1_problem* h, psl1_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (h)
        h->err = buf;
    else
        g_create_error = buf;
    return st;
}

#define CU(h, call)                                                                                  \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess)                                                                       \
            return fail((h), PSL1_ERR_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                        __FILE__, __LINE__);                                                         \
    } while (0)

template <typename T>
static psl1_status dalloc(psl1_problem* h, T** p, size_t count)
{
    if (count == 0) count = 1;
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, count * sizeof(T));
    if (e != cudaSuccess)
        return fail(h, PSL1_ERR_NOMEM, "cudaMalloc of %zu bytes failed: %s", count * sizeof(T),
                    cudaGetErrorString(e));
    h->allocs.push_back(q);
    *p = static_cast<T*>(q);
    return PSL1_OK;
}

#define TRY(x)                       \
    do {                             \
        psl1_status s_ = (x);        \
        if (s_ != PSL1_OK) return s_; \
    } while (0)

static psl1_status check_device_status(psl1_problem* h)
{
    DevStatus st{};
    CU(h, cudaMemcpyAsync(&st, h->d_status, sizeof st, cudaMemcpyDeviceToHost, h->stream));
    CU(h, cudaStreamSynchronize(h->stream));
    if (st.code != 0) {
        const char* what = st.code == PSL1_ERR_NOT_SPD ? "non-positive Cholesky pivot (D <= 0?)"
                           : st.code == PSL1_ERR_NONFINITE ? "non-finite value"
                                                           : "device error";
        return fail(h, (psl1_status)st.code, "%s in instance %d (stage %d, step %d)", what, st.inst, st.where,
                    st.info);
    }
    return PSL1_OK;
}

static psl1_status reset_status(psl1_problem* h)
{
    CU(h, cudaMemsetAsync(h->d_status, 0, sizeof(DevStatus), h->stream));
    if (h->d_flops) CU(h, cudaMemsetAsync(h->d_flops, 0, 4 * sizeof(double), h->stream));
    return PSL1_OK;
}

// Copy the device FLOP accumulators into the statistics (after a synchronising call).
static psl1_status read_flops(psl1_problem* h)
{
    double f[4] = {0, 0, 0, 0};
    CU(h, cudaMemcpyAsync(f, h->d_flops, sizeof f, cudaMemcpyDeviceToHost, h->stream));
    CU(h, cudaStreamSynchronize(h->stream));
    h->stats.flop_fine = f[0];
    h->stats.flop_coarse = f[1];
    h->stats.flop_serial = f[2];
    return PSL1_OK;
}

static bool finite_all(const double* p, int n)
{
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

extern "C" {

const char* psl1_last_error(psl1_h h) { return h ? h->err.c_str() : g_create_error.c_str(); }

void psl1_destroy(psl1_h h)
{
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->uni_graph) cudaGraphExecDestroy(h->uni_graph);
    if (h->soe_graph) cudaGraphExecDestroy(h->soe_graph);
    if (h->par_graph) cudaGraphExecDestroy(h->par_graph);
    for (void* p : h->allocs) cudaFree(p);
    for (auto& e : h->ev)
        if (e) cudaEventDestroy(e);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

// dpar / fpar as (hi, lo) float pairs for the double-float evaluation, and
// whether f can be evaluated in double-float (no manufactured source)
static void family_copies(InstDev& I)
{
    for (int i = 0; i < 8; ++i) {
        float h = (float)I.dpar[i];
        I.dpf[2 * i] = h;
        I.dpf[2 * i + 1] = (float)(I.dpar[i] - (double)h);
        h = (float)I.fpar[i];
        I.fpf[2 * i] = h;
        I.fpf[2 * i + 1] = (float)(I.fpar[i] - (double)h);
    }
    I.f_df = (I.fpar[4] == 0.0 && I.fpar[5] == 0.0) ? 1 : 0;
}

// Chebyshev-Lobatto collocation data of n intervals on [a, b] (Sec. 4.1), appended
// to pool: nodes x_j = (a+b)/2 + (b-a)/2 cos(j pi/n), sin(pi x_j), sin(2 pi x_j), and
// the first-derivative matrix scaled by 2/(b-a) with the entries the paper gives,
//   D_ij = (c_i/c_j) (-1)^{i+j} / (xi_i - xi_j),  c_0 = c_n = 2, else 1,
//   D_00 = (2n^2+1)/6,  D_nn = -(2n^2+1)/6,  D_jj = -xi_j / (2 (1 - xi_j^2)),
// where xi_i - xi_j = -2 sin((i+j) pi/2n) sin((i-j) pi/2n) and 1 - xi_j^2 =
// sin^2(j pi/n) are taken in these trigonometric forms (no cancellation).
static void cheb_tables(int n, double a, double b, std::vector<double>& pool)
{
    const int Q = n + 1;
    const size_t o = pool.size();
    pool.resize(o + 3 * (size_t)Q + (size_t)Q * Q);
    double* x = pool.data() + o;
    double* s1 = x + Q;
    double* s2 = s1 + Q;
    double* D = s2 + Q;
    const double h = M_PI / n, sc = 2.0 / (b - a);
    for (int j = 0; j < Q; ++j) {
        x[j] = 0.5 * (a + b) + 0.5 * (b - a) * std::cos(j * h);
        s1[j] = std::sin(M_PI * x[j]);
        s2[j] = std::sin(2.0 * M_PI * x[j]);
    }
    for (int i = 0; i < Q; ++i)
        for (int j = 0; j < Q; ++j) {
            double v;
            if (i == j) {
                if (i == 0)
                    v = (2.0 * n * n + 1.0) / 6.0;
                else if (i == n)
                    v = -(2.0 * n * n + 1.0) / 6.0;
                else {
                    const double sn = std::sin(i * h);
                    v = -std::cos(i * h) / (2.0 * sn * sn);
                }
            } else {
                const double ci = (i == 0 || i == n) ? 2.0 : 1.0, cj = (j == 0 || j == n) ? 2.0 : 1.0;
                const double diff = -2.0 * std::sin(0.5 * (i + j) * h) * std::sin(0.5 * (i - j) * h);
                v = (ci / cj) * (((i + j) & 1) ? -1.0 : 1.0) / diff;
            }
            D[(size_t)i * Q + j] = sc * v;
        }
}

static psl1_status validate(const psl1_instance& d, int P, int b)
{
    if (d.dim != 1 && d.dim != 2) return fail(nullptr, PSL1_ERR_ARG, "instance %d: dim must be 1 or 2", b);
    if (d.basis != PSL1_BASIS_SINE && d.basis != PSL1_BASIS_CHEB)
        return fail(nullptr, PSL1_ERR_ARG, "instance %d: unknown basis %d", b, d.basis);
    if (d.basis == PSL1_BASIS_CHEB && (d.dim != 1 || d.modes[0] < 2 || d.modes[0] > CHEB_NMAX))
        return fail(nullptr, PSL1_ERR_ARG, "instance %d: collocation needs dim 1 and 2 <= intervals <= %d", b,
                    CHEB_NMAX);
    const int mmax = d.dim == 1 ? KMAX_1D : MMAX_2D;
    for (int ax = 0; ax < d.dim; ++ax) {
        int M = d.modes[ax];
        if (M < 1 || M > mmax)
            return fail(nullptr, PSL1_ERR_ARG, "instance %d: modes[%d] = %d outside [1,%d]", b, ax, M, mmax);
        int Q = d.qnodes[ax] ? d.qnodes[ax] : 2 * M;
        if (Q < 2 || (Q & 1) || Q > 4 * mmax)
            return fail(nullptr, PSL1_ERR_ARG, "instance %d: quadrature nodes[%d] = %d must be even in [2,%d]", b, ax,
                        Q, 4 * mmax);
        if (!(d.hi[ax] > d.lo[ax]) || !std::isfinite(d.lo[ax]) || !std::isfinite(d.hi[ax]))
            return fail(nullptr, PSL1_ERR_ARG, "instance %d: empty domain along axis %d", b, ax);
    }
    if (d.nsteps < P || d.nsteps % P)
        return fail(nullptr, PSL1_ERR_ARG, "instance %d: nsteps %d must be a positive multiple of P=%d", b, d.nsteps, P);
    if (!(d.alpha > 0.0 && d.alpha <= 1.0)) return fail(nullptr, PSL1_ERR_ARG, "instance %d: alpha must be in (0,1]", b);
    if (!(d.T > 0.0) || !std::isfinite(d.T)) return fail(nullptr, PSL1_ERR_ARG, "instance %d: T must be > 0", b);
    if (!(d.hi[0] > d.lo[0]) || !std::isfinite(d.lo[0]) || !std::isfinite(d.hi[0]))
        return fail(nullptr, PSL1_ERR_ARG, "instance %d: empty domain", b);
    if (!finite_all(d.dpar, 8) || !finite_all(d.fpar, 8))
        return fail(nullptr, PSL1_ERR_ARG, "instance %d: non-finite coefficient parameters", b);
    return PSL1_OK;
}

// 2D: the layout of one CTA of a cluster of `split` CTAs that shares each coarse-sweep
// step (each CTA holds the node columns of ceil(Qhy / split) y pairs)
static Layout2D split_layout(const psl1_problem* h, int split)
{
    long long nT = 0, nN = 0, ntab = 0;
    for (const InstDev& I : h->inst) {
        const long long nq = (I.Qhy + split - 1) / split;
        nT = std::max(nT, (long long)I.Mx * (2 * nq + 1));
        nN = std::max(nN, (long long)I.Q * 2 * nq);
        ntab = std::max(ntab, (long long)I.Mx * I.Qh + (long long)I.My * I.Qhy);
    }
    return make_layout2d(h->prec, h->Kmax, nT, nN, ntab, h->max_smem - 1024, split);
}

// Use clusters of `split` CTAs for the 2D coarse sweep, if that configuration can run
// (its arrays fit the slot workspace, B split CTAs have slots, and the device can
// hold at least one such cluster); otherwise one CTA per instance.  Returns whether
// the requested setting was applied.
static bool apply_split(psl1_problem* h, int split)
{
    h->pa.split2d = 1;
    if (!h->pa.dim2 || split < 2) return split <= 1;
    const Layout2D L = split_layout(h, split);
    if (L.smem > h->max_smem - 1024 || L.gbytes > 8 * h->pa.work_stride || (long long)h->B * split > h->pa.nslots)
        return false;
    PathArgs t = h->pa;
    t.L2s = L;
    if (coarse_sweep_clusters(t, split) < 1) return false;
    h->pa.L2s = L;
    h->pa.split2d = split;
    return true;
}

// the automatic choice: the largest power of two <= 8 that leaves every instance's
// cluster room on the SMs (none once the batch alone fills them)
static void auto_split(psl1_problem* h)
{
    h->pa.split2d = 1;
    if (!h->pa.dim2) return;
    for (int c = 8; c >= 2; c /= 2)
        if ((long long)h->B * c <= h->nsm && apply_split(h, c)) return;
}

psl1_status psl1_create(psl1_h* out, int batch, const psl1_instance* in, int P, int precision, void* stream)
{
    if (!out) return fail(nullptr, PSL1_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (batch < 1 || !in) return fail(nullptr, PSL1_ERR_ARG, "batch must be >= 1 with an instance array");
    if (P < 1) return fail(nullptr, PSL1_ERR_ARG, "P must be >= 1");
    if (precision != PSL1_PREC_FP64 && precision != PSL1_PREC_MIXED && precision != PSL1_PREC_FP32)
        return fail(nullptr, PSL1_ERR_ARG, "unknown precision %d", precision);
    for (int b = 0; b < batch; ++b) TRY(validate(in[b], P, b));
    for (int b = 0; b < batch; ++b)
        if (in[b].basis == PSL1_BASIS_CHEB && precision != PSL1_PREC_FP64)
            return fail(nullptr, PSL1_ERR_ARG, "instance %d: the collocation scheme runs in PSL1_PREC_FP64", b);
    for (int b = 1; b < batch; ++b)
        if (in[b].dim != in[0].dim)
            return fail(nullptr, PSL1_ERR_ARG, "instance %d: all instances of a handle must have the same dim", b);
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev < 1)
        return fail(nullptr, PSL1_ERR_CUDA, "no usable CUDA device: %s", cudaGetErrorString(e));

    psl1_problem* h = new psl1_problem();
    h->B = batch;
    h->P = P;
    h->prec = precision;
    h->desc.assign(in, in + batch);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, dev);
    if (stream) {
        h->stream = (cudaStream_t)stream;
    } else {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete h;
            return fail(nullptr, PSL1_ERR_CUDA, "stream creation failed");
        }
        h->own_stream = true;
    }
    auto bail = [&](psl1_status st) {
        g_create_error = h->err;
        psl1_destroy(h);
        return st;
    };
#define CTRY(x)                                 \
    do {                                        \
        psl1_status s_ = (x);                   \
        if (s_ != PSL1_OK) return bail(s_);     \
    } while (0)

    // tables shared by instances (and axes) with the same (M, Q, interval)
    std::map<std::tuple<int, int, double, double>, int> tabid;
    std::vector<TableJob> jobs;
    auto table_for = [&](int M, int Q, double lo, double hi) {
        auto key = std::make_tuple(M, Q, lo, hi);
        auto it = tabid.find(key);
        if (it != tabid.end()) return it->second;
        TabDev t{};
        t.Mx = M;
        t.Qx = Q;
        t.Qh = Q / 2;
        long long o = h->tabElems;
        const long long mq = (long long)t.Mx * t.Qh;
        t.oX = o;
        o += t.Qh;
        t.oWq = o;
        o += t.Qh;
        t.oAux = o;
        o += 4LL * t.Qh;
        t.oSt = o;
        o += mq;
        t.oS = o;
        o += mq;
        t.oC = o;
        o += (long long)t.Qh * (2 * t.Mx + 1);
        t.oStd = o;
        o += mq;
        t.oSd = o;
        o += mq;
        t.oCd = o;
        o += (long long)t.Qh * (2 * t.Mx + 1);
        t.oDt = o;
        o += mq;
        t.oDtd = o;
        o += mq;
        t.oSt32 = o;
        o += (mq + 1) / 2;
        t.oDt32 = o;
        o += (mq + 1) / 2;
        t.oAux2 = o;
        o += 2LL * t.Qh;
        t.oWd = o;
        o += t.Qh;
        t.oAuxd = o;
        o += 4LL * t.Qh;
        t.oAux2d = o;
        o += 2LL * t.Qh;
        t.oS32 = o;
        o += (mq + 1) / 2;
        t.oC32 = o;
        o += ((long long)t.Qh * (2 * t.Mx + 1) + 1) / 2;
        h->tabElems = o;
        int id = (int)h->tabs.size();
        h->tabs.push_back(t);
        tabid[key] = id;
        TableJob j{};
        j.Mx = t.Mx;
        j.Qh = t.Qh;
        j.lo = lo;
        j.hi = hi;
        jobs.push_back(j);
        return id;
    };
    h->inst.resize(batch);
    long long nT2 = 0, nN2 = 0, ntab2 = 0;
    std::vector<double> cheb_pool;
    int Kc = 0;
    for (int b = 0; b < batch; ++b) {
        const psl1_instance& d = in[b];
        InstDev& I = h->inst[b];
        memset(&I, 0, sizeof I);
        I.dim = d.dim;
        I.basis = d.basis;
        I.inner_rtol = INNER_RTOL_DEFAULT;
        I.mc = 1;
        I.Mx = d.modes[0];
        I.My = d.dim == 2 ? d.modes[1] : 1;
        I.K = I.basis == PSL1_BASIS_CHEB ? I.Mx - 1 : I.Mx * I.My;
        I.nb = (I.K + TILE - 1) / TILE;
        I.Kp = I.nb * TILE;
        I.Q = d.qnodes[0] ? d.qnodes[0] : 2 * I.Mx;
        I.Qh = I.Q / 2;
        I.Qy = d.dim == 2 ? (d.qnodes[1] ? d.qnodes[1] : 2 * I.My) : 1;
        I.Qhy = I.Qy / 2;
        I.N = d.nsteps;
        I.P = P;
        I.m = I.N / P;
        I.alpha = d.alpha;
        I.T = d.T;
        I.dT = d.T / P;
        I.dt = d.T / I.N;
        I.lo0 = d.lo[0];
        I.hi0 = d.hi[0];
        double L = I.hi0 - I.lo0;
        I.cA = M_PI * M_PI / (L * L * L);
        for (int i = 0; i < 8; ++i) {
            I.dpar[i] = d.dpar[i];
            I.fpar[i] = d.fpar[i];
        }
        family_copies(I);
        I.tab = table_for(I.Mx, I.Q, I.lo0, I.hi0);
        if (I.dim == 2) {
            I.lo1 = d.lo[1];
            I.hi1 = d.hi[1];
            I.tabY = table_for(I.My, I.Qy, I.lo1, I.hi1);
            nT2 = std::max(nT2, (long long)I.Mx * (I.Qy + 1));
            nN2 = std::max(nN2, (long long)I.Q * I.Qy);
            ntab2 = std::max(ntab2, (long long)I.Mx * I.Qh + (long long)I.My * I.Qhy);
        } else {
            I.tabY = I.tab;
        }
        if (I.basis == PSL1_BASIS_CHEB) {   // nodes, sin(pi x), sin(2 pi x), derivative matrix
            I.oC = (long long)cheb_pool.size();
            cheb_tables(I.Mx, I.lo0, I.hi0, cheb_pool);
            Kc = std::max(Kc, I.K);
        }
        I.Nb = std::max(std::max(I.N, P), I.m) + 1;
        I.oK = h->sumK;
        h->sumK += I.K;
        I.oU = h->sumU;
        h->sumU += (long long)(P + 1) * I.K;
        I.oPK = h->sumPK;
        h->sumPK += (long long)P * I.K;
        I.oB = h->sumB;
        h->sumB += (I.Nb + 1) + (long long)P * I.m;
        I.oW = h->sumNK;
        h->sumNK += (long long)I.N * I.K;
        h->Kmax = std::max(h->Kmax, I.K);
        h->Kpmax = std::max(h->Kpmax, I.Kp);
        h->Qhmax = std::max(h->Qhmax, I.Qh);
        h->mmax = std::max(h->mmax, I.m);
        h->Nmax = std::max(h->Nmax, I.N);
    }
    int nbmax = h->Kpmax / TILE;
    int nslots = std::max(4 * h->nsm, batch);   // up to four F-stage CTAs per SM (autotuned)
    int max_smem = 0;
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    h->max_smem = max_smem;
    const bool two_d = in[0].dim == 2;
    SmemLayout lay{};
    Layout2D lay2{};
    if (two_d) {
        lay2 = make_layout2d(precision, h->Kmax, nT2, nN2, ntab2, max_smem - 1024);
        lay.total = lay2.smem;
        lay.fine = lay2.smem;
    } else {
        lay = make_layout(precision, h->Kmax, h->Kpmax, h->Qhmax, Kc);
    }
    if (lay.total > max_smem - 1024) {
        g_create_error = "instance too large for the shared-memory layout";
        psl1_destroy(h);
        return PSL1_ERR_ARG;
    }
    CTRY(dalloc(h, &h->d_inst, batch));
    CTRY(dalloc(h, &h->d_tab, h->tabs.size()));
    CTRY(dalloc(h, &h->d_tp, h->tabElems));
    CTRY(dalloc(h, &h->d_bp, h->sumB));
    CTRY(dalloc(h, &h->d_bpd, h->sumB));   // double-float pairs, 8 bytes each
    CTRY(dalloc(h, &h->d_u0, h->sumK));
    CTRY(dalloc(h, &h->d_Ua, h->sumU));
    CTRY(dalloc(h, &h->d_Ub, h->sumU));
    CTRY(dalloc(h, &h->d_Us, h->sumU));
    CTRY(dalloc(h, &h->d_Fv, h->sumPK));
    CTRY(dalloc(h, &h->d_Gold, h->sumPK));
    CTRY(dalloc(h, &h->d_incr, batch));
    CTRY(dalloc(h, &h->d_nfirst, batch));
    CTRY(dalloc(h, &h->d_active, batch));
    CTRY(dalloc(h, &h->d_counter, 1));
    CTRY(dalloc(h, &h->d_gmode, batch));
    if (cudaMemset(h->d_gmode, 0, sizeof(int) * batch) != cudaSuccess) {
        g_create_error = "cudaMemset failed";
        psl1_destroy(h);
        return PSL1_ERR_CUDA;
    }
    CTRY(dalloc(h, &h->d_status, 1));
    CTRY(dalloc(h, &h->d_flops, 4));
    if (!cheb_pool.empty()) CTRY(dalloc(h, &h->d_cheb, cheb_pool.size()));
    // per-slot workspace: the FP64 1D factor, or the 2D working arrays that do not fit in shared memory
    long long gb2 = lay2.gbytes;   // 2D: also room for the arrays of a cluster-split sweep CTA
    for (int c = 2; two_d && c <= 8; c *= 2) gb2 = std::max(gb2, split_layout(h, c).gbytes);
    long long work_stride = two_d ? std::max(1LL, (gb2 + 255) / 256 * 32)   // 256-byte aligned slots
                            : precision == PSL1_PREC_FP64 ? bp_elems(nbmax, TILE)
                            : 1;
    long long ring_stride = (long long)h->mmax * h->Kmax;
    CTRY(dalloc(h, &h->d_work, (size_t)nslots * work_stride));
    CTRY(dalloc(h, &h->d_ring, (size_t)nslots * ring_stride));
    CTRY(dalloc(h, &h->d_corr, (size_t)nslots * h->Kmax));
    // mixed-path coarse differences (double-float, 8 bytes per entry)
    long long dud_stride = precision == PSL1_PREC_FP64 ? 0 : (long long)P * h->Kmax;
    if (dud_stride) CTRY(dalloc(h, &h->d_dud, (size_t)nslots * dud_stride));
    // coarse-history terms of a slice's steps (double-float, 8 bytes per entry)
    long long hc_stride = precision == PSL1_PREC_FP64 ? 0 : (long long)h->mmax * h->Kmax;
    if (hc_stride) CTRY(dalloc(h, &h->d_hc, (size_t)nslots * hc_stride));
    // fine units, longest first (cost ~ m K^3)
    std::vector<int2> units;
    for (int b = 0; b < batch; ++b)
        for (int n = 0; n < P; ++n) units.push_back(make_int2(b, n));
    std::stable_sort(units.begin(), units.end(), [&](int2 x, int2 y) {
        const InstDev &a = h->inst[x.x], &c = h->inst[y.x];
        // cost per step: K^3 (1D), K (Qx + Qy) per operator application (2D)
        auto cost = [](const InstDev& I) {
            return I.dim == 2 ? (double)I.m * I.K * (I.Q + I.Qy) : (double)I.m * I.K * I.K * I.K;
        };
        double ca = cost(a), cc = cost(c);
        return ca > cc;
    });
    h->nunits = (int)units.size();
    CTRY(dalloc(h, &h->d_units, units.size()));
    // One CTA (or cluster) per instance runs each sequential chain: the coarse sweep
    // (P coarse steps, cost ~ K^3 or K (Qx + Qy) per step) and the serial solver (N fine
    // steps).  Launched longest first, the longest chains start on SMs of their own;
    // with more instances than SMs the shorter ones share.
    std::vector<int> order(2 * (size_t)batch);
    for (int b = 0; b < batch; ++b) order[b] = order[batch + b] = b;
    auto step_cost = [](const InstDev& I) {
        return I.dim == 2 ? (double)I.K * (I.Q + I.Qy) : (double)I.K * I.K * I.K;
    };
    std::stable_sort(order.begin(), order.begin() + batch, [&](int x, int y) {
        return step_cost(h->inst[x]) > step_cost(h->inst[y]);
    });
    std::stable_sort(order.begin() + batch, order.end(), [&](int x, int y) {
        return h->inst[x].N * step_cost(h->inst[x]) > h->inst[y].N * step_cost(h->inst[y]);
    });
    CTRY(dalloc(h, &h->d_order, order.size()));
    for (size_t t = 0; t < jobs.size(); ++t) {
        const TabDev& T = h->tabs[t];
        jobs[t].xh = h->d_tp + T.oX;
        jobs[t].wh = h->d_tp + T.oWq;
        jobs[t].aux = h->d_tp + T.oAux;
        jobs[t].St = h->d_tp + T.oSt;
        jobs[t].S = h->d_tp + T.oS;
        jobs[t].C = h->d_tp + T.oC;
        jobs[t].Std = h->d_tp + T.oStd;
        jobs[t].Sd = h->d_tp + T.oSd;
        jobs[t].Cd = h->d_tp + T.oCd;
        jobs[t].Dt = h->d_tp + T.oDt;
        jobs[t].Dtd = h->d_tp + T.oDtd;
        jobs[t].St32 = h->d_tp + T.oSt32;
        jobs[t].Dt32 = h->d_tp + T.oDt32;
        jobs[t].aux2 = h->d_tp + T.oAux2;
        jobs[t].Wd = h->d_tp + T.oWd;
        jobs[t].auxd = h->d_tp + T.oAuxd;
        jobs[t].aux2d = h->d_tp + T.oAux2d;
        jobs[t].S32 = h->d_tp + T.oS32;
        jobs[t].C32 = h->d_tp + T.oC32;
    }
    auto cu = [&](cudaError_t e2, const char* what) -> psl1_status {
        if (e2 != cudaSuccess) return fail(h, PSL1_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e2));
        return PSL1_OK;
    };
    CTRY(cu(cudaMemcpyAsync(h->d_inst, h->inst.data(), sizeof(InstDev) * batch, cudaMemcpyHostToDevice, h->stream),
            "copy instances"));
    CTRY(cu(cudaMemcpyAsync(h->d_tab, h->tabs.data(), sizeof(TabDev) * h->tabs.size(), cudaMemcpyHostToDevice,
                            h->stream), "copy tables"));
    CTRY(cu(cudaMemcpyAsync(h->d_units, units.data(), sizeof(int2) * units.size(), cudaMemcpyHostToDevice,
                            h->stream), "copy units"));
    CTRY(cu(cudaMemcpyAsync(h->d_order, order.data(), sizeof(int) * order.size(), cudaMemcpyHostToDevice,
                            h->stream), "copy instance order"));
    CTRY(cu(cudaMemsetAsync(h->d_status, 0, sizeof(DevStatus), h->stream), "status"));
    if (!cheb_pool.empty())
        CTRY(cu(cudaMemcpyAsync(h->d_cheb, cheb_pool.data(), sizeof(double) * cheb_pool.size(),
                                cudaMemcpyHostToDevice, h->stream), "copy collocation tables"));
    for (auto& j : jobs) CTRY(cu(launch_tables(j, h->stream), "table kernels"));
    CTRY(cu(launch_weights(h->d_inst, batch, h->d_bp, h->d_bpd, h->stream), "weight kernel"));
    // constants computed on the device (mu, muT, ...) are needed on the host copy too
    CTRY(cu(cudaMemcpyAsync(h->inst.data(), h->d_inst, sizeof(InstDev) * batch, cudaMemcpyDeviceToHost, h->stream),
            "read constants"));
    CTRY(cu(cudaStreamSynchronize(h->stream), "set-up"));
    for (auto& ev : h->ev) CTRY(cu(cudaEventCreate(&ev), "events"));
    // the allocation-free fine propagator's fixed array: its device address on this
    // device, looked up here so that psl1_fine_slice_noalloc needs no set-up
    CTRY(cu(noalloc_scratch_address(&h->d_noalloc), "address of the fixed scratch array"));

    PathArgs& a = h->pa;
    a.inst = h->d_inst;
    a.tab = h->d_tab;
    a.tp = h->d_tp;
    a.bp = h->d_bp;
    a.bpd = reinterpret_cast<const df*>(h->d_bpd);
    a.dud = reinterpret_cast<df*>(h->d_dud);
    a.dud_stride = dud_stride;
    a.hc = reinterpret_cast<df*>(h->d_hc);
    a.hc_stride = hc_stride;
    a.status = h->d_status;
    a.work = h->d_work;
    a.work_stride = work_stride;
    a.ring = h->d_ring;
    a.ring_stride = ring_stride;
    a.corr = h->d_corr;
    a.nslots = nslots;
    a.Kmax = h->Kmax;
    a.Kpmax = h->Kpmax;
    a.Qhmax = h->Qhmax;
    a.mmax = h->mmax;
    a.prec = precision;
    a.L = lay;
    a.flops = h->d_flops;
    a.flop_slot = 3;
    a.dim2 = two_d ? 1 : 0;
    a.L2 = lay2;
    a.incr = h->d_incr;
    a.loose_above = 0.0;
    a.refine_factor = 0.0;
    a.gmode = h->d_gmode;
    a.sweep_order = h->d_order;
    a.serial_order = h->d_order + batch;
    a.cheb = h->d_cheb;
    a.fstage_minb = 2;
    a.split2d = 1;
    auto_split(h);
    h->iters.assign(batch, 0);
    h->errlog.assign(batch, {});
    h->d_Ucur = h->d_Ua;
    *out = h;
    return PSL1_OK;
#undef CTRY
}

psl1_status psl1_set_D(psl1_h h, const double* dpar)
{
    if (!h || !dpar) return fail(h, PSL1_ERR_ARG, "NULL argument");
    if (!finite_all(dpar, 8 * h->B)) return fail(h, PSL1_ERR_ARG, "non-finite D parameters");
    for (int b = 0; b < h->B; ++b) {
        for (int i = 0; i < 8; ++i) h->inst[b].dpar[i] = h->desc[b].dpar[i] = dpar[8 * b + i];
        family_copies(h->inst[b]);
    }
    CU(h, cudaMemcpyAsync(h->d_inst, h->inst.data(), sizeof(InstDev) * h->B, cudaMemcpyHostToDevice, h->stream));
    CU(h, cudaStreamSynchronize(h->stream));
    return PSL1_OK;
}

psl1_status psl1_set_f(psl1_h h, const double* fpar)
{
    if (!h || !fpar) return fail(h, PSL1_ERR_ARG, "NULL argument");
    if (!finite_all(fpar, 8 * h->B)) return fail(h, PSL1_ERR_ARG, "non-finite f parameters");
    for (int b = 0; b < h->B; ++b) {
        for (int i = 0; i < 8; ++i) h->inst[b].fpar[i] = h->desc[b].fpar[i] = fpar[8 * b + i];
        family_copies(h->inst[b]);
    }
    CU(h, cudaMemcpyAsync(h->d_inst, h->inst.data(), sizeof(InstDev) * h->B, cudaMemcpyHostToDevice, h->stream));
    CU(h, cudaStreamSynchronize(h->stream));
    return PSL1_OK;
}

psl1_status psl1_set_u0(psl1_h h, const double* c)
{
    if (!h || !c) return fail(h, PSL1_ERR_ARG, "NULL argument");
    if (!finite_all(c, (int)h->sumK)) return fail(h, PSL1_ERR_NONFINITE, "u0 holds a non-finite value");
    CU(h, cudaMemcpyAsync(h->d_u0, c, sizeof(double) * h->sumK, cudaMemcpyHostToDevice, h->stream));
    CU(h, cudaStreamSynchronize(h->stream));
    h->u0_set = true;
    return PSL1_OK;
}

psl1_status psl1_set_u0_dev(psl1_h h, const double* c)
{
    if (!h || !c) return fail(h, PSL1_ERR_ARG, "NULL argument");
    CU(h, cudaMemcpyAsync(h->d_u0, c, sizeof(double) * h->sumK, cudaMemcpyDeviceToDevice, h->stream));
    h->u0_set = true;
    return PSL1_OK;
}

// candidate row chunks of the history stream (k_uni_hist), smallest first
static const int kUniChunks[] = {16, 32, 64, 128};

static psl1_status ensure_uniform_pools(psl1_problem* h)
{
    if (h->d_dW) return PSL1_OK;
    h->uni_maxchunks = (h->Nmax + kUniChunks[0] - 1) / kUniChunks[0];   // room for any candidate
    TRY(dalloc(h, &h->d_Wcur, h->sumK));
    TRY(dalloc(h, &h->d_dW, h->sumNK));
    TRY(dalloc(h, &h->d_part, (size_t)h->B * h->uni_maxchunks * h->Kmax));
    CU(h, cudaMemsetAsync(h->d_dW, 0, sizeof(double) * h->sumNK, h->stream));
    return PSL1_OK;
}

// Autotuning of the history stream: its row chunk sets the grid (chunks x
// instances CTAs) and so how much of HBM's latency is covered; the best value
// depends on the batch, K and N.  Every candidate is timed on the longest
// history launch (fine step Nmax - 1) after one warm-up launch, and the fastest
// is kept for the handle (the sums differ only in their association order).
static psl1_status tune_uniform_chunk(psl1_problem* h)
{
    const int j = h->Nmax - 1;
    if (j < 2) return PSL1_OK;
    float best = 0.f;
    int pick = h->uni_chunk;
    bool first = true;
    for (int c : kUniChunks) {
        CU(h, launch_uni_hist(h->pa, h->B, h->d_dW, j, h->d_part, c, h->uni_maxchunks, h->stream));
        CU(h, cudaEventRecord(h->ev[2], h->stream));
        CU(h, launch_uni_hist(h->pa, h->B, h->d_dW, j, h->d_part, c, h->uni_maxchunks, h->stream));
        CU(h, cudaEventRecord(h->ev[3], h->stream));
        CU(h, cudaEventSynchronize(h->ev[3]));
        float ms = 0.f;
        CU(h, cudaEventElapsedTime(&ms, h->ev[2], h->ev[3]));
        if (first || ms < best) {
            best = ms;
            pick = c;
            first = false;
        }
    }
    h->uni_chunk = pick;
    return PSL1_OK;
}

static double elapsed(cudaEvent_t a, cudaEvent_t b)
{
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    return ms;
}

static void count_work(psl1_problem* h, const std::vector<int>& nfirst, const std::vector<int>& active)
{
    for (int b = 0; b < h->B; ++b) {
        if (!active[b]) continue;
        const InstDev& I = h->inst[b];
        double steps = (double)(h->P - nfirst[b]) * I.m;
        h->stats.fine_steps += steps;
        h->stats.fine_step_modes += steps * I.K;
    }
}

// The uniform solver's launches: initial state, then per fine step j the
// history partial sums and the step (j = 0 has no history).
static cudaError_t enqueue_uniform(psl1_problem* h)
{
    cudaError_t e = launch_uni_init(h->pa, h->B, h->d_u0, h->d_Wcur, h->d_Us, h->stream);
    for (int j = 0; j < h->Nmax && e == cudaSuccess; ++j) {
        e = launch_uni_hist(h->pa, h->B, h->d_dW, j, h->d_part, h->uni_chunk, h->uni_maxchunks, h->stream);
        if (e == cudaSuccess)
            e = launch_uni_step(h->pa, h->B, h->d_Wcur, h->d_dW, h->d_Us, j, h->d_part, h->uni_chunk,
                                h->uni_maxchunks, h->stream);
    }
    return e;
}

// The fast uniform history: the exponentials of every instance (host, psl1_soe.cu),
// their device pool exp(-s), exp(-s nloc), w, and the L x K state of each instance.
static psl1_status ensure_soe_pools(psl1_problem* h)
{
    if (h->d_Y) return PSL1_OK;
    TRY(ensure_uniform_pools(h));
    std::vector<double> pool;
    h->soe_s.assign(h->B, {});
    h->soe_w.assign(h->B, {});
    long long oY = 0;
    for (int b = 0; b < h->B; ++b) {
        InstDev& I = h->inst[b];
        double sv[SOE_MAXL], wv[SOE_MAXL];
        const int L = soe_nodes(I.alpha, SOE_NLOC, I.N, SOE_EPS, SOE_MAXL, sv, wv);
        if (L < 0) return fail(h, PSL1_ERR_ARG, "instance %d: no fast-history exponentials", b);
        I.soeL = L;
        I.oS = (long long)pool.size();
        I.oY = oY;
        for (int i = 0; i < L; ++i) pool.push_back(std::exp(-sv[i]));
        for (int i = 0; i < L; ++i) pool.push_back(std::exp(-sv[i] * SOE_NLOC));
        for (int i = 0; i < L; ++i) pool.push_back(wv[i]);
        h->soe_s[b].assign(sv, sv + L);
        h->soe_w[b].assign(wv, wv + L);
        oY += (long long)L * I.K;
    }
    h->sumY = oY;
    TRY(dalloc(h, &h->d_soe, std::max<size_t>(pool.size(), 1)));
    TRY(dalloc(h, &h->d_Y, (size_t)std::max(oY, 1LL)));
    CU(h, cudaMemcpyAsync(h->d_soe, pool.data(), sizeof(double) * pool.size(), cudaMemcpyHostToDevice, h->stream));
    CU(h, cudaMemcpyAsync(h->d_inst, h->inst.data(), sizeof(InstDev) * h->B, cudaMemcpyHostToDevice, h->stream));
    CU(h, cudaStreamSynchronize(h->stream));
    return PSL1_OK;
}

// The fast uniform solver's launches: initial state, a cleared exponential
// state, then one fused history + step launch per fine step.
static cudaError_t enqueue_uniform_soe(psl1_problem* h)
{
    cudaError_t e = launch_uni_init(h->pa, h->B, h->d_u0, h->d_Wcur, h->d_Us, h->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(h->d_Y, 0, sizeof(double) * std::max(h->sumY, 1LL), h->stream);
    for (int j = 0; j < h->Nmax && e == cudaSuccess; ++j)
        e = launch_uni_soe_step(h->pa, h->B, h->d_Wcur, h->d_dW, h->d_Us, j, h->d_soe, h->d_Y, SOE_NLOC,
                                h->stream);
    return e;
}

// Capture an N-step launch sequence into a graph (once per handle).
static psl1_status capture(psl1_problem* h, cudaGraphExec_t* out, cudaError_t (*enq)(psl1_problem*), const char* what)
{
    cudaGraph_t g = nullptr;
    CU(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = enq(h);
    cudaError_t ee = cudaStreamEndCapture(h->stream, &g);
    if (e == cudaSuccess) e = ee;
    if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        *out = nullptr;
        return fail(h, PSL1_ERR_CUDA, "%s graph: %s", what, cudaGetErrorString(e));
    }
    return PSL1_OK;
}

psl1_status psl1_solve_serial(psl1_h h, int kind)
{
    if (!h) return fail(h, PSL1_ERR_ARG, "NULL handle");
    if (!h->u0_set) return fail(h, PSL1_ERR_STATE, "set u0 before solving");
    auto t0 = std::chrono::steady_clock::now();
    h->stats = psl1_stats{};
    TRY(reset_status(h));
    CU(h, cudaEventRecord(h->ev[0], h->stream));
    h->ser_kind = kind;
    if (kind == PSL1_SERIAL_HYBRID) {
        CU(h, launch_serial_hyb(h->pa, h->B, h->d_u0, h->d_Us, h->stream));
        h->stats.kernel_launches = 1;
        for (int b = 0; b < h->B; ++b) {
            h->stats.fine_steps += h->inst[b].N;
            h->stats.fine_step_modes += (double)h->inst[b].N * h->inst[b].K;
        }
    } else if (kind == PSL1_SERIAL_COARSE) {
        PathArgs exact = h->pa;   // the coarse solution itself: never the inexact G
        exact.loose_above = 0.0;
        CU(h, launch_coarse_sweep(exact, h->B, h->d_u0, nullptr, h->d_Us, nullptr, h->d_Gold, 1, h->d_nfirst,
                                  h->d_active, h->d_incr, h->stream));
        h->stats.kernel_launches = 1;
    } else if (kind == PSL1_SERIAL_UNIFORM) {
        TRY(ensure_uniform_pools(h));
        // The N-step sequence (a history launch and a step launch per fine step) is
        // captured into a CUDA graph on the first uniform solve of the handle and
        // replayed afterwards: every argument is a fixed pool or a step index, and
        // u0, D and f are read from device memory when the graph runs.
        if (!h->uni_graph) {
            TRY(tune_uniform_chunk(h));
            CU(h, cudaEventRecord(h->ev[0], h->stream));   // the timed solve starts after the tuning
            TRY(capture(h, &h->uni_graph, enqueue_uniform, "uniform solver"));
        }
        CU(h, cudaGraphLaunch(h->uni_graph, h->stream));
        h->stats.kernel_launches = 2 * h->Nmax;   // init + (N - 1) history + N step kernels
        for (int b = 0; b < h->B; ++b) {
            h->stats.fine_steps += h->inst[b].N;
            h->stats.fine_step_modes += (double)h->inst[b].N * h->inst[b].K;
        }
    } else if (kind == PSL1_SERIAL_UNIFORM_SOE) {
        TRY(ensure_soe_pools(h));
        if (!h->soe_graph) {
            TRY(capture(h, &h->soe_graph, enqueue_uniform_soe, "fast uniform solver"));
            CU(h, cudaEventRecord(h->ev[0], h->stream));
        }
        CU(h, cudaGraphLaunch(h->soe_graph, h->stream));
        h->stats.kernel_launches = 1 + h->Nmax;   // init + N fused history/step kernels
        for (int b = 0; b < h->B; ++b) {
            h->stats.fine_steps += h->inst[b].N;
            h->stats.fine_step_modes += (double)h->inst[b].N * h->inst[b].K;
        }
    } else {
        return fail(h, PSL1_ERR_ARG, "unknown serial kind %d", kind);
    }
    CU(h, cudaEventRecord(h->ev[1], h->stream));
    TRY(check_device_status(h));
    h->stats.ms_fine = elapsed(h->ev[0], h->ev[1]);
    TRY(read_flops(h));
    h->stats.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    h->ser_done = true;
    return PSL1_OK;
}

psl1_status psl1_keep_iterates(psl1_h h, int on)
{
    if (!h) return fail(h, PSL1_ERR_ARG, "NULL handle");
    h->keep_iterates = on != 0;
    return PSL1_OK;
}

static psl1_status snapshot(psl1_problem* h, const double* d)
{
    std::vector<double> v((size_t)h->sumU);
    CU(h, cudaMemcpyAsync(v.data(), d, sizeof(double) * h->sumU, cudaMemcpyDeviceToHost, h->stream));
    CU(h, cudaStreamSynchronize(h->stream));
    h->iterates.push_back(std::move(v));
    return PSL1_OK;
}

// Convergence verdict and statistics shared by the host-loop and graph modes.
static psl1_status finish_parareal(psl1_problem* h, double tol, int maxit, int* iters_out,
                                   std::chrono::steady_clock::time_point t0)
{
    h->par_done = true;
    int itmax = 0;
    bool all_conv = true;
    for (int b = 0; b < h->B; ++b) {
        itmax = std::max(itmax, h->iters[b]);
        bool conv = (!h->errlog[b].empty() && h->errlog[b].back() <= tol) || h->iters[b] >= h->P;
        if (!conv) all_conv = false;
    }
    TRY(read_flops(h));
    h->stats.iterations_max = itmax;
    if (iters_out) *iters_out = itmax;
    h->stats.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (!all_conv) return fail(h, PSL1_ERR_NOT_CONVERGED, "parareal stopped at max_iter=%d above tol", maxit);
    return PSL1_OK;
}

psl1_status psl1_set_graph(psl1_h h, int on)
{
    if (!h) return fail(h, PSL1_ERR_ARG, "NULL handle");
    h->graph_mode = on != 0;
    return PSL1_OK;
}

// The graph-mode iteration: a while node whose body is
//   F stage (U^k -> F_old), [inexact iterations: G_old brought into this
//   iteration's coarse-step mode], correction sweep (U^k -> U^{k+1}, e_k), U^k <- U^{k+1},
//   update (log e_k, retire converged instances, k += 1, loop condition).
// CTAs of the persistent F stage: the tuned count, at most one per workspace slot
static int fstage_grid(const psl1_problem* h)
{
    const int g = h->fgrid > 0 ? std::min(h->fgrid, h->pa.nslots) : h->pa.nslots;
    return std::min(h->nunits, g);
}

static psl1_status build_parareal_graph(psl1_problem* h)
{
    if (!h->d_iters) {
        TRY(dalloc(h, &h->d_iters, h->B));
        TRY(dalloc(h, &h->d_kstate, 2));
        TRY(dalloc(h, &h->d_errlog, (size_t)h->B * h->P));
        TRY(dalloc(h, &h->d_tol, 1));
    }
    cudaGraph_t g = nullptr;
    cudaGraphConditionalHandle cond;
    cudaGraphNodeParams np = {};
    cudaGraphNode_t wnode;
    cudaError_t e = cudaGraphCreate(&g, 0);
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) {
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = cond;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        e = cudaGraphAddNode(&wnode, g, nullptr, nullptr, 0, &np);
    }
    if (e == cudaSuccess) {
        cudaGraph_t body = np.conditional.phGraph_out[0];
        e = cudaStreamBeginCaptureToGraph(h->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            const int grid = fstage_grid(h);
            cudaError_t q = launch_fstage(h->pa, h->d_Ua, h->d_Fv, h->d_units, h->nunits, h->d_counter, h->d_nfirst,
                                          h->d_active, grid, h->stream);
            if (q == cudaSuccess && h->pa.loose_above > 0.0)
                q = launch_coarse_regold(h->pa, h->d_Ua, h->d_Gold, h->d_units, h->nunits, h->d_nfirst, h->d_active,
                                         grid, h->stream);
            if (q == cudaSuccess)
                q = launch_coarse_sweep(h->pa, h->B, h->d_u0, h->d_Ua, h->d_Ub, h->d_Fv, h->d_Gold, 0, h->d_nfirst,
                                        h->d_active, h->d_incr, h->stream);
            if (q == cudaSuccess)
                q = cudaMemcpyAsync(h->d_Ua, h->d_Ub, sizeof(double) * h->sumU, cudaMemcpyDeviceToDevice, h->stream);
            if (q == cudaSuccess)
                q = launch_pr_update(h->d_incr, h->d_active, h->d_nfirst, h->d_iters, h->d_errlog, h->d_counter,
                                     h->d_kstate, h->d_tol, cond, h->B, h->P, h->stream);
            cudaGraph_t out = nullptr;
            e = cudaStreamEndCapture(h->stream, &out);
            if (e == cudaSuccess) e = q;
        }
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&h->par_graph, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        h->par_graph = nullptr;
        return fail(h, PSL1_ERR_CUDA, "parareal graph: %s", cudaGetErrorString(e));
    }
    return PSL1_OK;
}

static psl1_status solve_parareal_graph(psl1_problem* h, double tol, int maxit)
{
    const int B = h->B, P = h->P;
    if (!h->par_graph) TRY(build_parareal_graph(h));
    std::vector<int> zeros(B, 0), ones(B, 1);
    const int kst[2] = {0, maxit};
    CU(h, cudaMemcpyAsync(h->d_active, ones.data(), sizeof(int) * B, cudaMemcpyHostToDevice, h->stream));
    CU(h, cudaEventRecord(h->ev[0], h->stream));
    CU(h, launch_coarse_sweep(h->pa, B, h->d_u0, nullptr, h->d_Ua, nullptr, h->d_Gold, 1, h->d_nfirst, h->d_active,
                              h->d_incr, h->stream));
    CU(h, cudaMemcpyAsync(h->d_nfirst, zeros.data(), sizeof(int) * B, cudaMemcpyHostToDevice, h->stream));
    CU(h, cudaMemcpyAsync(h->d_iters, zeros.data(), sizeof(int) * B, cudaMemcpyHostToDevice, h->stream));
    CU(h, cudaMemcpyAsync(h->d_kstate, kst, sizeof kst, cudaMemcpyHostToDevice, h->stream));
    CU(h, cudaMemcpyAsync(h->d_tol, &tol, sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CU(h, cudaMemsetAsync(h->d_counter, 0, sizeof(int), h->stream));
    CU(h, cudaGraphLaunch(h->par_graph, h->stream));
    CU(h, cudaEventRecord(h->ev[1], h->stream));
    std::vector<int> iters(B);
    std::vector<double> elog((size_t)B * P);
    CU(h, cudaMemcpyAsync(iters.data(), h->d_iters, sizeof(int) * B, cudaMemcpyDeviceToHost, h->stream));
    CU(h, cudaMemcpyAsync(elog.data(), h->d_errlog, sizeof(double) * elog.size(), cudaMemcpyDeviceToHost,
                          h->stream));
    TRY(check_device_status(h));
    int itmax = 0;
    for (int b = 0; b < B; ++b) {
        h->iters[b] = iters[b];
        h->errlog[b].assign(elog.begin() + (size_t)b * P, elog.begin() + (size_t)b * P + iters[b]);
        itmax = std::max(itmax, iters[b]);
    }
    std::vector<int> nfirst(B), active(B);
    for (int k = 0; k < itmax; ++k) {
        for (int b = 0; b < B; ++b) {
            nfirst[b] = k;
            active[b] = iters[b] > k;
        }
        count_work(h, nfirst, active);
    }
    h->stats.kernel_launches = 1 + (h->pa.loose_above > 0.0 ? 4 : 3) * itmax;
    h->d_Ucur = h->d_Ua;
    return PSL1_OK;
}

static psl1_status parareal_host(psl1_problem* h, int k0, const double* Uk0, double tol, int maxit, int* iters_out,
                                 std::chrono::steady_clock::time_point t0);

psl1_status psl1_solve_parareal(psl1_h h, double tol, int max_iter, int* iters_out)
{
    if (!h) return fail(h, PSL1_ERR_ARG, "NULL handle");
    if (!h->u0_set) return fail(h, PSL1_ERR_STATE, "set u0 before solving");
    if (!(tol >= 0.0)) return fail(h, PSL1_ERR_ARG, "tol must be >= 0");
    auto t0 = std::chrono::steady_clock::now();
    const int B = h->B, P = h->P;
    int maxit = (max_iter <= 0 || max_iter > P) ? P : max_iter;
    h->stats = psl1_stats{};
    h->iterates.clear();
    h->iters.assign(B, 0);
    h->errlog.assign(B, {});
    TRY(reset_status(h));
    if (h->graph_mode && !h->keep_iterates) {
        TRY(solve_parareal_graph(h, tol, maxit));
        return finish_parareal(h, tol, maxit, iters_out, t0);
    }
    return parareal_host(h, -1, nullptr, tol, maxit, iters_out, t0);
}

// The host-driven iteration.  k0 < 0: start from the coarse sweep (U^0, and
// G_old(n) = G_n(U^0_{0:n}) along it); k0 >= 0: resume from the checkpoint
// U^{k0} (host), with G_old(n) = G_n(U^{k0}_{0:n}) recomputed at those states --
// the values the interrupted iteration held, so the continuation is the same.
static psl1_status parareal_host(psl1_problem* h, int k0, const double* Uk0, double tol, int maxit, int* iters_out,
                                 std::chrono::steady_clock::time_point t0)
{
    const int B = h->B;
    std::vector<int> nfirst(B, 0), active(B, 1);
    std::vector<double> incr(B, 0.0);
    double* Uk = h->d_Ua;
    double* Uk1 = h->d_Ub;
    CU(h, cudaMemcpyAsync(h->d_active, active.data(), sizeof(int) * B, cudaMemcpyHostToDevice, h->stream));
    CU(h, cudaEventRecord(h->ev[0], h->stream));
    if (k0 < 0) {
        // step 1: U^0 by the coarse sweep, G_old(n) = G_n(U^0_{0:n})
        CU(h, launch_coarse_sweep(h->pa, B, h->d_u0, nullptr, Uk, nullptr, h->d_Gold, 1, h->d_nfirst, h->d_active,
                                  h->d_incr, h->stream));
    } else {
        CU(h, cudaMemcpyAsync(Uk, Uk0, sizeof(double) * h->sumU, cudaMemcpyHostToDevice, h->stream));
        // the last increment is not part of the checkpoint: zero keeps every resumed F stage refined
        CU(h, cudaMemsetAsync(h->d_incr, 0, sizeof(double) * B, h->stream));
        CU(h, cudaMemsetAsync(h->d_counter, 0, sizeof(int), h->stream));
        CU(h, launch_coarse_at(h->pa, Uk, h->d_Gold, h->d_units, h->nunits, h->d_counter, fstage_grid(h),
                               h->stream));
        CU(h, cudaMemsetAsync(h->d_gmode, 0, sizeof(int) * B, h->stream));   // G_old: refined values
    }
    CU(h, cudaEventRecord(h->ev[1], h->stream));
    h->stats.kernel_launches = 1;
    TRY(check_device_status(h));
    h->stats.ms_coarse += elapsed(h->ev[0], h->ev[1]);
    if (h->keep_iterates) TRY(snapshot(h, Uk));
    int k = k0 < 0 ? 0 : k0;
    for (; k < maxit; ++k) {
        for (int b = 0; b < B; ++b) nfirst[b] = k;
        count_work(h, nfirst, active);
        CU(h, cudaMemcpyAsync(h->d_nfirst, nfirst.data(), sizeof(int) * B, cudaMemcpyHostToDevice, h->stream));
        CU(h, cudaMemcpyAsync(h->d_active, active.data(), sizeof(int) * B, cudaMemcpyHostToDevice, h->stream));
        CU(h, cudaMemsetAsync(h->d_counter, 0, sizeof(int), h->stream));
        CU(h, cudaEventRecord(h->ev[0], h->stream));
        int grid = fstage_grid(h);
        CU(h, launch_fstage(h->pa, Uk, h->d_Fv, h->d_units, h->nunits, h->d_counter, h->d_nfirst, h->d_active,
                            grid, h->stream));
        CU(h, cudaEventRecord(h->ev[1], h->stream));
        if (h->pa.loose_above > 0.0) {
            CU(h, launch_coarse_regold(h->pa, Uk, h->d_Gold, h->d_units, h->nunits, h->d_nfirst, h->d_active, grid,
                                       h->stream));
            h->stats.kernel_launches += 1;
        }
        CU(h, launch_coarse_sweep(h->pa, B, h->d_u0, Uk, Uk1, h->d_Fv, h->d_Gold, 0, h->d_nfirst, h->d_active,
                                  h->d_incr, h->stream));
        CU(h, cudaEventRecord(h->ev[2], h->stream));
        h->stats.kernel_launches += 2;
        CU(h, cudaMemcpyAsync(incr.data(), h->d_incr, sizeof(double) * B, cudaMemcpyDeviceToHost, h->stream));
        TRY(check_device_status(h));
        h->stats.ms_fine += elapsed(h->ev[0], h->ev[1]);
        h->stats.ms_coarse += elapsed(h->ev[1], h->ev[2]);
        std::swap(Uk, Uk1);
        if (h->keep_iterates) TRY(snapshot(h, Uk));
        int nact = 0;
        for (int b = 0; b < B; ++b) {
            if (!active[b]) continue;
            h->errlog[b].push_back(incr[b]);
            h->iters[b] = k + 1;
            if (incr[b] <= tol)
                active[b] = 0;
            else
                ++nact;
        }
        if (nact == 0) {
            ++k;
            break;
        }
    }
    h->d_Ucur = Uk;
    return finish_parareal(h, tol, maxit, iters_out, t0);
}

psl1_status psl1_resume_parareal(psl1_h h, int k0, const double* Uk0, double tol, int max_iter, int* iters_out)
{
    if (!h || !Uk0) return fail(h, PSL1_ERR_ARG, "NULL argument");
    if (!h->u0_set) return fail(h, PSL1_ERR_STATE, "set u0 before solving");
    if (!(tol >= 0.0)) return fail(h, PSL1_ERR_ARG, "tol must be >= 0");
    const int P = h->P;
    int maxit = (max_iter <= 0 || max_iter > P) ? P : max_iter;
    if (k0 < 0 || k0 >= maxit) return fail(h, PSL1_ERR_ARG, "k0 must be in [0, max_iter)");
    auto t0 = std::chrono::steady_clock::now();
    h->stats = psl1_stats{};
    h->iterates.clear();
    h->iters.assign(h->B, k0);
    h->errlog.assign(h->B, {});
    TRY(reset_status(h));
    return parareal_host(h, k0, Uk0, tol, maxit, iters_out, t0);
}

psl1_status psl1_get_coeffs(psl1_h h, int which, double* out)
{
    if (!h || !out) return fail(h, PSL1_ERR_ARG, "NULL argument");
    const double* src = which == 0 ? h->d_Ucur : h->d_Us;
    if ((which == 0 && !h->par_done) || (which == 1 && !h->ser_done) || (which != 0 && which != 1))
        return fail(h, PSL1_ERR_STATE, "no result of that kind yet");
    CU(h, cudaMemcpyAsync(out, src, sizeof(double) * h->sumU, cudaMemcpyDeviceToHost, h->stream));
    CU(h, cudaStreamSynchronize(h->stream));
    return PSL1_OK;
}

psl1_status psl1_get_coeffs_dev(psl1_h h, int which, double* out)
{
    if (!h || !out) return fail(h, PSL1_ERR_ARG, "NULL argument");
    const double* src = which == 0 ? h->d_Ucur : h->d_Us;
    if ((which == 0 && !h->par_done) || (which == 1 && !h->ser_done) || (which != 0 && which != 1))
        return fail(h, PSL1_ERR_STATE, "no result of that kind yet");
    CU(h, cudaMemcpyAsync(out, src, sizeof(double) * h->sumU, cudaMemcpyDeviceToDevice, h->stream));
    return PSL1_OK;
}

psl1_status psl1_get_iterations(psl1_h h, int* it)
{
    if (!h || !it) return fail(h, PSL1_ERR_ARG, "NULL argument");
    for (int b = 0; b < h->B; ++b) it[b] = h->iters[b];
    return PSL1_OK;
}

psl1_status psl1_get_errlog(psl1_h h, int b, double* out, int cap, int* len)
{
    if (!h || b < 0 || b >= h->B) return fail(h, PSL1_ERR_ARG, "bad instance index");
    int n = (int)h->errlog[b].size();
    if (len) *len = n;
    if (out)
        for (int i = 0; i < n && i < cap; ++i) out[i] = h->errlog[b][i];
    return PSL1_OK;
}

psl1_status psl1_get_iterate(psl1_h h, int k, double* out)
{
    if (!h || !out) return fail(h, PSL1_ERR_ARG, "NULL argument");
    if (k < 0 || k >= (int)h->iterates.size())
        return fail(h, PSL1_ERR_STATE, "iterate %d not kept (enable psl1_keep_iterates before solving)", k);
    memcpy(out, h->iterates[k].data(), sizeof(double) * h->sumU);
    return PSL1_OK;
}

// ---------------------------------------------------------------- autotuning
// Candidates of the refined mixed step's FP32 inner CG tolerance: a looser
// inner solve takes fewer CG iterations and more refinement sweeps (each with
// a double-float residual); the best balance depends on K.
static const float kInnerRtol[] = {1e-7f, 1e-5f, 3e-4f};

static std::string tune_device_name()
{
    int d = 0;
    cudaDeviceProp pr{};
    if (cudaGetDevice(&d) != cudaSuccess || cudaGetDeviceProperties(&pr, d) != cudaSuccess) return "unknown";
    return pr.name;
}

// cache file: one JSON object per line, {"key": "...", "value": <number>}
static std::map<std::string, double> tune_read(const char* path)
{
    std::map<std::string, double> m;
    if (!path) return m;
    FILE* f = std::fopen(path, "r");
    if (!f) return m;
    char line[1024];
    while (std::fgets(line, sizeof line, f)) {
        const char* k = std::strstr(line, "\"key\": \"");
        const char* v = std::strstr(line, "\"value\": ");
        if (!k || !v) continue;
        k += 8;   // past "key": "
        const char* e = std::strchr(k, '"');
        if (!e) continue;
        m[std::string(k, e - k)] = std::strtod(v + 9, nullptr);
    }
    std::fclose(f);
    return m;
}

// one F stage (all slices, iteration 0) of the instances in `active`, timed on
// the second of two launches; optionally the slice-end states
static psl1_status fstage_trial(psl1_problem* h, const std::vector<int>& active, float* ms, std::vector<double>* Fv)
{
    std::vector<int> nf(h->B, 0);
    CU(h, cudaMemcpyAsync(h->d_nfirst, nf.data(), sizeof(int) * h->B, cudaMemcpyHostToDevice, h->stream));
    CU(h, cudaMemcpyAsync(h->d_active, active.data(), sizeof(int) * h->B, cudaMemcpyHostToDevice, h->stream));
    for (int rep = 0; rep < 2; ++rep) {
        CU(h, cudaMemsetAsync(h->d_counter, 0, sizeof(int), h->stream));
        if (rep == 1) CU(h, cudaEventRecord(h->ev[2], h->stream));
        CU(h, launch_fstage(h->pa, h->d_Ua, h->d_Fv, h->d_units, h->nunits, h->d_counter, h->d_nfirst, h->d_active,
                            fstage_grid(h), h->stream));
        if (rep == 1) CU(h, cudaEventRecord(h->ev[3], h->stream));
    }
    TRY(check_device_status(h));
    CU(h, cudaEventElapsedTime(ms, h->ev[2], h->ev[3]));
    if (Fv) {
        Fv->resize(h->sumPK);
        CU(h, cudaMemcpy(Fv->data(), h->d_Fv, sizeof(double) * h->sumPK, cudaMemcpyDeviceToHost));
    }
    return PSL1_OK;
}

psl1_status psl1_autotune(psl1_h h, const char* cache_path, int* from_cache)
{
    if (!h) return fail(h, PSL1_ERR_ARG, "NULL handle");
    if (!h->u0_set) return fail(h, PSL1_ERR_STATE, "set u0 before tuning");
    const std::string dev = tune_device_name();
    const char* prec = h->prec == PSL1_PREC_FP64 ? "fp64" : h->prec == PSL1_PREC_MIXED ? "mixed" : "fp32";
    const char* dim = h->pa.dim2 ? "2d" : "1d";
    std::map<std::string, double> cache = tune_read(cache_path);
    std::vector<std::pair<std::string, double>> fresh;
    int hits = 0, misses = 0;
    const double loose = h->pa.loose_above;
    h->pa.loose_above = 0.0;   // tune the refined step
    TRY(reset_status(h));
    CU(h, launch_coarse_sweep(h->pa, h->B, h->d_u0, nullptr, h->d_Ua, nullptr, h->d_Gold, 1, h->d_nfirst,
                              h->d_active, h->d_incr, h->stream));   // U^0, the states every trial starts from
    psl1_status st = PSL1_OK;
    // (1) inner tolerance per K bucket (powers of two), refined mixed sine-basis step
    if (h->prec == PSL1_PREC_MIXED) {
        std::map<int, std::vector<int>> buckets;
        for (int b = 0; b < h->B; ++b) {
            if (h->inst[b].basis != PSL1_BASIS_SINE) continue;
            int kb = 1;
            while (kb < h->inst[b].K) kb <<= 1;
            buckets[kb].push_back(b);
        }
        for (auto& bk : buckets) {
            char key[256];
            std::snprintf(key, sizeof key, "%s|%s|%s|inner_rtol|K<=%d", dev.c_str(), prec, dim, bk.first);
            auto set_rtol = [&](float r) -> psl1_status {
                for (int b : bk.second) h->inst[b].inner_rtol = r;
                CU(h, cudaMemcpyAsync(h->d_inst, h->inst.data(), sizeof(InstDev) * h->B, cudaMemcpyHostToDevice,
                                      h->stream));
                return PSL1_OK;
            };
            auto it = cache.find(key);
            if (it != cache.end()) {
                if ((st = set_rtol((float)it->second)) != PSL1_OK) break;
                ++hits;
                continue;
            }
            ++misses;
            std::vector<int> act(h->B, 0);
            for (int b : bk.second) act[b] = 1;
            std::vector<double> ref, F;
            float best_ms = 0.f, ms = 0.f;
            float best = kInnerRtol[0];
            if ((st = set_rtol(best)) != PSL1_OK || (st = fstage_trial(h, act, &best_ms, &ref)) != PSL1_OK) break;
            for (size_t c = 1; c < sizeof kInnerRtol / sizeof kInnerRtol[0] && st == PSL1_OK; ++c) {
                if ((st = set_rtol(kInnerRtol[c])) != PSL1_OK || (st = fstage_trial(h, act, &ms, &F)) != PSL1_OK) break;
                // keep a candidate only if its slice-end states agree with the default's to 1e-10
                double num = 0.0, den = 0.0;
                for (int b : bk.second) {
                    const InstDev& I = h->inst[b];
                    for (long long e = I.oPK; e < I.oPK + (long long)h->P * I.K; ++e) {
                        num = std::max(num, std::fabs(F[e] - ref[e]));
                        den = std::max(den, std::fabs(ref[e]));
                    }
                }
                if (num <= 1e-10 * den && ms < best_ms) {
                    best_ms = ms;
                    best = kInnerRtol[c];
                }
            }
            if (st != PSL1_OK || (st = set_rtol(best)) != PSL1_OK) break;
            fresh.push_back({key, (double)best});
        }
    }
    // (2) CTAs of the persistent F stage: one to four per SM
    if (st == PSL1_OK) {
        char key[256];
        std::snprintf(key, sizeof key, "%s|%s|%s|fstage_ctas_per_sm|units=%d|K<=%d", dev.c_str(), prec, dim, h->nunits,
                      h->Kmax);
        auto it = cache.find(key);
        if (it != cache.end()) {
            const int c = (int)it->second;   // CTAs per SM; 3 and 4 run the variants bounded for them
            h->fgrid = c * h->nsm;
            h->pa.fstage_minb = (c >= 3 && !h->pa.dim2) ? c : 2;
            ++hits;
        } else {
            ++misses;
            // candidates: (CTAs per SM, register bound) = (1, 2), (2, 2), (3, 3), (4, 4); 2D runs one
            // per SM.  A candidate whose CTAs do not all fit at once still runs correctly (the
            // queue is persistent, no CTA waits on another) and loses on time.
            std::vector<int> act(h->B, 1);
            int best = 0;
            float best_ms = 0.f;
            const int cands[4][2] = {{1, 2}, {2, 2}, {3, 3}, {4, 4}};
            for (int c = 0; c < (h->pa.dim2 ? 1 : 4); ++c) {
                const int g = cands[c][0] * h->nsm;
                if (g > h->pa.nslots) continue;
                h->fgrid = g;
                h->pa.fstage_minb = cands[c][1];
                float ms = 0.f;
                if ((st = fstage_trial(h, act, &ms, nullptr)) != PSL1_OK) break;
                if (best == 0 || ms < best_ms) {
                    best = c + 1;
                    best_ms = ms;
                }
            }
            if (best) {
                h->fgrid = cands[best - 1][0] * h->nsm;
                h->pa.fstage_minb = cands[best - 1][1];
            }
            if (st == PSL1_OK) fresh.push_back({key, (double)best});
        }
    }
    h->pa.loose_above = loose;
    if (h->par_graph) {   // the graph holds the launch configuration
        cudaGraphExecDestroy(h->par_graph);
        h->par_graph = nullptr;
    }
    if (st != PSL1_OK) return st;
    if (cache_path && !fresh.empty()) {
        FILE* f = std::fopen(cache_path, "a");
        if (!f) return fail(h, PSL1_ERR_ARG, "cannot write the tuning cache %s", cache_path);
        for (auto& kv : fresh) std::fprintf(f, "{\"key\": \"%s\", \"value\": %.9g}\n", kv.first.c_str(), kv.second);
        std::fclose(f);
    }
    if (from_cache) *from_cache = (misses == 0 && hits > 0) ? 1 : 0;
    return PSL1_OK;
}

psl1_status psl1_get_tuning(psl1_h h, int b, float* inner_rtol, int* fstage_ctas)
{
    if (!h || b < 0 || b >= h->B) return fail(h, PSL1_ERR_ARG, "bad argument");
    if (inner_rtol) *inner_rtol = h->inst[b].inner_rtol;
    if (fstage_ctas) *fstage_ctas = fstage_grid(h);
    return PSL1_OK;
}

psl1_status psl1_get_soe(psl1_h h, int b, double* s, double* w, int cap, int* len)
{
    if (!h || b < 0 || b >= h->B || !len || cap < 0) return fail(h, PSL1_ERR_ARG, "bad argument");
    if (!h->d_Y) TRY(ensure_soe_pools(h));
    const int L = (int)h->soe_s[b].size();
    *len = L;
    for (int i = 0; i < L && i < cap; ++i) {
        if (s) s[i] = h->soe_s[b][i];
        if (w) w[i] = h->soe_w[b][i];
    }
    return PSL1_OK;
}

psl1_status psl1_get_stats(psl1_h h, psl1_stats* st)
{
    if (!h || !st) return fail(h, PSL1_ERR_ARG, "NULL argument");
    *st = h->stats;
    return PSL1_OK;
}

// ---------------------------------------------------------------- single pieces
struct TmpDev {
    psl1_problem* h;
    std::vector<void*> p;
    ~TmpDev()
    {
        for (void* q : p) cudaFree(q);
    }
    double* get(size_t n)
    {
        void* q = nullptr;
        if (cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(double)) != cudaSuccess) return nullptr;
        p.push_back(q);
        return (double*)q;
    }
};

// ---------------------------------------------------------------- dense assembly (measurement of the choice)
psl1_status psl1_assemble(psl1_h h, int b, int method, int units, const double* D, float* A, float* ms)
{
    if (!h || !D || !A || b < 0 || b >= h->B || units < 1) return fail(h, PSL1_ERR_ARG, "bad argument");
    const InstDev& I = h->inst[b];
    if (I.dim != 1 || I.basis != PSL1_BASIS_SINE)
        return fail(h, PSL1_ERR_ARG, "dense assembly is defined for 1D sine-basis instances");
    if (method != PSL1_ASSEMBLE_TENSOR && method != PSL1_ASSEMBLE_MOMENTS)
        return fail(h, PSL1_ERR_ARG, "unknown assembly method %d", method);
    const int K = I.K, Q = I.Q, Qh = I.Qh;
    if (method == PSL1_ASSEMBLE_TENSOR && K > TC_KMAX)
        return fail(h, PSL1_ERR_ARG, "tensor-core assembly needs K <= %d (K = %d)", TC_KMAX, K);
    const int Kpad = (K + 127) / 128 * 128, Npad = (K + 15) / 16 * 16, Qpad = (Q + 63) / 64 * 64;
    const TabDev& T = h->tabs[I.tab];
    TmpDev t{h};
    double* dD = t.get((size_t)units * Q);
    double* tphi = t.get(((size_t)Kpad * Qpad + 3) / 4);               // BF16 table
    double* tcos = t.get(((size_t)Q * (2 * K + 1) + 1) / 2);           // FP32 cosines
    double* tw = t.get((Q + 1) / 2);                                   // FP32 weights
    double* twD = t.get(((size_t)units * Qpad + 1) / 2);                // FP32 w D
    double* tA = t.get(((size_t)units * K * K + 1) / 2);                // FP32 result
    double* tst = t.get(1);
    if (!dD || !tphi || !tcos || !tw || !twD || !tA || !tst) return fail(h, PSL1_ERR_NOMEM, "scratch allocation failed");
    auto* phiT = reinterpret_cast<__nv_bfloat16*>(tphi);
    float *cosT = reinterpret_cast<float*>(tcos), *w = reinterpret_cast<float*>(tw);
    float *wD = reinterpret_cast<float*>(twD), *dA = reinterpret_cast<float*>(tA);
    int* st = reinterpret_cast<int*>(tst);
    CU(h, cudaMemsetAsync(st, 0, sizeof(int), h->stream));
    CU(h, cudaMemcpyAsync(dD, D, sizeof(double) * units * Q, cudaMemcpyHostToDevice, h->stream));
    CU(h, launch_tc_tables(h->d_tp + T.oDt, h->d_tp + T.oC, h->d_tp + T.oWq, K, Qh, Kpad, Qpad, phiT, cosT, w,
                           h->stream));
    k_tc_weights<<<256, 256, 0, h->stream>>>(dD, w, units, Q, Qpad, wD);
    CU(h, cudaGetLastError());
    CU(h, cudaEventRecord(h->ev[2], h->stream));
    if (method == PSL1_ASSEMBLE_TENSOR)
        CU(h, launch_assemble_tc(phiT, wD, units, K, Npad, Kpad, Qpad, dA, st, h->stream));
    else
        CU(h, launch_assemble_th(cosT, wD, units, K, Qpad, Q, (float)I.cA, dA, h->stream));
    CU(h, cudaEventRecord(h->ev[3], h->stream));
    int hst = 0;
    CU(h, cudaMemcpyAsync(&hst, st, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CU(h, cudaMemcpyAsync(A, dA, sizeof(float) * units * K * K, cudaMemcpyDeviceToHost, h->stream));
    CU(h, cudaStreamSynchronize(h->stream));
    if (hst) return fail(h, PSL1_ERR_TIMEOUT, "tensor-core assembly: a bounded wait on the MMA barrier gave up");
    if (ms) {
        float e = 0.f;
        CU(h, cudaEventElapsedTime(&e, h->ev[2], h->ev[3]));
        *ms = e;
    }
    return PSL1_OK;
}

psl1_status psl1_step(psl1_h h, int b, const double* c, double te, double mu, const double* hist, double* out)
{
    if (!h || !c || !hist || !out || b < 0 || b >= h->B) return fail(h, PSL1_ERR_ARG, "bad argument");
    int K = h->inst[b].K;
    TmpDev t{h};
    double *dc = t.get(K), *dh = t.get(K), *dout = t.get(K);
    if (!dc || !dh || !dout) return fail(h, PSL1_ERR_NOMEM, "scratch allocation failed");
    TRY(reset_status(h));
    CU(h, cudaMemcpyAsync(dc, c, sizeof(double) * K, cudaMemcpyHostToDevice, h->stream));
    CU(h, cudaMemcpyAsync(dh, hist, sizeof(double) * K, cudaMemcpyHostToDevice, h->stream));
    CU(h, launch_one_step(h->pa, b, dc, dh, te, mu, dout, h->stream));
    CU(h, cudaMemcpyAsync(out, dout, sizeof(double) * K, cudaMemcpyDeviceToHost, h->stream));
    return check_device_status(h);
}

psl1_status psl1_fine_slice(psl1_h h, int b, int n, const double* U, double* V)
{
    if (!h || !U || !V || b < 0 || b >= h->B || n < 0 || n >= h->P) return fail(h, PSL1_ERR_ARG, "bad argument");
    const InstDev& I = h->inst[b];
    TmpDev t{h};
    double *dU = t.get((size_t)(n + 1) * I.K), *dV = t.get((size_t)(I.m + 1) * I.K);
    if (!dU || !dV) return fail(h, PSL1_ERR_NOMEM, "scratch allocation failed");
    TRY(reset_status(h));
    CU(h, cudaMemcpyAsync(dU, U, sizeof(double) * (n + 1) * I.K, cudaMemcpyHostToDevice, h->stream));
    CU(h, launch_one_slice(h->pa, b, n, dU, dV, h->stream));
    CU(h, cudaMemcpyAsync(V, dV, sizeof(double) * (I.m + 1) * I.K, cudaMemcpyDeviceToHost, h->stream));
    return check_device_status(h);
}

psl1_status psl1_fine_slice_noalloc(psl1_h h, int b, int n, const double* d_U, double* d_V)
{
    if (!h || !d_U || !d_V || b < 0 || b >= h->B || n < 0 || n >= h->P)
        return fail(h, PSL1_ERR_ARG, "bad argument");
    const InstDev& I = h->inst[b];
    // scratch: the fine-history ring, then the FP64 1D factor or the 2D working arrays
    // outside shared memory, then the coarse differences of the FP32-pipe paths
    long long ring = (long long)I.m * I.K;
    long long work = h->pa.dim2 ? h->pa.work_stride
                     : h->prec == PSL1_PREC_FP64 ? bp_elems(I.nb, TILE)
                     : 0;
    long long dud = h->prec == PSL1_PREC_FP64 ? 0 : (long long)(n + 1) * I.K;
    const long long need = noalloc_round(ring) + noalloc_round(work) + dud;
    if (need > NOALLOC_SCRATCH_DOUBLES)
        return fail(h, PSL1_ERR_ARG,
                    "instance %d needs %lld doubles of scratch (history ring %lld, factor or 2D arrays %lld, "
                    "coarse differences %lld, regions 256-byte aligned); the fixed allocation-free array holds %lld",
                    b, need, ring, work, dud, NOALLOC_SCRATCH_DOUBLES);
    TRY(reset_status(h));
    CU(h, launch_one_slice_noalloc(h->pa, h->d_noalloc, b, n, d_U, d_V, ring, work, dud, h->stream));
    return check_device_status(h);
}

psl1_status psl1_coarse_step(psl1_h h, int b, int n, const double* U, double* out)
{
    if (!h || !U || !out || b < 0 || b >= h->B || n < 0 || n >= h->P) return fail(h, PSL1_ERR_ARG, "bad argument");
    const InstDev& I = h->inst[b];
    TmpDev t{h};
    double *dU = t.get((size_t)(n + 1) * I.K), *dout = t.get(I.K);
    if (!dU || !dout) return fail(h, PSL1_ERR_NOMEM, "scratch allocation failed");
    TRY(reset_status(h));
    CU(h, cudaMemcpyAsync(dU, U, sizeof(double) * (n + 1) * I.K, cudaMemcpyHostToDevice, h->stream));
    CU(h, launch_one_coarse(h->pa, b, n, dU, dout, h->stream));
    CU(h, cudaMemcpyAsync(out, dout, sizeof(double) * I.K, cudaMemcpyDeviceToHost, h->stream));
    return check_device_status(h);
}

// ---------------------------------------------------------------- learned coarse correction
}  // extern "C"

struct psl1_mlp {
    MlpLayout L{};
    int nU = 0, nH = 0, nin = 0, width = 0, nout = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<void*> allocs;
    float *master = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr, *oscale = nullptr, *loss = nullptr;
    __nv_bfloat16 *w16 = nullptr, *wT = nullptr;
    int adam_t = 0;
    int bcap = 0;
    float *X0 = nullptr, *T = nullptr, *Y = nullptr, *dY = nullptr, *dH = nullptr, *dH2 = nullptr;
    float *pre[3] = {nullptr, nullptr, nullptr}, *act[3] = {nullptr, nullptr, nullptr};
    float *tA = nullptr, *tB = nullptr;   // transposes for the weight gradients
    int* tc_status = nullptr;             // set by a tensor-core product whose bounded wait gave up
    int S = 0;                 // sample slots in Z / R
    int Scap = 0;
    float *Z = nullptr, *R = nullptr;
    int* valid = nullptr;      // indices of the slots holding samples
    int nvalid = 0;
    std::string err;

    MlpTc tc() const { return {wT, tA, tB, tc_status}; }

    MlpDev dev() const
    {
        MlpDev d{};
        d.wT = wT;
        d.bias = master;
        long long oT = 0;
        for (int l = 0; l < 4; ++l) {
            d.oT[l] = oT;
            oT += (long long)L.din[l] * L.dout[l];
            d.ob[l] = L.ob[l];
        }
        d.oscale = oscale;
        d.nU = nU;
        d.nH = nH;
        d.nin = nin;
        d.width = width;
        d.nout = nout;
        d.on = 1;
        return d;
    }
};

static psl1_status mfail(psl1_mlp* h, psl1_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (h)
        h->err = buf;
    else
        g_create_error = buf;
    return st;
}

#define MCU(h, call)                                                                                 \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess)                                                                       \
            return mfail((h), PSL1_ERR_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                         __FILE__, __LINE__);                                                        \
    } while (0)

template <typename T>
static psl1_status malloc_m(psl1_mlp* h, T** p, size_t count)
{
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) return mfail(h, PSL1_ERR_NOMEM, "cudaMalloc of %zu bytes failed", count * sizeof(T));
    h->allocs.push_back(q);
    *p = static_cast<T*>(q);
    return PSL1_OK;
}

static psl1_status ensure_batch(psl1_mlp* h, int B)
{
    if (B <= h->bcap) return PSL1_OK;
    size_t W = h->width;
    TRY(malloc_m(h, &h->X0, (size_t)B * h->nin));
    TRY(malloc_m(h, &h->T, (size_t)B * h->nout));
    TRY(malloc_m(h, &h->Y, (size_t)B * h->nout));
    TRY(malloc_m(h, &h->dY, (size_t)B * h->nout));
    TRY(malloc_m(h, &h->dH, (size_t)B * W));
    TRY(malloc_m(h, &h->dH2, (size_t)B * W));
    for (int l = 0; l < 3; ++l) {
        TRY(malloc_m(h, &h->pre[l], (size_t)B * W));
        TRY(malloc_m(h, &h->act[l], (size_t)B * W));
    }
    const size_t wmax = std::max<size_t>(W, std::max(h->nin, h->nout));
    TRY(malloc_m(h, &h->tA, (size_t)B * wmax));
    TRY(malloc_m(h, &h->tB, (size_t)B * wmax));
    if (!h->tc_status) {
        float* st = nullptr;
        TRY(malloc_m(h, &st, 1));
        h->tc_status = reinterpret_cast<int*>(st);
        if (cudaMemsetAsync(h->tc_status, 0, sizeof(int), h->stream) != cudaSuccess)
            return mfail(h, PSL1_ERR_CUDA, "status word");
    }
    h->bcap = B;
    return PSL1_OK;
}

extern "C" {

const char* psl1_mlp_last_error(psl1_mlp_h h) { return h ? h->err.c_str() : g_create_error.c_str(); }

void psl1_mlp_destroy(psl1_mlp_h h)
{
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (void* p : h->allocs) cudaFree(p);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

psl1_status psl1_mlp_create(psl1_mlp_h* out, int nU, int nH, int width, int nout, unsigned long long seed,
                            void* stream)
{
    if (!out) return mfail(nullptr, PSL1_ERR_ARG, "out is NULL");
    *out = nullptr;
    int nin = nU + nH + 2;
    if (nU < 1 || nH < 0 || nin > MLP_MAX_IN || width < 1 || width > MLP_MAX_WIDTH || nout < 1 || nout > MLP_MAX_OUT)
        return mfail(nullptr, PSL1_ERR_ARG, "MLP sizes out of range (nU+nH+2 <= %d, width <= %d, nout <= %d)",
                     MLP_MAX_IN, MLP_MAX_WIDTH, MLP_MAX_OUT);
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1)
        return mfail(nullptr, PSL1_ERR_CUDA, "no usable CUDA device");
    psl1_mlp* h = new psl1_mlp();
    h->nU = nU;
    h->nH = nH;
    h->nin = nin;
    h->width = width;
    h->nout = nout;
    h->L = mlp_layout(nin, width, nout);
    if (stream) {
        h->stream = (cudaStream_t)stream;
    } else {
        cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
        h->own_stream = true;
    }
    auto bail = [&](psl1_status st) {
        g_create_error = h->err;
        psl1_mlp_destroy(h);
        return st;
    };
    long long n = h->L.nparam;
    psl1_status st;
    if ((st = malloc_m(h, &h->master, n)) || (st = malloc_m(h, &h->m, n)) || (st = malloc_m(h, &h->v, n)) ||
        (st = malloc_m(h, &h->grad, n)) || (st = malloc_m(h, &h->oscale, nout)) || (st = malloc_m(h, &h->loss, 1)) ||
        (st = malloc_m(h, &h->w16, n)) || (st = malloc_m(h, &h->wT, n)))
        return bail(st);
    std::vector<float> ones(nout, 1.0f);
    if (cudaMemsetAsync(h->m, 0, sizeof(float) * n, h->stream) != cudaSuccess ||
        cudaMemsetAsync(h->v, 0, sizeof(float) * n, h->stream) != cudaSuccess ||
        cudaMemcpyAsync(h->oscale, ones.data(), sizeof(float) * nout, cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
        mlp_init_params(h->master, h->L, seed, h->stream) != cudaSuccess ||
        mlp_refresh_bf16(h->master, h->w16, h->wT, nullptr, h->L, h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess) {
        h->err = "MLP initialisation failed";
        return bail(PSL1_ERR_CUDA);
    }
    *out = h;
    return PSL1_OK;
}

psl1_status psl1_mlp_nparams(psl1_mlp_h h, long long* n)
{
    if (!h || !n) return mfail(h, PSL1_ERR_ARG, "NULL argument");
    *n = h->L.nparam;
    return PSL1_OK;
}

psl1_status psl1_mlp_get_params(psl1_mlp_h h, float* params, float* oscale)
{
    if (!h) return mfail(h, PSL1_ERR_ARG, "NULL handle");
    if (params) MCU(h, cudaMemcpyAsync(params, h->master, sizeof(float) * h->L.nparam, cudaMemcpyDeviceToHost, h->stream));
    if (oscale) MCU(h, cudaMemcpyAsync(oscale, h->oscale, sizeof(float) * h->nout, cudaMemcpyDeviceToHost, h->stream));
    MCU(h, cudaStreamSynchronize(h->stream));
    return PSL1_OK;
}

psl1_status psl1_mlp_set_params(psl1_mlp_h h, const float* params, const float* oscale)
{
    if (!h) return mfail(h, PSL1_ERR_ARG, "NULL handle");
    if (params) MCU(h, cudaMemcpyAsync(h->master, params, sizeof(float) * h->L.nparam, cudaMemcpyHostToDevice, h->stream));
    if (oscale) MCU(h, cudaMemcpyAsync(h->oscale, oscale, sizeof(float) * h->nout, cudaMemcpyHostToDevice, h->stream));
    MCU(h, mlp_refresh_bf16(h->master, h->w16, h->wT, nullptr, h->L, h->stream));
    MCU(h, cudaStreamSynchronize(h->stream));
    return PSL1_OK;
}

// a tensor-core product of the network whose bounded barrier wait gave up
static psl1_status check_tc(psl1_mlp* h)
{
    if (!h->tc_status) return PSL1_OK;
    int st = 0;
    MCU(h, cudaMemcpyAsync(&st, h->tc_status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    MCU(h, cudaStreamSynchronize(h->stream));
    if (st) {
        cudaMemsetAsync(h->tc_status, 0, sizeof(int), h->stream);
        return mfail(h, PSL1_ERR_TIMEOUT, "tensor-core product: a bounded barrier wait gave up");
    }
    return PSL1_OK;
}

psl1_status psl1_mlp_forward(psl1_mlp_h h, int B, const float* z, float* y)
{
    if (!h || !z || !y || B < 1) return mfail(h, PSL1_ERR_ARG, "bad argument");
    TRY(ensure_batch(h, B));
    MCU(h, cudaMemcpyAsync(h->X0, z, sizeof(float) * B * h->nin, cudaMemcpyHostToDevice, h->stream));
    MCU(h, mlp_forward(h->X0, B, h->w16, h->master, h->L, h->pre, h->act, h->Y, h->tc(), h->stream));
    MCU(h, cudaMemcpyAsync(y, h->Y, sizeof(float) * B * h->nout, cudaMemcpyDeviceToHost, h->stream));
    MCU(h, cudaStreamSynchronize(h->stream));
    return check_tc(h);
}

psl1_status psl1_mlp_loss_grad(psl1_mlp_h h, int B, const float* z, const float* t, float* grad, float* loss)
{
    if (!h || !z || !t || B < 1) return mfail(h, PSL1_ERR_ARG, "bad argument");
    TRY(ensure_batch(h, B));
    MCU(h, cudaMemcpyAsync(h->X0, z, sizeof(float) * B * h->nin, cudaMemcpyHostToDevice, h->stream));
    MCU(h, cudaMemcpyAsync(h->T, t, sizeof(float) * B * h->nout, cudaMemcpyHostToDevice, h->stream));
    MCU(h, cudaMemsetAsync(h->loss, 0, sizeof(float), h->stream));
    MCU(h, mlp_forward(h->X0, B, h->w16, h->master, h->L, h->pre, h->act, h->Y, h->tc(), h->stream));
    MCU(h, mlp_backward(h->X0, B, h->T, h->w16, h->L, h->pre, h->act, h->Y, h->dY, h->dH, h->dH2, h->grad, h->loss,
                        h->tc(), h->stream));
    if (grad) MCU(h, cudaMemcpyAsync(grad, h->grad, sizeof(float) * h->L.nparam, cudaMemcpyDeviceToHost, h->stream));
    if (loss) MCU(h, cudaMemcpyAsync(loss, h->loss, sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    MCU(h, cudaStreamSynchronize(h->stream));
    return check_tc(h);
}

psl1_status psl1_mlp_adam_step(psl1_mlp_h h, const float* grad, float lr)
{
    if (!h || !grad) return mfail(h, PSL1_ERR_ARG, "bad argument");
    MCU(h, cudaMemcpyAsync(h->grad, grad, sizeof(float) * h->L.nparam, cudaMemcpyHostToDevice, h->stream));
    h->adam_t += 1;
    MCU(h, mlp_adam(h->master, h->grad, h->m, h->v, h->L.nparam, h->adam_t, lr, 0.9f, 0.999f, 1e-8f, h->stream));
    MCU(h, mlp_refresh_bf16(h->master, h->w16, h->wT, nullptr, h->L, h->stream));
    MCU(h, cudaStreamSynchronize(h->stream));
    return PSL1_OK;
}

psl1_status psl1_mlp_dataset(psl1_mlp_h mh, psl1_h data, int source, int iters)
{
    if (!mh || !data || !(source & (PSL1_DATA_TRAJECTORIES | PSL1_DATA_ITERATES)))
        return mfail(mh, PSL1_ERR_ARG, "bad argument");
    if ((source & PSL1_DATA_TRAJECTORIES) && (!data->ser_done || data->ser_kind != PSL1_SERIAL_HYBRID))
        return mfail(mh, PSL1_ERR_STATE, "trajectory samples need a serial HYBRID solve of the data problem");
    if ((source & PSL1_DATA_ITERATES) && (!data->u0_set || iters < 1))
        return mfail(mh, PSL1_ERR_STATE, "iterate samples need u0 and iters >= 1");
    if (data->pa.dim2) return mfail(mh, PSL1_ERR_ARG, "the learned coarse correction is defined for 1D instances");
    iters = std::min(iters, data->P);
    if (data->stream != mh->stream) MCU(mh, cudaStreamSynchronize(data->stream));
    const int B = data->B, P = data->P, BP = B * P;
    const int S = ((source & PSL1_DATA_TRAJECTORIES) ? BP : 0) + ((source & PSL1_DATA_ITERATES) ? BP * iters : 0);
    if (S > mh->Scap) {
        TRY(malloc_m(mh, &mh->Z, (size_t)S * mh->nin));
        TRY(malloc_m(mh, &mh->R, (size_t)S * mh->nout));
        TRY(malloc_m(mh, &mh->valid, (size_t)S));
        mh->Scap = S;
    }
    mh->S = S;
    MCU(mh, cudaMemsetAsync(mh->Z, 0, sizeof(float) * (size_t)S * mh->nin, mh->stream));
    MCU(mh, cudaMemsetAsync(mh->R, 0, sizeof(float) * (size_t)S * mh->nout, mh->stream));
    MCU(mh, cudaMemsetAsync(data->d_status, 0, sizeof(DevStatus), mh->stream));
    PathArgs run = data->pa;          // the data problem's own coarse propagator
    run.loose_above = 0.0;            // samples from refined F and G only
    run.refine_factor = 0.0;
    PathArgs feat = data->pa;         // feature / sample layout of this network
    feat.mlp = mh->dev();
    std::vector<int> valid;
    long long base = 0;
    if (source & PSL1_DATA_TRAJECTORIES) {
        // features and residuals of the plain L1 coarse propagator on S_hyb
        MCU(mh, cudaMemsetAsync(data->d_counter, 0, sizeof(int), mh->stream));
        MCU(mh, launch_coarse_dataset(feat, data->d_Us, data->d_units, data->nunits, data->d_counter, mh->Z, mh->R,
                                      std::min(data->nunits, feat.nslots), mh->stream));
        for (int s = 0; s < BP; ++s) valid.push_back(s);
        base = BP;
    }
    if (source & PSL1_DATA_ITERATES) {
        // iterations of parareal on the data problem; after each F stage the pairs
        // (z(U^k_{0:n}), F_old(n) - G_old(n)) of every slice n >= k become samples
        std::vector<int> nfirst(B, 0), active(B, 1);
        double* Uk = data->d_Ua;
        double* Uk1 = data->d_Ub;
        MCU(mh, cudaMemcpyAsync(data->d_active, active.data(), sizeof(int) * B, cudaMemcpyHostToDevice, mh->stream));
        MCU(mh, launch_coarse_sweep(run, B, data->d_u0, nullptr, Uk, nullptr, data->d_Gold, 1, data->d_nfirst,
                                    data->d_active, data->d_incr, mh->stream));
        for (int k = 0; k < iters; ++k) {
            for (int b = 0; b < B; ++b) nfirst[b] = k;
            MCU(mh, cudaMemcpyAsync(data->d_nfirst, nfirst.data(), sizeof(int) * B, cudaMemcpyHostToDevice, mh->stream));
            MCU(mh, cudaMemsetAsync(data->d_counter, 0, sizeof(int), mh->stream));
            MCU(mh, launch_fstage(run, Uk, data->d_Fv, data->d_units, data->nunits, data->d_counter, data->d_nfirst,
                                  data->d_active, std::min(data->nunits, run.nslots), mh->stream));
            MCU(mh, launch_iterate_dataset(feat, B, P, Uk, data->d_Fv, data->d_Gold, data->d_nfirst, mh->Z, mh->R,
                                           base + (long long)k * BP, mh->stream));
            MCU(mh, launch_coarse_sweep(run, B, data->d_u0, Uk, Uk1, data->d_Fv, data->d_Gold, 0, data->d_nfirst,
                                        data->d_active, data->d_incr, mh->stream));
            std::swap(Uk, Uk1);
            for (int b = 0; b < B; ++b)
                for (int n = k; n < P; ++n) valid.push_back((int)(base + (long long)k * BP + (long long)b * P + n));
        }
        data->d_Ucur = Uk;
    }
    mh->nvalid = (int)valid.size();
    MCU(mh, cudaMemcpyAsync(mh->valid, valid.data(), sizeof(int) * valid.size(), cudaMemcpyHostToDevice, mh->stream));
    MCU(mh, mlp_scale_targets(mh->R, S, mh->nvalid, mh->nout, mh->oscale, mh->stream));
    MCU(mh, cudaStreamSynchronize(mh->stream));
    DevStatus dst{};
    MCU(mh, cudaMemcpy(&dst, data->d_status, sizeof dst, cudaMemcpyDeviceToHost));
    if (dst.code != 0) return mfail(mh, (psl1_status)dst.code, "device error while generating samples");
    return PSL1_OK;
}

psl1_status psl1_mlp_train(psl1_mlp_h mh, psl1_h data, int epochs, int batch, float lr, unsigned long long seed,
                           float* loss_log)
{
    if (!mh || epochs < 0 || batch < 1) return mfail(mh, PSL1_ERR_ARG, "bad argument");
    if (mh->nvalid == 0) {
        if (!data) return mfail(mh, PSL1_ERR_STATE, "no samples: build a dataset or pass a data problem");
        TRY(psl1_mlp_dataset(mh, data, PSL1_DATA_TRAJECTORIES, 0));
    }
    const int S = mh->nvalid;
    TRY(ensure_batch(mh, batch));
    // Adam with a cosine learning-rate decay; each epoch visits the samples in the
    // order of an affine permutation (a j + c) mod S with gcd(a, S) = 1
    const int steps = std::max(1, S / batch);
    const long long total = (long long)epochs * steps;
    long long it = 0;
    auto gcd = [](long long x, long long y) {
        while (y) {
            long long t = x % y;
            x = y;
            y = t;
        }
        return x;
    };
    unsigned long long rs = seed * 6364136223846793005ULL + 1442695040888963407ULL;
    for (int ep = 0; ep < epochs; ++ep) {
        rs = rs * 6364136223846793005ULL + 1442695040888963407ULL;
        long long pa = (long long)((rs >> 33) % (unsigned long long)S) | 1;
        while (gcd(pa, S) != 1) pa += 2;
        long long pc = (long long)((rs >> 13) % (unsigned long long)S);
        MCU(mh, cudaMemsetAsync(mh->loss, 0, sizeof(float), mh->stream));
        for (int s = 0; s < steps; ++s, ++it) {
            float lr_t = 0.5f * lr * (1.0f + cosf(3.14159265f * (float)it / (float)std::max<long long>(total, 1)));
            MCU(mh, mlp_gather(mh->Z, mh->R, mh->valid, S, mh->nin, mh->nout, batch, pa, pc, (long long)s * batch,
                               mh->X0, mh->T, mh->stream));
            MCU(mh, mlp_forward(mh->X0, batch, mh->w16, mh->master, mh->L, mh->pre, mh->act, mh->Y, mh->tc(), mh->stream));
            MCU(mh, mlp_backward(mh->X0, batch, mh->T, mh->w16, mh->L, mh->pre, mh->act, mh->Y, mh->dY, mh->dH,
                                 mh->dH2, mh->grad, mh->loss, mh->tc(), mh->stream));
            mh->adam_t += 1;
            MCU(mh, mlp_adam(mh->master, mh->grad, mh->m, mh->v, mh->L.nparam, mh->adam_t, lr_t, 0.9f, 0.999f, 1e-8f,
                             mh->stream));
            MCU(mh, mlp_refresh_bf16(mh->master, mh->w16, mh->wT, nullptr, mh->L, mh->stream));
        }
        if (loss_log) {
            float l = 0.f;
            MCU(mh, cudaMemcpyAsync(&l, mh->loss, sizeof(float), cudaMemcpyDeviceToHost, mh->stream));
            MCU(mh, cudaStreamSynchronize(mh->stream));
            loss_log[ep] = l / steps;
        }
    }
    MCU(mh, cudaStreamSynchronize(mh->stream));
    return check_tc(mh);
}

psl1_status psl1_set_inexact_refinement(psl1_h h, double factor)
{
    if (!h) return fail(h, PSL1_ERR_ARG, "NULL handle");
    if (!(factor >= 0.0) || !std::isfinite(factor)) return fail(h, PSL1_ERR_ARG, "factor must be finite and >= 0");
    h->pa.refine_factor = factor;
    if (h->par_graph) {   // the graph holds the kernels' arguments
        cudaGraphExecDestroy(h->par_graph);
        h->par_graph = nullptr;
    }
    return PSL1_OK;
}

psl1_status psl1_set_sweep_split(psl1_h h, int ctas)
{
    if (!h) return fail(h, PSL1_ERR_ARG, "NULL handle");
    if (ctas != 0 && ctas != 1 && ctas != 2 && ctas != 4 && ctas != 8)
        return fail(h, PSL1_ERR_ARG, "cluster size must be 0 (automatic), 1, 2, 4 or 8");
    if (ctas > 1 && !h->pa.dim2) return fail(h, PSL1_ERR_ARG, "the split sweep is defined for 2D instances");
    const int before = h->pa.split2d;
    if (ctas == 0) {
        auto_split(h);
    } else if (!apply_split(h, ctas)) {
        apply_split(h, before);
        return fail(h, PSL1_ERR_ARG, "clusters of %d CTAs cannot run this batch's coarse sweep", ctas);
    }
    if (h->par_graph && h->pa.split2d != before) {   // the graph holds the launch configuration
        cudaGraphExecDestroy(h->par_graph);
        h->par_graph = nullptr;
    }
    return PSL1_OK;
}

psl1_status psl1_get_sweep_split(psl1_h h, int* ctas)
{
    if (!h || !ctas) return fail(h, PSL1_ERR_ARG, "NULL argument");
    *ctas = h->pa.split2d;
    return PSL1_OK;
}

psl1_status psl1_set_coarse_substeps(psl1_h h, int c)
{
    if (!h) return fail(h, PSL1_ERR_ARG, "NULL handle");
    int mmin = h->inst[0].m;
    for (int b = 0; b < h->B; ++b) mmin = std::min(mmin, h->inst[b].m);
    if (c < 1 || c > mmin) return fail(h, PSL1_ERR_ARG, "coarse substeps must be in [1, %d] (the smallest m)", mmin);
    if (c > 1 && h->pa.mlp.on)
        return fail(h, PSL1_ERR_ARG, "the learned coarse correction is defined on the one-step coarse propagator");
    // mc^-a b(d + r/mc), d < P, 1 <= r <= mc, per instance (b(x) = (x+1)^{1-a} - x^{1-a}), and
    // the substep size and mu, on the host
    std::vector<double> w;
    std::vector<float> wd;
    for (int b = 0; b < h->B; ++b) {
        InstDev& I = h->inst[b];
        I.mc = c;
        I.dtc = I.dT / c;
        I.muc = std::pow(I.dtc, I.alpha) * std::tgamma(2.0 - I.alpha);
        I.oBc = (long long)w.size();
        const double ma = std::pow((double)c, -I.alpha);
        for (int d = 0; d < h->P; ++d)
            for (int r = 1; r <= c; ++r) {
                const double x = d + (double)r / c;
                const double bx = std::pow(x + 1.0, 1.0 - I.alpha) - std::pow(x, 1.0 - I.alpha);
                const double v = ma * bx;
                w.push_back(v);
                const float hi = (float)v;
                wd.push_back(hi);
                wd.push_back((float)(v - (double)hi));
            }
    }
    if (w.size() > h->bcc_cap) {
        TRY(dalloc(h, &h->d_bcc, w.size()));
        TRY(dalloc(h, &h->d_bccd, w.size()));   // float pairs in 8-byte slots
        h->bcc_cap = w.size();
    }
    CU(h, cudaMemcpyAsync(h->d_bcc, w.data(), sizeof(double) * w.size(), cudaMemcpyHostToDevice, h->stream));
    CU(h, cudaMemcpyAsync(h->d_bccd, wd.data(), sizeof(float) * wd.size(), cudaMemcpyHostToDevice, h->stream));
    CU(h, cudaMemcpyAsync(h->d_inst, h->inst.data(), sizeof(InstDev) * h->B, cudaMemcpyHostToDevice, h->stream));
    CU(h, cudaStreamSynchronize(h->stream));
    h->pa.bcc = h->d_bcc;
    h->pa.bccd = reinterpret_cast<const df*>(h->d_bccd);
    if (h->par_graph) {   // the graph holds the kernels' arguments
        cudaGraphExecDestroy(h->par_graph);
        h->par_graph = nullptr;
    }
    return PSL1_OK;
}

psl1_status psl1_set_inexact_fine(psl1_h h, double above)
{
    if (!h) return fail(h, PSL1_ERR_ARG, "NULL handle");
    if (!(above >= 0.0) || !std::isfinite(above)) return fail(h, PSL1_ERR_ARG, "threshold must be finite and >= 0");
    h->pa.loose_above = above;
    if (h->par_graph) {   // the graph holds the kernels' arguments
        cudaGraphExecDestroy(h->par_graph);
        h->par_graph = nullptr;
    }
    return PSL1_OK;
}

psl1_status psl1_set_coarse(psl1_h h, psl1_mlp_h mh)
{
    if (!h) return fail(h, PSL1_ERR_ARG, "NULL handle");
    if (!mh) {
        h->pa.mlp = MlpDev{};
        if (h->par_graph) {
            cudaGraphExecDestroy(h->par_graph);
            h->par_graph = nullptr;
        }
        return PSL1_OK;
    }
    if (h->pa.dim2) return fail(h, PSL1_ERR_ARG, "the learned coarse correction is defined for 1D instances");
    if (h->inst[0].mc > 1)
        return fail(h, PSL1_ERR_ARG, "the learned coarse correction is defined on the one-step coarse propagator");
    for (int b = 0; b < h->B; ++b)
        if (h->inst[b].basis == PSL1_BASIS_CHEB)
            return fail(h, PSL1_ERR_ARG, "the learned coarse correction is defined for sine-basis instances");
    if (mh->stream != h->stream) CU(h, cudaStreamSynchronize(mh->stream));
    h->pa.mlp = mh->dev();
    if (h->par_graph) {   // the graph holds the kernels' arguments
        cudaGraphExecDestroy(h->par_graph);
        h->par_graph = nullptr;
    }
    return PSL1_OK;
}

}  // extern "C"
