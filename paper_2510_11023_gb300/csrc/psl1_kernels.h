// psl1_kernels.h -- host-side launch interface of the solver kernels
// (internal to the library; the public boundary is include/psl1.h).
#pragma once
#include <cuda_runtime.h>
#include "psl1_device.cuh"
#include "psl1_mlp.h"

namespace psl1 {

struct TableJob {
    int Mx, Qh;
    double lo, hi;
    double *xh, *wh, *St, *S, *C, *aux;
    double *Std, *Sd, *Cd;   // double-float copies (float pairs stored in 8-byte slots)
    double *Dt, *Dtd, *St32, *Dt32, *aux2;   // derivative table, FP32 copies, cos(2 pi x)
    double *Wd, *auxd, *aux2d;               // double-float copies of the weights and node functions
    double *S32, *C32;                       // FP32 copies of S and C (packed floats)
};

// Byte offsets of the per-CTA shared-memory regions (host-computed; -1 = absent).
struct SmemLayout {
    int cur, hist, nxt, F, v, wp, wm, fp, fm, g, bad;     // FP64 path (+ common)
    int cdf, wpd, wmd, fpd, fmd, gdf, ydf, x, rhs, z, red;   // FP32-pipe path
    int cgx, cgr, cgp, cgq, cgpl, cgdinv, cgred, cggs, cggh, cgpart;   // PCG inner solver
    int mpart;                                                   // split-transform partial sums
    int cm, cu, cdc, cr, cl, cpiv;                               // collocation step (FP64)
    int mz, mh0, mh1;                                            // learned correction inference (last)
    int fine;    // bytes used by kernels that never run the learned correction (everything before mz)
    int total;
};

// 2D working arrays: each region lives in shared memory when it fits (in the
// order listed: most used first), else in the CTA slot's global workspace.
enum Region2D {
    R2_BAD, R2_RED, R2_SPLIT, R2_DINV, R2_PX, R2_PR, R2_PP, R2_PQ, R2_TAB32, R2_T1, R2_T2, R2_Z, R2_WD32,
    R2_N1, R2_N2, R2_CDF, R2_XR, R2_RHS, R2_CUR, R2_HIST, R2_NXT, R2_F, R2_WD, R2_COUNT
};

struct Layout2D {
    int off[R2_COUNT];               // byte offset (shared memory or slot workspace); -1: absent
    unsigned char glob[R2_COUNT];    // 1: in the slot's global workspace
    int smem;                        // shared-memory bytes per CTA
    long long gbytes;                // global workspace bytes per slot
};

// Kmax: modes; nT: max Mx (Qyl + 1); nN: max Qx Qyl (Qyl: the node columns of one
// CTA, Qy unless the step is split); ntab: max Mx Qx/2 + My Qy/2; split > 1: the
// step is shared by a cluster of that many CTAs (adds the partial-sum buffers,
// always in shared memory).
Layout2D make_layout2d(int prec, int Kmax, long long nT, long long nN, long long ntab, int max_smem,
                       int split = 1);

// Pointers and sizes every solver kernel needs.
struct PathArgs {
    const InstDev* inst;
    const TabDev* tab;
    const double* tp;        // table pool
    const double* bp;        // L1 weight pool
    const df* bpd;           // the same weights as double-float (mixed history sums)
    df* dud;                 // per-CTA-slot coarse differences U_i - U_{i-1} (P x Kmax, double-float)
    long long dud_stride;
    df* hc;                  // per-CTA-slot coarse-history terms of a slice's m steps (mmax x Kmax), may be null
    long long hc_stride;
    DevStatus* status;
    double* work;            // per-CTA-slot workspace (FP64 factor; 2D arrays outside shared memory)
    long long work_stride;   // doubles per slot
    double* ring;            // per-CTA-slot fine history ring (m x K doubles)
    long long ring_stride;
    int nslots;              // slots available in work/ring
    int Kmax, Kpmax, Qhmax, mmax;
    int prec;                // PSL1_PREC_*
    SmemLayout L;            // shared-memory layout of the step kernels
    double* flops;           // algorithmic FLOP accumulators (by slot), may be null
    int flop_slot;           // 0 F stage, 1 coarse sweeps, 2 serial solvers, 3 single pieces
    MlpDev mlp;              // learned coarse correction (mlp.on = 0: plain L1 G)
    int dim2;                // 2D instances (the 2D layout below applies)
    Layout2D L2;
    const double* incr;      // last parareal increment e_k per instance (written by the correction sweep)
    double loose_above;      // > 0: inexact F stage while e_k > loose_above (MIXED only; 0: off)
    double refine_factor;    // > 0: refined F steps of slices n > k stop refining at refine_factor e_{k-1}
    const double* cheb;      // collocation pool (nodes, sines, derivative matrices), may be null
    int fstage_minb;         // 1D F stage: CTAs per SM its registers are bounded for (2, 3 or 4)
    const double* bcc;       // coarse-substep weights mc^-a b(d + r/mc) (FP64), may be null
    const df* bccd;          // the same as double-float
    int* gmode;              // per instance: 1 if the stored G_old values are FP32-step values
    double* corr;            // per-CTA-slot parareal corrections F_old(n) - G_old(n) of the sweep (Kmax)
    const int* sweep_order;  // instance of each coarse-sweep CTA (cluster), longest chain first; may be null
    const int* serial_order; // instance of each serial-solver CTA, longest chain first; may be null
    int split2d;             // 2D: CTAs of the cluster that shares each coarse-sweep step (1: none)
    Layout2D L2s;            // 2D: the layout of one CTA of such a cluster
};

// Kc: largest collocation K of the batch (0: none)
SmemLayout make_layout(int prec, int Kmax, int Kpmax, int Qhmax, int Kc = 0);

size_t step_smem_bytes(const PathArgs& a);
// the F stage and the serial fine sweep: the layout without the learned-correction buffers
size_t fine_smem_bytes(const PathArgs& a);

cudaError_t launch_tables(const TableJob& job, cudaStream_t s);
cudaError_t launch_weights(InstDev* inst, int B, double* bpool, double* bpool_df, cudaStream_t s);

// Parareal pieces.
cudaError_t launch_fstage(const PathArgs& a, const double* Uold, double* Fv, const int2* units, int nunits,
                          int* counter, const int* nfirst, const int* active, int grid, cudaStream_t s);
cudaError_t launch_coarse_sweep(const PathArgs& a, int B, const double* u0, const double* Uold, double* Unew,
                                const double* Fv, double* Gold, int init, const int* nfirst,
                                const int* active, double* incr, cudaStream_t s);
// Clusters of `split` CTAs (with layout L2s) that can be resident at once for the 2D
// coarse sweep (0 if none can, or the launch configuration is refused).
int coarse_sweep_clusters(const PathArgs& a, int split);
// G_old(n) = G_n(U_{0:n}) for every unit at given states (resumed parareal).
cudaError_t launch_coarse_at(const PathArgs& a, const double* Uk, double* Gold, const int2* units, int nunits,
                             int* counter, int grid, cudaStream_t s);
// Inexact early iterations: G_old(n), n >= nfirst, of every active instance whose
// coarse-step mode changes at this iteration, recomputed in the new mode.
cudaError_t launch_coarse_regold(const PathArgs& a, const double* Uk, double* Gold, const int2* units, int nunits,
                                 const int* nfirst, const int* active, int grid, cudaStream_t s);
// Serial solvers.
cudaError_t launch_serial_hyb(const PathArgs& a, int B, const double* u0, double* Us, cudaStream_t s);
cudaError_t launch_uni_init(const PathArgs& a, int B, const double* u0, double* Wcur, double* Us,
                            cudaStream_t s);
cudaError_t launch_uni_hist(const PathArgs& a, int B, const double* dW, int j, double* part, int chunk,
                            int maxchunks, cudaStream_t s);
cudaError_t launch_uni_step(const PathArgs& a, int B, double* Wcur, double* dW, double* Us, int j,
                            const double* part, int chunk, int maxchunks, cudaStream_t s);
// Uniform scheme with the fast (sum-of-exponentials) history: one launch per fine step j.
cudaError_t launch_uni_soe_step(const PathArgs& a, int B, double* Wcur, double* dW, double* Us, int j,
                                const double* soe, double* Y, int nloc, cudaStream_t s);
// Single pieces (one CTA).
cudaError_t launch_one_step(const PathArgs& a, int b, const double* c, const double* hist, double te,
                            double mu, double* out, cudaStream_t s);
cudaError_t launch_one_slice(const PathArgs& a, int b, int n, const double* U, double* V, cudaStream_t s);
cudaError_t launch_one_coarse(const PathArgs& a, int b, int n, const double* U, double* out, cudaStream_t s);

// Learned-correction training samples from a serial S_hyb solution (persistent CTAs over units).
cudaError_t launch_coarse_dataset(const PathArgs& a, const double* Us, const int2* units, int nunits, int* counter,
                                  float* Z, float* R, int grid, cudaStream_t s);

// Learned-correction samples (z(U^k_{0:n}), F_old(n) - G_old(n)) from one parareal iterate.
cudaError_t launch_iterate_dataset(const PathArgs& a, int B, int P, const double* Uk, const double* Fv,
                                   const double* Gold, const int* nfirst, float* Z, float* R, long long base,
                                   cudaStream_t s);

// Device-side bookkeeping of one parareal iteration inside the graph-mode loop:
// log the increments, retire converged instances, advance k and nfirst, reset the
// unit counter, and set the while-loop condition (any instance active and k < maxit).
// kstate = {k, maxit}.
cudaError_t launch_pr_update(const double* incr, int* active, int* nfirst, int* iters, double* errlog, int* counter,
                             int* kstate, const double* tol, cudaGraphConditionalHandle cond, int B, int P,
                             cudaStream_t s);

// Single slice with scratch from a fixed device array (no allocation).
constexpr long long NOALLOC_SCRATCH_DOUBLES = 512 * 1024;   // 4 MiB
// regions of the fixed array start on 256-byte (32-double) boundaries
constexpr long long noalloc_round(long long doubles) { return (doubles + 31) / 32 * 32; }
// device address of the fixed array on the current device (loads its module there)
cudaError_t noalloc_scratch_address(double** p);
cudaError_t launch_one_slice_noalloc(const PathArgs& a, double* scratch, int b, int n, const double* U, double* V,
                                     long long ring_doubles, long long work_doubles, long long dud_doubles,
                                     cudaStream_t s);

}  // namespace psl1
