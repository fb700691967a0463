/*
 * psl1.h -- C ABI of the GB300 parareal / L1 / sine-Galerkin solver for the
 * quasilinear Caputo subdiffusion equation (arXiv 2510.11023)
 *
 *     d^alpha_t u = div( D(x,t,u) grad u ) + f(x,t,u)   on a box Omega,
 *     u = 0 on the boundary,  u(.,0) = u0,  0 < alpha <= 1        (Sec. 1, Eq. MainPDE)
 *
 * Space: Galerkin in the L2-orthonormal sine basis
 *   1D  phi_k(x) = sqrt(2/L) sin(k pi (x-lo)/L),   k = 1..Mx
 *   2D  phi_kl(x,y) = phi_k(x) phi_l(y),  mode index i = (k-1)*My + (l-1)
 * with Gauss-Legendre quadrature (Qx [x Qy] nodes) for the D and f terms and
 * the identity mass matrix (Sec. 2.1, Eq. AForm / MainPDEWeakSemi).
 * Time: the semi-implicit L1 scheme (Sec. 2.1, Eq. L1Scheme and
 * NumericalSchemeSequential): D and f are evaluated at the previous time
 * level, so every step is one SPD solve (I + mu A(D)) c_new = history + mu F.
 * Parallel in time: parareal with the coarse propagator G_n (one L1 step of
 * size dT = T/P with the whole coarse history, Eq. CoarsePropagator) and the
 * fine propagator F_n (m = N/P fine steps whose history on [0,T_n] is taken
 * on the coarse grid, Sec. 2.2, Eq. L1Fine / NumericalSchemeFine /
 * FinePropagator), iterated as in Eq. (Parareal) and Fig. (parareal).
 *
 * Everything runs on one CUDA device in hand-written sm_103a kernels; there
 * is no CPU fallback: a call that needs the device fails with PSL1_ERR_CUDA
 * when none is usable.
 *
 * Conventions
 *  - Every function returns a psl1_status and never aborts the process; the
 *    text of the last failure is returned by psl1_last_error(handle) (or
 *    psl1_last_error(NULL) for a failed psl1_create).
 *  - Ownership: the caller owns every array it passes; the library copies
 *    what it keeps.  Host arrays are plain C arrays; "_dev" functions take
 *    device pointers and are ordered on the handle's stream.
 *  - A handle is not thread-safe; different handles are independent.
 *  - Coefficient vectors of a batch are concatenated instance after instance
 *    (instance b holds K_b = Mx*My doubles); "node" arrays hold the P+1
 *    coarse nodes T_0..T_P of every instance: sum_b (P+1)*K_b doubles.
 */
#ifndef PSL1_H
#define PSL1_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct psl1_problem* psl1_h;

typedef enum {
    PSL1_OK = 0,
    PSL1_ERR_ARG = -1,           /* invalid argument or size                       */
    PSL1_ERR_NOT_SPD = -2,       /* non-positive Cholesky pivot (D <= 0 somewhere)  */
    PSL1_ERR_NONFINITE = -3,     /* NaN / Inf produced or supplied                  */
    PSL1_ERR_CUDA = -4,          /* CUDA runtime failure or no usable device        */
    PSL1_ERR_TIMEOUT = -5,       /* a bounded device-side wait gave up              */
    PSL1_ERR_NOT_CONVERGED = -6, /* parareal stopped at max_iter above tolerance    */
    PSL1_ERR_STATE = -7,         /* call out of order (e.g. get before solve)       */
    PSL1_ERR_NOMEM = -8          /* device or host allocation failed                */
} psl1_status;

/* Precision of the solve (the history sums, L1 weights and parareal
 * correction are FP64 in every mode).
 *  FP64 : plain FP64 everywhere.  1D: transforms, assembly, Cholesky.  2D:
 *         sum-factorised (matrix-free) operator, Jacobi-preconditioned
 *         conjugate gradients to a relative residual of 1e-14.
 *  MIXED: FP32-pair ("double-float") transforms and residuals, an FP32 inner
 *         solver (conjugate gradients) inside iterative refinement against
 *         the FP64-accurate operator.
 *  FP32 : FP32 coefficient functions, a single FP32 inner solve and no
 *         refinement; 1D transforms in FP32 from FP32 tables.               */
enum { PSL1_PREC_FP64 = 0, PSL1_PREC_MIXED = 1, PSL1_PREC_FP32 = 2 };

/* Serial solvers.
 *  HYBRID : U_{n+1} = F_n(U_{0:n}), n = 0..P-1 -- the sequential fine sweep,
 *           the fixed point of parareal (Sec. 2.2, Eq. PararealConvergence).
 *  UNIFORM: the uniform L1 scheme on all N fine steps with the whole fine
 *           history (Sec. 2.1, Eq. NumericalSchemeSequential with dt = T/N).
 *  COARSE : U_{n+1} = G_n(U_{0:n}) -- the coarse sweep (parareal step 1).
 *  UNIFORM_SOE: the uniform scheme with a fast history (the paper's outlook,
 *           Conclusion item (i)): the weights b(x) of differences at least
 *           nloc = 16 steps old are replaced by a sum of exponentials
 *           sum_i w_i exp(-s_i x) (Gauss-Jacobi and composite Gauss-Legendre
 *           quadrature of b's Laplace-type integral; 5e-15 relative on
 *           [16, N] for N <= 8192, 38-80 exponentials), carried as an L x K
 *           state updated once per step: O((nloc + L) K) work per step
 *           instead of O(j K).  Captured into a CUDA graph on first use.    */
enum { PSL1_SERIAL_HYBRID = 0, PSL1_SERIAL_UNIFORM = 1, PSL1_SERIAL_COARSE = 2, PSL1_SERIAL_UNIFORM_SOE = 3 };

/* One problem instance.  Coefficient families (x, y physical coordinates):
 *   D = (d0 + d1/(1+u^2) * X1 + d2*u + d3*sin(pi x)) * X0,
 *       X_i = 1 + a_i sin(2 pi x) + b_i cos(2 pi y)      (b_i terms 2D only)
 *       dpar = {d0, d1, d2, d3, a0, b0, a1, b1}
 *   f = c0 cos u + c1 sin u + c2 u (1-u) + c3 sin(pi x) e^{-t}
 *       + c4 S1(x,t) + c5 S2(x,t),        fpar = {c0, c1, c2, c3, c4, c5, 0, 0}
 * S1, S2 are the manufactured sources of the exact solutions
 *   S1: u = (1 + t^alpha) sin(pi x)            with D = d0 + d1/(1+u^2)
 *   S2: u = (1 + t^2) sin(pi x)/(2 - cos pi x)  with D = d0 + d3 sin(pi x)
 * on (0,1) (1D only).                                                       */
typedef struct {
    int dim;          /* 1 or 2; every instance of a handle has the same dim  */
    int modes[2];     /* Mx, My (My unused in 1D); 1D: Mx <= 512;
                         2D: Mx, My <= 64 (K = Mx*My <= 4096)                  */
    int qnodes[2];    /* Qx, Qy Gauss-Legendre nodes; 0 selects 2*modes; even */
    int nsteps;       /* N: total fine L1 steps on [0,T]; a multiple of P     */
    double alpha;     /* fractional order, 0 < alpha <= 1                      */
    double T;         /* final time, > 0                                      */
    double lo[2];     /* Omega = (lo0,hi0) [x (lo1,hi1)]                      */
    double hi[2];
    double dpar[8];
    double fpar[8];
    int basis;        /* PSL1_BASIS_SINE (0, default) or PSL1_BASIS_CHEB    */
} psl1_instance;

/* Spatial scheme of an instance.
 *  SINE: Galerkin in the sine basis (above); the state is the K = Mx [My]
 *        modal coefficients.
 *  CHEB: Chebyshev-Lobatto collocation, the paper's own implementation
 *        (Sec. 4.1, Eq. NumericalSchemeMainSystem): 1D only, modes[0] = n
 *        intervals (2 <= n <= 64), nodes x_j = (lo+hi)/2 + (hi-lo)/2
 *        cos(j pi/n); the state is the K = n - 1 values at the interior
 *        nodes j = 1..n-1 (u = 0 at j = 0, n); div(D grad u) is Dm diag(D(u))
 *        Dm restricted to the interior (Dm the scaled first-derivative
 *        matrix); each step (I - mu N) u = hist + mu f is solved by LU with
 *        partial pivoting.  qnodes is ignored; handles with collocation
 *        instances run in PSL1_PREC_FP64 only, and the learned coarse
 *        correction is not defined for them.  A singular step matrix is
 *        reported as PSL1_ERR_NOT_SPD.                                       */
enum { PSL1_BASIS_SINE = 0, PSL1_BASIS_CHEB = 1 };

/* Per-solve statistics filled by the library (device times by CUDA events). */
typedef struct {
    int    iterations_max;   /* largest parareal iteration count of the batch   */
    int    kernel_launches;  /* launches of this library's kernels in the solve */
    double ms_total;         /* wall time of the last solve call (host clock)   */
    double ms_fine;          /* device time in fine-propagator launches         */
    double ms_coarse;        /* device time in coarse sweeps                    */
    double ms_history;       /* device time in history kernels                  */
    double fine_steps;       /* linearised fine steps executed (all instances)  */
    double fine_step_modes;  /* sum over executed fine steps of K               */
    double flop_fine;        /* algorithmic FLOPs done in fine-propagator launches */
    double flop_coarse;      /* algorithmic FLOPs done in coarse sweeps          */
    double flop_serial;      /* algorithmic FLOPs done by the serial solvers     */
} psl1_stats;

/* Create a batch of `batch` instances sharing the slice count P (every
 * instance's nsteps must be a multiple of P).  `cuda_stream` is a
 * cudaStream_t to order all work on, or NULL for a library-owned stream.
 * Builds the quadrature, trigonometric and L1 weight tables on the device.
 * Errors: PSL1_ERR_ARG for an invalid description, PSL1_ERR_CUDA,
 * PSL1_ERR_NOMEM.                                                          */
psl1_status psl1_create(psl1_h* out, int batch, const psl1_instance* inst, int P,
                        int precision, void* cuda_stream);

/* Replace the D / f family parameters (batch x 8 doubles, host).            */
psl1_status psl1_set_D(psl1_h h, const double* dpar);
psl1_status psl1_set_f(psl1_h h, const double* fpar);

/* Initial modal coefficients u0 (sum_b K_b doubles), host or device memory. */
psl1_status psl1_set_u0(psl1_h h, const double* coeffs);
psl1_status psl1_set_u0_dev(psl1_h h, const double* d_coeffs);

/* Serial solve of every instance (kind: PSL1_SERIAL_*).  The result at the
 * coarse nodes is kept in the "serial" slot (see psl1_get_coeffs).  The first
 * UNIFORM solve of a handle also autotunes the history stream (row chunk per
 * CTA, timed on the longest history launch) and captures the N-step launch
 * sequence into a CUDA graph that later UNIFORM solves replay.              */
psl1_status psl1_solve_serial(psl1_h h, int kind);

/* Parareal iteration (Eq. Parareal with the stored G_old of the flowchart):
 * init U^0 by the coarse sweep, then iterate until
 *   e_k = max_n ||U^{k+1}_n - U^k_n||_2 / max_n ||U^{k+1}_n||_2 <= tol
 * for every instance, or k = max_iter (max_iter <= 0 selects P).  Slices
 * n < k are already exact after k iterations and are not recomputed.
 * iters_out (may be NULL) receives the largest iteration count.  Returns
 * PSL1_ERR_NOT_CONVERGED (results still readable) if some instance stopped
 * at max_iter above tol.                                                    */
psl1_status psl1_solve_parareal(psl1_h h, double tol, int max_iter, int* iters_out);

/* Resume parareal from a checkpoint (no counterpart in the paper): U (host,
 * sum_b (P+1) K_b doubles) is the iterate U^{k0} of an earlier solve of the
 * same problem with the same coarse propagator after k0 iterations
 * (psl1_get_iterate or psl1_get_coeffs), 0 <= k0 < max_iter.  G_old(n) =
 * G_n(U^{k0}_{0:n}) is recomputed at those states -- the values the earlier
 * solve held -- and the iteration continues at k0 with slices n >= k0, so it
 * ends where the uninterrupted solve would (bitwise, the kernels being
 * deterministic; to rounding when a 2D sweep is split across a cluster,
 * whose G_old values come from another summation order) for every instance
 * still iterating at k0 (all instances are taken as active there).  Iteration counts include the k0 done before; the
 * increment log and kept iterates start at e_{k0} and U^{k0}.  The last
 * increment is not part of the checkpoint, so resumed F stages are refined
 * (inexact early iterations apply only to fresh solves).  Runs the host
 * loop (graph mode is not used).                                          */
psl1_status psl1_resume_parareal(psl1_h h, int k0, const double* U, double tol, int max_iter, int* iters_out);

/* Copy coefficients at the coarse nodes, sum_b (P+1) K_b doubles:
 * which = 0: the current parareal iterate, 1: the last serial solve.       */
psl1_status psl1_get_coeffs(psl1_h h, int which, double* out);
psl1_status psl1_get_coeffs_dev(psl1_h h, int which, double* d_out);

/* Per-instance parareal iteration counts (batch ints) and the increment log
 * e_k of instance b (cap entries; len receives the count).                  */
psl1_status psl1_get_iterations(psl1_h h, int* iters);
psl1_status psl1_get_errlog(psl1_h h, int b, double* out, int cap, int* len);

/* Iterate history: copy U^k (sum_b (P+1)K_b doubles) of parareal iteration k
 * of the last psl1_solve_parareal (0 <= k <= iterations) -- available when the
 * handle keeps iterates (psl1_keep_iterates(h, 1) before the solve).        */
psl1_status psl1_keep_iterates(psl1_h h, int on);
psl1_status psl1_get_iterate(psl1_h h, int k, double* out);

/* Graph mode of psl1_solve_parareal (on != 0; off by default): the whole
 * iteration -- F stage, correction sweep, and a one-CTA update that logs e_k,
 * retires converged instances and decides whether to continue -- runs as one
 * CUDA graph whose while loop is driven from the device (a conditional graph
 * node), so the host waits once per solve instead of once per iteration.
 * Results, iteration counts and increment logs are the same as in the host
 * loop (the kernels are the same and deterministic).  Per-kernel device times
 * (psl1_stats.ms_fine / ms_coarse) are not measured in this mode (0).  The
 * graph is built on the first graph-mode solve and rebuilt after
 * psl1_set_coarse; with psl1_keep_iterates on, the host loop is used.
 * No counterpart in the paper (its iteration is the same, Fig. parareal).     */
psl1_status psl1_set_graph(psl1_h h, int on);

/* Inexact early parareal iterations (off by default, above = 0).  With
 * above > 0, the F stage of iteration k runs the slices n > k with the FP32
 * step of PSL1_PREC_FP32 (FP32 transforms, D and f, one FP32 inner solve)
 * instead of the refined step, as long as the instance's last increment
 * e_{k-1} exceeds `above` (and always at k = 0); slice n = k, which starts
 * from exact states, keeps the refined step.  In the same iterations (and
 * in the initial coarse sweep) the coarse propagator G is evaluated with
 * the FP32 step as well.  When an instance's mode changes, its stored
 * values G_n(U^k_{0:n}), n >= k, are first recomputed in the new mode (one
 * parallel launch), so each iteration uses one G at both call sites of
 * Eq. Parareal.  The fixed point (the sequential F sweep S_hyb) and the
 * exactness of U^{k+1}_{0:k+1} are unchanged; the cheaper early iterations
 * perturb the iterate by about the FP32 step's error (~1e-6 relative),
 * which the later, refined iterations remove, so `above` should stay well
 * above that (the benchmark tries 1e-4 and 1e-5).  Affects MIXED instances
 * (1D and 2D); a no-op for FP64 and FP32.  psl1_solve_serial's coarse
 * solution always uses the refined G.  Rebuilds the parareal graph.
 * PSL1_ERR_ARG for negative or non-finite values.  No counterpart in the
 * paper (an implementation choice: its iteration, Eq. Parareal, uses the
 * same F and G throughout).                                                 */
psl1_status psl1_set_inexact_fine(psl1_h h, double above);

/* Looser refined F steps while the increment is large (off by default,
 * factor = 0; no counterpart in the paper -- an inexact-solve choice like
 * psl1_set_inexact_fine).  With factor > 0, in iteration k (e_{-1} taken as
 * 1), the refined steps of slices n > k (those not taking the FP32 step) stop their
 * iterative refinement once the measured or predicted correction is below
 * min(1e-6, factor e_{k-1}) of the iterate, instead of the full target
 * (1e-11 measured, 1e-13 predicted); those taking the FP32 step solve to
 * a relative residual of min(1e-4, factor e_{k-1}) instead of 1e-7 (the
 * coarse propagator's FP32 steps are unchanged, since G must be the same
 * function at both call sites).  Slice n = k keeps the full target,
 * so U^{k+1}_{0:k+1} stays exact, and the target tightens with e_k, so the
 * iteration still ends at S_hyb.  F is computed afresh in every iteration,
 * so no stored value has to be recomputed when the target changes.  MIXED
 * instances (1D and 2D); a no-op otherwise.  Rebuilds the parareal graph.
 * PSL1_ERR_ARG for negative or non-finite values.                          */
psl1_status psl1_set_inexact_refinement(psl1_h h, double factor);

/* Coarse propagator with c L1 substeps per slice (1 <= c <= the smallest m
 * of the batch; 1, the default, is the paper's one-step G of Eq.
 * CoarsePropagator).  G^(c)_n(U_{0:n}) is the fine propagator of Eq.
 * FinePropagator on the grid with c steps per slice (dt_c = dT/c, the coarse
 * history of Eq. L1Fine at r/c); c = m makes G the fine propagator itself.
 * Parareal still converges to the sequential fine sweep S_hyb (Eq.
 * PararealConvergence holds for any G); a finer G contracts faster per
 * iteration and costs c times more in the sequential coarse sweep -- the
 * coarse-fine balance the paper names as future work (Conclusion, item
 * (ii)).  Rejected while a learned correction is attached (it is defined on
 * the one-step G).  Rebuilds the parareal graph.                           */
psl1_status psl1_set_coarse_substeps(psl1_h h, int c);

/* 2D: the coarse sweep shares each coarse step among the CTAs of a
 * thread-block cluster (no counterpart in the paper; its sweep is one
 * sequential chain per instance).  With ctas > 1 every instance's sweep runs
 * on a cluster of that many CTAs: each CTA owns ~1/ctas of the y node
 * columns (the node values, D and f there, and their share of every
 * node-to-mode transform), the partial sums are added up through distributed
 * shared memory, and the mode-space vectors and CG iterations are carried
 * redundantly (identical in every CTA).  Results agree with the one-CTA sweep
 * to the rounding of the changed summation order.  ctas: 1, 2, 4 or 8; 0
 * (the default) chooses the largest of 8, 4, 2 for which the batch's
 * clusters fit on the SMs at once.  PSL1_ERR_ARG for other values, for 1D
 * handles with ctas > 1, or when the configuration cannot run (shared
 * memory, workspace, or no cluster of that size fits); the previous setting
 * stays then.  Rebuilds the parareal graph when it changes.
 * psl1_get_sweep_split returns the cluster size in use (1: none).          */
psl1_status psl1_set_sweep_split(psl1_h h, int ctas);
psl1_status psl1_get_sweep_split(psl1_h h, int* ctas);

/* Statistics of the last solve.                                             */
psl1_status psl1_get_stats(psl1_h h, psl1_stats* st);

/* Dense stiffness matrices of the 1D sine-basis instance b (Eq. AForm with
 * the Gauss quadrature of the step), for `units` sets of nodal diffusivities:
 *   A_u[k][l] = sum_q w_q D_u(x_q) phi_{k+1}'(x_q) phi_{l+1}'(x_q),
 * D: units x Q doubles at the Q nodes in ascending order (host); A: units x
 * K x K floats, row-major (host).  The solver never forms this matrix (it
 * applies the Toeplitz+Hankel form, O(QK) per step); this entry point
 * measures that choice against the dense contraction:
 *  PSL1_ASSEMBLE_TENSOR : A = Phi'^T diag(w D) Phi' as a GEMM on the tensor
 *      cores (tcgen05.mma kind::f16, BF16 operands, FP32 accumulation in
 *      tensor memory; one CTA per unit and 128-row block; K <= 256).  Each
 *      entry is within 2^-7 sqrt(A_kk A_ll) of the exact sum (BF16 rounding
 *      of both operands).
 *  PSL1_ASSEMBLE_MOMENTS: the 2K+1 moments g_s = sum_q w_q D_q cos(s pi
 *      th_q) in FP32, A_kl = cA k l (g_|k-l| + g_{k+l}).
 * ms (may be NULL) receives the device time of the assembly kernel alone.
 * Table set-up and copies are outside that time.  PSL1_ERR_TIMEOUT if a
 * bounded wait of the tensor-core kernel gave up.  No counterpart in the
 * paper (its implementation is collocation; the moment form is this
 * library's).                                                              */
enum { PSL1_ASSEMBLE_TENSOR = 0, PSL1_ASSEMBLE_MOMENTS = 1 };
psl1_status psl1_assemble(psl1_h h, int b, int method, int units, const double* D, float* A, float* ms);

/* Autotuning of the F stage for this handle's batch (no counterpart in the
 * paper).  Tuned by timing one F stage (iteration 0, every slice) per
 * candidate on the handle's own instances and u0 (set it first):
 *  - PSL1_PREC_MIXED: the relative residual of the FP32 inner CG of the
 *    refined step, per bucket of instances with K in (2^(j-1), 2^j]
 *    (candidates 1e-7 (default), 1e-5, 3e-4: a looser inner solve means
 *    fewer CG iterations and more double-float refinement sweeps); a
 *    candidate is kept only if its slice-end states agree with the
 *    default's to 1e-10 relative;
 *  - every precision: the persistent F stage's CTAs per SM -- one or two
 *    with the kernel's registers bounded for two, or three or four with
 *    them bounded for three or four (fewer registers, some spilling); 2D:
 *    one.
 * cache_path (may be NULL): a file of JSON lines {"key": ..., "value": ...}
 * keyed by device name, precision, dimension and bucket (or unit count);
 * cached choices are applied without timing, new ones are appended.
 * from_cache (may be NULL) receives 1 if every choice came from the cache.
 * The parareal graph is rebuilt on the next graph-mode solve.              */
psl1_status psl1_autotune(psl1_h h, const char* cache_path, int* from_cache);
/* The tuned inner tolerance of instance b and the F stage's CTA count.      */
psl1_status psl1_get_tuning(psl1_h h, int b, float* inner_rtol, int* fstage_ctas);

/* Exponents s and weights w (cap entries each, may be NULL) of the fast
 * history of instance b: b(x) ~ sum_i w_i exp(-s_i x) for 16 <= x <= N_b;
 * len receives their number (0 for alpha = 1, which has no history).       */
psl1_status psl1_get_soe(psl1_h h, int b, double* s, double* w, int cap, int* len);

/* ---- single pieces of the path, for checks at full size ----------------- */
/* One linearised step of instance b (Eq. NumericalSchemeSequential form):
 *   (I + mu A(D(t_e, c_prev))) c_new = hist + mu F(f(t_e, c_prev)),
 * host arrays of K_b doubles.                                               */
psl1_status psl1_step(psl1_h h, int b, const double* c_prev, double t_e, double mu,
                      const double* hist, double* c_new);

/* Fine propagator F_n of instance b on the coarse states U_0..U_n (host,
 * (n+1) K_b doubles); V receives U_{n,0..m} ((m+1) K_b doubles).           */
psl1_status psl1_fine_slice(psl1_h h, int b, int n, const double* U, double* V);

/* Allocation-free fine propagator (the paper has no counterpart; this is a
 * service to callers).  Same result as psl1_fine_slice, but the inputs and
 * outputs are device arrays the caller owns (d_U: (n+1) K_b doubles,
 * d_V: (m+1) K_b doubles) and the call allocates nothing: no cudaMalloc,
 * cudaFree or allocating library routine.  It is meant for callers that
 * cannot allocate device memory at the time they call -- for example a
 * real-time loop whose device memory was all planned before it started,
 * or code running under a memory manager that forbids new allocations --
 * after creating the handle where allocation was still allowed.
 * Scratch comes from one fixed 4 MiB device array compiled into the library
 * (512 Ki doubles), which every device that loads the library keeps until the
 * process exits.  It holds, each region starting on a 256-byte boundary:
 *   the fine-history ring, m K_b doubles;
 *   PSL1_PREC_FP64 1D: the blocked Cholesky factor, nb (nb+1)/2 32x32 blocks
 *     (nb = ceil(K_b/32)); 2D: the working arrays that do not fit in shared
 *     memory (none for small mode counts; the node arrays at 64 x 64 modes);
 *   PSL1_PREC_MIXED / FP32: the coarse differences U_i - U_{i-1}, (n+1) K_b
 *     entries of 8 bytes.
 * An instance whose scratch exceeds the array is rejected with PSL1_ERR_ARG
 * (the message gives the need).  psl1_create looks up the array's device
 * address with the handle's device current (this loads the library's kernel
 * module there, which is when the array is placed), so this call needs no
 * set-up of its own; a handle is invalid after cudaDeviceReset, the address
 * with it.  All calls share the array and it keeps the last call's contents;
 * every element is written before it is read, so nothing needs clearing, but
 * calls that overlap on the GPU (for instance from two handles on different
 * streams) race.  Ordered on the handle's stream; returns after the kernel
 * finished, with device-side failures reported as in psl1_fine_slice.       */
psl1_status psl1_fine_slice_noalloc(psl1_h h, int b, int n, const double* d_U, double* d_V);

/* Coarse propagator G_n of instance b on U_0..U_n (host); out: K_b doubles. */
psl1_status psl1_coarse_step(psl1_h h, int b, int n, const double* U, double* out);

/* ---- learned coarse correction (no counterpart in the paper) ------------
 * A reading of the learned coarse propagator: it corrects the L1 coarse
 * propagator rather than replacing it,
 *   G_theta(U_{0:n}) = G_n(U_{0:n}) + s o MLP(z_n),
 *   z_n = [k^2 U_n(k), k <= nU ; k^2 eta_n(k), k <= nH ; alpha ; T_n],
 *   eta_n = sum_{j<n} b_{n-j} (U_{j+1} - U_j)  (the coarse L1 history of Eq.
 *   NumericalSchemeSequential), modes beyond an instance's K read as 0,
 * MLP = Linear(nU+nH+2, W) SiLU Linear(W, W) SiLU Linear(W, W) SiLU
 * Linear(W, nout), applied to the first nout modes; BF16 weight copies,
 * FP32 accumulation, FP32 master weights and Adam state.  The output layer
 * starts at zero, so an untrained network is exactly the L1 G (its fallback).
 * Parareal converges to the sequential fine solution for ANY coarse
 * propagator (Eq. PararealConvergence); the network only changes the
 * number of iterations.  Flat parameter layout: W1[W][nin] b1[W] W2[W][W]
 * b2[W] W3[W][W] b3[W] W4[nout][W] b4[nout], nin = nU+nH+2.               */
typedef struct psl1_mlp* psl1_mlp_h;

/* nU + nH + 2 <= 320, W <= 512, nout <= 512; weights U(-1/sqrt(fan_in), +)
 * from a counter-based hash of (seed, index); output layer zero.          */
psl1_status psl1_mlp_create(psl1_mlp_h* out, int nU, int nH, int width, int nout,
                            unsigned long long seed, void* cuda_stream);
psl1_status psl1_mlp_nparams(psl1_mlp_h mh, long long* nparams);
/* FP32 master parameters (flat layout) and the nout output scales s (host). */
psl1_status psl1_mlp_get_params(psl1_mlp_h mh, float* params, float* oscale);
psl1_status psl1_mlp_set_params(psl1_mlp_h mh, const float* params, const float* oscale);
/* Raw network output (without s) for B feature rows z (B x nin, host).     */
psl1_status psl1_mlp_forward(psl1_mlp_h mh, int B, const float* z, float* y);
/* loss = mean (MLP(z) - t)^2 and its gradient w.r.t. every parameter.       */
psl1_status psl1_mlp_loss_grad(psl1_mlp_h mh, int B, const float* z, const float* t, float* grad,
                               float* loss);
/* One Adam step (b1 0.9, b2 0.999, eps 1e-8) with a caller-given gradient. */
psl1_status psl1_mlp_adam_step(psl1_mlp_h mh, const float* grad, float lr);
/* Build the training set from the instances of `data` (replacing any
 * previous one); source is a bit mask:
 *  PSL1_DATA_TRAJECTORIES: (z_n, U_{n+1} - G_n(U_{0:n})) on the sequential
 *      fine solution (needs psl1_solve_serial(data, PSL1_SERIAL_HYBRID));
 *  PSL1_DATA_ITERATES: runs `iters` parareal iterations on `data` with its
 *      current coarse propagator and takes, after each F stage, the pairs
 *      (z(U^k_{0:n}), F_n(U^k_{0:n}) - G_n(U^k_{0:n})) of every slice n >= k --
 *      the exact correction parareal applies, on the states it visits.
 * Targets are scaled per mode to unit RMS; s holds those RMS values.  The
 * parareal buffers of `data` are overwritten.                              */
enum { PSL1_DATA_TRAJECTORIES = 1, PSL1_DATA_ITERATES = 2 };
psl1_status psl1_mlp_dataset(psl1_mlp_h mh, psl1_h data, int source, int iters);
/* Train on the current training set (built from `data`'s trajectories if
 * none exists): minibatches of `batch` in a per-epoch affine permutation,
 * Adam with cosine-decayed learning rate lr.  loss_log (may be NULL)
 * receives the mean loss of each epoch.                                    */
psl1_status psl1_mlp_train(psl1_mlp_h mh, psl1_h data, int epochs, int batch, float lr,
                           unsigned long long seed, float* loss_log);
/* Use the learned correction in every coarse propagator of h (coarse sweeps,
 * G_old, psl1_coarse_step); NULL restores the plain L1 G.  mh must outlive
 * its use by h.  The correction is defined for 1D instances: a 2D handle
 * (here, and as `data` of psl1_mlp_dataset) gives PSL1_ERR_ARG.             */
psl1_status psl1_set_coarse(psl1_h h, psl1_mlp_h mh);
const char* psl1_mlp_last_error(psl1_mlp_h mh);
void psl1_mlp_destroy(psl1_mlp_h mh);

/* ---- measurement utility (no counterpart in the paper) ------------------ */
/* Measured FP64 and FP32 FMA throughput of the current device in TFLOP/s
 * (dependent FMA chains on every SM, best of three timed launches).  Used
 * as the roofline denominators of the ALU-bound kernels.                    */
psl1_status psl1_probe_peaks(double* fp64_tflops, double* fp32_tflops);
/* Measured FP64 tensor-core (mma.sync m8n8k4 f64) throughput in TFLOP/s:
 * four independent accumulators per warp, 8 CTAs of 256 threads per SM,
 * best of three timed launches.                                             */
psl1_status psl1_probe_dmma(double* fp64_tensor_tflops);

const char* psl1_last_error(psl1_h h);
void psl1_destroy(psl1_h h);

#ifdef __cplusplus
}
#endif
#endif /* PSL1_H */
