/* kcycle.h -- C ABI of the B300 kappa-cycle multigrid library (libkcycle.so).
 *
 * Method: Avnat & Yavneh, "On the recursive structure of multigrid cycles" (arXiv 2010.00626).
 * The cycle is Algorithm 3 (Section 2.1): relax nu1 times, restrict the residual, solve the
 * coarse problem by one recursive call with cycle counter kappa and, if kappa > 1, a second
 * call with kappa - 1, interpolate and correct, relax nu2 times. kappa = 1 is the V-cycle,
 * kappa = 2 the F-cycle, kappa >= levels the W-cycle (Proposition 2.1).
 *
 * Problem (Section 4): rotated anisotropic diffusion on the unit square, homogeneous Dirichlet
 * boundary, nine-point stencil of Section 4 scaled by 1/h^2 (h = 1/(n+1)); Galerkin coarse
 * operators A^{l+1} = R A^l P with full weighting R and bilinear P; damped Jacobi relaxation;
 * exact coarsest solve.
 *
 * Conventions shared by every entry point
 *   Grid layout   A grid function on the finest level is n*n doubles, row-major, interior points
 *                 only: element (i, j) (i = x index, j = y index, j+1 = north) is at [j*n + i].
 *                 Boundary values are zero and never stored.
 *   Pointers      Arguments documented "device" are CUDA device pointers to memory the caller
 *                 owns (for example torch CUDA tensors); "host" arguments are ordinary host
 *                 memory. The library keeps no reference to caller memory after a call returns.
 *                 Every device pointer must be 8-byte aligned.
 *   Streams       Work is queued on the handle's stream (mg_set_stream; default: a stream the
 *                 handle creates). Entry points that return results on the host synchronise that
 *                 stream; mg_kcycle, mg_kcycle_adjoint and mg_apply do not.
 *   Errors        Every entry point returns an mg_status code; nothing is thrown across the ABI.
 *                 Asynchronous CUDA errors surface at the next synchronising call as MG_ERR_CUDA.
 *                 mg_last_error() gives a text for the last failure on the calling thread.
 *   Threads       A handle must not be used from two host threads at once.
 */
#ifndef KCYCLE_H
#define KCYCLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mg_ctx* mg_handle;

typedef enum {
  MG_OK = 0,
  MG_NOT_CONVERGED = 1,   /* iteration limit reached before the tolerance           */
  MG_ERR_ARG = -1,        /* invalid argument (sizes, kappa <= 0, tol <= 0, ...)    */
  MG_ERR_NOMEM = -2,      /* device allocation failed                               */
  MG_ERR_CUDA = -3,       /* a CUDA call or kernel failed                           */
  MG_ERR_TIMEOUT = -4,    /* a device-side wait gave up                             */
  MG_ERR_STATE = -5       /* handle not usable (NULL, destroyed, or failed setup)   */
} mg_status;

/* Any counter >= the number of levels is the W-cycle (Proposition 2.1). */
#define MG_KAPPA_W 0x7fffffff

/* Options for mg_set_option / mg_get_option. */
typedef enum {
  MG_OPT_OMEGA = 1,        /* Jacobi damping (Section 4: between 0.8 and 0.87); default 0.8     */
  MG_OPT_COARSE_N = 2,     /* largest grid side handled by the single-CTA coarse-level kernel,
                              which walks the kappa recursion on the device; one of 1, 3, 7,
                              15, 31 (default), 63                                                */
  MG_OPT_LEVELS = 3,       /* read-only: number of levels                                          */
  MG_OPT_N = 4,            /* read-only: finest grid side                                          */
  MG_OPT_LAUNCHES = 5,     /* read-only: kernel launches in the last cycle graph built              */
  MG_OPT_COARSE_N32 = 6,   /* as MG_OPT_COARSE_N for the FP32 cycles of the mixed forms; default 31  */
  MG_OPT_COARSE_OP = 7,    /* coarse operators: 0 Galerkin R A P (default), 1 the Section 4 stencil
                              rediscretized on each coarse grid                                     */
  MG_OPT_STOP = 8,         /* mg_solve's stopping test: 0 ||f - A v||/||f|| <= tol (default);
                              1 ||v_k||/||v_0|| <= tol, the error reduction of Section 4 when f = 0  */
  MG_OPT_SMOOTHER = 9,     /* relaxation: 0 damped Jacobi (default); 1 alternating zebra line
                              Gauss-Seidel (Section 4, solvers 3-4): the k-th relaxation of a
                              smoothing step solves every row (k odd: x) or every column (k even: y)
                              exactly, even-indexed lines first, then odd-indexed ones, with no
                              damping; nu1 = nu2 = 2 is one relaxation in each direction; 2 zebra
                              along x only (every relaxation solves the rows). The adjoint entry
                              points return MG_ERR_ARG under the line smoothers.                 */
  MG_OPT_COARSENING = 10,  /* 0 full coarsening (default); 1 semi-coarsening along y only
                              (Section 4, solvers 5-6): every level keeps the n columns and halves
                              the rows, transfers are (1/4)[1 2 1] and linear interpolation across
                              rows, coarse operators Galerkin, smoother forced to 2 (x lines), and
                              the coarsest level is a single row solved exactly. Needs levels = k
                              and Galerkin operators (else MG_ERR_ARG). Reallocates the hierarchy;
                              the mixed-precision entry points return MG_ERR_ARG under it.      */
  MG_OPT_PRECOND = 11,     /* MGCG preconditioner: 0 one kappa-cycle B from zero (default); 1 the
                              symmetrised B + B^T - B^T A B (one cycle, the residual, one adjoint
                              cycle: error propagator (I - B^T A)(I - B A)), symmetric for every
                              kappa. Option 1 needs damped Jacobi, full coarsening and FP64:
                              mg_pcg returns MG_ERR_ARG otherwise, mg_pcg_mixed always.         */
  MG_OPT_CONV_X = 12,      /* convection b = (bx, by), x component (see MG_OPT_CONV_Y)          */
  MG_OPT_CONV_Y = 13,      /* y component: the problem becomes -div(K grad u) + b.grad u, the
                              non-symmetric test problem proposed in Section 5, with b.grad u by
                              first-order upwind differences (default 0: the Section 4 problem).
                              Nonzero b: damped Jacobi, full coarsening and FP64 only (otherwise
                              MG_ERR_ARG when set); mg_pcg, the mixed forms and the adjoint entry
                              points return MG_ERR_ARG. Galerkin products of the upwind operator
                              lose its upwind structure on coarse grids and the cycle can diverge;
                              MG_OPT_COARSE_OP = 1 (rediscretized upwind operators) is the stable
                              choice. Recomputes the stencils.                                    */
  MG_OPT_FUSED_CALL = 14,  /* 2: as 1, and each call two levels above the coarse-level
                              kernel's (not level 0), whose child calls' own children are condensed
                              (MG_OPT_CONDENSED_CHILDREN), runs with those child calls as one launch
                              of a 16-CTA cluster: pass A, per child call pass A, the condensed
                              matrix-vector product and pass B, then pass B; same results bit for
                              bit (measured no faster inside a graph: its 16 CTAs do that level's
                              passes on 16 SMs). 1 (default): with damped Jacobi and full
                              coarsening, each call at the
                              level just above the coarse-level kernel's (FP64 and FP32 cycles)
                              runs as one launch of a thread-block cluster with one CTA per tile
                              of that level, at most 16 (pass A over the tiles, the coarse walk on
                              one CTA, pass B), instead of three launches; same results bit for
                              bit. 0: three launches (the default for the instances of a batch,
                              whose concurrent branches need the SMs a cluster would hold while
                              one of them walks). Not applied at level 0, to adjoint cycles, to
                              levels of more than 16 tiles, or where the device cannot run the
                              cluster (three launches then).                                    */
  MG_OPT_TMA_PASSES = 15,  /* 1 (default): the FP32 cycles' passes at sides >= 255 with nu = 2 run as
                              persistent kernels whose input windows arrive by 2-D tensor copies
                              (TMA), double-buffered; 0: the shared-memory tile and register-pipeline
                              passes. Same arithmetic per point up to the order of FP32 rounding. Arrays
                              must be 16-byte aligned with pitches that are multiples of 4 floats (the
                              handle's own are), else the other passes run.                       */
  MG_OPT_CONDENSED_CHILDREN = 16, /* 1 (default): the two calls that a call just above the coarse-
                              kernel level makes there (counters k and k-1, the first from zero,
                              Algorithm 3), with everything below them, are one linear map of the
                              restricted residual, v = P_c f with c = min(k, levels - lc + 1);
                              the handle computes P_c once (FP64, by the coarse kernel run on unit
                              vectors) and applies it as one matrix-vector product over 16 CTAs
                              (inside the fused call, or as its own launch). Same linear map as
                              the call-by-call walk, rounded differently. Used where that level's
                              side is <= 31 and the maps take <= 64 MB; not for adjoint cycles.
                              0: the walk of the coarse-level kernel.                          */
  MG_OPT_DEEP_CALLS = 18,  /* 0 (off), 63, 127 (default), 255 or 511 (batch instances: 0 only): each
                              call at the largest level of side
                              <= this value runs, with every call below it, as one persistent
                              cooperative launch of one or two CTAs per SM: pass A over the level's
                              tiles, a grid barrier, the child calls (recursively, the two at the
                              coarse-kernel level as the condensed product of
                              MG_OPT_CONDENSED_CHILDREN), pass B, a grid barrier; the kappa
                              recursion walked on the device. Same tiles and per-point arithmetic
                              as the separate launches, so the same results bit for bit. Damped
                              Jacobi, full coarsening, symmetric operators, not adjoint cycles, and
                              only where the condensed maps exist (else the separate launches run).
                              Grid barrier waits are bounded (0.5 s): MG_ERR_TIMEOUT.           */
  MG_OPT_TEST_STALL_BARRIER = 19, /* Test hook for the deep calls' grid barriers. c >= 0: CTA c of
                              every persistent deep launch leaves as it starts, so the other CTAs'
                              first barrier wait runs out after its limit (0.5 s); they record the
                              timeout and leave, the cycle completes, and the next call that reads
                              the solve's result returns MG_ERR_TIMEOUT once (and clears the
                              barrier words). -1 (default): off. Makes no fault.                */
  MG_OPT_TEST_STALL_COPY = 17 /* Test hook for the bounded waits. t >= 0: the FP32 tensor-copy pass A
                              at level 0 arms the copy barrier of tile t (row-major tile index) but
                              issues no copy, so that CTA's wait runs out after its limit (0.5 s,
                              twice); the CTA records the timeout and returns, the launch and the
                              rest of the cycle complete, and the next call that reads the solve's
                              result returns MG_ERR_TIMEOUT once. -1 (default): off. Makes no
                              fault: every copy that is issued completes.                      */
} mg_option;

/* Set up the hierarchy for the Section 4 problem on an n x n interior grid.
 *   n       grid side, n = 2^k - 1 with 1 <= k <= 14
 *   eps     anisotropy, 0 < eps <= 1 (Section 4)
 *   theta   angle of strong diffusion in radians, |theta| <= 1e4 (the paper's phi;
 *           K = R(theta) diag(1,eps) R^T)
 *   levels  1 <= levels <= k; the coarsest grid side 2^(k-levels+1) - 1 must be <= 15
 *   nu1,nu2 pre- and post-relaxation sweeps, 0..8
 * The fine stencil, the Galerkin coarse stencils and the coarsest-level inverse are computed by
 * device kernels; every stencil entry is rounded once from its exact value (correctly rounded
 * cos/sin, exact Galerkin sums, zero-row-sum coarse centres), so it is reproducible bit for bit. Allocates the coarse-level arrays (about n*n/3 doubles per vector kind) and one
 * n*n temporary. On success *out owns them; release with mg_destroy.
 * Errors: MG_ERR_ARG for invalid sizes/parameters, MG_ERR_NOMEM, MG_ERR_CUDA. */
int mg_setup(int n, double eps, double theta, int levels, int nu1, int nu2, mg_handle* out);

/* Free everything the handle owns. Safe on NULL. */
int mg_destroy(mg_handle h);

int mg_set_option(mg_handle h, int key, double value);
int mg_get_option(mg_handle h, int key, double* value);

/* Queue all further work of this handle on the given cudaStream_t (NULL = the handle's own, a
 * non-blocking stream; pass cudaStreamLegacy to order work with the legacy default stream). */
int mg_set_stream(mg_handle h, void* cuda_stream);

/* One finest-level kappa-cycle in place (Algorithm 3): v <- kappa-cycle(v, f, A, 1, levels, kappa).
 *   v  device, n*n, in/out; f device, n*n, read-only; v and f must not overlap.
 *   kappa >= 1 (MG_KAPPA_W or any value >= levels gives the W-cycle).
 * Asynchronous on the handle's stream. */
int mg_kcycle(mg_handle h, double* v, const double* f, int kappa);

/* The adjoint cycle: the cycle whose zero-start map is the transpose B^T of the kappa-cycle's
 * zero-start map B. It swaps nu1 and nu2 and makes the coarse call with counter kappa-1 before
 * the call with kappa (transpose of the error propagator of Algorithm 3, with A symmetric,
 * a constant Jacobi diagonal and R = P^T/4). Same arguments and behaviour as mg_kcycle. */
int mg_kcycle_adjoint(mg_handle h, double* v, const double* f, int kappa);

/* Stand-alone solver (Section 4, first solver): repeat finest-level kappa-cycles from the initial
 * guess in v until ||f - A v||_2 / ||f||_2 <= tol or max_cycles cycles ran. The stopping test runs
 * on the device after every cycle (one graph launch for the whole solve).
 *   v device in/out (initial guess, then the solution); f device.
 *   tol > 0; max_cycles >= 1.
 *   cycles, final_relres  host, nullable: cycles run and the last relative residual.
 *   history               host, nullable, max_cycles doubles: relative residual after each cycle.
 * Returns MG_OK, or MG_NOT_CONVERGED if max_cycles ran without reaching tol. Synchronises. */
int mg_solve(mg_handle h, double* v, const double* f, int kappa, double tol, int max_cycles,
             int* cycles, double* final_relres, double* history);

/* mg_solve iterating the adjoint cycle (mg_kcycle_adjoint): solves A^T v = f, the adjoint problem
 * of a differentiable solve (lambda = A^-T dL/du). Same arguments and behaviour as mg_solve. */
int mg_solve_adjoint(mg_handle h, double* v, const double* f, int kappa, double tol, int max_cycles,
                     int* cycles, double* final_relres, double* history);

/* mg_solve on HOST buffers: copies f and the initial guess v to the device, solves, copies v
 * back. v, f: host, n*n doubles (page-locked memory gives the fastest copies). */
int mg_solve_host(mg_handle h, double* v, const double* f, int kappa, double tol, int max_cycles,
                  int* cycles, double* final_relres, double* history);

/* Conjugate gradients preconditioned by one kappa-cycle from a zero start per iteration (MGCG,
 * Section 4, second solver). x0 = 0; stops when ||r||_2/||b||_2 <= tol or after max_iters.
 *   x device out; b device. flexible != 0 uses beta = r_new.(z_new - z_old) / (r_old.z_old).
 *   iters, final_relres, history: as for mg_solve (history: max_iters doubles).
 * FP64 throughout. Allocates five n*n work vectors on first use. Synchronises. */
int mg_pcg(mg_handle h, double* x, const double* b, int kappa, double tol, int max_iters,
           int flexible, int* iters, double* final_relres, double* history);

/* Mixed precision (an extension of the paper's FP64 method): iterative refinement in FP64 around
 * FP32 kappa-cycles. Each iteration runs one FP32 kappa-cycle from zero on the FP32-rounded
 * residual, d = B32 r (relaxation, restriction and interpolation in FP32; the coarsest solve in
 * FP64), then x += d and r = f - A x in FP64, and tests ||r||_2/||f||_2 <= tol on the device.
 *   x device in/out (initial guess, then the solution, FP64); f device (FP64).
 *   iters, final_relres, history: as for mg_solve (history: max_iters doubles).
 * Allocates the FP32 level arrays (about 4n^2/3 floats per vector kind) on first use.
 * Returns MG_OK or MG_NOT_CONVERGED. Synchronises. */
int mg_solve_mixed(mg_handle h, double* x, const double* f, int kappa, double tol, int max_iters,
                   int* iters, double* final_relres, double* history);

/* One kappa-cycle in FP32 arithmetic in place (the inner cycle of mg_solve_mixed; coarsest solve
 * in FP64): v, f device float arrays, n*n, row-major. Asynchronous. */
int mg_kcycle_f32(mg_handle h, float* v, const float* f, int kappa);

/* MGCG with a mixed-precision preconditioner (an extension of the paper's FP64 method): the PCG
 * vectors, A p, the inner products and alpha/beta are FP64; each preconditioner application rounds
 * r to FP32, runs one FP32 kappa-cycle from zero (coarsest solve FP64) and widens z back to FP64.
 * Same arguments and behaviour as mg_pcg; the flexible beta (flexible != 0) suits this inexact
 * preconditioner. Allocates the FP32 level arrays on first use. Synchronises. */
int mg_pcg_mixed(mg_handle h, double* x, const double* b, int kappa, double tol, int max_iters,
                 int flexible, int* iters, double* final_relres, double* history);

/* out = A v on the finest level (device pointers, n*n each). Asynchronous. */
int mg_apply(mg_handle h, const double* v, double* out);

/* ||f - A v||_2 on the finest level; result to host *norm. Synchronises. */
int mg_residual_norm(mg_handle h, const double* v, const double* f, double* norm);

/* Parameter gradients of a loss L through u = A(theta, eps)^{-1} f: with lambda = A^{-T} dL/du,
 * dL/dtheta = -lambda^T (dA/dtheta) u and dL/deps = -lambda^T (dA/deps) u, dA/dp being the
 * derivative of the Section 4 stencil. lambda, u: device n*n. dtheta, deps: host. Synchronises. */
int mg_param_grads(mg_handle h, const double* lambda, const double* u, double* dtheta, double* deps);

/* Copy the per-level stencils computed on the device to host memory: out[l*9 + (dy+1)*3 + (dx+1)]
 * is the coefficient of v(i+dx, j+dy) in (A^l v)(i, j), l = 0 finest. out: host, max_levels*9.
 * The number of levels written goes to *written (nullable). Synchronises. */
int mg_stencils(mg_handle h, double* out, int max_levels, int* written);

/* Call counts of one kappa-cycle of this handle's hierarchy: calls_per_level[l] for l = 0..levels-1
 * (Proposition 2.2), the kernel launches of its cycle graph and the calls served by the coarse-level
 * kernel. All host, nullable; calls_per_level holds levels entries. No device work beyond computing
 * the condensed child-call maps if they are not built yet (which launches may be fused depends on
 * them). */
int mg_counters(mg_handle h, int kappa, long long* calls_per_level, long long* launches,
                long long* coarse_calls);

/* Launch shape of the level passes, for reports of SM occupancy: *n_level = the side of `level`
 * and *ctas = the CTAs of one pass-A or pass-B launch there that writes no residual sums, in the
 * FP64 cycle (fp32 = 0) or the FP32 cycle of the mixed forms (fp32 = 1; level 0 assumes caller
 * arrays aligned to 16 bytes, as mg_solve_mixed's own are). A pass that also writes residual sums
 * (the level-0 pass A of a stand-alone FP64 solve) uses 64 x 48 tiles where the others use 64 x 32;
 * FP64 levels below level 0 that one tile per SM covers run one such tile per CTA (on 148 SMs: 511
 * in 12 x 12 tiles of 44^2, 255 in 12 x 12 tiles of 22^2; not in the instances of a batch); in the
 * FP32 cycle at sides of 4095 and more the value is pass B's, pass A running as 112 x 16
 * tiles there. For a level handled inside the coarse-level kernel *ctas = 1, that kernel's one
 * CTA; for the level whose calls run as one cluster launch (MG_OPT_FUSED_CALL), the cluster's CTAs. Damped-Jacobi smoother with full coarsening only (else
 * MG_ERR_ARG). Host pointers, both required. No device work. */
int mg_level_grid(mg_handle h, int level, int fp32, int* n_level, int* ctas);

/* Run one finest-level kappa-cycle like mg_kcycle (from the initial guess in v), but launch by
 * launch with a CUDA event pair around every kernel instead of through a graph, and report each
 * launch: ms[r] its duration in milliseconds, kind[r] 0 = pass A (relax + residual + restrict),
 * 1 = pass B (interpolate + correct + relax), 2 = coarse-level kernel, 3 = whole-grid residual;
 * level[r] its level (0 finest); kinds 4 and 5 are zebra row and column relaxations, kind 6 a call
 * run as one cluster launch (pass A, the coarse-level walk, pass B; MG_OPT_FUSED_CALL), kind 7 a
 * call run with everything below it as one persistent launch (MG_OPT_DEEP_CALLS). Flags in
 * with_norm: bit 0 profiles the launches of a stand-alone solve cycle (with the residual partial
 * sums of its stopping test, formed by the first sweep of pass A at level 0 where mg_solve does so,
 * else by the last pass); bit 1 profiles instead the FP32 cycle of mg_solve_mixed (zero start on the
 * handle's FP32 level-0 arrays; v and f are then not used); bit 2 captures the launches with their
 * event pairs into a graph and replays it once (the pairs then hold no host launch latency, as in a
 * solve's graph).
 * ms, kind, level: host, nullable, max_records entries; *count: number of launches (may exceed
 * max_records). Measurement hook with no counterpart in the paper. Synchronises. */
int mg_profile_cycle(mg_handle h, double* v, const double* f, int kappa, int with_norm, int max_records,
                     double* ms, int* kind, int* level, int* count);

/* ||f - A v||_2 on the finest grid of the Section 4 operator for (n, eps, theta), computed WITHOUT
 * allocating anything. The paper has no counterpart: this exists for callers that cannot call
 * cudaMalloc at the point where they need the number -- for example code running while another
 * framework owns the whole device memory pool, a plug-in whose host application forbids device
 * allocation, or a timing loop that cannot afford the device-wide synchronisation an allocation
 * may cause. It needs no handle.
 *   n      grid side, n = 2^k - 1, at most 16383 (larger sizes return MG_ERR_ARG with a message)
 *   eps, theta as for mg_setup
 *   v, f   device, n*n doubles, row-major (caller-owned; only read)
 *   cuda_stream  cudaStream_t to queue on; NULL means the legacy default stream
 *   norm   host, receives the result
 * Scratch: one 5760-byte static device array in libkcycle.so, which every GPU that loads the
 * library holds until the process exits. The first call on a device looks up that array's device
 * address (cudaGetSymbolAddress) with the device current; make that first call before any stream
 * capture. Each call rewrites every scratch slot it reads, so nothing needs clearing between
 * calls, but all calls share the array: calls that overlap on the GPU (other streams, other host
 * threads) race and must be serialised by the caller. Synchronises the stream. */
int mg_residual_norm_noalloc(int n, double eps, double theta, const double* v, const double* f,
                             void* cuda_stream, double* norm);

/* Batched solves (an extension beyond the paper): many independent problems -- each with its own
 * grid side n_i, anisotropy eps_i and angle theta_i, so a ragged set of level hierarchies -- solved
 * by ONE CUDA-graph launch. The graph holds one branch per instance (its initialisation, then a
 * WHILE conditional node repeating {cycle, stopping test}); the branches are independent, so the
 * GPU runs the instances' kernels concurrently. */
typedef struct mg_batch_ctx* mg_batch;

/* Create `count` instances: n[i], eps[i], theta[i] as for mg_setup, levels[i] (NULL: all levels down
 * to 1x1), shared nu1, nu2. *out owns every hierarchy; release with mg_batch_destroy. */
int mg_batch_create(int count, const int* n, const double* eps, const double* theta, const int* levels,
                    int nu1, int nu2, mg_batch* out);

/* Autotuner of the batch's launch shapes, per distinct grid side (largest first), timed inside the
 * batch's concurrency: up to 64 instances of that side are solved together as batch branches of one
 * graph (4 iterations of the FP64 solve, or of the mixed solve when mixed != 0, on scratch arrays),
 * and the side's options are chosen by coordinate descent over
 *   1. the coarse-kernel threshold: FP64 7, 15, 31 (MG_OPT_COARSE_N); FP32 15, 31, 63 (COARSE_N32);
 *   2. fused calls (MG_OPT_FUSED_CALL) x condensed child calls (MG_OPT_CONDENSED_CHILDREN), on/off;
 *   3. for mixed solves of sides >= 1023, the FP32 passes (MG_OPT_TMA_PASSES) on/off;
 * keeping a change only when it is faster; the winner is applied to every instance of that side.
 * chosen (host, nullable, 2 ints per distinct side, largest side first): pairs (n, threshold); the
 * other choices can be read per instance with mg_batch_instance + mg_get_option. Allocates and frees
 * scratch arrays. Synchronises. */
int mg_batch_autotune(mg_batch b, int kappa, int mixed, int* chosen);

/* Solve every instance to ||f_i - A_i x_i|| / ||f_i|| <= tol from the initial guesses x_i, with
 * FP64 kappa-cycles (mixed == 0, as mg_solve) or FP32 kappa-cycles inside FP64 iterative refinement
 * (mixed != 0, as mg_solve_mixed). x, f: host arrays of `count` device pointers (n_i*n_i doubles
 * each). iters, relres: host, nullable, `count` entries. One graph launch; synchronises. Returns
 * MG_OK when every instance converged, MG_NOT_CONVERGED otherwise. */
int mg_batch_solve(mg_batch b, double* const* x, const double* const* f, int kappa, double tol,
                   int max_iters, int mixed, int* iters, double* relres);

/* mg_set_option on every instance of the batch (for example MG_OPT_SMOOTHER = 1: zebra line
 * relaxation everywhere, which also smooths the near-grid-aligned instances that damped Jacobi
 * cannot). Returns the first failing status, MG_ERR_ARG for read-only keys. Synchronises. */
int mg_batch_set_option(mg_batch b, int key, double value);

/* The handle of instance `index` (0-based) of the batch, for mg_get_option (the autotuner's choices)
 * or for solving that instance alone with mg_solve / mg_solve_mixed. The batch owns the handle: do
 * not destroy it; it is valid until mg_batch_destroy. Options set on it apply to the batch too (the
 * batch's graph is rebuilt on its next solve only through mg_batch_set_option or the autotuner, so
 * set per-instance options before the first mg_batch_solve). */
int mg_batch_instance(mg_batch b, int index, mg_handle* out);

/* The batch under the names of the problem-statement interface: mg_setup_batched is mg_batch_create
 * with every instance's full level count (levels = NULL); mg_solve_batched is mg_batch_solve with
 * FP64 kappa-cycles (mixed = 0) and at most 10000 cycles per instance, its cycle counts in `cycles`
 * (host, nullable, `count` entries). Same ownership and errors as those calls. */
int mg_setup_batched(int count, const int* n, const double* eps, const double* theta, int nu1, int nu2,
                     mg_batch* out);
int mg_solve_batched(mg_batch b, double* const* v, const double* const* f, int kappa, double tol, int* cycles);

int mg_batch_size(mg_batch b, int* count);
int mg_batch_destroy(mg_batch b);

/* Measured FP64 operation rate of the current device (fused multiply-adds per second, one add, mul
 * or fma counting as one operation): the ALU peak the FP64 level kernels are reported against.
 * A measurement hook with no counterpart in the paper. Synchronises the device. */
int mg_fp64_rate(double* ops_per_second);

/* Static string for a status code. */
const char* mg_status_string(int status);

/* Text of the last failure seen on the calling host thread ("" if none). */
const char* mg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* KCYCLE_H */
