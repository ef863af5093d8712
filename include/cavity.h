/*
 * cavity.h -- C ABI of the GB300 solver for electromagnetic scattering by an
 * open rectangular cavity in a perfectly conducting ground plane (Chen, Jiang,
 * Lai, Li, "A fast algorithm for the electromagnetic scattering from a large
 * rectangular cavity in three dimensions").
 *
 * Problem (Sec. 2): aperture Gamma = [0,a] x [0,b] in the ground plane x3 = 0,
 * cavity depth c, fill of horizontal layers with relative permittivity eps_l
 * (Sec. 4), free-space wavenumber kappa0, incident plane wave from direction
 * (theta, phi) with polarisation angle alpha (Sec. 7).  The solver follows
 * Algorithm I / II (Sec. 6): Fourier modes in x1, x2 (E123F), finite differences
 * and Gaussian elimination in x3 (Sec. 3, Sec. 4), the transparent boundary
 * condition (ENU1) with its singular integrals evaluated by FFT (Sec. 5), then
 * back-substitution (EInter) and inverse transforms for the interior field.
 *
 * Discretisation: Nx, Ny horizontal grid intervals (M = Nx-1, N = Ny-1 modes),
 * Nz vertical steps (h = c/Nz, aperture at level Nz).  The aperture unknowns are
 * ordered as in Appendix A: E1 over N1 = {0..M}x{1..N}, E2 over N2 =
 * {1..M}x{0..N}, E3 over N3 = {1..M}x{1..N}, each m-major; n_ap = 3MN + M + N.
 * Complex numbers are interleaved (re, im) pairs of double (complex128) or float
 * (complex64).
 *
 * Conventions for every call:
 *  - all work is issued on the CUDA stream given to cavity_setup; a call returns
 *    after that stream has finished the call's work, with its status;
 *  - inputs are read only and owned by the caller; outputs go into buffers the
 *    caller allocated; "device" buffers are CUDA device pointers of the device
 *    that was current at cavity_setup, "host" buffers are ordinary host memory;
 *  - the library allocates its own resident state (kernel table, per-mode
 *    profiles, preconditioner, Krylov workspaces) and frees it in
 *    cavity_destroy;
 *  - on error nothing is aborted: the call returns a status and
 *    cavity_last_error() describes it; outputs are then unspecified except where
 *    stated.
 *  - a context is not thread safe: one host thread at a time per context.
 *  - one device per process: the library raises the shared-memory limits of
 *    its kernels once per process, on the device current at that first use,
 *    so every context of a process must be set up on that device (on another
 *    device, a launch that needs the raised limit returns a CUDA error
 *    status, without a fault).  Use one process per GPU.
 */
#ifndef CAVITY_H
#define CAVITY_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cavity_ctx cavity_ctx;

typedef enum {
  CAVITY_OK = 0,
  CAVITY_EINVAL = 1,     /* invalid argument or unsupported size            */
  CAVITY_ENOMEM = 2,     /* device memory budget or allocation exceeded     */
  CAVITY_ESINGULAR = 3,  /* a per-mode pivot vanished: kappa0 is (nearly) a  */
                         /* discrete cavity resonance (Sec. 3, after (EJJ1)) */
  CAVITY_ENOCONV = 4,    /* the aperture solve stopped above its tolerance;  */
                         /* outputs are filled and the residual is reported  */
  CAVITY_ETIMEOUT = 5,   /* a bounded device wait gave up                    */
  CAVITY_ECUDA = 6       /* a CUDA runtime error                             */
} cavity_status;

enum { CAVITY_FP64 = 0, CAVITY_MIXED = 1 };          /* precision modes       */
/* cavity_apply only: the operator in pair-of-FP32 arithmetic (relative error
 * ~1e-12, complex128 vectors), the residual operator of CAVITY_MIXED solves */
enum { CAVITY_PAIR32 = 2 };
enum { CAVITY_OUT_APERTURE = 0, CAVITY_OUT_FIELD = 1 };
enum { CAVITY_MEM_DEVICE = 0, CAVITY_MEM_HOST = 1 };
enum { CAVITY_POL_THETA = 0, CAVITY_POL_PHI = 1 };

typedef struct {
  double a, b, c;        /* aperture [0,a]x[0,b], depth c                     */
  int nx, ny, nz;        /* grid intervals; nx, ny powers of two in [4, 1024]; */
                         /* nz >= 2                                            */
  int precision;         /* CAVITY_FP64: every step in FP64 (complex128 field) */
                         /* CAVITY_MIXED: FP64 elimination and FP64-accurate   */
                         /*   aperture solve (FP32 inner Krylov iterations with */
                         /*   FP64 residual refinement); FP32 transforms and a  */
                         /*   complex64 field                                  */
  int pad_factor;        /* period of the TBC convolution in aperture sides    */
                         /* (Sec. 5.2; it must exceed side + sqrt 2 max(a, b)  */
                         /* on each axis): 0 = per axis, 4 where that suffices */
                         /* (max/min < 2.12), else 8 or 16 (max/min < 11);    */
                         /* 4 = 4 on both axes (EINVAL if too short).  The FFT */
                         /* operator, and with it the Krylov solver, needs 4   */
                         /* on both axes; longer periods take the dense solver */
  double gmres_tol;      /* relative residual target of (EJ1)/(uT1); 0 -> 1e-12 */
  int gmres_restart;     /* Krylov basis size, at most 120; 0 -> 40            */
  int gmres_max_iter;    /* total inner iterations; 0 -> 400                   */
  double pivot_tol;      /* |pivot| below pivot_tol * max(1,|sigma-2|) is       */
                         /* reported as CAVITY_ESINGULAR; 0 -> 1e-12            */
  int khat_scheme;       /* kernel table F(G) of Sec. 5.2:                      */
                         /* CAVITY_KHAT_QUADRATURE (0): Gauss-Legendre, ~1e-13  */
                         /* CAVITY_KHAT_PAPER (1): the paper's scheme -- the    */
                         /*   same quadrature where 2 pi rho R <= 20 pi sqrt 2, */
                         /*   else the closed-form integral to infinity minus   */
                         /*   the asymptotic tail (two-term J0 and Fresnel      */
                         /*   expansions); an approximation, inaccurate near    */
                         /*   2 pi rho = kappa0                                 */
  int modes_m, modes_n;  /* aperture expansion truncated to the modes m <=      */
                         /* modes_m, n <= modes_n (Galerkin restriction of      */
                         /* (EJ1)/(uT1): the other aperture unknowns are zero    */
                         /* and their rows dropped), as in the paper's runs with */
                         /* few modes (Sec. 7, Table 2: M ~ 2a/lambda); 0 -> all */
                         /* (M = nx-1, N = ny-1); must not exceed M, N          */
  int aperture_solver;   /* how (EJ1)/(uT1) is solved (Algorithm I/II Step 3):  */
                         /* CAVITY_SOLVER_KRYLOV (0): matrix-free GMRES with the */
                         /*   FFT operator (see precision);                     */
                         /* CAVITY_SOLVER_DENSE (1): the paper's direct solve of */
                         /*   the kept block (every unknown of the modes m <=   */
                         /*   modes_m, n <= modes_n), assembled once per        */
                         /*   cavity_prepare from the per-axis factors of       */
                         /*   Sec. 5.2 and LU-factored with partial pivoting in */
                         /*   FP32; each solve refines x in FP64, the residual */
                         /*   from the block kept in FP64 (CAVITY_FP64, and    */
                         /*   the Parseval rule) or from the pair-of-FP32 FFT  */
                         /*   operator (CAVITY_MIXED), so the result meets     */
                         /*   gmres_tol like the Krylov path.                  */
                         /*   The kept block must have at most                 */
                         /*   CAVITY_DENSE_MAX_N unknowns (3 mm nn + mm + nn)  */
  int outer_rule;        /* outer integral of the TBC coefficients (Sec. 5.2): */
                         /* CAVITY_OUTER_TRAPEZOID (0): the trapezoid rule on  */
                         /*   the aperture nodes (rule D; every solver);       */
                         /* CAVITY_OUTER_PARSEVAL (1): exact by Parseval's     */
                         /*   identity on the torus -- each TBC block becomes  */
                         /*   Phi^H diag(F(G)) Phi, complex symmetric; dense   */
                         /*   solver only (the block is assembled in FP64 and  */
                         /*   also supplies the refinement's residual); the    */
                         /*   operator calls cavity_apply and                  */
                         /*   cavity_apply_noalloc apply rule D whatever this  */
                         /*   field says                                       */
} cavity_desc;
enum { CAVITY_KHAT_QUADRATURE = 0, CAVITY_KHAT_PAPER = 1 };
enum { CAVITY_SOLVER_KRYLOV = 0, CAVITY_SOLVER_DENSE = 1 };
enum { CAVITY_OUTER_TRAPEZOID = 0, CAVITY_OUTER_PARSEVAL = 1 };
#define CAVITY_DENSE_MAX_N 16384

/* Create a context for one cavity geometry and grid.  `cuda_stream` is a
 * cudaStream_t (NULL = legacy default stream).  Validates the descriptor;
 * CAVITY_EINVAL on any out-of-range field.  Allocates nothing that depends on
 * kappa0 or eps (that happens at the first cavity_solve / cavity_prepare). */
cavity_status cavity_setup(const cavity_desc* desc, void* cuda_stream,
                           cavity_ctx** out);

/* Steps 1-2 of Algorithm I/II (Sec. 6) for one wavenumber and layer profile:
 * the kernel table F(G) of Sec. 5.2 on the frequency box, the per-mode
 * elimination in x3 (Sec. 3 (LU1)-(EJJ1); Sec. 4 (con12)-(uTT1) and its closing
 * remark for more layers), and the block-diagonal preconditioner.  Layers are
 * given top to bottom: layer_levels[l] grid steps (>= 2 each, summing to nz)
 * with eps = eps_re[l] + i eps_im[l] (host arrays of length nlayers).  The
 * state is kept and reused by cavity_solve while (kappa0, layers) repeat.
 * CAVITY_ESINGULAR if a pivot of the elimination vanishes. */
cavity_status cavity_prepare(cavity_ctx* ctx, double kappa0, int nlayers,
                             const int* layer_levels, const double* eps_re,
                             const double* eps_im);

/* Solve for ndir incident plane waves (Sec. 7 parametrisation, host arrays of
 * length ndir) with the given wavenumber and layer profile (as for
 * cavity_prepare, which this call runs when the pair changed).
 *  aperture_out: ndir x n_ap complex128, the aperture coefficients E_{l,Nz}
 *                (required, never NULL).
 *  field_out:    required when out_mode == CAVITY_OUT_FIELD, else ignored:
 *                ndir x nz x S values, S = (nx+1)(ny-1) + (nx-1)(ny+1) +
 *                (nx-1)(ny-1), complex128 (FP64) or complex64 (MIXED): for each
 *                direction and level j = 1..nz the samples of E1 on
 *                p=0..nx, q=1..ny-1, then E2 on p=1..nx-1, q=0..ny, then E3 on
 *                p=1..nx-1, q=1..ny-1, each row-major in (p, q); at an interface
 *                level E3 is the upper layer's value.
 *  out_mem:      CAVITY_MEM_DEVICE or CAVITY_MEM_HOST for both outputs.
 *  iters_out, resid_out: host arrays of length ndir (may be NULL): Krylov
 *                iterations and final relative residual of (EJ1)/(uT1) per
 *                direction.  CAVITY_FP64: GMRES iterations of the direction.
 *                CAVITY_MIXED: block GMRES steps of the FP32 inner solves,
 *                summed over the FP64 refinement cycles (one step applies
 *                the operator to the whole group of up to 16 directions);
 *                the residual is the refinement's FP64 residual.
 * gmres_restart bounds the basis per direction (CAVITY_FP64) or the block
 * steps per refinement cycle (CAVITY_MIXED: min(gmres_restart, 30), at least
 * 2); gmres_max_iter bounds the iterations or block steps in total.
 * Returns CAVITY_ENOCONV (outputs filled) when a residual stays above
 * gmres_tol after gmres_max_iter iterations (CAVITY_FP64: when the true
 * residual, recomputed after GMRES stops on its estimate, exceeds
 * 10 gmres_tol). */
cavity_status cavity_solve(cavity_ctx* ctx, double kappa0, int nlayers,
                           const int* layer_levels, const double* eps_re,
                           const double* eps_im, int ndir, const double* theta,
                           const double* phi, const double* alpha, int out_mode,
                           int out_mem, void* aperture_out, void* field_out,
                           int* iters_out, double* resid_out);

/* Backscatter radar cross section (Sec. 7; formula from (EGa2):
 * sigma = (kappa0^2/pi) |e . (x_hat x L)|^2, L = int_Gamma (z x E)
 * exp(-i kappa0 x_hat.y) dy, x_hat = (sin t cos f, sin t sin f, cos t)).
 * aperture: ndir x n_ap complex128 (mem = CAVITY_MEM_DEVICE or _HOST) for the
 * wavenumber of the last prepare; obs_theta/obs_phi host arrays (length ndir);
 * pol selects e = theta_hat or phi_hat; sigma_out host array (length ndir). */
cavity_status cavity_rcs(cavity_ctx* ctx, int ndir, const void* aperture, int mem,
                         const double* obs_theta, const double* obs_phi, int pol,
                         double* sigma_out);

/* Release the context and all its device memory.  NULL is a no-op. */
void cavity_destroy(cavity_ctx* ctx);

/* Message of the last failed call on this context (or of the last failed
 * cavity_setup when ctx is NULL).  Owned by the library. */
const char* cavity_last_error(const cavity_ctx* ctx);

/* ---- step-level entry points (same conventions; device buffers) ----------
 * They expose the individual rows of the hot path so that each can be checked
 * on its own; cavity_solve is composed of exactly these steps. */

/* n_ap and the number of field samples per direction. */
cavity_status cavity_sizes(const cavity_ctx* ctx, long long* n_ap,
                           long long* field_per_dir);

/* Per-mode elimination results of the last prepare (Sec. 3/4):
 *  top:  5 x n_ap complex128 rows [tau | varsigma | 0...] laid out as
 *        tau over the aperture ordering (n_ap values: tau1 over N1, tau2 over
 *        N2, tau3 over N3) followed by varsigma over N1 and N2 (n1+n2 values);
 *        that is n_ap + n1 + n2 values in total.
 *  prof: (nz-1) x n_ap complex128 profiles P at levels j = 1..nz-1 (level-major,
 *        aperture ordering; E3 upper values at interfaces), may be NULL.
 *  profq:(nz-1) x (n1+n2) complex128 E3-driven profiles Q of E1/E2, may be NULL. */
cavity_status cavity_export_elimination(cavity_ctx* ctx, void* top, void* prof,
                                        void* profq);

/* The kernel table F(G)(rho) of Sec. 5.2 at rho = |(j1/Lx, j2/Ly)| for
 * j1 = 0..Px/2-1, j2 = 0..Py/2-1 (row-major, complex128), Px = 4 nx. */
cavity_status cavity_export_khat(cavity_ctx* ctx, void* khat);

/* The convolution periods chosen at setup, in aperture sides: Lx = pad_x a,
 * Ly = pad_y b; the kernel table of cavity_export_khat is
 * (pad_x nx / 2) x (pad_y ny / 2). */
cavity_status cavity_periods(const cavity_ctx* ctx, int* pad_x, int* pad_y);

/* Right-hand sides [g1; g2; 0] of (EJ1) for ndir directions (host angle
 * arrays) into out (ndir x n_ap complex128, device). */
cavity_status cavity_rhs(cavity_ctx* ctx, int ndir, const double* theta,
                         const double* phi, const double* alpha, void* out);

/* y = A x for the reduced aperture matrix of (EJ1)/(uT1): x, y ndir x n_ap
 * (device), complex128 when precision == CAVITY_FP64 or CAVITY_PAIR32 and
 * complex64 when CAVITY_MIXED.  Other precision values: CAVITY_EINVAL.  With a
 * truncated mode set (modes_m, modes_n) the rows of the dropped modes are 0. */
cavity_status cavity_apply(cavity_ctx* ctx, int ndir, int precision,
                           const void* x, void* y);

/* Allocation-free y = A x: the operator of cavity_apply, for callers that
 * may not allocate device memory -- for example a host application that owns
 * a fixed device memory budget and forbids libraries to call cudaMalloc in
 * its solve loop, where an allocation would also add an implicit device
 * synchronisation.  It needs a context that cavity_setup and cavity_prepare
 * built beforehand; the call itself allocates nothing.
 *  precision: CAVITY_FP64 (x, y complex128) or CAVITY_MIXED (FP32 operator,
 *             x, y complex64) only; CAVITY_PAIR32 and any other value return
 *             CAVITY_EINVAL.
 *  x, y:      ndir x n_ap device buffers of the context's device, caller-owned;
 *             y must not overlap x (the operator reads x while writing y).
 * The transform passes use a fixed 4 MiB device array inside the library
 * (held on every device that loads it, until exit) as scratch; sizes whose
 * scratch exceeds 4 MiB (e.g. more than about 2 directions at 64 x 64 in
 * FP64) are rejected with CAVITY_EINVAL and a message.  The first call on a
 * device looks up the array's device address; the context's device must be
 * current.  The call
 * synchronises the context's stream before it returns.  All calls share the
 * one array: calls that overlap on the GPU (other streams, other contexts,
 * other threads) race and must be serialised by the caller.  Nothing carries
 * over between calls: each call writes all scratch it reads.
 * The paper has no counterpart to this entry point. */
cavity_status cavity_apply_noalloc(cavity_ctx* ctx, int ndir, int precision,
                                   const void* x, void* y);

/* Interior field from given aperture coefficients (EInter + E123F): aperture
 * ndir x n_ap complex128, field as in cavity_solve for the context's precision. */
cavity_status cavity_field(cavity_ctx* ctx, int ndir, const void* aperture,
                           void* field);

/* Dense direct solve (Algorithm I/II Step 3) on the kept modes, step by step.
 *
 * cavity_dense_size: *n = number of kept unknowns, 3 mm nn + mm + nn with
 *   mm = modes_m, nn = modes_n (0 -> M, N); the kept block's rows and columns
 *   are these unknowns in Appendix A order (E1 over m = 0..mm, n = 1..nn, then
 *   E2 over m = 1..mm, n = 0..nn, then E3 over m = 1..mm, n = 1..nn, m-major).
 * cavity_dense_assemble (after cavity_prepare): writes the kept block of the
 *   matrix of (EJ1)/(uT1) -- the cavity part and the TBC integrals of Sec. 5.1
 *   under the discrete rule of Sec. 5.2 -- as complex64 into the device buffer
 *   a, row-major with leading dimension lda >= n (elements); entries carry
 *   FP32 rounding of sums over the frequency box.  CAVITY_EINVAL if n exceeds
 *   CAVITY_DENSE_MAX_N.
 * cavity_lu_factor: in-place LU factorisation with partial pivoting, P A = L U
 *   (L unit lower, U upper, both stored in a), of an n x n complex64 device
 *   matrix, row-major with leading dimension lda; ipiv (device, n ints)
 *   receives the row exchanged with row i at step i (0-based, as a sequence of
 *   exchanges).  *info (host) = -1, or the first step whose pivot column was
 *   exactly zero (the factors are then complete but U is singular and the call
 *   returns CAVITY_ESINGULAR).  1 <= n <= CAVITY_DENSE_MAX_N.
 * cavity_lu_solve: overwrites the nrhs right-hand sides b (device, complex64,
 *   right-hand side r at b + r ldb, ldb >= n) with the solutions of
 *   A x = b from cavity_lu_factor's output.  ipiv is read on the device and
 *   checked before b is touched: an entry outside 0..n-1 returns
 *   CAVITY_EINVAL with b unchanged.  b must not overlap lu or ipiv. */
cavity_status cavity_dense_size(const cavity_ctx* ctx, int* n);
cavity_status cavity_dense_assemble(cavity_ctx* ctx, void* a, int lda);
cavity_status cavity_lu_factor(cavity_ctx* ctx, void* a, int n, int lda, int* ipiv, int* info);
cavity_status cavity_lu_solve(cavity_ctx* ctx, const void* lu, int n, int lda, const int* ipiv,
                              int nrhs, void* b, int ldb);

/* ---- implementation options (chosen by the autotuner) ---------------------
 * Variants of the same arithmetic whose speed depends on the grid, the batch
 * and the device; results agree within the precision of the path (the FP32
 * operator variants to ~1e-7 relative, the group width within the solver
 * tolerance).  Set per context, at any time between calls; the
 * paper_2008_01966_gb300.autotune module times them and caches its choice.
 *  CAVITY_OPT_PASS_B_2048, CAVITY_OPT_PASS_C_2048: FP32 operator passes B and
 *      C on lines of 2048 points (512-point grid sides): 0 = each line on a
 *      pair of warps (one radix-2 step, then a 1024-point warp transform per
 *      warp; default), 1 = the block (Stockham) transform.
 *  CAVITY_OPT_GROUP_WIDTH: directions per group of the mixed solve's block
 *      Krylov iterations (one basis per group), 1..16; default 16.
 *  CAVITY_OPT_COARSE_MODES: two-level preconditioner of the mixed solve's
 *      inner FP32 iterations (Krylov solver): 0 (default) = the 3 x 3 block
 *      diagonal of each mode alone; mc > 0 = in addition the kept block of
 *      the modes m, n <= mc solved exactly with its FP32 LU factors (the
 *      coarse level, the modes that couple most through the TBC), factored
 *      at the first mixed solve after cavity_prepare or a change of mc; its
 *      3 mc^2 + 2 mc unknowns must not exceed CAVITY_DENSE_MAX_N.  Changes
 *      the iteration count, not the result beyond the solver tolerance.
 *  CAVITY_OPT_FIELD_FUSED: the complex64 field synthesis of square grids of
 *      32..512 points per side: 0 (default) = the fused persistent kernel at
 *      512 points per side (faster there), the two-pass kernels elsewhere;
 *      1 = the fused kernel on every square grid it supports; 2 = always the
 *      two-pass kernels.  The fields agree to FP32 rounding.  The FP32
 *      profiles are stored in the chosen kernel's layout at cavity_prepare,
 *      so a change takes effect at the next prepare (a solve re-prepares).
 * CAVITY_EINVAL for an unknown option or a value out of range. */
enum { CAVITY_OPT_PASS_B_2048 = 0, CAVITY_OPT_PASS_C_2048 = 1, CAVITY_OPT_GROUP_WIDTH = 2,
       CAVITY_OPT_COARSE_MODES = 3, CAVITY_OPT_FIELD_FUSED = 4, CAVITY_NUM_OPT = 5 };
cavity_status cavity_set_option(cavity_ctx* ctx, int option, int value);
cavity_status cavity_get_option(const cavity_ctx* ctx, int option, int* value);

/* ---- launch accounting (benchmark instrumentation, not part of the method) --
 * Every kernel the library launches belongs to one of CAVITY_NUM_KCLASS
 * classes (names from cavity_kernel_class).  Launches are always counted.
 * cavity_timing(ctx, 1) resets the counters and starts bracketing every launch
 * with CUDA events on the context's stream (adds a small host cost per launch);
 * cavity_timing(ctx, 0) stops.  cavity_timing_read synchronises the stream and
 * returns, per class, the summed event time in ms (0 when timing was off) and
 * the number of launches since the last reset; ms and launches are host arrays
 * of length nclass (<= CAVITY_NUM_KCLASS), either may be NULL.
 * cavity_kernel_class(k): the name of class k, a static string owned by the
 * library ("" for k outside 0..CAVITY_NUM_KCLASS-1). */
#define CAVITY_NUM_KCLASS 24
cavity_status cavity_timing(cavity_ctx* ctx, int enable);
cavity_status cavity_timing_read(cavity_ctx* ctx, int nclass, double* ms,
                                 long long* launches);
const char* cavity_kernel_class(int k);

#ifdef __cplusplus
}
#endif
#endif /* CAVITY_H */
