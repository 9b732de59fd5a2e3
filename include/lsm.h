/*
 * lsm.h - C ABI of the GB300 matrix-free elastic Lippmann-Schwinger solver.
 *
 * The library solves the discretised Lippmann-Schwinger (LS) equation for
 * the frequency-domain displacement u in a heterogeneous anisotropic elastic
 * medium split into a homogeneous isotropic background (lambda0, mu0, rho0)
 * and per-voxel contrasts dC (Voigt 6x6) and drho (Sec. 2, Eqs. 2-3, 8, 11):
 *
 *     A u = u - G * ( D.sigma + w^2 drho u ) = u0,   sigma_J = dC_JK eps_K(u),
 *
 * with eps the finite-difference Voigt strain (Eq. 18), D the central
 * difference divergence, G the sampled background Green's tensor and "*" a
 * zero-padded 3-D convolution evaluated by FFT (Eq. 21).  u0 is the
 * background field of a moment-tensor point source (Eqs. 13-16).  A u = u0
 * is solved with BiCGSTAB and the relative residual of Eq. 22.
 *
 * Conventions shared by every entry point:
 *   - grid n = {nx, ny, nz}; node (ix, iy, iz) sits at (ix, iy, iz) * dx metres;
 *   - a displacement field is 3 complex components, layout [c][iz][iy][ix]
 *     (x fastest), complex numbers interleaved (re, im): complex128 (16 B)
 *     unless an entry point says complex64;
 *   - dC is 21 planes of float64, layout [k][iz][iy][ix], k running over the
 *     upper triangle of the symmetric Voigt matrix row by row:
 *     (1,1),(1,2),...,(1,6),(2,2),...,(6,6); Voigt order 11,22,33,23,13,12
 *     (Sec. 3.1, Eq. 17); drho is one float64 plane [iz][iy][ix];
 *   - moment tensors are Voigt 6-vectors (M11, M22, M33, M23, M13, M12);
 *   - time dependence exp(-i w t): outgoing waves are exp(+i w r / c);
 *   - every pointer argument named as "device" must be CUDA device memory of
 *     the current device; the library never writes to caller inputs;
 *   - calls are ordered on the handle's stream and asynchronous with respect
 *     to the host unless they return host values (lsm_solve*, which
 *     synchronise that stream before returning);
 *   - errors are returned as lsm_status codes; no entry point aborts or traps;
 *     lsm_last_error() describes the most recent failure of a handle.
 *
 * Every path runs in hand-written CUDA kernels (sm_103a).  Nothing here
 * calls cuFFT or cuBLAS.
 */
#ifndef LSM_H
#define LSM_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lsm_ctx *lsm_t;

typedef enum {
    LSM_OK = 0,
    LSM_ERR_ARG = -1,        /* invalid argument (null pointer, size, unsupported grid) */
    LSM_ERR_CUDA = -2,       /* a CUDA runtime call failed */
    LSM_ERR_OOM = -3,        /* device allocation failed */
    LSM_ERR_BREAKDOWN = -4,  /* BiCGSTAB breakdown (rho, omega or <r^,v> vanished or non-finite) */
    LSM_ERR_NOCONV = -5,     /* iteration limit reached; the last iterate is returned */
    LSM_ERR_TIMEOUT = -6,    /* reserved for bounded device waits */
    LSM_WARN_SOURCE_ON_NODE = 1 /* lsm_source: a node coincides with the source; u0 = 0 there */
} lsm_status;

enum { LSM_FP64 = 0, LSM_MIXED = 1 };
enum { LSM_GREEN_EXACT = 0, LSM_GREEN_PAPER = 1 };
enum { LSM_KERNEL_DIFF = 0, LSM_KERNEL_H = 1 };
enum { LSM_RESIDUAL_DFLOAT = 0, LSM_RESIDUAL_FP64 = 1 };

typedef struct {
    int precision;     /* LSM_FP64: complex128 throughout.
                          LSM_MIXED: complex64 FFTs/contractions with an outer residual
                          b - A x of Eq. 22 (see residual) and iterative refinement in
                          complex128 storage; FP64-accurate inner products. */
    int green;         /* LSM_GREEN_EXACT: full isotropic solution of Eq. 7 (default).
                          LSM_GREEN_PAPER: near field Eq. A.4 + far field Eq. A.5. */
    double tol;        /* target relative residual of Eq. 22 (default 1e-10) */
    int maxit;         /* BiCGSTAB iteration limit per solve (FP64) or per inner solve (mixed) */
    double inner_tol;  /* mixed: the tightest relative tolerance an FP32 inner solve is asked for.
                          Each inner solve aims at 0.1 * tol / (current FP64 relres),
                          clamped to [inner_tol, 0.1] (default 1e-6) */
    int max_outer;     /* mixed: refinement steps limit (default 8) */
    int taper;         /* absorbing boundary (Eq. 25): width in nodes of the layer in which the
                          contrast sources are weighted by prod_a [1 - exp(-l_a^2 / (N_a dx^2))],
                          l_a = distance to the outer node plane along axis a, N_a = nodes along a;
                          0 = none (default) */
    int graph;         /* 1 (default): the BiCGSTAB iteration kernels of a solve are captured once
                          into a CUDA graph (two iterations per graph, kernels of stopped systems
                          return at once) and replayed, one host synchronisation per replay;
                          the graph is kept with the solver workspace and reused by later solves
                          of the same batch size.  0: every kernel is launched from the host. */
    int kernel;        /* LSM_KERNEL_DIFF (default): the derivative in H of Eq. 9 is taken as the
                          central difference (Eq. 18's stencil) of the contrast stress, so three
                          source components are transformed each way against 6 spectra.
                          LSM_KERNEL_H: Eq. 21 literally, with H_iJ sampled from the analytic
                          derivative of the Green's tensor (Appendix A, Eqs. A.6-A.11 for
                          LSM_GREEN_PAPER) and transformed: 9 forward transforms (6 stress, 3
                          density), 24 spectra (18 H, 6 G), about 4x the spectrum memory.  The
                          adjoint calls (lsm_adjoint, lsm_solve_adjoint, lsm_gradient) and
                          lsm_apply_static return LSM_ERR_ARG for it. */
    int residual;      /* LSM_MIXED: arithmetic of the outer residual's operator apply.
                          LSM_RESIDUAL_FP64 (default): FP64.  LSM_RESIDUAL_DFLOAT: double-float
                          pairs (two FP32 words, about 48 significand bits, unit roundoff near
                          2^-48; see lsm_apply_df) on the FP32 pipe, with the iterate scaled by a
                          power of two to RMS(b) ~ 1 first: several times faster on this GPU,
                          whose FP64 rate is 1/64 of its FP32 rate, but narrower than FP64.
                          Adjoint solves always use FP64.  Ignored for LSM_FP64 handles. */
    int fused_dots;    /* LSM_MIXED, 1 (default): the inner products of an FP32 BiCGSTAB
                          iteration (<r^, v> for alpha, <t, s> and <t, t> for omega) are summed in
                          the epilogue of the operator apply that writes v and t, where that
                          epilogue is the warp-per-line inverse x transform (grid sides 8, 32 and
                          128 with the default schedule; forward solves), instead of by two vector
                          kernels that read the vectors again.  0: always the vector kernels.
                          Both sum exact products with compensation into FP64 totals; the results
                          agree to rounding.  FP64 iterations always use the vector kernels. */
} lsm_opts;

/* Fill *o with the defaults listed above.  o: host pointer, not null. */
void lsm_default_opts(lsm_opts *o);

/*
 * Create a handle for one medium at one angular frequency omega [rad/s].
 * Sec. 2 (Eqs. 2-3) defines the split into background and contrast;
 * Appendix A and Eq. 21 define the Green's tensor whose spectrum is built here.
 *
 *   out      host pointer receiving the handle (set to NULL on failure)
 *   n        host int[3] = {nx, ny, nz}; each n_a >= 2 and 2 n_a must factor into
 *            2, 3 and 5 with 2 n_a <= 512
 *   dx       grid spacing [m], > 0
 *   lambda0, mu0, rho0  background Lame parameters [Pa] and density [kg/m^3], mu0 > 0,
 *            lambda0 + 2 mu0 > 0, rho0 > 0
 *   dC       device float64, 21 * nz*ny*nx values (layout above); copied
 *   drho     device float64, nz*ny*nx values; copied
 *   omega    angular frequency [rad/s], > 0
 *   opts     host pointer or NULL for defaults
 *   stream   cudaStream_t (as void*) all work of this handle is ordered on; NULL = legacy default
 *
 * The library owns copies of the contrast (FP64, plus FP32 in LSM_MIXED), the
 * octant-symmetric Green spectrum, and the workspaces.  Synchronises the
 * stream before returning (setup only).
 */
lsm_status lsm_create(lsm_t *out, const int n[3], double dx,
                      double lambda0, double mu0, double rho0,
                      const double *dC, const double *drho,
                      double omega, const lsm_opts *opts, void *stream);

/*
 * Create a handle for the medium of `base` at another angular frequency.
 * The contrast storage is shared (reference counted) with `base`; the new
 * handle builds its own Green spectrum (Eq. 21) and workspaces.  Same
 * options and stream as `base`.  Handles sharing a medium may be solved
 * together by lsm_solve_batched.
 */
lsm_status lsm_create_shared(lsm_t *out, lsm_t base, double omega);

/*
 * Background field of a moment-tensor point source (Eqs. 13-16, t0 = 0):
 *   u0_i(x) = -M_jk dG_ij/dx_k (x - xs).
 *   M   host double[6], Voigt (M11, M22, M33, M23, M13, M12)
 *   xs  host double[3], source position [m]
 *   u0  device complex128, 3 * nz*ny*nx (written)
 * Returns LSM_WARN_SOURCE_ON_NODE (and u0 = 0 on that node, the cell
 * average of an odd function) when a node coincides with xs.  Synchronises
 * the handle's stream to read that flag.
 */
lsm_status lsm_source(lsm_t h, const double M[6], const double xs[3], void *u0);

/*
 * Background fields of nm moment tensors at one source position (Eqs. 13-16),
 * as nm calls of lsm_source would give them; the Green's-tensor derivative
 * (the transcendental part) is evaluated once per node for all of them.
 *   nm  1 .. 4096
 *   M   host double[6 * nm], tensor m at M[6m .. 6m+5] in lsm_source's order
 *   xs  host double[3], source position [m]
 *   u0  host array of nm device pointers, each complex128 3 * nz*ny*nx (written)
 * LSM_ERR_ARG for nm out of range, a null pointer or a non-finite input;
 * LSM_WARN_SOURCE_ON_NODE as for lsm_source.  Synchronises the stream once.
 */
lsm_status lsm_source_moments(lsm_t h, int nm, const double *M, const double xs[3], void *const *u0);

/*
 * One application of the LS operator (Eqs. 19-21): Au = A u in FP64.
 *   u, Au  device complex128, 3 * nz*ny*nx; u != Au required (no aliasing).
 */
lsm_status lsm_apply(lsm_t h, const void *u, void *Au);

/*
 * The same operator in FP32 arithmetic (complex64 FFTs and contraction):
 *   u, Au  device complex64, 3 * nz*ny*nx; u != Au.
 * Only for handles created with LSM_MIXED (else LSM_ERR_ARG).
 */
lsm_status lsm_apply_c64(lsm_t h, const void *u, void *Au);

/*
 * The operator of lsm_apply in double-float arithmetic: every real quantity of
 * the path (field, strain, stress, contrast, spectra, twiddles) is carried as
 * an unevaluated sum hi + lo of two FP32 numbers; sums use two-sum, products
 * the exact FMA product error (Dekker 1971).  Normwise relative error a few
 * times 2^-48 times the FFT depth, far below the tolerances FP32 can certify,
 * at the FP32 pipe's rate.  FP32's exponent range applies: entries of u and
 * of the intermediate fields must stay within about 1e-30 .. 1e30 in modulus
 * (the mixed solver scales its iterate first; this entry point does not).
 *   u, Au  device complex128, 3 * nz*ny*nx; u != Au.  Au is written as
 *          complex128 (the pairs are converted in place at the end).
 * Either operator form (lsm_opts.kernel).  Only for handles created with
 * LSM_MIXED and LSM_RESIDUAL_DFLOAT (else LSM_ERR_ARG).
 */
lsm_status lsm_apply_df(lsm_t h, const void *u, void *Au);

/*
 * Adjoint operator A^H v in FP64 (the transposes of the apply's steps in
 * reverse order: conjugate Green spectrum, conjugate derivative factors,
 * transposed contrast and strain maps).
 *   v, AHv  device complex128, 3 * nz*ny*nx; v != AHv.
 */
lsm_status lsm_adjoint(lsm_t h, const void *v, void *AHv);

/*
 * Solve A x = b with BiCGSTAB (Sec. 3.2) to the handle's tolerance on the
 * relative residual of Eq. 22.
 *   b       device complex128, 3 * nz*ny*nx (right-hand side, e.g. lsm_source's u0)
 *   x       device complex128, 3 * nz*ny*nx; on entry the initial guess (zeros for
 *           none), on exit the solution (the last iterate on LSM_ERR_NOCONV)
 *   iters   host int* or NULL: BiCGSTAB iterations (mixed: total inner iterations)
 *   relres  host double* or NULL: the true residual ||b - A x|| / ||b|| at exit, from an
 *           FP64 apply (LSM_FP64) or the mixed mode's residual apply (double-float by
 *           default, see lsm_opts.residual), not the recursively updated one
 * Synchronises the handle's stream.
 */
lsm_status lsm_solve(lsm_t h, const void *b, void *x, int *iters, double *relres);

/*
 * Solve nsys independent systems together (frequencies x sources).  All
 * handles must share one medium (lsm_create_shared) and one precision;
 * systems that use the same handle share its Green spectrum.  Each kernel
 * of the solve runs over all unconverged systems in one launch; converged
 * systems are masked out.
 *   hs      host array of nsys handles (repeats allowed)
 *   b, x    host arrays of nsys device pointers, as in lsm_solve
 *   iters, relres, status  host arrays of nsys entries, or NULL
 * Returns LSM_OK when every system converged, else the first failing status.
 */
lsm_status lsm_solve_batched(int nsys, const lsm_t *hs, const void *const *b, void *const *x,
                             int *iters, double *relres, lsm_status *status);

/*
 * Adjoint solve A^H x = b (BiCGSTAB with the adjoint apply, same options and stopping rule as
 * lsm_solve).  With b = R^T g (receiver-sampling adjoint of a misfit gradient g) the solution is
 * the adjoint field lambda of the discrete-adjoint gradient of the LS solution (Sec. 3.2, Eq. 21).
 *   b, x, iters, relres  as in lsm_solve (relres is ||b - A^H x|| / ||b||).
 */
lsm_status lsm_solve_adjoint(lsm_t h, const void *b, void *x, int *iters, double *relres);

/*
 * Replace the medium's contrast (all handles sharing it see the change; the Green spectra do not
 * depend on the contrast and are kept).  dC, drho: device float64, layouts as in lsm_create; copied.
 */
lsm_status lsm_set_contrast(lsm_t h, const double *dC, const double *drho);

/*
 * Contrast gradient of the LS solution (discrete adjoint of Eqs. 8, 11 and 18): for the forward
 * solution u (A u = u0) and an adjoint field lam (A^H lam = r), writes the gradient of
 * Re<lam, K (Dv dC eps(u) + w^2 drho u)> = Re<r, du> with respect to
 *   gC    device float64 [21][nz][ny][nx]: the 21 packed Voigt contrast planes (an off-diagonal
 *         entry counts both of its symmetric positions),
 *   grho  device float64 [nz][ny][nx]: the density contrast;
 * accumulate != 0 adds to gC and grho (sums over frequencies and sources), else overwrites.
 * u, lam: device complex128, 3 * nz*ny*nx.
 */
lsm_status lsm_gradient(lsm_t h, const void *u, const void *lam, double *gC, double *grho, int accumulate);

/*
 * Moment-tensor gradient gM_J = Re<lam, d u0/d M_J> (Eqs. 13-16; u0 is linear in M), J over the
 * Voigt components (M11, M22, M33, M23, M13, M12), for a source at xs [m].
 *   lam  device complex128, 3 * nz*ny*nx;  gM  host double[6] (written).  Synchronises the stream.
 */
lsm_status lsm_source_gradient(lsm_t h, const double xs[3], const void *lam, double gM[6]);

/*
 * Receiver time traces from frequency-domain receiver data (Sec. 4.1.2: solve at the positive and
 * negative frequencies up to Nyquist, inverse Fourier transform).  With exp(-i w t) and a real
 * medium U(-f) = conj(U(f)), so positive frequencies f_k = k df (k = 0..nf-1) suffice:
 *   u(t_j) = df [W_0 U_0 + 2 Re sum_{k>=1} W_k U_k exp(-2 pi i f_k t_j)],  t_j = j dt,
 * W_k the Ricker spectrum 2 f^2/(sqrt(pi) fp^3) exp(-f^2/fp^2) exp(+2 pi i f t0).
 *   nf       1..12288 frequencies;  df  spacing [Hz]
 *   ntr      traces (e.g. receivers x 3 components);  spectra  device complex128 [nf][ntr]
 *   nt, dt   samples and interval [s];  fp  Ricker peak frequency [Hz];  t0  delay [s]
 *   traces   device float64 [ntr][nt] (written);  stream  cudaStream_t (as void*)
 */
lsm_status lsm_time_traces(int nf, double df, int ntr, const void *spectra, int nt, double dt, double fp, double t0,
                           double *traces, void *stream);

/*
 * Receiver seismograms of one moment-tensor source, the whole chain of Sec. 4.1.2: for each
 * frequency f_k = k df, k = 1 .. nf-1, the background field (Eqs. 13-16) and the LS solution of
 * A_k u_k = u0_k (BiCGSTAB to the handle's tolerance, Eq. 22), the three displacement components
 * read at the receiver nodes, then the time traces of lsm_time_traces (k = 0 contributes nothing:
 * the Ricker weight vanishes at f = 0).  The frequencies are solved in waves of up to `wave`
 * systems, each wave one lsm_solve_batched over handles created with lsm_create_shared.
 *   base     handle of the medium; its options (precision, tolerance, operator form, taper) are
 *            used, its own frequency is not
 *   nf, df   2 <= nf <= 12288 frequencies f_k = k df [Hz], df > 0
 *   M, xs    host double[6] moment tensor (Voigt, as lsm_source), host double[3] position [m]
 *   nrec     number of receivers (>= 1);  rec  host int[3 * nrec]: node indices (ix, iy, iz) of
 *            receiver r at rec[3r .. 3r+2], each inside the grid
 *   nt, dt, fp, t0  samples, interval [s], Ricker peak frequency [Hz] and delay [s], as in
 *            lsm_time_traces
 *   traces   device float64 [nrec][3][nt] (written when the call returns LSM_OK or
 *            LSM_WARN_SOURCE_ON_NODE): trace 3 r + c is component c at receiver r
 *   wave     1 .. 256 systems per batched solve
 *   iters, relres  host int[nf] / double[nf] or NULL: per frequency as lsm_solve reports them
 *            (entry 0 is 0)
 * Allocates, for the duration of the call, the [nf][3 nrec] receiver spectra and per wave the
 * handles' Green spectra and two fields per frequency; the base handle's solver workspace grows to
 * `wave` systems and stays.  Returns the first failing status of a solve (traces not written),
 * LSM_WARN_SOURCE_ON_NODE if a node coincides with the source (u0 = 0 there), else LSM_OK.
 * Synchronises the stream.
 */
lsm_status lsm_seismograms(lsm_t base, int nf, double df, const double M[6], const double xs[3], int nrec,
                           const int *rec, int nt, double dt, double fp, double t0, double *traces, int wave,
                           int *iters, double *relres);

/* Number of kernel launches the library has issued on this handle (diagnostics). */
long long lsm_launch_count(lsm_t h);

/*
 * FFT schedules (no counterpart in the paper).  Each apply stage can run one of
 * a few kernel variants: v[0] strain + contraction: 0 = stress kernel, then the
 * divergence with the forward x pass, 1 = contraction and divergence fused in
 * one z-marching kernel (no stress round trip through memory); v[1] forward
 * x pass, v[2] forward y pass, v[4] inverse y pass, v[5] inverse x pass and
 * epilogue: 0 = compile-time two-step FFT where the line length allows it
 * (16..512), 1 = runtime mixed-radix Stockham engine, 2 = the same with half
 * its tile; v[3] z pass with the Green multiply: 0..2 as above (0 is the
 * register-resident kernel in FP32), 3 = the shared-memory two-step kernel.
 * Every variant computes the same operator.  precision: LSM_FP64 (the FP64
 * applies) or LSM_MIXED (the FP32 applies of a mixed handle).  The schedule
 * belongs to the medium (all handles sharing it); setting one drops the
 * captured iteration graphs.  LSM_ERR_ARG for an invalid variant.
 */
lsm_status lsm_set_schedule(lsm_t h, int precision, const int v[6]);
lsm_status lsm_get_schedule(lsm_t h, int precision, int v[6]);

/*
 * The project's tuner: times `reps` batched applies (1..100) of nsys systems
 * (1..64, the batch size the solves will use) under every variant set, per
 * precision the handle runs, with CUDA events around each stage, and keeps for
 * every stage the fastest variant.  The chosen schedules are returned in v64
 * and v32 (host int[6] each, may be NULL; v32 is all 0 for an LSM_FP64
 * handle).  Sizes the solver workspace for nsys systems and allocates 1 + nsys
 * 3N complex128 buffers for the duration; resets the stage timer's totals;
 * synchronises the stream.
 */
lsm_status lsm_autotune(lsm_t h, int nsys, int reps, int v64[6], int v32[6]);

/*
 * Diagnostic (no counterpart in the paper): conj(a) . b over n complex64
 * elements, accumulated exactly as the mixed solver's FP32 BiCGSTAB inner
 * products are (each FP32 product split exactly with an FMA, compensated FP32
 * partial sums over 16 elements, FP64 totals and FP64 cross-thread sums).
 *   a, b  device complex64, n elements; out host double[2] = (re, im)
 * LSM_ERR_ARG for a null pointer or n < 0.  Allocates a small scratch buffer;
 * synchronises the handle's stream.
 */
lsm_status lsm_dot_c64(lsm_t h, long long n, const void *a, const void *b, double out[2]);

/*
 * Diagnostics for roofline measurement (no counterpart in the paper).
 * lsm_timer_start(h, enable): zero the totals and the executed-apply counters, and (enable != 0)
 * from now on record a CUDA event pair on the handle's stream around every launch of every stage
 * of the operator apply, on every handle that shares h's medium.  Stages: 0 strain +
 * contraction, 1 contrast source + x FFT, 2 y FFT, 3 z FFT + Green multiply + inverse z FFT,
 * 4 inverse y FFT, 5 inverse x FFT + epilogue.  Synchronises the stream.
 * lsm_timer_read: synchronise, then write total milliseconds and launches per slot
 * (slot = 6 * p + stage, p = 0 for FP64 applies and the mixed solver's double-float residual
 * applies, 1 for FP32 applies) and the number of system-level operator applies executed in
 * FP64 or double-float (applies[0]) and FP32 (applies[1]) since lsm_timer_start; systems masked
 * out of a batched launch are not counted.  Any out-pointer may be NULL.
 */
lsm_status lsm_timer_start(lsm_t h, int enable);
lsm_status lsm_timer_read(lsm_t h, double ms[12], long long launches[12], long long applies[2]);

/*
 * FP64 operator apply that allocates nothing (the paper has no counterpart).  It serves callers
 * that cannot call cudaMalloc when they apply the operator: a process whose device memory was
 * reserved up front by another allocator (for instance a serving framework whose caching
 * allocator holds the device), or a loop that must not stop halfway on an out-of-memory error or
 * on the device-wide synchronisation cudaMalloc may bring.  Same result as lsm_apply; the handle
 * itself must already exist (lsm_create allocates).
 *   u, Au  device complex128, 3 * nz*ny*nx; u != Au.
 * The workspace is one library-wide array in device global memory of 64 MiB, present on every
 * GPU that loads the library until the process exits.  A grid needs 384 * nx * ny * (nz + 2)
 * bytes of it plus 256 (the largest cubic grid the library accepts that fits is 54^3); a grid
 * that needs more is rejected with LSM_ERR_ARG, and so is a call made while another device than
 * the handle's is current.  The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress), so make that first call before any stream capture.  All calls share
 * the one array and each call leaves its contents behind; nothing in it needs to start at zero.
 * Calls whose work overlaps on the GPU (different streams, or different handles without
 * ordering between them) race on the array: order them on one stream.
 */
lsm_status lsm_apply_static(lsm_t h, const void *u, void *Au);

/* Release every device buffer the handle owns (shared contrast when its last user goes). */
void lsm_destroy(lsm_t h);

/* Text of the most recent error on h (or of the last failed create when h is NULL). */
const char *lsm_last_error(lsm_t h);

#ifdef __cplusplus
}
#endif
#endif /* LSM_H */
