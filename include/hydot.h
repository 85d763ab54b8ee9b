/*
 * hydot.h -- C ABI of libhydot, the GB300 (sm_103a) hot path of the Born-approximation
 * method for hyperspectral diffuse optical tomography (Saibaba, Kilmer, Miller & Fantini,
 * "Fast algorithms for Hyperspectral Diffuse Optical Tomography", arXiv:1410.0986).
 *
 * What the library computes
 *   - Fields (Section 2.2, eqn:discincident and eqn:multipleshifted; Section 3): for every
 *     wavelength lambda_j and every source s / detector d, the discrete diffusion solve
 *         A_j phi = e_cell,
 *     A_j = K + sigma_j M + sigma'_j R restated as a cell-centred finite-volume 7-point
 *     operator on a box of nx*ny*nz cells of side h: interior faces D_j*h, absorption
 *     mu_a,j*h^3, Robin faces 2 D_j h^2 / (h + 4 A D_j) (A = 0: Dirichlet), and for a
 *     modulated source an extra i*omega*h^3/c_medium on the diagonal. mu_a,j = sum_c
 *     eps_c(lambda_j) c_bg,c and D_j = 1 / (3 (mu_a,j + mu_s'(lambda_j))).
 *     The adjoint (detector) fields are the same solves with the detector cell as source
 *     (Section 2.1, reciprocity).
 *   - Born rows (eqn:lippschwin, eqn:perturbation, eqn:measurement):
 *         J[(s,d,lambda),(c,x)] = -h^3 eps_c(lambda) phi_s(x;lambda) phi_d(x;lambda).
 *   - Implicit products y = J x and g += J^T y with the fields resident.
 *
 * Conventions (all calls)
 *   - Voxel index x = (k*ny + j)*nx + i (i fastest), N = nx*ny*nz.
 *   - A wavelength slice [lam0, lam0+nlam) is addressed by its own arrays: phi_src is
 *     [nlam][n_src][N] and phi_det is [nlam][n_det][N] for that slice only.
 *   - Rows of J / entries of y inside a slice: r = (s*n_det + d)*nlam + (lambda - lam0)
 *     (wavelength fastest, then detector, then source: E_k = I (x) I (x) diag(eps_k)).
 *   - Columns of J / entries of x and g: c*N + x (chromophore-major).
 *   - Element type of every bulk array: double for HYDOT_FP64, float for HYDOT_MIXED;
 *     with omega != 0 the fields are complex (interleaved re, im) of that precision.
 *   - Bulk arrays (fields, J, x, y, g) are DEVICE pointers owned by the caller; the
 *     library never frees them. Work is enqueued on the context's stream and is complete
 *     when that stream is synchronised (hydot_solve_fields synchronises it itself).
 *   - Every call returns a hydot_status; on error, hydot_last_error(ctx) describes it.
 *     No call aborts the process or throws across the ABI.
 */
#ifndef HYDOT_H
#define HYDOT_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hydot_ctx hydot_ctx; /* opaque: device coefficient tables, workspace, stream */

typedef enum {
  HYDOT_OK = 0,
  HYDOT_ERR_ARG = -1,           /* invalid argument; nothing was enqueued */
  HYDOT_ERR_OOM = -2,           /* a device or host allocation failed */
  HYDOT_ERR_CUDA = -3,          /* a CUDA call failed (message holds cudaGetErrorString) */
  HYDOT_ERR_NOT_CONVERGED = -4, /* some field missed its tolerance: best iterate written; or the
                                 * host eigensolver of a sketch or deflation step did not converge
                                 * (the message says which; outputs are then not valid) */
  HYDOT_ERR_TIMEOUT = -5,       /* a bounded device wait gave up */
  HYDOT_ERR_STATE = -6,         /* call not valid for this context (e.g. complex Born) */
  HYDOT_ERR_HOST = -7           /* a host-side failure other than an allocation (for example a
                                 * worker thread that could not start); the message says what */
} hydot_status;

typedef enum {
  HYDOT_FP64 = 0,  /* FP64 Jacobi-PCG (COCG when omega != 0), no refinement */
  HYDOT_MIXED = 1  /* FP32 inner PCG/COCG with iterative refinement: the iterate and its residual
                    * are double-float (two FP32 words, about 48 significant bits) computed with
                    * FP32 error-free transformations; per-field sums and tests in FP64 */
} hydot_precision;

typedef struct {
  /* grid */
  int nx, ny, nz;          /* cells per axis, each >= 1 */
  double h_mm;             /* cell side, mm, > 0 */
  double robin_A[6];       /* Robin coefficient per face -x,+x,-y,+y,-z,+z (eqn:robin); 0 = Dirichlet */
  /* medium (host arrays, copied during hydot_setup) */
  int n_lambda;            /* wavelengths, >= 1 */
  int n_chrom;             /* chromophore species, 1..16 */
  const double* eps;       /* [n_lambda][n_chrom] extinction, /mm/mM */
  const double* c_bg;      /* [n_chrom] background concentration, mM */
  const double* mus_prime; /* [n_lambda] reduced scattering, /mm */
  double omega;            /* modulation, rad/ns; 0 => continuous wave, real fields */
  double c_medium;         /* speed of light in the medium, mm/ns (used when omega != 0) */
  /* optodes (host arrays, copied): cell indices (i, j, k), all distinct from each other */
  int n_src, n_det;
  const int* src_ijk;      /* [n_src][3] */
  const int* det_ijk;      /* [n_det][3] */
  /* solver */
  int precision;           /* hydot_precision */
  double tol;              /* stop when ||b - A x||_2 <= tol ||b||_2 ...                    */
  double tol_cw;           /* ... and max_i |b - A x|_i / (|A||x| + |b|)_i <= tol_cw (0: off) */
  double inner_tol;        /* HYDOT_MIXED: residual reduction per FP32 inner solve (0: 1e-5)  */
  int max_iter;            /* cap on Krylov iterations per field, all cycles together (0: 20000) */
  int deflation_k;         /* size of the recycled deflation basis, 0..32 (0: off)            */
  int max_lambda_per_call; /* largest nlam passed to hydot_solve_fields (0: n_lambda)          */
  double cw_floor;         /* >= 0. With c = cw_floor > 0 the componentwise test of a field f at
                            * wavelength j uses |b - A x|_i / (|A||x| + |b| + theta_f)_i with
                            * theta_f = c * sigma_j * min |x_f| over its partner optode cells
                            * (detectors for a source field, sources for a detector field;
                            * sigma_j = mu_a h^2 / D in the operator scaled by 1/(D h)). Since
                            * (A/(D h)) 1 >= sigma_j entrywise and A^-1 >= 0, the residual entries
                            * this admits change the field by at most tol_cw * c times its smallest
                            * partner value anywhere, so c = tau / tol_cw keeps every Born entry
                            * J[(s,d,.),.] within about tau of its row maximum while cells far from
                            * every optode stop driving refinement. 0: plain componentwise test.
                            * With omega != 0 the same holds with |x| the modulus and sigma_j the
                            * real part: the frequency term is one imaginary shift i w on every
                            * cell, so |A^-1| = |int_0^inf e^(-t Re A) e^(-i w t) dt| <= (Re A)^-1
                            * entrywise, and Re A is the continuous-wave operator. */
} hydot_problem;

typedef struct {
  int n_fields;            /* fields solved by the call */
  int n_not_converged;     /* fields that missed tol / tol_cw within max_iter */
  int iters_max;           /* Krylov iterations of the slowest field (all cycles) */
  double iters_mean;       /* mean Krylov iterations per field */
  int cycles_max;          /* refinement cycles of the slowest field */
  double resid_max;        /* largest final ||b - A x||_2 / ||b||_2 (FP64) */
  double cw_max;           /* largest final componentwise backward error */
} hydot_stats;

/* Version of this ABI (major*10000 + minor*100 + patch). */
int hydot_version(void);

/* Validates *p, copies its host arrays, computes the per-wavelength coefficients
 * (mu_a, D, the scaled absorption and Robin terms), allocates the workspace for
 * max_lambda_per_call*(n_src+n_det) simultaneous fields and, when deflation_k > 0, builds the
 * recycled deflation basis. stream: a cudaStream_t (NULL = the legacy default stream).
 * On success *out owns everything the library allocated; free it with hydot_destroy.
 * Errors: HYDOT_ERR_ARG (bad sizes, optodes outside the grid or sharing a cell, bad
 * tolerances), HYDOT_ERR_OOM, HYDOT_ERR_CUDA. On error *out is NULL. */
int hydot_setup(const hydot_problem* p, void* stream, hydot_ctx** out);

/* Sets the stream later calls enqueue on. */
int hydot_set_stream(hydot_ctx* ctx, void* stream);

/* Fields for wavelengths [lam0, lam0+nlam) (eqn:multipleshifted for each source and detector):
 * writes phi_src [nlam][n_src][N] and phi_det [nlam][n_det][N] (device, caller-owned).
 * Either pointer may be NULL to skip that set (its solves are not run).
 * Synchronises the stream (convergence is decided on the device and polled). If st is not
 * NULL it receives the statistics. Returns HYDOT_ERR_NOT_CONVERGED (best iterates written)
 * when a field missed tol / tol_cw within max_iter. */
int hydot_solve_fields(hydot_ctx* ctx, int lam0, int nlam, void* phi_src, void* phi_det,
                       hydot_stats* st);

/* Field solves of several contexts in one call: a batch of independent problems of uneven size
 * (one phantom per context, e.g. frequency-domain phantoms of different grid sizes), each solved as
 * hydot_solve_fields(ctxs[i], lam0[i], nlam[i], phi_src[i], phi_det[i], &st[i]) would. The
 * contexts run concurrently, each from its own host thread on the stream its context holds, so
 * small grids overlap on the GPU instead of queueing behind one another; give every context its
 * own stream (hydot_set_stream) or the work serialises on the shared one. All contexts must be
 * on the caller's current device and distinct (a context repeated in the list is HYDOT_ERR_ARG:
 * its workspace would be shared by two threads). phi_src / phi_det entries follow the rules of
 * hydot_solve_fields; st and status may be NULL, else they receive n entries (status: each
 * context's own return code, its message in hydot_last_error of that context; when the lists
 * themselves are rejected, no context runs, every status entry holds that code and the message is
 * in hydot_last_error(NULL)). Synchronous.
 * Returns the first error other than HYDOT_ERR_NOT_CONVERGED in list order, else
 * HYDOT_ERR_NOT_CONVERGED when any field missed its tolerance, else HYDOT_OK. */
int hydot_solve_batch(hydot_ctx* const* ctxs, int n, const int* lam0, const int* nlam, void* const* phi_src,
                      void* const* phi_det, hydot_stats* st, int* status);

/* Born rows [row0, row0+nrows) of the slice [lam0, lam0+nlam) into J (device, row-major,
 * leading dimension ldJ >= n_chrom*N elements): J[r-row0][c*N + x]. Continuous wave only
 * (HYDOT_ERR_STATE otherwise). Rows outside the slice are HYDOT_ERR_ARG. Asynchronous. */
int hydot_born_assemble(hydot_ctx* ctx, const void* phi_src, const void* phi_det, int lam0, int nlam,
                        long long row0, long long nrows, void* J, long long ldJ);

/* y = J x for the slice: x [n_chrom*N], y [n_src*n_det*nlam] (overwritten). Continuous wave
 * only. Asynchronous; uses library workspace, so calls on one context must not overlap. */
int hydot_born_apply(hydot_ctx* ctx, const void* phi_src, const void* phi_det, int lam0, int nlam,
                     const void* x, void* y);

/* g += J^T y for the slice: y [n_src*n_det*nlam], g [n_chrom*N] (accumulated, so calls over
 * consecutive slices sum to the full product). Continuous wave only. Asynchronous. */
int hydot_born_apply_T(hydot_ctx* ctx, const void* phi_src, const void* phi_det, int lam0, int nlam,
                       const void* y, void* g);

/* Adjoint fields (Section 5: the misfit gradient -dmu/dp^T H^T (y - H mu) needs H^T times a data
 * vector; since phi_d = A^-1 e_d and A is symmetric, sum_d y[s,d,lambda] phi_d = A^-1 (sum_d
 * y[s,d,lambda] e_d), one solve per source and wavelength instead of the stored detector fields):
 *     A_lambda psi[a][s] = sum_d y[(s*n_det + d)*nlam + a] e_(detector cell d)
 * for every source s and wavelength lambda = lam0 + a of the slice. y: DEVICE [n_src*n_det*nlam]
 * (slice rows as for hydot_born_apply); psi: DEVICE [nlam][n_src][N], written. The same solver,
 * tolerances and refinement as hydot_solve_fields (each right-hand side normalised to unit 2-norm,
 * the norm applied to the output; the componentwise floor weighs the field against its own source
 * cell); starts from zero. Continuous wave only (HYDOT_ERR_STATE otherwise); needs
 * nlam * n_src <= max_lambda_per_call * (n_src + n_det). Synchronises the stream. */
int hydot_solve_adjoint(hydot_ctx* ctx, int lam0, int nlam, const void* y, void* psi, hydot_stats* st);

/* g += J^T y for the slice from the source fields and the adjoint fields of y:
 *     g[c*N + x] += -h^3 sum_lambda eps_c(lambda) sum_s phi_s(x; lambda) psi_s(x; lambda).
 * phi_src [nlam][n_src][N], psi [nlam][n_src][N] (hydot_solve_adjoint), g [n_chrom*N] (accumulated).
 * Equals hydot_born_apply_T without the detector fields. Continuous wave only. Asynchronous. */
int hydot_born_apply_T_adjoint(hydot_ctx* ctx, const void* phi_src, const void* psi, int lam0, int nlam, void* g);

/* y = J x for one wavelength slice in FP32 without allocating device memory and without a
 * context. The paper has no counterpart: this exists for callers that cannot allocate device
 * memory themselves (code running where cudaMalloc is not allowed, or whose allocator is owned
 * by someone else). The computation is hydot_born_apply's; its per-block partial sums and the
 * slice's extinction coefficients are kept in a 16 MiB file-scope device array that every GPU
 * holds from the library's load until the process exits.
 *   N, n_src, n_det, n_chrom, nlam: sizes (>= 1, n_chrom <= 16); h_mm: cell side.
 *   eps: HOST [nlam][n_chrom] extinction coefficients of the slice's wavelengths.
 *   phi_src [nlam][n_src][N], phi_det [nlam][n_det][N], x [n_chrom*N], y [n_src*n_det*nlam]:
 *   DEVICE float arrays owned by the caller, layouts as for hydot_born_apply.
 *   stream: a cudaStream_t (NULL = legacy default stream); the call is asynchronous on it.
 * Limits: nlam*n_chrom <= 8192 and nlam*ceil(n_src/32)*ceil(n_det/32)*ceil(N/1024) <= 4096
 * (16 MiB of partial sums); larger sizes return HYDOT_ERR_ARG with a message from
 * hydot_last_error(NULL). The first call on a device, with that device current, looks up the
 * array's device address (cudaGetSymbolAddress) once; make that first call before any stream
 * capture. eps is copied to the device by cudaMemcpyAsync on stream: from pageable memory the
 * call returns once eps has been read, from pinned memory eps must stay valid and unchanged until
 * the stream has run the copy. All calls share the array, which keeps the last call's contents
 * (nothing in it needs to start at zero): calls that overlap on the GPU, on any streams of one
 * device, race. Devices with an index of 64 or more are rejected (HYDOT_ERR_CUDA). */
int hydot_born_apply_noalloc(long long N, int n_src, int n_det, int n_chrom, int nlam, double h_mm,
                             const double* eps, const float* phi_src, const float* phi_det, const float* x,
                             float* y, void* stream);

/* Kernels whose time the instrumentation below accumulates. */
typedef enum {
  HYDOT_KERNEL_DIR = 0,        /* inner PCG pass 1: p = D^-1 r + beta p, gamma = p^T A p */
  HYDOT_KERNEL_UPDATE = 1,     /* inner PCG pass 2: x += alpha p, r -= alpha A p, rho */
  HYDOT_KERNEL_RESIDUAL = 2,   /* residual of the refinement iterate (double-float on the mixed
                                * paths, FP64 on the FP64 paths) and its test, once per cycle */
  HYDOT_KERNEL_BORN_ROWS = 3,  /* Born-row assembly */
  HYDOT_KERNEL_APPLY = 4,      /* J x (partial sums) */
  HYDOT_KERNEL_APPLY_T = 5,    /* J^T y (partial sums) */
  HYDOT_KERNEL_SKETCH_RANGE = 6,   /* tensor-core Y = J Omega (work counted in flops) */
  HYDOT_KERNEL_SKETCH_PROJECT = 7, /* tensor-core B^T += J^T Q (work counted in flops) */
  HYDOT_KERNEL_ITER = 8,       /* one inner Krylov iteration of the slice's active fields, all its
                                * passes together; timed per group of 8 iterations (one CUDA-graph
                                * replay or 8 direct iterations), so "launches" counts iterations */
  HYDOT_KERNEL_SWEEP = 9,      /* single-sweep inner CG iteration (real FP32 fields): p, s = A p,
                                * x, r, u = D^-1 r, A u and both inner products in one pass */
  HYDOT_KERNEL_PRIME = 10,     /* once per refinement cycle before the single-sweep iterations:
                                * the first inner products from r_0 (reads r) */
  HYDOT_KERNEL_COUNT = 11
} hydot_kernel;

/* Instrumentation: on != 0 makes later calls record CUDA events around each launch of the
 * kernels above (on the context's stream) and count the algorithmic bytes each launch moves
 * (the bytes the operation must read and write once: 12 B per cell and active field for
 * HYDOT_KERNEL_DIR, 20 B for HYDOT_KERNEL_UPDATE in FP32, 24 B for HYDOT_KERNEL_SWEEP, 4 B for
 * HYDOT_KERNEL_PRIME, 12 B for HYDOT_KERNEL_RESIDUAL, the rows
 * written for HYDOT_KERNEL_BORN_ROWS, the fields read for the products, and for HYDOT_KERNEL_ITER
 * 6 N w per active field and iteration: the Krylov vectors x, r and p read and written once, the
 * least any CG iteration moves). Inner iterations replayed from a CUDA graph are timed as whole
 * groups (HYDOT_KERNEL_ITER only); the per-pass kinds are timed when the passes are launched
 * directly. Resets the totals. */
int hydot_set_kernel_timing(hydot_ctx* ctx, int on);

/* Totals since the last hydot_set_kernel_timing: summed device time in ms, launches, and
 * algorithmic bytes of `kernel` (a hydot_kernel). Synchronises the context's stream. Any output
 * pointer may be NULL. */
int hydot_kernel_stats(hydot_ctx* ctx, int kernel, double* ms, long long* launches, double* bytes);

/* Iteration and launch form of the inner solves (HYDOT_MIXED, real fields, nx % 4 == 0). An inner
 * CG iteration is either two passes over memory (the default) or one sweep (the Chronopoulos-Gear
 * recurrences: both inner products of an iteration from one pass; the environment variable
 * HYDOT_SINGLE_SWEEP=1 at hydot_setup selects it). With single sweeps a refinement
 * cycle's iterations run either launched (groups of 8 replayed from a CUDA graph, the host polling
 * one word per group) or as one persistent cooperative launch: co-resident blocks iterate over
 * (field, column) work items with a grid-wide barrier after each iteration and stop on the device
 * when no field is still iterating (every barrier wait is bounded: one that runs out ends the call
 * with HYDOT_ERR_TIMEOUT). Both do the same arithmetic (the same bits). While *mode is -1 the solver
 * times whole cycles in each, per active cell-iteration, and then keeps the faster (1: persistent,
 * 0: launched; always 0 with two-pass iterations); HYDOT_PERSISTENT=0 or 1 at hydot_setup fixes
 * the choice (1 also selects single sweeps). ns_launched / ns_persistent: measured ns per cell-iteration (0 if not timed). Any
 * output pointer may be NULL. */
int hydot_get_launch_mode(const hydot_ctx* ctx, int* mode, double* ns_launched, double* ns_persistent);

/* Inner iterations of the rolling passes replay a CUDA graph per group of 8 iterations when on
 * != 0 (the default, unless the environment variable HYDOT_NO_GRAPHS was set at hydot_setup);
 * with on == 0 every pass is launched directly, which lets the instrumentation time each pass on
 * its own. Results are bitwise identical either way. */
int hydot_set_graphs(hydot_ctx* ctx, int on);

/* Number of kernels this context has launched since hydot_setup (instrumentation: lets a
 * caller count the library's launches inside a timed region). */
long long hydot_kernel_launches(const hydot_ctx* ctx);

/* Autotuning of the inner passes (HYDOT_MIXED, real fields, nx % 4 == 0). The two passes stream
 * TMA slabs of `planes` z-planes through `buffers` shared-memory buffers; the variants below give
 * bitwise identical results and differ in data in flight and blocks per SM. While *variant is
 * -1 the solver times groups of inner iterations with each variant in turn (within the first
 * solves of the context) and then keeps the fastest per cell-iteration; the environment variable
 * HYDOT_ROLL_VARIANT=<index> fixes the choice at setup. */
#define HYDOT_ROLL_VARIANTS 4

/* The chosen variant (-1 while tuning, or when the context does not use these passes) and, for
 * each variant i < HYDOT_ROLL_VARIANTS, its planes, buffers and measured ns per cell-iteration
 * (0 if not timed yet). Any output pointer may be NULL; arrays hold HYDOT_ROLL_VARIANTS entries. */
int hydot_get_tuning(const hydot_ctx* ctx, int* variant, int* planes, int* buffers, double* ns_per_cell);

/* Absorption perturbation for the nonlinear forward model (eqn:lippschwin without the Born
 * approximation): later hydot_solve_fields calls solve (A_lambda + h^3 diag(dmu_a)) phi = e with
 * dmu_a(x; lambda) = sum_c eps_c(lambda) dc[c][x], the diffusion coefficient staying the
 * background's. dc: HOST double [n_chrom][N] concentration changes (mM), copied; NULL removes the
 * perturbation. Perturbed solves run the generic (non-TMA) inner kernels; results stay FP32 fields
 * with FP64 refinement (or FP64 throughout), to the context's tolerances. Synchronous. */
int hydot_set_absorption(hydot_ctx* ctx, const double* dc);

/* Shift-invariant initial guesses (Section 3, 3.2; the base operator at the mean shift, Section
 * 6.1). Builds, for every source and detector field, an orthonormal basis V (m vectors, FP32) of the
 * Krylov space K_m(Ahat_0, e_cell) of the base operator Ahat_0 = Lg + mean(sigma) I + sum_f
 * mean(bhat_f) B_f (the scaled operator of the coefficient table, averaged over the wavelengths),
 * with Lanczos and full reorthogonalisation, together with the Lanczos tridiagonal and the
 * boundary blocks V^T B_f V. From then on hydot_solve_fields starts every field of every wavelength
 * j from the Galerkin projection x_j = V (V^T Ahat_j V)^-1 V^T e_cell, formed from those small
 * matrices without products with Ahat_j, instead of from zero; the solves still converge to the
 * context's tolerances (the guess changes where the iteration starts, not where it stops).
 * m: 1..64 (capped at N), or 0 to remove the bases. Device memory: (n_src+n_det)*m*N*4 bytes,
 * plus small tables. Continuous-wave contexts only (HYDOT_ERR_STATE for omega != 0), and not
 * together with deflation_k > 0 (HYDOT_ERR_STATE); m outside 0..64: HYDOT_ERR_ARG. With an
 * absorption perturbation set (hydot_set_absorption) the guess ignores it. Synchronous. */
int hydot_set_shift_guess(hydot_ctx* ctx, int m);

/* The initial guesses themselves, in field units phi = x / (D h), for the wavelengths lam0 ..
 * lam0+nlam-1: phi_src [nlam][n_src][N], phi_det [nlam][n_det][N], DEVICE, element type as for
 * hydot_solve_fields (FP32 for HYDOT_MIXED, FP64 for HYDOT_FP64). nlam*(n_src+n_det) must not exceed
 * the context's simultaneous fields (max_lambda_per_call*(n_src+n_det)). HYDOT_ERR_STATE when no
 * bases are built. Asynchronous on the context's stream. */
int hydot_shift_guess_fields(hydot_ctx* ctx, int lam0, int nlam, void* phi_src, void* phi_det);

/* Shape reconstruction with parametric level sets (Section 5: eqn:pals, eqn:minimization,
 * Algorithm alg:opt) on a compressed Born operator J ~ U diag(S) V^T (U with orthonormal columns,
 * e.g. from hydot_sketch_factor or the recursive compression).
 * Shape: mu(r) = H_eps(phi(r) - tau), phi(r) = sum_k alpha_k psi(beta_k |r - chi_k|_nu), |v|_nu =
 * sqrt(|v|^2 + nu^2), psi(t) = (1 - t)_+^4 (4t + 1) (Wendland's compactly supported C2 function),
 * H_eps(t) = 1/2 + arctan(pi t / eps) / pi; the points r are the voxel centres ((i + 1/2) h, ...)
 * in mm. Parameters p = [alpha (n), beta (n), chi_x (n), chi_y (n), chi_z (n)], n = n_basis in 1..8,
 * host FP64 [5 n]. Measurements y = sum_c c_c E_c H mu: J applied to the chromophore-major vector
 * (c_0 mu, c_1 mu, ...). Errors: HYDOT_ERR_ARG for a bad size, pointer or model constant. */
typedef struct {
  double tau, eps, nu;   /* level, width of the smoothed Heaviside, smoothing of |r| (mm) */
  double gamma;          /* discrepancy factor: stop when |y - D(p) c| <= gamma * noise_norm */
  double noise_norm;     /* |eta|, the norm of the measurement noise (0: run to the iteration limits) */
  double lm_nu0;         /* initial Levenberg-Marquardt damping, relative to max diag(J^T J) */
  int max_outer;         /* alternations between the c step and the p steps */
  int max_inner;         /* Levenberg-Marquardt trial steps per alternation */
  int fix_c;             /* 1: c is known and kept (shape only), 0: c is estimated too */
} hydot_pals_options;

typedef struct {
  int evaluations;       /* shape + projection evaluations */
  int accepted;          /* accepted Levenberg-Marquardt steps */
  double residual0;      /* |y - D(p0) c0| */
  double residual;       /* |y - D(p) c| at the returned p, c */
} hydot_pals_result;

/* Algorithm alg:opt: alternate the linear least-squares step for c (skipped with fix_c) and
 * Levenberg-Marquardt steps (J^T J + nu I) dp = -J^T eps on p (nu divided by 3 after an accepted
 * step, multiplied by 4 after a rejected one), until the residual meets the discrepancy principle or
 * the iteration limits, or an alternation stops reducing it. All in the rank coordinates:
 * |y - D c|^2 = (|y|^2 - |U^T y|^2) + |U^T y - S M c|^2 with M[:, c] = V_c^T mu(p), and the
 * Jacobian -S sum_c c_c V_c^T dmu/dp; mu and dmu/dp come from a kernel over the voxels, the products
 * from tall-skinny FP32 kernels with FP64 sums, the small systems are solved on the host (FP64).
 * U: DEVICE FP32 [rows][rank] (row stride ldU); S: HOST FP64 [rank]; V: DEVICE FP32
 * [n_chrom * N][rank] (row stride ldV), rows chromophore-major; y: DEVICE FP32 [rows];
 * p: HOST [5 n_basis] initial guess in, result out; c: HOST [n_chrom] initial (or known)
 * concentrations in, result out; res: may be NULL. Synchronous. */
int hydot_pals_reconstruct(hydot_ctx* ctx, const float* U, long long ldU, long long rows, const double* S,
                           const float* V, long long ldV, int rank, const float* y, int n_basis, double* p,
                           double* c, const hydot_pals_options* opt, hydot_pals_result* res);

/* mu(r) at every voxel for the parameters p: mu DEVICE FP32 [N]. Synchronous. */
int hydot_pals_shape(hydot_ctx* ctx, int n_basis, const double* p, double tau, double eps, double nu, float* mu);

/* One evaluation of the reconstruction: A[c][k][q] = sum_x V[(c, x)][k] F[x][q] with
 * F = [mu, dmu/dp] (q < 1 + 5 n_basis), for the tests and for inspection. V as above; A HOST FP64
 * [n_chrom][rank][1 + 5 n_basis]. Synchronous. */
int hydot_pals_project(hydot_ctx* ctx, const float* V, long long ldV, int rank, int n_basis, const double* p,
                       double tau, double eps, double nu, double* A);

/* The metrics of Section 6.2 between a true shape mu and a recovered one (DEVICE FP32 [N]):
 * relative L2 error |mu - mu_hat| / |mu| and the Dice coefficient 2 |A and B| / (|A| + |B|) of the
 * voxel sets where each exceeds `level` (1 when both are empty). Outputs may be NULL. Synchronous. */
int hydot_shape_compare(hydot_ctx* ctx, const float* mu, const float* mu_hat, double level, double* rel_l2,
                        double* dice);

/* Failure-path self-test (no counterpart in the paper), with `polls` polls (1..2^22) per wait
 * instead of the kernels' own limits: (1) one thread waits on a shared-memory mbarrier that nothing
 * arrives at, through the bounded poll loop the pipelined kernels use for their TMA and
 * tensor-core waits; (2) in a cooperative launch of two blocks only one arrives at the grid barrier
 * of the persistent inner solve, so its bounded wait runs out. Each raises the device error flag
 * and returns. The call returns HYDOT_ERR_TIMEOUT when both waits gave up (HYDOT_ERR_STATE if one
 * did not), and the context stays usable (the flag is cleared). Synchronises the stream. */
int hydot_wait_selftest(hydot_ctx* ctx, int polls);

/* Randomised sketch of J, pass 1 (Appendix A.1, alg:randsvd: Y = A Omega with Gaussian Omega):
 *   Y[r][k] = sum_(c,x) J[r,(c,x)] Omega[(c,x),k]
 * for the rows r of the sources src0 .. src0+nsrc-1 (the row block H_i of Section 4.1 for a block of
 * sources) and the wavelengths of the slice [lam0, lam0+nlam); row r = ((s - src0)*n_det + d)*nlam
 * + (lambda - lam0). phi_src/phi_det: the slice's fields of all sources/detectors.
 * omega_t: DEVICE BF16 (raw 16-bit) [n_chrom][ncols][N], Omega transposed per chromophore.
 * Y: DEVICE float [nsrc*n_det*nlam][ldY], 16-byte aligned, ldY >= 224 and ldY % 4 == 0; columns
 * >= ncols are written as 0. Computed on the tensor cores (BF16 operands, FP32 accumulation).
 * Needs HYDOT_MIXED, omega == 0, N divisible by 8 and ncols <= 224. Synchronises the stream;
 * HYDOT_ERR_TIMEOUT if a bounded device wait gave up. */
int hydot_sketch_range(hydot_ctx* ctx, const void* phi_src, const void* phi_det, int lam0, int nlam, int src0,
                       int nsrc, const void* omega_t, int ncols, float* Y, long long ldY);

/* Randomised sketch of J, pass 2 (B = Q^T A): Bt[(c,x)][k] += sum_r J[r,(c,x)] Q[r][k] over the rows
 * r of the sources src0 .. src0+nsrc-1 and the slice, so calls over consecutive slices merge the
 * row blocks into B^T (Section 4.2). Q: DEVICE float [nsrc*n_det*nlam][ldQ] (those rows of the
 * orthonormal range basis, ordered as in hydot_sketch_range), Bt: DEVICE float [n_chrom*N][ldB],
 * ldB >= 224, accumulated. Tensor cores, same requirements as hydot_sketch_range. Synchronises the
 * stream. */
int hydot_sketch_project(hydot_ctx* ctx, const void* phi_src, const void* phi_det, int lam0, int nlam, int src0,
                         int nsrc, const float* Q, int ncols, long long ldQ, float* Bt, long long ldB);

/* Orthonormal basis of range(Y) in place (the basis step of alg:randsvd): two rounds of
 * Y <- Y V diag(lambda^-1/2) from the Gram Y^T Y = V diag(lambda) V^T (FP32 products, FP64 sums across
 * 64-row blocks, eigen-decomposition in FP64 on the host). Directions whose
 * singular value is below 1e-6 of the largest become zero columns; *rank_out (may be NULL) gets the
 * number kept, *smax_out (may be NULL) the largest singular value of the input Y. The columns come
 * out in descending order of singular value. Y: DEVICE float [rows][ldY], first ncols (<= 224)
 * columns. Synchronous. */
int hydot_sketch_orthonormalize(hydot_ctx* ctx, float* Y, long long rows, int ncols, long long ldY, int* rank_out,
                                double* smax_out);

/* Adaptive rank (the error estimator of alg:randsvd): Q DEVICE float [rows][ldQ], nq <= 224
 * orthonormal columns in descending singular-value order (hydot_sketch_orthonormalize), Y2 DEVICE
 * float [rows][ldY2] = A Omega_2 for k (1..32) further Gaussian columns. *rank receives the smallest
 * r (at least 1) with || Y2 - Q_r Q_r^T Y2 ||_2 <= tol * s1, where Q_r are the first r columns and s1
 * is the caller's scale (the largest singular value of A Omega_1); nq when none qualifies.
 * *estimate (may be NULL) receives || Y2 - Q_r Q_r^T Y2 ||_2 / s1 for that r. Products in FP32, sums across
 * 64-row blocks in FP64.
 * Synchronous. */
int hydot_sketch_rank(hydot_ctx* ctx, const float* Q, long long ldQ, long long rows, int nq, const float* Y2,
                      long long ldY2, int k, double s1, double tol, int* rank, double* estimate);

/* Agglomeration of the low-rank factors of two stacked row blocks (Section 4.3, Algorithm
 * alg:recursive): [H1; H2] ~ [U1 diag(S1) V1^T; U2 diag(S2) V2^T] is recompressed to U diag(S) V^T
 * with U = [U1 E1; U2 E2] (rows m1 + m2), keeping the singular values of [diag(S1) V1^T; diag(S2)
 * V2^T] above tol times the largest (at most max_rank of them). Inputs: U1 [m1][ldU1], V1 [n][ldV1]
 * (r1 columns), likewise block 2, all DEVICE float; S1, S2 HOST double. Outputs: U DEVICE float
 * [m1+m2][ldU], V DEVICE float [n][ldV] (not aliasing the inputs), S HOST double [r1+r2] (first
 * *rank_out entries set), *rank_out the merged rank. The Gram of the stacked factors is formed from
 * tall-skinny products (FP32 products, FP64 block sums) and diagonalised in FP64 on the host. Synchronous. */
int hydot_sketch_merge(hydot_ctx* ctx, const float* U1, long long ldU1, long long m1, const double* S1, const float* V1,
                       long long ldV1, int r1, const float* U2, long long ldU2, long long m2, const double* S2,
                       const float* V2, long long ldV2, int r2, long long n, double tol, int max_rank, float* U,
                       long long ldU, double* S, float* V, long long ldV, int* rank_out);

/* Rank-`rank` factors J ~ U diag(S) V^T from Q (the orthonormal range basis, rows x ncols) and
 * Bt = (Q^T J)^T (nb = n_chrom*N rows): the Gram of Bt (FP32 products, FP64 block sums) gives U_B and S
 * (descending), then
 * V = Bt U_B diag(1/S) and U = Q U_B (Section 4.4's final recompression). U: DEVICE float
 * [rows][ldU], V: DEVICE float [nb][ldV], S: HOST double [rank]. Synchronous. */
int hydot_sketch_factor(hydot_ctx* ctx, const float* Q, long long rows, long long ldQ, const float* Bt, long long nb,
                        long long ldB, int ncols, int rank, float* U, long long ldU, double* S, float* V,
                        long long ldV);

/* Geometric bisection tree of the sources (Section 4.1, Algorithm alg:geom), which orders the row
 * blocks for the recursive compression: the box [x_lo, x_hi] x [y_lo, y_hi] is split across its
 * longer side (the first on a tie) at the midpoint, the positions at or below the split coordinate
 * going to the first side, recursively, until a cell holds at most leaf_max positions (or below 64
 * levels). A side without positions is dropped, and a split that leaves one side empty makes no
 * node. xy: HOST double [n][2]. Outputs, HOST: order int [n], the position indices leaf by leaf,
 * depth first, first side first; nodes int [2n][4] = (lo, hi, first child, second child), a node
 * covering order[lo .. hi-1], children -1 for a leaf; *n_nodes the number of nodes written (at most
 * 2n - 1) and *root the index of the root. Host arithmetic only (no GPU, no context); n >= 1 and
 * leaf_max >= 1, else HYDOT_ERR_ARG with the message in hydot_last_error(NULL). */
int hydot_source_tree(const double* xy, int n, double x_lo, double y_lo, double x_hi, double y_hi, int leaf_max,
                      int* order, int* nodes, int* n_nodes, int* root);

/* Last error message of ctx; with ctx NULL, that of the calling thread's last failed call that
 * has no context (hydot_setup, the context-free Born call). */
const char* hydot_last_error(const hydot_ctx* ctx);

/* Frees everything hydot_setup allocated. NULL is ignored. */
void hydot_destroy(hydot_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* HYDOT_H */
