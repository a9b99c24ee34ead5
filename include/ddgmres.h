/*
 * ddgmres.h -- C ABI of the data-driven GMRES library for 2D FDFD solves (sm_103a).
 *
 * The library solves A f = b, where A is the finite-difference frequency-domain
 * operator of Maxwell's equations for the 2D TM polarisation (Ez), and can
 * augment GMRES with a predicted subspace V (data-driven GMRES):
 *   Eq. 1   [curl curl - omega^2 eps / c^2] E = -i omega mu0 J, discretised on a
 *           periodic Yee grid with stretched-coordinate PML (Sec. II).
 *   Eq. 2   GMRES: f_i = argmin over K_i(A, b) of ||A f - b||.
 *   Eq. 3-4 data-driven GMRES: f_i = argmin over V + K_i(A~, b~),
 *           A~ = P_perp(A V) A, b~ = P_perp(A V) b; update rule of the supplement
 *           (Eqs. S1-S7: A V = C R, Arnoldi on A~, block least squares).
 *
 * Conventions shared by every call
 *  - Complex vectors are interleaved (re, im) pairs: a complex128 vector of
 *    length D is `double[2*D]`, a complex64 vector is `float[2*D]`.
 *  - Grid vectors are row-major [ny][nx]: cell (i, j) at index j*nx + i.
 *  - Pointer arguments are DEVICE pointers unless marked (host).  The caller
 *    owns every buffer it passes; the library never frees them.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Calls are stream-ordered; calls that return ddg_info fill it on return
 *    (they synchronise `stream`).
 *  - Handles (ddg_context, ddg_op) belong to the device that was current when
 *    they were created; use one ddg_context per host thread / stream.
 *  - No C++ exception crosses this boundary.  On error the call returns a
 *    status != DDG_OK and ddg_last_error() describes it.
 */
#ifndef DDGMRES_H
#define DDGMRES_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DDG_OK = 0,
    DDG_EINVAL = 1,      /* bad argument: sizes, tolerances, non-finite or non-positive eps */
    DDG_ENOMEM = 2,      /* device allocation failed */
    DDG_ECUDA = 3,       /* a CUDA runtime call failed (message in ddg_last_error) */
    DDG_ENOCONV = 4,     /* iteration cap reached before the tolerance; x holds the best iterate */
    DDG_EBREAKDOWN = 5,  /* reserved: unrecoverable Arnoldi breakdown */
    DDG_ETIMEOUT = 6,    /* a bounded device wait gave up (a bulk copy into shared memory did not
                            complete within the wait limit, 1 s by default); the solve's outputs
                            are not valid */
    DDG_ESINGULAR = 7    /* a small dense factorisation failed */
} ddg_status;

/* Precision of the Krylov loop. */
typedef enum {
    DDG_C128 = 0,        /* everything in complex128 / FP64 */
    DDG_C64_REFINE = 1,  /* Arnoldi vectors and matvecs in complex64 (FP32 sums inside a
                            block, FP64 across blocks); true residual r = b - A x, Givens
                            rotations, Hessenberg least squares and the update of x in FP64.
                            Every restart recomputes r in FP64 (iterative refinement). */
    DDG_C64_ONLY = 2     /* the Krylov loop as DDG_C64_REFINE, and the residual r = b - A x of
                            every restart also in complex64 (from the operator's FP32 copy):
                            no FP64 refinement; a cycle runs until its estimate reaches
                            tol * ||b||.  For tolerances of about 1e-5 and above (FP32
                            round-off bounds the attainable residual); the Givens rotations,
                            the small least-squares problem and the x buffer stay FP64.
                            Not accepted by gmres_solve_noalloc. */
} ddg_precision;

/* Problem description (host struct).  Units: metres. */
typedef struct {
    int nx, ny;          /* cells along x (fastest index) and y */
    double dx;           /* cell size h (square cells) */
    double wavelength;   /* vacuum wavelength; k0 = 2 pi / wavelength */
    int npml_x, npml_y;  /* PML thickness in cells (0 = none) on both ends of x / y */
    double pml_order;    /* polynomial grading order m of the PML conductivity */
    double pml_R;        /* target normal-incidence reflection R of the PML */
} ddg_grid;

/* Per-solve result (host struct). */
typedef struct {
    int iters;                       /* Arnoldi steps (matvecs in the Krylov loop) */
    int cycles;                      /* restart cycles (each starts from an FP64 residual) */
    int converged;                   /* 1 if true_rel_residual <= tol */
    int fallback_used;               /* augmented solve ran as plain GMRES (V rejected) */
    int breakdown;                   /* an Arnoldi step hit an invariant subspace */
    double true_rel_residual;        /* ||b - A x|| / ||b||, FP64, recomputed at the end */
    double first_step_rel_residual;  /* augmented: ||P_perp b|| / ||b|| = min over V (Eq. 6) */
} ddg_info;

typedef struct ddg_context ddg_context;   /* workspace + tuning, one per stream */
typedef struct ddg_op ddg_op;             /* the operator A(eps, omega) of one problem */

/* Status text; never NULL. */
const char* ddg_status_str(ddg_status s);
/* Last error message of the calling thread; never NULL. */
const char* ddg_last_error(void);
/* Library version as 10000*major + 100*minor + patch. */
int ddg_version(void);

/* Kernel classes of the solver, for ddg_context_profile_read. */
typedef enum {
    DDG_K_STEP = 0,       /* q_j = w / h, w = A q_j (stencil) */
    DDG_K_DOTS = 1,       /* Gram-Schmidt projections [C Q]^H w */
    DDG_K_UPDATE = 2,     /* Gram-Schmidt updates w -= [C Q] h (+ norm, Givens) */
    DDG_K_RESIDUAL = 3,   /* cycle start: r = b - A x (FP64), augmented projection */
    DDG_K_CYCLE_END = 4,  /* back substitution and x += V z + Q y */
    DDG_K_SETUP = 5,      /* augmentation set-up (A V, Cholesky QR twice), PCA fit */
    DDG_K_NCLASSES = 6
} ddg_kernel_class;

/* Context: owns the device workspace (grown on demand, reused across calls). */
ddg_status ddg_context_create(ddg_context** ctx);
ddg_status ddg_context_destroy(ddg_context* ctx);
/* Bytes of device workspace the context currently holds. */
long long ddg_context_workspace_bytes(const ddg_context* ctx);
/* Kernels launched through this context since it was created. */
long long ddg_context_launches(const ddg_context* ctx);
/* Profiling: with enable != 0 every later launch is bracketed by CUDA events on
   its stream and each kernel adds its algorithmic bytes (the bytes the method
   must move: every vector element read or written once) to a device counter.
   Enabling (or disabling) clears the accumulators. */
ddg_status ddg_context_profile_enable(ddg_context* ctx, int enable);
/* Accumulated device time (ms), algorithmic bytes and launch count of one
   ddg_kernel_class since profiling was enabled.  Synchronises the device. */
ddg_status ddg_context_profile_read(ddg_context* ctx, int cls, double* ms, double* bytes,
                                    long long* launches);
/* Gram-Schmidt scheme of the Arnoldi step (Eq. S2 and its reorthogonalisation). */
typedef enum {
    DDG_ORTH_CGS2 = 0,   /* classical Gram-Schmidt applied twice per step: 4 passes over the
                            basis, 2 reductions per step */
    DDG_ORTH_DCGS2 = 1   /* default: the second pass of step i-1 is merged into the single
                            reduction of step i and the Hessenberg column corrected
                            algebraically (delayed reorthogonalisation, Bielich et al.,
                            Parallel Computing 112, 2022): 2 passes over the basis per step */
} ddg_orthogonalization;
ddg_status ddg_context_set_orthogonalization(ddg_context* ctx, int scheme);
/* Solve loop of the delayed scheme (no paper counterpart): with `enable` (the
   default) a batched solve's restart cycles, after its set-up, run as ONE
   CUDA graph launch: a device-side WHILE over cycles (cycle-start residual,
   then an IF for the cycle's Arnoldi steps -- the first step and a nested
   WHILE over [8 x (reduction, sweep), step advance] that ends when every
   solve has left its cycle or the restart length is reached -- and an IF for
   the cycle end), which ends when every solve has converged or stopped, a
   bounded wait gave up, or maxit + 2 cycles have run; the host reads the
   results once.  Otherwise the host launches every kernel, reads the counts
   at every cycle start and polls the device every 8 steps.  Both give the
   same results (same kernels, same order).  Per-kernel profiling
   (ddg_context_profile_enable) uses the host-driven loop. */
ddg_status ddg_context_set_graphs(ddg_context* ctx, int enable);
/* Storage of the Krylov basis [C | Q] in complex64 solves (no paper
   counterpart; compressed-basis GMRES, Aliaga et al., Int. J. High Perform.
   Comput. Appl. 36, 2022): with `half` the basis vectors are stored in IEEE
   half (4 bytes per complex value) and read back into FP32 for every product
   and sum; everything else is unchanged (FP32 arithmetic, FP64 true residual
   judging convergence, so the tolerance is met as before).  It halves the
   bytes of the Gram-Schmidt passes, which dominate the solve; the Arnoldi
   relation then holds to half precision (~5e-4), which can add Krylov steps
   when a restart cycle reduces the residual a lot.  Default 0 (the basis in
   FP32).  Ignored for DDG_C128. */
ddg_status ddg_context_set_basis_storage(ddg_context* ctx, int half);
/* Data-free preconditioner, the baseline the data-driven subspace is compared
   with (Sec. III, the benchmark against data-free preconditioners, and the
   supplement's section on them): kind 1 = Jacobi, M = D(A), the diagonal of A
   (the stencil's centre coefficient).  The supplement applies it on the left
   (D(A)^-1 A); here it is applied on the right: GMRES runs on A M^-1, which is
   similar to D(A)^-1 A (same spectrum), and x += M^-1 Q y, so the residual
   minimised, the stopping rule and the augmentation stay those of A f = b.
   kind 0 (default) = none.  For the indefinite FDFD operator with PML Jacobi
   slows convergence.  Returns DDG_EINVAL for any other kind. */
ddg_status ddg_context_set_preconditioner(ddg_context* ctx, int kind);
/* Augmented solves: when the V-only relative residual ||b~|| / ||b|| of the first
   cycle (Eq. 6's minimum over V) exceeds `threshold`, the predicted subspace is
   judged to have failed: its least-squares step is kept (x += V R^-1 C^H b) and
   the solve continues as plain GMRES (info.fallback_used = 1).  Default 0.5;
   a threshold >= 1 never falls back. */
ddg_status ddg_context_set_fallback(ddg_context* ctx, double threshold);
/* Restarted augmented solves (the paper does not restart): the first `cycles`
   restart cycles run data-driven GMRES with V (Eqs. 3-4, S1-S7); later cycles
   continue as plain GMRES from the current iterate.  Default 1 (the paper's
   method for the first cycle); 0 keeps only the least-squares step over V;
   a value >= maxit keeps V in every cycle. */
ddg_status ddg_context_set_augmented_cycles(ddg_context* ctx, int cycles);
/* Restart policy of augmented solves, in full (no paper counterpart; the
   paper does not restart): the first `cycles` restart cycles use all k
   columns of V; later cycles keep the leading `keep` columns (A V = C R is
   triangular in the column order, so their factors are the leading columns of
   C and the leading block of R: nothing is recomputed) and keep = 0 continues
   as plain GMRES.  With wavelength = 0 this sets the default for every solve
   (ddg_context_set_augmented_cycles sets `cycles` alone); with a wavelength in
   metres (> 0, matched to 1e-9 relative) the policy of the solves whose
   operator has that wavelength, which overrides the default (one set of
   problems, e.g. one device at two wavelengths, may need two policies).
   Order V so that the vectors worth keeping come first.
   cycles >= 0, 0 <= keep <= 32, else DDG_EINVAL. */
ddg_status ddg_context_set_augmented_policy(ddg_context* ctx, double wavelength, int cycles, int keep);
/* Limit of the bounded device waits of the solver (no paper counterpart): an
   Arnoldi kernel waits at most `ns` nanoseconds for a bulk copy of basis
   columns into shared memory (default 1e9, 1 s).  A wait that runs out stops
   that block's reduction; the block still waits for the copies it issued, at
   the 1 s default, before it exits, and the call returns DDG_ETIMEOUT (the
   solve's outputs are not valid; the context stays usable).  A limit of 0
   tests each copy once without waiting, so that waits run out on purpose
   (which exercises that path).
   0 <= ns <= 1e10, else DDG_EINVAL. */
ddg_status ddg_context_set_wait_limit(ddg_context* ctx, long long ns);
/* Largest device workspace the context may hold, in bytes (0, the default:
   no limit).  A call that needs more returns DDG_ENOMEM without allocating
   (and a workspace above a new limit is freed at once).  Serves callers with
   a memory budget, and makes the allocation-failure path testable. */
ddg_status ddg_context_set_workspace_limit(ddg_context* ctx, long long bytes);
/* Inner-cycle relative tolerance for DDG_C64_REFINE (a cycle ends once its
   least-squares residual falls below eta times the cycle's starting residual).
   Default 1e-5.  Must be in (0, 1). */
ddg_status ddg_context_set_inner_tol(ddg_context* ctx, double eta);

/*
 * fdfd_operator -- set up A(eps, omega) of Eq. 1 (Sec. II) on the Yee grid:
 *   (A x)_{i,j} = -[ (1/sxb_i)((x_{i+1,j}-x_{i,j})/sxf_i - (x_{i,j}-x_{i-1,j})/sxf_{i-1})
 *                  + (1/syb_j)((x_{i,j+1}-x_{i,j})/syf_j - (x_{i,j}-x_{i,j-1})/syf_{j-1}) ]
 *                - (k0 h)^2 eps_{i,j} x_{i,j},          indices periodic (mod nx, ny),
 * i.e. Eq. 1 times h^2, with stretch s(p) = 1 - i smax (d(p)/L)^m at integer
 * nodes (sxb) and half nodes p = i + 1/2 (sxf), d(p) the depth into the PML in
 * cells, smax = -(m+1) ln(R) / (2 k0 h L).
 *   g    (host)  grid description; nx, ny >= 3; nx*ny < 2^31; 0 <= npml <= n/2; R in (0,1).
 *   eps  device, ny*nx doubles, row-major; every value finite and > 0, else DDG_EINVAL.
 *   A    (host)  receives the new handle; the operator keeps its own copy of eps.
 * Synchronises `stream` (the eps check reads back one flag).
 */
ddg_status fdfd_operator(const ddg_grid* g, const double* eps, ddg_op** A, void* stream);
ddg_status fdfd_operator_destroy(ddg_op* A);
/* Number of unknowns D = nx*ny of the operator (0 for NULL). */
long long fdfd_operator_size(const ddg_op* A);

/* y = A x in complex128 (x, y: device, 2*D doubles, must not overlap). */
ddg_status fdfd_apply(const ddg_op* A, const double* x, double* y, void* stream);
/* y = A x in complex64 (coefficients rounded to FP32; x, y: 2*D floats). */
ddg_status fdfd_apply_c64(const ddg_op* A, const float* x, float* y, void* stream);

/*
 * fdfd_source -- b = -i (k0 h) J (Eq. 1 right-hand side times h^2 up to the
 * constant mu0 c): a line current on column i_src with Gaussian profile
 * J_j = exp(-(j - j_c)^2 / (2 sigma^2)) along y, zero elsewhere.
 *   b  device, 2*D doubles (written in full).  0 <= i_src < nx, sigma > 0.
 */
ddg_status fdfd_source(const ddg_op* A, int i_src, double sigma_cells, double j_c,
                       double* b, void* stream);

/*
 * gmres_solve -- restarted GMRES(restart) for A x = b (Eq. 2), classical
 * Gram-Schmidt with one reorthogonalisation (Eq. S2 applied twice), complex
 * Givens least squares in FP64.  Stops when the FP64 true relative residual
 * ||b - A x|| / ||b|| <= tol, or after maxit Arnoldi steps (DDG_ENOCONV).
 *   b     device, 2*D doubles.
 *   x     device, 2*D doubles: in = initial guess x0, out = solution.
 *   tol   in (0, 1);  restart in [1, 1024];  maxit >= 1.
 *   info  (host) may be NULL.
 */
ddg_status gmres_solve(ddg_context* ctx, const ddg_op* A, const double* b, double* x,
                       double tol, int restart, int maxit, ddg_precision prec,
                       ddg_info* info, void* stream);

/*
 * augmented_gmres_solve -- data-driven GMRES (Eqs. 3-4, supplement S1-S7):
 * A V = C R by Cholesky QR applied twice (FP64), b~ = b - C C^H b, Arnoldi on
 * A~ = (I - C C^H) A with B = C^H A Q kept, the block least-squares problem
 * decoupled into y = argmin ||H y - ||b~|| e1|| and x_V = C^H b - B y, and
 * f = V R^-1 x_V + Q y.  Restarts solve the residual equation with the same V.
 *   U     device, D x k complex128, column-major (column n at U + 2*D*n), the
 *         predicted vectors v_1..v_k; need not be orthonormal.
 *   k     1 <= k <= 32.  If A U is numerically rank deficient the solve runs as
 *         plain GMRES and info.fallback_used = 1 (status DDG_OK).
 * Other arguments as gmres_solve.
 */
ddg_status augmented_gmres_solve(ddg_context* ctx, const ddg_op* A, const double* b,
                                 const double* U, int k, double* x, double tol,
                                 int restart, int maxit, ddg_precision prec,
                                 ddg_info* info, void* stream);

/*
 * Batched forms: n independent solves (uneven grid sizes allowed) advanced
 * together, every kernel launch covering all solves still running.
 *   A, b, x, U  (host) arrays of n handles / device pointers.
 *   info        (host) array of n results, may be NULL.
 * Returns DDG_ENOCONV if any solve missed the tolerance.
 */
ddg_status gmres_solve_batched(ddg_context* ctx, int n, const ddg_op* const* A,
                               const double* const* b, double* const* x, double tol,
                               int restart, int maxit, ddg_precision prec,
                               ddg_info* info, void* stream);
ddg_status augmented_gmres_solve_batched(ddg_context* ctx, int n, const ddg_op* const* A,
                                         const double* const* b, const double* const* U,
                                         int k, double* const* x, double tol, int restart,
                                         int maxit, ddg_precision prec, ddg_info* info,
                                         void* stream);

/*
 * gmres_solve_trajectories -- Krylov subspace recycling along design
 * trajectories (Sec. I names recycling across a sequence of related solves as
 * prior art, and the supplement's update rule is that of GCROT): n_traj
 * trajectories of n_steps correlated problems each (an optimisation's
 * successive designs), solved step by step.  Step t of every trajectory runs in
 * one batched augmented solve (augmented_gmres_solve_batched) whose subspace
 * is [U (the k predicted vectors of that problem) | x_{t-1} (the same
 * trajectory's solution of step t-1)]; step 0 uses U alone, or plain GMRES when
 * U is NULL (k = 0).  Every solve starts from x = 0 (the previous solution
 * enters through the subspace: its least-squares step already contains it).
 *   A, b, x, U, info  (host) arrays of n_traj * n_steps entries,
 *                     trajectory-major (entry r * n_steps + t); a trajectory
 *                     keeps one grid size; U may be NULL (then k = 0).
 *   k                 0 <= k <= 31 predicted vectors per problem.
 *   other arguments   as augmented_gmres_solve_batched (the context's options
 *                     apply to every step).
 * The subspaces are assembled in a buffer the context keeps (n_traj (k+1) D
 * complex128).  Returns DDG_ENOCONV if any solve missed the tolerance.
 */
ddg_status gmres_solve_trajectories(ddg_context* ctx, int n_traj, int n_steps, const ddg_op* const* A,
                                    const double* const* b, const double* const* U, int k, double* const* x,
                                    double tol, int restart, int maxit, ddg_precision prec, ddg_info* info,
                                    void* stream);

/*
 * gmres_solve_queue -- a queue of n independent solves of Eq. 2 / Eqs. 3-4
 * (the paper is silent on batching; library plumbing for workloads of hundreds
 * of correlated solves on uneven grids) run as groups of
 * `width` consecutive solves, each group one batched solve
 * (augmented_gmres_solve_batched when U is not NULL, else gmres_solve_batched).
 * `nlanes` lanes work at once, lane l with context lanes[l] and stream
 * streams[l] on its own host thread; a lane takes the next group as soon as its
 * previous group has finished, so one group's slowest solves run beside the
 * next group's.  Which width and how many lanes suit a workload is found by
 * timing (the package's autotuner).  Returns when every solve has finished.
 *   lanes    (host) nlanes distinct contexts, 1 <= nlanes <= 8; their options
 *            (precision of the basis, graphs, preconditioner) apply per group.
 *   streams  (host) nlanes streams (distinct when not NULL; NULL entries = the
 *            legacy default stream), or NULL for all.
 *   width    >= 1 solves per group.
 *   A, b, U, x, info: as the batched forms (n entries; U may be NULL).
 * Returns DDG_ENOCONV if any solve missed the tolerance; on any other error
 * the lanes stop taking groups and the first error is returned (solves of
 * groups never taken keep their x and info untouched).
 */
ddg_status gmres_solve_queue(ddg_context* const* lanes, void* const* streams, int nlanes,
                             int width, int n, const ddg_op* const* A,
                             const double* const* b, const double* const* U, int k,
                             double* const* x, double tol, int restart, int maxit,
                             ddg_precision prec, ddg_info* info);

/*
 * gmres_solve_queue_trajectories -- the solve queue over design trajectories
 * with recycling (no paper counterpart beyond gmres_solve_trajectories): the
 * n_traj trajectories of n_steps problems (host arrays of n_traj * n_steps
 * entries, trajectory-major, as gmres_solve_trajectories) are taken in groups
 * of traj_per_group consecutive trajectories by nlanes concurrent lanes, each
 * group solved by gmres_solve_trajectories on the lane's context and stream
 * (step t of the group's trajectories in one batch, subspace [U | x_{t-1}]).
 * Concurrent lanes fill the GPU that one group's per-step batches leave
 * idle.  Every solve's result is that of gmres_solve_trajectories on its own
 * trajectory.  Other arguments and the return value as gmres_solve_queue.
 */
ddg_status gmres_solve_queue_trajectories(ddg_context* const* lanes, void* const* streams, int nlanes,
                                          int traj_per_group, int n_traj, int n_steps, const ddg_op* const* A,
                                          const double* const* b, const double* const* U, int k, double* const* x,
                                          double tol, int restart, int maxit, ddg_precision prec, ddg_info* info);

/*
 * pca_fit -- principal components of training fields (Sec. III, "Principal
 * component analysis": an incomplete SVD of the matrix whose columns are the
 * training fields; uncentred, no normalisation).  U receives the k leading left
 * singular vectors of F, computed by the method of snapshots in FP64: G = F^H F,
 * its top-k eigenpairs by block subspace iteration (k + 16 vectors) with
 * Rayleigh-Ritz, u_c = F w_c / sigma_c.  Singular vectors are defined up to a
 * unit phase (and a rotation inside repeated singular values).
 *   F      device, D x M complex128, column-major (field m at F + 2*D*m).
 *   U      device, D x k complex128, column-major, written in full.
 *   sigma  (host) k doubles (sigma_1 >= ... >= sigma_k), may be NULL.
 *   1 <= k <= min(32, M), M <= D, M <= 8192.  Uses the context's workspace
 *   (about (slices + 1) * M^2 * 16 bytes, slices <= 64); synchronises `stream`
 *   when sigma is requested.
 */
ddg_status pca_fit(ddg_context* ctx, const double* F, long long D, int M, int k, double* U,
                   double* sigma, void* stream);

/*
 * Subspace predictor (Sec. III, "Convolutional neural network", Fig. 3a): a CNN
 * mapping the permittivity to k complex vectors v_1..v_k that span the
 * predicted subspace, trained with the projection loss (Eq. 5) and Adam
 * (Methods).  Architecture: `levels` resolutions with channels[l] channels, two
 * 3x3 convolutions + ReLU per level, 2x2 average pooling between encoder levels,
 * nearest 2x upsampling concatenated with the encoder output of the same level
 * in the decoder, a 1x1 head to 2k channels (pair (2c, 2c+1) = (Re, Im) of v_c).
 * Inputs per cell: (eps - 2.1)/10.15, (wavelength - 1.3 um)/0.25 um, PML mask,
 * source profile exp(-(j - j_c)^2 / (2 sigma^2)) on column i_src.
 * Parameters: a flat FP32 vector, per layer the weights [Cout][Cin][kh][kw]
 * then the biases, layers in the order enc0a, enc0b, ..., enc{L-1}b,
 * dec{L-2}a, dec{L-2}b, ..., dec0b, head.  The forward pass uses BF16 weights
 * and activations with FP32 accumulation; gradients and Adam are FP32.
 * A batch must share one grid size, with nx and ny divisible by 2^(levels-1).
 */
typedef struct ddg_predictor ddg_predictor;
/* k complex outputs (1..16); channels: `levels` (1..8) host ints.  Weights start at 0. */
ddg_status predictor_create(int k, int levels, const int* channels, ddg_predictor** P);
/* predictor_create_with_field -- the same network with two more input channels:
   the real and imaginary parts of an approximate field of the grid, normalised
   to max |f| = 1 (the paper's networks take a cheap approximate field as input,
   Sec. III and Methods; here e.g. the field of the unpatterned background, one
   solve per grid and wavelength).  Set it with predictor_set_input_field
   before any forward or training call on that grid. */
ddg_status predictor_create_with_field(int k, int levels, const int* channels, ddg_predictor** P);
/* f: device, ny*nx complex128 (row-major), copied (normalised) into the
   predictor; DDG_EINVAL for a network created without the field input. */
ddg_status predictor_set_input_field(ddg_predictor* P, const double* f, int nx, int ny, void* stream);
/* predictor_set_output_base -- a fixed offset added to the network's output
   (no paper counterpart; the paper gives no architecture): the predicted
   vectors become v_c = scale * U_c + CNN(eps)_c.  With U a data-derived basis
   (for instance the leading principal components of the training fields,
   pca_fit) and the head initialised at zero, training starts from that basis
   and learns permittivity-dependent corrections.  The offset is not trained.
     U  device, D x k complex128 column-major (column c at U + 2 D c), D = nx ny;
        NULL removes the offset.
   The offset serves every problem of that grid size (one offset per grid
   size; setting it again replaces it).  A forward, prediction or training
   call with a problem of a grid size that has no offset, while any offset is
   set, is refused (DDG_EINVAL).  U = NULL removes every offset. */
ddg_status predictor_set_output_base(ddg_predictor* P, const double* U, int nx, int ny, double scale, void* stream);
/* predictor_set_output_base_wavelength -- as predictor_set_output_base, for
   the problems of this grid at one vacuum wavelength (metres, > 0; matched to
   1e-9 relative).  A problem takes the offset of its grid and wavelength if
   there is one, else its grid's offset for every wavelength.  Serves one
   network conditioned on the wavelength with a data-derived basis per
   wavelength (the fields of one device at two wavelengths differ). */
ddg_status predictor_set_output_base_wavelength(ddg_predictor* P, const double* U, int nx, int ny,
                                                double wavelength, double scale, void* stream);
ddg_status predictor_destroy(ddg_predictor* P);
long long predictor_num_params(const ddg_predictor* P);
/* Number k of predicted complex vectors (0 for NULL). */
int predictor_num_outputs(const ddg_predictor* P);
/* Kernels launched by this predictor since it was created. */
long long predictor_launches(const ddg_predictor* P);
/* 3x3 convolutions on the tensor cores (no paper counterpart).  `enable` is a
   set of bits: 1 (the default) = the forward convolutions, 2 = the backward
   convolutions: the gradient w.r.t. a layer's input (run as a forward
   convolution from the output to the input channels with flipped taps) and
   w.r.t. its weights (a GEMM over the pixels: output channels x (tap, input
   channel)).  Layers whose channel counts are multiples of 16 (at most 256
   outputs forward and backward-data, at most 128 for the weight gradient)
   run on tcgen05 (BF16 operands, FP32 accumulation in tensor memory), and so
   does the first layer's forward (at most 16 input channels, read from a copy
   of the input zero-padded to 16 channels, with zero weights for the
   padding); the others, the head and the bias gradients use CUDA cores.  The forward paths
   give the same results up to FP32 summation order; with bit 2 the masked
   output gradient enters both backward products rounded to BF16 (the
   CUDA-core path keeps it in FP32).  Bit 4 (with bit 1; the default is
   1 | 4): a forward convolution whose input is one plain tensor (not the
   decoder's upsampled concatenation), on a grid that is a multiple of 16 x 8
   pixels and whose weights and two 18 x 10 halo tiles fit in shared memory,
   loads its input tiles by TMA (cp.async.bulk.tensor) and reads the nine taps
   as descriptor offsets into the loaded tile, with no gather on the SM; same
   K order and results as the gather.  A tensor-core wait that gives up makes
   the call return DDG_ETIMEOUT.  0 <= enable <= 7, else DDG_EINVAL. */
ddg_status predictor_set_tensor_cores(ddg_predictor* P, int enable);
/* theta: host, n = predictor_num_params floats.  Setting resets the Adam state. */
ddg_status predictor_set_params(ddg_predictor* P, const float* theta, long long n);
ddg_status predictor_get_params(const ddg_predictor* P, float* theta, long long n);
/* Raw network output for n problems: y device FP32 [n][ny][nx][2k]. */
ddg_status predictor_forward(ddg_predictor* P, int n, const ddg_op* const* A, int i_src, double sigma,
                             double j_c, float* y, void* stream);
/* subspace_predict -- the predicted subspace of each problem, orthonormal:
   the network's k vectors (with the output offset, as predictor_forward)
   orthonormalised on the device by Cholesky QR applied twice in FP64
   (G = V^H V = L L^H, V <- V L^-H), so U[s]^H U[s] = I to FP64 round-off and
   span U[s] = span of the raw output.  A vector whose Cholesky pivot falls
   below 1e-13 of the largest (already spanned by the vectors before it) is
   returned as a zero column.  U[s] device, D x k complex128 column-major
   (ready for augmented_gmres_solve).  Synchronises. */
ddg_status subspace_predict(ddg_predictor* P, int n, const ddg_op* const* A, int i_src, double sigma,
                            double j_c, double* const* U, void* stream);
/* Training loss: 0 = projection loss (Eq. 5), the default: f[s] are solved
   fields; 1 = residual loss (Eq. 6), unsupervised: f[s] are the right-hand
   sides b (l = min over z of ||A V z - b||^2 / ||b||^2 with the problem's own A;
   its gradient is A^H applied to Eq. 5's gradient in W = A V, with
   A^H x = conj(S_b A S_b^-1 conj(x)), S_b = diag(sxb_i syb_j)). */
ddg_status predictor_set_loss(ddg_predictor* P, int kind);
/* Mean training loss over the batch (f[s]: device, D complex128 each: the
   solved fields, or the right-hand sides for the residual loss) and its
   gradient (kept inside the predictor; also copied to `grad`, device FP32
   [nparams], when not NULL).  Synchronises. */
ddg_status predictor_loss_grad(ddg_predictor* P, int n, const ddg_op* const* A, int i_src, double sigma,
                               double j_c, const double* const* f, double* loss, float* grad, void* stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) with the last gradient;
   skipped (weights and moments unchanged) when the last loss was not finite. */
ddg_status predictor_adam_step(ddg_predictor* P, float lr, void* stream);
/* predictor_loss_grad followed by predictor_adam_step. */
ddg_status predictor_train_step(ddg_predictor* P, int n, const ddg_op* const* A, int i_src, double sigma,
                                double j_c, const double* const* f, float lr, double* loss, void* stream);
/* Checkpoint of the weights, Adam moments and step, with a checksum; load checks
   the architecture and the checksum (DDG_EINVAL on mismatch). */
ddg_status predictor_save(const ddg_predictor* P, const char* path);
ddg_status predictor_load(ddg_predictor* P, const char* path);

/*
 * fdfd_solve_host -- the path of a user who holds permittivities and wants
 * fields, from and to HOST memory in one call (Eq. 1 set up, Eqs. 3-4 solved;
 * no paper counterpart beyond that): for each of n problems the permittivity
 * is copied to the device, the operator (fdfd_operator) and the source
 * (fdfd_source) are built, the subspace [U_fixed[s] | the predictor's k
 * vectors] is assembled (subspace_predict when P is not NULL) and
 * augmented_gmres_solve_batched runs, or plain GMRES (gmres_solve_batched)
 * when there is neither P nor U_fixed; the solution is copied back.
 *   grids     (host) n problem descriptions (with P: one grid size; the
 *             wavelengths may differ, e.g. one device at two wavelengths).
 *   eps_host  (host) n pointers to ny*nx doubles, row-major (pinned memory
 *             lets the copies run asynchronously).
 *   i_src, sigma, j_c  the source of every problem, as fdfd_source.
 *   U_fixed   NULL, or (host array of) n DEVICE pointers to D x k_fixed
 *             complex128 column-major bases placed before the predicted
 *             vectors (e.g. the principal components of each problem's
 *             wavelength, to be kept across restarts with
 *             ddg_context_set_augmented_policy); k_fixed = 0 without it, else
 *             1 <= k_fixed and k_fixed + k <= 32.
 *   x_host    (host) n pointers to 2*D doubles: the fields (x0 = 0).
 *   tol, restart, maxit, prec, info: as the batched solves.
 * The device copies of eps, b, x and the subspace live in a buffer that the
 * context keeps and grows (about (8 + 32 + 16 (k_fixed + k)) D bytes per
 * problem).
 * Returns the solve's status (DDG_ENOCONV: fields copied back, some solve
 * missed the tolerance); on other errors x_host is not written.
 * Synchronises `stream`.
 */
ddg_status fdfd_solve_host(ddg_context* ctx, ddg_predictor* P, int n, const ddg_grid* grids,
                           const double* const* eps_host, int i_src, double sigma, double j_c,
                           const double* const* U_fixed, int k_fixed, double tol, int restart, int maxit,
                           ddg_precision prec, double* const* x_host, ddg_info* info, void* stream);

/*
 * gmres_solve_noalloc -- gmres_solve without any device allocation.  (The paper
 * has no counterpart: this is a library convenience.)
 *
 * Some callers cannot let a library call cudaMalloc: their device memory is
 * owned in full by another allocator (a framework's caching allocator or a
 * fixed budget that a stray cudaMalloc would break), or they cannot afford the
 * device-wide synchronisation that cudaMalloc and cudaFree may cause.  This
 * entry point needs no ddg_context: its whole workspace lives in one static
 * device array of DDG_NOALLOC_SCRATCH_BYTES bytes, which every GPU that loads
 * the library holds until the process exits.  It runs one plain restarted
 * GMRES solve with the same Arnoldi kernels as gmres_solve (delayed
 * reorthogonalisation).  Supported precisions: DDG_C128 and DDG_C64_REFINE
 * (DDG_C64_ONLY returns DDG_EINVAL).  Having no context, it takes none of a
 * context's options: the basis is always stored in the arithmetic type (FP32
 * for DDG_C64_REFINE), there is no preconditioner, the step loop is launched by
 * the host, and the DDG_C64_REFINE inner tolerance is fixed at 1e-5.  It polls
 * the solve's state by synchronising the stream every 16 Arnoldi steps (no
 * pinned buffer, no events), so it trades some speed against gmres_solve for
 * having no allocation.
 *   - Sizes whose workspace exceeds the array are rejected with DDG_EINVAL
 *     (about (restart + 4) * D * 8 bytes for DDG_C64_REFINE, twice that for
 *     DDG_C128, plus O(restart^2) bytes: D = 128 x 128 fits restart = 200).
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress); make that first call before any stream capture.
 *   - Every call shares the array and it keeps the last call's contents (the
 *     call initialises what must start at zero).  Calls that overlap on the GPU
 *     (other streams, other host threads) race on it and must be serialised.
 * Other arguments and results as gmres_solve; the caller still owns b, x and A.
 */
#define DDG_NOALLOC_SCRATCH_BYTES (32LL << 20)
ddg_status gmres_solve_noalloc(const ddg_op* A, const double* b, double* x, double tol, int restart,
                               int maxit, ddg_precision prec, ddg_info* info, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* DDGMRES_H */
