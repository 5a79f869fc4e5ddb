/*
 * seedcg.h - C ABI of the GB300 (sm_103a) Improved Seed-CG library.
 *
 * The library solves many Hermitian positive-definite systems
 *     M x^j = b^j,  j = 1..nrhs,   M = D^dag D,   D = 1 - kappa H_Wilson
 * with the Improved Seed-CG method of Abdel-Rehim, Morgan and Wilcox
 * ("Seed methods for linear equations in lattice QCD problems with multiple
 * right-hand sides", Lattice 2008): the first system is solved by Lanczos
 * (Algorithm 1) past convergence with periodic re-orthogonalisation (PO),
 * its stored basis V seeds every other system through the Galerkin
 * projection of Eq. (1) updated with the LU factorisation of T (Eq. 2), and
 * standard CG finishes the seeded systems (Section 2).
 *
 * Conventions shared by every call (Section 3 names the operator only as
 * "Wilson fermions"; these are the conventions this library fixes):
 *   - site index s = x + Lx*(y + Ly*(z + Lz*t)); mu = 0,1,2,3 <-> x,y,z,t.
 *   - gauge field: complex128 (re, im interleaved doubles) [site][mu][a][b],
 *     U_mu(x) with colour row a, column b.
 *   - spinor field: complex128 [site][spin 4][colour 3]; a batch of n spinor
 *     fields is n such fields back to back.
 *   - (D psi)(x) = psi(x) - kappa sum_mu [ (1 - g_mu) U_mu(x) psi(x+mu)
 *                                         + (1 + g_mu) U_mu(x-mu)^dag psi(x-mu) ],
 *     periodic in x,y,z and antiperiodic in t (a factor -1 on hops that wrap
 *     t); chiral gamma basis g_k = [[0,-i s_k],[i s_k,0]], g_4 = [[0,1],[1,0]];
 *     D^dag = g5 D g5, g5 = diag(1,1,-1,-1).
 *
 * Memory: a pointer argument documented as "host or device" may be either;
 * the library asks the CUDA runtime which one it is.  Device pointers must
 * be on the device that was current at seedcg_create.  All device work is
 * ordered on the caller's stream (NULL = legacy default stream); every call
 * returns after that work has completed unless documented otherwise.
 *
 * Errors: every call returns a seedcg_status.  Arguments are checked before
 * any device work; on failure seedcg_last_error() describes it.  No call
 * throws across the ABI.  A handle is not thread-safe: one caller at a time.
 */
#ifndef SEEDCG_H
#define SEEDCG_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct seedcg_handle seedcg_handle;

typedef enum {
    SEEDCG_OK = 0,
    SEEDCG_ERR_ARG = -1,            /* invalid argument (nothing was run)          */
    SEEDCG_ERR_OOM = -2,            /* device allocation failed                    */
    SEEDCG_ERR_CUDA = -3,           /* a CUDA runtime call failed                  */
    SEEDCG_ERR_NOT_CONVERGED = -4,  /* an iteration limit was hit; X = best iterate */
    SEEDCG_ERR_BREAKDOWN = -5,      /* delta_i = 0 in the LU of T (M not HPD)      */
    SEEDCG_ERR_NAN = -6,            /* a NaN/Inf appeared in a scalar              */
    SEEDCG_ERR_TIMEOUT = -7         /* a bounded device wait ran out               */
} seedcg_status;

typedef enum {
    SEEDCG_FP64 = 0,          /* every vector, V and the dslash in FP64                  */
    SEEDCG_MIXED_V32 = 1,     /* FP32 dslash and vectors, V in complex64, FP64 scalars    */
    SEEDCG_MIXED_VBF16 = 2    /* as MIXED_V32 but V stored in bf16 (tensor-core projections) */
} seedcg_precision;

typedef struct {
    int m_max;             /* largest Krylov dimension m stored in V (Algorithm 1, "m");
                              0 = default 4000 */
    double past_factor;    /* >= 1: run RHS 1 to m = max(m_conv + extra_iters,
                              ceil(past_factor * m_conv)), capped by m_max (Section 2:
                              "solved past the convergence limit")                  */
    int precision;         /* seedcg_precision                                          */
    double reliable_delta; /* mixed CG: recompute the FP64 true residual whenever the
                              iterated residual fell by this factor (default 0.1)      */
    int po_passes;         /* 1 = classical Gram-Schmidt, 2 = CGS2 (default 1)         */
    int seed_mode;         /* 0 = literal per-iteration updates (Algorithm 1 steps 3-7;
                              FP64 only), 1 = blocked: x^1 by the LU recurrence of steps
                              3 and 6, the systems j >= 2 by Eq. (1) after the Lanczos run,
                              2 = classic repeated seeding, the comparison variant of
                              Section 1: each system in turn is run by Lanczos from its
                              current guess to convergence (past_factor and extra_iters
                              are not used) and seeds the systems after it by Eq. (1);
                              CG then finishes any system still above tol;
                              3 = no seeding: standard CG for every system from x_0
                              (no Lanczos, no basis), the baseline Section 3 measures
                              the seeded systems against; seedcg_solve only           */
    int x0_given;          /* 1: X holds initial guesses x_0^j on entry                */
    int cg_maxiter;        /* CG iteration cap per system (default 20000)               */
    int stop_after_seed;   /* 1: return the seeded guesses without running CG (tests)  */
    int poll_every;        /* iterations between host polls of device flags (default 32) */
    int use_tensor_cores;  /* bf16 basis only: 1 (default) projections V^dag X of more than
                              two vectors (the Eq. (1) seeds) on tcgen05 and the
                              two-vector PO projection on SIMT (measured faster: it is a
                              bandwidth-bound GEMV); 2: every projection on tcgen05;
                              0: every projection on SIMT */
    int use_guess;         /* 1: start every system from the learned guess x_0 = net(b)
                              (weights set by seedcg_guess_set_weights/_train); a system
                              whose guess has ||b - M x_0|| >= ||b|| starts from 0 */
    int resid_mode;        /* 0 (default): B holds b of M x = b, and ||b - M x|| <= tol ||b||
                              (FP64) is the stopping criterion.  1: B holds eta of the
                              original system D x = eta (Section 3 monitors its residual);
                              the solve forms b = D^dag eta, and ||eta - D x|| <= tol ||eta||,
                              recomputed in FP64, is the binding criterion: systems that miss
                              it continue CG with a tighter M tolerance (up to six rounds).
                              seedcg_solve only. */
    int po_guard;          /* 1 (default): a PO step (Algorithm 1 step 8) that finds the stored
                              basis far from orthonormal ends the Lanczos run at i - 1: a
                              projection pass leaving ||v_i|| < 1/2 (v_i within 30 degrees of
                              the stored space), or re-orthogonalisation lengthening f by more
                              than 1 % (impossible for an orthonormal basis).  0: step 8 runs
                              as printed whatever it finds (the run still ends if v_i vanishes
                              or a scalar is not finite). */
} seedcg_options;

typedef struct {
    /* filled by seedcg_solve; the array pointers are caller-owned host arrays
       of nrhs entries each, or NULL to skip them */
    int m_conv;            /* first i with beta_i |zeta_i/delta_i| <= tol ||b^1||        */
    int m;                 /* Lanczos iterations run (basis size)                       */
    int po_count;          /* periodic re-orthogonalisation steps taken                 */
    int cg_iters_max;      /* CG iterations of the slowest seeded system                */
    int reliable_updates;  /* FP64 residual recomputations in the CG phase              */
    int* iters;            /* per RHS: Lanczos iterations (j=1) + CG iterations         */
    int* matvecs;          /* per RHS: applications of D or D^dag                        */
    double* true_resid;    /* per RHS: ||b - M x|| / ||b||, FP64                         */
    float ms_total, ms_lanczos, ms_po, ms_seed, ms_cg;   /* device-event phase times    */
    double* true_resid_D;  /* per RHS: ||eta - D x|| / ||eta||, FP64; written only when
                              resid_mode = 1 (NULL to skip)                               */
} seedcg_info;

/* Fill *opt with the defaults documented above. */
void seedcg_default_options(seedcg_options* opt);

/*
 * Create a solver for one gauge field (Section 3: one configuration, many
 * right-hand sides).  dims = {Lx, Ly, Lz, Lt}, each >= 2 and even.
 * gauge: host or device, complex128 [V][4][3][3]; copied, the caller keeps
 * ownership.  kappa: hopping parameter.  opt may be NULL (defaults).
 * Returns SEEDCG_ERR_ARG for bad dims/pointers, SEEDCG_ERR_OOM/CUDA on
 * device failures; *h is NULL on failure.
 */
seedcg_status seedcg_create(seedcg_handle** h, const int dims[4], const double* gauge,
                            double kappa, const seedcg_options* opt);

/* Change options of an existing handle (takes effect at the next solve). */
seedcg_status seedcg_set_options(seedcg_handle* h, const seedcg_options* opt);

/*
 * Solve M x^j = b^j for j = 1..nrhs (Section 2, Algorithm 1 + CG).
 * B: host or device, complex128 [nrhs][V][4][3], read only.
 * X: host or device, same layout; on entry x_0^j if opt.x0_given, on exit the
 *    solutions (or the seeded guesses if opt.stop_after_seed).
 * tol: relative residual; convergence is ||b - M x|| <= tol ||b|| in FP64.
 * extra_iters: Lanczos iterations past m_conv (see seedcg_options.past_factor).
 * reorth_period: k of Algorithm 1 (PO every k iterations), 0 = none.
 * info: NULL or filled on return (also on NOT_CONVERGED).
 * stream: cudaStream_t or NULL.
 */
seedcg_status seedcg_solve(seedcg_handle* h, int nrhs, const double* B, double* X, double tol,
                           int extra_iters, int reorth_period, seedcg_info* info,
                           void* stream);

/*
 * Several gauge fields at once (each handle one field, e.g. lattices of
 * different sizes): for every field, Algorithm 1 on its first right-hand side
 * and the Eq. (1) seeds of its others; then ONE batched CG over the seeded
 * systems of all fields (a multi-field multi-RHS dslash per half-step, the
 * iteration chunks replayed as a CUDA graph).  hs: nfields (1..16) distinct
 * handles of the same precision mode and device; nrhs[f], B[f], X[f] as in
 * seedcg_solve for field f (host or device; at most 512 systems in total).
 * infos: NULL or nfields entries.  The options of each handle apply to its
 * Lanczos run; those of hs[0] to the CG phase.
 */
seedcg_status seedcg_batch_solve(seedcg_handle** hs, int nfields, const int* nrhs,
                                 const double* const* B, double* const* X, double tol,
                                 int extra_iters, int reorth_period, seedcg_info* infos,
                                 void* stream);

/*
 * Apply the operator to n spinor fields (for parity checks and for forming
 * b = D^dag eta): the Wilson operator of Section 3, D = 1 - kappa H with the
 * projector, gamma-basis and boundary conventions stated at the top of this
 * header, D^dag = g5 D g5, and M = D^dag D, the matrix Algorithm 1 and the CG
 * of Section 2 solve with.  op: 0 = D, 1 = D^dag, 2 = M = D^dag D.  prec: 0 = FP64
 * arithmetic, 1 = FP32 arithmetic (inputs rounded to FP32, result widened).
 * in/out: device pointers, complex128 [n][V][4][3]; they may not overlap.
 * multi = 1 uses the multi-RHS kernel (links staged once per site tile for
 * all n fields), 0 the single-RHS kernel n times.
 */
seedcg_status seedcg_apply(seedcg_handle* h, int op, int prec, int multi, int n,
                           const double* in, double* out, void* stream);

/*
 * Even-odd preconditioned operator (Section 3 solves the even-odd system):
 * with the sites split by parity (x + y + z + t even / odd; every lattice
 * extent must be even), the odd-site Schur complement A = 1 - kappa^2 H_oe H_eo,
 * where D = 1 - kappa H.  Half-lattice vectors are complex128
 * [n][V/2][4][3] holding the odd sites in lexicographic site order.
 * op: 0 = A, 1 = A^dag (= gamma5 A gamma5), 2 = A^dag A.  prec: 0 = FP64,
 * 1 = FP32 arithmetic.  in/out: device pointers that may not alias.
 * SEEDCG_ERR_ARG for odd extents, host pointers or bad op/prec.
 */
seedcg_status seedcg_apply_eo(seedcg_handle* h, int op, int prec, int n, const double* in,
                              double* out, void* stream);
/* phi = eta_o + kappa H_oe eta_e, the right-hand side of A x_o = phi for D x = eta.
   eta: device, full [n][V][4][3]; phi: device, half [n][V/2][4][3]; FP64. */
seedcg_status seedcg_eo_source(seedcg_handle* h, int n, const double* eta, double* phi, void* stream);
/*
 * Improved Seed-CG on the even-odd system (Section 3 solves A^dag A x_o = A^dag phi):
 * for each right-hand side eta (device, full [nrhs][V][4][3]) phi = eta_o + kappa H_oe eta_e
 * and b = A^dag phi are formed in FP64, Algorithm 1 runs on A^dag A with the handle's
 * options on the device-resident engine of seedcg_solve (every precision mode and seeding
 * form seed_mode 0-3: Lanczos with the LU of T, PO, Eq. (1) seeds, the batched CG with FP64
 * reliable updates), on odd-site half vectors; then x_e = eta_e + kappa H_eo x_o gives the
 * full solution x (device, full; on entry x_0 if opt.x0_given, of which the odd sites are
 * used).  The binding criterion is ||b - A^dag A x_o|| <= tol ||b|| in FP64
 * (info->true_resid); info->true_resid_D, when not NULL, receives the original system's
 * ||eta - D x|| / ||eta|| in FP64.  info->matvecs counts applications of the full-lattice
 * D: one A^dag A (four half-lattice hops) counts 2.  use_guess and resid_mode = 1 are
 * refused (SEEDCG_ERR_ARG).  Afterwards seedcg_get_basis returns odd-site half vectors
 * [count][V/2][4][3]; seedcg_project_basis and seedcg_deflate_guess refuse the basis.
 */
seedcg_status seedcg_solve_eo(seedcg_handle* h, int nrhs, const double* eta, double* x, double tol,
                              int extra_iters, int reorth_period, seedcg_info* info, void* stream);
/* The full solution of D x = eta from x_o: x_e = eta_e + kappa H_eo x_o.
   x_odd: device, half; eta, x: device, full; FP64. */
seedcg_status seedcg_eo_reconstruct(seedcg_handle* h, int n, const double* x_odd, const double* eta,
                                    double* x, void* stream);

/*
 * seedcg_apply for callers that cannot allocate device memory, e.g. a host
 * framework whose caching allocator has reserved the GPU's memory for its own
 * pool, or a caller that cannot afford the allocation and implicit
 * synchronisation of cudaMalloc / cudaFree on every call.  (The paper has no
 * counterpart: this is a property of the library, not of the method.)
 * Same arguments, layouts and results as seedcg_apply; in and out are the
 * caller's device buffers on the handle's GPU (host, pinned or unregistered
 * memory is refused with SEEDCG_ERR_ARG before any kernel runs).  The scratch (internal copies of in, the
 * intermediate and the output) is one fixed 16 MiB device array that every
 * GPU loading this library holds until the process exits; the call returns
 * SEEDCG_ERR_ARG, with a message, when 3 * n * V * 12 * (16 B for prec 0,
 * 8 B for prec 1) exceeds 16 MiB.  No device memory is allocated or freed.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture.  All calls share the one array and every call
 * overwrites it before reading it: calls that overlap on the GPU (other
 * streams, other threads, other handles on the same device) race.
 */
seedcg_status seedcg_apply_noalloc(seedcg_handle* h, int op, int prec, int multi, int n,
                                   const double* in, double* out, void* stream);

/*
 * After a solve: copy the Lanczos scalars of RHS 1 (alpha_1..m, beta_1..m,
 * delta_1..m; Eq. 2) into caller host arrays of `cap` doubles (any may be
 * NULL).  Returns the number m written via *m_out.
 */
seedcg_status seedcg_get_lanczos(const seedcg_handle* h, int cap, double* alpha, double* beta,
                                 double* delta, int* m_out);

/*
 * After a solve: copy stored basis vectors v_first .. v_first+count-1 (0-based)
 * as complex128 [count][V][4][3] into `out` (host or device).  Works for every
 * V precision (the stored values are widened).
 */
seedcg_status seedcg_get_basis(seedcg_handle* h, int first, int count, double* out);

/*
 * After a solve: C[a][j] = v_a^dag x_j, the projection of nvec spinor fields
 * onto the first `rows` stored basis vectors (the contraction that Algorithm 1
 * step 8 and Eq. (1) perform against V).  X: device, complex128 [nvec][V][4][3];
 * C: host, complex128 [rows][nvec].  use_tensor_cores = 1 takes the tcgen05
 * path when V is stored in bf16 (x_j rounded to bf16 for the product), 0 the
 * SIMT path (x_j rounded to the working precision).
 */
seedcg_status seedcg_project_basis(seedcg_handle* h, int rows, int nvec, const double* X,
                                   double* C, int use_tensor_cores, void* stream);

/*
 * Host only: the nev smallest eigenpairs of the symmetric tridiagonal matrix
 * with alpha[0..m-1] on the diagonal and beta[0..m-2] beside it (T_m of Eq. 2's
 * Lanczos run), by Sturm-sequence bisection and inverse iteration.  theta: nev
 * ascending values; S: row-major [m][nev], S[a*nev + j] = entry a of eigenvector
 * j (unit length).  SEEDCG_ERR_ARG for bad sizes or NULL pointers.
 */
seedcg_status seedcg_tridiag_lowest(int m, const double* alpha, const double* beta, int nev, double* theta,
                                   double* S);

/*
 * Deflated initial guesses from the last solve's stored basis (the premise of
 * Sections 1-2: the basis built past convergence holds accurate low
 * eigenvectors).  The nev (<= 64) smallest Ritz pairs (theta_j, y_j = V s_j) of
 * T_m give, for each of nr new right-hand sides b (same gauge field), the
 * Galerkin guess x0 = Y c with (Y^dag M Y) c = Y^dag b, in FP64.  B, X0: device,
 * complex128 [nr][V][4][3]; ritz_values: host, nev doubles, or NULL.  Pass X0
 * with x0_given = 1 to a later seedcg_solve.  SEEDCG_ERR_BREAKDOWN if Y^dag M Y
 * is not positive definite.
 */
seedcg_status seedcg_deflate_guess(seedcg_handle* h, int nev, int nr, const double* B, double* X0,
                                   double* ritz_values, void* stream);

/*
 * Learned initial guess (the project's extension; the paper has none): a
 * gauge-covariant nearest-neighbour network of three layers, 1 -> 8 -> 8 -> 1
 * channels,
 *   out_co(x) = sum_ci [ W_0 in_ci(x) + sum_{d=+-mu} W_d U(x,d) in_ci(x+d) ],
 * U(x,+mu) = U_mu(x), U(x,-mu) = U_mu(x-mu)^dag with the operator's boundary
 * sign; W_d[co][ci] a complex 4x4 spin matrix; ReLU on real and imaginary
 * parts after layers 1 and 2; input b/||b||, output times ||b||.
 * Weights: complex128 (host) [11520] = layer 1 [9][8][1][4][4], layer 2
 * [9][8][8][4][4], layer 3 [9][1][8][4][4], directions 0, +x,-x,+y,-y,+z,-z,+t,-t.
 * B, X, X0: host or device, complex128 [n][V][4][3].  Storage is bf16 (the
 * activations, their gradients and the weights the layers read), accumulation
 * FP32; the 8 -> 8 layer's contraction (K = 288 complex terms per output) runs on
 * the tcgen05 tensor cores, forward and backward through the data; Adam keeps
 * FP32 master weights (what guess_get_weights returns) and sums the gradient
 * in FP64.  SEEDCG_ERR_TIMEOUT if a bounded tensor-core wait expired.
 */
seedcg_status seedcg_guess_set_weights(seedcg_handle* h, const double* w);
seedcg_status seedcg_guess_get_weights(seedcg_handle* h, double* w);
/* loss = mean_k ||net(b_k) - x_k||^2 / ||x_k||^2 and, if grad is not NULL, its
   gradient dL/dRe(W) + i dL/dIm(W) (complex128 host [11520]) */
seedcg_status seedcg_guess_loss_grad(seedcg_handle* h, int npairs, const double* B, const double* X,
                                     double* loss, double* grad, void* stream);
/* Adam (beta = 0.9, 0.999, eps = 1e-8) over `epochs` passes of the pairs in
   their given order, mini-batches of `batch`; *final_loss = last epoch's mean.
   There is no random-number seed: training draws nothing at random (the weights
   come from seedcg_guess_set_weights, the order of the pairs from the caller),
   so a run is reproducible from its inputs alone; `stream` orders the work as in
   seedcg_solve. */
seedcg_status seedcg_guess_train(seedcg_handle* h, int npairs, const double* B, const double* X,
                                 int epochs, int batch, double lr, double* final_loss, void* stream);
/* X0[k] = net(B[k]) */
seedcg_status seedcg_guess_predict(seedcg_handle* h, int n, const double* B, double* X0, void* stream);

/*
 * Measurement helper: time `reps` launches of the multi-RHS dslash D on n
 * internal spinor fields (prec 0 = FP64, 1 = FP32) with CUDA events on
 * `stream`, writing a 512 MB buffer between launches when flush_l2 != 0 so
 * that every launch starts from a cold L2.  *ms_per_launch receives the mean.
 */
seedcg_status seedcg_time_dslash(seedcg_handle* h, int prec, int n, int reps, int flush_l2,
                                 float* ms_per_launch, void* stream);

/*
 * Failure-detection self-check (no counterpart in the paper): one thread waits
 * on an mbarrier that nothing arrives at, through the bounded wait that the
 * tensor-core kernels use for every mbarrier, with a limit of limit_ms (0, 1000]
 * milliseconds instead of their 1 s.  *kernel_status receives what the kernel
 * reports: SEEDCG_ERR_TIMEOUT when the wait gave up as it must.  Returns
 * SEEDCG_OK when the launch ran and the status was read (the context stays
 * usable), SEEDCG_ERR_ARG for a bad limit or NULL pointer.
 */
seedcg_status seedcg_selftest_bounded_wait(double limit_ms, int* kernel_status);

/* Number of CUDA kernels this library has launched in this process (all
   handles, all threads); differences around a call count its launches. */
unsigned long long seedcg_kernel_launches(void);

/* Message for the last failing call on h (never NULL). */
const char* seedcg_last_error(const seedcg_handle* h);

/* Free everything the handle owns.  NULL is ignored. */
void seedcg_destroy(seedcg_handle* h);

#ifdef __cplusplus
}
#endif
#endif /* SEEDCG_H */
