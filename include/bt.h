/*
 * bt.h -- C ABI of libbt: preconditioned conjugate gradient for symmetric
 * positive definite block-tridiagonal systems S x = b on an NVIDIA GB300
 * (sm_103a), preconditioned by the parametrised multi-splitting polynomial
 * preconditioner of arXiv 2503.15269 at its optimal parameters.
 *
 * The matrix (Sec. 2.1, Eq. 1): N diagonal blocks D_i (n x n, SPD) and N-1
 * off-diagonal blocks O_i = S[i, i+1], with S[i+1, i] = O_i^T; blocks are
 * dense.  Indices are 0-based here (the paper counts from 1).
 *
 * The preconditioner (Sec. 3.1 and Sec. 3.5): with a = 1, b = -1,
 *     M^-1 = (alpha_0 I + alpha_1 H + ... + alpha_{m-1} H^{m-1}) G,
 * alpha_0 = 1, where G = G_opt (block tridiagonal) and H = H_opt (block
 * pentadiagonal with zero +-1 blocks) have the closed forms of Sec. 4.1:
 *     E_i = D_i^-1 O_i D_{i+1}^-1
 *     G[i,i] = D_i^-1,  G[i,i+1] = -E_i,  G[i+1,i] = -E_i^T
 *     H[i,i] = E_{i-1}^T O_{i-1} + E_i O_i^T,  H[i,i+2] = E_i O_{i+1},
 *     H[i+2,i] = E_{i+1}^T O_i^T.
 * It is applied as in Sec. 4.2: y_0 = G r, y_j = H y_{j-1}, z = sum alpha_j y_j.
 * Other members of the family (bt_params.a in [0, 1), b = 1 - 2a) use, with
 * the block Jacobi matrix H_J = B_d^-1 C_d,
 *     G_ab = B_d^-1 + a B_d^-1 C_d B_d^-1   (E_i above scaled by a)
 *     H_ab = a H_J^2 + (1 - a) H_J          (a H_opt plus the +-1 blocks
 *            -(1-a) D_i^-1 O_i and -(1-a) D_{i+1}^-1 O_i^T),
 * the block form of the multi-splitting of Sec. 3.1.
 *
 * Conventions for every call below:
 *   - Array arguments named D, O, b, x, r, z, y are DEVICE pointers to
 *     float64 data, row-major within each block: D is [N][n][n], O is
 *     [N-1][n][n], vectors are [N*n] (block i at offset i*n).  The caller
 *     owns them; the library never frees them and keeps no pointer to D or
 *     O after bt_setup* returns (it copies what it needs).
 *   - Arrays named N, n, d_off, o_off, vec_off, iters, status are HOST
 *     arrays.
 *   - Work is queued on params->stream (a cudaStream_t; NULL = legacy
 *     default stream).  Calls that return device-computed scalars through
 *     host pointers (iters, status) synchronise that stream; the *_async
 *     variants do not.
 *   - Every call returns a bt_status.  On BT_ERR_ARG / BT_ERR_PARAM nothing
 *     was launched.  bt_last_error gives the detail of the last failure.
 *   - A handle is used by one host thread and one stream at a time.
 */
#ifndef BT_H_
#define BT_H_

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  BT_OK = 0,
  BT_ERR_ARG = 1,             /* bad pointer, size or layout                        */
  BT_ERR_PARAM = 2,           /* parameter outside what the method admits (a, m, alpha) */
  BT_ERR_NOT_SPD = 3,         /* a diagonal block D_i failed Cholesky (pivot <= 0)  */
  BT_ERR_NO_CONVERGENCE = 4,  /* maxit (or max_outer) reached; x holds the last iterate */
  BT_ERR_BREAKDOWN = 5,       /* p.q <= 0: S or M^-1 is not positive definite       */
  BT_ERR_NONFINITE = 6,       /* NaN/Inf met in b or during the iteration           */
  BT_ERR_TIMEOUT = 7,         /* the device loop ran past params->cycle_budget      */
  BT_ERR_CUDA = 8,            /* a CUDA runtime call failed                         */
  BT_ERR_ALLOC = 9,           /* device allocation failed                           */
  BT_ERR_STATE = 10           /* call not valid for this handle (e.g. batched vs single) */
} bt_status;

typedef enum {
  BT_FP64 = 0,   /* everything in float64                                            */
  BT_MIXED = 1   /* float32 SpMV/preconditioner inside float64 iterative refinement   */
} bt_precision;

#define BT_MAX_M 8      /* largest polynomial order m accepted                 */
#define BT_MAX_BLOCK 64 /* largest block size n accepted (BT_FP64 handles: n <= 48, the
                           shared-memory pipeline needs two stages of five blocks) */

typedef struct bt_params {
  double a;            /* multi-splitting weight, b = 1 - 2a (Sec. 3.1).  Admissible
                          set C_g (Sec. 3.3): a in [0,1], else BT_ERR_PARAM.  a = 1 is
                          the optimum (Thm. 3.2); a = 0 is block Jacobi, a = 1/2 the
                          stair splittings alone, a = 1/3 equal weights.  a < 1 takes
                          alpha = all ones only (H_ab has negative eigenvalues, where
                          other coefficients can make M^-1 indefinite).  For a < 1
                          and m >= 2 the handle also keeps the +-1 blocks of H_ab
                          (two more block arrays) and H sweeps stream five arrays
                          instead of three; n <= 36 (float64) or 48 (mixed) then,
                          else BT_ERR_ARG from setup.  bt_pcg_solve_multi and
                          bt_pcg_solve_noalloc implement a = 1 only (BT_ERR_PARAM). */
  int m;               /* polynomial order, 1..BT_MAX_M.                           */
  const double* alpha; /* HOST array of m coefficients (Eq. with polynomial
                          coefficients, Sec. 3.5); alpha[0] must be 1 and
                          q(h) = sum_j alpha_j h^j positive on [0, 1] (then M^-1
                          is SPD for every S: the eigenvalues of M^-1 S are
                          q(h)(1-h) over the eigenvalues h in [0, 1) of H_opt);
                          every alpha_j >= 0 qualifies (Thm. 3.3's setting), so
                          do the coefficients of bt_alpha_chebyshev.  Checked
                          exactly (Sturm sequence), else BT_ERR_PARAM.
                          NULL = all ones (the "Optimal" preconditioner).           */
  int precision;       /* bt_precision                                             */
  double tol_inner;    /* BT_MIXED: relative tolerance of each float32 inner solve;
                          0 = sqrt(tol) clamped to [1e-6, 1e-4] (two refinement
                          steps reach tol; 1e-4 at tol = 1e-8); 1e-5 for
                          bt_pcg_solve_multi.                                       */
  int max_outer;       /* BT_MIXED: refinement steps; 0 = 30.                      */
  int use_x0;          /* 1: x holds the initial guess on entry; 0: start from 0.  */
  long long cycle_budget; /* device clock cycles one solve may take before it stops
                          with BT_ERR_TIMEOUT; 0 = 2^34 (about 8 s).                */
  void* stream;        /* cudaStream_t                                             */
  int ctas_per_sm;     /* persistent CTAs per SM; 0 = autotuned/default.           */
  int group_ctas;      /* single-instance solves: CTAs of the persistent kernel that
                          split the block rows (>= 1); 0 = automatic: float64
                          instances whose block arrays fit in the shared memory of
                          one CTA (about 200 KB, e.g. N = 16, n = 6) or of a cluster
                          of 2, 4 or 8 CTAs (e.g. N = 128, n = 12 on 8) run on the
                          shared-memory engine (every block loaded once per solve,
                          halo rows read from the neighbouring CTAs' shared
                          memory), others take a CTA count chosen from N;
                          -1, -2, -4, -8 = the shared-memory engine on a cluster of
                          that many CTAs (BT_ERR_ARG from setup where it does not
                          fit, or leaves a CTA fewer than two block rows).        */
  int stage_kb;        /* shared-memory pipeline stage size in KiB; 0 = default.   */
  int h_matrix_free;   /* 1: apply H_opt = H_J^2 matrix-free, H_J v = -D^-1 (O_{i-1}^T
                          v_{i-1} + O_i v_{i+1}) from the D^-1 and O blocks the handle
                          keeps anyway, two sweeps per application: no Hd, Hu, Hl
                          blocks are formed or stored (3 of 7 block arrays; for
                          problems bound by memory capacity), 4 instead of 3 block
                          reads per application.  a = 1 only; not for
                          bt_pcg_solve_multi or bt_pcg_solve_noalloc (BT_ERR_PARAM). */
  int mrhs_engine;     /* bt_pcg_solve_multi's block products: 0 = automatic (tensor
                          cores where supported: n a multiple of 8, n <= 48; float32
                          SIMT otherwise), 1 = float32 SIMT, 2 = tensor cores (3xTF32
                          split, float32 accumulation; BT_ERR_ARG where unsupported). */
  int mixed_strict_fp64; /* BT_MIXED: 1 = float64 where the mixed method needs it
                          most: every D_i factored (Cholesky, D_i^-1) in float64,
                          then rounded to float32 with the E and H blocks formed
                          from it, and the inner CG step scalars (alpha = rho / p.q,
                          beta = rho' / rho) divided in float64.  0 (default) =
                          float32 factor with a float64 refactor of the blocks
                          whose pivots show cond(D_i) > 1e3, float32 divisions of
                          the step scalars (float64 dot products either way).     */
} bt_params;

typedef struct bt_ctx* bt_handle;

/* Fill *p with the defaults: a = 1, m = 2, alpha = NULL, BT_FP64, everything
 * else 0 (= automatic). */
void bt_params_init(bt_params* p);

/* Check *params against the admissible sets (a, m, alpha, precision and the
 * other fields as documented above) on the host, without touching the GPU:
 * BT_OK, BT_ERR_PARAM, or BT_ERR_ARG for params == NULL.  bt_setup* run the
 * same check. */
bt_status bt_params_check(const bt_params* params);

/* Single instance setup (Sec. 4.1).  Copies D and O into the library's
 * layout, factors every D_i by Cholesky in float64, forms D_i^-1, E_i and
 * (m >= 2) the H blocks, in float64 (BT_FP64) or float32 from the float64
 * Cholesky factor (BT_MIXED).  Returns BT_ERR_NOT_SPD if some D_i is not
 * positive definite (bt_last_error gives the block and the failing pivot).
 * Synchronises params->stream.  N >= 1, 1 <= n <= BT_MAX_BLOCK. */
bt_status bt_setup(int N, int n, const double* D, const double* O,
                   const bt_params* params, bt_handle* out);

/* Recompute every per-block factor of an existing handle (single or batched)
 * from new values of D and O with the same sizes and packing as at setup: the
 * same kernels as bt_setup*, no allocation, queued on the handle's stream
 * without synchronisation (so it can sit inside a timed or captured region).
 * A non-SPD block is reported by the next bt_setup_status call. */
bt_status bt_refactor(bt_handle h, const double* D, const double* O);

/* Synchronise the handle's stream; BT_ERR_NOT_SPD if the last setup or
 * refactor met a diagonal block that is not positive definite, else BT_OK. */
bt_status bt_setup_status(bt_handle h);

/* z = M^-1 r, one application of the preconditioner (Sec. 4.2), in the
 * handle's working precision (float32 blocks for BT_MIXED).  r, z: [N*n]. */
bt_status bt_apply_precond(bt_handle h, const double* r, double* z);

/* y = S x (Eq. 1) with the float64 blocks.  x, y: [N*n]. */
bt_status bt_spmv(bt_handle h, const double* x, double* y);

/* y = S x with the float32 blocks of a BT_MIXED handle (the product the inner
 * solve uses); float64 in and out.  BT_ERR_STATE on a BT_FP64 handle. */
bt_status bt_spmv_f32(bt_handle h, const double* x, double* y);

/* Solve S x = b by PCG (the textbook method the paper cites), stopping when
 * ||r_k||_2 <= tol ||b||_2 on the recursive residual (BT_FP64) or on the
 * float64 true residual b - S x (BT_MIXED).  One persistent kernel keeps the
 * whole iteration on the device.  *iters = number of products S p (float32
 * inner products summed over refinement steps for BT_MIXED).  b == 0 gives
 * x = 0, iters = 0.  Synchronises the stream. */
bt_status bt_pcg_solve(bt_handle h, const double* b, double* x, double tol, int maxit,
                       int* iters);

/* bt_pcg_solve without host synchronisation: the iteration count and status
 * go to the DEVICE ints d_iters[0], d_status[0] (either may be NULL). */
bt_status bt_pcg_solve_async(bt_handle h, const double* b, double* x, double tol, int maxit,
                             int* d_iters, int* d_status);

/* Details of the last bt_pcg_solve / batched solve of instance k (0 for a
 * single instance): refinement steps taken and the final relative residual
 * ||b - S x|| / ||b|| that the device measured (float64 true residual for
 * BT_MIXED; the recursive residual for BT_FP64).  Host outputs. */
bt_status bt_solve_info(bt_handle h, int k, int* outer, double* rel_residual);

/* Many right-hand sides (a BT_MIXED single-instance handle): solve
 * S X = B for nrhs <= 64 columns at once.  The columns run independent PCG
 * recurrences (own alpha, beta, stopping test) that share every block sweep,
 * so each block product becomes an n x n by n x 64 contraction; float32
 * inner solves inside float64 refinement on each column's true residual, as
 * in bt_pcg_solve.  B, X: DEVICE [N*n][nrhs] float64, row-major.  iters and
 * status (HOST arrays of nrhs, may be NULL) receive per-column results; the
 * call returns the first non-OK status.  Requires n % 4 == 0 and n <= 64
 * (else BT_ERR_ARG).  The first call
 * allocates the many-RHS workspace on the handle.  Synchronises the stream. */
bt_status bt_pcg_solve_multi(bt_handle h, const double* B, double* X, int nrhs, double tol,
                             int maxit, int* iters, int* status);

/* Refinement steps and final relative true residual of column j of the last
 * bt_pcg_solve_multi. */
bt_status bt_multi_info(bt_handle h, int j, int* outer, double* rel_residual);

/* Batched setup: B independent instances of sizes N[k] x n[k], packed back
 * to back: instance k's D starts at D + d_off[k], its O at O + o_off[k]
 * (element offsets, HOST arrays).  Same work as bt_setup per instance. */
bt_status bt_setup_batched(int B, const int* N, const int* n, const long long* d_off,
                           const long long* o_off, const double* D, const double* O,
                           const bt_params* params, bt_handle* out);

/* Solve all B instances in one persistent launch: each CTA pulls instances
 * from a device work queue ordered largest first and keeps per-instance
 * convergence state.  Instance k's b and x start at b + vec_off[k] and
 * x + vec_off[k]; vec_off == NULL means packed back to back in instance
 * order.  iters[k], status[k] (HOST arrays of B) receive per-instance
 * results; the call returns the first non-OK status, else BT_OK. */
bt_status bt_pcg_solve_batched(bt_handle h, const double* b, double* x, const long long* vec_off,
                               double tol, int maxit, int* iters, int* status);

/* Same without any host synchronisation or host-side output (suitable for
 * stream capture): per-instance iteration counts and statuses are written to
 * the DEVICE arrays d_iters[B], d_status[B] (either may be NULL).  vec_off
 * is the packing given at bt_setup_batched (back to back). */
bt_status bt_pcg_solve_batched_async(bt_handle h, const double* b, double* x, double tol,
                                     int maxit, int* d_iters, int* d_status);

/* Capture bt_pcg_solve_batched_async(h, b, x, tol, maxit, d_iters, d_status)
 * once into a CUDA graph owned by the handle; bt_graph_launch replays it on
 * the handle's stream.  A new capture replaces the previous one. */
bt_status bt_graph_capture_batched(bt_handle h, const double* b, double* x, double tol,
                                   int maxit, int* d_iters, int* d_status);

/* Capture one whole step of a batched workload -- bt_refactor(h, D, O)
 * followed by bt_pcg_solve_batched_async(h, b, x, tol, maxit, d_iters,
 * d_status) -- into the handle's CUDA graph (replacing any earlier capture).
 * Each bt_graph_launch then re-forms every preconditioner block (Sec. 4.1)
 * from the values D, O hold at that moment and solves all instances, with no
 * host work between the setup kernels and the persistent solve.  D, O, b, x
 * (DEVICE) must keep their addresses and the packing given at setup; a
 * non-SPD block is reported by bt_setup_status after the replay. */
bt_status bt_graph_capture_refactor_solve(bt_handle h, const double* D, const double* O,
                                          const double* b, double* x, double tol, int maxit,
                                          int* d_iters, int* d_status);
bt_status bt_graph_launch(bt_handle h);

/* Adjoint of x = S^-1 b (kernel only): given x and g = S^-1 (dL/dx) for each
 * instance (both packed like b), write dL/dD_i = -g_i x_i^T and
 * dL/dO_i = -(g_i x_{i+1}^T + x_i g_{i+1}^T) into gD, gO (DEVICE, same
 * packing as the D and O given at setup).  The caller obtains g with a second
 * solve on the same handle (S is symmetric). */
bt_status bt_adjoint_blocks(bt_handle h, const double* x, const double* g, double* gD,
                            double* gO);

/* bt_pcg_solve_noalloc -- a solve for callers that cannot allocate device
 * memory (the paper has no counterpart; this is a property of the library).
 * Some callers may not call cudaMalloc: a real-time control loop whose
 * memory is fixed at start-up (cudaMalloc can synchronise the device and has
 * no latency bound), or a plug-in inside a host application that owns the
 * GPU's memory budget.  This entry point runs the same setup kernels and
 * persistent PCG kernel as bt_setup + bt_pcg_solve on one instance, but every
 * buffer they need besides the caller's D, O, b and x (block copies, D_i^-1,
 * E_i, H blocks, work vectors, control words) lives in one static device
 * array of BT_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds
 * until the process exits.  Nothing is allocated and no handle is created.
 *   - Arguments as for bt_setup and bt_pcg_solve (D, O, b, x device float64,
 *     row-major blocks; params as for bt_setup, including params->stream);
 *     *iters (host, may be NULL) receives the iteration count.
 *   - Sizes whose buffers do not fit in the array are rejected with
 *     BT_ERR_ARG before anything runs: for BT_FP64 with m = 2 the limit is
 *     about 56 N n^2 + 88 N n bytes <= 16 MiB (N = 128, n = 32 fits).
 *   - The first call in each CUDA context of a device looks up the array's
 *     device address (with that device current) and keeps it for later calls
 *     in the same context; after cudaDeviceReset, or when the device's primary
 *     context is destroyed and made anew, the module is loaded again and the
 *     next call looks the address up afresh.  The lookup may load the module,
 *     so make a device's first call while no CUDA stream capture is under way
 *     in the process.
 *   - Every call shares the array, which keeps the last call's contents; each
 *     call clears what must start at zero.  Calls that overlap on the GPU race
 *     on the array: issue them one after another.
 *   - Synchronises params->stream; returns the solve status (as bt_pcg_solve)
 *     or BT_ERR_NOT_SPD from the setup. */
#define BT_NOALLOC_SCRATCH_BYTES (16u << 20)
bt_status bt_pcg_solve_noalloc(int N, int n, const double* D, const double* O, const double* b,
                               double* x, double tol, int maxit, const bt_params* params,
                               int* iters);

/* bt_alpha_chebyshev -- polynomial coefficients beyond grid search (the
 * paper's stated future work, Sec. 6), host only: for a bound rho on the
 * spectral radius of H_opt (0 < rho < 1), the alpha[0..m-1] (alpha_0 = 1)
 * that make the eigenvalues q(h)(1-h) of M^-1 S closest to constant over
 * [0, rho] in the minimax sense: p(h) = T_m((2h - rho)/rho) / T_m((2 - rho)/rho)
 * (Chebyshev, p(1) = 1), q(h) = (1 - p(h)) / (1 - h).  The spread of the
 * preconditioned spectrum is then (1 + e)/(1 - e), e = 1/T_m((2 - rho)/rho).
 * m = 2 gives alpha = (1, 1/(1 - rho)).  The coefficients alternate in sign
 * for m >= 3; q stays positive on [0, 1].  A rho below the true spectral
 * radius leaves M^-1 SPD but loses the bound.  BT_ERR_ARG on bad arguments. */
bt_status bt_alpha_chebyshev(int m, double rho, double* alpha);

/* bt_autotune -- choose the persistent kernel's launch shape for this handle
 * by timing its own solves of b (DEVICE, packed as for the solve calls):
 * batched handles try stage sizes of 64, 72 and 80 KiB, single-instance
 * handles two mappings: the shared-memory engine on clusters of 1, 2, 4 and
 * 8 CTAs (where they fit; reported as *group_ctas = -C) and the persistent
 * kernel with 1, N/16, N/8, N/4 and N/2 CTAs per instance (shapes that do
 * not fit are skipped); each candidate
 * runs one untimed and `trials` timed
 * solves (CUDA events on the handle's stream) and the fastest stays
 * configured for later calls (a captured CUDA graph is dropped).  x (DEVICE)
 * holds a solve in the chosen shape on return; *stage_kb and *group_ctas
 * (may be NULL) report the shape.  With the environment variable
 * BT_TUNE_CACHE naming a file, a shape recorded there for the same handle
 * layout (batched or not, variant, precision, m, instance count and sizes,
 * SM count) is configured without timing, and a newly timed one is appended
 * (one JSON object per line).  Synchronises the stream.  Not for the
 * many-RHS engine, which has its own shape. */
bt_status bt_autotune(bt_handle h, const double* b, double* x, double tol, int maxit, int trials, int* stage_kb,
                      int* group_ctas);

/* bt_estimate_rho -- the bound rho that bt_alpha_chebyshev takes, per
 * instance of a handle with a = 1 (stored or matrix-free H): power iteration
 * on H_opt, using that M^-1 S = I - H_opt at m = 1 (Sec. 3.5), i.e.
 *     v <- (v - G_opt (S v)) / || . ||,   rho[k] = ||v - G_opt S v||, ||v|| = 1,
 * `iters` steps from the fixed start vector v_i = 1 + sin(i)/10 (i the element
 * index within the instance), S in float64 and G_opt in the handle's
 * precision.  rho[k] (HOST array of the handle's instance count) approaches
 * rho(H_opt), mostly from below (H_opt is not symmetric, so the norm ratio
 * may also end a little above it); the top eigenvalues of H_opt come in pairs
 * with close neighbours, so convergence is slow (within about 1e-3 after 400
 * steps on the LQR family): add a margin before passing it on.  Three launches per step
 * on the handle's stream, then synchronises.  BT_ERR_PARAM for a < 1. */
bt_status bt_estimate_rho(bt_handle h, int iters, double* rho);

/* bt_set_history -- per-iteration history of later solves on h: hist (DEVICE,
 * [instances][len][3] doubles, owned by the caller, which keeps it alive)
 * receives for PCG iteration k < len of instance i: the relative residual
 * ||r_k|| / ||rhs|| of the PCG run it belongs to (for BT_MIXED the float32
 * inner solve of its refinement step), alpha_k and beta_k (the CG scalars;
 * with them the Lanczos tridiagonal of M^-1 S).  Iterations of successive
 * refinement steps follow one another.  len = 0 turns it off. */
bt_status bt_set_history(bt_handle h, double* hist, int len);

/* bt_ritz_rho -- the bound for bt_alpha_chebyshev from Ritz values (the
 * paper's future work names a spectral estimate): `iters` iterations of PCG
 * on S x = b with M^-1 = G_opt (m = 1, whose M^-1 S = I - H_opt, Sec. 3.5),
 * then per instance rho[k] = 1 - lambda_min(T), T the Lanczos tridiagonal
 * of the CG scalars, its smallest eigenvalue by Sturm bisection on the host.
 * Converges much faster than bt_estimate_rho (extreme Ritz values); for
 * BT_MIXED the scalars come from float32 iterations.  b (DEVICE, packed as
 * for the solves) should excite the whole spectrum (random entries do).
 * a = 1 handles; synchronises. */
bt_status bt_ritz_rho(bt_handle h, const double* b, int iters, double* rho);

/* bt_lqr_schur -- form the systems S lam = gamma of B LQR problems on the
 * device: the construction of the test matrices of Sec. 5 (an LQR problem as
 * an equality-constrained QP, its KKT system, the Schur complement with
 * respect to the Hessian).  Problem k has N[k] knots, state size n[k] and
 * input size m[k] (HOST arrays; 1 <= n[k], m[k] <= 48).  The QP over
 * z = (x_0, u_0, x_1, ..., u_{N-2}, x_{N-1}) is
 *     min 1/2 z^T G z + g^T z  s.t.  x_0 = c_0,  x_{k+1} - A_k x_k - B_k u_k = c_{k+1},
 * G = blkdiag(Q_0, R_0, ..., R_{N-2}, Q_{N-1}), g = (q_0, r_0, ..., q_{N-1}),
 * and with S = C G^-1 C^T, gamma = -(c + C G^-1 g) in blocks:
 *     D_0 = Q_0^-1,  D_k = Q_k^-1 + A_{k-1} Q_{k-1}^-1 A_{k-1}^T + B_{k-1} R_{k-1}^-1 B_{k-1}^T,
 *     O_k = -Q_k^-1 A_k^T.
 * DEVICE inputs, float64, row-major blocks, problems packed back to back:
 *     A [sum (N-1)][n][n], Bm [sum (N-1)][n][m], Q [sum N][n][n] (SPD),
 *     R [sum (N-1)][m][m] (SPD), q [sum N][n], r [sum (N-1)][m], c [sum N][n]
 * (A, Bm, R, r may be NULL when every N[k] = 1).  DEVICE outputs in exactly
 * the layout bt_setup_batched takes: D [sum N][n][n], O [sum (N-1)][n][n]
 * (d_off[k] = sum_{j<k} N_j n_j^2, o_off[k] = sum_{j<k} (N_j-1) n_j^2) and
 * gamma [sum N][n] (vec_off[k] = sum_{j<k} N_j n_j).  Arithmetic in
 * double-float pairs (two float32 numbers with error-free products and sums,
 * about 48 significand bits) on the float32 pipe, inputs split on load and
 * every result rounded once to float64: agrees with a float64 formation to
 * about 1e-13 relative to the block norms at these condition numbers.  One
 * CTA per 16 knots of a problem.  Queued on `stream` (a cudaStream_t),
 * then synchronised: returns BT_ERR_NOT_SPD if some Q_k or R_k has a
 * non-positive Cholesky pivot (*bad_inst, *bad_row name the first one if
 * non-NULL; for R_k the row is k), BT_ERR_ARG on bad sizes or pointers. */
bt_status bt_lqr_schur(int B, const int* N, const int* n, const int* m, const double* A, const double* Bm,
                       const double* Q, const double* R, const double* q, const double* r, const double* c,
                       double* D, double* O, double* gamma, void* stream, int* bad_inst, int* bad_row);

/* bt_lqr_refactor -- bt_lqr_schur fused with the refactor of a handle: forms
 * S and gamma of B LQR problems (the construction above) and writes S
 * straight into h's block arrays (D, O in float64 and float32, the
 * library's column-major slots), then factors every D_k from the float32
 * copy just written (Sec. 4.3's block Cholesky, D_k^-1 = W^T W with
 * W = L^-1; float64 for the blocks the float32 factor refuses, as in
 * bt_refactor) and forms E and the H blocks (Sec. 4.1).  No D or O array
 * passes through device memory in the caller's layout and nothing is copied
 * into the library layout.  h must be a BT_MIXED handle of the optimum (a =
 * 1, stored H blocks, not mixed_strict_fp64) created by bt_setup or
 * bt_setup_batched with the problems' shapes: instance k has N[k] = h's N_k
 * block rows and state size n[k] = h's n_k (<= 48); m (HOST, one entry per
 * instance) gives the input sizes.  A, Bm, Q, R, q, r, c as for
 * bt_lqr_schur (DEVICE); gamma (DEVICE, [sum N][n], h's vector packing)
 * receives the right-hand sides.  Afterwards h holds exactly what
 * bt_refactor of bt_lqr_schur's D and O leaves.  Synchronises h's stream;
 * BT_ERR_NOT_SPD if some Q_k or R_k has a non-positive pivot (*bad_inst,
 * *bad_row as for bt_lqr_schur; h's blocks are then unspecified until the
 * next successful refactor) or some D_k is not SPD (bt_last_error names it),
 * BT_ERR_STATE for a handle of another kind, BT_ERR_ARG on bad sizes or
 * pointers. */
bt_status bt_lqr_refactor(bt_handle h, const int* m, const double* A, const double* Bm, const double* Q,
                          const double* R, const double* q, const double* r, const double* c, double* gamma,
                          int* bad_inst, int* bad_row);

/* bt_lqr_recover_factored -- bt_lqr_recover for the problems of the last
 * successful bt_lqr_refactor on h, from the factors that call formed and h
 * keeps (W = L^-1 of every Q_k and R_k, in double-float pairs): per knot
 *     x_k = -W^T W (q_k + lam_k - A_k^T lam_{k+1}),
 *     u_k = -W_R^T W_R (r_k - B_k^T lam_{k+1}),
 * two triangular products each instead of a Cholesky factorization.  Q and
 * R must be those of that call (they are not read again); m (HOST) must
 * equal its m, else BT_ERR_STATE (also before any bt_lqr_refactor).  A, Bm,
 * q, r, lambda (DEVICE) and the outputs x, u (DEVICE) as for
 * bt_lqr_recover.  Synchronises h's stream. */
bt_status bt_lqr_recover_factored(bt_handle h, const int* m, const double* A, const double* Bm, const double* q,
                                  const double* r, const double* lambda, double* x, double* u);

/* bt_lqr_recover -- the primal solution of the QP above from the solution
 * lam of S lam = gamma: z = -G^-1 (g + C^T lam), i.e.
 *     x_k = -Q_k^-1 (q_k + lam_k - A_k^T lam_{k+1})  (no A term at k = N-1),
 *     u_k = -R_k^-1 (r_k - B_k^T lam_{k+1}),
 * by a float64 Cholesky solve per block.  Inputs as for bt_lqr_schur plus
 * lambda [sum N][n] (DEVICE); outputs x [sum N][n], u [sum (N-1)][m]
 * (DEVICE).  Synchronises `stream`; BT_ERR_NOT_SPD as above. */
bt_status bt_lqr_recover(int B, const int* N, const int* n, const int* m, const double* A, const double* Bm,
                         const double* Q, const double* R, const double* q, const double* r,
                         const double* lambda, double* x, double* u, void* stream);

/* Detail of the last failure on h: instance, block row and a value (the
 * failing Cholesky pivot, or the offending p.q).  Any pointer may be NULL. */
bt_status bt_last_error(bt_handle h, int* instance, int* block, double* value);

/* Bytes of device memory the handle holds. */
long long bt_device_bytes(bt_handle h);

/* Release everything the handle owns.  NULL is ignored. */
void bt_destroy(bt_handle h);

const char* bt_status_string(bt_status s);

#ifdef __cplusplus
}
#endif
#endif /* BT_H_ */
