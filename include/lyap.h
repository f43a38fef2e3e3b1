/*
 * lyap.h -- C ABI of the GB300 projection solver for large symmetric Lyapunov
 * and Sylvester equations (Palitta & Simoncini, "Computationally enhanced
 * projection methods for symmetric Sylvester and Lyapunov matrix equations").
 *
 *   Lyapunov : A X + X A + C C^T = 0            (eq. 1.1 with B = A, C1 = C2 = C)
 *   Sylvester: A X + X B + C1 C2^T = 0          (eq. 5.1)
 *
 * A and B are sparse, symmetric negative definite; C1 (n1 x s) and C2 (n2 x s)
 * are tall.  The solution is returned as low-rank factors: X ~= Z Z^T
 * (Lyapunov) or X ~= Z1 Z2^T (Sylvester).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Status: every function returns an int status (lyap_status below) and never
 *    throws or aborts.  lyap_status_string() gives a static description.
 *  - Memory: the library never allocates device memory.  The caller provides one
 *    device workspace of the size lyap_workspace_size() reports; the handle
 *    lives in host memory (malloc) and owns two CUDA streams and a few events.
 *  - Dense blocks (C, V, Z) are row-major: row i of an n x s block holds its s
 *    values contiguously (leading dimension s, or the ld argument).
 *  - Pointers flagged LYAP_MEM_HOST are host memory (pinned or pageable); the
 *    library copies them to or from the workspace inside the call.
 *  - Streams are passed as void* holding a cudaStream_t (NULL = legacy stream).
 *    All work is ordered on the caller's stream, except that lyap_solve runs the
 *    convergence checks of a finished chunk of steps on the handle's second stream
 *    while the next chunk runs on the caller's; it synchronises both before it
 *    returns, once the convergence decision is known on the host.
 *  - Calling order: create -> solve -> (residual_norm)* -> factor -> destroy.
 *    factor may be called once per solve.
 */
#ifndef LYAP_H
#define LYAP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LYAP_OK = 0,
  LYAP_NOT_CONVERGED = 1,  /* maxit reached; history and factor are still valid    */
  LYAP_ERR_ARG = 2,        /* invalid argument, size or calling order              */
  LYAP_ERR_NONFINITE = 3,  /* NaN/Inf met in the data or in a coefficient          */
  LYAP_ERR_BREAKDOWN = 4,  /* CholQR2 pivot <= 0: rank-deficient block (the paper
                              assumes full rank, Sec. 2; deflation not implemented) */
  LYAP_ERR_NOT_NEGDEF = 5, /* lambda_i + lambda_j >= 0 met: A is not negative definite */
  LYAP_ERR_TCAP = 6,       /* the factor needs more than tcap columns              */
  LYAP_ERR_TIMEOUT = 7,    /* a bounded device wait gave up                        */
  LYAP_ERR_CUDA = 8,       /* a CUDA runtime call failed                           */
  LYAP_ERR_WORKSPACE = 9,  /* workspace too small or misaligned (256 B)            */
  LYAP_ERR_EIGEN = 10      /* the eigensolver of T_m did not converge (residual test) */
} lyap_status;

enum { LYAP_F64 = 0, LYAP_F32 = 1 };            /* element types              */
enum { LYAP_MEM_DEVICE = 0, LYAP_MEM_HOST = 1 }; /* where a pointer lives       */
/* bulk number type of the basis, the SpMM and the row arithmetic of a solve */
enum { LYAP_PREC_F64 = 0, LYAP_PREC_MIXED = 1, LYAP_PREC_F32X2 = 2 };

/* lyap_options.check_every: the adaptive check schedule */
enum { LYAP_CHECK_ADAPTIVE = -1 };

/* Sparse matrix in CSR form, read only during lyap_workspace_size and lyap_create.
 * Column indices of each row need not be sorted; the matrix must be symmetric
 * (the method relies on it, Sec. 2) -- symmetry is not checked. */
typedef struct {
  int64_t n;              /* rows = columns                                  */
  int64_t nnz;            /* stored entries                                  */
  const int64_t* rowptr;  /* n + 1 offsets                                   */
  const int32_t* col;     /* nnz column indices in [0, n)                    */
  const void* val;        /* nnz values of type val_dtype                    */
  int val_dtype;          /* LYAP_F64 or LYAP_F32                            */
  int mem;                /* LYAP_MEM_DEVICE or LYAP_MEM_HOST (all 3 arrays) */
} lyap_csr;

typedef struct {
  int maxit;             /* iteration cap (default 1000)                                    */
  int check_every;       /* d: test the residual at every d-th space dimension (Sec. 6);
                            default 1.  LYAP_CHECK_ADAPTIVE: every m <= 8, then every 8th m
                            until the residual trend (a line through log10 of the last 16
                            checked residuals) predicts tol within reach, then every m; when a
                            check meets tol, the m skipped since the last failing check are
                            checked too, and m is the first of them meeting tol.  Skipped
                            entries of the history are NaN                                   */
  double trunc_eps;      /* truncation threshold eps of the reduced solution (eq. 2.5), relative
                            to ||C1||_F ||C2||_F: the discarded eigenvalues (singular values for
                            Sylvester) have a tail of Frobenius norm <= eps ||C1|| ||C2||.
                            0 (default): eps = min(1e-12, tol / (10 (||T_m|| + ||J_m||))), so that
                            the truncation changes the residual by at most tol / 10 (it moves
                            A X + X B by at most (||A|| + ||B||) eps ||C1|| ||C2||; with ||C|| = 1
                            the paper uses 1e-12)                                                */
  int precision;         /* LYAP_PREC_F64: basis, SpMM and factor in fp64.
                            LYAP_PREC_MIXED: basis, SpMM and factor in fp32; per-thread sums in
                            fp32, combined across the GPU as float pairs.
                            LYAP_PREC_F32X2: basis, SpMM, sums and factor in float pairs
                            (hi + lo, about 48 bits) computed on the fp32 pipe; operator values
                            as fp32 when given as LYAP_F32, else as float pairs; block sizes 1-4.
                            In every mode the Cholesky factors, the reduced eigenproblem and the
                            residual are fp64 (default F64)                                    */
  int sell_sigma;        /* SELL-C-sigma sorting window in rows (1 = no sorting; default 1) */
  int pass2_blocks;      /* k: basis blocks buffered per Z update in the second pass
                            (default 16)                                                   */
  int check_batch;       /* most convergence checks evaluated per batch (default 32)        */
  int zcap;              /* columns of Z the workspace can stage for LYAP_MEM_HOST output of
                            lyap_factor (default 0: device output only)                    */
} lyap_options;

typedef struct lyap_handle lyap_handle;

/* Fills *opt with the defaults listed above. */
void lyap_default_options(lyap_options* opt);

/* Bytes of device workspace lyap_create needs for this problem (Alg. 1 storage:
 * 3s basis vectors per operator (Sec. 3.3), the SELL copy of A and B, the
 * coefficient log of T_m up to maxit, and check/factor scratch).  B = NULL for
 * a Lyapunov equation.  Reads the rowptr arrays (copying them if on device). */
int lyap_workspace_size(const lyap_csr* A, const lyap_csr* B, int s,
                        const lyap_options* opt, size_t* bytes);

/* Sets up a solve of A X + X B + C1 C2^T = 0 (Alg. 1 steps 1-2).
 *  A, B      : operators (B = NULL for Lyapunov; then C2 must be NULL too)
 *  C1, C2    : fp64 n1 x s and n2 x s row-major, in c_mem memory
 *  s         : block size, 1 <= s <= 8
 *  tol       : stop at the first m with ||R_m||_F / (||C1||_F ||C2||_F) <= tol
 *  workspace : device memory of ws_bytes >= lyap_workspace_size(), 256-B aligned,
 *              owned by the caller, not touched by anyone else until destroy
 *  stream    : cudaStream_t for the copies and the SELL-C-sigma build
 * The inputs are copied; the caller may free them after the call returns. */
int lyap_create(const lyap_csr* A, const lyap_csr* B, const double* C1,
                const double* C2, int c_mem, int s, double tol,
                const lyap_options* opt, void* workspace, size_t ws_bytes,
                void* stream, lyap_handle** out);

/* Large A, small dense B (Sec. 5.2, Alg. 5): only A is projected.  B = P Upsilon P^T is
 * diagonalised once in lyap_smallb_create; every check then evaluates the residual of the
 * reduced equation T_m Y + Y B + E_1 gamma_1 C2^T = 0 as Alg. 5 does, and lyap_factor returns
 * Z1 = V_m (Q Y1) (n1 x t, by the two-pass device) and Z2 = P Y2 (n2 x t) from the truncation
 * Y~ ~= Y1 Y2^T of the reduced solution in the eigenbases of T_m and B.
 *  B         : fp64 n2 x n2 row-major, symmetric (its symmetric part is used), in c_mem memory
 *  n2        : 1 <= n2 <= s * opt.maxit
 *  C1, C2    : fp64 n1 x s and n2 x s row-major, in c_mem memory
 * Other arguments, ownership and the returned handle are those of lyap_create; lyap_solve,
 * lyap_residual_norm, lyap_projected_matrix (op 0), lyap_factor (Z2 required) and
 * lyap_destroy apply.  The inputs are copied.  LYAP_ERR_NONFINITE if B or C2 holds a NaN or Inf. */
int lyap_smallb_workspace_size(const lyap_csr* A, int n2, int s,
                               const lyap_options* opt, size_t* bytes);
int lyap_smallb_create(const lyap_csr* A, const double* B, int n2, const double* C1,
                       const double* C2, int c_mem, int s, double tol,
                       const lyap_options* opt, void* workspace, size_t ws_bytes,
                       void* stream, lyap_handle** out);

/* Pass 1 (Alg. 1 steps 3-7): block Lanczos (Alg. 2: the block MGS projections and a Cholesky
 * QR normalisation, formed from one reduction per step), the cheap residual norm of Prop. 3.1 / Alg. 3
 * (Alg. 4 for Sylvester) at every check_every-th step, until tol or maxit.
 * Steps run in chunks ahead of their checks: the chunk after the one whose checks
 * find convergence has already been launched, and is discarded, including any sweep
 * error it reports.
 * Returns LYAP_OK, LYAP_NOT_CONVERGED or an error. */
int lyap_solve(lyap_handle* h, void* stream);

/* Relative residual history of the last solve: hist_host[m-1] for m = 1..*m_out
 * (NaN where the check period skipped m).  Writes at most cap entries;
 * *m_out is the final iteration count m.  Host memory. */
int lyap_residual_norm(lyap_handle* h, double* hist_host, int cap, int* m_out);

/* The projected matrix T_m = V_m^T A V_m of the last solve (J_m for op = 1 in a
 * Sylvester solve), built from the logged block Lanczos coefficients (Sec. 2):
 * LAPACK lower band storage ab[d + i*ldab] = T_m[i+d][i], d = 0..s, i = 0..s*m-1,
 * with the symmetric part of tau_jj on the diagonal blocks and tau_{j+1,j} below
 * them; gamma (C = V_1 gamma) and tau_{m+1,m}, both s x s row-major.  Host memory;
 * any pointer may be NULL.  Requires 1 <= m <= the Lanczos steps run by the last
 * solve (also after a solve that returned an error, for diagnosis). */
int lyap_projected_matrix(lyap_handle* h, int op, int m, double* ab, int ldab,
                          double* gamma, double* tau_next);

/* Alg. 1 steps 8-9 with the two-pass device of Sec. 3.3 (4.1 for Sylvester):
 * truncates the reduced solution (eq. 2.5) and accumulates Z = V_m (Q_m Ycheck)
 * while regenerating the basis from the logged coefficients.
 *  Z1, Z2  : n1 x tcap and n2 x tcap row-major (leading dims ldz1, ldz2 >= tcap),
 *            element type z_dtype (LYAP_F64, or LYAP_F32 in mixed precision),
 *            in z_mem memory; columns beyond *t_out are left untouched.
 *            Z2 must be NULL for Lyapunov.  Host output needs opt.zcap >= tcap.
 *  t_out   : the rank t kept by the truncation.
 * Returns LYAP_ERR_TCAP (with *t_out set) if t > tcap. */
int lyap_factor(lyap_handle* h, void* Z1, int64_t ldz1, void* Z2, int64_t ldz2,
                int z_dtype, int z_mem, int tcap, int* t_out, void* stream);

/* Phase timings in milliseconds (CUDA events on the caller's stream):
 * out[0] create, out[1] solve, out[2] factor, out[3] block Lanczos steps run by the
 * last solve (>= m: the iteration runs ahead of the checks by up to check_batch - 1),
 * out[4] convergence checks of the last solve (sum over batches),
 * out[5] block Lanczos sweeps of the last solve (sum over chunks),
 * out[6] number of kernels the library launched since lyap_create,
 * out[7] block Lanczos steps the last solve ran past its converged m (the speculative chunk),
 * out[8] convergence checks it evaluated past that m, out[9] convergence checks it evaluated.
 * The chunk of steps launched ahead of its checks is sized from the residual history known
 * so far: log10 of the residual extrapolated over the last 16 checked m to the steps still
 * needed, times 1.25, between 4 and twice the previous chunk (at most check_batch); the
 * convergence test is unchanged. */
int lyap_phase_times(lyap_handle* h, double* out, int cap);

/* Releases the handle's streams and events and the handle itself.  The caller
 * frees the workspace afterwards. */
int lyap_destroy(lyap_handle* h);

/* Allocation-free evaluation of the relative residual ||R_m||_F / beta^2 for a projected
 * matrix the caller supplies: the residual norm of the Lyapunov equation computed from the
 * eigenvalues and the first and last s rows of the eigenvectors of the block tridiagonal T_m,
 * exactly as the convergence check of lyap_solve does.  The paper has no counterpart: this
 * entry point is an addition of this library.  It runs the kernels of lyap_solve's
 * convergence check, but every byte of their scratch sits in one fixed device array compiled
 * into the library, so the call makes no cudaMalloc, cudaFree or other allocating call.  It
 * is meant for callers that cannot allocate device memory at the point where they need a
 * residual: code running inside another framework whose caching allocator already holds the
 * free device memory (a raw cudaMalloc there fails or fragments that pool), and real-time or
 * embedded loops whose memory is fixed at set-up and may not change afterwards.
 *  ab        : device memory, lower band of T_m, ab[d + i*ldab] = T_m[i+d][i] for
 *              d = 0..s and i < s*m (the layout lyap_projected_matrix returns); ldab >= s+1
 *  gamma     : device memory, s x s row-major, C = V_1 gamma
 *  tau_next  : device memory, s x s row-major, tau_{m+1,m}
 *  beta      : ||C||_F  (> 0)
 *  rel_out   : device memory, receives the relative residual (a double)
 *  status_out: device memory, receives LYAP_OK or the error status of the evaluation (an int)
 *  stream    : cudaStream_t the work is ordered on; the call returns after enqueueing
 * Limits: 1 <= s <= 4 and s*m <= 256; anything larger returns LYAP_ERR_ARG.
 * Set-up: with lazy module loading (the CUDA default), a device gets the library's device
 * code and this array (about 6 MiB) only when the library first runs a kernel there, and
 * that load allocates device memory.  So make the first call on each device at set-up, while
 * memory can still be allocated and before any stream capture; that first call also looks
 * the array's address up (cudaGetSymbolAddress) with the device current.  From then on the
 * array stays held on that device until the process exits, and calls allocate nothing.
 * All calls share the one array and each call clears what must start at zero, so calls
 * whose work overlaps on the GPU (concurrent streams or threads) race and must be
 * serialised. */
int lyap_residual_noalloc(int s, int m, const double* ab, int ldab, const double* gamma,
                          const double* tau_next, double beta, double* rel_out,
                          int* status_out, void* stream);

const char* lyap_status_string(int status);

/* ---- batched solves ------------------------------------------------------------------
 * Many independent Lyapunov equations A_b X + X A_b + C_b C_b^T = 0 (b < count) of uneven
 * size and block size, solved together: every block Lanczos sweep (Alg. 2 with CholQR2) of all
 * instances with the same s is one persistent launch over a list of row tiles of all of them,
 * one iteration of all groups is replayed from a CUDA graph, and the convergence checks
 * (Prop. 3.1, Alg. 3) of the instances run on several streams.  Each instance follows the
 * same method and stopping test as a single lyap_solve; its results (history, m, factor)
 * are read per instance.  The paper treats one equation at a time; the batch is an addition.
 *  A        : count CSR operators (host or device memory, read during lyap_batch_create)
 *  C        : count pointers to n_b x s_b row-major fp64 blocks, memory kind c_mem
 *  s        : count block sizes (1, 2, 3, 4 or 8)
 *  tol      : count tolerances on ||R||_F / ||C||_F^2
 *  opt      : shared options (maxit, precision, check_batch, pass2_blocks; sell_sigma must be 1)
 * The workspace (one caller-owned device buffer, 256-byte aligned) holds every instance's
 * state plus a few shared scratch pools for the checks and the factor; its size comes from
 * lyap_batch_workspace_size with the same arguments. */
typedef struct lyap_batch lyap_batch;

int lyap_batch_workspace_size(int count, const lyap_csr* A, const int* s, const lyap_options* opt,
                              size_t* bytes);
int lyap_batch_create(int count, const lyap_csr* A, const double* const* C, int c_mem, const int* s,
                      const double* tol, const lyap_options* opt, void* workspace, size_t ws_bytes,
                      void* stream, lyap_batch** out);

/* Solves every instance to its tolerance or maxit.  autotune != 0 first times the batched
 * sweeps for each block size over a set of row-tile heights and CTAs per SM (by running
 * iteration 1, which any configuration recomputes identically) and keeps the fastest;
 * otherwise the previous choice, or the default (4096 rows, full occupancy), is used.
 * Returns LYAP_OK when every instance converged, LYAP_NOT_CONVERGED when some reached
 * maxit, or the first error status of an instance (per-instance statuses: lyap_batch_status). */
int lyap_batch_solve(lyap_batch* b, int autotune, void* stream);

/* status[i] and m[i] (iterations) of every instance after lyap_batch_solve (either may be NULL). */
int lyap_batch_status(lyap_batch* b, int* status, int* m);

/* Relative residual history of instance i (as lyap_residual_norm). */
int lyap_batch_residual_norm(lyap_batch* b, int i, double* hist_host, int cap, int* m_out);

/* Low-rank factor of instance i into device memory Z (n_i x tcap row-major, leading dimension
 * ldz >= tcap), as lyap_factor; instances are factored one call at a time. */
int lyap_batch_factor(lyap_batch* b, int i, void* Z, int64_t ldz, int z_dtype, int tcap, int* t_out,
                      void* stream);

/* Chosen sweep configuration per block-size group: out[3g] = s, out[3g+1] = rows per tile,
 * out[3g+2] = CTAs per SM; returns the number of groups written. */
int lyap_batch_tuning(lyap_batch* b, int* out, int cap);

/* out[0] create ms, [1] solve ms, [2] Lanczos sweep ms (graph replays), [3] check ms,
 * [4] instance-iterations run, [5] kernels launched (graph replays count their kernels),
 * [6] graph replays. */
int lyap_batch_phase_times(lyap_batch* b, double* out, int cap);

int lyap_batch_destroy(lyap_batch* b);

/* ---- extended Krylov space with preconditioned inner solves (Sec. 4) --------------------------
 * Galerkin projection onto K_m(A, C) + K_m(A^{-1}, A^{-1} C): blocks of 2s columns, W =
 * [A V_j^(1), A^{-1} V_j^(2)], block Gram-Schmidt against every stored block (twice; Sec. 4's
 * three-term version loses orthogonality quickly in floating point) and CholQR2; T_m by explicit
 * projection; the convergence check is Prop. 3.1 / Alg. 3 with block size 2s.  The paper applies
 * A^{-1} by direct solves; here they are conjugate gradients on M = -A (SPD) to relative
 * residual inner_tol, with one of three preconditioners:
 *   0  Jacobi scaling;
 *   1  IC(0) of M (zero fill, Meijerink and van der Vorst) for a 5-point operator on the nx x ny
 *      grid, factored on the device along the grid's anti-diagonals and applied as
 *      P = B^T B with B = sum_{t=0}^{3} T^t D^{-1}, T = -D^{-1} N (L = D + N), a truncated Neumann
 *      series of L^{-1}: sparse products only, symmetric positive definite by construction;
 *   2  the same application with factor values corrected by a network (three 3x3 convolutions,
 *      5 -> 16 -> 16 -> 3 channels, ReLU, bf16 activations, fp32 accumulation, the 16 -> 16 layer
 *      on the tensor cores): d = d0 exp(y0), lw = lw0 (1 + y1), ls = ls0 (1 + y2) from the
 *      operator's stencil row over its diagonal, trained on the device with Adam on the solve
 *      pairs (b, A^{-1} b) of the method's first inner solves (the first is A^{-1} C), with the
 *      energy-norm loss (1/K) sum_k ||P b_k - x_k||_M^2 / ||x_k||_M^2.  IC(0) judges it: the trained
 *      network is used only when its loss is below IC(0)'s, and a network-preconditioned solve that
 *      needs more than twice the last IC(0) solve's iterations is redone with IC(0).
 *  A : CSR with fp64 values (host or device memory, read during create); s in {1, 2, 4}
 *  C : n x s row-major fp64, memory kind c_mem
 *  nx, ny : grid of the unknowns (x fastest, nx * ny = n) for preconditioners 1 and 2; 0, 0 for
 *           none.  IC(0) needs a 5-point pattern, positive diagonal, positive pivots and nx <= 1024
 *           (lyap_ek_precond_status tells).
 * The basis is stored (n x 2s per iteration, maxit + 1 blocks) and the factor is formed from it. */
typedef struct lyap_ek lyap_ek;

int lyap_ek_workspace_size(const lyap_csr* A, int s, int maxit, int nx, int ny, size_t* bytes);
int lyap_ek_create(const lyap_csr* A, const double* C, int c_mem, int s, double tol, int maxit,
                   double inner_tol, int nx, int ny, void* workspace, size_t ws_bytes, void* stream,
                   lyap_ek** out);
/* 0 when IC(0) exists on the context's grid; otherwise a bit set: 1 an entry outside the
 * 5-point pattern, 2 a non-positive diagonal, 4 a non-positive pivot, 8 nx > 1024; -1 no grid. */
int lyap_ek_precond_status(lyap_ek* e);
/* precond 0 Jacobi, 1 IC(0), 2 the network: the first train_solves inner solves use IC(0) and
 * provide the training pairs (at most 4 columns), then train_iters Adam steps with learning
 * rate lr; LYAP_ERR_ARG when preconditioner 1 or 2 is not available. */
int lyap_ek_solve(lyap_ek* e, int precond, int train_solves, int train_iters, float lr, void* stream);
int lyap_ek_residual_norm(lyap_ek* e, double* hist_host, int cap, int* m_out);
/* Z: device fp64, n x tcap row-major, leading dimension ldz >= tcap */
int lyap_ek_factor(lyap_ek* e, double* Z, int64_t ldz, int tcap, int* t_out, void* stream);
/* out[0] solve ms, [1] training ms, [2] training loss before (IC(0)'s), [3] after, [4] inner
 * solves ns, [5] network-preconditioned solves redone with IC(0), [6] 1 when the trained
 * network was accepted, then the ns iteration counts, then the ns preconditioner kinds. */
int lyap_ek_stats(lyap_ek* e, double* out, int cap);
/* Energy-norm loss and gradient of the network for caller parameters (host floats, length
 * lyap_ek_param_count(); layout w1[16][5][9], b1[16], w2[16][16][9], b2[16], w3[3][16][9],
 * b3[3], tap k = 3 dy + dx reading (x + dx - 1, y + dy - 1)) over K <= 4 device pairs (n x K
 * column-major B and X with A X = B); grad is a host array of the same length.  Overwrites the
 * context's network parameters. */
int lyap_ek_net_grad(lyap_ek* e, const float* params, int K, const double* B, const double* X,
                     double* loss, double* grad, void* stream);
/* Z = P R for K <= 4 device columns (n x K column-major): kind 1 IC(0), kind 2 the network's
 * values (with params, host, when not NULL: then they replace the context's parameters). */
int lyap_ek_precond_apply(lyap_ek* e, int kind, const float* params, int K, const double* R,
                          double* Z, void* stream);
/* The factor values d (diagonal), lw (west), ls (south) of kind 1 or 2 into host arrays of n.
 * A blocking copy: call it once the context's work on its stream has finished. */
int lyap_ek_precond_values(lyap_ek* e, int kind, double* d, double* lw, double* ls);
int lyap_ek_param_count(void);
/* T_m of the extended space (block size 2s) in the band layout of lyap_projected_matrix, with
 * gamma (gamma_1 padded with zero columns) and tau_{m+1,m}; m up to the steps run, also after a
 * solve that stopped with an error.  For tests. */
int lyap_ek_projected_matrix(lyap_ek* e, int m, double* ab, int ldab, double* gamma, double* tau_next);
int lyap_ek_destroy(lyap_ek* e);

/* Generalised Lyapunov equation A X E + E X A + C C^T = 0 with E symmetric positive definite (the
 * example with a mass matrix, Sec. 6).  With E = L L^T it is the standard equation for
 * L^{-1} A L^{-T} and L^{-1} C, solved by Alg. 1-3 without forming L: the block Lanczos basis V
 * is E-orthonormal (the Krylov space of E^{-1} A from E^{-1} C), T_m = V^T A V, and the history
 * is that residual norm relative to ||L^{-1} C||_F^2.  Each step solves with E by Jacobi-
 * preconditioned conjugate gradients to relative residual inner_tol (an E-solve that stops short
 * of it ends the solve with LYAP_ERR_BREAKDOWN) and E-orthogonalises against every stored block
 * twice.  The basis is stored (n x s per iteration, maxit + 1 blocks) and lyap_gen_factor returns
 * Z with X ~= Z Z^T in the original coordinates.
 *  A, E : CSR with fp64 values, same n (host or device memory, read during create); s in {1, 2, 4}
 *  C    : n x s row-major fp64, memory kind c_mem */
typedef struct lyap_gen lyap_gen;

int lyap_gen_workspace_size(const lyap_csr* A, const lyap_csr* E, int s, int maxit, size_t* bytes);
int lyap_gen_create(const lyap_csr* A, const lyap_csr* E, const double* C, int c_mem, int s,
                    double tol, int maxit, double inner_tol, void* workspace, size_t ws_bytes,
                    void* stream, lyap_gen** out);
int lyap_gen_solve(lyap_gen* g, void* stream);
int lyap_gen_residual_norm(lyap_gen* g, double* hist_host, int cap, int* m_out);
/* Z: device fp64, n x tcap row-major, leading dimension ldz >= tcap */
int lyap_gen_factor(lyap_gen* g, double* Z, int64_t ldz, int tcap, int* t_out, void* stream);
/* out[0] solve ms, [1] solves with E, [2] their conjugate-gradient iterations, [3] the most in one */
int lyap_gen_stats(lyap_gen* g, double* out, int cap);
int lyap_gen_destroy(lyap_gen* g);

#ifdef __cplusplus
}
#endif
#endif /* LYAP_H */
