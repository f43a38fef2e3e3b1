// Internal declarations shared by the translation units of liblyap.so.
//
// Data layout in device memory (all inside the caller's workspace):
//   * SELL-C-sigma copy of each operator: slices of C = 32 rows, column-major
//     inside a slice (entry j of row r of slice k at slice_ptr[k] + 32*j + r),
//     padded entries point at the row itself with value 0.
//   * basis ring: three n x s row-major blocks V[0..2] plus the work block W
//     (only the last 3s basis vectors are kept, Sec. 3.3).
//   * coefficient log: per iteration j a record of LOG_NREC s x s fp64 blocks
//     (the MGS coefficients of both sweeps, the two CholQR2 factors and the
//     three blocks of T_m they define), which is all the second pass needs.
//   * per-CTA partial sums of the s x s reductions (fixed grid, reduced in a
//     fixed order by the last CTA, so every run is bitwise reproducible).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>
#include "lyap.h"

#include <vector>

#define LYAP_SLICE 32
#define LYAP_MAX_S 8

// records in one iteration's log entry (each s*s doubles, row-major)
enum {
  REC_APREV = 0,  // alpha_{j-1}: first MGS sweep against V_{j-1}
  REC_ADIAG,      // alpha_j    : first MGS sweep against V_j
  REC_BPREV,      // second MGS sweep against V_{j-1}
  REC_BDIAG,      // second MGS sweep against V_j
  REC_R1,         // first CholQR factor (upper)
  REC_R2,         // second CholQR factor (upper)
  REC_TNEXT,      // tau_{j+1,j} = R2 R1
  REC_TDIAG,      // tau_{jj}   = alpha_j + beta_j (raw)
  REC_TPREV,      // tau_{j-1,j} = alpha_{j-1} + beta_{j-1} (raw)
  REC_CROSS,      // V_j^T V_{j-1} (rounding-level, used by the fused MGS algebra)
  LOG_NREC
};

// device error bits (OR-ed into a word in the workspace)
enum {
  DERR_BREAKDOWN = 1,
  DERR_NONFINITE = 2,
  DERR_NOTNEGDEF = 4,
  DERR_TIMEOUT = 8,
  DERR_BOUNDS = 16,
  DERR_EIGEN = 32,
};

// One operator (A or B) and its Krylov recurrence state.
struct OpDev {
  int64_t n = 0;
  int64_t nslices = 0;
  int64_t sell_nnz = 0;
  int64_t* slice_ptr = nullptr;  // nslices + 1
  int32_t* slice_w = nullptr;    // nslices
  int32_t* sell_col = nullptr;   // sell_nnz
  void* sell_val = nullptr;      // sell_nnz, fp64 or fp32
  int32_t* perm = nullptr;       // n (SELL row -> original row), nullptr when sigma == 1
  int val_pair = 0;              // SELL values stored as float pairs (float-pair bulk, values not exact in fp32)
  void* V[3] = {nullptr, nullptr, nullptr};
  void* W = nullptr;
  double* C = nullptr;           // fp64 copy of the right-hand side (n x s)
  double* log = nullptr;         // (maxit + 1) * LOG_NREC * s * s; entry 0 = initial QR of C
  double* partials = nullptr;    // sweep_grid * max_nacc
  unsigned int* counter = nullptr;
  double beta = 0.0;             // ||C||_F (host copy after init)
};

struct Plan {
  int s = 1;
  int sylv = 0;
  int n2 = 0;             // size of a small dense B (Sec. 5.2: only A is projected), 0 otherwise
  int bulk = LYAP_PREC_F64;  // bulk number type of the basis: LYAP_PREC_F64, _MIXED (fp32), _F32X2 (pairs)
  int maxit = 1000;
  int sweep_grid = 0;     // CTAs of the reducing sweep of a block Lanczos step (and of the init sweeps)
  int sweep_grid_b = 0;   // CTAs of the sweep writing V_{j+1}
  int check_batch = 32;   // full-size (nmax) slots that fit in the check area (the factor uses one)
  int check_batch_req = 32;  // checks per batch asked for; a batch's slots are sized by its largest m
  int nmax = 0;           // largest reduced dimension s * maxit
  int pass2_blocks = 16;
  int zcap = 0;
  size_t total = 0;
  // byte offsets inside the workspace
  struct OpOff {
    size_t slice_ptr, slice_w, sell_col, sell_val, perm, V[3], W, C, log, partials, counter;
    int64_t n, nslices, sell_nnz;
    int val_pair;
  } op[2];
  size_t hist = 0, flags = 0, chk_err = 0, check = 0, check_bytes = 0, factor = 0, factor_bytes = 0, zstage = 0,
         staging = 0, staging_bytes = 0, smallb = 0, smallb_bytes = 0;
};

// per-check scratch (fp64 unless noted), one slot per check in a batch
struct CheckSlot {
  double* d;     // N
  double* e;     // N
  double* rows;  // 2 s N   (E_1^T P then E_m^T P)
  double* lam;   // N
  double* a;     // N s     (Q^T E_1 gamma)
  double* w;     // N s     (Q^T E_m tau^T)
  double* part;  // N
  double* twk;   // 2 N N   (twisted factorisation pivots, [k][i] layout)
};

size_t check_slot_bytes(int s, int nmax);
int batch_nmax(int s, int m_hi);

// A small dense B of A X + X B + C1 C2^T = 0 (Sec. 5.2): B = P Upsilon P^T computed once
struct SmallB {
  double* P = nullptr;      // n2 x n2, eigenvector j in column j
  double* ups = nullptr;    // n2 eigenvalues, ascending
  double* ctil = nullptr;   // n2 x s: P^T C2
  double* parts = nullptr;  // check_batch x n2 per-row sums of Alg. 5
  int* d_n2 = nullptr;      // n2 on the device (inner dimension of the factor's products)
  double c2norm = 0.0;      // ||C2||_F
};

struct lyap_handle {
  Plan plan;
  SmallB smallb;
  char* ws = nullptr;
  OpDev op[2];
  int s = 1;
  double tol = 1e-8;
  lyap_options opt;
  double* hist = nullptr;       // device, maxit
  int* flags = nullptr;         // device: [0] error bits, [1] first converged m, [2] first m whose check failed
  int* chk_err = nullptr;       // device, maxit: error bits of the check at each m
  char* check_ws = nullptr;
  char* factor_ws = nullptr;
  char* zstage = nullptr;
  int solved = 0;
  int factored = 0;
  int m = 0;                    // iterations of the last solve
  int converged = 0;
  int lanczos_done = 0;         // iterations whose blocks exist
  int checked = 0;              // largest m the last solve checked
  int nchecks = 0;              // checks the last solve evaluated
  int checks_past = 0;          // of those, checks at m past its converged m
  double* hist_host = nullptr;  // pinned copy
  int* flags_host = nullptr;    // pinned
  cudaStream_t side = nullptr;  // second stream (checks)
  cudaEvent_t ev[8];
  float times_ms[8];
  int64_t launches = 0;          // kernels launched since lyap_create
};

// CTAs (or row tiles) of one sweep over one operator: the size of its partials area
constexpr int kMaxSweepGrid = 2048;

// ---- batched solves: per-instance state and row tiles (device resident) --------
struct BInst {
  OpDev op;       // the instance's operator (its log, ring blocks, partials and counter)
  int* flags;     // its error bits
  int* step;      // [0] next iteration j (1-based), [1] 1 while the instance iterates
  int ntiles;     // tiles of this instance in its group's list
  int maxit;
};
struct BTile {
  int inst;       // index into the BInst array
  int local;      // tile index within the instance (its partials slot)
  int64_t lo, hi; // rows [lo, hi), lo a multiple of the SELL slice height
};

// ---- launch helpers implemented in the .cu files --------------------------
// sell.cu
int sell_plan_host(const lyap_csr* A, int sigma, int64_t* nslices, int64_t* sell_nnz);

// step.cu: one block Lanczos step of one operator (two sweeps), its initial block, the second pass
int max_nacc(int s);
int step_supported(int bulk, int s);
void step_blocks_per_sm(int s, int bulk, int pair, int* per_sm_a, int* per_sm_b);
int launch_init_block(OpDev& op, int s, int bulk, int grid, int* d_flags, cudaStream_t st);
int launch_lanczos_step(OpDev& op, int s, int bulk, int grid_a, int grid_b, int j, int* d_flags, cudaStream_t st);
void launch_pass2(OpDev& op, int s, int bulk, int grid, int j, const void* vp, int64_t ldp, const void* vc,
                  int64_t ldc, void* vn, int64_t ldn, cudaStream_t st);
void launch_pass2_v1(OpDev& op, int s, int bulk, int grid, void* vn, int64_t ldn, cudaStream_t st);

// lanczos.cu: the batched sweeps (many instances per launch)
int launch_batch_step(int s, int bulk_f32, const BInst* d_inst, const BTile* d_tiles, int ntiles, int grid,
                      cudaStream_t st);
int batch_blocks_per_sm(int s, int bulk_f32);

// check.cu
int launch_check_batch(lyap_handle* h, int m_lo, int m_hi, cudaStream_t st);
int launch_check_list(lyap_handle* h, const int* ms, int nchk, cudaStream_t st);
int launch_eigen_for_factor(lyap_handle* h, int opi, int m, cudaStream_t st);

// api.cu (used by the batched solver)
lyap_options resolve_options(const lyap_options* opt);
int valid_block(int s);
int validate_csr(const lyap_csr* A);
int create_handle(const lyap_csr* A, const lyap_csr* B, const double* C1, const double* C2, int c_mem, int s,
                  double tol, const lyap_options* opt, void* workspace, size_t ws_bytes, void* stream, int external,
                  lyap_handle** out, int n2 = 0);
int make_plan(const lyap_csr* A, const lyap_csr* B, int s, const lyap_options& o, Plan& p, int external, int n2 = 0);
void solve_begin(lyap_handle* h, cudaStream_t st);
int solve_end(lyap_handle* h, int done, int m_final, int result, cudaStream_t st);
int round_status(lyap_handle* h);
// the m of (from, upto] the check schedule (period or adaptive) evaluates, given the history on
// the host up to m = known
void pick_checks(const lyap_handle* h, int from, int upto, int known, std::vector<int>& out);

// factor.cu
int dense_eigh(double* K, int n, int ld, double* ev, double* V, double* scratch, int* cnt, cudaStream_t st);
size_t factor_ws_bytes(int s, int nmax, int sylv);
size_t pass2_ws_bytes(int64_t n, int s, int kb, int bulk);
int run_factor_basis(lyap_handle* h, const double* basis, int64_t n, double* Z, int64_t ldz, int tcap, int* t_out,
                     cudaStream_t st);
int run_factor(lyap_handle* h, void* Z1, int64_t ldz1, void* Z2, int64_t ldz2, int z_dtype, int tcap, int* t_out,
               cudaStream_t st);

#define LYAP_CUDA_TRY(x)                         \
  do {                                           \
    cudaError_t e_ = (x);                        \
    if (e_ != cudaSuccess) return LYAP_ERR_CUDA; \
  } while (0)

__host__ __device__ inline int64_t lyap_align256(int64_t x) { return (x + 255) & ~int64_t(255); }
