// C ABI of liblyap: workspace planning, set-up, the pass-1 driver (Alg. 1) and the
// factor step.  See include/lyap.h for the contract of every entry point.
#include "common.cuh"

#include <limits.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

size_t factor_ws_bytes(int s, int nmax, int sylv);
size_t pass2_ws_bytes(int64_t n, int s, int kb, int bulk);
int sell_build(const lyap_csr* A, const int64_t* d_rowptr, const int32_t* d_col, const void* d_val, int sigma,
               int bulk, OpDev& op, int* d_flags, cudaStream_t st);

namespace {


// CTAs of the two sweeps of a block Lanczos step: as many as fit on the device at once (one
// wave), at most one per 256 rows.  The reduction order depends on the grid, so results are
// reproducible run to run on a given GPU model.
void sweep_grids_for(int64_t n, int s, int bulk, int pair, int* grid_a, int* grid_b) {
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 152;
  int pa = 1, pb = 1;
  step_blocks_per_sm(s, bulk, pair, &pa, &pb);
  const int64_t byrows = (n + 255) / 256;
  auto clamp = [&](int64_t g) {
    if (g > byrows) g = byrows;
    if (g < 1) g = 1;
    if (g > kMaxSweepGrid) g = kMaxSweepGrid;
    return (int)g;
  };
  *grid_a = clamp((int64_t)sms * pa);
  *grid_b = clamp((int64_t)sms * pb);
}

int valid_s(int s) { return s == 1 || s == 2 || s == 3 || s == 4 || s == 8; }

int check_csr(const lyap_csr* A) {
  if (!A || A->n <= 0 || A->nnz < 0 || !A->rowptr || (A->nnz > 0 && (!A->col || !A->val))) return LYAP_ERR_ARG;
  if (A->val_dtype != LYAP_F64 && A->val_dtype != LYAP_F32) return LYAP_ERR_ARG;
  if (A->mem != LYAP_MEM_DEVICE && A->mem != LYAP_MEM_HOST) return LYAP_ERR_ARG;
  if (A->n > INT_MAX - 64) return LYAP_ERR_ARG;
  return LYAP_OK;
}

lyap_options resolve(const lyap_options* opt) {
  lyap_options o;
  lyap_default_options(&o);
  if (opt) {
    if (opt->maxit > 0) o.maxit = opt->maxit;
    if (opt->check_every > 0 || opt->check_every == LYAP_CHECK_ADAPTIVE) o.check_every = opt->check_every;
    o.trunc_eps = opt->trunc_eps > 0 ? opt->trunc_eps : 0.0;
    o.precision = opt->precision;
    if (opt->sell_sigma > 0) o.sell_sigma = opt->sell_sigma;
    if (opt->pass2_blocks >= 2) o.pass2_blocks = opt->pass2_blocks;
    if (opt->check_batch > 0) o.check_batch = opt->check_batch;
    if (opt->zcap > 0) o.zcap = opt->zcap;
  }
  if (o.check_batch > 256) o.check_batch = 256;
  return o;
}

size_t staging_bytes(const lyap_csr* A) {
  if (!A || A->mem != LYAP_MEM_HOST) return 0;
  const size_t vw = A->val_dtype == LYAP_F64 ? 8 : 4;
  return lyap_align256((int64_t)(sizeof(int64_t) * (A->n + 1))) + lyap_align256((int64_t)(sizeof(int32_t) * A->nnz)) +
         lyap_align256((int64_t)(vw * A->nnz));
}

}  // namespace

lyap_options resolve_options(const lyap_options* opt) { return resolve(opt); }
int valid_block(int s) { return valid_s(s); }
int validate_csr(const lyap_csr* A) { return check_csr(A); }

// external: the check slots, factor scratch and host staging of Z are lent by a caller (a batch)
int make_plan(const lyap_csr* A, const lyap_csr* B, int s, const lyap_options& o, Plan& p, int external, int n2) {
  p.s = s;
  p.sylv = B != nullptr;
  p.n2 = n2;
  p.bulk = o.precision;
  p.maxit = o.maxit;
  p.check_batch = o.check_batch;
  p.check_batch_req = o.check_batch;
  p.nmax = s * o.maxit;
  p.pass2_blocks = o.pass2_blocks;
  p.zcap = o.zcap;
  const size_t w = p.bulk == LYAP_PREC_MIXED ? 4 : 8;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t r = off;
    off += lyap_align256((int64_t)bytes);
    return r;
  };
  int64_t nmaxop = 0;
  for (int k = 0; k < 1 + p.sylv; ++k) {
    const lyap_csr* M = k == 0 ? A : B;
    int64_t nsl = 0, snnz = 0;
    int rc = sell_plan_host(M, o.sell_sigma, &nsl, &snnz);
    if (rc != LYAP_OK) return rc;
    Plan::OpOff& q = p.op[k];
    q.val_pair = p.bulk == LYAP_PREC_F32X2 && M->val_dtype == LYAP_F64;
    const size_t wv = p.bulk == LYAP_PREC_F64 ? 8 : (q.val_pair ? 8 : 4);
    q.n = M->n;
    q.nslices = nsl;
    q.sell_nnz = snnz;
    q.slice_ptr = take(sizeof(int64_t) * (nsl + 1));
    q.slice_w = take(sizeof(int32_t) * nsl);
    q.sell_col = take(sizeof(int32_t) * (size_t)snnz);
    q.sell_val = take(wv * (size_t)snnz);
    q.perm = take(o.sell_sigma > 1 ? sizeof(int32_t) * (size_t)M->n : 0);
    for (int r = 0; r < 3; ++r) q.V[r] = take(w * (size_t)M->n * s);
    q.W = take(w * (size_t)M->n * s);
    q.C = take(sizeof(double) * (size_t)M->n * s);
    q.log = take(sizeof(double) * (size_t)(o.maxit + 1) * LOG_NREC * s * s);
    q.partials = take(sizeof(double) * (size_t)kMaxSweepGrid * max_nacc(s));
    q.counter = take(256);
    nmaxop = std::max<int64_t>(nmaxop, M->n);
  }
  p.sweep_grid = 0;  // set at create (needs the device)
  p.hist = take(sizeof(double) * (size_t)o.maxit);
  p.flags = take(256);
  p.chk_err = take(sizeof(int) * (size_t)o.maxit);
  // the check slots hold per-eigenpair fp64 scratch (O(nmax^2) each): cap their total at 16 GiB
  if (external) {
    p.check_batch = 1;
    p.check_bytes = 0;
    p.factor_bytes = factor_ws_bytes(s, p.nmax, p.sylv);  // lent: the pass-2 buffers follow it
    p.staging_bytes = staging_bytes(A) + staging_bytes(B);
    p.staging = take(p.staging_bytes);
    p.total = off;
    return LYAP_OK;
  }
  {
    const size_t per = (size_t)(1 + p.sylv) * check_slot_bytes(s, p.nmax);
    const size_t cap = (size_t)16 << 30;
    if ((size_t)p.check_batch * per > cap) p.check_batch = (int)std::max<size_t>(1, cap / per);
  }
  p.check_bytes = (size_t)(1 + p.sylv) * p.check_batch * check_slot_bytes(s, p.nmax);
  p.check = take(p.check_bytes);
  // the small-B factor works on a stacked kernel of N + n2 <= 2 nmax rows, as the two-sided one
  p.factor_bytes = factor_ws_bytes(s, p.nmax, p.sylv || n2 > 0);
  size_t p2 = 0;
  for (int k = 0; k < 1 + p.sylv; ++k) p2 += pass2_ws_bytes(p.op[k].n, s, o.pass2_blocks, p.bulk);
  p.factor = take(p.factor_bytes + p2);
  p.zstage = take(o.zcap > 0 ? sizeof(double) * (size_t)o.zcap * (A->n + (B ? B->n : n2)) : 0);
  p.staging_bytes = staging_bytes(A) + staging_bytes(B);
  p.staging = take(p.staging_bytes);
  if (n2 > 0) {
    // B copy (then its reflectors), P, upsilon, P^T C2, C2, Alg. 5 row sums, eigen scratch, ints
    const size_t nn = (size_t)n2 * n2;
    p.smallb_bytes = lyap_align256((int64_t)(sizeof(double) * nn)) * 2 + lyap_align256((int64_t)(sizeof(double) * n2)) +
                     2 * lyap_align256((int64_t)(sizeof(double) * (size_t)n2 * s)) +
                     lyap_align256((int64_t)(sizeof(double) * (size_t)o.check_batch * n2)) +
                     lyap_align256((int64_t)(sizeof(double) * (4 * (size_t)n2 + 3 * nn))) + 256;
    p.smallb = take(p.smallb_bytes);
  }
  p.total = off;
  return LYAP_OK;
}

namespace {

template <typename T>
T* at(char* ws, size_t off) {
  return reinterpret_cast<T*>(ws + off);
}

__global__ void k_init_flags(int* flags, double* hist, int* chk_err, int maxit) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    flags[0] = 0;
    flags[1] = INT_MAX;
    flags[2] = INT_MAX;
  }
  if (i < maxit) {
    hist[i] = __longlong_as_double(0x7ff8000000000000LL);
    chk_err[i] = 0;
  }
}

int status_from_bits(int bits) {
  // root causes first: a breakdown leaves a degenerate block whose later use may overflow
  if (bits & DERR_BOUNDS) return LYAP_ERR_ARG;
  if (bits & DERR_BREAKDOWN) return LYAP_ERR_BREAKDOWN;
  if (bits & DERR_NONFINITE) return LYAP_ERR_NONFINITE;
  if (bits & DERR_NOTNEGDEF) return LYAP_ERR_NOT_NEGDEF;
  if (bits & DERR_TIMEOUT) return LYAP_ERR_TIMEOUT;
  if (bits & DERR_EIGEN) return LYAP_ERR_EIGEN;
  return LYAP_OK;
}

}  // namespace

extern "C" {

void lyap_default_options(lyap_options* opt) {
  if (!opt) return;
  opt->maxit = 1000;
  opt->check_every = 1;
  opt->trunc_eps = 0.0;
  opt->precision = LYAP_PREC_F64;
  opt->sell_sigma = 1;
  opt->pass2_blocks = 16;
  opt->check_batch = 32;
  opt->zcap = 0;
}

const char* lyap_status_string(int status) {
  switch (status) {
    case LYAP_OK: return "ok";
    case LYAP_NOT_CONVERGED: return "not converged within maxit";
    case LYAP_ERR_ARG: return "invalid argument or calling order";
    case LYAP_ERR_NONFINITE: return "non-finite value in data or coefficients";
    case LYAP_ERR_BREAKDOWN: return "CholQR2 breakdown: rank-deficient block";
    case LYAP_ERR_NOT_NEGDEF: return "operator is not negative definite";
    case LYAP_ERR_TCAP: return "factor rank exceeds tcap";
    case LYAP_ERR_TIMEOUT: return "bounded device wait expired";
    case LYAP_ERR_CUDA: return "CUDA runtime error";
    case LYAP_ERR_WORKSPACE: return "workspace too small or misaligned";
    case LYAP_ERR_EIGEN: return "reduced eigensolver did not converge";
    default: return "unknown status";
  }
}

int lyap_workspace_size(const lyap_csr* A, const lyap_csr* B, int s, const lyap_options* opt, size_t* bytes) {
  if (!bytes || !valid_s(s)) return LYAP_ERR_ARG;
  int rc = check_csr(A);
  if (rc != LYAP_OK) return rc;
  if (B && (rc = check_csr(B)) != LYAP_OK) return rc;
  lyap_options o = resolve(opt);
  if (o.precision != LYAP_PREC_F64 && o.precision != LYAP_PREC_MIXED && o.precision != LYAP_PREC_F32X2)
    return LYAP_ERR_ARG;
  if (!step_supported(o.precision, s)) return LYAP_ERR_ARG;
  Plan p;
  rc = make_plan(A, B, s, o, p, 0);
  if (rc != LYAP_OK) return rc;
  *bytes = p.total;
  return LYAP_OK;
}

}  // extern "C"

// lyap_create's work; external = 1 leaves the check, factor and Z staging areas to the caller
int create_handle(const lyap_csr* A, const lyap_csr* B, const double* C1, const double* C2, int c_mem, int s,
                  double tol, const lyap_options* opt, void* workspace, size_t ws_bytes, void* stream, int external,
                  lyap_handle** out, int n2) {
  if (!out || !valid_s(s) || !C1 || !(tol >= 0.0)) return LYAP_ERR_ARG;
  if (n2 == 0 && (B == nullptr) != (C2 == nullptr)) return LYAP_ERR_ARG;
  if (c_mem != LYAP_MEM_DEVICE && c_mem != LYAP_MEM_HOST) return LYAP_ERR_ARG;
  int rc = check_csr(A);
  if (rc != LYAP_OK) return rc;
  if (B && (rc = check_csr(B)) != LYAP_OK) return rc;
  lyap_options o = resolve(opt);
  if (o.precision != LYAP_PREC_F64 && o.precision != LYAP_PREC_MIXED && o.precision != LYAP_PREC_F32X2)
    return LYAP_ERR_ARG;
  if (!step_supported(o.precision, s)) return LYAP_ERR_ARG;
  Plan p;
  rc = make_plan(A, B, s, o, p, external, n2);
  if (rc != LYAP_OK) return rc;
  if (!workspace || ws_bytes < p.total || (reinterpret_cast<uintptr_t>(workspace) & 255)) return LYAP_ERR_WORKSPACE;
  *out = nullptr;
  lyap_handle* h = new (std::nothrow) lyap_handle();
  if (!h) return LYAP_ERR_ARG;
  sweep_grids_for(std::max(A->n, B ? B->n : (int64_t)0), s, p.bulk, p.op[0].val_pair || (p.sylv && p.op[1].val_pair),
                  &p.sweep_grid, &p.sweep_grid_b);
  h->plan = p;
  h->ws = static_cast<char*>(workspace);
  h->s = s;
  h->tol = tol;
  h->opt = o;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  for (int i = 0; i < 8; ++i) h->ev[i] = nullptr;
  auto fail = [&](int code) {
    lyap_destroy(h);
    return code;
  };
  if (cudaEventCreate(&h->ev[0]) != cudaSuccess || cudaEventCreate(&h->ev[1]) != cudaSuccess) return fail(LYAP_ERR_CUDA);
  cudaEventRecord(h->ev[0], st);
  if (cudaMallocHost(&h->hist_host, sizeof(double) * o.maxit) != cudaSuccess) return fail(LYAP_ERR_CUDA);
  if (cudaMallocHost(&h->flags_host, sizeof(int) * 8) != cudaSuccess) return fail(LYAP_ERR_CUDA);
  h->hist = at<double>(h->ws, p.hist);
  h->flags = at<int>(h->ws, p.flags);
  h->chk_err = at<int>(h->ws, p.chk_err);
  h->check_ws = h->ws + p.check;
  h->factor_ws = h->ws + p.factor;
  h->zstage = h->ws + p.zstage;
  k_init_flags<<<(o.maxit + 255) / 256, 256, 0, st>>>(h->flags, h->hist, h->chk_err, o.maxit);
  h->launches = 1;
  char* stage = h->ws + p.staging;
  for (int k = 0; k < 1 + p.sylv; ++k) {
    const lyap_csr* M = k == 0 ? A : B;
    const double* Ck = k == 0 ? C1 : C2;
    OpDev& op = h->op[k];
    const Plan::OpOff& q = p.op[k];
    op.n = q.n;
    op.nslices = q.nslices;
    op.sell_nnz = q.sell_nnz;
    op.slice_ptr = at<int64_t>(h->ws, q.slice_ptr);
    op.slice_w = at<int32_t>(h->ws, q.slice_w);
    op.sell_col = at<int32_t>(h->ws, q.sell_col);
    op.sell_val = h->ws + q.sell_val;
    op.perm = o.sell_sigma > 1 ? at<int32_t>(h->ws, q.perm) : nullptr;
    op.val_pair = q.val_pair;
    for (int r = 0; r < 3; ++r) op.V[r] = h->ws + q.V[r];
    op.W = h->ws + q.W;
    op.C = at<double>(h->ws, q.C);
    op.log = at<double>(h->ws, q.log);
    op.partials = at<double>(h->ws, q.partials);
    op.counter = at<unsigned int>(h->ws, q.counter);
    if (cudaMemsetAsync(op.counter, 0, 256, st) != cudaSuccess) return fail(LYAP_ERR_CUDA);
    const int64_t* rp = M->rowptr;
    const int32_t* cl = M->col;
    const void* vl = M->val;
    if (M->mem == LYAP_MEM_HOST) {
      const size_t vw = M->val_dtype == LYAP_F64 ? 8 : 4;
      int64_t* drp = reinterpret_cast<int64_t*>(stage);
      stage += lyap_align256((int64_t)(sizeof(int64_t) * (M->n + 1)));
      int32_t* dcl = reinterpret_cast<int32_t*>(stage);
      stage += lyap_align256((int64_t)(sizeof(int32_t) * M->nnz));
      void* dvl = stage;
      stage += lyap_align256((int64_t)(vw * M->nnz));
      if (cudaMemcpyAsync(drp, rp, sizeof(int64_t) * (M->n + 1), cudaMemcpyHostToDevice, st) != cudaSuccess ||
          cudaMemcpyAsync(dcl, cl, sizeof(int32_t) * M->nnz, cudaMemcpyHostToDevice, st) != cudaSuccess ||
          cudaMemcpyAsync(dvl, vl, vw * M->nnz, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return fail(LYAP_ERR_CUDA);
      rp = drp;
      cl = dcl;
      vl = dvl;
    }
    rc = sell_build(M, rp, cl, vl, o.sell_sigma, p.bulk, op, h->flags, st);
    if (rc != LYAP_OK) return fail(rc);
    h->launches += 1;
    const cudaMemcpyKind kind = c_mem == LYAP_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    if (cudaMemcpyAsync(op.C, Ck, sizeof(double) * (size_t)op.n * s, kind, st) != cudaSuccess)
      return fail(LYAP_ERR_CUDA);
  }
  if (cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking) != cudaSuccess) return fail(LYAP_ERR_CUDA);
  for (int i = 2; i < 8; ++i)
    if (cudaEventCreate(&h->ev[i]) != cudaSuccess) return fail(LYAP_ERR_CUDA);
  cudaEventRecord(h->ev[1], st);
  if (cudaStreamSynchronize(st) != cudaSuccess) return fail(LYAP_ERR_CUDA);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, h->ev[0], h->ev[1]);
  for (int i = 0; i < 8; ++i) h->times_ms[i] = 0.f;
  h->times_ms[0] = ms;
  if (cudaMemcpy(h->flags_host, h->flags, sizeof(int) * 2, cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(LYAP_ERR_CUDA);
  rc = status_from_bits(h->flags_host[0]);
  if (rc != LYAP_OK) return fail(rc);
  *out = h;
  return LYAP_OK;
}

// resets the history and flags and builds V_1 (CholQR2 of C) for every operator
void solve_begin(lyap_handle* h, cudaStream_t st) {
  const Plan& p = h->plan;
  k_init_flags<<<(p.maxit + 255) / 256, 256, 0, st>>>(h->flags, h->hist, h->chk_err, p.maxit);
  h->launches += 1;
  for (int k = 0; k < 1 + p.sylv; ++k)
    h->launches += launch_init_block(h->op[k], h->s, p.bulk, p.sweep_grid, h->flags, st);
}

// records the outcome of a solve (m, convergence, iterations run), copies the history to
// the host and reads beta for the factor; records ev[1] and synchronises the stream
int solve_end(lyap_handle* h, int done, int m_final, int result, cudaStream_t st) {
  const Plan& p = h->plan;
  h->m = m_final;
  h->converged = result == LYAP_OK;
  h->lanczos_done = done;
  h->solved = 1;
  h->factored = 0;
  h->op[0].beta = 0.0;
  LYAP_CUDA_TRY(cudaMemcpyAsync(h->hist_host, h->hist, sizeof(double) * p.maxit, cudaMemcpyDeviceToHost, st));
  double betas[2] = {0.0, 0.0};
  for (int k = 0; k < 1 + p.sylv; ++k)
    LYAP_CUDA_TRY(
        cudaMemcpyAsync(&betas[k], h->op[k].log + REC_TDIAG * h->s * h->s, sizeof(double), cudaMemcpyDeviceToHost, st));
  cudaEventRecord(h->ev[1], st);
  LYAP_CUDA_TRY(cudaStreamSynchronize(st));
  for (int k = 0; k < 1 + p.sylv; ++k) h->op[k].beta = betas[k];
  return LYAP_OK;
}

// status of a check round: error bits, or the first failed check before the first converged m
int round_status(lyap_handle* h) {
  int rc = status_from_bits(h->flags_host[0]);
  if (rc == LYAP_OK && h->flags_host[2] < h->flags_host[1]) {
    int eb = 0;
    LYAP_CUDA_TRY(cudaMemcpy(&eb, h->chk_err + h->flags_host[2] - 1, sizeof(int), cudaMemcpyDeviceToHost));
    rc = status_from_bits(eb);
    if (rc == LYAP_OK) rc = LYAP_ERR_EIGEN;
  }
  return rc;
}

// Predicted first m with a residual <= tol: least-squares line through log10 of the last 16
// residuals on record (m <= known; skipped m are NaN), extrapolated to log10(tol).  Returns
// false without a prediction (fewer than 4 values, a slope >= 0, or tol <= 0).
bool predict_converged_m(const double* hist, int known, double tol, double* m_star) {
  int n = 0;
  double sx = 0, sy = 0, sxx = 0, sxy = 0;
  for (int m = known; m >= 1 && n < 16; --m) {
    const double v = hist[m - 1];
    if (!(v > 0.0) || !isfinite(v)) continue;
    const double y = log10(v);
    sx += m;
    sy += y;
    sxx += (double)m * m;
    sxy += m * y;
    ++n;
  }
  if (n < 4 || !(tol > 0.0)) return false;
  const double den = n * sxx - sx * sx;
  const double slope = den != 0.0 ? (n * sxy - sx * sy) / den : 0.0;
  if (!(slope < 0.0)) return false;
  const double icpt = (sy - slope * sx) / n;
  *m_star = (log10(tol) - icpt) / slope;
  return isfinite(*m_star);
}

// Size of the next chunk of block Lanczos steps (launched ahead of its checks).  The steps of a
// chunk run while the checks of the previous one are evaluated; the checks that find convergence
// leave the chunk after it discarded.  From the history known on the host, the number of steps
// still needed beyond those already launched is predicted (above); the next chunk covers 1.25
// times that, between 4 steps and min(2 x the previous chunk, the check batch).  The chunk size
// does not change the convergence test: the first checked m with rel <= tol is the result.
int next_chunk(const double* hist, int known, int launched, int prev, int cap, double tol) {
  const int hi_cap = std::min(2 * prev, cap);
  const int lo_cap = std::min(4, hi_cap);
  double m_star = 0.0;
  if (!predict_converged_m(hist, known, tol, &m_star)) return hi_cap;
  const double need = 1.25 * (m_star - launched);
  if (!(need < hi_cap)) return hi_cap;
  return std::max(lo_cap, (int)ceil(need));
}

// The m of (from, upto] whose residual is evaluated.  A period d >= 1 takes the multiples of d
// (Sec. 6).  The adaptive schedule takes every m <= kDenseHead, every kSparseStride-th m after
// that, and every m from the predicted first converged m minus a margin on: the margin is 2 plus
// a quarter of the distance the prediction extrapolates over, so a prediction made from far away
// opens the dense window early.  Checks skipped before the first converged one are evaluated
// afterwards.  (A stride growing with m measured slower on the batched workload: the checks it
// saves are outweighed by the longer stretches a late window leaves to that catch-up.)
constexpr int kDenseHead = 8;
constexpr int kSparseStride = 8;
void pick_checks(const lyap_handle* h, int from, int upto, int known, std::vector<int>& out) {
  out.clear();
  const int d = h->opt.check_every;
  if (d >= 1) {
    for (int m = from + 1; m <= upto; ++m)
      if (m % d == 0) out.push_back(m);
    return;
  }
  double m_star = 0.0;
  const bool pred = predict_converged_m(h->hist_host, known, h->tol, &m_star);
  const double dense_from = pred ? m_star - (2.0 + 0.25 * std::max(0.0, m_star - known)) : 1e300;
  for (int m = from + 1; m <= upto; ++m)
    if (m <= kDenseHead || m % kSparseStride == 0 || (double)m >= dense_from) out.push_back(m);
}

extern "C" {

int lyap_create(const lyap_csr* A, const lyap_csr* B, const double* C1, const double* C2, int c_mem, int s,
                double tol, const lyap_options* opt, void* workspace, size_t ws_bytes, void* stream,
                lyap_handle** out) {
  return create_handle(A, B, C1, C2, c_mem, s, tol, opt, workspace, ws_bytes, stream, 0, out);
}

int lyap_smallb_workspace_size(const lyap_csr* A, int n2, int s, const lyap_options* opt, size_t* bytes) {
  if (!bytes || !valid_s(s) || n2 < 1) return LYAP_ERR_ARG;
  int rc = check_csr(A);
  if (rc != LYAP_OK) return rc;
  lyap_options o = resolve(opt);
  if (o.precision != LYAP_PREC_F64 && o.precision != LYAP_PREC_MIXED && o.precision != LYAP_PREC_F32X2)
    return LYAP_ERR_ARG;
  if (!step_supported(o.precision, s) || n2 > s * o.maxit) return LYAP_ERR_ARG;
  Plan p;
  rc = make_plan(A, nullptr, s, o, p, 0, n2);
  if (rc != LYAP_OK) return rc;
  *bytes = p.total;
  return LYAP_OK;
}

}  // extern "C"

namespace {

// B <- (B + B^T) / 2 in place (n2 x n2 row-major); *bad set if an entry is not finite
__global__ void k_symmetrize(double* B, int n2, int* bad) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n2 * n2) return;
  if (!isfinite(B[idx])) atomicOr(bad, 1);
  const int r = (int)(idx / n2), c = (int)(idx % n2);
  if (r >= c) return;
  const double v = 0.5 * (B[(size_t)r * n2 + c] + B[(size_t)c * n2 + r]);
  B[(size_t)r * n2 + c] = v;
  B[(size_t)c * n2 + r] = v;
}

// ct = P^T C2 (n2 x s); column i of P is the eigenvector of upsilon_i
__global__ void k_ptc(const double* __restrict__ P, const double* __restrict__ C2, int n2, int s,
                      double* __restrict__ ct) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n2) return;
  for (int c = 0; c < s; ++c) {
    double acc = 0.0;
    for (int r = 0; r < n2; ++r) acc = fma(P[(size_t)r * n2 + i], C2[(size_t)r * s + c], acc);
    ct[(size_t)i * s + c] = acc;
  }
}

}  // namespace

extern "C" {

int lyap_smallb_create(const lyap_csr* A, const double* B, int n2, const double* C1, const double* C2, int c_mem,
                       int s, double tol, const lyap_options* opt, void* workspace, size_t ws_bytes, void* stream,
                       lyap_handle** out) {
  if (!out || !B || !C2 || n2 < 1) return LYAP_ERR_ARG;
  if (c_mem != LYAP_MEM_DEVICE && c_mem != LYAP_MEM_HOST) return LYAP_ERR_ARG;
  lyap_options o = resolve(opt);
  if (n2 > s * o.maxit) return LYAP_ERR_ARG;
  int rc = create_handle(A, nullptr, C1, nullptr, c_mem, s, tol, opt, workspace, ws_bytes, stream, 0, out, n2);
  if (rc != LYAP_OK) return rc;
  lyap_handle* h = *out;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  auto fail = [&](int code) {
    lyap_destroy(h);
    *out = nullptr;
    return code;
  };
  const size_t nn = (size_t)n2 * n2;
  char* p = h->ws + h->plan.smallb;
  auto take = [&](size_t bytes) { char* r = p; p += lyap_align256((int64_t)bytes); return r; };
  double* Bk = (double*)take(sizeof(double) * nn);
  SmallB& sb = h->smallb;
  sb.P = (double*)take(sizeof(double) * nn);
  sb.ups = (double*)take(sizeof(double) * n2);
  sb.ctil = (double*)take(sizeof(double) * (size_t)n2 * s);
  double* C2d = (double*)take(sizeof(double) * (size_t)n2 * s);
  sb.parts = (double*)take(sizeof(double) * (size_t)h->opt.check_batch * n2);
  double* scratch = (double*)take(sizeof(double) * (4 * (size_t)n2 + 3 * nn));
  int* ints = (int*)take(256);
  sb.d_n2 = ints;
  const cudaMemcpyKind kind = c_mem == LYAP_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  if (cudaMemcpyAsync(Bk, B, sizeof(double) * nn, kind, st) != cudaSuccess ||
      cudaMemcpyAsync(C2d, C2, sizeof(double) * (size_t)n2 * s, kind, st) != cudaSuccess ||
      cudaMemcpyAsync(sb.d_n2, &n2, sizeof(int), cudaMemcpyHostToDevice, st) != cudaSuccess)
    return fail(LYAP_ERR_CUDA);
  if (cudaMemsetAsync(ints + 2, 0, sizeof(int), st) != cudaSuccess) return fail(LYAP_ERR_CUDA);
  k_symmetrize<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(Bk, n2, ints + 2);
  int bad = 0;
  if (cudaMemcpyAsync(&bad, ints + 2, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return fail(LYAP_ERR_CUDA);
  if (bad) return fail(LYAP_ERR_NONFINITE);
  // B = P Upsilon P^T, once (the reduced equations of every m share it)
  rc = dense_eigh(Bk, n2, n2, sb.ups, sb.P, scratch, ints + 1, st);
  if (rc != LYAP_OK) return fail(rc);
  k_ptc<<<(n2 + 127) / 128, 128, 0, st>>>(sb.P, C2d, n2, s, sb.ctil);
  h->launches += 5;
  std::vector<double> c2h((size_t)n2 * s);
  if (cudaMemcpyAsync(c2h.data(), C2d, sizeof(double) * c2h.size(), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return fail(LYAP_ERR_CUDA);
  double nrm = 0.0;
  for (double v : c2h) nrm += v * v;
  sb.c2norm = sqrt(nrm);
  if (!(sb.c2norm > 0.0) || !std::isfinite(sb.c2norm)) return fail(LYAP_ERR_NONFINITE);
  return cudaGetLastError() == cudaSuccess ? LYAP_OK : fail(LYAP_ERR_CUDA);
}

int lyap_solve(lyap_handle* h, void* stream) {
  if (!h) return LYAP_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaStream_t sd = h->side;
  const Plan& p = h->plan;
  const int s = h->s;
  cudaEventRecord(h->ev[0], st);
  solve_begin(h, st);
  // Lanczos chunks run on the caller's stream and the checks of a finished chunk on the side
  // stream, so chunk c+1 (speculative: the checks of chunk c may find convergence) overlaps the
  // checks of chunk c.  Step j writes only log record j and the checks of chunk c read records
  // up to its last step, so the two never touch the same data.  Each chunk reports sweep errors
  // in its own word (two words, alternating), so an error in a speculative chunk past the
  // converged m does not fail the solve.
  int* cw = h->flags + 8;
  LYAP_CUDA_TRY(cudaMemsetAsync(cw, 0, 2 * sizeof(int), st));
  cudaEvent_t c_beg[2] = {h->ev[2], h->ev[6]}, c_end[2] = {h->ev[3], h->ev[7]};
  auto launch_chunk = [&](int from, int upto, int c) {
    int* fw = cw + (c & 1);
    cudaEventRecord(c_beg[c & 1], st);
    for (int k = 0; k < 1 + p.sylv; ++k)
      for (int j = from + 1; j <= upto; ++j)
        h->launches += launch_lanczos_step(h->op[k], s, p.bulk, p.sweep_grid, p.sweep_grid_b, j, fw, st);
    cudaEventRecord(c_end[c & 1], st);
  };
  // checks in batches: as many as fit in the check area with slots sized by the batch's largest m
  std::vector<int> todo;
  std::vector<unsigned char> was_checked((size_t)p.maxit + 1, 0);
  int nchecks = 0;
  auto launch_checks = [&](const std::vector<int>& ms) {
    size_t i = 0;
    while (i < ms.size()) {
      size_t n = std::min(ms.size() - i, (size_t)p.check_batch_req);
      while (n > 1 && (size_t)(1 + p.sylv) * n * check_slot_bytes(s, batch_nmax(s, ms[i + n - 1])) > p.check_bytes)
        --n;
      h->launches += launch_check_list(h, ms.data() + i, (int)n, sd);
      for (size_t k = i; k < i + n; ++k) was_checked[ms[k]] = 1;
      i += n;
    }
    nchecks += (int)ms.size();
  };
  int chunk = std::min(4, p.check_batch_req);
  int done = std::min(p.maxit, chunk);  // last step of the chunk being checked
  int checked = 0;                      // largest m already checked
  int known = 0;                        // largest m whose history value is on the host
  int c = 0;                            // index of the chunk being checked
  int result = LYAP_NOT_CONVERGED;
  int m_final = p.maxit;
  float t_lanczos = 0.f, t_check = 0.f;
  launch_chunk(0, done, 0);
  int rc = LYAP_OK;
  while (true) {
    LYAP_CUDA_TRY(cudaStreamWaitEvent(sd, c_end[c & 1], 0));
    cudaEventRecord(h->ev[5], sd);
    const int first_new = checked + 1;
    pick_checks(h, checked, done, known, todo);
    launch_checks(todo);
    checked = done;
    cudaEventRecord(h->ev[4], sd);
    LYAP_CUDA_TRY(cudaMemcpyAsync(h->flags_host, h->flags, sizeof(int) * 3, cudaMemcpyDeviceToHost, sd));
    LYAP_CUDA_TRY(cudaMemcpyAsync(h->flags_host + 3, cw + (c & 1), sizeof(int), cudaMemcpyDeviceToHost, sd));
    LYAP_CUDA_TRY(cudaMemcpyAsync(h->hist_host + first_new - 1, h->hist + first_new - 1,
                                  sizeof(double) * (checked - first_new + 1), cudaMemcpyDeviceToHost, sd));
    // the next chunk, launched while the checks run (steps past the converged m are discarded)
    chunk = next_chunk(h->hist_host, known, done, chunk, p.check_batch_req, h->tol);
    const int next = std::min(p.maxit, done + chunk);
    if (next > done) {
      LYAP_CUDA_TRY(cudaMemsetAsync(cw + ((c + 1) & 1), 0, sizeof(int), st));
      launch_chunk(done, next, c + 1);
    }
    LYAP_CUDA_TRY(cudaGetLastError());
    LYAP_CUDA_TRY(cudaStreamSynchronize(sd));
    known = checked;
    float a = 0.f, b = 0.f;
    cudaEventElapsedTime(&a, c_beg[c & 1], c_end[c & 1]);
    cudaEventElapsedTime(&b, h->ev[5], h->ev[4]);
    t_lanczos += a;
    t_check += b;
    // a sweep error in the checked chunk, or a check that failed before (or without)
    // convergence, is the result
    h->flags_host[0] |= h->flags_host[3];
    rc = round_status(h);
    if (rc != LYAP_OK) break;
    if (h->flags_host[1] != INT_MAX) {
      // the adaptive schedule may have skipped m just before the first converged one: check
      // them, so that m is the first converged m after the last check that failed the test (a
      // period d keeps the multiples of d, Sec. 6)
      int mc = h->flags_host[1], last = mc - 1;
      while (last >= 1 && !was_checked[last]) --last;
      todo.clear();
      if (h->opt.check_every == LYAP_CHECK_ADAPTIVE)
        for (int m = last + 1; m < mc; ++m) todo.push_back(m);
      if (!todo.empty()) {
        cudaEventRecord(h->ev[5], sd);
        launch_checks(todo);
        cudaEventRecord(h->ev[4], sd);
        LYAP_CUDA_TRY(cudaMemcpyAsync(h->flags_host, h->flags, sizeof(int) * 3, cudaMemcpyDeviceToHost, sd));
        LYAP_CUDA_TRY(cudaStreamSynchronize(sd));
        float bf = 0.f;
        cudaEventElapsedTime(&bf, h->ev[5], h->ev[4]);
        t_check += bf;
        h->flags_host[0] |= h->flags_host[3];
        rc = round_status(h);
        if (rc != LYAP_OK) break;
      }
      m_final = h->flags_host[1];
      result = LYAP_OK;
      break;
    }
    if (next == done) break;
    done = next;
    ++c;
  }
  // the speculative chunk may still be running on the caller's stream
  LYAP_CUDA_TRY(cudaStreamSynchronize(st));
  if (rc != LYAP_OK) {
    h->lanczos_done = done;
    h->solved = 0;
    return rc;
  }
  int rc_end = solve_end(h, done, m_final, result, st);
  if (rc_end != LYAP_OK) return rc_end;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, h->ev[0], h->ev[1]);
  h->times_ms[1] = ms;
  h->times_ms[4] = t_check;
  h->times_ms[5] = t_lanczos;
  h->checked = checked;
  h->nchecks = nchecks;
  h->checks_past = 0;
  for (int m = h->m + 1; m <= p.maxit; ++m) h->checks_past += was_checked[m];
  return result;
}

int lyap_residual_norm(lyap_handle* h, double* hist_host, int cap, int* m_out) {
  if (!h || !h->solved) return LYAP_ERR_ARG;
  if (m_out) *m_out = h->m;
  if (hist_host && cap > 0) {
    const int n = std::min(cap, h->m);
    memcpy(hist_host, h->hist_host, sizeof(double) * n);
  }
  return h->converged ? LYAP_OK : LYAP_NOT_CONVERGED;
}

int lyap_projected_matrix(lyap_handle* h, int op, int m, double* ab, int ldab, double* gamma, double* tau_next) {
  if (!h || op < 0 || op > h->plan.sylv || m < 1 || m > h->lanczos_done) return LYAP_ERR_ARG;
  const int s = h->s, SS = s * s, N = s * m;
  if (ab && ldab < s + 1) return LYAP_ERR_ARG;
  std::vector<double> rec((size_t)(m + 1) * LOG_NREC * SS);
  LYAP_CUDA_TRY(cudaMemcpy(rec.data(), h->op[op].log, sizeof(double) * rec.size(), cudaMemcpyDeviceToHost));
  auto R = [&](int j, int kind) { return rec.data() + ((size_t)j * LOG_NREC + kind) * SS; };
  if (gamma) memcpy(gamma, R(0, REC_TNEXT), sizeof(double) * SS);
  if (tau_next) memcpy(tau_next, R(m, REC_TNEXT), sizeof(double) * SS);
  if (ab) {
    for (int i = 0; i < N; ++i)
      for (int d = 0; d <= s; ++d) {
        const int r = i + d;
        double v = 0.0;
        if (r < N) {
          const int J = r / s, Jc = i / s;
          if (J == Jc) v = 0.5 * (R(J + 1, REC_TDIAG)[(r % s) * s + i % s] + R(J + 1, REC_TDIAG)[(i % s) * s + r % s]);
          else if (J == Jc + 1) v = R(Jc + 1, REC_TNEXT)[(r % s) * s + i % s];
        }
        ab[d + (size_t)i * ldab] = v;
      }
  }
  return LYAP_OK;
}

int lyap_factor(lyap_handle* h, void* Z1, int64_t ldz1, void* Z2, int64_t ldz2, int z_dtype, int z_mem, int tcap,
                int* t_out, void* stream) {
  if (!h || !h->solved || h->factored || !Z1 || !t_out || tcap < 0) return LYAP_ERR_ARG;
  if ((h->plan.sylv != 0 || h->plan.n2 > 0) != (Z2 != nullptr)) return LYAP_ERR_ARG;
  if (z_dtype != LYAP_F64 && z_dtype != LYAP_F32) return LYAP_ERR_ARG;
  if (z_dtype == LYAP_F32 && h->plan.bulk != LYAP_PREC_MIXED) return LYAP_ERR_ARG;
  if (ldz1 < tcap || (Z2 && ldz2 < tcap)) return LYAP_ERR_ARG;
  if (z_mem != LYAP_MEM_DEVICE && z_mem != LYAP_MEM_HOST) return LYAP_ERR_ARG;
  if (z_mem == LYAP_MEM_HOST && tcap > h->plan.zcap) return LYAP_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaEventRecord(h->ev[0], st);
  void* z1 = Z1;
  void* z2 = Z2;
  int64_t l1 = ldz1, l2 = ldz2;
  const size_t zw = z_dtype == LYAP_F64 ? 8 : 4;
  if (z_mem == LYAP_MEM_HOST) {
    z1 = h->zstage;
    l1 = tcap;
    if (Z2) {
      z2 = h->zstage + lyap_align256((int64_t)(zw * (size_t)h->op[0].n * tcap));
      l2 = tcap;
    }
  }
  int rc = run_factor(h, z1, l1, z2, l2, z_dtype, tcap, t_out, st);
  if (rc != LYAP_OK) return rc;
  if (z_mem == LYAP_MEM_HOST && *t_out > 0) {
    const int t = *t_out;
    LYAP_CUDA_TRY(cudaMemcpy2DAsync(Z1, zw * ldz1, z1, zw * l1, zw * t, h->op[0].n, cudaMemcpyDeviceToHost, st));
    if (Z2)
      LYAP_CUDA_TRY(cudaMemcpy2DAsync(Z2, zw * ldz2, z2, zw * l2, zw * t, h->plan.n2 > 0 ? h->plan.n2 : h->op[1].n,
                                      cudaMemcpyDeviceToHost, st));
  }
  cudaEventRecord(h->ev[1], st);
  LYAP_CUDA_TRY(cudaStreamSynchronize(st));
  LYAP_CUDA_TRY(cudaMemcpy(h->flags_host, h->flags, sizeof(int) * 2, cudaMemcpyDeviceToHost));
  rc = status_from_bits(h->flags_host[0]);
  if (rc != LYAP_OK) return rc;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, h->ev[0], h->ev[1]);
  h->times_ms[2] = ms;
  h->factored = 1;
  return LYAP_OK;
}

int lyap_phase_times(lyap_handle* h, double* out, int cap) {
  if (!h || !out) return LYAP_ERR_ARG;
  for (int i = 0; i < cap && i < 6; ++i) out[i] = h->times_ms[i];
  if (cap > 3) out[3] = (double)h->lanczos_done;
  if (cap > 6) out[6] = (double)h->launches;
  if (cap > 7) out[7] = (double)(h->lanczos_done - h->m);  // steps run past the converged m
  if (cap > 8) out[8] = (double)h->checks_past;            // checks evaluated past it
  if (cap > 9) out[9] = (double)h->nchecks;                // checks evaluated in all
  return LYAP_OK;
}

int lyap_destroy(lyap_handle* h) {
  if (!h) return LYAP_OK;
  if (h->side) cudaStreamDestroy(h->side);
  for (int i = 0; i < 8; ++i)
    if (h->ev[i]) cudaEventDestroy(h->ev[i]);
  if (h->hist_host) cudaFreeHost(h->hist_host);
  if (h->flags_host) cudaFreeHost(h->flags_host);
  delete h;
  return LYAP_OK;
}

}  // extern "C"
