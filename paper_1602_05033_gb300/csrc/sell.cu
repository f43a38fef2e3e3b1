// CSR -> SELL-C-sigma conversion (C = 32 rows per slice, rows sorted by length
// inside windows of sigma rows).  The integer planning (row permutation, slice
// widths and offsets) runs on the host from the row pointers; the copy of the
// nnz column indices and values into the padded, slice-column-major layout runs
// on the device.
#include "common.cuh"

#include <algorithm>
#include <numeric>
#include <vector>

namespace {

struct SellPlanHost {
  std::vector<int32_t> perm;      // empty when sigma == 1
  std::vector<int32_t> width;     // per slice
  std::vector<int64_t> slice_ptr; // nslices + 1
};

int read_rowptr(const lyap_csr* A, std::vector<int64_t>& rp) {
  rp.resize((size_t)A->n + 1);
  if (A->mem == LYAP_MEM_HOST) {
    std::copy(A->rowptr, A->rowptr + A->n + 1, rp.begin());
  } else {
    if (cudaMemcpy(rp.data(), A->rowptr, sizeof(int64_t) * (A->n + 1), cudaMemcpyDeviceToHost) != cudaSuccess)
      return LYAP_ERR_CUDA;
  }
  if (rp[0] != 0 || rp[A->n] != A->nnz) return LYAP_ERR_ARG;
  for (int64_t i = 0; i < A->n; ++i)
    if (rp[i + 1] < rp[i]) return LYAP_ERR_ARG;
  return LYAP_OK;
}

int plan(const lyap_csr* A, int sigma, SellPlanHost& p) {
  std::vector<int64_t> rp;
  int st = read_rowptr(A, rp);
  if (st != LYAP_OK) return st;
  const int64_t n = A->n;
  const int64_t nsl = (n + LYAP_SLICE - 1) / LYAP_SLICE;
  std::vector<int32_t> len((size_t)n);
  for (int64_t i = 0; i < n; ++i) len[i] = (int32_t)(rp[i + 1] - rp[i]);
  if (sigma > 1) {
    p.perm.resize((size_t)n);
    std::iota(p.perm.begin(), p.perm.end(), 0);
    for (int64_t w0 = 0; w0 < n; w0 += sigma) {
      const int64_t w1 = std::min<int64_t>(n, w0 + sigma);
      std::stable_sort(p.perm.begin() + w0, p.perm.begin() + w1,
                       [&](int32_t a, int32_t b) { return len[a] > len[b]; });
    }
  }
  p.width.assign((size_t)nsl, 0);
  p.slice_ptr.assign((size_t)nsl + 1, 0);
  for (int64_t k = 0; k < nsl; ++k) {
    int32_t w = 0;
    for (int l = 0; l < LYAP_SLICE; ++l) {
      const int64_t r = k * LYAP_SLICE + l;
      if (r >= n) break;
      const int32_t row = p.perm.empty() ? (int32_t)r : p.perm[r];
      w = std::max(w, len[row]);
    }
    p.width[k] = w;
    p.slice_ptr[k + 1] = p.slice_ptr[k] + (int64_t)w * LYAP_SLICE;
  }
  return LYAP_OK;
}

// an operator value in the stored type: fp64, fp32, or a float pair (hi = fl32(v), lo = fl32(v - hi))
template <typename Tout>
__device__ __forceinline__ Tout sell_value(double v) { return Tout(v); }
template <>
__device__ __forceinline__ float2 sell_value<float2>(double v) {
  const float h = (float)v;
  return make_float2(h, (float)(v - (double)h));
}

template <typename Tin, typename Tout>
__global__ void k_sell_fill(int64_t n, int64_t nsl, const int64_t* __restrict__ rowptr,
                            const int32_t* __restrict__ col, const Tin* __restrict__ val,
                            const int32_t* __restrict__ perm, const int64_t* __restrict__ slice_ptr,
                            const int32_t* __restrict__ width, int32_t* __restrict__ scol,
                            Tout* __restrict__ sval, int* flags) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t k = t / LYAP_SLICE;
  const int lane = (int)(t % LYAP_SLICE);
  if (k >= nsl) return;
  const int64_t r = k * LYAP_SLICE + lane;
  const int64_t row = r < n ? (perm ? (int64_t)perm[r] : r) : -1;
  const int w = width[k];
  int64_t b = 0, len = 0;
  if (row >= 0) {
    b = rowptr[row];
    len = rowptr[row + 1] - b;
  }
  const int32_t pad_col = row >= 0 ? (int32_t)row : 0;
  for (int j = 0; j < w; ++j) {
    const int64_t e = slice_ptr[k] + (int64_t)j * LYAP_SLICE + lane;
    if (j < len) {
      const int32_t c = col[b + j];
      if (c < 0 || c >= n) {
        atomicOr(flags, DERR_BOUNDS);
        scol[e] = pad_col;
        sval[e] = sell_value<Tout>(0.0);
      } else {
        scol[e] = c;
        const Tin v = val[b + j];
        if (!isfinite((double)v)) atomicOr(flags, DERR_NONFINITE);
        sval[e] = sell_value<Tout>((double)v);
      }
    } else {
      scol[e] = pad_col;
      sval[e] = sell_value<Tout>(0.0);
    }
  }
}

}  // namespace

int sell_plan_host(const lyap_csr* A, int sigma, int64_t* nslices, int64_t* sell_nnz) {
  SellPlanHost p;
  int st = plan(A, sigma, p);
  if (st != LYAP_OK) return st;
  *nslices = (int64_t)p.width.size();
  *sell_nnz = p.slice_ptr.back();
  return LYAP_OK;
}

// d_rowptr/d_col/d_val: the CSR arrays in device memory (the caller's, or staged copies)
int sell_build(const lyap_csr* A, const int64_t* d_rowptr, const int32_t* d_col, const void* d_val, int sigma,
               int bulk, OpDev& op, int* d_flags, cudaStream_t st) {
  SellPlanHost p;
  int rc = plan(A, sigma, p);
  if (rc != LYAP_OK) return rc;
  if ((int64_t)p.width.size() != op.nslices || p.slice_ptr.back() != op.sell_nnz) return LYAP_ERR_ARG;
  LYAP_CUDA_TRY(cudaMemcpyAsync(op.slice_ptr, p.slice_ptr.data(), sizeof(int64_t) * p.slice_ptr.size(),
                                cudaMemcpyHostToDevice, st));
  LYAP_CUDA_TRY(cudaMemcpyAsync(op.slice_w, p.width.data(), sizeof(int32_t) * p.width.size(),
                                cudaMemcpyHostToDevice, st));
  if (!p.perm.empty()) {
    LYAP_CUDA_TRY(cudaMemcpyAsync(op.perm, p.perm.data(), sizeof(int32_t) * p.perm.size(),
                                  cudaMemcpyHostToDevice, st));
  } else {
    op.perm = nullptr;
  }
  const int64_t threads = op.nslices * LYAP_SLICE;
  const int bs = 256;
  const int64_t grid = (threads + bs - 1) / bs;
#define LYAP_FILL(TIN, TOUT)                                                                                     \
  k_sell_fill<TIN, TOUT><<<(unsigned)grid, bs, 0, st>>>(A->n, op.nslices, d_rowptr, d_col, (const TIN*)d_val, op.perm, \
                                                     op.slice_ptr, op.slice_w, op.sell_col, (TOUT*)op.sell_val, d_flags)
  // stored type: fp64 (fp64 bulk), fp32 (fp32 bulk, and float-pair bulk with fp32 input values), pairs
  if (A->val_dtype == LYAP_F64) {
    if (bulk == LYAP_PREC_MIXED) LYAP_FILL(double, float);
    else if (bulk == LYAP_PREC_F32X2) LYAP_FILL(double, float2);
    else LYAP_FILL(double, double);
  } else {
    if (bulk == LYAP_PREC_F64) LYAP_FILL(float, double);
    else LYAP_FILL(float, float);
  }
#undef LYAP_FILL
  LYAP_CUDA_TRY(cudaGetLastError());
  // the host vectors must outlive the async copies
  LYAP_CUDA_TRY(cudaStreamSynchronize(st));
  return LYAP_OK;
}
