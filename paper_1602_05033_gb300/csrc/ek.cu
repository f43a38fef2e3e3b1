// Extended Krylov projection (Sec. 4) with the solves with A done by preconditioned conjugate
// gradients on the GPU, preconditioned by Jacobi scaling, by IC(0) applied through a truncated
// Neumann series, or by IC(0) values corrected by a small network trained on solve pairs that the
// method itself produces (ekprec.cuh).  The CG iterations run on an internal stream, eight at a
// time replayed from a CUDA graph.
//
// Basis blocks V_j = [V_j^(1), V_j^(2)] have S = 2s columns; [C, A^{-1} C] = V_1 gamma.  Step j:
// W = [A V_j^(1), A^{-1} V_j^(2)], block Gram-Schmidt against every stored block (twice), CholQR2
// -> V_{j+1}; tau_jj = V_j^T A V_j and tau_{j+1,j} = V_{j+1}^T A V_j by explicit projection.  These
// go into a coefficient log with block size S, so the convergence check (Prop. 3.1, Alg. 3) and the
// factor (eq. 2.5) are the standard ones with block size 2s.  Sec. 4's three-term orthogonalisation
// loses orthogonality quickly in floating point, hence the full Gram-Schmidt (the space is small).
#include "common.cuh"

#include <cuda_bf16.h>
#include <float.h>
#include <math.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

namespace {

constexpr int kT = 256;
constexpr int kGrid = 304;           // CTAs of the reduction kernels (fixed: deterministic sums)
constexpr int kTile = 1024;          // pixels per weight-gradient tile of the CUDA-core layers

struct Csr {
  int64_t n;
  const int64_t* rowptr;
  const int32_t* col;
  const double* val;
};

// ---- fixed-order reductions: per-CTA partials, then one CTA sums them in CTA order --------
template <int NV>
__device__ void cta_partials(double (&v)[NV], double* __restrict__ partials) {
  __shared__ double red[kT / 32][NV > 0 ? NV : 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double x = v[k];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) red[warp][k] = x;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < NV; k += blockDim.x) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w][k];
    partials[(size_t)blockIdx.x * NV + k] = t;
  }
  __syncthreads();
}

// out[k] = sum over CTAs of partials (one CTA, fixed order)
__global__ void k_sum_partials(const double* __restrict__ partials, int nparts, int nv, double* __restrict__ out) {
  for (int k = threadIdx.x; k < nv; k += blockDim.x) {
    double t = 0.0;
    for (int b = 0; b < nparts; ++b) t += partials[(size_t)b * nv + k];
    out[k] = t;
  }
}

// ---- sparse products --------------------------------------------------------------------
// Y = sgn * A X for S columns (row-major, leading dimensions ldx, ldy)
template <int S>
__global__ void k_spmm(Csr A, const double* __restrict__ X, int ldx, double* __restrict__ Y, int ldy, double sgn) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < A.n; i += (int64_t)gridDim.x * blockDim.x) {
    double acc[S];
#pragma unroll
    for (int a = 0; a < S; ++a) acc[a] = 0.0;
    for (int64_t e = A.rowptr[i]; e < A.rowptr[i + 1]; ++e) {
      const double v = A.val[e];
      const double* x = X + (int64_t)A.col[e] * ldx;
#pragma unroll
      for (int a = 0; a < S; ++a) acc[a] = fma(v, x[a], acc[a]);
    }
#pragma unroll
    for (int a = 0; a < S; ++a) Y[i * ldy + a] = sgn * acc[a];
  }
}

void spmm(const Csr& A, int S, const double* X, int ldx, double* Y, int ldy, double sgn, cudaStream_t st) {
  const int g = (int)std::min<int64_t>((A.n + kT - 1) / kT, 8192);
  switch (S) {
    case 1: k_spmm<1><<<g, kT, 0, st>>>(A, X, ldx, Y, ldy, sgn); break;
    case 2: k_spmm<2><<<g, kT, 0, st>>>(A, X, ldx, Y, ldy, sgn); break;
    case 4: k_spmm<4><<<g, kT, 0, st>>>(A, X, ldx, Y, ldy, sgn); break;
    case 8: k_spmm<8><<<g, kT, 0, st>>>(A, X, ldx, Y, ldy, sgn); break;
  }
}

// ---- block Gram-Schmidt pieces ----------------------------------------------------------
// partials of P_b = X_b^T W for nb blocks X_b (n x S, consecutive, block stride bstride)
template <int S>
__global__ void k_proj(const double* __restrict__ X, int64_t bstride, int nb, const double* __restrict__ W, int64_t n,
                       double* __restrict__ partials) {
  const int b = blockIdx.y;
  double acc[S * S];
#pragma unroll
  for (int k = 0; k < S * S; ++k) acc[k] = 0.0;
  const double* Xb = X + (size_t)b * bstride;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double x[S], w[S];
#pragma unroll
    for (int a = 0; a < S; ++a) {
      x[a] = Xb[i * S + a];
      w[a] = W[i * S + a];
    }
#pragma unroll
    for (int a = 0; a < S; ++a)
#pragma unroll
      for (int c = 0; c < S; ++c) acc[a * S + c] = fma(x[a], w[c], acc[a * S + c]);
  }
  cta_partials<S * S>(acc, partials + (size_t)b * gridDim.x * S * S);
}

// P[b] = sum of its partials (one CTA per block)
__global__ void k_proj_sum(const double* __restrict__ partials, int nparts, int nv, double* __restrict__ P) {
  const int b = blockIdx.x;
  for (int k = threadIdx.x; k < nv; k += blockDim.x) {
    double t = 0.0;
    for (int c = 0; c < nparts; ++c) t += partials[((size_t)b * nparts + c) * nv + k];
    P[(size_t)b * nv + k] = t;
  }
}

// W -= sum_b X_b P_b
template <int S>
__global__ void k_subtract(const double* __restrict__ X, int64_t bstride, int nb, const double* __restrict__ P,
                           double* __restrict__ W, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double w[S];
#pragma unroll
    for (int a = 0; a < S; ++a) w[a] = W[i * S + a];
    for (int b = 0; b < nb; ++b) {
      const double* xb = X + (size_t)b * bstride + i * S;
      const double* pb = P + (size_t)b * S * S;
#pragma unroll
      for (int a = 0; a < S; ++a) {
        const double xa = xb[a];
#pragma unroll
        for (int c = 0; c < S; ++c) w[c] = fma(-xa, pb[a * S + c], w[c]);
      }
    }
#pragma unroll
    for (int a = 0; a < S; ++a) W[i * S + a] = w[a];
  }
}

// W <- W R^{-1} (R upper triangular, S x S row-major)
template <int S>
__global__ void k_trsm(double* __restrict__ W, int64_t n, const double* __restrict__ R) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double w[S];
#pragma unroll
    for (int a = 0; a < S; ++a) w[a] = W[i * S + a];
#pragma unroll
    for (int c = 0; c < S; ++c) {
      double t = w[c];
#pragma unroll
      for (int a = 0; a < c; ++a) t = fma(-w[a], R[a * S + c], t);
      w[c] = t / R[c * S + c];
    }
#pragma unroll
    for (int a = 0; a < S; ++a) W[i * S + a] = w[a];
  }
}

// dst[:, off:off+w] = src[:, 0:w] (row-major, leading dimensions), scaled
__global__ void k_copy_cols(const double* __restrict__ src, int lds, double* __restrict__ dst, int ldd, int off, int w,
                            int64_t n, double scale) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * w; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / w;
    const int c = (int)(t % w);
    dst[i * ldd + off + c] = scale * src[i * lds + c];
  }
}

// ---- preconditioned conjugate gradients on M = -A (SPD) for s columns ----------------------
// scalars per column (device): [0] rz, [1] alpha, [2] beta, [3] rr, [4] bb, [5] active (as double)
constexpr int kSc = 6;

// x = 0, r = -B, bb = ||B||^2 per column; B has leading dimension ldb
template <int s>
__global__ void k_cg_start(const double* __restrict__ B, int ldb, double* __restrict__ x, double* __restrict__ r,
                           int64_t n, double* __restrict__ partials) {
  double acc[s];
#pragma unroll
  for (int c = 0; c < s; ++c) acc[c] = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
#pragma unroll
    for (int c = 0; c < s; ++c) {
      const double b = B[i * ldb + c];
      x[i * s + c] = 0.0;
      r[i * s + c] = -b;
      acc[c] = fma(b, b, acc[c]);
    }
  cta_partials<s>(acc, partials);
}

// Jacobi: z = r / diag(M); partials z.r and z.r_old (r_old = r + alpha q)
template <int s>
__global__ void k_cg_jacobi(const double* __restrict__ mdinv, const double* __restrict__ r, const double* __restrict__ q,
                            const double* __restrict__ sc, double* __restrict__ z, int64_t n, int first,
                            double* __restrict__ partials) {
  double acc[2 * s];
#pragma unroll
  for (int k = 0; k < 2 * s; ++k) acc[k] = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double d = mdinv[i];
#pragma unroll
    for (int c = 0; c < s; ++c) {
      const double rc = r[i * s + c];
      const double zc = d * rc;
      z[i * s + c] = zc;
      acc[c] = fma(zc, rc, acc[c]);
      if (!first) acc[s + c] = fma(zc, rc + sc[c * kSc + 1] * q[i * s + c], acc[s + c]);
    }
  }
  cta_partials<2 * s>(acc, partials);
}

// partials z.r and z.r_old for a preconditioner applied elsewhere
template <int s>
__global__ void k_cg_zdots(const double* __restrict__ r, const double* __restrict__ q, const double* __restrict__ sc,
                           const double* __restrict__ z, int64_t n, int first, double* __restrict__ partials) {
  double acc[2 * s];
#pragma unroll
  for (int k = 0; k < 2 * s; ++k) acc[k] = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
#pragma unroll
    for (int c = 0; c < s; ++c) {
      const double rc = r[i * s + c], zc = z[i * s + c];
      acc[c] = fma(zc, rc, acc[c]);
      if (!first) acc[s + c] = fma(zc, rc + sc[c * kSc + 1] * q[i * s + c], acc[s + c]);
    }
  cta_partials<2 * s>(acc, partials);
}

// beta (Polak-Ribiere, for a preconditioner that may vary), new rz; first: rz only, beta = 0
__global__ void k_cg_beta(const double* __restrict__ zdots, double* __restrict__ sc, int s, int first) {
  const int c = threadIdx.x;
  if (c >= s) return;
  double* q = sc + c * kSc;
  const double zr = zdots[c], zro = zdots[s + c];
  const bool act = q[5] != 0.0;
  q[2] = (!first && act && q[0] != 0.0) ? (zr - zro) / q[0] : 0.0;
  if (act) q[0] = zr;
}

// p = z + beta p (active columns)
template <int s>
__global__ void k_cg_dir(const double* __restrict__ z, double* __restrict__ p, const double* __restrict__ sc, int64_t n) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * s; t += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(t % s);
    if (sc[c * kSc + 5] != 0.0) p[t] = z[t] + sc[c * kSc + 2] * p[t];
  }
}

// q = M p; partials p.q
template <int s>
__global__ void k_cg_matvec(Csr A, const double* __restrict__ p, double* __restrict__ q, double* __restrict__ partials) {
  double acc[s];
#pragma unroll
  for (int c = 0; c < s; ++c) acc[c] = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < A.n; i += (int64_t)gridDim.x * blockDim.x) {
    double t[s];
#pragma unroll
    for (int c = 0; c < s; ++c) t[c] = 0.0;
    for (int64_t e = A.rowptr[i]; e < A.rowptr[i + 1]; ++e) {
      const double v = -A.val[e];
      const double* x = p + (int64_t)A.col[e] * s;
#pragma unroll
      for (int c = 0; c < s; ++c) t[c] = fma(v, x[c], t[c]);
    }
#pragma unroll
    for (int c = 0; c < s; ++c) {
      q[i * s + c] = t[c];
      acc[c] = fma(p[i * s + c], t[c], acc[c]);
    }
  }
  cta_partials<s>(acc, partials);
}

__global__ void k_cg_alpha(const double* __restrict__ pq, double* __restrict__ sc, int s) {
  const int c = threadIdx.x;
  if (c >= s) return;
  double* q = sc + c * kSc;
  q[1] = (q[5] != 0.0 && pq[c] > 0.0) ? q[0] / pq[c] : 0.0;
}

// x += alpha p, r -= alpha q; partials r.r
template <int s>
__global__ void k_cg_update(double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p,
                            const double* __restrict__ q, const double* __restrict__ sc, int64_t n,
                            double* __restrict__ partials) {
  double acc[s];
#pragma unroll
  for (int c = 0; c < s; ++c) acc[c] = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
#pragma unroll
    for (int c = 0; c < s; ++c) {
      const double al = sc[c * kSc + 1];
      x[i * s + c] = fma(al, p[i * s + c], x[i * s + c]);
      const double rc = fma(-al, q[i * s + c], r[i * s + c]);
      r[i * s + c] = rc;
      acc[c] = fma(rc, rc, acc[c]);
    }
  cta_partials<s>(acc, partials);
}

// rr, and the stopping test ||r|| <= tol ||b||
__global__ void k_cg_conv(const double* __restrict__ rr, double* __restrict__ sc, int s, double tol2, int start) {
  const int c = threadIdx.x;
  if (c >= s) return;
  double* q = sc + c * kSc;
  if (start) {
    q[4] = rr[c];
    q[3] = rr[c];
    q[5] = rr[c] > 0.0 ? 1.0 : 0.0;
    q[0] = 0.0;
    return;
  }
  q[3] = rr[c];
  if (!(rr[c] > tol2 * q[4])) q[5] = 0.0;
}

// ---- preconditioners on the operator's grid (IC(0), truncated Neumann application, network) ---
#include "ekprec.cuh"

// 1 / diag(-A)
__global__ void k_mdinv(Csr A, double* __restrict__ d) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < A.n; i += (int64_t)gridDim.x * blockDim.x) {
    double a = 0.0;
    for (int64_t e = A.rowptr[i]; e < A.rowptr[i + 1]; ++e)
      if (A.col[e] == i) a = A.val[e];
    d[i] = a < 0.0 ? -1.0 / a : 0.0;
  }
}

int grid_for(int64_t n) { return (int)std::min<int64_t>((n + kT - 1) / kT, kGrid); }

constexpr int kPairCap = 4;     // training pairs (columns of the first inner solves)
constexpr int kTrainBlocks = 2 + 2 * (kQ + 2) + 7;  // n x kPairCap blocks of the training pass
constexpr int kL2WGrid = 152;   // CTAs of the tensor-core weight-gradient kernel

}  // namespace

namespace {

struct EkLayout {
  size_t total = 0, basis = 0, W = 0, AV = 0, C = 0, mdinv = 0, vec = 0, partials = 0, small = 0, log = 0, hist = 0,
         flags = 0, chk = 0, check = 0, check_bytes = 0, factor = 0, factor_bytes = 0, csr = 0, pairs = 0, prec = 0;
  int pair_cap = 0;
};

int64_t wpart_rows_bytes(int64_t n) {
  const int64_t ntiles = (n + kTile - 1) / kTile;
  const int64_t a = ntiles * std::max(kNW1, kNW3);
  const int64_t b = (int64_t)kL2WGrid * kWarpsW * kNW2;
  return (int64_t)sizeof(double) * std::max(a, b);
}

size_t prec_bytes(int64_t n) {
  size_t b = 0;
  auto add = [&](size_t x) { b += lyap_align256((int64_t)x); };
  add(sizeof(double) * n * 5);                    // stencil
  add(sizeof(double) * n);                        // pivots
  add(sizeof(double) * n * 6);                    // IC(0) and learned values
  add(sizeof(float) * n * kNin);                  // features
  add(sizeof(__nv_bfloat16) * n * kCh * 4);       // a1, a2, g1, g2
  add(sizeof(float) * n * kNout * 2);             // y, gy
  add(sizeof(double) * n * 3);                    // value gradients
  add(sizeof(double) * n * kPairCap * kTrainBlocks);  // training blocks
  add(sizeof(double) * n * 4 * 3);                // application scratch (s <= 4)
  add(sizeof(float) * kNW * 4);                   // th, m1, m2, initial th
  add(sizeof(__nv_bfloat16) * kNW);               // thq
  add(sizeof(double) * kNW);                      // grad
  add((size_t)wpart_rows_bytes(n));               // weight-gradient partials
  add(sizeof(double) * 32);                       // loss coefficients
  add(256);                                       // flags
  return b;
}

EkLayout ek_layout(const lyap_csr* A, int s, int maxit, int grid_image) {
  EkLayout L;
  const int S = 2 * s;
  const int64_t n = A->n;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t r = off; off += lyap_align256((int64_t)bytes); return r; };
  L.csr = take(sizeof(int64_t) * (n + 1) + 8) ;
  take(sizeof(int32_t) * A->nnz);
  take(sizeof(double) * A->nnz);
  L.basis = take(sizeof(double) * (size_t)(maxit + 1) * n * S);
  L.W = take(sizeof(double) * n * S);
  L.AV = take(sizeof(double) * n * S);
  L.C = take(sizeof(double) * n * s);
  L.mdinv = take(sizeof(double) * n);
  L.vec = take(sizeof(double) * n * s * 5);
  L.partials = take(sizeof(double) * (size_t)kGrid * (maxit + 2) * S * S);
  L.small = take(sizeof(double) * ((size_t)(maxit + 2) * S * S + 128));
  L.log = take(sizeof(double) * (size_t)(maxit + 1) * LOG_NREC * S * S);
  L.hist = take(sizeof(double) * maxit);
  L.flags = take(256);
  L.chk = take(sizeof(int) * maxit);
  const int nmax = S * maxit;
  L.check_bytes = std::max(check_slot_bytes(S, nmax), (size_t)1 << 20);
  L.check = take(L.check_bytes);
  L.factor_bytes = factor_ws_bytes(S, nmax, 0);
  L.factor = take(L.factor_bytes);
  L.pair_cap = kPairCap;
  L.pairs = take(sizeof(double) * n * L.pair_cap * 2);
  L.prec = grid_image ? take(prec_bytes(n)) : 0;
  L.total = off;
  return L;
}

template <typename T>
T* at(char* base, size_t off) { return reinterpret_cast<T*>(base + off); }

// two dot products u.v and u.w (n doubles each) -> partials
__global__ void k_dot2(const double* __restrict__ u, const double* __restrict__ v, const double* __restrict__ w, int64_t n,
                       double* __restrict__ partials) {
  double acc[2] = {0.0, 0.0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    acc[0] = fma(u[i], v[i], acc[0]);
    acc[1] = fma(u[i], w[i], acc[1]);
  }
  cta_partials<2>(acc, partials);
}

// Y -= X (n * c values)
__global__ void k_sub(double* __restrict__ Y, const double* __restrict__ X, int64_t m) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < m; t += (int64_t)gridDim.x * blockDim.x)
    Y[t] -= X[t];
}

__global__ void k_init_ek(double* __restrict__ hist, int* __restrict__ flags, int* __restrict__ chk_err, int maxit) {
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

}  // namespace

// ---------------------------------------------------------------------------------------------
// preconditioner state of a context on an nx x ny grid
struct EkPrec {
  Grid g{0, 0};
  int status = -1;               // 0: IC(0) exists; otherwise why not (1 pattern, 2 diagonal, 4 pivot)
  double *sten = nullptr, *piv = nullptr;
  double *d0 = nullptr, *lw0 = nullptr, *ls0 = nullptr;  // IC(0)
  double *d1 = nullptr, *lw1 = nullptr, *ls1 = nullptr;  // the network's values
  float* feats = nullptr;
  __nv_bfloat16 *a1 = nullptr, *a2 = nullptr, *g1 = nullptr, *g2 = nullptr;
  float *y = nullptr, *gy = nullptr;
  double *gd = nullptr, *gw = nullptr, *gs = nullptr;
  double* train = nullptr;       // kTrainBlocks blocks of n x kPairCap
  double* app = nullptr;         // 3 blocks of n x 4: the application's Horner scratch
  float *th = nullptr, *m1 = nullptr, *m2 = nullptr, *th_init = nullptr;
  __nv_bfloat16* thq = nullptr;
  double *grad = nullptr, *wpart = nullptr, *coef = nullptr;
  int* bad = nullptr;
};

struct lyap_ek {
  int s = 1, S = 2, maxit = 0;
  int64_t n = 0;
  int nx = 0, ny = 0;
  double tol = 1e-8, inner_tol = 1e-10;
  int inner_maxit = 20000;
  Csr A;
  EkLayout L;
  char* ws = nullptr;
  double *basis = nullptr, *AV = nullptr, *C = nullptr, *mdinv = nullptr;
  double *x = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr;
  double *partials = nullptr, *small = nullptr, *sc = nullptr, *P = nullptr, *dR = nullptr;
  double* log = nullptr;
  double *pair_b = nullptr, *pair_x = nullptr;
  int npairs = 0;
  EkPrec pc;
  int trained = 0, adam_t = 0, last_jacobi_its = 0, last_ic0_its = 0, fallbacks = 0;
  // the conjugate-gradient iterations run on an internal stream; eight of them at a time are
  // replayed from a CUDA graph per preconditioner kind (state 0: not captured, 1: captured,
  // -1: capture failed, direct launches)
  cudaStream_t cgs = nullptr;
  cudaEvent_t cg_ev[2] = {};
  cudaGraphExec_t cg_graph[3] = {};
  int cg_state[3] = {0, 0, 0};
  lyap_handle hk;  // the check and factor kernels' view: block size S, the log below
  int m = 0, done = 0;
  std::vector<int> inner_its, inner_kind;
  double times[8] = {};
  double loss0 = -1.0, loss1 = -1.0;
  cudaEvent_t ev[4] = {};
};

namespace {

// ---- block Gram-Schmidt with deterministic sums ---------------------------------------------
void project(lyap_ek* e, const double* X, int nb, const double* Wm, cudaStream_t st) {
  const int S = e->S;
  const int g = grid_for(e->n);
  dim3 grid(g, nb);
  switch (S) {
    case 1: k_proj<1><<<grid, kT, 0, st>>>(X, e->n * S, nb, Wm, e->n, e->partials); break;
    case 2: k_proj<2><<<grid, kT, 0, st>>>(X, e->n * S, nb, Wm, e->n, e->partials); break;
    case 4: k_proj<4><<<grid, kT, 0, st>>>(X, e->n * S, nb, Wm, e->n, e->partials); break;
    case 8: k_proj<8><<<grid, kT, 0, st>>>(X, e->n * S, nb, Wm, e->n, e->partials); break;
  }
  k_proj_sum<<<nb, 64, 0, st>>>(e->partials, g, S * S, e->P);
}

void subtract(lyap_ek* e, const double* X, int nb, double* Wm, cudaStream_t st) {
  const int g = grid_for(e->n) * 4;
  switch (e->S) {
    case 1: k_subtract<1><<<g, kT, 0, st>>>(X, e->n * 1, nb, e->P, Wm, e->n); break;
    case 2: k_subtract<2><<<g, kT, 0, st>>>(X, e->n * 2, nb, e->P, Wm, e->n); break;
    case 4: k_subtract<4><<<g, kT, 0, st>>>(X, e->n * 4, nb, e->P, Wm, e->n); break;
    case 8: k_subtract<8><<<g, kT, 0, st>>>(X, e->n * 8, nb, e->P, Wm, e->n); break;
  }
}

bool chol_upper_host(const double* G, double* R, int S) {
  for (int i = 0; i < S * S; ++i) R[i] = 0.0;
  for (int j = 0; j < S; ++j) {
    double d = G[j * S + j];
    for (int k = 0; k < j; ++k) d -= R[k * S + j] * R[k * S + j];
    if (!(d > 0.0) || !std::isfinite(d)) return false;
    R[j * S + j] = sqrt(d);
    for (int i = j + 1; i < S; ++i) {
      double t = 0.5 * (G[j * S + i] + G[i * S + j]);
      for (int k = 0; k < j; ++k) t -= R[k * S + j] * R[k * S + i];
      R[j * S + i] = t / R[j * S + j];
    }
  }
  return true;
}

// CholQR2 of Wm in place; gamma = R2 R1 (S x S row-major, host)
int cholqr2(lyap_ek* e, double* Wm, std::vector<double>& gamma, cudaStream_t st) {
  const int S = e->S;
  std::vector<double> G(S * S), R(S * S), acc(S * S, 0.0);
  for (int pass = 0; pass < 2; ++pass) {
    project(e, Wm, 1, Wm, st);
    LYAP_CUDA_TRY(cudaMemcpyAsync(G.data(), e->P, sizeof(double) * S * S, cudaMemcpyDeviceToHost, st));
    LYAP_CUDA_TRY(cudaStreamSynchronize(st));
    if (!chol_upper_host(G.data(), R.data(), S)) return LYAP_ERR_BREAKDOWN;
    LYAP_CUDA_TRY(cudaMemcpyAsync(e->dR, R.data(), sizeof(double) * S * S, cudaMemcpyHostToDevice, st));
    const int g = grid_for(e->n) * 4;
    switch (S) {
      case 1: k_trsm<1><<<g, kT, 0, st>>>(Wm, e->n, e->dR); break;
      case 2: k_trsm<2><<<g, kT, 0, st>>>(Wm, e->n, e->dR); break;
      case 4: k_trsm<4><<<g, kT, 0, st>>>(Wm, e->n, e->dR); break;
      case 8: k_trsm<8><<<g, kT, 0, st>>>(Wm, e->n, e->dR); break;
    }
    if (pass == 0) acc = R;
    else {
      std::vector<double> t(S * S, 0.0);
      for (int i = 0; i < S; ++i)
        for (int j = 0; j < S; ++j)
          for (int k = 0; k < S; ++k) t[i * S + j] += R[i * S + k] * acc[k * S + j];
      acc = t;
    }
    LYAP_CUDA_TRY(cudaStreamSynchronize(st));  // dR is reused
  }
  gamma = acc;
  return LYAP_OK;
}

// ---- the preconditioner's application, Z = P_q R on C columns -------------------------------
Vals vals_of(const EkPrec& pc, int kind) {
  return kind == 2 ? Vals{pc.d1, pc.lw1, pc.ls1} : Vals{pc.d0, pc.lw0, pc.ls0};
}

template <int C>
void apply_P_t(const EkPrec& pc, const Vals& v, int64_t n, const double* R, int ldr, double* Z, int ldz, cudaStream_t st) {
  const int gr = grid_for(n) * 4;
  double* U = pc.app;
  double* Ya = pc.app + n * 4;
  double* Yb = pc.app + n * 8;
  k_h_first<C><<<gr, kT, 0, st>>>(R, ldr, v.d, U, Ya, n);
  double *cur = Ya, *nxt = Yb;
  for (int j = 0; j < kQ; ++j) {
    k_h_fwd<C><<<gr, kT, 0, st>>>(U, cur, v, pc.g, nxt);
    std::swap(cur, nxt);
  }
  // cur = B_q R; then B_q^T by Horner steps w <- y - N^T D^{-1} w, ping-pong in the free buffers
  const double* y = cur;
  double* wa = cur == Ya ? Yb : Ya;
  double* wb = U;
  const double* w0 = y;
  for (int j = 0; j < kQ; ++j) {
    double* out = (j % 2 == 0) ? wa : wb;
    k_h_bwd<C><<<gr, kT, 0, st>>>(y, w0, v, pc.g, out);
    w0 = out;
  }
  k_h_last<C><<<gr, kT, 0, st>>>(w0, v.d, Z, ldz, n);
}

void apply_P(const EkPrec& pc, int kind, int C, int64_t n, const double* R, int ldr, double* Z, int ldz, cudaStream_t st) {
  const Vals v = vals_of(pc, kind);
  switch (C) {
    case 1: apply_P_t<1>(pc, v, n, R, ldr, Z, ldz, st); break;
    case 2: apply_P_t<2>(pc, v, n, R, ldr, Z, ldz, st); break;
    case 3: apply_P_t<3>(pc, v, n, R, ldr, Z, ldz, st); break;
    case 4: apply_P_t<4>(pc, v, n, R, ldr, Z, ldz, st); break;
  }
}

// ---- the network: forward into the learned values, loss and gradient over K pairs ------------
void net_forward(lyap_ek* e, cudaStream_t st) {
  EkPrec& pc = e->pc;
  const int64_t n = e->n;
  const int gp = (int)std::min<int64_t>((n + kT - 1) / kT, 4096);
  const int gm = (int)std::min<int64_t>(((n + 15) / 16 + kWarpsW - 1) / kWarpsW, 4096);
  k_l1_fwd<<<gp, kT, 0, st>>>(pc.feats, pc.thq + oW1, pc.th + oB1, pc.g, pc.a1);
  k_l2_fwd<<<gm, 256, 0, st>>>(pc.a1, pc.thq + oW2, pc.th + oB2, pc.g, pc.a2);
  k_l3_fwd<<<gp, kT, 0, st>>>(pc.a2, pc.thq + oW3, pc.th + oB3, pc.g, pc.y);
  k_net_vals<<<grid_for(n) * 4, kT, 0, st>>>(pc.y, vals_of(pc, 1), n, pc.d1, pc.lw1, pc.ls1);
}

// training blocks (n x K each, K <= kPairCap): R, X, Ur, Yr[0..q], Ug, Yg[0..q], E, ME, G, T1, T2, lamA, lamB
struct TrainBufs {
  double *R, *X, *Ur, *Yr[kQ + 1], *Ug, *Yg[kQ + 1], *E, *ME, *G, *T1, *T2, *la, *lb;
};

TrainBufs train_bufs(const lyap_ek* e) {
  TrainBufs b;
  double* p = e->pc.train;
  const size_t blk = (size_t)e->n * kPairCap;
  int k = 0;
  auto next = [&]() { return p + blk * (k++); };
  b.R = next();
  b.X = next();
  b.Ur = next();
  for (int j = 0; j <= kQ; ++j) b.Yr[j] = next();
  b.Ug = next();
  for (int j = 0; j <= kQ; ++j) b.Yg[j] = next();
  b.E = next();
  b.ME = next();
  b.G = next();
  b.T1 = next();
  b.T2 = next();
  b.la = next();
  b.lb = next();
  return b;
}

template <int C>
void horner_fwd_store(const EkPrec& pc, const Vals& v, int64_t n, const double* R, double* U, double* const* Y,
                      cudaStream_t st) {
  const int gr = grid_for(n) * 4;
  k_h_first<C><<<gr, kT, 0, st>>>(R, C, v.d, U, Y[0], n);
  for (int j = 0; j < kQ; ++j) k_h_fwd<C><<<gr, kT, 0, st>>>(U, Y[j], v, pc.g, Y[j + 1]);
}

// lambda_q = Lq; forward iterates Y[0..q] of the other argument; gradient into gd, gw, gs
template <int C>
void reverse_pass(const EkPrec& pc, const Vals& v, int64_t n, const double* Lq, double* const* Y, double* la, double* lb,
                  cudaStream_t st) {
  const int gr = grid_for(n) * 4;
  const double* lam = Lq;
  double* outs[2] = {la, lb};
  for (int j = kQ - 1; j >= 0; --j) {
    double* out = outs[j % 2];
    k_h_rev<C><<<gr, kT, 0, st>>>(lam, Y[j], Y[j + 1], v, pc.g, out, pc.gd, pc.gw, pc.gs);
    lam = out;
  }
  k_h_rev_last<C><<<gr, kT, 0, st>>>(lam, Y[0], v.d, n, pc.gd);
}

// the energy loss of the current network over K pairs in tb.R, tb.X (M X = R, interleaved) and its
// gradient into pc.grad; the loss goes to pc.coef[0]; pc.coef[8 .. 8 + K) must hold x_k^T M x_k
template <int C>
int net_loss_grad_t(lyap_ek* e, const TrainBufs& tb, cudaStream_t st) {
  EkPrec& pc = e->pc;
  const int64_t n = e->n;
  const int gr = grid_for(n) * 4;
  LYAP_CUDA_TRY(cudaMemsetAsync(pc.grad, 0, sizeof(double) * kNW, st));
  net_forward(e, st);
  const Vals v = vals_of(pc, 2);
  // U = B R (iterates kept), E = B^T U - X
  horner_fwd_store<C>(pc, v, n, tb.R, tb.Ur, tb.Yr, st);
  const double* y = tb.Yr[kQ];
  const double* w0 = y;
  for (int j = 0; j < kQ; ++j) {
    double* out = (j % 2 == 0) ? tb.T1 : tb.T2;
    k_h_bwd<C><<<gr, kT, 0, st>>>(y, w0, v, pc.g, out);
    w0 = out;
  }
  k_h_last<C><<<gr, kT, 0, st>>>(w0, v.d, tb.E, C, n);
  k_sub<<<gr, kT, 0, st>>>(tb.E, tb.X, n * C);
  // ME = M E (M = -A); loss terms and G = 2 M E / (K x^T M x)
  spmm(e->A, C, tb.E, C, tb.ME, C, -1.0, st);
  k_coldots<C><<<kGrid, kT, 0, st>>>(tb.E, tb.ME, n, e->partials);
  k_sum_partials<<<1, 64, 0, st>>>(e->partials, kGrid, C, pc.coef + 16);
  k_energy_terms<<<1, 32, 0, st>>>(pc.coef + 16, pc.coef + 8, C, pc.coef);
  k_scale_cols<<<gr, kT, 0, st>>>(tb.ME, pc.coef + 1, 0.0, C, n, tb.G);
  // B G (iterates kept); gradient of sum_k [(B r_k)^T B' g_k + (B g_k)^T B' r_k]
  horner_fwd_store<C>(pc, v, n, tb.G, tb.Ug, tb.Yg, st);
  LYAP_CUDA_TRY(cudaMemsetAsync(pc.gd, 0, sizeof(double) * n * 3, st));
  reverse_pass<C>(pc, v, n, tb.Yr[kQ], tb.Yg, tb.la, tb.lb, st);
  reverse_pass<C>(pc, v, n, tb.Yg[kQ], tb.Yr, tb.la, tb.lb, st);
  k_net_gy<<<gr, kT, 0, st>>>(pc.gd, pc.gw, pc.gs, pc.d1, vals_of(pc, 1), n, pc.gy);
  // back through the convolutions
  const int gp = (int)std::min<int64_t>((n + kT - 1) / kT, 4096);
  const int gm = (int)std::min<int64_t>(((n + 15) / 16 + kWarpsW - 1) / kWarpsW, 4096);
  const int nt = (int)((n + kTile - 1) / kTile);
  k_l3_bwd_data<<<gp, kT, 0, st>>>(pc.gy, pc.thq + oW3, pc.a2, pc.g, pc.g2);
  k_l3_bwd_w<<<nt, kT, 0, st>>>(pc.gy, pc.a2, pc.g, pc.wpart);
  k_rows_sum<<<(kNW3 + 127) / 128, 128, 0, st>>>(pc.wpart, nt, kNW3, pc.grad + oW3);
  k_l2_bwd_data<<<gm, 256, 0, st>>>(pc.g2, pc.thq + oW2, pc.a1, pc.g, pc.g1);
  k_l2_bwd_w<<<kL2WGrid, kWarpsW * 32, 0, st>>>(pc.g2, pc.a1, pc.g, pc.wpart);
  k_rows_sum<<<(kNW2 + 127) / 128, 128, 0, st>>>(pc.wpart, kL2WGrid * kWarpsW, kNW2, pc.grad + oW2);
  k_l1_bwd_w<<<nt, kT, 0, st>>>(pc.g1, pc.feats, pc.g, pc.wpart);
  k_rows_sum<<<(kNW1 + 127) / 128, 128, 0, st>>>(pc.wpart, nt, kNW1, pc.grad + oW1);
  return LYAP_OK;
}

int net_loss_grad(lyap_ek* e, int K, const TrainBufs& tb, cudaStream_t st) {
  switch (K) {
    case 1: return net_loss_grad_t<1>(e, tb, st);
    case 2: return net_loss_grad_t<2>(e, tb, st);
    case 3: return net_loss_grad_t<3>(e, tb, st);
    case 4: return net_loss_grad_t<4>(e, tb, st);
  }
  return LYAP_ERR_ARG;
}

// x_k^T M x_k of the pairs into pc.coef[8 .. 8 + K)
int pair_norms(lyap_ek* e, int K, const TrainBufs& tb, cudaStream_t st) {
  spmm(e->A, K, tb.X, K, tb.ME, K, -1.0, st);
  switch (K) {
    case 1: k_coldots<1><<<kGrid, kT, 0, st>>>(tb.X, tb.ME, e->n, e->partials); break;
    case 2: k_coldots<2><<<kGrid, kT, 0, st>>>(tb.X, tb.ME, e->n, e->partials); break;
    case 3: k_coldots<3><<<kGrid, kT, 0, st>>>(tb.X, tb.ME, e->n, e->partials); break;
    case 4: k_coldots<4><<<kGrid, kT, 0, st>>>(tb.X, tb.ME, e->n, e->partials); break;
    default: return LYAP_ERR_ARG;
  }
  k_sum_partials<<<1, 64, 0, st>>>(e->partials, kGrid, K, e->pc.coef + 8);
  return LYAP_OK;
}

// pairs (b_k, x_k) with A x_k = b_k, column-major n x K each, into tb.R = B and tb.X = -X (M = -A)
void load_pairs(lyap_ek* e, int K, const double* B, const double* X, const TrainBufs& tb, cudaStream_t st) {
  const int64_t n = e->n;
  const int g = (int)std::min<int64_t>((n + kT - 1) / kT, 8192);
  for (int c = 0; c < K; ++c) {
    k_copy_cols<<<g, kT, 0, st>>>(B + (size_t)c * n, 1, tb.R, K, c, 1, n, 1.0);
    k_copy_cols<<<g, kT, 0, st>>>(X + (size_t)c * n, 1, tb.X, K, c, 1, n, -1.0);
  }
}

void reset_params(lyap_ek* e, cudaStream_t st) {
  EkPrec& pc = e->pc;
  cudaMemcpyAsync(pc.th, pc.th_init, sizeof(float) * kNW, cudaMemcpyDeviceToDevice, st);
  cudaMemsetAsync(pc.m1, 0, sizeof(float) * 2 * kNW, st);
  k_cast_params<<<(kNW + 255) / 256, 256, 0, st>>>(pc.th, pc.thq, kNW);
  e->adam_t = 0;
}

// Adam steps on the stored pairs; the trained network is kept only if it lowered the loss below
// the initial one, which is IC(0)'s (the last layer starts at zero)
int net_train(lyap_ek* e, int iters, float lr, cudaStream_t st) {
  EkPrec& pc = e->pc;
  const int K = e->npairs;
  if (K < 1) return LYAP_ERR_ARG;
  const TrainBufs tb = train_bufs(e);
  load_pairs(e, K, e->pair_b, e->pair_x, tb, st);
  int rc = pair_norms(e, K, tb, st);
  if (rc != LYAP_OK) return rc;
  for (int it = 0; it <= iters; ++it) {
    rc = net_loss_grad(e, K, tb, st);
    if (rc != LYAP_OK) return rc;
    if (it == 0) LYAP_CUDA_TRY(cudaMemcpyAsync(&e->loss0, pc.coef, sizeof(double), cudaMemcpyDeviceToHost, st));
    if (it == iters) break;
    ++e->adam_t;
    k_adam<<<(kNW + 255) / 256, 256, 0, st>>>(pc.th, pc.grad, pc.m1, pc.m2, pc.thq, kNW, lr, 0.9f, 0.999f, 1e-8f,
                                              e->adam_t);
  }
  LYAP_CUDA_TRY(cudaMemcpyAsync(&e->loss1, pc.coef, sizeof(double), cudaMemcpyDeviceToHost, st));
  LYAP_CUDA_TRY(cudaStreamSynchronize(st));
  LYAP_CUDA_TRY(cudaGetLastError());
  e->trained = (std::isfinite(e->loss1) && e->loss1 < e->loss0) ? 1 : -1;
  return LYAP_OK;
}

// ---- preconditioned conjugate gradients for A X = B (s columns), on M = -A ------------------
// kind 0: Jacobi; 1: IC(0) by the truncated Neumann series; 2: the network's values, same application
template <int s>
int pcg_t(lyap_ek* e, const double* B, int ldb, int kind, int* its, cudaStream_t caller) {
  const int64_t n = e->n;
  const double tol2 = e->inner_tol * e->inner_tol;
  cudaStream_t st = e->cgs ? e->cgs : caller;
  if (e->cgs) {
    LYAP_CUDA_TRY(cudaEventRecord(e->cg_ev[0], caller));
    LYAP_CUDA_TRY(cudaStreamWaitEvent(st, e->cg_ev[0], 0));
  }
  k_cg_start<s><<<kGrid, kT, 0, st>>>(B, ldb, e->x, e->r, n, e->partials);
  k_sum_partials<<<1, 64, 0, st>>>(e->partials, kGrid, s, e->small);
  k_cg_conv<<<1, 32, 0, st>>>(e->small, e->sc, s, tol2, 1);
  auto precond = [&](int first) {
    if (kind != 0) {
      apply_P(e->pc, kind, s, n, e->r, s, e->z, s, st);
      k_cg_zdots<s><<<kGrid, kT, 0, st>>>(e->r, e->q, e->sc, e->z, n, first, e->partials);
    } else {
      k_cg_jacobi<s><<<kGrid, kT, 0, st>>>(e->mdinv, e->r, e->q, e->sc, e->z, n, first, e->partials);
    }
    k_sum_partials<<<1, 64, 0, st>>>(e->partials, kGrid, 2 * s, e->small);
    k_cg_beta<<<1, 32, 0, st>>>(e->small, e->sc, s, first);
  };
  auto iteration = [&]() {
    k_cg_matvec<s><<<kGrid, kT, 0, st>>>(e->A, e->p, e->q, e->partials);
    k_sum_partials<<<1, 64, 0, st>>>(e->partials, kGrid, s, e->small);
    k_cg_alpha<<<1, 32, 0, st>>>(e->small, e->sc, s);
    k_cg_update<s><<<kGrid, kT, 0, st>>>(e->x, e->r, e->p, e->q, e->sc, n, e->partials);
    k_sum_partials<<<1, 64, 0, st>>>(e->partials, kGrid, s, e->small);
    k_cg_conv<<<1, 32, 0, st>>>(e->small, e->sc, s, tol2, 0);
    precond(0);
    k_cg_dir<s><<<kGrid * 4, kT, 0, st>>>(e->z, e->p, e->sc, n);
  };
  constexpr int kBlock = 8;  // iterations between the host's convergence reads
  // the block of kBlock iterations as a graph: every argument is fixed per context and kind
  if (e->cgs && e->cg_state[kind] == 0) {
    cudaGraph_t g = nullptr;
    bool ok = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      for (int k = 0; k < kBlock; ++k) iteration();
      ok = cudaStreamEndCapture(st, &g) == cudaSuccess && g != nullptr;
    }
    ok = ok && cudaGraphInstantiate(&e->cg_graph[kind], g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    if (!ok) {
      e->cg_graph[kind] = nullptr;
      cudaGetLastError();  // a failed capture leaves no sticky error; the block runs as launches
    }
    e->cg_state[kind] = ok ? 1 : -1;
  }
  precond(1);
  LYAP_CUDA_TRY(cudaMemcpyAsync(e->p, e->z, sizeof(double) * n * s, cudaMemcpyDeviceToDevice, st));
  std::vector<double> hsc(kSc * s);
  int it = 0;
  for (; it < e->inner_maxit;) {
    if (e->cg_state[kind] == 1 && e->inner_maxit - it >= kBlock) {
      LYAP_CUDA_TRY(cudaGraphLaunch(e->cg_graph[kind], st));
      it += kBlock;
    } else {
      for (int k = 0; k < kBlock && it < e->inner_maxit; ++k, ++it) iteration();
    }
    LYAP_CUDA_TRY(cudaMemcpyAsync(hsc.data(), e->sc, sizeof(double) * kSc * s, cudaMemcpyDeviceToHost, st));
    LYAP_CUDA_TRY(cudaStreamSynchronize(st));
    LYAP_CUDA_TRY(cudaGetLastError());
    bool any = false;
    for (int c = 0; c < s; ++c) any = any || hsc[c * kSc + 5] != 0.0;
    if (!any) break;
  }
  if (e->cgs) {
    LYAP_CUDA_TRY(cudaEventRecord(e->cg_ev[1], st));
    LYAP_CUDA_TRY(cudaStreamWaitEvent(caller, e->cg_ev[1], 0));
  }
  *its = it;
  for (int c = 0; c < s; ++c)
    if (!std::isfinite(hsc[c * kSc + 3])) return LYAP_ERR_NONFINITE;
  return it >= e->inner_maxit ? LYAP_NOT_CONVERGED : LYAP_OK;
}

int pcg_once(lyap_ek* e, const double* B, int ldb, int kind, int* its, cudaStream_t st) {
  switch (e->s) {
    case 1: return pcg_t<1>(e, B, ldb, kind, its, st);
    case 2: return pcg_t<2>(e, B, ldb, kind, its, st);
    case 4: return pcg_t<4>(e, B, ldb, kind, its, st);
  }
  return LYAP_ERR_ARG;
}

// The network's solve is accepted when it reaches the inner tolerance within twice the iterations
// of the last IC(0) solve; otherwise (or when it went non-finite) the solve is redone with IC(0),
// which judges and backs up the network.  *used tells which preconditioner produced the solution.
int pcg(lyap_ek* e, const double* B, int ldb, int kind, int* its, int* used, cudaStream_t st) {
  *used = kind;
  if (kind == 2) {
    const int cap = e->inner_maxit;
    e->inner_maxit = std::min(cap, std::max(100, 2 * e->last_ic0_its));
    const int rc = pcg_once(e, B, ldb, 2, its, st);
    e->inner_maxit = cap;
    if (rc == LYAP_OK) return rc;
    ++e->fallbacks;
    kind = 1;
    *used = 1;
  }
  const int rc = pcg_once(e, B, ldb, kind, its, st);
  if (rc == LYAP_OK || rc == LYAP_NOT_CONVERGED) {
    if (kind == 1) e->last_ic0_its = *its;
    if (kind == 0) e->last_jacobi_its = *its;
  }
  return rc;
}

// solution X (n x s, in e->x) of A X = B into dst columns [off, off+s) (leading dimension ldd);
// keeps (B, X) as training pairs while there is room
void take_solution(lyap_ek* e, const double* B, int ldb, double* dst, int ldd, int off, bool keep, cudaStream_t st) {
  const int64_t n = e->n;
  const int g = (int)std::min<int64_t>((n * e->s + kT - 1) / kT, 8192);
  k_copy_cols<<<g, kT, 0, st>>>(e->x, e->s, dst, ldd, off, e->s, n, 1.0);
  if (!keep) return;
  for (int c = 0; c < e->s && e->npairs < e->L.pair_cap; ++c, ++e->npairs) {
    k_copy_cols<<<g, kT, 0, st>>>(B + c, ldb, e->pair_b + (size_t)e->npairs * n, 1, 0, 1, n, 1.0);
    k_copy_cols<<<g, kT, 0, st>>>(e->x + c, e->s, e->pair_x + (size_t)e->npairs * n, 1, 0, 1, n, 1.0);
  }
}

void init_params_host(std::vector<float>& th) {
  // the initialisation law of the network: w1 ~ normal(0, 0.1 / sqrt(5)), w2 ~ normal(0, 0.1 / 4),
  // zero biases, zero last layer (the preconditioner starts as IC(0) exactly); a fixed-seed
  // generator of this library (64-bit LCG, Box-Muller)
  th.assign(kNW, 0.f);
  unsigned long long st = 0x2545F4914F6CDD1DULL;
  auto uni = [&]() {
    st = st * 6364136223846793005ULL + 1442695040888963407ULL;
    return ((st >> 11) + 0.5) * (1.0 / 9007199254740992.0);
  };
  auto nrm = [&]() { return sqrt(-2.0 * log(uni())) * cos(6.283185307179586 * uni()); };
  for (int k = 0; k < kCh * kNin * 9; ++k) th[oW1 + k] = (float)(0.1 / sqrt((double)kNin) * nrm());
  for (int k = 0; k < kCh * kCh * 9; ++k) th[oW2 + k] = (float)(0.1 / 4.0 * nrm());
}

// stencil, IC(0) and the network's initial state on the grid; pc.status tells whether IC(0) exists
int prec_setup(lyap_ek* e, cudaStream_t st) {
  EkPrec& pc = e->pc;
  const int64_t n = e->n;
  char* c = e->ws + e->L.prec;
  auto take = [&](size_t bytes) { char* r2 = c; c += lyap_align256((int64_t)bytes); return r2; };
  pc.g = Grid{e->nx, e->ny};
  pc.sten = reinterpret_cast<double*>(take(sizeof(double) * n * 5));
  pc.piv = reinterpret_cast<double*>(take(sizeof(double) * n));
  pc.d0 = reinterpret_cast<double*>(take(sizeof(double) * n * 6));
  pc.lw0 = pc.d0 + n;
  pc.ls0 = pc.d0 + 2 * n;
  pc.d1 = pc.d0 + 3 * n;
  pc.lw1 = pc.d0 + 4 * n;
  pc.ls1 = pc.d0 + 5 * n;
  pc.feats = reinterpret_cast<float*>(take(sizeof(float) * n * kNin));
  pc.a1 = reinterpret_cast<__nv_bfloat16*>(take(sizeof(__nv_bfloat16) * n * kCh * 4));
  pc.a2 = pc.a1 + n * kCh;
  pc.g1 = pc.a1 + 2 * n * kCh;
  pc.g2 = pc.a1 + 3 * n * kCh;
  pc.y = reinterpret_cast<float*>(take(sizeof(float) * n * kNout * 2));
  pc.gy = pc.y + n * kNout;
  pc.gd = reinterpret_cast<double*>(take(sizeof(double) * n * 3));
  pc.gw = pc.gd + n;
  pc.gs = pc.gd + 2 * n;
  pc.train = reinterpret_cast<double*>(take(sizeof(double) * n * kPairCap * kTrainBlocks));
  pc.app = reinterpret_cast<double*>(take(sizeof(double) * n * 4 * 3));
  pc.th = reinterpret_cast<float*>(take(sizeof(float) * kNW * 4));
  pc.m1 = pc.th + kNW;
  pc.m2 = pc.th + 2 * kNW;
  pc.th_init = pc.th + 3 * kNW;
  pc.thq = reinterpret_cast<__nv_bfloat16*>(take(sizeof(__nv_bfloat16) * kNW));
  pc.grad = reinterpret_cast<double*>(take(sizeof(double) * kNW));
  pc.wpart = reinterpret_cast<double*>(take((size_t)wpart_rows_bytes(n)));
  pc.coef = reinterpret_cast<double*>(take(sizeof(double) * 32));
  pc.bad = reinterpret_cast<int*>(take(256));
  LYAP_CUDA_TRY(cudaMemsetAsync(pc.bad, 0, sizeof(int), st));
  k_stencil<<<grid_for(n) * 4, kT, 0, st>>>(e->A, pc.g, pc.sten, pc.feats, pc.bad);
  int bad = 0;
  LYAP_CUDA_TRY(cudaMemcpyAsync(&bad, pc.bad, sizeof(int), cudaMemcpyDeviceToHost, st));
  LYAP_CUDA_TRY(cudaStreamSynchronize(st));
  if (bad == 0 && e->nx <= 1024) {
    const int threads = (e->nx + 31) / 32 * 32;
    k_ic0_wave<<<1, threads, 0, st>>>(pc.sten, pc.g, pc.piv, pc.bad);
    k_ic0_vals<<<grid_for(n) * 4, kT, 0, st>>>(pc.sten, pc.piv, pc.g, pc.d0, pc.lw0, pc.ls0);
    LYAP_CUDA_TRY(cudaMemcpyAsync(&bad, pc.bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    LYAP_CUDA_TRY(cudaStreamSynchronize(st));
  } else if (bad == 0) {
    bad = 8;  // grids wider than one CTA: no IC(0)
  }
  pc.status = bad;
  std::vector<float> th;
  init_params_host(th);
  LYAP_CUDA_TRY(cudaMemcpyAsync(pc.th_init, th.data(), sizeof(float) * kNW, cudaMemcpyHostToDevice, st));
  reset_params(e, st);
  if (pc.status == 0) net_forward(e, st);
  LYAP_CUDA_TRY(cudaStreamSynchronize(st));
  return cudaGetLastError() == cudaSuccess ? LYAP_OK : LYAP_ERR_CUDA;
}

}  // namespace

extern "C" {

int lyap_ek_workspace_size(const lyap_csr* A, int s, int maxit, int nx, int ny, size_t* bytes) {
  if (!A || !bytes || (s != 1 && s != 2 && s != 4) || maxit < 1) return LYAP_ERR_ARG;
  int rc = validate_csr(A);
  if (rc != LYAP_OK) return rc;
  if (A->val_dtype != LYAP_F64) return LYAP_ERR_ARG;
  if (nx < 0 || ny < 0 || ((nx || ny) && (int64_t)nx * ny != A->n)) return LYAP_ERR_ARG;
  if (nx > 0 && A->n >= INT_MAX) return LYAP_ERR_ARG;  // grid kernels index nodes in 32 bits
  *bytes = ek_layout(A, s, maxit, nx > 0).total;
  return LYAP_OK;
}

}  // extern "C"

namespace {
// events and pinned host buffers of a context (the object itself stays)
void ek_release(lyap_ek* e) {
  for (int i = 0; i < 4; ++i)
    if (e->ev[i]) cudaEventDestroy(e->ev[i]);
  for (int k = 0; k < 3; ++k)
    if (e->cg_graph[k]) cudaGraphExecDestroy(e->cg_graph[k]);
  for (int k = 0; k < 2; ++k)
    if (e->cg_ev[k]) cudaEventDestroy(e->cg_ev[k]);
  if (e->cgs) cudaStreamDestroy(e->cgs);
  if (e->hk.ev[0]) cudaEventDestroy(e->hk.ev[0]);
  if (e->hk.ev[1]) cudaEventDestroy(e->hk.ev[1]);
  if (e->hk.hist_host) cudaFreeHost(e->hk.hist_host);
  if (e->hk.flags_host) cudaFreeHost(e->hk.flags_host);
}
}  // namespace

extern "C" {

int lyap_ek_destroy(lyap_ek* e) {
  if (!e) return LYAP_OK;
  ek_release(e);
  delete e;
  return LYAP_OK;
}

int lyap_ek_create(const lyap_csr* A, const double* C, int c_mem, int s, double tol, int maxit, double inner_tol, int nx,
                   int ny, void* workspace, size_t ws_bytes, void* stream, lyap_ek** out) {
  if (!out || !C || !(tol >= 0.0) || !(inner_tol > 0.0)) return LYAP_ERR_ARG;
  size_t need = 0;
  int rc = lyap_ek_workspace_size(A, s, maxit, nx, ny, &need);
  if (rc != LYAP_OK) return rc;
  if (!workspace || ws_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255)) return LYAP_ERR_WORKSPACE;
  if (c_mem != LYAP_MEM_DEVICE && c_mem != LYAP_MEM_HOST) return LYAP_ERR_ARG;
  lyap_ek* e = new (std::nothrow) lyap_ek();
  if (!e) return LYAP_ERR_ARG;
  auto fail = [&](int code) {
    lyap_ek_destroy(e);
    return code;
  };
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  e->s = s;
  e->S = 2 * s;
  e->maxit = maxit;
  e->n = A->n;
  e->nx = nx;
  e->ny = ny;
  e->tol = tol;
  e->inner_tol = inner_tol;
  e->L = ek_layout(A, s, maxit, nx > 0);
  e->ws = static_cast<char*>(workspace);
  const int64_t n = A->n;
  const int S = e->S;
  char* w = e->ws;
  // CSR copy (fp64 values)
  int64_t* rp = at<int64_t>(w, e->L.csr);
  int32_t* cl = reinterpret_cast<int32_t*>(reinterpret_cast<char*>(rp) + lyap_align256((int64_t)(sizeof(int64_t) * (n + 1) + 8)));
  double* vl = reinterpret_cast<double*>(reinterpret_cast<char*>(cl) + lyap_align256((int64_t)(sizeof(int32_t) * A->nnz)));
  const cudaMemcpyKind kind = A->mem == LYAP_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  if (cudaMemcpyAsync(rp, A->rowptr, sizeof(int64_t) * (n + 1), kind, st) != cudaSuccess ||
      cudaMemcpyAsync(cl, A->col, sizeof(int32_t) * A->nnz, kind, st) != cudaSuccess ||
      cudaMemcpyAsync(vl, A->val, sizeof(double) * A->nnz, kind, st) != cudaSuccess)
    return fail(LYAP_ERR_CUDA);
  e->A = Csr{n, rp, cl, vl};
  e->basis = at<double>(w, e->L.basis);
  e->AV = at<double>(w, e->L.AV);
  e->C = at<double>(w, e->L.C);
  e->mdinv = at<double>(w, e->L.mdinv);
  double* v = at<double>(w, e->L.vec);
  e->x = v;
  e->r = v + n * s;
  e->z = v + 2 * n * s;
  e->p = v + 3 * n * s;
  e->q = v + 4 * n * s;
  e->partials = at<double>(w, e->L.partials);
  e->small = at<double>(w, e->L.small);
  // small: [0, 32) reduction results, [32, 56) CG scalars, [64, 128) R of CholQR, [128, ...) P blocks
  e->sc = e->small + 32;
  e->dR = e->small + 64;
  e->P = e->small + 128;
  e->log = at<double>(w, e->L.log);
  e->pair_b = at<double>(w, e->L.pairs);
  e->pair_x = e->pair_b + (size_t)n * e->L.pair_cap;
  if (cudaMemcpyAsync(e->C, C, sizeof(double) * n * s,
                      c_mem == LYAP_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return fail(LYAP_ERR_CUDA);
  k_mdinv<<<grid_for(n) * 4, kT, 0, st>>>(e->A, e->mdinv);
  if (nx > 0) {
    rc = prec_setup(e, st);
    if (rc != LYAP_OK) return fail(rc);
  }
  // the check and factor view
  lyap_handle& hk = e->hk;
  hk.plan.s = S;
  hk.plan.sylv = 0;
  hk.plan.bulk = LYAP_PREC_F64;
  hk.plan.maxit = maxit;
  hk.plan.nmax = S * maxit;
  hk.plan.check_batch = 1;
  hk.plan.check_batch_req = 1;
  hk.plan.factor_bytes = e->L.factor_bytes;
  hk.s = S;
  hk.tol = tol;
  lyap_default_options(&hk.opt);
  hk.opt.maxit = maxit;
  hk.op[0].n = n;
  hk.op[0].log = e->log;
  hk.hist = at<double>(w, e->L.hist);
  hk.flags = at<int>(w, e->L.flags);
  hk.chk_err = at<int>(w, e->L.chk);
  hk.check_ws = w + e->L.check;
  hk.factor_ws = w + e->L.factor;
  for (int i = 0; i < 8; ++i) hk.ev[i] = nullptr;
  if (cudaEventCreate(&hk.ev[0]) != cudaSuccess || cudaEventCreate(&hk.ev[1]) != cudaSuccess) return fail(LYAP_ERR_CUDA);
  for (int i = 0; i < 4; ++i)
    if (cudaEventCreate(&e->ev[i]) != cudaSuccess) return fail(LYAP_ERR_CUDA);
  if (cudaStreamCreateWithFlags(&e->cgs, cudaStreamNonBlocking) != cudaSuccess) return fail(LYAP_ERR_CUDA);
  for (int i = 0; i < 2; ++i)
    if (cudaEventCreateWithFlags(&e->cg_ev[i], cudaEventDisableTiming) != cudaSuccess) return fail(LYAP_ERR_CUDA);
  if (cudaMallocHost(&hk.hist_host, sizeof(double) * maxit) != cudaSuccess) return fail(LYAP_ERR_CUDA);
  if (cudaMallocHost(&hk.flags_host, sizeof(int) * 8) != cudaSuccess) return fail(LYAP_ERR_CUDA);
  if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess) return fail(LYAP_ERR_CUDA);
  *out = e;
  return LYAP_OK;
}

int lyap_ek_precond_status(lyap_ek* e) { return e ? (e->nx > 0 ? e->pc.status : -1) : -1; }

// precond: 0 Jacobi, 1 IC(0), 2 the network (the first train_solves inner solves use IC(0) and
// provide its training pairs, then train_iters Adam steps with learning rate lr)
int lyap_ek_solve(lyap_ek* e, int precond, int train_solves, int train_iters, float lr, void* stream) {
  if (!e || precond < 0 || precond > 2) return LYAP_ERR_ARG;
  if (precond > 0 && (e->nx == 0 || e->pc.status != 0)) return LYAP_ERR_ARG;
  if (precond == 2 && (train_solves < 1 || train_iters < 0 || !(lr > 0.f))) return LYAP_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t n = e->n;
  const int s = e->s, S = e->S;
  lyap_handle& hk = e->hk;
  cudaEventRecord(e->ev[0], st);
  k_init_ek<<<(e->maxit + 255) / 256, 256, 0, st>>>(hk.hist, hk.flags, hk.chk_err, e->maxit);
  LYAP_CUDA_TRY(cudaMemsetAsync(e->log, 0, sizeof(double) * (size_t)(e->maxit + 1) * LOG_NREC * S * S, st));
  e->inner_its.clear();
  e->inner_kind.clear();
  e->npairs = 0;
  e->trained = 0;
  e->loss0 = e->loss1 = -1.0;
  e->last_ic0_its = 0;
  hk.solved = 0;
  hk.factored = 0;
  if (precond == 2) reset_params(e, st);
  float t_train = 0.f;
  // beta = ||C||_F
  k_dot2<<<kGrid, kT, 0, st>>>(e->C, e->C, e->C, n * s, e->partials);
  k_sum_partials<<<1, 64, 0, st>>>(e->partials, kGrid, 2, e->small);
  double bb[2];
  LYAP_CUDA_TRY(cudaMemcpyAsync(bb, e->small, sizeof(bb), cudaMemcpyDeviceToHost, st));
  LYAP_CUDA_TRY(cudaStreamSynchronize(st));
  const double beta = sqrt(bb[0]);
  auto kind_now = [&]() { return precond == 2 ? (e->trained == 1 ? 2 : 1) : precond; };
  auto collect = [&]() { return precond == 2 && e->trained == 0 && (int)e->inner_its.size() < train_solves; };
  // [C, A^{-1} C] = V_1 gamma
  double* V1 = e->basis;
  const int gcp = (int)std::min<int64_t>((n * S + kT - 1) / kT, 8192);
  k_copy_cols<<<gcp, kT, 0, st>>>(e->C, s, V1, S, 0, s, n, 1.0);
  int its = 0, used = 0;
  e->fallbacks = 0;
  const bool keep0 = collect();
  int rc = pcg(e, e->C, s, kind_now(), &its, &used, st);
  if (rc == LYAP_ERR_NONFINITE) return rc;
  e->inner_its.push_back(its);
  e->inner_kind.push_back(used);
  take_solution(e, e->C, s, V1, S, s, keep0, st);
  std::vector<double> gamma;
  rc = cholqr2(e, V1, gamma, st);
  if (rc != LYAP_OK) return rc;
  {
    // record 0: gamma_1 = gamma(:, 1:s) padded with zero columns, beta
    std::vector<double> rec(LOG_NREC * S * S, 0.0);
    for (int a = 0; a < S; ++a)
      for (int b = 0; b < s; ++b) rec[REC_TNEXT * S * S + a * S + b] = gamma[a * S + b];
    rec[REC_TDIAG * S * S] = beta;
    LYAP_CUDA_TRY(cudaMemcpyAsync(e->log, rec.data(), sizeof(double) * rec.size(), cudaMemcpyHostToDevice, st));
    LYAP_CUDA_TRY(cudaStreamSynchronize(st));
  }
  int result = LYAP_NOT_CONVERGED, m_final = e->maxit, done = 0;
  for (int j = 1; j <= e->maxit; ++j) {
    if (precond == 2 && e->trained == 0 && (int)e->inner_its.size() >= train_solves) {
      cudaEventRecord(e->ev[2], st);
      rc = net_train(e, train_iters, lr, st);
      if (rc != LYAP_OK) return rc;
      cudaEventRecord(e->ev[3], st);
      LYAP_CUDA_TRY(cudaStreamSynchronize(st));
      cudaEventElapsedTime(&t_train, e->ev[2], e->ev[3]);
    }
    double* Vj = e->basis + (size_t)(j - 1) * n * S;
    double* Vn = e->basis + (size_t)j * n * S;
    spmm(e->A, S, Vj, S, e->AV, S, 1.0, st);
    k_copy_cols<<<gcp, kT, 0, st>>>(e->AV, S, Vn, S, 0, s, n, 1.0);
    const bool keep = collect();
    rc = pcg(e, Vj + s, S, kind_now(), &its, &used, st);
    if (rc == LYAP_ERR_NONFINITE) return rc;
    e->inner_its.push_back(its);
    e->inner_kind.push_back(used);
    take_solution(e, Vj + s, S, Vn, S, s, keep, st);
    // block Gram-Schmidt against every stored block, twice, then CholQR2
    for (int pass = 0; pass < 2; ++pass) {
      project(e, e->basis, j, Vn, st);
      subtract(e, e->basis, j, Vn, st);
    }
    rc = cholqr2(e, Vn, gamma, st);
    if (rc != LYAP_OK) return rc;
    // tau_jj = V_j^T A V_j, tau_{j+1,j} = V_{j+1}^T A V_j  (V_j, V_{j+1} are consecutive blocks)
    project(e, Vj, 2, e->AV, st);
    double* rec = e->log + (size_t)j * LOG_NREC * S * S;
    LYAP_CUDA_TRY(cudaMemcpyAsync(rec + REC_TDIAG * S * S, e->P, sizeof(double) * S * S, cudaMemcpyDeviceToDevice, st));
    LYAP_CUDA_TRY(cudaMemcpyAsync(rec + REC_TNEXT * S * S, e->P + S * S, sizeof(double) * S * S, cudaMemcpyDeviceToDevice, st));
    // the convergence check at m = j (Prop. 3.1, Alg. 3 with block size 2s)
    launch_check_batch(&hk, j, j, st);
    LYAP_CUDA_TRY(cudaMemcpyAsync(hk.flags_host, hk.flags, sizeof(int) * 3, cudaMemcpyDeviceToHost, st));
    LYAP_CUDA_TRY(cudaStreamSynchronize(st));
    LYAP_CUDA_TRY(cudaGetLastError());
    done = j;
    hk.lanczos_done = j;
    const int rs = round_status(&hk);
    if (rs != LYAP_OK) return rs;
    if (hk.flags_host[1] != INT_MAX) {
      m_final = hk.flags_host[1];
      result = LYAP_OK;
      break;
    }
  }
  e->m = m_final;
  e->done = done;
  rc = solve_end(&hk, done, m_final, result, st);
  if (rc != LYAP_OK) return rc;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e->ev[0], hk.ev[1]);
  e->times[0] = ms;
  e->times[1] = t_train;
  return result;
}

int lyap_ek_residual_norm(lyap_ek* e, double* hist, int cap, int* m_out) {
  if (!e) return LYAP_ERR_ARG;
  return lyap_residual_norm(&e->hk, hist, cap, m_out);
}

int lyap_ek_factor(lyap_ek* e, double* Z, int64_t ldz, int tcap, int* t_out, void* stream) {
  if (!e || !Z || !t_out || !e->hk.solved || ldz < tcap) return LYAP_ERR_ARG;
  return run_factor_basis(&e->hk, e->basis, e->n, Z, ldz, tcap, t_out, static_cast<cudaStream_t>(stream));
}

// out[0] solve ms, [1] training ms, [2] loss before training, [3] after, [4] inner solves ns,
// [5] network solves redone with IC(0), [6] 1 when the trained network was accepted, then the ns
// iteration counts and the ns preconditioner kinds (0 Jacobi, 1 IC(0), 2 network) up to cap
int lyap_ek_stats(lyap_ek* e, double* out, int cap) {
  if (!e || !out) return LYAP_ERR_ARG;
  const int ns = (int)e->inner_its.size();
  const double head[7] = {e->times[0], e->times[1], e->loss0, e->loss1, (double)ns, (double)e->fallbacks,
                          e->trained == 1 ? 1.0 : 0.0};
  int k = 0;
  for (; k < 7 && k < cap; ++k) out[k] = head[k];
  for (int i = 0; i < ns && k < cap; ++i, ++k) out[k] = (double)e->inner_its[i];
  for (int i = 0; i < ns && k < cap; ++i, ++k) out[k] = (double)e->inner_kind[i];
  return LYAP_OK;
}

// energy-norm loss and gradient of the network for caller parameters over caller pairs
int lyap_ek_net_grad(lyap_ek* e, const float* params, int K, const double* B, const double* X, double* loss,
                     double* grad, void* stream) {
  if (!e || !params || K < 1 || K > kPairCap || !B || !X || !loss || !grad || e->nx == 0 || e->pc.status != 0)
    return LYAP_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  EkPrec& pc = e->pc;
  LYAP_CUDA_TRY(cudaMemcpyAsync(pc.th, params, sizeof(float) * kNW, cudaMemcpyHostToDevice, st));
  k_cast_params<<<(kNW + 255) / 256, 256, 0, st>>>(pc.th, pc.thq, kNW);
  const TrainBufs tb = train_bufs(e);
  load_pairs(e, K, B, X, tb, st);
  int rc = pair_norms(e, K, tb, st);
  if (rc == LYAP_OK) rc = net_loss_grad(e, K, tb, st);
  if (rc != LYAP_OK) return rc;
  LYAP_CUDA_TRY(cudaMemcpyAsync(grad, pc.grad, sizeof(double) * kNW, cudaMemcpyDeviceToHost, st));
  LYAP_CUDA_TRY(cudaMemcpyAsync(loss, pc.coef, sizeof(double), cudaMemcpyDeviceToHost, st));
  LYAP_CUDA_TRY(cudaStreamSynchronize(st));
  return cudaGetLastError() == cudaSuccess ? LYAP_OK : LYAP_ERR_CUDA;
}

// Z = P_q R for K columns (device, column-major n x K each) with the IC(0) values (kind 1) or the
// network's (kind 2; params: host parameters to evaluate it with, or NULL for the current ones)
int lyap_ek_precond_apply(lyap_ek* e, int kind, const float* params, int K, const double* R, double* Z, void* stream) {
  if (!e || (kind != 1 && kind != 2) || K < 1 || K > 4 || !R || !Z || e->nx == 0 || e->pc.status != 0)
    return LYAP_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  EkPrec& pc = e->pc;
  if (kind == 2 && params) {
    LYAP_CUDA_TRY(cudaMemcpyAsync(pc.th, params, sizeof(float) * kNW, cudaMemcpyHostToDevice, st));
    k_cast_params<<<(kNW + 255) / 256, 256, 0, st>>>(pc.th, pc.thq, kNW);
    net_forward(e, st);
  }
  const int64_t n = e->n;
  const TrainBufs tb = train_bufs(e);
  const int g = (int)std::min<int64_t>((n + kT - 1) / kT, 8192);
  for (int c = 0; c < K; ++c) k_copy_cols<<<g, kT, 0, st>>>(R + (size_t)c * n, 1, tb.R, K, c, 1, n, 1.0);
  apply_P(pc, kind, K, n, tb.R, K, tb.X, K, st);
  for (int c = 0; c < K; ++c) k_copy_cols<<<g, kT, 0, st>>>(tb.X + c, K, Z + (size_t)c * n, 1, 0, 1, n, 1.0);
  LYAP_CUDA_TRY(cudaStreamSynchronize(st));
  return cudaGetLastError() == cudaSuccess ? LYAP_OK : LYAP_ERR_CUDA;
}

// the factor values (d, lw, ls; host arrays of n) of IC(0) (kind 1) or of the network (kind 2)
int lyap_ek_precond_values(lyap_ek* e, int kind, double* d, double* lw, double* ls) {
  if (!e || (kind != 1 && kind != 2) || !d || !lw || !ls || e->nx == 0 || e->pc.status != 0) return LYAP_ERR_ARG;
  const Vals v = vals_of(e->pc, kind);
  const size_t b = sizeof(double) * e->n;
  LYAP_CUDA_TRY(cudaMemcpy(d, v.d, b, cudaMemcpyDeviceToHost));
  LYAP_CUDA_TRY(cudaMemcpy(lw, v.lw, b, cudaMemcpyDeviceToHost));
  LYAP_CUDA_TRY(cudaMemcpy(ls, v.ls, b, cudaMemcpyDeviceToHost));
  return LYAP_OK;
}

int lyap_ek_param_count(void) { return kNW; }

int lyap_ek_projected_matrix(lyap_ek* e, int m, double* ab, int ldab, double* gamma, double* tau_next) {
  if (!e) return LYAP_ERR_ARG;
  return lyap_projected_matrix(&e->hk, 0, m, ab, ldab, gamma, tau_next);
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// Generalised Lyapunov equation A X E + E X A + C C^T = 0 with E symmetric positive definite (the
// mass-matrix example of Sec. 6).  With E = L L^T it is the standard equation for
// A~ = L^{-1} A L^{-T} and C~ = L^{-1} C, whose solution is X~ = L^T X L.  L is never formed: the
// block Lanczos basis of A~ is V~ = L^T V with V E-orthonormal (V^T E V = I) spanning the Krylov
// space of E^{-1} A from E^{-1} C.  Then T_m = V~^T A~ V~ = V^T A V, C~ = V~_1 gamma with
// C = E V_1 gamma, and the relation A~ V~_m = V~_m T_m + V~_{m+1} tau E_m^T holds, so the check
// (Prop. 3.1 / Alg. 3) is the standard one on T_m and measures the transformed residual, and the
// factor is Z = V_m (Q Ycheck) directly, since X = L^{-T} X~ L^{-1} = V Y V^T.
// Step j: W = E^{-1} A V_j by conjugate gradients on E (Jacobi preconditioned; E is well
// conditioned), E-orthogonalisation against every stored block twice (coefficients V_i^T (E W)
// with E W by a sparse product), E-CholQR2, and tau_jj = V_j^T A V_j, tau_{j+1,j} = V_{j+1}^T A V_j.
// The basis is stored: replaying the recurrence from the logged coefficients drifts on these
// operators, so the factor is accumulated from the stored blocks.
struct lyap_gen {
  lyap_ek e;      // the CG solves (e.A = -E), block Gram-Schmidt, the check and factor view
  Csr Aop{};      // A
  double* EW = nullptr;
  size_t total = 0;
  int iters = 0, solves = 0, max_iters = 0;
};

namespace {

struct GenLayout {
  size_t csrA = 0, csrE = 0, basis = 0, AV = 0, EW = 0, C = 0, mdinv = 0, vec = 0, partials = 0, small = 0, log = 0,
         hist = 0, flags = 0, chk = 0, check = 0, factor = 0, total = 0;
  size_t factor_bytes = 0;
};

GenLayout gen_layout(const lyap_csr* A, const lyap_csr* E, int s, int maxit) {
  GenLayout G;
  const int64_t n = A->n;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t r = off; off += lyap_align256((int64_t)bytes); return r; };
  G.csrA = take(sizeof(int64_t) * (n + 1) + 8);
  take(sizeof(int32_t) * A->nnz);
  take(sizeof(double) * A->nnz);
  G.csrE = take(sizeof(int64_t) * (n + 1) + 8);
  take(sizeof(int32_t) * E->nnz);
  take(sizeof(double) * E->nnz);
  G.basis = take(sizeof(double) * (size_t)(maxit + 1) * n * s);
  G.AV = take(sizeof(double) * n * s);
  G.EW = take(sizeof(double) * n * s);
  G.C = take(sizeof(double) * n * s);
  G.mdinv = take(sizeof(double) * n);
  G.vec = take(sizeof(double) * n * s * 5);
  G.partials = take(sizeof(double) * (size_t)kGrid * (maxit + 2) * s * s);
  G.small = take(sizeof(double) * ((size_t)(maxit + 2) * s * s + 128));
  G.log = take(sizeof(double) * (size_t)(maxit + 1) * LOG_NREC * s * s);
  G.hist = take(sizeof(double) * maxit);
  G.flags = take(256);
  G.chk = take(sizeof(int) * maxit);
  G.check = take(std::max(check_slot_bytes(s, s * maxit), (size_t)1 << 20));
  G.factor_bytes = factor_ws_bytes(s, s * maxit, 0);
  G.factor = take(G.factor_bytes);
  G.total = off;
  return G;
}

__global__ void k_scale(double* __restrict__ v, int64_t n, double a) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) v[i] *= a;
}

// CSR arrays into the workspace at offset off (fp64 values, scaled by sgn)
int copy_csr(const lyap_csr* A, char* w, size_t off, double sgn, Csr* out, cudaStream_t st) {
  const int64_t n = A->n;
  int64_t* rp = at<int64_t>(w, off);
  int32_t* cl = reinterpret_cast<int32_t*>(reinterpret_cast<char*>(rp) + lyap_align256((int64_t)(sizeof(int64_t) * (n + 1) + 8)));
  double* vl = reinterpret_cast<double*>(reinterpret_cast<char*>(cl) + lyap_align256((int64_t)(sizeof(int32_t) * A->nnz)));
  const cudaMemcpyKind kind = A->mem == LYAP_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  if (cudaMemcpyAsync(rp, A->rowptr, sizeof(int64_t) * (n + 1), kind, st) != cudaSuccess ||
      cudaMemcpyAsync(cl, A->col, sizeof(int32_t) * A->nnz, kind, st) != cudaSuccess ||
      cudaMemcpyAsync(vl, A->val, sizeof(double) * A->nnz, kind, st) != cudaSuccess)
    return LYAP_ERR_CUDA;
  if (sgn != 1.0) k_scale<<<grid_for(A->nnz) * 4, kT, 0, st>>>(vl, A->nnz, sgn);
  *out = Csr{n, rp, cl, vl};
  return LYAP_OK;
}

// W (n x s) E-orthonormalised twice (CholQR2 with Gram matrices W^T (E W)); gamma = R2 R1 (host)
int cholqr2_E(lyap_gen* g, double* Wm, std::vector<double>& gamma, cudaStream_t st) {
  lyap_ek* e = &g->e;
  const int S = e->S;
  std::vector<double> G(S * S), R(S * S), acc(S * S, 0.0);
  for (int pass = 0; pass < 2; ++pass) {
    spmm(e->A, S, Wm, S, g->EW, S, -1.0, st);  // E W (e->A holds -E)
    project(e, Wm, 1, g->EW, st);
    LYAP_CUDA_TRY(cudaMemcpyAsync(G.data(), e->P, sizeof(double) * S * S, cudaMemcpyDeviceToHost, st));
    LYAP_CUDA_TRY(cudaStreamSynchronize(st));
    if (!chol_upper_host(G.data(), R.data(), S)) return LYAP_ERR_BREAKDOWN;
    LYAP_CUDA_TRY(cudaMemcpyAsync(e->dR, R.data(), sizeof(double) * S * S, cudaMemcpyHostToDevice, st));
    const int gt = grid_for(e->n) * 4;
    switch (S) {
      case 1: k_trsm<1><<<gt, kT, 0, st>>>(Wm, e->n, e->dR); break;
      case 2: k_trsm<2><<<gt, kT, 0, st>>>(Wm, e->n, e->dR); break;
      case 4: k_trsm<4><<<gt, kT, 0, st>>>(Wm, e->n, e->dR); break;
    }
    if (pass == 0) acc = R;
    else {
      std::vector<double> t(S * S, 0.0);
      for (int i = 0; i < S; ++i)
        for (int j = 0; j < S; ++j)
          for (int k = 0; k < S; ++k) t[i * S + j] += R[i * S + k] * acc[k * S + j];
      acc = t;
    }
    LYAP_CUDA_TRY(cudaStreamSynchronize(st));  // dR is reused
  }
  gamma = acc;
  return LYAP_OK;
}

// dst <- E^{-1} B (n x s) by conjugate gradients on E; counts the iterations
int solve_E(lyap_gen* g, const double* B, double* dst, cudaStream_t st) {
  lyap_ek* e = &g->e;
  int its = 0, used = 0;
  const int rc = pcg(e, B, e->s, 0, &its, &used, st);  // (-E) X = B
  if (rc == LYAP_ERR_NONFINITE) return rc;
  g->iters += its;
  g->solves += 1;
  g->max_iters = std::max(g->max_iters, its);
  if (rc == LYAP_NOT_CONVERGED) return LYAP_ERR_BREAKDOWN;  // an E-solve short of its tolerance
  const int gcp = (int)std::min<int64_t>((e->n * e->s + kT - 1) / kT, 8192);
  k_copy_cols<<<gcp, kT, 0, st>>>(e->x, e->s, dst, e->s, 0, e->s, e->n, -1.0);
  return LYAP_OK;
}

}  // namespace

extern "C" {

int lyap_gen_workspace_size(const lyap_csr* A, const lyap_csr* E, int s, int maxit, size_t* bytes) {
  if (!A || !E || !bytes || (s != 1 && s != 2 && s != 4) || maxit < 1) return LYAP_ERR_ARG;
  int rc = validate_csr(A);
  if (rc == LYAP_OK) rc = validate_csr(E);
  if (rc != LYAP_OK) return rc;
  if (A->val_dtype != LYAP_F64 || E->val_dtype != LYAP_F64 || E->n != A->n) return LYAP_ERR_ARG;
  *bytes = gen_layout(A, E, s, maxit).total;
  return LYAP_OK;
}

int lyap_gen_destroy(lyap_gen* g) {
  if (!g) return LYAP_OK;
  ek_release(&g->e);
  delete g;
  return LYAP_OK;
}

int lyap_gen_create(const lyap_csr* A, const lyap_csr* E, const double* C, int c_mem, int s, double tol, int maxit,
                    double inner_tol, void* workspace, size_t ws_bytes, void* stream, lyap_gen** out) {
  if (!out || !C || !(tol >= 0.0) || !(inner_tol > 0.0)) return LYAP_ERR_ARG;
  size_t need = 0;
  int rc = lyap_gen_workspace_size(A, E, s, maxit, &need);
  if (rc != LYAP_OK) return rc;
  if (!workspace || ws_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255)) return LYAP_ERR_WORKSPACE;
  if (c_mem != LYAP_MEM_DEVICE && c_mem != LYAP_MEM_HOST) return LYAP_ERR_ARG;
  lyap_gen* g = new (std::nothrow) lyap_gen();
  if (!g) return LYAP_ERR_ARG;
  auto fail = [&](int code) {
    lyap_gen_destroy(g);
    return code;
  };
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const GenLayout G = gen_layout(A, E, s, maxit);
  lyap_ek* e = &g->e;
  e->s = s;
  e->S = s;
  e->maxit = maxit;
  e->n = A->n;
  e->tol = tol;
  e->inner_tol = inner_tol;
  e->ws = static_cast<char*>(workspace);
  g->total = G.total;
  const int64_t n = A->n;
  char* w = e->ws;
  if (copy_csr(A, w, G.csrA, 1.0, &g->Aop, st) != LYAP_OK || copy_csr(E, w, G.csrE, -1.0, &e->A, st) != LYAP_OK)
    return fail(LYAP_ERR_CUDA);
  e->basis = at<double>(w, G.basis);
  e->AV = at<double>(w, G.AV);
  g->EW = at<double>(w, G.EW);
  e->C = at<double>(w, G.C);
  e->mdinv = at<double>(w, G.mdinv);
  double* v = at<double>(w, G.vec);
  e->x = v;
  e->r = v + n * s;
  e->z = v + 2 * n * s;
  e->p = v + 3 * n * s;
  e->q = v + 4 * n * s;
  e->partials = at<double>(w, G.partials);
  e->small = at<double>(w, G.small);
  e->sc = e->small + 32;
  e->dR = e->small + 64;
  e->P = e->small + 128;
  e->log = at<double>(w, G.log);
  if (cudaMemcpyAsync(e->C, C, sizeof(double) * n * s,
                      c_mem == LYAP_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return fail(LYAP_ERR_CUDA);
  k_mdinv<<<grid_for(n) * 4, kT, 0, st>>>(e->A, e->mdinv);  // 1 / diag(E)
  lyap_handle& hk = e->hk;
  hk.plan.s = s;
  hk.plan.sylv = 0;
  hk.plan.bulk = LYAP_PREC_F64;
  hk.plan.maxit = maxit;
  hk.plan.nmax = s * maxit;
  hk.plan.check_batch = 1;
  hk.plan.check_batch_req = 1;
  hk.plan.factor_bytes = G.factor_bytes;
  hk.s = s;
  hk.tol = tol;
  lyap_default_options(&hk.opt);
  hk.opt.maxit = maxit;
  hk.op[0].n = n;
  hk.op[0].log = e->log;
  hk.hist = at<double>(w, G.hist);
  hk.flags = at<int>(w, G.flags);
  hk.chk_err = at<int>(w, G.chk);
  hk.check_ws = w + G.check;
  hk.factor_ws = w + G.factor;
  for (int i = 0; i < 8; ++i) hk.ev[i] = nullptr;
  if (cudaEventCreate(&hk.ev[0]) != cudaSuccess || cudaEventCreate(&hk.ev[1]) != cudaSuccess) return fail(LYAP_ERR_CUDA);
  for (int i = 0; i < 4; ++i)
    if (cudaEventCreate(&e->ev[i]) != cudaSuccess) return fail(LYAP_ERR_CUDA);
  if (cudaStreamCreateWithFlags(&e->cgs, cudaStreamNonBlocking) != cudaSuccess) return fail(LYAP_ERR_CUDA);
  for (int i = 0; i < 2; ++i)
    if (cudaEventCreateWithFlags(&e->cg_ev[i], cudaEventDisableTiming) != cudaSuccess) return fail(LYAP_ERR_CUDA);
  if (cudaMallocHost(&hk.hist_host, sizeof(double) * maxit) != cudaSuccess) return fail(LYAP_ERR_CUDA);
  if (cudaMallocHost(&hk.flags_host, sizeof(int) * 8) != cudaSuccess) return fail(LYAP_ERR_CUDA);
  if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess) return fail(LYAP_ERR_CUDA);
  *out = g;
  return LYAP_OK;
}

int lyap_gen_solve(lyap_gen* g, void* stream) {
  if (!g) return LYAP_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  lyap_ek* e = &g->e;
  const int64_t n = e->n;
  const int s = e->s, SS = s * s;
  lyap_handle& hk = e->hk;
  cudaEventRecord(e->ev[0], st);
  k_init_ek<<<(e->maxit + 255) / 256, 256, 0, st>>>(hk.hist, hk.flags, hk.chk_err, e->maxit);
  LYAP_CUDA_TRY(cudaMemsetAsync(e->log, 0, sizeof(double) * (size_t)(e->maxit + 1) * LOG_NREC * SS, st));
  hk.solved = 0;
  hk.factored = 0;
  g->iters = g->solves = g->max_iters = 0;
  // V_1 gamma = E^{-1} C with V_1 E-orthonormal: C = E V_1 gamma, C~ = V~_1 gamma
  double* V1 = e->basis;
  int rc = solve_E(g, e->C, V1, st);
  if (rc != LYAP_OK) return rc;
  std::vector<double> gamma;
  rc = cholqr2_E(g, V1, gamma, st);
  if (rc != LYAP_OK) return rc;
  {
    // record 0: gamma and beta = ||C~||_F = ||gamma||_F
    double b2 = 0.0;
    for (double x : gamma) b2 += x * x;
    std::vector<double> rec(LOG_NREC * SS, 0.0);
    for (int k = 0; k < SS; ++k) rec[REC_TNEXT * SS + k] = gamma[k];
    rec[REC_TDIAG * SS] = sqrt(b2);
    LYAP_CUDA_TRY(cudaMemcpyAsync(e->log, rec.data(), sizeof(double) * rec.size(), cudaMemcpyHostToDevice, st));
    LYAP_CUDA_TRY(cudaStreamSynchronize(st));
  }
  int result = LYAP_NOT_CONVERGED, m_final = e->maxit, done = 0;
  for (int j = 1; j <= e->maxit; ++j) {
    double* Vj = e->basis + (size_t)(j - 1) * n * s;
    double* Vn = e->basis + (size_t)j * n * s;
    spmm(g->Aop, s, Vj, s, e->AV, s, 1.0, st);  // A V_j
    rc = solve_E(g, e->AV, Vn, st);            // W = E^{-1} A V_j
    if (rc != LYAP_OK) return rc;
    // E-orthogonalisation against every stored block, twice, then E-CholQR2
    for (int pass = 0; pass < 2; ++pass) {
      spmm(e->A, s, Vn, s, g->EW, s, -1.0, st);
      project(e, e->basis, j, g->EW, st);
      subtract(e, e->basis, j, Vn, st);
    }
    rc = cholqr2_E(g, Vn, gamma, st);
    if (rc != LYAP_OK) return rc;
    // tau_jj = V_j^T A V_j, tau_{j+1,j} = V_{j+1}^T A V_j (consecutive blocks)
    project(e, Vj, 2, e->AV, st);
    double* rec = e->log + (size_t)j * LOG_NREC * SS;
    LYAP_CUDA_TRY(cudaMemcpyAsync(rec + REC_TDIAG * SS, e->P, sizeof(double) * SS, cudaMemcpyDeviceToDevice, st));
    LYAP_CUDA_TRY(cudaMemcpyAsync(rec + REC_TNEXT * SS, e->P + SS, sizeof(double) * SS, cudaMemcpyDeviceToDevice, st));
    launch_check_batch(&hk, j, j, st);
    LYAP_CUDA_TRY(cudaMemcpyAsync(hk.flags_host, hk.flags, sizeof(int) * 3, cudaMemcpyDeviceToHost, st));
    LYAP_CUDA_TRY(cudaStreamSynchronize(st));
    LYAP_CUDA_TRY(cudaGetLastError());
    done = j;
    hk.lanczos_done = j;
    const int rs = round_status(&hk);
    if (rs != LYAP_OK) return rs;
    if (hk.flags_host[1] != INT_MAX) {
      m_final = hk.flags_host[1];
      result = LYAP_OK;
      break;
    }
  }
  e->m = m_final;
  e->done = done;
  rc = solve_end(&hk, done, m_final, result, st);
  if (rc != LYAP_OK) return rc;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e->ev[0], hk.ev[1]);
  e->times[0] = ms;
  return result;
}

int lyap_gen_residual_norm(lyap_gen* g, double* hist, int cap, int* m_out) {
  if (!g) return LYAP_ERR_ARG;
  return lyap_residual_norm(&g->e.hk, hist, cap, m_out);
}

int lyap_gen_factor(lyap_gen* g, double* Z, int64_t ldz, int tcap, int* t_out, void* stream) {
  if (!g || !Z || !t_out || !g->e.hk.solved || ldz < tcap) return LYAP_ERR_ARG;
  return run_factor_basis(&g->e.hk, g->e.basis, g->e.n, Z, ldz, tcap, t_out, static_cast<cudaStream_t>(stream));
}

// out[0] solve ms, [1] E-solves, [2] their conjugate-gradient iterations in all, [3] the most in one
int lyap_gen_stats(lyap_gen* g, double* out, int cap) {
  if (!g || !out) return LYAP_ERR_ARG;
  const double v[4] = {g->e.times[0], (double)g->solves, (double)g->iters, (double)g->max_iters};
  for (int k = 0; k < 4 && k < cap; ++k) out[k] = v[k];
  return LYAP_OK;
}

}  // extern "C"
