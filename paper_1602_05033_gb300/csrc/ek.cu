// Extended Krylov projection (Sec. 4) with the solves with A done by preconditioned conjugate
// gradients on the GPU, preconditioned by Jacobi scaling or by a small convolutional network
// (three 3x3 convolutions, 1 -> 16 -> 16 -> 1 channels, ReLU, bf16 activations with fp32
// accumulation) trained on solve pairs that the method itself produces.
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
constexpr int kCh = 16;              // CNN channels
constexpr int kGrid = 304;           // CTAs of the reduction kernels (fixed: deterministic sums)
constexpr int kTile = 1024;          // pixels per weight-gradient tile
constexpr int kNW = kCh * 9 + kCh + kCh * kCh * 9 + kCh + kCh * 9 + 1;  // CNN parameters
// parameter offsets: w1 [c][k], b1 [c], w2 [co][ci][k], b2 [co], w3 [ci][k], b3
constexpr int oW1 = 0, oB1 = oW1 + kCh * 9, oW2 = oB1 + kCh, oB2 = oW2 + kCh * kCh * 9, oW3 = oB2 + kCh,
              oB3 = oW3 + kCh * 9;

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

// ---- convolutional preconditioner (bf16 activations, fp32 accumulation) --------------------
struct Img {
  int nx, ny;
};

__device__ __forceinline__ float bf(const __nv_bfloat16 v) { return __bfloat162float(v); }

// x0 = bf16(r_c / ||r_c||) for column c of r (leading dimension s)
__global__ void k_cnn_in(const double* __restrict__ r, int s, int c, const double* __restrict__ rr,
                         __nv_bfloat16* __restrict__ x0, int64_t n) {
  const double inv = rr[0] > 0.0 ? 1.0 / sqrt(rr[0]) : 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x0[i] = __float2bfloat16((float)(r[i * s + c] * inv));
}

// out[co][p] = act(b[co] + sum_ci sum_taps w[co][ci][k] in[ci](p + tap)); weights read as bf16
template <int CI, int CO, bool RELU>
__global__ void k_conv(const __nv_bfloat16* __restrict__ in, const __nv_bfloat16* __restrict__ wq,
                       const float* __restrict__ bias, __nv_bfloat16* __restrict__ out, float* __restrict__ out32, Img im) {
  __shared__ float w[CO * CI * 9];
  __shared__ float b[CO];
  for (int k = threadIdx.x; k < CO * CI * 9; k += blockDim.x) w[k] = bf(wq[k]);
  for (int k = threadIdx.x; k < CO; k += blockDim.x) b[k] = bias[k];
  __syncthreads();
  const int64_t n = (int64_t)im.nx * im.ny;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const int y = (int)(p / im.nx), x = (int)(p % im.nx);
    float acc[CO];
#pragma unroll
    for (int co = 0; co < CO; ++co) acc[co] = b[co];
#pragma unroll
    for (int dy = 0; dy < 3; ++dy) {
      const int yy = y + dy - 1;
      if (yy < 0 || yy >= im.ny) continue;
#pragma unroll
      for (int dx = 0; dx < 3; ++dx) {
        const int xx = x + dx - 1;
        if (xx < 0 || xx >= im.nx) continue;
        const int64_t q = (int64_t)yy * im.nx + xx;
#pragma unroll
        for (int ci = 0; ci < CI; ++ci) {
          const float v = bf(in[(int64_t)ci * n + q]);
#pragma unroll
          for (int co = 0; co < CO; ++co) acc[co] = fmaf(w[(co * CI + ci) * 9 + dy * 3 + dx], v, acc[co]);
        }
      }
    }
#pragma unroll
    for (int co = 0; co < CO; ++co) {
      const float v = RELU ? fmaxf(acc[co], 0.f) : acc[co];
      if (out) out[(int64_t)co * n + p] = __float2bfloat16(v);
      if (out32) out32[(int64_t)co * n + p] = v;
    }
  }
}

// preconditioned residual z_c = mdinv r_c - ||r_c|| y: Jacobi scaling of M = -A plus the network's
// correction (the network approximates A^{-1} - diag(A)^{-1} on unit residuals; z ~ M^{-1} r)
__global__ void k_cnn_out(const float* __restrict__ y, const double* __restrict__ rr, const double* __restrict__ mdinv,
                          const double* __restrict__ r, double* __restrict__ z, int s, int c, int64_t n) {
  const double sc = -sqrt(fmax(rr[0], 0.0));
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    z[i * s + c] = mdinv[i] * r[i * s + c] + sc * (double)y[i];
}

// y += r / diag(A) for the unit residual b / ||b|| (||b||^2 in bb[0]): the Jacobi part of the
// preconditioner in the training loss
__global__ void k_add_jacobi(float* __restrict__ y, const double* __restrict__ mdinv, const double* __restrict__ b,
                             const double* __restrict__ bb, int64_t n) {
  const double inv = 1.0 / sqrt(bb[0]);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] += (float)(-mdinv[i] * b[i] * inv);
}

// backward through one convolution: gin[ci][p] = mask(ci, p) * sum_co sum_taps w[co][ci][k] gout[co](p - tap)
// (mask: the layer input's ReLU, from its bf16 activation > 0); gout fp32
template <int CI, int CO>
__global__ void k_conv_bwd_data(const float* __restrict__ gout, const __nv_bfloat16* __restrict__ wq,
                                const __nv_bfloat16* __restrict__ act_in, float* __restrict__ gin, Img im) {
  __shared__ float w[CO * CI * 9];
  for (int k = threadIdx.x; k < CO * CI * 9; k += blockDim.x) w[k] = bf(wq[k]);
  __syncthreads();
  const int64_t n = (int64_t)im.nx * im.ny;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const int y = (int)(p / im.nx), x = (int)(p % im.nx);
    float acc[CI];
#pragma unroll
    for (int ci = 0; ci < CI; ++ci) acc[ci] = 0.f;
#pragma unroll
    for (int dy = 0; dy < 3; ++dy) {
      const int yy = y - (dy - 1);  // the output at yy used the input at yy + dy - 1 = y
      if (yy < 0 || yy >= im.ny) continue;
#pragma unroll
      for (int dx = 0; dx < 3; ++dx) {
        const int xx = x - (dx - 1);
        if (xx < 0 || xx >= im.nx) continue;
        const int64_t q = (int64_t)yy * im.nx + xx;
#pragma unroll
        for (int co = 0; co < CO; ++co) {
          const float g = gout[(int64_t)co * n + q];
#pragma unroll
          for (int ci = 0; ci < CI; ++ci) acc[ci] = fmaf(w[(co * CI + ci) * 9 + dy * 3 + dx], g, acc[ci]);
        }
      }
    }
#pragma unroll
    for (int ci = 0; ci < CI; ++ci) gin[(int64_t)ci * n + p] = bf(act_in[(int64_t)ci * n + p]) > 0.f ? acc[ci] : 0.f;
  }
}

// weight and bias gradients of one convolution, per tile of kTile pixels:
// gw[co][ci][k] = sum_p gout[co](p) in[ci](p + tap), gb[co] = sum_p gout[co](p)
template <int CI, int CO>
__global__ void k_conv_bwd_w(const float* __restrict__ gout, const __nv_bfloat16* __restrict__ in, Img im,
                             double* __restrict__ partials) {
  constexpr int NWG = CO * CI * 9 + CO;
  const int64_t n = (int64_t)im.nx * im.ny;
  const int64_t p0 = (int64_t)blockIdx.x * kTile;
  const int64_t p1 = p0 + kTile < n ? p0 + kTile : n;
  for (int wi = threadIdx.x; wi < NWG; wi += blockDim.x) {
    double acc = 0.0;
    if (wi < CO * CI * 9) {
      const int co = wi / (CI * 9), ci = (wi / 9) % CI, k = wi % 9;
      const int dy = k / 3 - 1, dx = k % 3 - 1;
      float part = 0.f;
      int cnt = 0;
      for (int64_t p = p0; p < p1; ++p) {
        const int y = (int)(p / im.nx) + dy, x = (int)(p % im.nx) + dx;
        if (y < 0 || y >= im.ny || x < 0 || x >= im.nx) continue;
        part = fmaf(gout[(int64_t)co * n + p], bf(in[(int64_t)ci * n + (int64_t)y * im.nx + x]), part);
        if (++cnt == 64) {
          acc += part;
          part = 0.f;
          cnt = 0;
        }
      }
      acc += part;
    } else {
      const int co = wi - CO * CI * 9;
      for (int64_t p = p0; p < p1; ++p) acc += gout[(int64_t)co * n + p];
    }
    partials[(size_t)blockIdx.x * NWG + wi] = acc;
  }
}

// grad[off + k] += sum over tiles of partials[.][k]
__global__ void k_wgrad_sum(const double* __restrict__ partials, int ntiles, int nwg, double* __restrict__ grad) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nwg; k += gridDim.x * blockDim.x) {
    double t = 0.0;
    for (int b = 0; b < ntiles; ++b) t += partials[(size_t)b * nwg + k];
    grad[k] += t;
  }
}

// gy = coef * (r_scaled - A y) from Ay (double) ; also partials y.Ay, y.r_scaled
__global__ void k_energy_grad(const float* __restrict__ y, const double* __restrict__ Ay, const __nv_bfloat16* __restrict__ x0,
                              const double* __restrict__ coef, float* __restrict__ gy, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    gy[i] = (float)(coef[0] * ((double)bf(x0[i]) - Ay[i]));
}

// Adam on the fp32 master parameters; the bf16 copy is what the kernels read
__global__ void k_adam(float* __restrict__ th, const double* __restrict__ g, float* __restrict__ m1, float* __restrict__ m2,
                       __nv_bfloat16* __restrict__ thq, int nw, float lr, float b1, float b2, float eps, int t) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nw) return;
  const float gk = (float)g[k];
  m1[k] = b1 * m1[k] + (1.f - b1) * gk;
  m2[k] = b2 * m2[k] + (1.f - b2) * gk * gk;
  const float mh = m1[k] / (1.f - powf(b1, (float)t)), vh = m2[k] / (1.f - powf(b2, (float)t));
  th[k] -= lr * mh / (sqrtf(vh) + eps);
  thq[k] = __float2bfloat16(th[k]);
}

__global__ void k_cast_params(const float* __restrict__ th, __nv_bfloat16* __restrict__ thq, int nw) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nw) thq[k] = __float2bfloat16(th[k]);
}

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

}  // namespace

namespace {

struct EkLayout {
  size_t total = 0, basis = 0, W = 0, AV = 0, C = 0, mdinv = 0, vec = 0, partials = 0, small = 0, log = 0, hist = 0,
         flags = 0, chk = 0, check = 0, check_bytes = 0, factor = 0, factor_bytes = 0, csr = 0, pairs = 0, cnn = 0;
  int pair_cap = 0;
};

size_t cnn_bytes(int64_t n) {
  size_t b = 0;
  auto add = [&](size_t x) { b += lyap_align256((int64_t)x); };
  add(sizeof(float) * kNW * 3);                  // th, m1, m2
  add(sizeof(__nv_bfloat16) * kNW);              // thq
  add(sizeof(__nv_bfloat16) * n * (1 + 2 * kCh)); // x0, a1, a2
  add(sizeof(float) * n * (1 + 2 * kCh + 1));    // y32, g1, g2, gy
  add(sizeof(double) * kNW);                     // grad
  add(sizeof(double) * ((n + kTile - 1) / kTile) * (kCh * kCh * 9 + kCh)); // wpart
  add(sizeof(double) * n);                        // Ay
  add(sizeof(double) * 8);                        // coef
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
  L.pair_cap = 4 * s;
  L.pairs = take(sizeof(double) * n * L.pair_cap * 2);
  L.cnn = grid_image ? take(cnn_bytes(n)) : 0;
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

// A y for the network's fp32 output y
__global__ void k_spmv_f(Csr A, const float* __restrict__ y, double* __restrict__ Ay) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < A.n; i += (int64_t)gridDim.x * blockDim.x) {
    double t = 0.0;
    for (int64_t e = A.rowptr[i]; e < A.rowptr[i + 1]; ++e) t = fma(A.val[e], (double)y[A.col[e]], t);
    Ay[i] = t;
  }
}

// y.Ay and y.b -> partials
__global__ void k_dot_y(const float* __restrict__ y, const double* __restrict__ Ay, const double* __restrict__ b, int64_t n,
                        double* __restrict__ partials) {
  double acc[2] = {0.0, 0.0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    acc[0] = fma((double)y[i], Ay[i], acc[0]);
    acc[1] = fma((double)y[i], b[i], acc[1]);
  }
  cta_partials<2>(acc, partials);
}

// per pair: coef[0] = b.b, coef[1] = b.x (reduced), coef[2] = y.Ay, coef[3] = y.b (reduced).
// With rhat = b/||b||, xhat = x/||b||: ex = xhat^T (-A) xhat = -xhat.rhat, the loss term
// (y - xhat)^T (-A) (y - xhat) / ex = (-y.Ay + 2 y.rhat + ex) / ex, gradient coefficient 2/(ex K)
__global__ void k_energy_coef(double* __restrict__ coef, int K) {
  if (threadIdx.x) return;
  const double nb = sqrt(coef[0]);
  const double ex = -coef[1] / coef[0];
  const double L = (-coef[2] + 2.0 * coef[3] / nb + ex) / ex;
  coef[4] = 2.0 / (ex * K);
  coef[5] += L / K;
  coef[6] = 1.0 / nb;
}

__global__ void k_energy_gy(const double* __restrict__ Ay, const double* __restrict__ b, const double* __restrict__ coef,
                            float* __restrict__ gy, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    gy[i] = (float)(coef[4] * (b[i] * coef[6] - Ay[i]));
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
  // CNN parameters (fp32 master, Adam moments, bf16 copy) and activations
  float *th = nullptr, *m1 = nullptr, *m2 = nullptr, *y32 = nullptr, *g1 = nullptr, *g2 = nullptr, *gy = nullptr;
  __nv_bfloat16 *thq = nullptr, *x0 = nullptr, *a1 = nullptr, *a2 = nullptr;
  double *grad = nullptr, *wpart = nullptr, *Ay = nullptr, *coef = nullptr;
  int trained = 0, adam_t = 0, last_jacobi_its = 0, fallbacks = 0;
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

// ---- the network ------------------------------------------------------------------------------
// y = N(rsrc_c / ||rsrc_c||) into y32 (activations kept for the backward pass); rr = ||rsrc_c||^2
void cnn_forward(lyap_ek* e, const double* rsrc, int ldr, int c, const double* rr, cudaStream_t st) {
  const int64_t n = e->n;
  Img im{e->nx, e->ny};
  const int g = (int)std::min<int64_t>((n + kT - 1) / kT, 4096);
  k_cnn_in<<<g, kT, 0, st>>>(rsrc, ldr, c, rr, e->x0, n);
  k_conv<1, kCh, true><<<g, kT, 0, st>>>(e->x0, e->thq + oW1, e->th + oB1, e->a1, nullptr, im);
  k_conv<kCh, kCh, true><<<g, kT, 0, st>>>(e->a1, e->thq + oW2, e->th + oB2, e->a2, nullptr, im);
  k_conv<kCh, 1, false><<<g, kT, 0, st>>>(e->a2, e->thq + oW3, e->th + oB3, nullptr, e->y32, im);
}

// adds the energy-loss gradient of pair k (of K) to e->grad and its loss term to coef[5]
void cnn_pair_grad(lyap_ek* e, const double* b, const double* x, int K, cudaStream_t st) {
  const int64_t n = e->n;
  Img im{e->nx, e->ny};
  const int g = (int)std::min<int64_t>((n + kT - 1) / kT, 4096);
  k_dot2<<<kGrid, kT, 0, st>>>(b, b, x, n, e->partials);
  k_sum_partials<<<1, 64, 0, st>>>(e->partials, kGrid, 2, e->coef);
  cnn_forward(e, b, 1, 0, e->coef, st);
  k_add_jacobi<<<g, kT, 0, st>>>(e->y32, e->mdinv, b, e->coef, n);
  k_spmv_f<<<g, kT, 0, st>>>(e->A, e->y32, e->Ay);
  k_dot_y<<<kGrid, kT, 0, st>>>(e->y32, e->Ay, b, n, e->partials);
  k_sum_partials<<<1, 64, 0, st>>>(e->partials, kGrid, 2, e->coef + 2);
  k_energy_coef<<<1, 32, 0, st>>>(e->coef, K);
  k_energy_gy<<<g, kT, 0, st>>>(e->Ay, b, e->coef, e->gy, n);
  const int nt = (int)((n + kTile - 1) / kTile);
  // layer 3: data gradient into a2's channels (masked by a2 > 0), weight gradient
  k_conv_bwd_data<kCh, 1><<<g, kT, 0, st>>>(e->gy, e->thq + oW3, e->a2, e->g2, im);
  k_conv_bwd_w<kCh, 1><<<nt, kT, 0, st>>>(e->gy, e->a2, im, e->wpart);
  k_wgrad_sum<<<(kCh * 9 + 1 + 127) / 128, 128, 0, st>>>(e->wpart, nt, kCh * 9 + 1, e->grad + oW3);
  // layer 2
  k_conv_bwd_data<kCh, kCh><<<g, kT, 0, st>>>(e->g2, e->thq + oW2, e->a1, e->g1, im);
  k_conv_bwd_w<kCh, kCh><<<nt, kT, 0, st>>>(e->g2, e->a1, im, e->wpart);
  k_wgrad_sum<<<(kCh * kCh * 9 + kCh + 127) / 128, 128, 0, st>>>(e->wpart, nt, kCh * kCh * 9 + kCh, e->grad + oW2);
  // layer 1 (its input needs no gradient)
  k_conv_bwd_w<1, kCh><<<nt, kT, 0, st>>>(e->g1, e->x0, im, e->wpart);
  k_wgrad_sum<<<(kCh * 9 + kCh + 127) / 128, 128, 0, st>>>(e->wpart, nt, kCh * 9 + kCh, e->grad + oW1);
}

// loss and gradient over the stored pairs (grad and coef[5] reset first)
void cnn_grad_all(lyap_ek* e, cudaStream_t st) {
  cudaMemsetAsync(e->grad, 0, sizeof(double) * kNW, st);
  cudaMemsetAsync(e->coef + 5, 0, sizeof(double), st);
  for (int k = 0; k < e->npairs; ++k)
    cnn_pair_grad(e, e->pair_b + (size_t)k * e->n, e->pair_x + (size_t)k * e->n, e->npairs, st);
}

int cnn_train(lyap_ek* e, int iters, float lr, cudaStream_t st) {
  if (e->npairs == 0) return LYAP_ERR_ARG;
  for (int it = 0; it < iters; ++it) {
    cnn_grad_all(e, st);
    if (it == 0) {
      LYAP_CUDA_TRY(cudaMemcpyAsync(&e->loss0, e->coef + 5, sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    ++e->adam_t;
    k_adam<<<(kNW + 255) / 256, 256, 0, st>>>(e->th, e->grad, e->m1, e->m2, e->thq, kNW, lr, 0.9f, 0.999f, 1e-8f, e->adam_t);
  }
  cnn_grad_all(e, st);
  LYAP_CUDA_TRY(cudaMemcpyAsync(&e->loss1, e->coef + 5, sizeof(double), cudaMemcpyDeviceToHost, st));
  LYAP_CUDA_TRY(cudaStreamSynchronize(st));
  // a network whose training diverged is not used (the solves stay with Jacobi)
  e->trained = std::isfinite(e->loss1) ? 1 : -1;
  return cudaGetLastError() == cudaSuccess ? LYAP_OK : LYAP_ERR_CUDA;
}

// ---- preconditioned conjugate gradients for A X = B (s columns), on M = -A ------------------
template <int s>
int pcg_t(lyap_ek* e, const double* B, int ldb, int use_cnn, int* its, cudaStream_t st) {
  const int64_t n = e->n;
  const double tol2 = e->inner_tol * e->inner_tol;
  k_cg_start<s><<<kGrid, kT, 0, st>>>(B, ldb, e->x, e->r, n, e->partials);
  k_sum_partials<<<1, 64, 0, st>>>(e->partials, kGrid, s, e->small);
  k_cg_conv<<<1, 32, 0, st>>>(e->small, e->sc, s, tol2, 1);
  auto precond = [&](int first) {
    if (use_cnn) {
      for (int c = 0; c < s; ++c) {
        cnn_forward(e, e->r, s, c, e->sc + c * kSc + 3, st);
        const int g = (int)std::min<int64_t>((n + kT - 1) / kT, 4096);
        k_cnn_out<<<g, kT, 0, st>>>(e->y32, e->sc + c * kSc + 3, e->mdinv, e->r, e->z, s, c, n);
      }
      k_cg_zdots<s><<<kGrid, kT, 0, st>>>(e->r, e->q, e->sc, e->z, n, first, e->partials);
    } else {
      k_cg_jacobi<s><<<kGrid, kT, 0, st>>>(e->mdinv, e->r, e->q, e->sc, e->z, n, first, e->partials);
    }
    k_sum_partials<<<1, 64, 0, st>>>(e->partials, kGrid, 2 * s, e->small);
    k_cg_beta<<<1, 32, 0, st>>>(e->small, e->sc, s, first);
  };
  precond(1);
  LYAP_CUDA_TRY(cudaMemcpyAsync(e->p, e->z, sizeof(double) * n * s, cudaMemcpyDeviceToDevice, st));
  std::vector<double> hsc(kSc * s);
  int it = 0;
  for (; it < e->inner_maxit;) {
    for (int k = 0; k < 8 && it < e->inner_maxit; ++k, ++it) {
      k_cg_matvec<s><<<kGrid, kT, 0, st>>>(e->A, e->p, e->q, e->partials);
      k_sum_partials<<<1, 64, 0, st>>>(e->partials, kGrid, s, e->small);
      k_cg_alpha<<<1, 32, 0, st>>>(e->small, e->sc, s);
      k_cg_update<s><<<kGrid, kT, 0, st>>>(e->x, e->r, e->p, e->q, e->sc, n, e->partials);
      k_sum_partials<<<1, 64, 0, st>>>(e->partials, kGrid, s, e->small);
      k_cg_conv<<<1, 32, 0, st>>>(e->small, e->sc, s, tol2, 0);
      precond(0);
      k_cg_dir<s><<<kGrid * 4, kT, 0, st>>>(e->z, e->p, e->sc, n);
    }
    LYAP_CUDA_TRY(cudaMemcpyAsync(hsc.data(), e->sc, sizeof(double) * kSc * s, cudaMemcpyDeviceToHost, st));
    LYAP_CUDA_TRY(cudaStreamSynchronize(st));
    LYAP_CUDA_TRY(cudaGetLastError());
    bool any = false;
    for (int c = 0; c < s; ++c) any = any || hsc[c * kSc + 5] != 0.0;
    if (!any) break;
  }
  *its = it;
  for (int c = 0; c < s; ++c)
    if (!std::isfinite(hsc[c * kSc + 3])) return LYAP_ERR_NONFINITE;
  return it >= e->inner_maxit ? LYAP_NOT_CONVERGED : LYAP_OK;
}

int pcg_once(lyap_ek* e, const double* B, int ldb, int use_cnn, int* its, cudaStream_t st) {
  switch (e->s) {
    case 1: return pcg_t<1>(e, B, ldb, use_cnn, its, st);
    case 2: return pcg_t<2>(e, B, ldb, use_cnn, its, st);
    case 4: return pcg_t<4>(e, B, ldb, use_cnn, its, st);
  }
  return LYAP_ERR_ARG;
}

// The network's solve is accepted when it reaches the inner tolerance within 3x the iterations of
// the last Jacobi solve; otherwise (or if it went non-finite: a nonlinear preconditioner need not
// keep z.r > 0) the solve is redone with Jacobi, which judges and backs up the network.
// *used_cnn tells which preconditioner produced the solution.
int pcg(lyap_ek* e, const double* B, int ldb, int use_cnn, int* its, int* used_cnn, cudaStream_t st) {
  *used_cnn = 0;
  if (use_cnn) {
    const int cap = e->inner_maxit;
    e->inner_maxit = std::max(200, 3 * e->last_jacobi_its);
    int rc = pcg_once(e, B, ldb, 1, its, st);
    e->inner_maxit = cap;
    if (rc == LYAP_OK) {
      *used_cnn = 1;
      return rc;
    }
    ++e->fallbacks;
  }
  int rc = pcg_once(e, B, ldb, 0, its, st);
  if (rc == LYAP_OK || rc == LYAP_NOT_CONVERGED) e->last_jacobi_its = *its;
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
  // the oracle's initialisation law: normal(0, 0.1) for w1, normal(0, 0.1/sqrt(C)) for w2, w3,
  // normal(0, 0.01) for b1, b2, zero b3 (a fixed-seed generator of this library)
  th.assign(kNW, 0.f);
  unsigned long long st = 0x2545F4914F6CDD1DULL;
  auto uni = [&]() {
    st = st * 6364136223846793005ULL + 1442695040888963407ULL;
    return ((st >> 11) + 0.5) * (1.0 / 9007199254740992.0);
  };
  auto nrm = [&]() { return sqrt(-2.0 * log(uni())) * cos(6.283185307179586 * uni()); };
  for (int k = 0; k < kCh * 9; ++k) th[oW1 + k] = (float)(0.1 * nrm());
  for (int k = 0; k < kCh; ++k) th[oB1 + k] = (float)(0.01 * nrm());
  for (int k = 0; k < kCh * kCh * 9; ++k) th[oW2 + k] = (float)(0.1 / 4.0 * nrm());
  for (int k = 0; k < kCh; ++k) th[oB2 + k] = (float)(0.01 * nrm());
  // the last layer starts at zero: the preconditioner starts as Jacobi scaling exactly
}

}  // namespace

extern "C" {

int lyap_ek_workspace_size(const lyap_csr* A, int s, int maxit, int nx, int ny, size_t* bytes) {
  if (!A || !bytes || (s != 1 && s != 2 && s != 4) || maxit < 1) return LYAP_ERR_ARG;
  int rc = validate_csr(A);
  if (rc != LYAP_OK) return rc;
  if (A->val_dtype != LYAP_F64) return LYAP_ERR_ARG;
  if ((nx || ny) && (int64_t)nx * ny != A->n) return LYAP_ERR_ARG;
  *bytes = ek_layout(A, s, maxit, nx > 0).total;
  return LYAP_OK;
}

}  // extern "C"

namespace {
// events and pinned host buffers of a context (the object itself stays)
void ek_release(lyap_ek* e) {
  for (int i = 0; i < 4; ++i)
    if (e->ev[i]) cudaEventDestroy(e->ev[i]);
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
    char* c = w + e->L.cnn;
    auto take = [&](size_t bytes) { char* r2 = c; c += lyap_align256((int64_t)bytes); return r2; };
    e->th = reinterpret_cast<float*>(take(sizeof(float) * kNW * 3));
    e->m1 = e->th + kNW;
    e->m2 = e->th + 2 * kNW;
    e->thq = reinterpret_cast<__nv_bfloat16*>(take(sizeof(__nv_bfloat16) * kNW));
    e->x0 = reinterpret_cast<__nv_bfloat16*>(take(sizeof(__nv_bfloat16) * n * (1 + 2 * kCh)));
    e->a1 = e->x0 + n;
    e->a2 = e->a1 + n * kCh;
    e->y32 = reinterpret_cast<float*>(take(sizeof(float) * n * (2 + 2 * kCh)));
    e->g1 = e->y32 + n;
    e->g2 = e->g1 + n * kCh;
    e->gy = e->g2 + n * kCh;
    e->grad = reinterpret_cast<double*>(take(sizeof(double) * kNW));
    e->wpart = reinterpret_cast<double*>(take(sizeof(double) * ((n + kTile - 1) / kTile) * (kCh * kCh * 9 + kCh)));
    e->Ay = reinterpret_cast<double*>(take(sizeof(double) * n));
    e->coef = reinterpret_cast<double*>(take(sizeof(double) * 8));
    std::vector<float> th;
    init_params_host(th);
    if (cudaMemcpyAsync(e->th, th.data(), sizeof(float) * kNW, cudaMemcpyHostToDevice, st) != cudaSuccess)
      return fail(LYAP_ERR_CUDA);
    cudaMemsetAsync(e->m1, 0, sizeof(float) * 2 * kNW, st);
    k_cast_params<<<(kNW + 255) / 256, 256, 0, st>>>(e->th, e->thq, kNW);
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
  if (cudaMallocHost(&hk.hist_host, sizeof(double) * maxit) != cudaSuccess) return fail(LYAP_ERR_CUDA);
  if (cudaMallocHost(&hk.flags_host, sizeof(int) * 8) != cudaSuccess) return fail(LYAP_ERR_CUDA);
  if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess) return fail(LYAP_ERR_CUDA);
  *out = e;
  return LYAP_OK;
}

// precond: 0 Jacobi, 1 the network (the first train_steps inner solves use Jacobi and provide
// its training pairs, then train_iters Adam steps, learning rate lr)
int lyap_ek_solve(lyap_ek* e, int precond, int train_steps, int train_iters, float lr, void* stream) {
  if (!e || (precond != 0 && precond != 1) || (precond == 1 && e->nx == 0)) return LYAP_ERR_ARG;
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
  hk.solved = 0;
  hk.factored = 0;
  float t_train = 0.f;
  // beta = ||C||_F
  k_dot2<<<kGrid, kT, 0, st>>>(e->C, e->C, e->C, n * s, e->partials);
  k_sum_partials<<<1, 64, 0, st>>>(e->partials, kGrid, 2, e->small);
  double bb[2];
  LYAP_CUDA_TRY(cudaMemcpyAsync(bb, e->small, sizeof(bb), cudaMemcpyDeviceToHost, st));
  LYAP_CUDA_TRY(cudaStreamSynchronize(st));
  const double beta = sqrt(bb[0]);
  auto use_cnn = [&]() { return precond == 1 && e->trained == 1; };
  auto collect = [&]() { return precond == 1 && e->trained == 0; };
  // [C, A^{-1} C] = V_1 gamma
  double* V1 = e->basis;
  const int gcp = (int)std::min<int64_t>((n * S + kT - 1) / kT, 8192);
  k_copy_cols<<<gcp, kT, 0, st>>>(e->C, s, V1, S, 0, s, n, 1.0);
  int its = 0, used = 0;
  e->fallbacks = 0;
  int rc = pcg(e, e->C, s, use_cnn(), &its, &used, st);
  if (rc == LYAP_ERR_NONFINITE) return rc;
  e->inner_its.push_back(its);
  e->inner_kind.push_back(used);
  take_solution(e, e->C, s, V1, S, s, collect(), st);
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
    if (precond == 1 && e->trained == 0 && (int)e->inner_its.size() >= train_steps) {
      cudaEventRecord(e->ev[2], st);
      rc = cnn_train(e, train_iters, lr, st);
      if (rc != LYAP_OK) return rc;
      cudaEventRecord(e->ev[3], st);
      LYAP_CUDA_TRY(cudaStreamSynchronize(st));
      cudaEventElapsedTime(&t_train, e->ev[2], e->ev[3]);
    }
    double* Vj = e->basis + (size_t)(j - 1) * n * S;
    double* Vn = e->basis + (size_t)j * n * S;
    spmm(e->A, S, Vj, S, e->AV, S, 1.0, st);
    k_copy_cols<<<gcp, kT, 0, st>>>(e->AV, S, Vn, S, 0, s, n, 1.0);
    rc = pcg(e, Vj + s, S, use_cnn(), &its, &used, st);
    if (rc == LYAP_ERR_NONFINITE) return rc;
    e->inner_its.push_back(its);
    e->inner_kind.push_back(used);
    take_solution(e, Vj + s, S, Vn, S, s, collect(), st);
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

// out[0] solve ms, [1] training ms, [2] loss before training, [3] loss after, [4] inner solves,
// [5] network solves redone with Jacobi, then the inner iteration counts (negative: solved with
// the network) up to cap
int lyap_ek_stats(lyap_ek* e, double* out, int cap) {
  if (!e || !out) return LYAP_ERR_ARG;
  const double head[6] = {e->times[0], e->times[1], e->loss0, e->loss1, (double)e->inner_its.size(), (double)e->fallbacks};
  int k = 0;
  for (; k < 6 && k < cap; ++k) out[k] = head[k];
  for (size_t i = 0; i < e->inner_its.size() && k < cap; ++i, ++k)
    out[k] = e->inner_kind[i] ? -(double)e->inner_its[i] : (double)e->inner_its[i];
  return LYAP_OK;
}

// loss and gradient of the network over caller-given pairs (device, n x K column-major each,
// A x_k = b_k) with the caller's parameters (host, the layout of the parameter vector);
// for testing the training kernels against an independent implementation
int lyap_ek_cnn_grad(lyap_ek* e, const float* params, int K, const double* B, const double* X, double* loss,
                     double* grad, void* stream) {
  if (!e || !params || K < 1 || !B || !X || !loss || !grad || e->nx == 0) return LYAP_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  LYAP_CUDA_TRY(cudaMemcpyAsync(e->th, params, sizeof(float) * kNW, cudaMemcpyHostToDevice, st));
  k_cast_params<<<(kNW + 255) / 256, 256, 0, st>>>(e->th, e->thq, kNW);
  cudaMemsetAsync(e->grad, 0, sizeof(double) * kNW, st);
  cudaMemsetAsync(e->coef + 5, 0, sizeof(double), st);
  for (int k = 0; k < K; ++k) cnn_pair_grad(e, B + (size_t)k * e->n, X + (size_t)k * e->n, K, st);
  LYAP_CUDA_TRY(cudaMemcpyAsync(grad, e->grad, sizeof(double) * kNW, cudaMemcpyDeviceToHost, st));
  LYAP_CUDA_TRY(cudaMemcpyAsync(loss, e->coef + 5, sizeof(double), cudaMemcpyDeviceToHost, st));
  LYAP_CUDA_TRY(cudaStreamSynchronize(st));
  return cudaGetLastError() == cudaSuccess ? LYAP_OK : LYAP_ERR_CUDA;
}

int lyap_ek_param_count(void) { return kNW; }

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
