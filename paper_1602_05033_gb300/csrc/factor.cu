// Low-rank factor at convergence (Alg. 1 steps 8-9) with the two-pass device (Sec. 3.3).
//
// The paper truncates the eigendecomposition of Y~ = -(e_i^T S e_j / (lambda_i + lambda_j))
// (Sec. 3.2) and forms Q_m Ycheck with the full eigenvector matrix Q_m.  On this
// GPU both O((sm)^3) steps are replaced by exact-arithmetic equivalents that cost
// O(sm t^2):
//  * Y~ is positive semidefinite with fast-decaying spectrum, so a pivoted
//    Cholesky factorisation Y~ ~= L L^T, stopped when the trace of the remainder
//    is below 1e-2 of the truncation threshold, captures its numerical range;
//    the eigendecomposition of L^T L (t x t, Jacobi) then gives the eigenpairs of
//    L L^T, truncated by the paper's rule (discarded tail <= eps).
//  * L = Y~(:,P) L_PP^{-T} (Nystrom form of the pivoted factor), and column p of
//    Q Y~ is -(T_m + lambda_p I)^{-1} E_1 gamma a_p (because Q a = E_1 gamma), an
//    SND band solve; hence Q L = B L_PP^{-T} without Q.
// M = Q Ycheck is then accumulated into Z = sum_j V_j E_j^T M while the basis is
// regenerated from the logged coefficients (k blocks buffered per GEMM update).
#include "common.cuh"
#include "ff.cuh"

#include <float.h>
#include <math.h>
#include <vector>
#include <algorithm>

void check_slot0(lyap_handle* h, int opi, double** lam, double** a, double** w);

namespace {

constexpr int kPcThreads = 1024;
// the parallel Jacobi kernel pairs at most 1024 index pairs per round (shared arrays)
constexpr int kTmaxCap = 2000;

struct FactorWs {
  double* L;      // tmax x nn   (row k = k-th pivoted column)
  int* piv;       // tmax
  int* tcount;    // [0] t after pivoted Cholesky, [1] kept t'
  double* K;      // tmax x tmax
  double* Vk;     // tmax x tmax
  double* ev;     // tmax
  double* chol;   // tmax x (s+1) x nmax   band Cholesky scratch, one per pivot
  double* B;      // nn x tmax  (Lanczos coordinates, row-major)
  double* M;      // nn x tmax
};

// ---- pivoted Cholesky of the PSD matrix Y~ (generalised to the 2N stacked Sylvester form)
// entry(i, j) = -(a_i . a_j) / (l_i + l_j), rows 0..nn-1 with a (nn x s) and l (nn)
__global__ void __launch_bounds__(kPcThreads) k_pivoted_cholesky(const double* __restrict__ lam,
                                                                 const double* __restrict__ a, int nn, int s,
                                                                 int tmax, double stop, FactorWs f,
                                                                 double* __restrict__ dg) {
  __shared__ double rv[kPcThreads / 32];
  __shared__ int ri[kPcThreads / 32];
  __shared__ double rs[kPcThreads / 32];
  __shared__ int s_p;
  __shared__ double s_sq, s_tr;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < nn; i += blockDim.x) {
    double q = 0.0;
    for (int c = 0; c < s; ++c) q += a[(size_t)i * s + c] * a[(size_t)i * s + c];
    dg[i] = -q / (2.0 * lam[i]);
  }
  __syncthreads();
  int k = 0;
  for (; k < tmax; ++k) {
    // argmax (lowest index on ties) and trace of the remaining diagonal
    double best = -1.0, tr = 0.0;
    int bi = nn;
    for (int i = tid; i < nn; i += blockDim.x) {
      const double v = dg[i];
      if (v > 0.0) tr += v;
      if (v > best) { best = v; bi = i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
      tr += __shfl_xor_sync(0xffffffffu, tr, o);
    }
    if (lane == 0) { rv[warp] = best; ri[warp] = bi; rs[warp] = tr; }
    __syncthreads();
    if (tid == 0) {
      double b = rv[0], t = rs[0];
      int bi0 = ri[0];
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
        if (rv[w] > b || (rv[w] == b && ri[w] < bi0)) { b = rv[w]; bi0 = ri[w]; }
        t += rs[w];
      }
      s_p = bi0;
      s_tr = t;
      s_sq = b > 0.0 ? sqrt(b) : 0.0;
    }
    __syncthreads();
    if (!(s_tr > stop) || s_p >= nn || !(s_sq > 0.0)) break;
    const int p = s_p;
    const double sq = s_sq;
    const double lp = lam[p];
    double ap[2 * LYAP_MAX_S];
    for (int c = 0; c < s; ++c) ap[c] = a[(size_t)p * s + c];
    for (int i = tid; i < nn; i += blockDim.x) {
      double y = 0.0;
      if (dg[i] > -1.0) {  // not yet pivoted
        double dot = 0.0;
        for (int c = 0; c < s; ++c) dot += a[(size_t)i * s + c] * ap[c];
        y = -dot / (lam[i] + lp);
        for (int l = 0; l < k; ++l) y -= f.L[(size_t)l * nn + i] * f.L[(size_t)l * nn + p];
        y /= sq;
      }
      f.L[(size_t)k * nn + i] = (i == p) ? sq : y;
    }
    __syncthreads();
    for (int i = tid; i < nn; i += blockDim.x) {
      if (i == p) dg[i] = -2.0;  // mark pivoted
      else if (dg[i] > -1.0) dg[i] -= f.L[(size_t)k * nn + i] * f.L[(size_t)k * nn + i];
    }
    if (tid == 0) f.piv[k] = p;
    __syncthreads();
  }
  if (tid == 0) f.tcount[0] = k;
}

// out = L(:, lo:lo+cnt)^T L(:, lo:lo+cnt)  (t x t); the rows of f.L are the pivoted columns of
// the factor, so this is the Gram matrix of the factor's rows lo..lo+cnt-1
__global__ void k_gram_L(FactorWs f, int nn, int lo, int cnt, int tmax, double* __restrict__ out) {
  const int t = f.tcount[0];
  const int a = blockIdx.x, b = blockIdx.y * blockDim.x + threadIdx.x;
  if (a >= t || b >= t) return;
  double acc = 0.0;
  for (int i = lo; i < lo + cnt; ++i) acc += f.L[(size_t)a * nn + i] * f.L[(size_t)b * nn + i];
  out[(size_t)a * tmax + b] = acc;
}

// ---- eigenpairs of the symmetric t x t matrix K (eigenvalues to f.ev, eigenvectors to the columns
// of f.Vk), in three steps:
//  1. Householder reduction K = H T H^T to tridiagonal form (one CTA; the reflector vectors
//     overwrite K below its subdiagonal);
//  2. per eigenvalue (one thread each): bisection with Sturm counts on T, inverse iteration with
//     the tridiagonal LU (partial pivoting), then the back-transformation by the reflectors;
//  3. re-orthogonalisation of the vectors of eigenvalues closer than 1e-10 ||K|| (one warp).
// The scratch of step 1 (d, e, reflector scales) lives in f.chol, free once the shifted solves have
// run; the U rows of step 2 (3 t^2 doubles) in a scratch area of their own.  O(t^3) fp64 work once,
// against O(t^3) per sweep for cyclic Jacobi on one SM.
__global__ void __launch_bounds__(1024) k_tridiag(FactorWs f, int tmax) {
  const int t = f.tcount[0];
  double* K = f.K;
  double* d = f.chol;
  double* e = f.chol + tmax;
  double* bet = f.chol + 2 * (size_t)tmax;
  double* pv = f.chol + 3 * (size_t)tmax;  // work vector
  __shared__ double red[32];
  __shared__ double s_val;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  auto block_sum = [&](double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[wid] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      double a = 0.0;
      for (int w = 0; w < nw; ++w) a += red[w];
      s_val = a;
    }
    __syncthreads();
    return s_val;
  };
  for (int k = 0; k + 2 < t; ++k) {
    const int n1 = t - k - 1;  // rows k+1 .. t-1
    double loc = 0.0;
    for (int i = threadIdx.x; i < n1; i += blockDim.x) {
      const double x = K[(size_t)(k + 1 + i) * tmax + k];
      loc += x * x;
    }
    const double xx = block_sum(loc);
    const double x0 = K[(size_t)(k + 1) * tmax + k];
    const double alpha = xx > 0.0 ? (x0 >= 0.0 ? -sqrt(xx) : sqrt(xx)) : 0.0;
    // v = x - alpha e_1, H = I - beta v v^T with beta = 2 / v^T v = 1 / (alpha (alpha - x0))
    const double beta = xx > 0.0 ? 1.0 / (alpha * (alpha - x0)) : 0.0;
    __syncthreads();
    if (threadIdx.x == 0) {
      d[k] = K[(size_t)k * tmax + k];
      e[k] = xx > 0.0 ? alpha : x0;
      bet[k] = beta;
      K[(size_t)(k + 1) * tmax + k] = x0 - alpha;  // v_0; v_i = x_i below it
    }
    __syncthreads();
    if (beta == 0.0) continue;
    // p = beta A v over the trailing block A = K[k+1.., k+1..]
    for (int i = threadIdx.x; i < n1; i += blockDim.x) {
      const double* row = K + (size_t)(k + 1 + i) * tmax + (k + 1);
      double acc = 0.0;
      for (int j = 0; j < n1; ++j) acc = fma(row[j], K[(size_t)(k + 1 + j) * tmax + k], acc);
      pv[i] = beta * acc;
    }
    __syncthreads();
    loc = 0.0;
    for (int i = threadIdx.x; i < n1; i += blockDim.x) loc += pv[i] * K[(size_t)(k + 1 + i) * tmax + k];
    const double vtp = block_sum(loc);
    // q = p - (beta/2)(v^T p) v;  A <- A - v q^T - q v^T
    const double h = 0.5 * beta * vtp;
    for (int i = threadIdx.x; i < n1; i += blockDim.x) pv[i] -= h * K[(size_t)(k + 1 + i) * tmax + k];
    __syncthreads();
    for (int idx = threadIdx.x; idx < n1 * n1; idx += blockDim.x) {
      const int i = idx / n1, j = idx % n1;
      const double vi = K[(size_t)(k + 1 + i) * tmax + k], vj = K[(size_t)(k + 1 + j) * tmax + k];
      double& a = K[(size_t)(k + 1 + i) * tmax + (k + 1 + j)];
      a = a - vi * pv[j] - pv[i] * vj;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (t >= 2) {
      d[t - 2] = K[(size_t)(t - 2) * tmax + (t - 2)];
      e[t - 2] = K[(size_t)(t - 1) * tmax + (t - 2)];
      bet[t - 2] = 0.0;
    }
    if (t >= 1) {
      d[t - 1] = K[(size_t)(t - 1) * tmax + (t - 1)];
      e[t - 1] = 0.0;
      bet[t - 1] = 0.0;
    }
  }
}

// number of eigenvalues of the tridiagonal (d, e) below x (Sturm count, tiny pivots replaced)
__device__ int tri_count(const double* __restrict__ d, const double* __restrict__ e, int t, double x, double pivmin) {
  int c = 0;
  double q = d[0] - x;
  if (fabs(q) <= pivmin) q = -pivmin;
  c += q < 0.0;
  for (int k = 1; k < t; ++k) {
    q = (d[k] - x) - e[k - 1] * e[k - 1] / q;
    if (fabs(q) <= pivmin) q = -pivmin;
    c += q < 0.0;
  }
  return c;
}

// step 2: eigenvalue i by bisection, its tridiagonal eigenvector by inverse iteration, then the
// eigenvector of K by the reflectors of k_tridiag (applied last to first)
__global__ void k_tri_eigvec(FactorWs f, int tmax, double* __restrict__ U3) {
  const int t = f.tcount[0];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= t) return;
  const double* d = f.chol;
  const double* e = f.chol + tmax;
  const double* bet = f.chol + 2 * (size_t)tmax;
  double* z = f.Vk + i;  // column i, stride tmax
  const size_t ld = (size_t)tmax;
  double lo = INFINITY, hi = -INFINITY;
  for (int k = 0; k < t; ++k) {
    const double r = (k > 0 ? fabs(e[k - 1]) : 0.0) + (k + 1 < t ? fabs(e[k]) : 0.0);
    lo = fmin(lo, d[k] - r);
    hi = fmax(hi, d[k] + r);
  }
  const double span = fmax(fmax(fabs(lo), fabs(hi)), DBL_MIN);
  lo -= 4.0 * DBL_EPSILON * span;
  hi += 4.0 * DBL_EPSILON * span;
  const double pivmin = DBL_MIN * fmax(1.0, span * span);
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (!(hi - lo > 2.0 * DBL_EPSILON * span) || mid <= lo || mid >= hi) break;
    if (tri_count(d, e, t, mid, pivmin) <= i) lo = mid;
    else hi = mid;
  }
  const double lam = 0.5 * (lo + hi);
  f.ev[i] = lam;
  // inverse iteration on T - lam I: LU with partial pivoting, U with two superdiagonals
  const double tiny = DBL_EPSILON * span + DBL_MIN;
  for (int k = 0; k < t; ++k) z[k * ld] = 1.0 + 0.1 * (double)((k * 7 + i * 13) % 11) / 11.0;
  for (int itr = 0; itr < 3; ++itr) {
    // forward elimination with the right-hand side z; the factors are recomputed each iteration
    double a0 = d[0] - lam, b0 = t > 1 ? e[0] : 0.0, c0 = 0.0;  // current row: diag, super1, super2
    double r0 = z[0];
    // rows of U (diagonal and two superdiagonals): row k of thread i at U3 + 3 (k t + i)
    double* U = U3 + (size_t)i * 3;
    const size_t us = (size_t)3 * t;
    for (int k = 0; k + 1 < t; ++k) {
      double a1 = e[k], b1 = d[k + 1] - lam, c1 = k + 2 < t ? e[k + 1] : 0.0, r1 = z[(k + 1) * ld];
      if (fabs(a1) > fabs(a0)) {  // swap rows k and k+1
        double tmp;
        tmp = a0; a0 = a1; a1 = tmp;
        tmp = b0; b0 = b1; b1 = tmp;
        tmp = c0; c0 = c1; c1 = tmp;
        tmp = r0; r0 = r1; r1 = tmp;
      }
      if (fabs(a0) < tiny) a0 = a0 < 0.0 ? -tiny : tiny;
      const double l = a1 / a0;
      U[(size_t)k * us] = a0;
      U[(size_t)k * us + 1] = b0;
      U[(size_t)k * us + 2] = c0;
      z[k * ld] = r0;
      a0 = b1 - l * b0;
      b0 = c1 - l * c0;
      c0 = 0.0;
      r0 = r1 - l * r0;
    }
    if (fabs(a0) < tiny) a0 = a0 < 0.0 ? -tiny : tiny;
    U[(size_t)(t - 1) * us] = a0;
    U[(size_t)(t - 1) * us + 1] = 0.0;
    U[(size_t)(t - 1) * us + 2] = 0.0;
    z[(t - 1) * ld] = r0;
    double x1 = 0.0, x2 = 0.0, nrm = 0.0;
    for (int k = t - 1; k >= 0; --k) {
      const double x = (z[k * ld] - U[(size_t)k * us + 1] * x1 - U[(size_t)k * us + 2] * x2) / U[(size_t)k * us];
      z[k * ld] = x;
      nrm = fmax(nrm, fabs(x));
      x2 = x1;
      x1 = x;
    }
    const double sc = nrm > 0.0 ? 1.0 / nrm : 1.0;
    for (int k = 0; k < t; ++k) z[k * ld] *= sc;
  }
  // back-transformation: z <- H_0 H_1 ... H_{t-3} z
  for (int k = t - 3; k >= 0; --k) {
    const double b = bet[k];
    if (b == 0.0) continue;
    double dot = 0.0;
    for (int r = k + 1; r < t; ++r) dot = fma(f.K[(size_t)r * tmax + k], z[r * ld], dot);
    const double g = b * dot;
    for (int r = k + 1; r < t; ++r) z[r * ld] -= g * f.K[(size_t)r * tmax + k];
  }
  double n2 = 0.0;
  for (int k = 0; k < t; ++k) n2 = fma(z[k * ld], z[k * ld], n2);
  const double inv = n2 > 0.0 ? 1.0 / sqrt(n2) : 0.0;
  for (int k = 0; k < t; ++k) z[k * ld] *= inv;
}

// step 3: groups of eigenvalues closer than 1e-10 max |lambda| get their vectors orthonormalised
// (modified Gram-Schmidt in ascending order, one warp)
__global__ void k_tri_reorth(FactorWs f, int tmax) {
  const int t = f.tcount[0];
  const int lane = threadIdx.x;
  double big = 0.0;
  for (int k = 0; k < t; ++k) big = fmax(big, fabs(f.ev[k]));
  const double tol = 1e-10 * big;
  for (int i = 1; i < t; ++i) {
    int j0 = i;
    while (j0 > 0 && f.ev[i] - f.ev[j0 - 1] <= tol && i - j0 < 64) --j0;
    for (int j = j0; j < i; ++j) {
      double dot = 0.0;
      for (int k = lane; k < t; k += 32) dot = fma(f.Vk[(size_t)k * tmax + j], f.Vk[(size_t)k * tmax + i], dot);
      for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
      for (int k = lane; k < t; k += 32) f.Vk[(size_t)k * tmax + i] -= dot * f.Vk[(size_t)k * tmax + j];
      __syncwarp();
    }
    if (j0 < i) {
      double n2 = 0.0;
      for (int k = lane; k < t; k += 32) n2 = fma(f.Vk[(size_t)k * tmax + i], f.Vk[(size_t)k * tmax + i], n2);
      for (int o = 16; o > 0; o >>= 1) n2 += __shfl_xor_sync(0xffffffffu, n2, o);
      const double inv = n2 > 0.0 ? 1.0 / sqrt(n2) : 0.0;
      for (int k = lane; k < t; k += 32) f.Vk[(size_t)k * tmax + i] *= inv;
      __syncwarp();
    }
  }
}

// B[:, k] = -(T_m + lambda_{p_k} I)^{-1} E_1 gamma a_{p_k}; one thread per pivot, banded Cholesky
// of the SPD matrix -(T_m + lambda I) in (s+1) x N band storage.
__global__ void k_shifted_solves(const double* __restrict__ log, int s, int m, const double* __restrict__ lam,
                                 const double* __restrict__ a, FactorWs f, int tmax, int nmax, int col_off,
                                 int piv_lo, int piv_hi, int* flags) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int t = f.tcount[0];
  if (k >= t) return;
  const int p = f.piv[k];
  if (p < piv_lo || p >= piv_hi) return;  // pivot belongs to the other operator (Sylvester)
  const int N = s * m, SS = s * s;
  const double shift = lam[p];
  double* Lb = f.chol + (size_t)k * (s + 1) * nmax;  // Lb[d*N + j] = L[j+d][j]
  auto Tval = [&](int i, int c) -> double {            // T_m[i][c], i >= c, i - c <= s
    const int J = i / s, Jc = c / s;
    if (J == Jc) {
      const double* D = log + (size_t)(J + 1) * LOG_NREC * SS + REC_TDIAG * SS;
      return 0.5 * (D[(i % s) * s + (c % s)] + D[(c % s) * s + (i % s)]);
    }
    if (J == Jc + 1) return log[(size_t)(Jc + 1) * LOG_NREC * SS + REC_TNEXT * SS + (i % s) * s + (c % s)];
    return 0.0;
  };
  bool ok = true;
  for (int j = 0; j < N; ++j) {
    double djj = -(Tval(j, j) + shift);
    for (int kk = max(0, j - s); kk < j; ++kk) djj -= Lb[(size_t)(j - kk) * N + kk] * Lb[(size_t)(j - kk) * N + kk];
    if (!(djj > 0.0)) { ok = false; djj = DBL_MIN; }
    const double ljj = sqrt(djj);
    Lb[j] = ljj;
    for (int i = j + 1; i <= min(N - 1, j + s); ++i) {
      double v = -Tval(i, j);
      for (int kk = max(0, i - s); kk < j; ++kk) v -= Lb[(size_t)(i - kk) * N + kk] * Lb[(size_t)(j - kk) * N + kk];
      Lb[(size_t)(i - j) * N + j] = v / ljj;
    }
  }
  if (!ok) atomicOr(flags, DERR_NOTNEGDEF);
  // rhs r = -(E_1 gamma a_p): solve L y = r, L^T x = y  => x = (-(T+lam I))^{-1} r = -(T + lam I)^{-1}(-E1 gamma a_p)
  // we want B = -(T+lam I)^{-1} E1 gamma a_p = (-(T + lam I))^{-1} E1 gamma a_p
  const double* gam = log + REC_TNEXT * SS;
  double* x = f.B + col_off + k;  // column k of B, stride tmax
  const size_t ld = (size_t)tmax;
  for (int j = 0; j < N; ++j) {
    double r = 0.0;
    if (j < s)
      for (int c = 0; c < s; ++c) r += gam[j * s + c] * a[(size_t)p * s + c];
    for (int kk = max(0, j - s); kk < j; ++kk) r -= Lb[(size_t)(j - kk) * N + kk] * x[(size_t)kk * ld];
    x[(size_t)j * ld] = r / Lb[j];
  }
  for (int j = N - 1; j >= 0; --j) {
    double r = x[(size_t)j * ld];
    for (int i = j + 1; i <= min(N - 1, j + s); ++i) r -= Lb[(size_t)(i - j) * N + j] * x[(size_t)i * ld];
    x[(size_t)j * ld] = r / Lb[j];
  }
}

// X = B L_PP^{-T} in place (row-wise forward substitution with L_PP[a][k] = L[k][p_a])
__global__ void k_apply_lpp(FactorWs f, int nrows, int nn, int tmax) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  const int t = f.tcount[0];
  if (r >= nrows) return;
  double* x = f.B + (size_t)r * tmax;
  for (int aa = 0; aa < t; ++aa) {
    double v = x[aa];
    const int pa = f.piv[aa];
    for (int kk = 0; kk < aa; ++kk) v -= x[kk] * f.L[(size_t)kk * nn + pa];
    x[aa] = v / f.L[(size_t)aa * nn + pa];
  }
}

// M[:, c] = X V[:, order[c]] for the kept columns
__global__ void k_form_M(FactorWs f, int nrows, int tmax, const int* __restrict__ order, int tk, int row_off,
                         double* __restrict__ M, int ldm) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  const int t = f.tcount[0];
  if (r >= nrows || c >= tk) return;
  const int oc = order[c];
  double acc = 0.0;
  for (int kk = 0; kk < t; ++kk) acc += f.B[(size_t)(row_off + r) * tmax + kk] * f.Vk[(size_t)kk * tmax + oc];
  M[(size_t)r * ldm + c] = acc;
}

// C[r][c] = scale[c] * sum_k op(A)[r][k] op(B)[k][bcol(c)], op = identity or transpose,
// bcol(c) = order ? order[c] : c; rows x cols outputs, inner dimension read from *kdim (a
// device count).  Small dense products of the factor step (t <= 2000), one thread per output.
__global__ void k_small_gemm(const double* __restrict__ A, int lda, int transA, const double* __restrict__ B,
                             int ldb, int transB, const int* __restrict__ order, const double* __restrict__ scale,
                             double* __restrict__ C, int ldc, int rows, int cols, const int* __restrict__ kdim) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  if (r >= rows || c >= cols) return;
  const int K = *kdim;
  const int bc = order ? order[c] : c;
  const size_t sa_r = transA ? 1 : (size_t)lda, sa_k = transA ? (size_t)lda : 1;
  const size_t sb_k = transB ? 1 : (size_t)ldb, sb_c = transB ? (size_t)ldb : 1;
  double acc = 0.0;
  for (int k = 0; k < K; ++k) acc = fma(A[r * sa_r + k * sa_k], B[k * sb_k + bc * sb_c], acc);
  C[(size_t)r * ldc + c] = scale ? acc * scale[c] : acc;
}

void small_gemm(const double* A, int lda, int transA, const double* B, int ldb, int transB, const int* order,
                const double* scale, double* C, int ldc, int rows, int cols, const int* kdim, cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return;
  k_small_gemm<<<dim3((rows + 127) / 128, cols), 128, 0, st>>>(A, lda, transA, B, ldb, transB, order, scale, C, ldc,
                                                                rows, cols, kdim);
}

// fixed-order block sum (all threads get the result); red holds one slot per warp
__device__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
  return t;
}

// R factors of the Householder QR of the two N x t blocks of the stacked pivoted-Cholesky
// factor (block 0: rows 0..N-1, block 1: rows N..2N-1; f.L row k holds column k).  The
// columns are copied to W (column k at W + k N) and reduced in place; R (t x t, row-major,
// rows >= N zero) is written out.  Only R is needed: Y~ = L_A L_B^T = U_A (R_A R_B^T) U_B^T.
__global__ void __launch_bounds__(1024) k_householder_r(const double* __restrict__ Lrows, int nn, int Na, int Nb,
                                                        const int* __restrict__ tcount, double* __restrict__ Wa,
                                                        double* __restrict__ Wb, double* __restrict__ Ra,
                                                        double* __restrict__ Rb, int tmax) {
  __shared__ double red[32];
  __shared__ double s_vn2;
  const int t = *tcount;
  const int lo = blockIdx.x == 0 ? 0 : Na;
  const int N = blockIdx.x == 0 ? Na : Nb;  // rows of this block's part
  double* W = blockIdx.x == 0 ? Wa : Wb;
  double* R = blockIdx.x == 0 ? Ra : Rb;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (size_t idx = tid; idx < (size_t)t * N; idx += blockDim.x) {
    const int k = (int)(idx / N), i = (int)(idx % N);
    W[idx] = Lrows[(size_t)k * nn + lo + i];
  }
  for (int idx = tid; idx < t * t; idx += blockDim.x) R[(size_t)(idx / t) * tmax + idx % t] = 0.0;
  __syncthreads();
  const int kend = t < N ? t : N;
  for (int k = 0; k < kend; ++k) {
    double* x = W + (size_t)k * N;
    double ss = 0.0;
    for (int i = k + tid; i < N; i += blockDim.x) ss = fma(x[i], x[i], ss);
    const double tot = block_sum(ss, red);
    if (tid == 0) {
      const double xk = x[k], nrm = sqrt(tot);
      const double alpha = xk >= 0.0 ? -nrm : nrm;
      const double vk = xk - alpha;
      x[k] = vk;
      s_vn2 = tot - xk * xk + vk * vk;
      R[(size_t)k * tmax + k] = alpha;
    }
    __syncthreads();
    const double vn2 = s_vn2;
    if (vn2 > 0.0) {
      for (int j = k + 1 + warp; j < t; j += nw) {
        double* y = W + (size_t)j * N;
        double d = 0.0;
        for (int i = k + lane; i < N; i += 32) d = fma(x[i], y[i], d);
        for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
        const double fct = 2.0 * d / vn2;
        for (int i = k + lane; i < N; i += 32) y[i] = fma(-fct, x[i], y[i]);
      }
    }
    __syncthreads();
  }
  for (int idx = tid; idx < t * t; idx += blockDim.x) {
    const int i = idx / t, j = idx % t;
    if (i < j && i < N) R[(size_t)i * tmax + j] = W[(size_t)j * N + i];
  }
}

// One-sided (Hestenes) Jacobi SVD of the t x t matrix G stored by columns (column j at
// G + j tmax): columns are rotated in round-robin pairs until mutually orthogonal, so G V =
// U Sigma with V accumulated by columns; sig[j] = ||G(:, j)||.  Singular values come out with
// absolute error ~ eps ||G||, without squaring the condition as a Gram matrix would.
__global__ void __launch_bounds__(1024) k_onesided_jacobi(double* __restrict__ G, double* __restrict__ V,
                                                          const int* __restrict__ tcount, int tmax,
                                                          double* __restrict__ sig) {
  __shared__ int s_rot;
  const int t = *tcount;
  const int tp = t + (t & 1);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int idx = tid; idx < t * t; idx += blockDim.x) V[(size_t)(idx / t) * tmax + idx % t] = (idx / t == idx % t);
  __syncthreads();
  for (int sweep = 0; sweep < 60 && t > 1; ++sweep) {
    if (tid == 0) s_rot = 0;
    __syncthreads();
    for (int round = 0; round < tp - 1; ++round) {
      for (int k = warp; k < tp / 2; k += nw) {
        const int i0 = k == 0 ? 0 : 1 + (k - 1 + round) % (tp - 1);
        const int j0 = 1 + (tp - 2 - k + round) % (tp - 1);
        const int p = min(i0, j0), q = max(i0, j0);
        if (q >= t) continue;
        double* gp = G + (size_t)p * tmax;
        double* gq = G + (size_t)q * tmax;
        double al = 0.0, be = 0.0, ga = 0.0;
        for (int i = lane; i < t; i += 32) {
          al = fma(gp[i], gp[i], al);
          be = fma(gq[i], gq[i], be);
          ga = fma(gp[i], gq[i], ga);
        }
        for (int o = 16; o > 0; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          ga += __shfl_xor_sync(0xffffffffu, ga, o);
        }
        if (!(ga != 0.0 && fabs(ga) > 1e-15 * sqrt(al * be))) continue;
        const double ze = (be - al) / (2.0 * ga);
        const double tt = (ze >= 0.0 ? 1.0 : -1.0) / (fabs(ze) + sqrt(1.0 + ze * ze));
        const double c = 1.0 / sqrt(1.0 + tt * tt), sn = c * tt;
        double* vp = V + (size_t)p * tmax;
        double* vq = V + (size_t)q * tmax;
        for (int i = lane; i < t; i += 32) {
          const double a = gp[i], b = gq[i];
          gp[i] = c * a - sn * b;
          gq[i] = sn * a + c * b;
          const double va = vp[i], vb = vq[i];
          vp[i] = c * va - sn * vb;
          vq[i] = sn * va + c * vb;
        }
        if (lane == 0) atomicAdd(&s_rot, 1);
      }
      __syncthreads();
    }
    const int rot = s_rot;
    __syncthreads();
    if (rot == 0) break;
  }
  for (int j = warp; j < t; j += nw) {
    double n2 = 0.0;
    for (int i = lane; i < t; i += 32) n2 = fma(G[(size_t)j * tmax + i], G[(size_t)j * tmax + i], n2);
    for (int o = 16; o > 0; o >>= 1) n2 += __shfl_xor_sync(0xffffffffu, n2, o);
    if (lane == 0) sig[j] = sqrt(n2);
  }
}

// stacked nodes mu = [lambda; upsilon] and rows c = [a; b] of the 2N x 2N PSD kernel
// -(c_x . c_y)/(mu_x + mu_y), whose off-diagonal block is the Sylvester Y~
__global__ void k_stack(const double* __restrict__ la, const double* __restrict__ aa, const double* __restrict__ lb,
                        const double* __restrict__ ab, int N, int s, double* __restrict__ mu,
                        double* __restrict__ c) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * N) return;
  const bool A = i < N;
  const int r = A ? i : i - N;
  mu[i] = A ? la[r] : lb[r];
  for (int k = 0; k < s; ++k) c[(size_t)i * s + k] = A ? aa[(size_t)r * s + k] : ab[(size_t)r * s + k];
}

// ---- Z += Vbuf (n x K) * Mg (K x t) -------------------------------------------
template <typename TV, typename TZ>
__global__ void __launch_bounds__(256) k_gemm_accum(int64_t n, int K, int t, const TV* __restrict__ Vb, int64_t ldv,
                                                    const double* __restrict__ Mg, int64_t ldm, TZ* __restrict__ Z,
                                                    int64_t ldz) {
  constexpr int BM = 64, BN = 64, BK = 16;
  __shared__ TZ As[BK][BM + 1];
  __shared__ TZ Bs[BK][BN];
  const int64_t row0 = (int64_t)blockIdx.x * BM;
  const int col0 = blockIdx.y * BN;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;  // 16 x 16 threads, 4 x 4 outputs each
  TZ acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = TZ(0);
  for (int k0 = 0; k0 < K; k0 += BK) {
    for (int idx = threadIdx.x; idx < BM * BK; idx += blockDim.x) {
      const int r = idx / BK, kk = idx % BK;
      const int64_t gr = row0 + r;
      As[kk][r] = (gr < n && k0 + kk < K) ? TZ(Vb[gr * ldv + k0 + kk]) : TZ(0);
    }
    for (int idx = threadIdx.x; idx < BK * BN; idx += blockDim.x) {
      const int kk = idx / BN, c = idx % BN;
      Bs[kk][c] = (k0 + kk < K && col0 + c < t) ? TZ(Mg[(int64_t)(k0 + kk) * ldm + col0 + c]) : TZ(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      TZ av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t gr = row0 + ty * 4 + i;
    if (gr >= n) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gc = col0 + tx * 4 + j;
      if (gc < t) Z[gr * ldz + gc] += acc[i][j];
    }
  }
}

// Z += Vbuf M with float pairs: V holds rows of S pairs per block (the S high parts, then the S
// low parts), Z holds pairs in the 8 bytes of each of its doubles until k_pairs_to_double
// (BM x BN tiles, 256 threads of 4 x 4 outputs: BM = 4 * 256 / (BN / 4))
template <int S, int BN>
__global__ void __launch_bounds__(256) k_gemm_accum_ff(int64_t n, int K, int t, const float* __restrict__ Vb,
                                                       int64_t ldv, const float2* __restrict__ Mp, int64_t ldm,
                                                       float2* __restrict__ Z, int64_t ldz) {
  constexpr int TXN = BN / 4, BM = 4 * (256 / TXN), BK = 16;
  __shared__ ff As[BK][BM + 1];
  __shared__ ff Bs[BK][BN];
  const int64_t row0 = (int64_t)blockIdx.x * BM;
  const int col0 = blockIdx.y * BN;
  const int tx = threadIdx.x % TXN, ty = threadIdx.x / TXN;
  ff acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = ff_make(0.f, 0.f);
  for (int k0 = 0; k0 < K; k0 += BK) {
    for (int idx = threadIdx.x; idx < BM * BK; idx += blockDim.x) {
      const int r = idx / BK, kk = idx % BK;
      const int64_t gr = row0 + r;
      const int k = k0 + kk;
      ff v = ff_make(0.f, 0.f);
      if (gr < n && k < K) {
        // value k of row gr: block k / S, column k % S
        const float* p = Vb + 2 * (gr * ldv + (int64_t)(k / S) * S);
        v = ff_make(p[k % S], p[S + k % S]);
      }
      As[kk][r] = v;
    }
    for (int idx = threadIdx.x; idx < BK * BN; idx += blockDim.x) {
      const int kk = idx / BN, c = idx % BN;
      const float2 b = (k0 + kk < K && col0 + c < t) ? Mp[(int64_t)(k0 + kk) * ldm + col0 + c] : make_float2(0.f, 0.f);
      Bs[kk][c] = ff_make(b.x, b.y);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      ff av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) ff_acc(acc[i][j], av[i], bv[j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t gr = row0 + ty * 4 + i;
    if (gr >= n) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gc = col0 + tx * 4 + j;
      if (gc < t) {
        const float2 z = Z[gr * ldz + gc];
        const ff r = ff_add(ff_make(z.x, z.y), ff_norm(acc[i][j]));
        Z[gr * ldz + gc] = make_float2(r.hi, r.lo);
      }
    }
  }
}

// doubles -> the pairs nearest them, in place (rows x cols of leading dimension ld)
__global__ void k_double_to_pairs(double* A, int64_t rows, int64_t ld, int cols) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * cols) return;
  double* a = A + (i / cols) * ld + (i % cols);
  const ff p = ff_from_double(*a);
  *reinterpret_cast<float2*>(a) = make_float2(p.hi, p.lo);
}

// the pairs accumulated in Z's doubles -> their fp64 values
__global__ void k_pairs_to_double(double* Z, int64_t n, int64_t ldz, int t) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * t) return;
  double* z = Z + (i / t) * ldz + (i % t);
  const float2 p = *reinterpret_cast<const float2*>(z);
  *z = (double)p.x + (double)p.y;
}

template <typename TZ>
__global__ void k_zero_cols(TZ* Z, int64_t n, int64_t ldz, int t) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * t) return;
  Z[(i / t) * ldz + (i % t)] = TZ(0);
}

void gemm_accum(int bulk, int s, int z_f32, int64_t n, int K, int t, const void* Vb, int64_t ldv, const double* Mg,
                int64_t ldm, void* Z, int64_t ldz, cudaStream_t st) {
  if (t <= 0 || K <= 0) return;
  dim3 grid((unsigned)((n + 63) / 64), (unsigned)((t + 63) / 64));
  if (bulk == LYAP_PREC_F32X2) {
    // the column tile (16, 32 or 64 wide; 256, 128 or 64-row tiles) with the fewest padded
    // columns: the pair products are the cost, re-reading the basis rows per column tile is not
    const float2* Mp = reinterpret_cast<const float2*>(Mg);  // converted in place by the caller
    const int w64 = (t + 63) / 64 * 64, w32 = (t + 31) / 32 * 32, w16 = (t + 15) / 16 * 16;
    const int bn = w16 < w32 ? 16 : (w32 < w64 ? 32 : 64);
    dim3 gf((unsigned)((n + 4096 / bn - 1) / (4096 / bn)), (unsigned)((t + bn - 1) / bn));
#define LYAP_GFF(SS_)                                                                                          \
  if (bn == 16)                                                                                                \
    k_gemm_accum_ff<SS_, 16><<<gf, 256, 0, st>>>(n, K, t, (const float*)Vb, ldv, Mp, ldm, (float2*)Z, ldz);     \
  else if (bn == 32)                                                                                           \
    k_gemm_accum_ff<SS_, 32><<<gf, 256, 0, st>>>(n, K, t, (const float*)Vb, ldv, Mp, ldm, (float2*)Z, ldz);     \
  else                                                                                                         \
    k_gemm_accum_ff<SS_, 64><<<gf, 256, 0, st>>>(n, K, t, (const float*)Vb, ldv, Mp, ldm, (float2*)Z, ldz)
    switch (s) {
      case 1: LYAP_GFF(1); break;
      case 2: LYAP_GFF(2); break;
      case 3: LYAP_GFF(3); break;
      case 4: LYAP_GFF(4); break;
    }
#undef LYAP_GFF
  } else if (bulk == LYAP_PREC_MIXED && z_f32) {
    k_gemm_accum<float, float><<<grid, 256, 0, st>>>(n, K, t, (const float*)Vb, ldv, Mg, ldm, (float*)Z, ldz);
  } else if (bulk == LYAP_PREC_MIXED) {
    k_gemm_accum<float, double><<<grid, 256, 0, st>>>(n, K, t, (const float*)Vb, ldv, Mg, ldm, (double*)Z, ldz);
  } else {
    k_gemm_accum<double, double><<<grid, 256, 0, st>>>(n, K, t, (const double*)Vb, ldv, Mg, ldm, (double*)Z, ldz);
  }
}

FactorWs carve(char* base, int s, int nmax2, int tmax, int nmax) {
  FactorWs f;
  char* p = base;
  auto take = [&](size_t bytes) { char* r = p; p += lyap_align256((int64_t)bytes); return r; };
  f.L = (double*)take(sizeof(double) * (size_t)tmax * nmax2);
  f.piv = (int*)take(sizeof(int) * (size_t)tmax);
  f.tcount = (int*)take(sizeof(int) * 4);
  f.K = (double*)take(sizeof(double) * (size_t)tmax * tmax);
  f.Vk = (double*)take(sizeof(double) * (size_t)tmax * tmax);
  f.ev = (double*)take(sizeof(double) * (size_t)tmax);
  f.chol = (double*)take(sizeof(double) * (size_t)tmax * (s + 1) * nmax);
  f.B = (double*)take(sizeof(double) * (size_t)nmax2 * tmax);
  f.M = (double*)take(sizeof(double) * (size_t)nmax2 * tmax);
  return f;
}

// second pass for one operator: regenerate V_1..V_m and accumulate Z += V_j E_j^T M
int second_pass(lyap_handle* h, int opi, const double* M, int ldm, int tk, void* Z, int64_t ldz, int z_f32,
                cudaStream_t st) {
  OpDev& op = h->op[opi];
  const int s = h->s, m = h->m, kb = h->plan.pass2_blocks;
  const int bulk = h->plan.bulk;
  const size_t w = bulk == LYAP_PREC_MIXED ? 4 : 8;
  const int64_t n = op.n;
  const int64_t ldb = (int64_t)kb * s;
  char* buf[2] = {reinterpret_cast<char*>(op.V[0]) + 0, nullptr};
  // the pass-2 buffers sit after the factor scratch: operator 0's pair, then operator 1's
  buf[0] = h->factor_ws + h->plan.factor_bytes +
           (opi ? 2 * (size_t)lyap_align256((int64_t)(h->op[0].n * ldb * w)) : 0);
  buf[1] = buf[0] + lyap_align256((int64_t)(n * ldb * w));
  auto pos = [&](int j) -> char* {  // block j (1-based)
    const int g = (j - 1) / kb, c = (j - 1) % kb;
    return buf[g & 1] + (size_t)c * s * w;
  };
  if (tk > 0 && bulk == LYAP_PREC_F32X2) {
    // the pair GEMM reads M as pairs: rows 0..m s - 1, columns 0..tk - 1, converted in place
    const int64_t tot = (int64_t)m * s * tk;
    k_double_to_pairs<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(const_cast<double*>(M), (int64_t)m * s, ldm, tk);
    h->launches += 1;
  }
  if (tk > 0) {
    const int64_t tot = n * tk;
    if (z_f32) k_zero_cols<float><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>((float*)Z, n, ldz, tk);
    else k_zero_cols<double><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>((double*)Z, n, ldz, tk);
    h->launches += 1;
  }
  launch_pass2_v1(op, s, bulk, h->plan.sweep_grid, pos(1), ldb, st);
  h->launches += 1;
  for (int j = 1; j <= m; ++j) {
    if (j < m) {
      const void* vp = j > 1 ? pos(j - 1) : pos(j);
      launch_pass2(op, s, bulk, h->plan.sweep_grid, j, vp, ldb, pos(j), ldb, pos(j + 1), ldb, st);
      h->launches += 1;
    }
    const bool group_end = (j % kb == 0) || j == m;
    if (group_end && tk > 0) {
      const int g = (j - 1) / kb;
      const int j0 = g * kb + 1;
      const int nblk = j - j0 + 1;
      gemm_accum(bulk, s, z_f32, n, nblk * s, tk, buf[g & 1], ldb, M + (size_t)(j0 - 1) * s * ldm, ldm, Z, ldz, st);
      h->launches += 1;
    }
  }
  if (bulk == LYAP_PREC_F32X2 && tk > 0) {
    const int64_t tot = n * tk;
    k_pairs_to_double<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>((double*)Z, n, ldz, tk);
    h->launches += 1;
  }
  return cudaGetLastError() == cudaSuccess ? LYAP_OK : LYAP_ERR_CUDA;
}

}  // namespace

size_t factor_ws_bytes(int s, int nmax, int sylv) {
  const int nmax2 = sylv ? 2 * nmax : nmax;
  const int tmax = nmax2 < kTmaxCap ? nmax2 : kTmaxCap;
  size_t b = 0;
  auto add = [&](size_t bytes) { b += lyap_align256((int64_t)bytes); };
  add(sizeof(double) * (size_t)tmax * nmax2);
  add(sizeof(int) * (size_t)tmax);
  add(sizeof(int) * 4);
  add(sizeof(double) * (size_t)tmax * tmax);
  add(sizeof(double) * (size_t)tmax * tmax);
  add(sizeof(double) * (size_t)tmax);
  add(sizeof(double) * (size_t)tmax * (s + 1) * nmax);
  add(sizeof(double) * (size_t)nmax2 * tmax);
  add(sizeof(double) * (size_t)nmax2 * tmax);
  add(sizeof(double) * (size_t)nmax2);  // diagonal scratch of the pivoted Cholesky
  add(sizeof(int) * (size_t)tmax);      // kept-column order
  if (!sylv) add(sizeof(double) * 3 * (size_t)tmax * tmax);  // U rows of the tridiagonal inverse iteration
  if (sylv) {
    add(sizeof(double) * (size_t)nmax2);          // stacked nodes
    add(sizeof(double) * (size_t)nmax2 * s);      // stacked rows
    for (int k = 0; k < 6; ++k) add(sizeof(double) * (size_t)tmax * tmax);  // R_A, R_B, G, V_G, R1, R2
    for (int k = 0; k < 2; ++k) add(sizeof(double) * (size_t)tmax * nmax);  // Householder work
    add(sizeof(double) * 3 * (size_t)tmax);       // column scales, singular values
  }
  return b;
}

size_t pass2_ws_bytes(int64_t n, int s, int kb, int bulk) {
  const size_t w = bulk == LYAP_PREC_MIXED ? 4 : 8;
  return 2 * (size_t)lyap_align256((int64_t)(n * (int64_t)kb * s * w));
}

// eps of eq. 2.5: the option, or, when it is 0, min(1e-12, tol / (10 (||T_m|| + ||J_m||))), so that
// the truncation moves the residual by at most tol / 10 (J_m = T_m for Lyapunov).  ||T_m|| is the
// largest |eigenvalue|, the first or last of the ascending list.
int trunc_eps_of(lyap_handle* h, const double* lam_a, const double* lam_b, int N, double* eps, cudaStream_t st,
                 int Nb = -1) {
  if (Nb < 0) Nb = N;
  if (h->opt.trunc_eps > 0.0) {
    *eps = h->opt.trunc_eps;
    return LYAP_OK;
  }
  double ends[4] = {0.0, 0.0, 0.0, 0.0};
  LYAP_CUDA_TRY(cudaMemcpyAsync(&ends[0], lam_a, sizeof(double), cudaMemcpyDeviceToHost, st));
  LYAP_CUDA_TRY(cudaMemcpyAsync(&ends[1], lam_a + N - 1, sizeof(double), cudaMemcpyDeviceToHost, st));
  if (lam_b) {
    LYAP_CUDA_TRY(cudaMemcpyAsync(&ends[2], lam_b, sizeof(double), cudaMemcpyDeviceToHost, st));
    LYAP_CUDA_TRY(cudaMemcpyAsync(&ends[3], lam_b + Nb - 1, sizeof(double), cudaMemcpyDeviceToHost, st));
  }
  LYAP_CUDA_TRY(cudaStreamSynchronize(st));
  const double na = fmax(fabs(ends[0]), fabs(ends[1]));
  const double nb = lam_b ? fmax(fabs(ends[2]), fabs(ends[3])) : na;
  double e = 1e-12;
  if (na + nb > 0.0 && isfinite(na + nb)) e = fmin(e, h->tol / (10.0 * (na + nb)));
  *eps = e;
  return LYAP_OK;
}

// Sylvester factors (Sec. 5.1): Y~_ij = -(a_i . b_j)/(lambda_i + upsilon_j) is the off-diagonal
// block of the 2N x 2N positive semidefinite kernel -(c_x . c_y)/(mu_x + mu_y) on the stacked
// nodes mu = [lambda; upsilon] and rows c = [a; b] (a Schur product of a Gram matrix and the
// Cauchy matrix -1/(mu_x + mu_y), all mu < 0).  Its pivoted Cholesky factor [L_A; L_B] gives
// Y~ ~= L_A L_B^T with an error below the remainder's trace.  With the Householder R factors
// L_A = U_A R_A, L_B = U_B R_B and the SVD R_A R_B^T = U_G Sigma V_G^T (one-sided Jacobi),
//   Y1 = L_A R_B^T V_G,t Sigma_t^{-1/2},   Y2 = L_B R_A^T U_G,t Sigma_t^{1/2}
//                                             = L_B R_A^T (G V_G)_t Sigma_t^{-1/2} Sigma_t^{-1},
// so Y1 Y2^T is the truncated SVD of L_A L_B^T and only kept singular values are divided by.
// As in the Lyapunov case Q L_A and P L_B come from shifted band solves, so M1 = Q Y1 and
// M2 = P Y2 are formed without Q or P; the truncation keeps the fewest singular values whose
// discarded tail has Frobenius norm <= eps = trunc_eps ||C1||_F ||C2||_F.
int run_factor_sylv(lyap_handle* h, void* Z1, int64_t ldz1, void* Z2, int64_t ldz2, int z_dtype, int tcap, int* t_out,
                    cudaStream_t st) {
  const int s = h->s, m = h->m, N = s * m, N2 = 2 * N;
  const int nmax = h->plan.nmax, nmax2 = 2 * nmax;
  const int tmax = nmax2 < kTmaxCap ? nmax2 : kTmaxCap;
  FactorWs f = carve(h->factor_ws, s, nmax2, tmax, nmax);
  char* p = reinterpret_cast<char*>(f.M) + lyap_align256((int64_t)(sizeof(double) * (size_t)nmax2 * tmax));
  auto take = [&](size_t bytes) { char* r = p; p += lyap_align256((int64_t)bytes); return r; };
  double* dg = (double*)take(sizeof(double) * nmax2);
  int* order_d = (int*)take(sizeof(int) * tmax);
  double* mu = (double*)take(sizeof(double) * nmax2);
  double* cst = (double*)take(sizeof(double) * (size_t)nmax2 * s);
  const size_t tt = (size_t)tmax * tmax;
  double* RA = (double*)take(sizeof(double) * tt);
  double* RB = (double*)take(sizeof(double) * tt);
  double* Gc = (double*)take(sizeof(double) * tt);
  double* VG = (double*)take(sizeof(double) * tt);
  double* R1 = (double*)take(sizeof(double) * tt);
  double* R2 = (double*)take(sizeof(double) * tt);
  double* WA = (double*)take(sizeof(double) * (size_t)tmax * nmax);
  double* WBh = (double*)take(sizeof(double) * (size_t)tmax * nmax);
  double* scl = (double*)take(sizeof(double) * 3 * (size_t)tmax);
  double* sig_d = scl + 2 * (size_t)tmax;

  // 1. eigenvalues and first-block rows of both projected matrices (Alg. 4 steps 1-4)
  h->launches += launch_eigen_for_factor(h, 0, m, st);
  h->launches += launch_eigen_for_factor(h, 1, m, st);
  double *la, *aa, *wa, *lb, *ab, *wb;
  check_slot0(h, 0, &la, &aa, &wa);
  check_slot0(h, 1, &lb, &ab, &wb);
  k_stack<<<(N2 + 127) / 128, 128, 0, st>>>(la, aa, lb, ab, N, s, mu, cst);
  // 2. pivoted Cholesky of the stacked kernel
  double teps = 0.0;
  int rc_e = trunc_eps_of(h, la, lb, N, &teps, st);
  if (rc_e != LYAP_OK) return rc_e;
  const double eps_abs = teps * h->op[0].beta * h->op[1].beta;
  k_pivoted_cholesky<<<1, kPcThreads, 0, st>>>(mu, cst, N2, s, tmax, 1e-2 * eps_abs, f, dg);
  h->launches += 2;
  LYAP_CUDA_TRY(cudaMemcpyAsync(h->flags_host + 2, f.tcount, sizeof(int), cudaMemcpyDeviceToHost, st));
  LYAP_CUDA_TRY(cudaStreamSynchronize(st));
  const int tpc = h->flags_host[2];
  if (tpc <= 0) {
    *t_out = 0;
    return LYAP_OK;
  }
  // 3. [Q L_A; P L_B] by shifted band solves with T_m (rows 0..N-1) and J_m (rows N..2N-1)
  const int nthr = 64;
  k_shifted_solves<<<(tpc + nthr - 1) / nthr, nthr, 0, st>>>(h->op[0].log, s, m, mu, cst, f, tmax, nmax, 0, 0, N2,
                                                             h->flags);
  k_shifted_solves<<<(tpc + nthr - 1) / nthr, nthr, 0, st>>>(h->op[1].log, s, m, mu, cst, f, tmax, nmax, N * tmax,
                                                             0, N2, h->flags);
  k_apply_lpp<<<(N2 + 127) / 128, 128, 0, st>>>(f, N2, N2, tmax);
  // 4. R_A, R_B; G = R_A R_B^T by columns (G(:, j) = R_A R_B(j, :)^T); its one-sided Jacobi SVD
  k_householder_r<<<2, 1024, 0, st>>>(f.L, N2, N, N, f.tcount, WA, WBh, RA, RB, tmax);
  small_gemm(RB, tmax, 0, RA, tmax, 1, nullptr, nullptr, Gc, tmax, tpc, tpc, f.tcount, st);
  k_onesided_jacobi<<<1, 1024, 0, st>>>(Gc, VG, f.tcount, tmax, sig_d);
  h->launches += 6;
  std::vector<double> sig(tpc);
  LYAP_CUDA_TRY(cudaMemcpyAsync(sig.data(), sig_d, sizeof(double) * tpc, cudaMemcpyDeviceToHost, st));
  LYAP_CUDA_TRY(cudaStreamSynchronize(st));
  // 5. truncation on the singular values, non-increasing (eq. 2.5 applied to the SVD of Y~)
  std::vector<int> order(tpc);
  for (int i = 0; i < tpc; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return sig[x] > sig[y]; });
  std::vector<double> tail(tpc + 1, 0.0);
  for (int i = tpc - 1; i >= 0; --i) tail[i] = tail[i + 1] + sig[order[i]] * sig[order[i]];
  int tk = 0;
  while (tk < tpc && !(sqrt(tail[tk]) <= eps_abs)) ++tk;
  while (tk > 0 && !(sig[order[tk - 1]] > 0.0)) --tk;
  *t_out = tk;
  if (tk > tcap) return LYAP_ERR_TCAP;
  std::vector<double> sc(2 * (size_t)tmax, 0.0);
  for (int c = 0; c < tk; ++c) {
    const double sg = sig[order[c]];
    sc[c] = 1.0 / sqrt(sg);
    sc[tmax + c] = 1.0 / (sg * sqrt(sg));
  }
  if (tk > 0) {
    LYAP_CUDA_TRY(cudaMemcpyAsync(order_d, order.data(), sizeof(int) * tk, cudaMemcpyHostToDevice, st));
    LYAP_CUDA_TRY(cudaMemcpyAsync(scl, sc.data(), sizeof(double) * 2 * tmax, cudaMemcpyHostToDevice, st));
    // 6. R1 = R_B^T V_G,t Sigma^{-1/2}, R2 = R_A^T (G V_G)_t Sigma^{-3/2}; M1 = (Q L_A) R1, M2 = (P L_B) R2
    small_gemm(RB, tmax, 1, VG, tmax, 1, order_d, scl, R1, tmax, tpc, tk, f.tcount, st);
    small_gemm(RA, tmax, 1, Gc, tmax, 1, order_d, scl + tmax, R2, tmax, tpc, tk, f.tcount, st);
    small_gemm(f.B, tmax, 0, R1, tmax, 0, nullptr, nullptr, f.M, tmax, N, tk, f.tcount, st);
    small_gemm(f.B + (size_t)N * tmax, tmax, 0, R2, tmax, 0, nullptr, nullptr, f.M + (size_t)N * tmax, tmax, N, tk,
               f.tcount, st);
    h->launches += 4;
  }
  // 7. second passes: Z1 = V_m M1, Z2 = U_m M2
  int rc = second_pass(h, 0, f.M, tmax, tk, Z1, ldz1, z_dtype == LYAP_F32, st);
  if (rc != LYAP_OK) return rc;
  rc = second_pass(h, 1, f.M + (size_t)N * tmax, tmax, tk, Z2, ldz2, z_dtype == LYAP_F32, st);
  if (rc != LYAP_OK) return rc;
  LYAP_CUDA_TRY(cudaStreamSynchronize(st));  // keeps the host vectors alive until the copies ran
  return LYAP_OK;
}

// Lyapunov factor up to M = Q_m Ycheck (N x tk, leading dimension tmax, in the factor scratch):
// steps 1-5 of the truncation; *t_out = tk (0: nothing to accumulate)
int factor_core(lyap_handle* h, int tcap, int* t_out, double** M_out, int* ldm_out, cudaStream_t st) {
  const int s = h->s, m = h->m, N = s * m;
  const int nmax = h->plan.nmax;
  const int tmax = nmax < kTmaxCap ? nmax : kTmaxCap;
  FactorWs f = carve(h->factor_ws, s, nmax, tmax, nmax);
  char* after = reinterpret_cast<char*>(f.M) + lyap_align256((int64_t)(sizeof(double) * (size_t)nmax * tmax));
  double* dg = reinterpret_cast<double*>(after);
  int* order_d = reinterpret_cast<int*>(after + lyap_align256((int64_t)(sizeof(double) * nmax)));
  double* ew = reinterpret_cast<double*>(reinterpret_cast<char*>(order_d) + lyap_align256((int64_t)(sizeof(int) * tmax)));

  // 1. eigenvalues lambda and rows a = (Q^T E_1 gamma) of T_m (Alg. 3 steps 1-4)
  h->launches += launch_eigen_for_factor(h, 0, m, st);
  double *lam, *a, *w;
  check_slot0(h, 0, &lam, &a, &w);
  // 2. pivoted Cholesky of Y~ = -(a_i . a_j)/(lambda_i + lambda_j)
  const double beta2 = h->op[0].beta * h->op[0].beta;
  double teps = 0.0;
  int rc_e = trunc_eps_of(h, lam, nullptr, N, &teps, st);
  if (rc_e != LYAP_OK) return rc_e;
  const double eps_abs = teps * beta2;
  k_pivoted_cholesky<<<1, kPcThreads, 0, st>>>(lam, a, N, s, tmax, 1e-2 * eps_abs, f, dg);
  h->launches += 1;
  LYAP_CUDA_TRY(cudaMemcpyAsync(h->flags_host + 2, f.tcount, sizeof(int), cudaMemcpyDeviceToHost, st));
  LYAP_CUDA_TRY(cudaStreamSynchronize(st));
  const int tpc = h->flags_host[2];
  *M_out = f.M;
  *ldm_out = tmax;
  if (tpc <= 0) {
    *t_out = 0;
    return LYAP_OK;
  }
  // 3. B = Q Y~(:,P) by shifted SND band solves, X = B L_PP^{-T} (= Q L)
  const int nthr = 64;
  k_shifted_solves<<<(tpc + nthr - 1) / nthr, nthr, 0, st>>>(h->op[0].log, s, m, lam, a, f, tmax, nmax, 0, 0, N,
                                                             h->flags);
  k_apply_lpp<<<(N + 127) / 128, 128, 0, st>>>(f, N, N, tmax);
  h->launches += 2;
  // 4. K = L^T L and its eigendecomposition (eigenpairs of L L^T)
  k_gram_L<<<dim3(tpc, (tpc + 127) / 128), 128, 0, st>>>(f, N, 0, N, tmax, f.K);
  k_tridiag<<<1, 1024, 0, st>>>(f, tmax);
  k_tri_eigvec<<<(tpc + 63) / 64, 64, 0, st>>>(f, tmax, ew);
  k_tri_reorth<<<1, 32, 0, st>>>(f, tmax);
  h->launches += 4;
  std::vector<double> ev(tpc);
  LYAP_CUDA_TRY(cudaMemcpyAsync(ev.data(), f.ev, sizeof(double) * tpc, cudaMemcpyDeviceToHost, st));
  LYAP_CUDA_TRY(cudaStreamSynchronize(st));
  // truncation (eq. 2.5): eigenvalues non-increasing; keep the fewest so that the
  // discarded tail has Frobenius norm <= eps; negative values are never kept
  std::vector<int> order(tpc);
  for (int i = 0; i < tpc; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return ev[x] > ev[y]; });
  std::vector<double> tail(tpc + 1, 0.0);
  for (int i = tpc - 1; i >= 0; --i) tail[i] = tail[i + 1] + ev[order[i]] * ev[order[i]];
  int tk = 0;
  while (tk < tpc && !(sqrt(tail[tk]) <= eps_abs)) ++tk;
  int npos = 0;
  for (int i = 0; i < tpc; ++i) npos += ev[i] > 0.0;
  if (tk > npos) tk = npos;
  *t_out = tk;
  if (tk > tcap) return LYAP_ERR_TCAP;
  if (tk > 0) LYAP_CUDA_TRY(cudaMemcpyAsync(order_d, order.data(), sizeof(int) * tk, cudaMemcpyHostToDevice, st));
  // 5. M = X V(:, kept) = Q Ycheck, then the second pass Z = sum_j V_j E_j^T M
  if (tk > 0) {
    k_form_M<<<dim3((N + 127) / 128, tk), 128, 0, st>>>(f, N, tmax, order_d, tk, 0, f.M, tmax);
    h->launches += 1;
  }
  LYAP_CUDA_TRY(cudaStreamSynchronize(st));  // the order vector above is a local host buffer
  return LYAP_OK;
}

namespace {

// ---- large A, small B (Sec. 5.2, Alg. 5): only A is projected; B = P Upsilon P^T once ------------
// stacked nodes mu = [lambda (N); upsilon (n2)] and rows c = [a (N x s); ctil = P^T C2 (n2 x s)]
__global__ void k_smallb_stack(const double* __restrict__ lam, const double* __restrict__ a, int N,
                               const double* __restrict__ ups, const double* __restrict__ ct, int n2, int s,
                               double* __restrict__ mu, double* __restrict__ c) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N + n2) return;
  const bool A = i < N;
  const int r = A ? i : i - N;
  mu[i] = A ? lam[r] : ups[r];
  for (int k = 0; k < s; ++k) c[(size_t)i * s + k] = A ? a[(size_t)r * s + k] : ct[(size_t)r * s + k];
}

// out[i][k] = -(ctil_i . c_{p_k}) / (upsilon_i + mu_{p_k}): the B rows of the stacked kernel at the
// pivots, before the multiplication by P
__global__ void k_smallb_brows(FactorWs f, int N, int n2, int s, const double* __restrict__ mu,
                               const double* __restrict__ c, double* __restrict__ out, int ldo) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  const int t = f.tcount[0];
  if (i >= n2 || k >= t) return;
  const int p = f.piv[k];
  double dot = 0.0;
  for (int q = 0; q < s; ++q) dot = fma(c[(size_t)(N + i) * s + q], c[(size_t)p * s + q], dot);
  out[(size_t)i * ldo + k] = -dot / (mu[N + i] + mu[p]);
}

// the rows of M2 (n2 x tk, leading dimension tmax) into the caller's Z2 (fp64 or fp32)
template <typename TZ>
__global__ void k_copy_z2(const double* __restrict__ M2, int ldm, int n2, int tk, TZ* __restrict__ Z, int64_t ldz) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n2 * tk) return;
  const int r = (int)(idx / tk), c = (int)(idx % tk);
  Z[(size_t)r * ldz + c] = (TZ)M2[(size_t)r * ldm + c];
}

}  // namespace

// Eigenpairs of the symmetric n x n matrix K (row-major, leading dimension ld; overwritten):
// eigenvalues ascending into ev, eigenvector j into column j of V (leading dimension ld).  scratch:
// 4 n + 3 n^2 doubles; cnt: one device int.  Same kernels as the factor's t x t problem.
int dense_eigh(double* K, int n, int ld, double* ev, double* V, double* scratch, int* cnt, cudaStream_t st) {
  if (n <= 0) return LYAP_OK;
  FactorWs f{};
  f.K = K;
  f.Vk = V;
  f.ev = ev;
  f.chol = scratch;
  f.tcount = cnt;
  LYAP_CUDA_TRY(cudaMemcpyAsync(cnt, &n, sizeof(int), cudaMemcpyHostToDevice, st));
  k_tridiag<<<1, 1024, 0, st>>>(f, ld);
  k_tri_eigvec<<<(n + 63) / 64, 64, 0, st>>>(f, ld, scratch + 4 * (size_t)ld);
  k_tri_reorth<<<1, 32, 0, st>>>(f, ld);
  LYAP_CUDA_TRY(cudaStreamSynchronize(st));  // n lives on the host stack
  return cudaGetLastError() == cudaSuccess ? LYAP_OK : LYAP_ERR_CUDA;
}

// Z1 = V_m (Q Y1) by the second pass and Z2 = P Y2, with Y~ = -(a_k . ctil_j)/(lambda_k + upsilon_j)
// ~= Y1 Y2^T truncated (the end of Sec. 5.2); the truncated SVD as in the two-sided case, on the
// stacked kernel with nodes [lambda; upsilon] and rows [a; ctil] (unequal halves N and n2).
int run_factor_smallb(lyap_handle* h, void* Z1, int64_t ldz1, void* Z2, int64_t ldz2, int z_dtype, int tcap,
                      int* t_out, cudaStream_t st) {
  const int s = h->s, m = h->m, N = s * m;
  const int n2 = h->plan.n2, NT = N + n2;
  const int nmax = h->plan.nmax, nmax2 = 2 * nmax;
  const int tmax = nmax2 < kTmaxCap ? nmax2 : kTmaxCap;
  FactorWs f = carve(h->factor_ws, s, nmax2, tmax, nmax);
  char* p = reinterpret_cast<char*>(f.M) + lyap_align256((int64_t)(sizeof(double) * (size_t)nmax2 * tmax));
  auto take = [&](size_t bytes) { char* r = p; p += lyap_align256((int64_t)bytes); return r; };
  double* dg = (double*)take(sizeof(double) * nmax2);
  int* order_d = (int*)take(sizeof(int) * tmax);
  double* mu = (double*)take(sizeof(double) * nmax2);
  double* cst = (double*)take(sizeof(double) * (size_t)nmax2 * s);
  const size_t tt = (size_t)tmax * tmax;
  double* RA = (double*)take(sizeof(double) * tt);
  double* RB = (double*)take(sizeof(double) * tt);
  double* Gc = (double*)take(sizeof(double) * tt);
  double* VG = (double*)take(sizeof(double) * tt);
  double* R1 = (double*)take(sizeof(double) * tt);
  double* R2 = (double*)take(sizeof(double) * tt);
  double* WA = (double*)take(sizeof(double) * (size_t)tmax * nmax);
  double* WBh = (double*)take(sizeof(double) * (size_t)tmax * nmax);
  double* scl = (double*)take(sizeof(double) * 3 * (size_t)tmax);
  double* sig_d = scl + 2 * (size_t)tmax;
  const SmallB& sb = h->smallb;

  // 1. eigenvalues and rows a of T_m (Alg. 5 steps 1-4), stacked with those of B
  h->launches += launch_eigen_for_factor(h, 0, m, st);
  double *la, *aa, *wa;
  check_slot0(h, 0, &la, &aa, &wa);
  k_smallb_stack<<<(NT + 127) / 128, 128, 0, st>>>(la, aa, N, sb.ups, sb.ctil, n2, s, mu, cst);
  // 2. pivoted Cholesky of the stacked kernel
  double teps = 0.0;
  int rc_e = trunc_eps_of(h, la, sb.ups, N, &teps, st, n2);
  if (rc_e != LYAP_OK) return rc_e;
  const double eps_abs = teps * h->op[0].beta * sb.c2norm;
  k_pivoted_cholesky<<<1, kPcThreads, 0, st>>>(mu, cst, NT, s, tmax, 1e-2 * eps_abs, f, dg);
  h->launches += 2;
  LYAP_CUDA_TRY(cudaMemcpyAsync(h->flags_host + 2, f.tcount, sizeof(int), cudaMemcpyDeviceToHost, st));
  LYAP_CUDA_TRY(cudaStreamSynchronize(st));
  const int tpc = h->flags_host[2];
  if (tpc <= 0) {
    *t_out = 0;
    return LYAP_OK;
  }
  // 3. [Q L_A; P L_B]: the A rows by shifted band solves with T_m (every pivot, A or B side), the
  //    B rows as P times the kernel's B rows at the pivots; then L_PP^{-T} on all rows
  const int nthr = 64;
  k_shifted_solves<<<(tpc + nthr - 1) / nthr, nthr, 0, st>>>(h->op[0].log, s, m, mu, cst, f, tmax, nmax, 0, 0, NT,
                                                             h->flags);
  k_smallb_brows<<<dim3((n2 + 127) / 128, tpc), 128, 0, st>>>(f, N, n2, s, mu, cst, f.M, tmax);
  small_gemm(sb.P, n2, 0, f.M, tmax, 0, nullptr, nullptr, f.B + (size_t)N * tmax, tmax, n2, tpc, sb.d_n2, st);
  k_apply_lpp<<<(NT + 127) / 128, 128, 0, st>>>(f, NT, NT, tmax);
  // 4. R_A, R_B; G = R_A R_B^T; its one-sided Jacobi SVD
  k_householder_r<<<2, 1024, 0, st>>>(f.L, NT, N, n2, f.tcount, WA, WBh, RA, RB, tmax);
  small_gemm(RB, tmax, 0, RA, tmax, 1, nullptr, nullptr, Gc, tmax, tpc, tpc, f.tcount, st);
  k_onesided_jacobi<<<1, 1024, 0, st>>>(Gc, VG, f.tcount, tmax, sig_d);
  h->launches += 8;
  std::vector<double> sig(tpc);
  LYAP_CUDA_TRY(cudaMemcpyAsync(sig.data(), sig_d, sizeof(double) * tpc, cudaMemcpyDeviceToHost, st));
  LYAP_CUDA_TRY(cudaStreamSynchronize(st));
  // 5. truncation on the singular values, non-increasing (eq. 2.5 applied to the SVD of Y~)
  std::vector<int> order(tpc);
  for (int i = 0; i < tpc; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return sig[x] > sig[y]; });
  std::vector<double> tail(tpc + 1, 0.0);
  for (int i = tpc - 1; i >= 0; --i) tail[i] = tail[i + 1] + sig[order[i]] * sig[order[i]];
  int tk = 0;
  while (tk < tpc && !(sqrt(tail[tk]) <= eps_abs)) ++tk;
  while (tk > 0 && !(sig[order[tk - 1]] > 0.0)) --tk;
  *t_out = tk;
  if (tk > tcap) return LYAP_ERR_TCAP;
  std::vector<double> sc(2 * (size_t)tmax, 0.0);
  for (int c = 0; c < tk; ++c) {
    const double sg = sig[order[c]];
    sc[c] = 1.0 / sqrt(sg);
    sc[tmax + c] = 1.0 / (sg * sqrt(sg));
  }
  if (tk > 0) {
    LYAP_CUDA_TRY(cudaMemcpyAsync(order_d, order.data(), sizeof(int) * tk, cudaMemcpyHostToDevice, st));
    LYAP_CUDA_TRY(cudaMemcpyAsync(scl, sc.data(), sizeof(double) * 2 * tmax, cudaMemcpyHostToDevice, st));
    // 6. R1 = R_B^T V_G,t Sigma^{-1/2}, R2 = R_A^T (G V_G)_t Sigma^{-3/2}; M1 = (Q L_A) R1, M2 = (P L_B) R2
    small_gemm(RB, tmax, 1, VG, tmax, 1, order_d, scl, R1, tmax, tpc, tk, f.tcount, st);
    small_gemm(RA, tmax, 1, Gc, tmax, 1, order_d, scl + tmax, R2, tmax, tpc, tk, f.tcount, st);
    small_gemm(f.B, tmax, 0, R1, tmax, 0, nullptr, nullptr, f.M, tmax, N, tk, f.tcount, st);
    small_gemm(f.B + (size_t)N * tmax, tmax, 0, R2, tmax, 0, nullptr, nullptr, f.M + (size_t)N * tmax, tmax, n2, tk,
               f.tcount, st);
    const int64_t tot = (int64_t)n2 * tk;
    if (z_dtype == LYAP_F32)
      k_copy_z2<float><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(f.M + (size_t)N * tmax, tmax, n2, tk,
                                                                     (float*)Z2, ldz2);
    else
      k_copy_z2<double><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(f.M + (size_t)N * tmax, tmax, n2, tk,
                                                                      (double*)Z2, ldz2);
    h->launches += 5;
  }
  // 7. Z1 = V_m M1 by the second pass
  int rc = second_pass(h, 0, f.M, tmax, tk, Z1, ldz1, z_dtype == LYAP_F32, st);
  if (rc != LYAP_OK) return rc;
  LYAP_CUDA_TRY(cudaStreamSynchronize(st));
  return LYAP_OK;
}

int run_factor(lyap_handle* h, void* Z1, int64_t ldz1, void* Z2, int64_t ldz2, int z_dtype, int tcap, int* t_out,
               cudaStream_t st) {
  if (h->plan.n2 > 0) return run_factor_smallb(h, Z1, ldz1, Z2, ldz2, z_dtype, tcap, t_out, st);
  if (h->plan.sylv) return run_factor_sylv(h, Z1, ldz1, Z2, ldz2, z_dtype, tcap, t_out, st);
  double* M = nullptr;
  int ldm = 0;
  int rc = factor_core(h, tcap, t_out, &M, &ldm, st);
  if (rc != LYAP_OK || *t_out == 0) return rc;
  rc = second_pass(h, 0, M, ldm, *t_out, Z1, ldz1, z_dtype == LYAP_F32, st);
  if (rc != LYAP_OK) return rc;
  LYAP_CUDA_TRY(cudaStreamSynchronize(st));  // keeps the host vectors alive until the copies ran
  return LYAP_OK;
}

// factor from a stored basis (blocks of n x s, consecutive): Z = sum_j V_j M_j, fp64
int run_factor_basis(lyap_handle* h, const double* basis, int64_t n, double* Z, int64_t ldz, int tcap, int* t_out,
                     cudaStream_t st) {
  double* M = nullptr;
  int ldm = 0;
  int rc = factor_core(h, tcap, t_out, &M, &ldm, st);
  if (rc != LYAP_OK) return rc;
  const int tk = *t_out, s = h->s;
  if (tk > 0) {
    const int64_t tot = n * tk;
    k_zero_cols<double><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(Z, n, ldz, tk);
    for (int j = 0; j < h->m; ++j)
      gemm_accum(LYAP_PREC_F64, s, 0, n, s, tk, basis + (size_t)j * n * s, s, M + (size_t)j * s * ldm, ldm, Z, ldz, st);
    h->launches += 1 + h->m;
  }
  LYAP_CUDA_TRY(cudaStreamSynchronize(st));
  return cudaGetLastError() == cudaSuccess ? LYAP_OK : LYAP_ERR_CUDA;
}
