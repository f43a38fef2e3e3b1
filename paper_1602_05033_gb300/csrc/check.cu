// Convergence check of Alg. 1 step 6 by Prop. 3.1 / Alg. 3 (Alg. 4 for Sylvester).
//
// Prop. 3.1 needs every eigenvalue of T_m and the first and last s components of
// every eigenvector.  The paper tridiagonalises T_m (band reduction) and runs a
// tridiagonal eigensolver on the CPU (Alg. 3 steps 1-3).  On this GPU fp64 runs
// at 1/64 of the fp32 rate, and a band reduction is a long chain of dependent
// rotations that cannot use more than one SM; so for a batch of consecutive m
// (one slot each) the kernels
//   1. copy the band of T_m (fp64, and fp32 scaled by its largest entry) and find
//      its Gershgorin interval;
//   2. bisect every eigenvalue on the fp32 band itself (Sturm counts from an
//      unpivoted LDL^T of T_m - x I, O(N s^2) each), giving estimates accurate to
//      a few eps32 ||T||;
//   3. refine every eigenpair in fp64 on the block-tridiagonal T_m itself:
//      estimates closer than the fp32 tolerance are first bisected again in fp64;
//      then inverse iteration from the estimate (fp32 solves, then one fp64 step
//      at the settled Rayleigh quotient, more only if the residual test asks),
//      with the banded LU (partial pivoting) of T_m - sigma I; estimates still
//      closer than the fp64 tolerance form a cluster, iterated as a subspace and
//      split by Rayleigh-Ritz so that its vectors stay orthonormal.  The full
//      eigenvector is available, so its first and last s rows give
//      a_i = (Q^T E_1 gamma)_i and w_i = (Q^T E_m tau^T)_i (Alg. 3 steps 3-5);
//   4. accumulate ||e_i^T S D_i^{-1} W||^2 per i (Alg. 3 steps 7-10);
//   5. sum, take sqrt(2 sum)/beta^2 and record the history and the first converged m.
// Every fp64 step runs one thread per eigenpair across the whole GPU.  Reductions
// are in a fixed order.
#include "common.cuh"
#include "ff.cuh"

#include <float.h>
#include <limits.h>
#include <math.h>
#ifdef LYAP_DEBUG
#include <stdio.h>
#endif

namespace {

constexpr int kMaxCluster = 16;
constexpr int kMaxChecks = 256;  // checks per batch (the check_batch option is capped there)
constexpr int kClusterBlocks = 16;  // blocks per check of k_invit_clusters
constexpr int kClusterWarps = 64;   // warps per check of k_invit_clusters (4 per block)
// Members of a group of fp32 estimates larger than this get fp64 estimates by multisection with
// Sturm counts on the fp64 band, and are then regrouped at the fp64 tolerance below (1: every
// group).  Estimates that stay farther apart than that tolerance are iterated one by one with
// their fp64 estimate as a fixed shift; closer ones as a subspace (k_invit_clusters), which keeps
// the vectors of close eigenvalues orthonormal: a single vector's error is its residual over the
// gap to its neighbour.  On the 2D Laplacian tests the subspace path for pairs closer than
// 1e-6 ||T|| keeps every history within a fifth of the 1e-10 bound; at 1e-9 ||T|| the errors of
// close singletons reached 2.6 times it.
#ifndef LYAP_REFINE_AT
#define LYAP_REFINE_AT 1
#endif
constexpr int kRefineAt = LYAP_REFINE_AT;
#ifndef LYAP_TOL64_FLOOR
#define LYAP_TOL64_FLOOR 1e-6
#endif
constexpr double kTol64Floor = LYAP_TOL64_FLOOR;
constexpr int kIters32 = 3;   // fp32 inverse iterations at the estimate before the fp64 ones
constexpr int kRounds32 = 2;  // fp32 rounds of a cluster before its fp64 rounds
constexpr int kMaxIters = 12; // fp64 inverse iterations (Rayleigh-quotient shifts) until converged
constexpr int kMaxRounds = 10;  // cluster rounds (Rayleigh-Ritz between them); converged clusters stop early
constexpr double kSettle = 1e-12;  // |change of the Rayleigh quotient| / ||T|| after which one more step is run
constexpr double kResTol = 1e-11;  // accepted ||T x - lambda x|| relative to ||T||
#ifndef LYAP_REFINE_RES
#define LYAP_REFINE_RES 1e-10
#endif
#ifndef LYAP_PAIR_INVIT
#define LYAP_PAIR_INVIT 1
#endif
constexpr double kRefineRes = LYAP_REFINE_RES;  // width at which multisection stops, relative to ||T||
constexpr bool kPairInvit = LYAP_PAIR_INVIT;    // singleton iteration in float pairs (else fp64)
// threads per block of k_invit (each thread iterates one eigenpair alone; smaller blocks, spread
// over more SM sub-partitions, measured slower on the n = 1e6 workload)
#ifndef LYAP_INVIT_THREADS
#define LYAP_INVIT_THREADS 32
#endif
constexpr int kInvitThreads = LYAP_INVIT_THREADS;

struct Slot {
  double* hdr;   // [0] Gershgorin lo, [1] hi (scaled), [2] max e^2 (scaled), [3] scale, [4] fp32 cluster
                 // tolerance, [6] fp64 cluster tolerance
  float* Tb32;   // (s+1) x N   fp32 copy of the band of T_m / scale, Tb32[d*N + c] = T_m[c+d][c] / scale
  double* est;   // nmax   fp32 eigenvalue estimates (unscaled)
  double* lam;   // nmax   fp64 eigenvalues
  double* part;  // nmax
  double* Tb;    // (s+1) x N   fp64 band of T_m, Tb[d*N + c] = T_m[c+d][c]
  double* a;     // nmax x s
  double* w;     // nmax x s
  int* clist;    // [0] number of clusters, then (first index, size) pairs
  double* X;     // nmax x nmax, [k][i]: component k of eigenvector i
  double* U;     // nmax x (2s+1) x nmax, [k][e][i]: row k of the LU factor of thread i
  double* etol;  // nmax   cluster tolerance of each estimate (fp32 one, or fp64 one once refined)
  double* Xc;    // nmax x nmax, [i][k]: eigenvector i of a cluster member, contiguous
  float2* Tbf;   // (s+1) x N   the fp64 band as float pairs (hi, lo), same indexing as Tb
};

__host__ __device__ constexpr size_t slot_doubles(int s, int nmax) {
  return 8 + ((size_t)(s + 1) * nmax + 1) / 2 /* Tb32 */ + 3 * (size_t)nmax + (size_t)(s + 1) * nmax + 2 * (size_t)s * nmax +
         ((size_t)nmax + 16) /* cluster list */ + (size_t)nmax * nmax + (size_t)(2 * s + 1) * nmax * nmax +
         (size_t)nmax /* etol */ + (size_t)nmax * nmax /* Xc */ + (size_t)(s + 1) * nmax /* Tbf */;
}

__device__ inline Slot get_slot(double* base, int s, int nmax, int idx) {
  Slot sl;
  double* p = base + (size_t)idx * slot_doubles(s, nmax);
  sl.hdr = p; p += 8;
  sl.Tb32 = reinterpret_cast<float*>(p);
  p += ((size_t)(s + 1) * nmax + 1) / 2;
  sl.est = p; p += nmax;
  sl.lam = p; p += nmax;
  sl.part = p; p += nmax;
  sl.Tb = p; p += (size_t)(s + 1) * nmax;
  sl.a = p; p += (size_t)s * nmax;
  sl.w = p; p += (size_t)s * nmax;
  sl.clist = reinterpret_cast<int*>(p); p += (size_t)nmax + 16;
  sl.X = p; p += (size_t)nmax * nmax;
  sl.U = p; p += (size_t)(2 * s + 1) * nmax * nmax;
  sl.etol = p; p += nmax;
  sl.Xc = p; p += (size_t)nmax * nmax;
  sl.Tbf = reinterpret_cast<float2*>(p);
  return sl;
}

struct CheckArgs {
  const double* log;  // coefficient log of this operator
  double* slots;      // slot array for this operator
  int s;
  int nmax;
  int nchk;
  int* flags;
  int* chk_err;       // per-m error bits of the check (index m - 1)
  int ms[kMaxChecks]; // slot c holds the check at m = ms[c]
};

// T_m[i][c] for i >= c, i - c <= s: symmetric part of tau_jj on the diagonal blocks,
// tau_{j+1,j} below them (Sec. 2)
__device__ inline double tval(const double* __restrict__ log, int s, int i, int c) {
  const int SS = s * s;
  const int J = i / s, Jc = c / s;
  if (J == Jc) {
    const double* D = log + (size_t)(J + 1) * LOG_NREC * SS + REC_TDIAG * SS;
    return 0.5 * (D[(i % s) * s + (c % s)] + D[(c % s) * s + (i % s)]);
  }
  if (J == Jc + 1) return log[(size_t)(Jc + 1) * LOG_NREC * SS + REC_TNEXT * SS + (i % s) * s + (c % s)];
  return 0.0;
}
__device__ inline double tsym(const double* __restrict__ log, int s, int i, int c) {
  if (i < c) { const int t = i; i = c; c = t; }
  return (i - c <= s) ? tval(log, s, i, c) : 0.0;
}

// T_m[r][c] from the slot's fp64 band (zero outside the band)
__device__ __forceinline__ double tband(const double* __restrict__ Tb, int N, int S, int r, int c) {
  const int d = r > c ? r - c : c - r;
  return d <= S ? __ldg(Tb + (size_t)d * N + (r < c ? r : c)) : 0.0;
}

// 1. per check: the fp64 band of T_m and an fp32 copy scaled by its largest entry, the Gershgorin
// interval of T_m / scale and the fp32 grouping tolerance
__global__ void __launch_bounds__(256) k_setup_band(CheckArgs g) {
  __shared__ double red[3][8];
  const int c_idx = blockIdx.x;
  const int m = g.ms[c_idx];
  const int s = g.s, N = s * m;
  Slot sl = get_slot(g.slots, s, g.nmax, c_idx);
  double mx = 0.0, lo = INFINITY, hi = -INFINITY;
  for (int t = threadIdx.x; t < (s + 1) * N; t += blockDim.x) {
    const int d = t / N, c = t % N;
    const double v = c + d < N ? tval(g.log, s, c + d, c) : 0.0;
    sl.Tb[t] = v;
    const ff vf = ff_from_double(v);
    sl.Tbf[t] = make_float2(vf.hi, vf.lo);
    mx = fmax(mx, fabs(v));
  }
  __syncthreads();
  for (int i = threadIdx.x; i < N; i += blockDim.x) {  // Gershgorin discs by rows
    double r = 0.0;
    for (int d = 1; d <= s; ++d) {
      if (i + d < N) r += fabs(sl.Tb[(size_t)d * N + i]);
      if (i - d >= 0) r += fabs(sl.Tb[(size_t)d * N + i - d]);
    }
    lo = fmin(lo, sl.Tb[i] - r);
    hi = fmax(hi, sl.Tb[i] + r);
  }
  for (int o = 16; o > 0; o >>= 1) {
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    red[0][w] = mx;
    red[1][w] = lo;
    red[2][w] = hi;
  }
  __syncthreads();
  __shared__ double sc;
  if (threadIdx.x == 0) {
    double a = 0.0, l = INFINITY, h = -INFINITY;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      a = fmax(a, red[0][k]);
      l = fmin(l, red[1][k]);
      h = fmax(h, red[2][k]);
    }
    if (!(a > 0.0)) a = 1.0;
    const double span = fmax(fabs(l), fabs(h)) / a;
    sl.hdr[0] = l / a - 8.0 * FLT_EPSILON * span;
    sl.hdr[1] = h / a + 8.0 * FLT_EPSILON * span;
    sl.hdr[2] = 0.0;
    sl.hdr[3] = a;
    // estimates closer than this form a group refined in fp64.  Sturm counts of the fp32 band
    // leave errors up to about 20 eps32 ||T|| on the Laplacian workloads at N < 130; the
    // tolerance keeps at least a factor two over that (the acceptance test of a singleton allows
    // half of it)
    sl.hdr[4] = 8.0 * sqrt((double)N) * FLT_EPSILON * a * span;
    sl.clist[0] = 0;
    sc = 1.0 / a;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < (s + 1) * N; t += blockDim.x) sl.Tb32[t] = (float)(sl.Tb[t] * sc);
  for (int t = threadIdx.x; t < N; t += blockDim.x) {
    sl.part[t] = 0.0;  // retry marks of k_invit
    sl.lam[t] = __longlong_as_double(0x7ff8000000000000LL);  // every eigenvalue must be written
  }
}

// Number of eigenvalues of the fp32 band below x: inertia of the unpivoted LDL^T of T - x I, a
// tiny pivot replaced by -pivmin (the fp32 counterpart of band_sturm below)
template <int S>
__device__ int band_sturm32(const float* __restrict__ Tb, int N, float x, float pivmin) {
  float dinv[S], L[S][S];
#pragma unroll
  for (int r = 0; r < S; ++r) {
    dinv[r] = 0.f;
#pragma unroll
    for (int t = 0; t < S; ++t) L[r][t] = 0.f;
  }
  int cnt = 0;
  for (int k = 0; k < N; ++k) {
    float w[S], nl[S];
#pragma unroll
    for (int r = S - 1; r >= 0; --r) {
      const int j = k - 1 - r;
      float v = j >= 0 ? Tb[(size_t)(r + 1) * N + j] : 0.f;
#pragma unroll
      for (int q = S - 1; q > r; --q) v = fmaf(-w[q], L[r][q - r - 1], v);
      w[r] = v;
      nl[r] = v * dinv[r];
    }
    float dk = Tb[k] - x;
#pragma unroll
    for (int r = 0; r < S; ++r) dk = fmaf(-nl[r], w[r], dk);
    if (fabsf(dk) <= pivmin) dk = -pivmin;
    cnt += dk < 0.f;
#pragma unroll
    for (int r = S - 1; r > 0; --r) {
      dinv[r] = dinv[r - 1];
#pragma unroll
      for (int t = 0; t < S; ++t) L[r][t] = L[r - 1][t];
    }
    dinv[0] = 1.f / dk;
#pragma unroll
    for (int t = 0; t < S; ++t) L[0][t] = nl[t];
  }
  return cnt;
}

// 2. fp32 multisection of every eigenvalue on the band itself, one warp per eigenvalue index:
// the 32 lanes count the eigenvalues below 32 interior points of the bracket at once, so a round
// narrows it 33-fold (about 5 rounds from the Gershgorin interval to fp32 resolution, where
// bisection takes 24 dependent Sturm counts)
template <int S>
__global__ void k_bisect_band32(CheckArgs g) {
  const int c_idx = blockIdx.y;
  const int m = g.ms[c_idx];
  const int N = S * m;
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);  // one index per warp
  if (i >= N) return;
  Slot sl = get_slot(g.slots, S, g.nmax, c_idx);
  float lo = (float)sl.hdr[0], hi = (float)sl.hdr[1];
  const float pivmin = 16.f * FLT_MIN;
  const unsigned full = 0xffffffffu;
  for (int round = 0; round < 16; ++round) {
    if (!(hi - lo > 2.f * FLT_EPSILON * fmaxf(fabsf(lo), fabsf(hi)))) break;
    const float x = lo + (hi - lo) * ((float)(lane + 1) / 33.f);
    const int c = band_sturm32<S>(sl.Tb32, N, x, pivmin);
    const unsigned below = __ballot_sync(full, c <= i);
    const int top = below ? 31 - __clz(below) : -1;  // last point at or below lambda_i
    const float nlo = __shfl_sync(full, x, top < 0 ? 0 : top);
    const float nhi = __shfl_sync(full, x, top < 31 ? top + 1 : 31);
    const float lo2 = top < 0 ? lo : nlo, hi2 = top < 31 ? nhi : hi;
    if (!(hi2 - lo2 < hi - lo)) break;  // no progress at this resolution
    lo = lo2;
    hi = hi2;
  }
  if (lane == 0) sl.est[i] = 0.5 * ((double)lo + (double)hi) * sl.hdr[3];
}

// 2b. per-estimate cluster tolerance: members of fp32 groups larger than kRefineAt get the
// fp64 grouping tolerance (and are refined by 2c), all others the fp32 one
__global__ void k_mark_refine(CheckArgs g) {
  const int c_idx = blockIdx.x;
  const int m = g.ms[c_idx];
  const int N = g.s * m;
  Slot sl = get_slot(g.slots, g.s, g.nmax, c_idx);
  const double tol32 = sl.hdr[4];
  const double span = fmax(fabs(sl.hdr[0]), fabs(sl.hdr[1]));
  // refined estimates are accurate to a few eps64 ||T||, so a refined singleton converges to its
  // own eigenvalue whenever its neighbours are farther than the fp64 tolerance; closer ones
  // (near-duplicate Ritz values of the finite-precision recurrence reach 1e-10 ||T||) are grouped
  // and resolved together
  const double tnorm = sl.hdr[3] * span;
  const double tol64 = fmax(8.0 * sqrt((double)N) * DBL_EPSILON * tnorm, kTol64Floor * tnorm);
  if (threadIdx.x == 0) sl.hdr[6] = tol64;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    if (i > 0 && sl.est[i] - sl.est[i - 1] <= tol32) continue;
    int c = 1;
    while (i + c < N && sl.est[i + c] - sl.est[i + c - 1] <= tol32) ++c;
    const double t = c > kRefineAt ? tol64 : tol32;
    for (int v = 0; v < c; ++v) sl.etol[i + v] = t;
  }
}

// Number of eigenvalues of T_m below x: inertia of the unpivoted LDL^T factorisation of
// T_m - x I on the fp64 band (Sylvester's law of inertia), a tiny pivot replaced by -pivmin.
// The last S rows of L and D stay in registers: w_r = (L D)[k][k-r], L[k][k-r] = w_r / d_{k-r},
// d_k = T_kk - x - sum_r L[k][k-r] w_r.
template <int S>
__device__ int band_sturm(const double* __restrict__ Tb, int N, double x, double pivmin) {
  double dinv[S], L[S][S];  // row r (= k-1-r) : 1/d and its sub-diagonal entries L[row][row-1-t]
#pragma unroll
  for (int r = 0; r < S; ++r) {
    dinv[r] = 0.0;
#pragma unroll
    for (int t = 0; t < S; ++t) L[r][t] = 0.0;
  }
  int cnt = 0;
  for (int k = 0; k < N; ++k) {
    double w[S], nl[S];
    // columns k-S .. k-1 (r = S-1 .. 0 means column k-1-r)
#pragma unroll
    for (int r = S - 1; r >= 0; --r) {
      const int j = k - 1 - r;
      double v = j >= 0 ? __ldg(Tb + (size_t)(r + 1) * N + j) : 0.0;
#pragma unroll
      for (int q = S - 1; q > r; --q) v = fma(-w[q], L[r][q - r - 1], v);  // L[j][k-1-q]
      w[r] = v;
      nl[r] = v * dinv[r];
    }
    double dk = __ldg(Tb + k) - x;
#pragma unroll
    for (int r = 0; r < S; ++r) dk = fma(-nl[r], w[r], dk);
    if (fabs(dk) <= pivmin) dk = -pivmin;
    cnt += dk < 0.0;
    // shift the window: the new row becomes row 0
#pragma unroll
    for (int r = S - 1; r > 0; --r) {
      dinv[r] = dinv[r - 1];
#pragma unroll
      for (int t = 0; t < S; ++t) L[r][t] = L[r - 1][t];
    }
    dinv[0] = 1.0 / dk;
#pragma unroll
    for (int t = 0; t < S; ++t) L[0][t] = nl[t];
  }
  return cnt;
}

// band_sturm in float pairs on the pair band: the same recurrence with every operation on the
// fp32 pipe (about 48 significant bits; the counts resolve eigenvalues to ~1e-13 ||T||)
template <int S>
__device__ int band_sturm_ff(const float2* __restrict__ Tb, int N, ff x, float pivmin) {
  ff dinv[S], L[S][S];
#pragma unroll
  for (int r = 0; r < S; ++r) {
    dinv[r] = ff_make(0.f, 0.f);
#pragma unroll
    for (int t = 0; t < S; ++t) L[r][t] = ff_make(0.f, 0.f);
  }
  const ff nx = ff_make(-x.hi, -x.lo);
  const ff one = ff_make(1.f, 0.f);
  int cnt = 0;
  for (int k = 0; k < N; ++k) {
    ff w[S], nl[S];
#pragma unroll
    for (int r = S - 1; r >= 0; --r) {
      const int j = k - 1 - r;
      const float2 t = j >= 0 ? __ldg(Tb + (size_t)(r + 1) * N + j) : make_float2(0.f, 0.f);
      ff v = ff_make(t.x, t.y);
#pragma unroll
      for (int q = S - 1; q > r; --q) ff_sub_acc(v, w[q], L[r][q - r - 1]);
      w[r] = ff_norm(v);
      nl[r] = ff_mul(w[r], dinv[r]);
    }
    const float2 t = __ldg(Tb + k);
    ff dk = ff_add(ff_make(t.x, t.y), nx);
#pragma unroll
    for (int r = 0; r < S; ++r) ff_sub_acc(dk, nl[r], w[r]);
    dk = ff_norm(dk);
    if (fabsf(dk.hi) <= pivmin) dk = ff_make(-pivmin, 0.f);
    cnt += dk.hi < 0.f;
#pragma unroll
    for (int r = S - 1; r > 0; --r) {
      dinv[r] = dinv[r - 1];
#pragma unroll
      for (int t2 = 0; t2 < S; ++t2) L[r][t2] = L[r - 1][t2];
    }
    dinv[0] = ff_div(one, dk);
#pragma unroll
    for (int t2 = 0; t2 < S; ++t2) L[0][t2] = nl[t2];
  }
  return cnt;
}

// 2c. multisection of the marked estimates, one warp per eigenvalue index: the 32 lanes count the
// eigenvalues below 32 interior points of the bracket at once (float-pair Sturm counts on the
// pair band), so a round narrows it 33-fold; started from the fp32 estimate +- the fp32 grouping
// tolerance (widened to the Gershgorin interval if the counts show the eigenvalue outside it),
// stopped at kRefineRes ||T||: four rounds.  The estimate only has to separate eigenvalues at the
// fp64 grouping tolerance (>= 1e-6 ||T||) and to serve as a shift; the eigenvalue itself is the
// Rayleigh quotient of the converged vector.
template <int S>
__global__ void k_refine64(CheckArgs g, int round) {
  const int c_idx = blockIdx.y;
  const int m = g.ms[c_idx];
  const int N = S * m;
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);  // one index per warp
  if (i >= N) return;
  Slot sl = get_slot(g.slots, S, g.nmax, c_idx);
  const double tol32 = sl.hdr[4];
  // round 0: members of fp32 groups; round 1: the singletons marked for a retry by k_invit
  if (round == 0 ? !(sl.etol[i] < tol32) : sl.part[i] == 0.0) return;
  const double sc = sl.hdr[3];
  const double glo = sl.hdr[0] * sc, ghi = sl.hdr[1] * sc;
  const double span = fmax(fabs(glo), fabs(ghi));
  const float pivmin = 1e-30f * (float)fmax(1.0, span * span);
  const unsigned full = 0xffffffffu;
  double lo = sl.est[i] - tol32, hi = sl.est[i] + tol32;
  {
    const int c = lane < 2 ? band_sturm_ff<S>(sl.Tbf, N, ff_from_double(lane == 0 ? lo : hi), pivmin) : 0;
    const int clo = __shfl_sync(full, c, 0), chi = __shfl_sync(full, c, 1);
    if (clo > i) lo = glo;
    if (chi <= i) hi = ghi;
  }
  for (int round = 0; round < 40; ++round) {
    if (!(hi - lo > kRefineRes * span)) break;
    const double x = lo + (hi - lo) * ((double)(lane + 1) / 33.0);
    const int c = band_sturm_ff<S>(sl.Tbf, N, ff_from_double(x), pivmin);
    // lambda_i >= x exactly when fewer than i + 1 eigenvalues lie below x
    const unsigned below = __ballot_sync(full, c <= i);
    const int top = below ? 31 - __clz(below) : -1;  // last point at or below lambda_i
    const double nlo = __shfl_sync(full, x, top < 0 ? 0 : top);
    const double nhi = __shfl_sync(full, x, top < 31 ? top + 1 : 31);
    const double lo2 = top < 0 ? lo : nlo, hi2 = top < 31 ? nhi : hi;
    if (!(hi2 - lo2 < hi - lo)) break;  // no progress at this resolution
    lo = lo2;
    hi = hi2;
  }
  if (lane == 0) sl.est[i] = 0.5 * (lo + hi);
}

__device__ inline double hash_unit(unsigned int k, unsigned int i) {
  // splitmix64 (Steele, Lea and Flood's mixing function) of the key (i, k): start vectors with
  // no structure along the rows, so no eigenvector of T_m is nearly missing from them
  unsigned long long z = ((unsigned long long)i << 32 | k) + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * 0x1.0p-52 - 1.0;  // in [-1, 1)
}

// the per-eigenvalue scratch (U rows, vector entries) is far larger than L2, so every
// row step of the sequential sweeps would wait one DRAM round trip; prefetch kPf rows ahead
constexpr int kPf = 8;
__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// (T_m - sigma I)[r][c] from the fp64 band, zero outside the matrix
template <int S>
__device__ __forceinline__ double mval(const double* __restrict__ Tb, int N, double sigma, int r, int c) {
  if (r >= N || c >= N || c < 0) return 0.0;
  const double v = tband(Tb, N, S, r, c);
  return r == c ? v - sigma : v;
}

// X[:, col] <- (T_m - sigma I)^{-1} (xscale X[:, col]) by a banded LU with partial pivoting; returns
// max_k |X[k, col]| of the result
// (bandwidth S; U gets 2S+1 diagonals).  The active (S+1) x (2S+1) window, the pivot swaps
// (predicated selects) and the back-substitution window live in registers: every index is a
// compile-time constant.  U rows go to per-thread scratch ([k][e][tid] layout, coalesced).
// R is the arithmetic type: fp32 for the cheap first iterations (the entries of T_m - sigma I are
// formed in fp64 and then rounded, so the shift stays exact), fp64 to finish.  U points at the
// double scratch reinterpreted as R.
template <int S, typename R = double>
__device__ double solve1(const double* __restrict__ Tb, int N, double sigma, R tiny, double xscale,
                         double* __restrict__ X, size_t ld, int col, R* __restrict__ U, int tid, size_t ldu) {
  constexpr int W = 2 * S + 1;
  // a thread's U entries are doubles at ((k W + e) ldu + tid); an fp32 solve stores its value in
  // the first half of the same double, so no thread ever touches another's scratch
  constexpr size_t us = sizeof(double) / sizeof(R);
  R win[S + 1][W];
  R yw[S + 1];
#pragma unroll
  for (int r = 0; r <= S; ++r) {
#pragma unroll
    for (int c = 0; c < W; ++c) win[r][c] = (R)mval<S>(Tb, N, sigma, r, c);
    yw[r] = r < N ? (R)(X[(size_t)r * ld + col] * xscale) : R(0);
  }
  for (int k = 0; k < N; ++k) {
    if (k + S + 1 + kPf < N) prefetch_l2(X + (size_t)(k + S + 1 + kPf) * ld + col);
    const int nr = min(S, N - 1 - k);
    R best = fabs(win[0][0]);
    int p = 0;
#pragma unroll
    for (int r = 1; r <= S; ++r) {
      const R a = fabs(win[r][0]);
      if (r <= nr && a > best) { best = a; p = r; }
    }
#pragma unroll
    for (int r = 1; r <= S; ++r) {
      const bool sw = p == r;
#pragma unroll
      for (int c = 0; c < W; ++c) {
        const R a = win[0][c], b = win[r][c];
        win[0][c] = sw ? b : a;
        win[r][c] = sw ? a : b;
      }
      const R a = yw[0], b = yw[r];
      yw[0] = sw ? b : a;
      yw[r] = sw ? a : b;
    }
    if (fabs(win[0][0]) < tiny) win[0][0] = win[0][0] < 0.0 ? -tiny : tiny;
    const R pinv = R(1) / win[0][0];
#pragma unroll
    for (int r = 1; r <= S; ++r) {
      const R l = r <= nr ? win[r][0] * pinv : R(0);
#pragma unroll
      for (int c = 1; c < W; ++c) win[r][c] = fma(-l, win[0][c], win[r][c]);
      yw[r] = fma(-l, yw[0], yw[r]);
    }
#pragma unroll
    for (int c = 0; c < W; ++c) U[(((size_t)k * W + c) * ldu + tid) * us] = win[0][c];
    X[(size_t)k * ld + col] = (double)yw[0];
#pragma unroll
    for (int r = 0; r < S; ++r) {
#pragma unroll
      for (int c = 0; c < W - 1; ++c) win[r][c] = win[r + 1][c + 1];
      win[r][W - 1] = R(0);
      yw[r] = yw[r + 1];
    }
    const int rn = k + S + 1;
#pragma unroll
    for (int c = 0; c < W; ++c) win[S][c] = (R)mval<S>(Tb, N, sigma, rn, k + 1 + c);
    yw[S] = rn < N ? (R)(X[(size_t)rn * ld + col] * xscale) : R(0);
  }
  double amax = 0.0;
  R xs[W - 1];  // xs[e - 1] = x_{k+e}; entries beyond N stay 0 (so do their U coefficients)
#pragma unroll
  for (int e = 0; e < W - 1; ++e) xs[e] = R(0);
  for (int k = N - 1; k >= 0; --k) {
    if (k >= kPf) {
      const int kp = k - kPf;
      prefetch_l2(X + (size_t)kp * ld + col);
#pragma unroll
      for (int e = 0; e < W; ++e) prefetch_l2(U + (((size_t)kp * W + e) * ldu + tid) * us);
    }
    R t = (R)X[(size_t)k * ld + col];
#pragma unroll
    for (int e = 1; e < W; ++e) t = fma(-U[(((size_t)k * W + e) * ldu + tid) * us], xs[e - 1], t);
    const R xk = t / U[(((size_t)k * W) * ldu + tid) * us];
    X[(size_t)k * ld + col] = (double)xk;
    amax = fmax(amax, fabs((double)xk));
#pragma unroll
    for (int e = W - 2; e > 0; --e) xs[e] = xs[e - 1];
    xs[0] = xk;
  }
  return amax;
}

// x^T T x and x^T x for column col in one pass (register window of 2S+1 entries of x)
template <int S>
__device__ void rq_pass(const double* __restrict__ Tb, int N, const double* __restrict__ X, size_t ld, int col,
                        double* num, double* den) {
  double xw[2 * S + 1];  // x_{k-S} .. x_{k+S}
#pragma unroll
  for (int j = 0; j <= 2 * S; ++j) {
    const int r = j - S;
    xw[j] = (r >= 0 && r < N) ? X[(size_t)r * ld + col] : 0.0;
  }
  double nu = 0.0, de = 0.0;
  for (int k = 0; k < N; ++k) {
    if (k + S + 1 + kPf < N) prefetch_l2(X + (size_t)(k + S + 1 + kPf) * ld + col);
    double tx = 0.0;
#pragma unroll
    for (int j = 0; j <= 2 * S; ++j) {
      const int c = k - S + j;
      if (c >= 0 && c < N) tx = fma(tband(Tb, N, S, k, c), xw[j], tx);
    }
    nu = fma(xw[S], tx, nu);
    de = fma(xw[S], xw[S], de);
#pragma unroll
    for (int j = 0; j < 2 * S; ++j) xw[j] = xw[j + 1];
    const int r = k + S + 1;
    xw[2 * S] = r < N ? X[(size_t)r * ld + col] : 0.0;
  }
  *num = nu;
  *den = de;
}

// x^T T x for column i of X (one band matrix-vector pass)
__device__ double rquot(const double* __restrict__ Tb, int s, int N, const double* __restrict__ X, size_t ld, int i) {
  double num = 0.0;
  for (int k = 0; k < N; ++k) {
    double tx = 0.0;
    for (int c = max(0, k - s); c <= min(N - 1, k + s); ++c) tx = fma(tband(Tb, N, s, k, c), X[(size_t)c * ld + i], tx);
    num = fma(X[(size_t)k * ld + i], tx, num);
  }
  return num;
}

// Rayleigh quotient and ||T x - rq x|| (two passes)
__device__ void rayleigh(const double* __restrict__ Tb, int s, int N, const double* __restrict__ X, size_t ld, int i,
                         double* rq, double* res) {
  const double num = rquot(Tb, s, N, X, ld, i);
  *rq = num;
  double r2 = 0.0;
  for (int k = 0; k < N; ++k) {
    double tx = 0.0;
    for (int c = max(0, k - s); c <= min(N - 1, k + s); ++c) tx = fma(tband(Tb, N, s, k, c), X[(size_t)c * ld + i], tx);
    const double d = tx - num * X[(size_t)k * ld + i];
    r2 = fma(d, d, r2);
  }
  *res = sqrt(r2);
}

__device__ double normalize_col(double* X, size_t ld, int N, int i) {
  double n2 = 0.0;
  for (int k = 0; k < N; ++k) n2 = fma(X[(size_t)k * ld + i], X[(size_t)k * ld + i], n2);
  const double inv = n2 > 0.0 ? 1.0 / sqrt(n2) : 0.0;
  for (int k = 0; k < N; ++k) X[(size_t)k * ld + i] *= inv;
  return n2;
}



// ---- singleton inverse iteration in float pairs ------------------------------------------------
// The vector lives in the eigenvector array as pairs (hi, lo in the 8 bytes of an entry) until it
// has converged; then its first and last S rows are rewritten as doubles for write_aw.  fp64 runs
// at 1/64 of the fp32 rate on this GPU, so the pair arithmetic (about 48 significant bits, a few
// fp32 operations per pair operation) finishes the same iteration several times sooner.
template <typename R>
__device__ __forceinline__ R from_ff(ff v);
template <>
__device__ __forceinline__ float from_ff<float>(ff v) { return v.hi; }
template <>
__device__ __forceinline__ fd from_ff<fd>(ff v) { return fd(v); }
__device__ __forceinline__ float2 to_f2(float x) { return make_float2(x, 0.f); }
__device__ __forceinline__ float2 to_f2(fd x) { return make_float2(x.v.hi, x.v.lo); }
__device__ __forceinline__ float lead(float x) { return x; }
__device__ __forceinline__ float lead(fd x) { return x.v.hi; }

// (T_m - sigma I)[r][c] from the pair band (nsig = -sigma), zero outside the matrix
template <int S>
__device__ __forceinline__ ff mval_ff(const float2* __restrict__ Tb, int N, ff nsig, int r, int c) {
  if (r >= N || c >= N || c < 0) return ff_make(0.f, 0.f);
  const int d = r > c ? r - c : c - r;
  if (d > S) return ff_make(0.f, 0.f);
  const float2 t = __ldg(Tb + (size_t)d * N + (r < c ? r : c));
  const ff v = ff_make(t.x, t.y);
  return r == c ? ff_add(v, nsig) : v;
}

// X[:, col] <- (T_m - sigma I)^{-1} (xscale X[:, col]) with X holding pairs: the banded LU with
// partial pivoting of solve1, in fp32 (R = float: leading parts only) or in pairs (R = fd).
// Returns max_k |x_k| (leading parts); not finite if the solve overflowed.
template <int S, typename R>
__device__ float solve_pair(const float2* __restrict__ Tb, int N, ff sigma, R tiny, ff xscale, float2* __restrict__ X,
                            size_t ld, int col, R* __restrict__ U, int tid, size_t ldu) {
  constexpr int W = 2 * S + 1;
  constexpr size_t us = sizeof(double) / sizeof(R);
  const ff nsig = ff_make(-sigma.hi, -sigma.lo);
  const R xsc = from_ff<R>(xscale);
  auto ldx = [&](int r) -> R {
    const float2 v = X[(size_t)r * ld + col];
    return from_ff<R>(ff_make(v.x, v.y)) * xsc;
  };
  R win[S + 1][W];
  R yw[S + 1];
#pragma unroll
  for (int r = 0; r <= S; ++r) {
#pragma unroll
    for (int c = 0; c < W; ++c) win[r][c] = from_ff<R>(mval_ff<S>(Tb, N, nsig, r, c));
    yw[r] = r < N ? ldx(r) : R(0);
  }
  for (int k = 0; k < N; ++k) {
    if (k + S + 1 + kPf < N) prefetch_l2(X + (size_t)(k + S + 1 + kPf) * ld + col);
    const int nr = min(S, N - 1 - k);
    R best = fabs(win[0][0]);
    int p = 0;
#pragma unroll
    for (int r = 1; r <= S; ++r) {
      const R a = fabs(win[r][0]);
      if (r <= nr && a > best) { best = a; p = r; }
    }
#pragma unroll
    for (int r = 1; r <= S; ++r) {
      const bool sw = p == r;
#pragma unroll
      for (int c = 0; c < W; ++c) {
        const R a = win[0][c], b = win[r][c];
        win[0][c] = sw ? b : a;
        win[r][c] = sw ? a : b;
      }
      const R a = yw[0], b = yw[r];
      yw[0] = sw ? b : a;
      yw[r] = sw ? a : b;
    }
    if (fabs(win[0][0]) < tiny) win[0][0] = lead(win[0][0]) < 0.f ? -tiny : tiny;
    const R pinv = R(1) / win[0][0];
#pragma unroll
    for (int r = 1; r <= S; ++r) {
      const R l = r <= nr ? win[r][0] * pinv : R(0);
#pragma unroll
      for (int c = 1; c < W; ++c) win[r][c] = fma(-l, win[0][c], win[r][c]);
      yw[r] = fma(-l, yw[0], yw[r]);
    }
#pragma unroll
    for (int c = 0; c < W; ++c) U[(((size_t)k * W + c) * ldu + tid) * us] = win[0][c];
    X[(size_t)k * ld + col] = to_f2(yw[0]);
#pragma unroll
    for (int r = 0; r < S; ++r) {
#pragma unroll
      for (int c = 0; c < W - 1; ++c) win[r][c] = win[r + 1][c + 1];
      win[r][W - 1] = R(0);
      yw[r] = yw[r + 1];
    }
    const int rn = k + S + 1;
#pragma unroll
    for (int c = 0; c < W; ++c) win[S][c] = from_ff<R>(mval_ff<S>(Tb, N, nsig, rn, k + 1 + c));
    yw[S] = rn < N ? ldx(rn) : R(0);
  }
  float amax = 0.f;
  R xs[W - 1];
#pragma unroll
  for (int e = 0; e < W - 1; ++e) xs[e] = R(0);
  for (int k = N - 1; k >= 0; --k) {
    if (k >= kPf) {
      const int kp = k - kPf;
      prefetch_l2(X + (size_t)kp * ld + col);
#pragma unroll
      for (int e = 0; e < W; ++e) prefetch_l2(U + (((size_t)kp * W + e) * ldu + tid) * us);
    }
    const float2 xv = X[(size_t)k * ld + col];
    R t = from_ff<R>(ff_make(xv.x, xv.y));
#pragma unroll
    for (int e = 1; e < W; ++e) t = fma(-U[(((size_t)k * W + e) * ldu + tid) * us], xs[e - 1], t);
    const R xk = t / U[(((size_t)k * W) * ldu + tid) * us];
    X[(size_t)k * ld + col] = to_f2(xk);
    amax = fmaxf(amax, fabsf(lead(xk)));
    if (!isfinite(lead(xk))) amax = INFINITY;
#pragma unroll
    for (int e = W - 2; e > 0; --e) xs[e] = xs[e - 1];
    xs[0] = xk;
  }
  return amax;
}

// x^T T x and x^T x (pairs) for column col of the pair vectors, one pass with a window of 2S+1
template <int S>
__device__ void rq_pair(const float2* __restrict__ Tb, int N, const float2* __restrict__ X, size_t ld, int col, ff* num,
                        ff* den) {
  ff xw[2 * S + 1];
  auto ldv = [&](int r) -> ff {
    if (r < 0 || r >= N) return ff_make(0.f, 0.f);
    const float2 v = X[(size_t)r * ld + col];
    return ff_make(v.x, v.y);
  };
#pragma unroll
  for (int j = 0; j <= 2 * S; ++j) xw[j] = ldv(j - S);
  ff nu = ff_make(0.f, 0.f), de = ff_make(0.f, 0.f);
  const ff zero = ff_make(0.f, 0.f);
  for (int k = 0; k < N; ++k) {
    if (k + S + 1 + kPf < N) prefetch_l2(X + (size_t)(k + S + 1 + kPf) * ld + col);
    ff tx = zero;
#pragma unroll
    for (int j = 0; j <= 2 * S; ++j) {
      const int c = k - S + j;
      if (c >= 0 && c < N) ff_acc(tx, mval_ff<S>(Tb, N, zero, k, c), xw[j]);
    }
    tx = ff_norm(tx);
    ff_acc(nu, xw[S], tx);
    ff_acc(de, xw[S], xw[S]);
    nu = ff_norm(nu);
    de = ff_norm(de);
#pragma unroll
    for (int j = 0; j < 2 * S; ++j) xw[j] = xw[j + 1];
    xw[2 * S] = ldv(k + S + 1);
  }
  *num = nu;
  *den = de;
}

// ||T x - theta x|| (pairs, leading part returned) for the pair vector of column col
template <int S>
__device__ double resid_pair(const float2* __restrict__ Tb, int N, const float2* __restrict__ X, size_t ld, int col,
                             ff theta) {
  const ff zero = ff_make(0.f, 0.f);
  const ff nth = ff_make(-theta.hi, -theta.lo);
  ff r2 = zero;
  for (int k = 0; k < N; ++k) {
    ff tx = zero;
    for (int c = max(0, k - S); c <= min(N - 1, k + S); ++c) {
      const float2 v = X[(size_t)c * ld + col];
      ff_acc(tx, mval_ff<S>(Tb, N, c == k ? nth : zero, k, c), ff_make(v.x, v.y));
    }
    tx = ff_norm(tx);
    ff_acc(r2, tx, tx);
    r2 = ff_norm(r2);
  }
  return sqrt(ff_to_double(r2));
}

// The inverse iteration of one singleton (the fp64 loop of k_invit, in pairs).  Returns false
// if a value went non-finite (the caller then runs the fp64 iteration from a fresh vector);
// otherwise the vector is normalised, its first and last S rows are doubles in X, and *lam and
// *res hold its Rayleigh quotient and residual norm.
template <int S>
__device__ bool invit_pair(Slot& sl, int N, size_t ld, int i, double est, bool refined, double tolc, double tnorm,
                           double* lam, double* res) {
  float2* X = reinterpret_cast<float2*>(sl.X);
  for (int k = 0; k < N; ++k) X[(size_t)k * ld + i] = make_float2((float)hash_unit((unsigned)k, (unsigned)i), 0.f);
  const ff estf = ff_from_double(est);
  const ff one = ff_make(1.f, 0.f);
  const double tiny = 8.0 * 0x1.0p-48 * tnorm + 1e-30;
  const fd tinyf(tiny);
  ff xscale = one, sigma = estf;
  bool warm = true;
  {
    float* U32 = reinterpret_cast<float*>(sl.U);
    const float tiny32 = FLT_EPSILON * (float)tnorm + FLT_MIN;
    for (int it = 0; it < kIters32 && warm; ++it) {
      const float amax = solve_pair<S, float>(sl.Tbf, N, estf, tiny32, xscale, X, ld, i, U32, i, ld);
      warm = isfinite(amax) && amax > 0.f;
      xscale = ff_make(warm ? 1.f / amax : 1.f, 0.f);
    }
  }
  ff rq = estf;
  if (warm) {
    ff num, den;
    rq_pair<S>(sl.Tbf, N, X, ld, i, &num, &den);
    warm = isfinite(num.hi) && isfinite(den.hi) && den.hi > 0.f;
    if (warm) {
      rq = ff_div(num, den);
      xscale = ff_from_double(1.0 / sqrt(ff_to_double(den)));
    }
  }
  if (!warm) {
    for (int k = 0; k < N; ++k) X[(size_t)k * ld + i] = make_float2((float)hash_unit((unsigned)k, (unsigned)i), 0.f);
    rq = estf;
    xscale = one;
  }
  // Rayleigh-quotient shifts while the iterate is dominated by the wanted eigenvector: for an
  // fp32 estimate within half its tolerance; for a refined estimate (kRefineRes ||T|| from the
  // eigenvalue, neighbours at least the fp64 tolerance away) within a thousandth of that
  auto may_shift = [&](ff q) {
    const double d = fabs(ff_to_double(q) - est);
    return d <= 0.5 * tolc + 8.0 * tiny && (!refined || d <= 1e-3 * tolc);
  };
  double prev = ff_to_double(rq);
  if (warm && may_shift(rq)) sigma = rq;
  int extra = -1;
  for (int it = 0; it < kMaxIters; ++it) {
    const float amax = solve_pair<S, fd>(sl.Tbf, N, sigma, tinyf, xscale, X, ld, i, reinterpret_cast<fd*>(sl.U), i, ld);
    if (!isfinite(amax)) return false;
    ff num, den;
    rq_pair<S>(sl.Tbf, N, X, ld, i, &num, &den);
    if (!(isfinite(num.hi) && isfinite(den.hi) && den.hi > 0.f)) return false;
    rq = ff_div(num, den);
    xscale = ff_from_double(1.0 / sqrt(ff_to_double(den)));
    const double rqd = ff_to_double(rq);
    if (extra == 0) break;
    if (extra > 0) --extra;
    if (extra < 0 && (warm || it >= 1) && fabs(rqd - prev) <= kSettle * tnorm) extra = 0;
    prev = rqd;
    if ((warm || it >= 1) && may_shift(rq)) sigma = rq;
  }
  for (int k = 0; k < N; ++k) {
    const float2 v = X[(size_t)k * ld + i];
    const ff y = ff_mul(ff_make(v.x, v.y), xscale);
    X[(size_t)k * ld + i] = make_float2(y.hi, y.lo);
  }
  ff num, den;
  rq_pair<S>(sl.Tbf, N, X, ld, i, &num, &den);
  if (!(isfinite(num.hi) && isfinite(den.hi) && den.hi > 0.f)) return false;
  // the residual of the converged pair vector (the acceptance test of the caller)
  rq = ff_div(num, den);
  *res = resid_pair<S>(sl.Tbf, N, X, ld, i, rq);
  // one fp64 inverse-iteration step at the pair Rayleigh quotient brings every component to
  // fp64 accuracy (the pair vector is accurate to about 2^-48 absolute, which the tiny last
  // components of converged Ritz vectors would feel); its Rayleigh quotient is the eigenvalue
  double* Xd = reinterpret_cast<double*>(X);
  for (int k = 0; k < N; ++k) {
    const float2 a = X[(size_t)k * ld + i];
    Xd[(size_t)k * ld + i] = (double)a.x + (double)a.y;
  }
  solve1<S>(sl.Tb, N, ff_to_double(rq), DBL_EPSILON * tnorm + DBL_MIN, 1.0, Xd, ld, i, sl.U, i, ld);
  double nu, de;
  rq_pass<S>(sl.Tb, N, Xd, ld, i, &nu, &de);
  if (!(isfinite(nu) && isfinite(de) && de > 0.0)) return false;
  *lam = nu / de;
  const double sc = 1.0 / sqrt(de);
  for (int k = 0; k < N; k = (k + 1 == S && N - S > S) ? N - S : k + 1)  // rows 0..S-1 and N-S..N-1, once
    Xd[(size_t)k * ld + i] *= sc;
  return isfinite(*lam) && isfinite(*res);
}

// first and last s components of eigenvectors i..i+c-1 ->
// a_i = (Q^T E_1 gamma)_i, w_i = (Q^T E_m tau^T)_i
template <int S>
__device__ void write_aw(const CheckArgs& g, Slot& sl, int m, int N, size_t ld, int i, int c) {
  const double* gam = g.log + REC_TNEXT * S * S;                                  // gamma (record 0)
  const double* tau = g.log + (size_t)m * LOG_NREC * S * S + REC_TNEXT * S * S;  // tau_{m+1,m}
  for (int v = 0; v < c; ++v) {
    const int iv = i + v;
    for (int cc = 0; cc < S; ++cc) {
      double av = 0.0, wv = 0.0;
      for (int t = 0; t < S; ++t) {
        av = fma(sl.X[(size_t)t * ld + iv], gam[t * S + cc], av);
        wv = fma(sl.X[(size_t)(N - S + t) * ld + iv], tau[cc * S + t], wv);
      }
      sl.a[(size_t)iv * S + cc] = av;
      sl.w[(size_t)iv * S + cc] = wv;
    }
  }
}

// 3. fp64 eigenpairs by inverse / Rayleigh-quotient iteration, one thread per eigenvalue
// (cluster leaders iterate their whole cluster as a subspace)
template <int S>
__global__ void k_invit(CheckArgs g, int round) {
  const int c_idx = blockIdx.y;
  const int m = g.ms[c_idx];
  const int N = S * m;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  Slot sl = get_slot(g.slots, S, g.nmax, c_idx);
  const size_t ld = (size_t)g.nmax;
  // round 1 retries the singletons of round 0 whose iteration settled away from their fp32
  // estimate (marked in part[]), now from fp64 estimates refined in between
  const bool retry = round == 1;
  if (retry && sl.part[i] == 0.0) return;
  const double tolc = retry ? sl.hdr[6] : sl.etol[i];
  const double tnorm = sl.hdr[3] * fmax(fabs(sl.hdr[0]), fabs(sl.hdr[1]));
  const double tiny = DBL_EPSILON * tnorm + DBL_MIN;
  int c = 1;
  if (retry) {
    if ((i > 0 && sl.est[i] - sl.est[i - 1] <= tolc) || (i + 1 < N && sl.est[i + 1] - sl.est[i] <= tolc)) {
      atomicOr(g.chk_err + m - 1, DERR_EIGEN);
#ifdef LYAP_DEBUG
      printf("eig fail retry m=%d N=%d i=%d est=%.17g tolc=%.4g\n", m, N, i, sl.est[i], tolc);
#endif
      return;
    }
  } else {
    // groups: consecutive estimates closer than the larger of their two tolerances.  A chain of
    // more than kMaxCluster such estimates (the tolerance floor chains eigenvalues that are tiny
    // against ||T|| but well apart, as the extended Krylov T_m has) is cut into groups of at most
    // kMaxCluster, each cut at the widest gap of its window so that the subspace iterations on
    // either side see well separated shifts; a cut narrower than four times the accuracy of the
    // refined estimates is an error.
    auto linked = [&](int a) { return sl.est[a] - sl.est[a - 1] <= fmax(sl.etol[a], sl.etol[a - 1]); };
    auto gap = [&](int a) { return sl.est[a] - sl.est[a - 1]; };
    int s0 = i;
    while (s0 > 0 && linked(s0)) --s0;
    int st = s0;
    for (;;) {  // the same partition of the chain in every thread
      int L = 1;
      while (st + L < N && L <= kMaxCluster && linked(st + L)) ++L;
      int len = L;
      if (L > kMaxCluster) {
        int best = st + 1;
        for (int p = st + 2; p <= st + kMaxCluster; ++p)
          if (gap(p) > gap(best)) best = p;
        len = best - st;
      }
      if (i < st + len) {
        c = len;
        break;
      }
      st += len;
    }
    if (i != st) return;  // not a leader
    const double cut_min = 4.0 * kRefineRes * tnorm + 8.0 * sqrt((double)N) * DBL_EPSILON * tnorm;
    if (st > s0 && !(gap(st) > cut_min)) {
      atomicOr(g.chk_err + m - 1, DERR_EIGEN);
#ifdef LYAP_DEBUG
      printf("eig fail cut m=%d N=%d i=%d est=%.17g prev=%.17g\n", m, N, i, sl.est[i], sl.est[i - 1]);
#endif
    }
  }
  if (c == 1) {
    const double est = sl.est[i];
    const bool refined = retry || tolc < sl.hdr[4];
    double rq = est, res = 0.0;
    if (!kPairInvit || !invit_pair<S>(sl, N, ld, i, est, refined, tolc, tnorm, &rq, &res)) {
    // fp64 from a fresh vector where the pair iteration overflowed
    for (int k = 0; k < N; ++k) sl.X[(size_t)k * ld + i] = hash_unit((unsigned)k, (unsigned)i);
    double sigma = est, prev = est, xscale = 1.0;
    // fp32 inverse iterations at the estimate (fp32 rate, half the scratch traffic) bring the
    // vector to fp32 accuracy; fp64 Rayleigh-quotient steps then finish it in one or two solves
    // (near-duplicate eigenvalues of T_m can put several tiny pivots in one factorisation; their
    // growth can overflow fp32, in which case the eigenpair restarts in fp64 from a fresh vector)
    bool warm = true;
    {
      float* U32 = reinterpret_cast<float*>(sl.U);
      const float tiny32 = FLT_EPSILON * (float)tnorm + FLT_MIN;
      // between fp32 solves the iterate is scaled by its largest entry; only the last one gets
      // its fp64 Rayleigh quotient
      for (int it = 0; it < kIters32 && warm; ++it) {
        const double amax = solve1<S, float>(sl.Tb, N, est, tiny32, xscale, sl.X, ld, i, U32, i, ld);
        warm = isfinite(amax) && amax > 0.0;
        xscale = warm ? 1.0 / amax : 1.0;
      }
      if (warm) {
        double num, den;
        rq_pass<S>(sl.Tb, N, sl.X, ld, i, &num, &den);
        warm = isfinite(num) && isfinite(den) && den > 0.0;
        rq = num / den;
        xscale = 1.0 / sqrt(den);
      }
      if (!warm) {
        for (int k = 0; k < N; ++k) sl.X[(size_t)k * ld + i] = hash_unit((unsigned)k, (unsigned)i);
        rq = est;
        xscale = 1.0;
      }
      prev = rq;
      if (warm && !refined && fabs(rq - est) <= 0.5 * tolc + 8.0 * tiny) sigma = rq;
    }
    int extra = -1;  // iterations still to run after the Rayleigh quotient settled
    for (int it = 0; it < kMaxIters; ++it) {
      solve1<S>(sl.Tb, N, sigma, tiny, xscale, sl.X, ld, i, sl.U, i, ld);
      double num, den;
      rq_pass<S>(sl.Tb, N, sl.X, ld, i, &num, &den);
      rq = num / den;
      xscale = 1.0 / sqrt(den);
      if (extra == 0) break;
      if (extra > 0) --extra;
      // settled: one more Rayleigh-quotient step brings the vector to full precision (from a
      // fresh start the first step cannot count as settled)
      if (extra < 0 && (warm || it >= 1) && fabs(rq - prev) <= kSettle * tnorm) extra = 0;
      prev = rq;
      // Rayleigh-quotient shifts while the iterate is dominated by the wanted eigenvector; an
      // fp64-refined estimate is already within a few eps ||T|| and stays the shift, so the
      // iteration cannot drift to a neighbour closer than the fp32 tolerance
      if (!refined && (warm || it >= 1) && fabs(rq - est) <= 0.5 * tolc + 8.0 * tiny) sigma = rq;
    }
    for (int k = 0; k < N; ++k) sl.X[(size_t)k * ld + i] *= xscale;
    rayleigh(sl.Tb, S, N, sl.X, ld, i, &rq, &res);
    }
    sl.lam[i] = rq;
#ifdef LYAP_DEBUG
    if (!(rq < 0.0))
      printf("invit lam>=0 m=%d N=%d i=%d est=%.17g rq=%.17g res=%.3e refined=%d retry=%d tolc=%.4g tnorm=%.4g\n", m, N,
             i, est, rq, res, (int)refined, (int)retry, tolc, tnorm);
#endif
    // the windows est +- tolc/2 of different groups are disjoint, so this also excludes
    // two singletons converging to the same eigenpair
    if (!(res <= kResTol * tnorm) || !isfinite(rq) || fabs(rq - est) > 0.5 * tolc) {
      if (!refined) {  // an fp32 estimate off by more than half the tolerance: retry in round 1
        sl.part[i] = 1.0;
        return;
      }
      atomicOr(g.chk_err + m - 1, DERR_EIGEN);
#ifdef LYAP_DEBUG
      printf("eig fail m=%d N=%d i=%d c=1 est=%.17g rq=%.17g res=%.3e tnorm=%.3e tolc=%.3e\n", m, N, i, est, rq, res,
             tnorm, tolc);
#endif
    }
  } else {
    // clusters are refined by one warp each in k_invit_clusters
    const int e = atomicAdd(sl.clist, 1);
    sl.clist[2 + 2 * e] = i;
    sl.clist[3 + 2 * e] = c;
    return;
  }
  write_aw<S>(g, sl, m, N, ld, i, 1);
}

// warp-wide sum (fixed shuffle order)
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// x_u^T T x_v over the rows the lane owns (contiguous vectors)
template <int S>
__device__ double lane_xTy(const double* __restrict__ Tb, int N, const double* __restrict__ xu,
                           const double* __restrict__ xv, int lane) {
  double acc = 0.0;
  for (int k = lane; k < N; k += 32) {
    double tx = 0.0;
    for (int c = max(0, k - S); c <= min(N - 1, k + S); ++c) tx = fma(tband(Tb, N, S, k, c), xv[c], tx);
    acc = fma(xu[k], tx, acc);
  }
  return acc;
}

// ||T x - theta x||^2 over the rows the lane owns (contiguous vector)
template <int S>
__device__ double lane_res2(const double* __restrict__ Tb, int N, const double* __restrict__ x, double theta,
                            int lane) {
  double r2 = 0.0;
  for (int k = lane; k < N; k += 32) {
    double tx = 0.0;
    for (int c = max(0, k - S); c <= min(N - 1, k + S); ++c) tx = fma(tband(Tb, N, S, k, c), x[c], tx);
    const double d = tx - theta * x[k];
    r2 = fma(d, d, r2);
  }
  return r2;
}

// the pack list of a slot sits in the unused tail of its cluster list (the list itself takes at
// most 2 + N ints of the 2 nmax + 32): [0] number of packs, then the first group of each pack
// and the end of the list
__device__ __forceinline__ int* pack_list(const Slot& sl, int nmax) { return sl.clist + nmax + 8; }

// 3a. groups packed greedily, in list order, into packs (one warp each in k_invit_clusters) of at
// most `cap` members, a larger group alone.  When the launch holds more warps than the GPU keeps
// resident (`dense`), the fp64 pipe is the limit and packs take up to 32 members; otherwise the
// members are spread evenly over the 64 warps a check gets (latency is the limit there).  One
// warp per check, the sizes read 32 at a time.
__global__ void k_pack_clusters(CheckArgs g, int dense) {
  const int c_idx = blockIdx.x;
  const int m = g.ms[c_idx];
  Slot sl = get_slot(g.slots, g.s, g.nmax, c_idx);
  const int lane = threadIdx.x;
  const int ncl = sl.clist[0];
  int* pk = pack_list(sl, g.nmax);
  int cap = 32;
  if (!dense) {
    int tm = 0;
    for (int base = 0; base < ncl; base += 32) {
      int cv = base + lane < ncl ? sl.clist[3 + 2 * (base + lane)] : 0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) cv += __shfl_xor_sync(0xffffffffu, cv, o);
      tm += cv;
    }
    cap = min(32, max(2, (tm + kClusterWarps - 1) / kClusterWarps));
  }
  int np = 0, tot = 0;
  for (int base = 0; base < ncl; base += 32) {
    const int cv = base + lane < ncl ? sl.clist[3 + 2 * (base + lane)] : 0;
    const int n = min(32, ncl - base);
    for (int t = 0; t < n; ++t) {
      const int c = __shfl_sync(0xffffffffu, cv, t);
      if (np == 0 || tot + c > cap) {
        if (lane == 0) pk[1 + np] = base + t;
        ++np;
        tot = 0;
      }
      tot += c;
    }
  }
  if (lane == 0) {
    pk[1 + np] = ncl;
    pk[0] = np;
  }
}

// 3b. groups of close estimates.  Lane v of a group iterates member v with its own estimate as
// a fixed shift (a Rayleigh-quotient shift could carry the last member to the eigenvalue just
// outside the group); after every step the group is re-orthonormalised (MGS, twice), and between
// rounds it is split by Rayleigh-Ritz, so the vectors of near-equal eigenvalues stay orthonormal.
// One warp takes a pack of groups (up to 32 members): the banded solves, which dominate, run on
// all the pack's lanes at once (the fp64 pipe spends the same time on a warp instruction
// whatever its active lanes), and the warp-wide orthonormalisation and Rayleigh-Ritz steps take
// the pack's groups in turn.  Every group keeps its own round state, so its result does not
// depend on the pack it lands in.  The members' vectors live contiguously in Xc (member i at
// Xc + i nmax), so the row loops coalesce.
template <int S>
__global__ void __launch_bounds__(128, 1) k_invit_clusters(CheckArgs g) {
  constexpr int WPB = kClusterWarps / kClusterBlocks;
  constexpr int kPackMax = 16;  // groups per pack (every group has at least two members)
  enum : int { kDone = 1, kPolish = 2, kFin = 4, kOvf = 8, kF64 = 16 };
  __shared__ double Hs[WPB][kMaxCluster][kMaxCluster];
  __shared__ double Vs[WPB][kMaxCluster][kMaxCluster];
  __shared__ double ths[WPB][32];  // Ritz values by member lane
  __shared__ int ords[WPB][kMaxCluster];
  __shared__ int qis[WPB][kPackMax], qcs[WPB][kPackMax], qos[WPB][kPackMax], qss[WPB][kPackMax];
  const int c_idx = blockIdx.y;
  const int m = g.ms[c_idx];
  const int N = S * m;
  Slot sl = get_slot(g.slots, S, g.nmax, c_idx);
  const size_t ld = (size_t)g.nmax;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const double tnorm = sl.hdr[3] * fmax(fabs(sl.hdr[0]), fabs(sl.hdr[1]));
  const double tiny = DBL_EPSILON * tnorm + DBL_MIN;
  const int* pk = pack_list(sl, g.nmax);
  const int npk = pk[0];
  double (*H)[kMaxCluster] = Hs[w];
  double (*V)[kMaxCluster] = Vs[w];
  double* theta = ths[w];
  int* ord = ords[w];
  int* qi = qis[w];  // first eigenvalue index of each group of the pack
  int* qc = qcs[w];  // its size
  int* qo = qos[w];  // its first lane
  int* qs = qss[w];  // its state bits
  for (int p = blockIdx.x * WPB + w; p < npk; p += gridDim.x * WPB) {
    const int e0 = pk[1 + p], nq = pk[2 + p] - e0;
    int myq = -1, myv = 0, off = 0;
    for (int q = 0; q < nq; ++q) {
      const int i = sl.clist[2 + 2 * (e0 + q)], c = sl.clist[3 + 2 * (e0 + q)];
      if (lane >= off && lane < off + c) {
        myq = q;
        myv = lane - off;
      }
      if (lane == 0) {
        qi[q] = i;
        qc[q] = c;
        qo[q] = off;
        qs[q] = 0;
      }
      off += c;
    }
    __syncwarp();
    const int me = myq >= 0 ? qi[myq] + myv : 0;  // eigenvalue index of the lane's member
    double shift = myq >= 0 ? sl.est[me] : 0.0;
    double* xme = sl.Xc + (size_t)me * ld;
    for (int q = 0; q < nq; ++q)
      for (int v = 0; v < qc[q]; ++v)
        for (int k = lane; k < N; k += 32)
          sl.Xc[(size_t)(qi[q] + v) * ld + k] = hash_unit((unsigned)k, (unsigned)(qi[q] + v));
    __syncwarp();
    // rounds at the fixed shifts until every member's residual passes, then one polishing round
    // at the Ritz values (Rayleigh-quotient shifts once the subspace is right); a group whose
    // fp32 round overflows restarts in fp64 from fresh vectors
    for (int round = 0; round < kMaxRounds + 1; ++round) {
      bool any = false;
      for (int q = 0; q < nq; ++q) {
        int st = qs[q];
        if (!(st & kFin)) {
          if (st & kDone) st |= (st & kPolish) ? kFin : kPolish;
          else if (round == kMaxRounds) st |= kFin;
        }
        any = any || !(st & kFin);
        __syncwarp();
        if (lane == 0) qs[q] = st;
      }
      __syncwarp();
      if (!any) break;
      const int mst = myq >= 0 ? qs[myq] : kFin;
      const bool live = !(mst & kFin);
      const bool pol = live && (mst & kPolish);
      const int r32 = (mst & kF64) ? 0 : kRounds32;
      if (pol) shift = theta[lane];
      for (int it = 0; it < 2; ++it) {
        if (live && (it == 0 || !pol)) {
          if (round < r32 && !pol)
            solve1<S, float>(sl.Tb, N, shift, FLT_EPSILON * (float)tnorm + FLT_MIN, 1.0, xme, 1, 0,
                             reinterpret_cast<float*>(sl.U), me, ld);
          else
            solve1<S>(sl.Tb, N, shift, tiny, 1.0, xme, 1, 0, sl.U, me, ld);
        }
        __syncwarp();
        for (int q = 0; q < nq; ++q) {
          const int st = qs[q];
          if ((st & kFin) || (it == 1 && (st & kPolish))) continue;
          const int c = qc[q];
          double* xc = sl.Xc + (size_t)qi[q] * ld;
          bool ovf = false;
          for (int pass = 0; pass < 2; ++pass)
            for (int v = 0; v < c; ++v) {
              double* xv = xc + (size_t)v * ld;
              for (int u = 0; u < v; ++u) {
                const double* xu = xc + (size_t)u * ld;
                double d = 0.0;
                for (int k = lane; k < N; k += 32) d = fma(xu[k], xv[k], d);
                d = warp_sum(d);
                for (int k = lane; k < N; k += 32) xv[k] = fma(-d, xu[k], xv[k]);
                __syncwarp();
              }
              double n2 = 0.0;
              for (int k = lane; k < N; k += 32) n2 = fma(xv[k], xv[k], n2);
              n2 = warp_sum(n2);
              if (!(n2 > 0.0) || !isfinite(n2)) {
                // the squared norm under- or overflowed: scale by the largest entry first
                double amax = 0.0;
                for (int k = lane; k < N; k += 32) amax = fmax(amax, fabs(xv[k]));
                amax = warp_max(amax);
                if (amax > 0.0 && isfinite(amax)) {
                  const double ia = 1.0 / amax;
                  n2 = 0.0;
                  for (int k = lane; k < N; k += 32) {
                    xv[k] *= ia;
                    n2 = fma(xv[k], xv[k], n2);
                  }
                  n2 = warp_sum(n2);
                }
              }
              const bool good = n2 > 0.0 && isfinite(n2);
              const double inv = good ? 1.0 / sqrt(n2) : 0.0;
              for (int k = lane; k < N; k += 32) xv[k] *= inv;
              __syncwarp();
              // a vector lost to overflow or cancellation restarts the group from fresh vectors in
              // fp64 (in any round: a zero vector would otherwise stay zero and pass every test)
              if (!good) ovf = true;
            }
          if (ovf) {
            __syncwarp();
            if (lane == 0) qs[q] = st | kOvf;
          }
          __syncwarp();
        }
      }
      for (int q = 0; q < nq; ++q) {
        const int st = qs[q];
        if (st & kFin) continue;
        const int c = qc[q], i = qi[q];
        double* xc = sl.Xc + (size_t)i * ld;
        if (st & kOvf) {
          for (int v = 0; v < c; ++v)
            for (int k = lane; k < N; k += 32) xc[(size_t)v * ld + k] = hash_unit((unsigned)k, (unsigned)(i + v));
          __syncwarp();
          if (lane == 0) qs[q] = (st & ~kOvf) | kF64;
          __syncwarp();
          continue;
        }
        // Rayleigh-Ritz
        for (int u = 0; u < c; ++u)
          for (int v = u; v < c; ++v) {
            const double h = warp_sum(lane_xTy<S>(sl.Tb, N, xc + (size_t)u * ld, xc + (size_t)v * ld, lane));
            if (lane == 0) {
              H[u][v] = h;
              H[v][u] = h;
            }
          }
        __syncwarp();
        if (lane == 0) {
          for (int u = 0; u < c; ++u)
            for (int v = 0; v < c; ++v) V[u][v] = u == v ? 1.0 : 0.0;
          for (int sweep = 0; sweep < 30; ++sweep) {
            double offd = 0.0, tot = 0.0;
            for (int u = 0; u < c; ++u)
              for (int v = 0; v < c; ++v) {
                tot += H[u][v] * H[u][v];
                if (u != v) offd += H[u][v] * H[u][v];
              }
            if (!(offd > 1e-32 * tot)) break;
            for (int a = 0; a < c; ++a)
              for (int b = a + 1; b < c; ++b) {
                if (H[a][b] == 0.0) continue;
                const double tq = (H[b][b] - H[a][a]) / (2.0 * H[a][b]);
                const double t = (tq >= 0 ? 1.0 : -1.0) / (fabs(tq) + sqrt(tq * tq + 1.0));
                const double cs = 1.0 / sqrt(t * t + 1.0), sn = t * cs;
                for (int k = 0; k < c; ++k) {
                  const double ha = H[a][k], hb = H[b][k];
                  H[a][k] = cs * ha - sn * hb;
                  H[b][k] = sn * ha + cs * hb;
                }
                for (int k = 0; k < c; ++k) {
                  const double ha = H[k][a], hb = H[k][b];
                  H[k][a] = cs * ha - sn * hb;
                  H[k][b] = sn * ha + cs * hb;
                  const double va = V[k][a], vb = V[k][b];
                  V[k][a] = cs * va - sn * vb;
                  V[k][b] = sn * va + cs * vb;
                }
              }
          }
          for (int v = 0; v < c; ++v) ord[v] = v;
          for (int a = 1; a < c; ++a) {
            const int t = ord[a];
            int b = a - 1;
            while (b >= 0 && H[ord[b]][ord[b]] > H[t][t]) {
              ord[b + 1] = ord[b];
              --b;
            }
            ord[b + 1] = t;
          }
          for (int v = 0; v < c; ++v) theta[qo[q] + v] = H[ord[v]][ord[v]];
        }
        __syncwarp();
        for (int k = lane; k < N; k += 32) {
          double row[kMaxCluster], out[kMaxCluster];
          for (int v = 0; v < c; ++v) row[v] = xc[(size_t)v * ld + k];
          for (int v = 0; v < c; ++v) {
            double t = 0.0;
            for (int u = 0; u < c; ++u) t = fma(row[u], V[u][ord[v]], t);
            out[v] = t;
          }
          for (int v = 0; v < c; ++v) xc[(size_t)v * ld + k] = out[v];
        }
        __syncwarp();
        if (round < ((st & kF64) ? 0 : kRounds32) || (st & kPolish)) continue;
        // the group has converged once every member's residual passes
        bool ok = true;
        for (int v = 0; v < c; ++v) {
          const double r2 = warp_sum(lane_res2<S>(sl.Tb, N, xc + (size_t)v * ld, theta[qo[q] + v], lane));
          ok = ok && sqrt(r2) <= kResTol * tnorm;
        }
        if (ok && lane == 0) qs[q] = st | kDone;
        __syncwarp();
      }
    }
    // final Rayleigh quotients and residual test; the first and last S rows go back to X for
    // the a and w rows
    for (int q = 0; q < nq; ++q) {
      const int i = qi[q], c = qc[q];
      for (int v = 0; v < c; ++v) {
        const double* xv = sl.Xc + (size_t)(i + v) * ld;
        double x2 = 0.0;
        for (int k = lane; k < N; k += 32) x2 = fma(xv[k], xv[k], x2);
        x2 = warp_sum(x2);
        const double num = warp_sum(lane_xTy<S>(sl.Tb, N, xv, xv, lane)) / x2;
        const double r2 = warp_sum(lane_res2<S>(sl.Tb, N, xv, num, lane)) / x2;
        if (lane < S) {
          sl.X[(size_t)lane * ld + i + v] = xv[lane];
          sl.X[(size_t)(N - S + lane) * ld + i + v] = xv[N - S + lane];
        }
        if (lane == 0) {
          sl.lam[i + v] = num;
          const bool inside =
              num >= sl.est[i] - 0.5 * sl.etol[i] && num <= sl.est[i + c - 1] + 0.5 * sl.etol[i + c - 1];
          // the vectors leave the rounds normalised: anything else is a lost vector
          const bool unit = fabs(x2 - 1.0) <= 1e-6;
          if (!(sqrt(r2) <= kResTol * tnorm) || !isfinite(num) || !inside || !unit) {
            atomicOr(g.chk_err + m - 1, DERR_EIGEN);
#ifdef LYAP_DEBUG
            printf("eig fail m=%d N=%d i=%d c=%d v=%d rq=%.17g res=%.3e tnorm=%.3e est[i]=%.17g est[i+c-1]=%.17g "
                   "etol=%.4g state=%d x2=%.6g\n",
                   m, N, i, c, v, num, sqrt(r2), tnorm, sl.est[i], sl.est[i + c - 1], sl.etol[i], qs[q], x2);
#endif
          }
        }
      }
      __syncwarp();
      if (lane == 0) write_aw<S>(g, sl, m, N, ld, i, c);
      __syncwarp();
    }
  }
}

// one warp per row i of Y~ W: ||sum_j (a_i.a_j)/(lam_i+lam_j) w_j||^2
__global__ void k_cauchy_lyap(CheckArgs g) {
  const int c_idx = blockIdx.y;
  const int m = g.ms[c_idx];
  const int s = g.s, N = s * m;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * (blockDim.x >> 5) + warp;
  if (i >= N) return;
  Slot sl = get_slot(g.slots, s, g.nmax, c_idx);
  double ai[LYAP_MAX_S], acc[LYAP_MAX_S];
  for (int c = 0; c < s; ++c) {
    ai[c] = sl.a[(size_t)i * s + c];
    acc[c] = 0.0;
  }
  const double li = sl.lam[i];
  bool bad = false;
  for (int j = lane; j < N; j += 32) {
    double dot = 0.0;
    for (int c = 0; c < s; ++c) dot = fma(ai[c], sl.a[(size_t)j * s + c], dot);
    const double den = li + sl.lam[j];
    bad |= !(den < 0.0);
    const double f = dot / den;
    for (int c = 0; c < s; ++c) acc[c] = fma(f, sl.w[(size_t)j * s + c], acc[c]);
  }
  double tot = 0.0;
  for (int c = 0; c < s; ++c) {
    double v = acc[c];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    tot = fma(v, v, tot);
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) {
    atomicOr(g.chk_err + m - 1, DERR_NOTNEGDEF);
#ifdef LYAP_DEBUG
    printf("not negdef m=%d N=%d i=%d lam_i=%.17g est_i=%.17g etol_i=%.4g\n", m, N, i, li, sl.est[i], sl.etol[i]);
#endif
  }
  if (lane == 0) sl.part[i] = tot;
}

// Sylvester: one warp per row i (rows of Y~ G, A side) or column j (Y~^T F, B side)
__global__ void k_cauchy_sylv(CheckArgs ga, CheckArgs gb, int side) {
  const int c_idx = blockIdx.y;
  const int m = ga.ms[c_idx];
  const int s = ga.s, N = s * m;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * (blockDim.x >> 5) + warp;
  if (i >= N) return;
  Slot sa = get_slot(ga.slots, s, ga.nmax, c_idx);
  Slot sb = get_slot(gb.slots, s, gb.nmax, c_idx);
  // side 0: row i of A-side against all j of B-side with G = sb.w; side 1: swapped with F = sa.w
  const Slot& me = side == 0 ? sa : sb;
  const Slot& ot = side == 0 ? sb : sa;
  double ai[LYAP_MAX_S], acc[LYAP_MAX_S];
  for (int c = 0; c < s; ++c) {
    ai[c] = me.a[(size_t)i * s + c];
    acc[c] = 0.0;
  }
  const double li = me.lam[i];
  bool bad = false;
  for (int j = lane; j < N; j += 32) {
    double dot = 0.0;
    for (int c = 0; c < s; ++c) dot = fma(ai[c], ot.a[(size_t)j * s + c], dot);
    const double den = li + ot.lam[j];
    bad |= !(den < 0.0);
    const double f = dot / den;
    for (int c = 0; c < s; ++c) acc[c] = fma(f, ot.w[(size_t)j * s + c], acc[c]);
  }
  double tot = 0.0;
  for (int c = 0; c < s; ++c) {
    double v = acc[c];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    tot = fma(v, v, tot);
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(ga.chk_err + m - 1, DERR_NOTNEGDEF);
  if (lane == 0) me.part[i] = tot;
}

// large A, small B (Alg. 5): one warp per eigenpair j of B,
//   part_j = ||sum_k (ctil_j . a_k) / (upsilon_j + lambda_k) w_k||^2,
// (e_j^T S) D_j^{-1} W with S = (P^T C2 gamma^T)(E_1^T Q), D_j = upsilon_j I + Lambda, W = Q^T E_m tau^T
__global__ void k_cauchy_smallb(CheckArgs g, const double* __restrict__ ups, const double* __restrict__ ct, int n2,
                                double* __restrict__ parts) {
  const int c_idx = blockIdx.y;
  const int m = g.ms[c_idx];
  const int s = g.s, N = s * m;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j = blockIdx.x * (blockDim.x >> 5) + warp;
  if (j >= n2) return;
  Slot sl = get_slot(g.slots, s, g.nmax, c_idx);
  double cj[LYAP_MAX_S], acc[LYAP_MAX_S];
  for (int c = 0; c < s; ++c) {
    cj[c] = ct[(size_t)j * s + c];
    acc[c] = 0.0;
  }
  const double uj = ups[j];
  bool bad = false;
  for (int k = lane; k < N; k += 32) {
    double dot = 0.0;
    for (int c = 0; c < s; ++c) dot = fma(cj[c], sl.a[(size_t)k * s + c], dot);
    const double den = uj + sl.lam[k];
    bad |= !(den < 0.0);
    const double f = dot / den;
    for (int c = 0; c < s; ++c) acc[c] = fma(f, sl.w[(size_t)k * s + c], acc[c]);
  }
  double tot = 0.0;
  for (int c = 0; c < s; ++c) {
    double v = acc[c];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    tot = fma(v, v, tot);
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(g.chk_err + m - 1, DERR_NOTNEGDEF);
  if (lane == 0) parts[(size_t)c_idx * n2 + j] = tot;
}

// Alg. 5's residual: sqrt(sum_j part_j) / (||C1||_F ||C2||_F); history and convergence flags
__global__ void k_finalize_smallb(CheckArgs g, const double* __restrict__ parts, int n2, double c2norm, double* hist,
                                  double tol, int* first_conv) {
  const int c_idx = blockIdx.x;
  const int m = g.ms[c_idx];
  __shared__ double red[256];
  double t = 0.0;
  for (int j = threadIdx.x; j < n2; j += blockDim.x) t += parts[(size_t)c_idx * n2 + j];
  red[threadIdx.x] = t;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double beta = g.log[REC_TDIAG * g.s * g.s];
    const double rel = sqrt(red[0]) / (beta * c2norm);
    hist[m - 1] = rel;
    if (g.chk_err[m - 1] != 0 || !isfinite(rel)) {
      if (!isfinite(rel)) atomicOr(g.chk_err + m - 1, DERR_NONFINITE);
      atomicMin(first_conv + 1, m);
    } else if (rel <= tol) {
      atomicMin(first_conv, m);
    }
  }
}

// sum of the per-row parts in a fixed order; history entry and convergence flag
__global__ void k_finalize(CheckArgs ga, CheckArgs gb, int sylv, double* hist, double tol, int* first_conv) {
  const int c_idx = blockIdx.x;
  const int m = ga.ms[c_idx];
  const int s = ga.s, N = s * m;
  Slot sa = get_slot(ga.slots, s, ga.nmax, c_idx);
  __shared__ double red[256];
  double t = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) t += sa.part[i];
  if (sylv) {
    Slot sb = get_slot(gb.slots, s, gb.nmax, c_idx);
    for (int i = threadIdx.x; i < N; i += blockDim.x) t += sb.part[i];
  }
  red[threadIdx.x] = t;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
#ifdef LYAP_DEBUG
  if (threadIdx.x == 0 && !isfinite(red[0])) {
    int nl = 0, na = 0, nw = 0, np = 0;
    for (int i = 0; i < N; ++i) {
      nl += !isfinite(sa.lam[i]);
      np += !isfinite(sa.part[i]);
      for (int c = 0; c < s; ++c) {
        na += !isfinite(sa.a[(size_t)i * s + c]);
        nw += !isfinite(sa.w[(size_t)i * s + c]);
      }
    }
    int first = -1;
    for (int i = 0; i < N && first < 0; ++i)
      if (!isfinite(sa.part[i])) first = i;
    printf("nonfinite m=%d N=%d lam %d a %d w %d part %d first part %d lam %.6g est %.6g etol %.3g clist %d\n", m, N, nl,
           na, nw, np, first, first >= 0 ? sa.lam[first] : 0.0, first >= 0 ? sa.est[first] : 0.0,
           first >= 0 ? sa.etol[first] : 0.0, sa.clist[0]);
  }
#endif
  if (threadIdx.x == 0) {
    const int SS = s * s;
    const double betaA = ga.log[REC_TDIAG * SS];
    double res, scale;
    if (sylv) {
      const double betaB = gb.log[REC_TDIAG * SS];
      res = sqrt(red[0]);
      scale = betaA * betaB;
    } else {
      res = sqrt(2.0 * red[0]);
      scale = betaA * betaA;
    }
    const double rel = res / scale;
    hist[m - 1] = rel;
    // a failed check at m counts only if no earlier m converged (the host compares
    // the first failing m with the first converged m)
    if (ga.chk_err[m - 1] != 0 || !isfinite(rel)) {
      if (!isfinite(rel)) atomicOr(ga.chk_err + m - 1, DERR_NONFINITE);
      atomicMin(first_conv + 1, m);
    } else if (rel <= tol) {
      atomicMin(first_conv, m);
    }
  }
}

// nslots slots of leading dimension nmax per operator, operator 1's after operator 0's
CheckArgs make_args(lyap_handle* h, int opi, const int* ms, int nchk, int nmax, int nslots) {
  CheckArgs g;
  g.log = h->op[opi].log;
  g.s = h->s;
  g.nmax = nmax;
  const size_t sd = slot_doubles(h->s, nmax);
  g.slots = reinterpret_cast<double*>(h->check_ws) + sd * (size_t)(opi * nslots);
  g.nchk = nchk;
  for (int c = 0; c < kMaxChecks; ++c) g.ms[c] = c < nchk ? ms[c] : 0;
  g.flags = h->flags;
  g.chk_err = h->chk_err;
  return g;
}

int eigen_pipeline(const CheckArgs& g, int nmax_batch, cudaStream_t st) {
  k_setup_band<<<g.nchk, 256, 0, st>>>(g);
  dim3 gv((nmax_batch + 31) / 32, g.nchk);
  dim3 gr((nmax_batch + 7) / 8, g.nchk);  // eight warps a block, one eigenvalue a warp
  dim3 gi((nmax_batch + kInvitThreads - 1) / kInvitThreads, g.nchk);
  switch (g.s) {
    case 1: k_bisect_band32<1><<<gr, 256, 0, st>>>(g); break;
    case 2: k_bisect_band32<2><<<gr, 256, 0, st>>>(g); break;
    case 3: k_bisect_band32<3><<<gr, 256, 0, st>>>(g); break;
    case 4: k_bisect_band32<4><<<gr, 256, 0, st>>>(g); break;
    case 8: k_bisect_band32<8><<<gr, 256, 0, st>>>(g); break;
  }
  // refined estimates for the members of fp32 groups; the singleton iteration; refined
  // estimates and a second iteration for the singletons whose fp32 estimate proved too far off
  k_mark_refine<<<g.nchk, 256, 0, st>>>(g);
  for (int round = 0; round < 2; ++round) {
    switch (g.s) {
      case 1: k_refine64<1><<<gr, 256, 0, st>>>(g, round); break;
      case 2: k_refine64<2><<<gr, 256, 0, st>>>(g, round); break;
      case 3: k_refine64<3><<<gr, 256, 0, st>>>(g, round); break;
      case 4: k_refine64<4><<<gr, 256, 0, st>>>(g, round); break;
      case 8: k_refine64<8><<<gr, 256, 0, st>>>(g, round); break;
    }
    if (round == 1) break;
    switch (g.s) {
      case 1: k_invit<1><<<gi, kInvitThreads, 0, st>>>(g, 0); break;
      case 2: k_invit<2><<<gi, kInvitThreads, 0, st>>>(g, 0); break;
      case 3: k_invit<3><<<gi, kInvitThreads, 0, st>>>(g, 0); break;
      case 4: k_invit<4><<<gi, kInvitThreads, 0, st>>>(g, 0); break;
      case 8: k_invit<8><<<gi, kInvitThreads, 0, st>>>(g, 0); break;
    }
  }
  switch (g.s) {
    case 1: k_invit<1><<<gi, kInvitThreads, 0, st>>>(g, 1); break;
    case 2: k_invit<2><<<gi, kInvitThreads, 0, st>>>(g, 1); break;
    case 3: k_invit<3><<<gi, kInvitThreads, 0, st>>>(g, 1); break;
    case 4: k_invit<4><<<gi, kInvitThreads, 0, st>>>(g, 1); break;
    case 8: k_invit<8><<<gi, kInvitThreads, 0, st>>>(g, 1); break;
  }
  // groups: packed into warps of up to 32 members; 16 blocks of 4 warps per check take the packs
  // in turn (the SM count is read once: a process uses one GPU model)
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  // two blocks of k_invit_clusters (254 registers a thread) fit on an SM
  k_pack_clusters<<<g.nchk, 32, 0, st>>>(g, g.nchk * kClusterWarps >= 8 * sms);
  dim3 gc(kClusterBlocks, g.nchk);
  switch (g.s) {
    case 1: k_invit_clusters<1><<<gc, 128, 0, st>>>(g); break;
    case 2: k_invit_clusters<2><<<gc, 128, 0, st>>>(g); break;
    case 3: k_invit_clusters<3><<<gc, 128, 0, st>>>(g); break;
    case 4: k_invit_clusters<4><<<gc, 128, 0, st>>>(g); break;
    case 8: k_invit_clusters<8><<<gc, 128, 0, st>>>(g); break;
  }
  return 9;
}

}  // namespace

size_t check_slot_bytes(int s, int nmax) { return slot_doubles(s, nmax) * sizeof(double); }

// leading dimension of the slots of a batch whose largest check is at m_hi
int batch_nmax(int s, int m_hi) { return (s * m_hi + 7) / 8 * 8; }

// Evaluates the checks at m = ms[0..nchk-1] (ascending, nchk <= the check batch); the slots of
// the batch have leading dimension batch_nmax(s, ms[nchk-1]) and must fit in the check area (the
// caller sizes the batch).
int launch_check_list(lyap_handle* h, const int* ms, int nchk, cudaStream_t st) {
  if (nchk <= 0) return 0;
  int nl = 0;
  const int m_hi = ms[nchk - 1];
  const int nmax_batch = h->s * m_hi;
  const int nb = batch_nmax(h->s, m_hi);
  CheckArgs ga = make_args(h, 0, ms, nchk, nb, nchk);
  nl += eigen_pipeline(ga, nmax_batch, st);
  CheckArgs gb = ga;
  const int wpb = 8;
  dim3 gc((nmax_batch + wpb - 1) / wpb, nchk);
  if (h->plan.n2 > 0) {
    const int n2 = h->plan.n2;
    k_cauchy_smallb<<<dim3((n2 + wpb - 1) / wpb, nchk), wpb * 32, 0, st>>>(ga, h->smallb.ups, h->smallb.ctil, n2,
                                                                          h->smallb.parts);
    k_finalize_smallb<<<nchk, 256, 0, st>>>(ga, h->smallb.parts, n2, h->smallb.c2norm, h->hist, h->tol, h->flags + 1);
    return nl + 2;
  }
  if (h->plan.sylv) {
    gb = make_args(h, 1, ms, nchk, nb, nchk);
    nl += eigen_pipeline(gb, nmax_batch, st);
    k_cauchy_sylv<<<gc, wpb * 32, 0, st>>>(ga, gb, 0);
    k_cauchy_sylv<<<gc, wpb * 32, 0, st>>>(ga, gb, 1);
    nl += 2;
  } else {
    k_cauchy_lyap<<<gc, wpb * 32, 0, st>>>(ga);
    nl += 1;
  }
  k_finalize<<<nchk, 256, 0, st>>>(ga, gb, h->plan.sylv, h->hist, h->tol, h->flags + 1);
  return nl + 1;
}

// every m = m_lo..m_hi that the check period d selects (m % d == 0)
int launch_check_batch(lyap_handle* h, int m_lo, int m_hi, cudaStream_t st) {
  const int every = h->opt.check_every > 0 ? h->opt.check_every : 1;
  int ms[kMaxChecks];
  int n = 0;
  for (int m = m_lo; m <= m_hi && n < kMaxChecks; ++m)
    if (m % every == 0) ms[n++] = m;
  return launch_check_list(h, ms, n, st);
}

// Eigenvalues and a, w rows of T_m (slot 0 of operator opi) for the factor step.
int launch_eigen_for_factor(lyap_handle* h, int opi, int m, cudaStream_t st) {
  CheckArgs g = make_args(h, opi, &m, 1, h->plan.nmax, h->plan.check_batch);
  return eigen_pipeline(g, h->s * m, st);
}

// device pointers of slot 0 of operator opi (factor step reads lam and a)
void check_slot0(lyap_handle* h, int opi, double** lam, double** a, double** w) {
  const size_t sd = slot_doubles(h->s, h->plan.nmax);
  double* p = reinterpret_cast<double*>(h->check_ws) + sd * (size_t)(opi * h->plan.check_batch);
  const int nmax = h->plan.nmax, s = h->s;
  p += 8 + ((size_t)(s + 1) * nmax + 1) / 2;  // hdr, Tb32
  p += nmax;              // est
  *lam = p;
  p += 2 * (size_t)nmax;        // lam, part
  p += (size_t)(s + 1) * nmax;  // fp64 band
  *a = p;
  p += (size_t)s * nmax;
  *w = p;
}

// ---------------------------------------------------------------------------------
// Allocation-free residual evaluation (lyap_residual_noalloc in include/lyap.h).
//
// The scratch of one check (the slot of the kernels above, a coefficient log in the
// format they read, the history entry and the error words) lives in a file-scope
// device array sized for s <= 4 and s*m <= 256.  Host code must not use the array's
// name as a device address: it is looked up once per device with cudaGetSymbolAddress.
// ---------------------------------------------------------------------------------
#include <mutex>

namespace {

constexpr int kNoAllocMaxS = 4;
constexpr int kNoAllocMaxN = 256;  // s * m
constexpr size_t kNoAllocSlot = slot_doubles(kNoAllocMaxS, kNoAllocMaxN);  // one check slot
constexpr size_t kNoAllocLog = (size_t)(kNoAllocMaxN + 1) * LOG_NREC * kNoAllocMaxS * kNoAllocMaxS;
constexpr size_t kNoAllocInts = 4 + kNoAllocMaxN;  // flags, per-m error bits
constexpr size_t kNoAllocDoubles = kNoAllocSlot + kNoAllocLog + kNoAllocMaxN + (kNoAllocInts + 1) / 2;

__device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

// copies the caller's T_m band, gamma, tau_{m+1,m} and beta into the log format the
// check kernels read; clears the error words
__global__ void k_noalloc_pack(int s, int m, const double* __restrict__ ab, int ldab, const double* __restrict__ gam,
                               const double* __restrict__ tau, double beta, double* __restrict__ log, int* ints) {
  const int SS = s * s;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < (m + 1) * SS; t += gridDim.x * blockDim.x) {
    const int j = t / SS, k = t % SS, a = k / s, b = k % s;
    double* rec = log + (size_t)j * LOG_NREC * SS;
    if (j == 0) {
      rec[REC_TNEXT * SS + k] = gam[k];
      if (k == 0) rec[REC_TDIAG * SS] = beta;
      continue;
    }
    // diagonal block j: T_m[(j-1)s + a][(j-1)s + b], band entry of the lower triangle
    const int r = (j - 1) * s + a, c = (j - 1) * s + b;
    const int lo = r > c ? c : r, d = r > c ? r - c : c - r;
    rec[REC_TDIAG * SS + k] = ab[d + (size_t)lo * ldab];
    // sub-diagonal block below it (tau_{j+1,j}, upper triangular), or the caller's tau for j = m
    double tn = 0.0;
    if (j < m) {
      if (a <= b) tn = ab[(s + a - b) + (size_t)((j - 1) * s + b) * ldab];
    } else {
      tn = tau[k];
    }
    rec[REC_TNEXT * SS + k] = tn;
  }
  if (blockIdx.x == 0)
    for (int t = threadIdx.x; t < (int)kNoAllocInts; t += blockDim.x) ints[t] = (t >= 1 && t < 4) ? INT_MAX : 0;
}

__device__ int noalloc_status(int bits) {
  if (bits & DERR_BREAKDOWN) return LYAP_ERR_BREAKDOWN;
  if (bits & DERR_NONFINITE) return LYAP_ERR_NONFINITE;
  if (bits & DERR_NOTNEGDEF) return LYAP_ERR_NOT_NEGDEF;
  if (bits & DERR_EIGEN) return LYAP_ERR_EIGEN;
  return bits ? LYAP_ERR_EIGEN : LYAP_OK;
}

__global__ void k_noalloc_out(int m, const double* __restrict__ hist, const int* __restrict__ chk_err, double* rel_out,
                              int* status_out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    *rel_out = hist[m - 1];
    *status_out = noalloc_status(chk_err[m - 1]);
  }
}

std::mutex g_noalloc_mu;
void* g_noalloc_addr[64] = {};

}  // namespace

extern "C" int lyap_residual_noalloc(int s, int m, const double* ab, int ldab, const double* gamma,
                                     const double* tau_next, double beta, double* rel_out, int* status_out,
                                     void* stream) {
  if (s < 1 || s > kNoAllocMaxS || m < 1 || s * m > kNoAllocMaxN || ldab < s + 1) return LYAP_ERR_ARG;
  if (!ab || !gamma || !tau_next || !rel_out || !status_out || !(beta > 0.0)) return LYAP_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return LYAP_ERR_CUDA;
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
      // the host-side symbol is not a device address: ask the runtime, with dev current
      if (cudaGetSymbolAddress(&g_noalloc_addr[dev], g_noalloc_scratch) != cudaSuccess) {
        g_noalloc_addr[dev] = nullptr;
        return LYAP_ERR_CUDA;
      }
    }
    base = g_noalloc_addr[dev];
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double* slot = static_cast<double*>(base);
  double* log = slot + kNoAllocSlot;
  double* hist = log + kNoAllocLog;
  int* ints = reinterpret_cast<int*>(hist + kNoAllocMaxN);  // [0] error bits, [1..2] first converged / failed m
  int* chk_err = ints + 4;
  k_noalloc_pack<<<8, 256, 0, st>>>(s, m, ab, ldab, gamma, tau_next, beta, log, ints);
  CheckArgs g;
  g.log = log;
  g.slots = slot;
  g.s = s;
  g.nmax = kNoAllocMaxN;
  g.nchk = 1;
  g.ms[0] = m;
  g.flags = ints;
  g.chk_err = chk_err;
  eigen_pipeline(g, s * m, st);
  k_cauchy_lyap<<<dim3((s * m + 7) / 8, 1), 256, 0, st>>>(g);
  k_finalize<<<1, 256, 0, st>>>(g, g, 0, hist, -1.0, ints + 1);
  k_noalloc_out<<<1, 32, 0, st>>>(m, hist, chk_err, rel_out, status_out);
  return cudaGetLastError() == cudaSuccess ? LYAP_OK : LYAP_ERR_CUDA;
}
