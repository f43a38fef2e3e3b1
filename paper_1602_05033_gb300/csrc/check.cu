// Convergence check of Alg. 1 step 6 by Prop. 3.1 / Alg. 3 (Alg. 4 for Sylvester).
//
// For a batch of consecutive iteration counts m (one slot each) the kernels
//   1. build T_m from the coefficient log and reduce it to a tridiagonal F_m = P^T T_m P
//      by Givens bulge chasing, accumulating only the first and last s rows of P
//      (Alg. 3 step 1; the paper uses LAPACK's band reduction for this);
//   2. find every eigenvalue of F_m by bisection on Sturm counts (Alg. 3 step 2);
//   3. for each eigenvalue, build the eigenvector of F_m by a twisted
//      factorisation and project it on the 2s tracked rows of P, giving the
//      first and last s components of the eigenvector of T_m (Alg. 3 step 3),
//      then a_i = (Q^T E_1 gamma)_i and w_i = (Q^T E_m tau^T)_i (steps 4-5);
//   4. accumulate ||e_i^T S D_i^{-1} W||^2 per i (steps 7-10);
//   5. sum, take sqrt(2 sum)/beta^2 and record the history and the first
//      converged m.
// Everything runs in fp64.  Reductions are in a fixed order.
#include "common.cuh"

#include <float.h>
#include <limits.h>
#include <math.h>

namespace {

constexpr int kBandThreads = 512;
constexpr int kGroup = 8;  // lanes per concurrent Givens rotation
constexpr int kDelta = 4;  // stage lag between consecutive sweeps (non-overlapping windows for b >= 2)

struct Slot {
  double* hdr;   // [0] Gershgorin lo, [1] hi, [2] max e^2
  double* d;
  double* e;
  double* e2;
  double* rows;  // 2s x nmax
  double* lam;
  double* a;     // nmax x s
  double* w;     // nmax x s
  double* part;  // nmax
  double* dp;    // nmax x nmax, [k][i]
  double* dm;    // nmax x nmax, [k][i]
};

__host__ __device__ inline size_t slot_doubles(int s, int nmax) {
  return 8 + 5 * (size_t)nmax + 4 * (size_t)s * nmax + 2 * (size_t)nmax * nmax;
}

__device__ inline Slot get_slot(double* base, int s, int nmax, int idx) {
  Slot sl;
  double* p = base + (size_t)idx * slot_doubles(s, nmax);
  sl.hdr = p; p += 8;
  sl.d = p; p += nmax;
  sl.e = p; p += nmax;
  sl.e2 = p; p += nmax;
  sl.lam = p; p += nmax;
  sl.part = p; p += nmax;
  sl.rows = p; p += 2 * (size_t)s * nmax;
  sl.a = p; p += (size_t)s * nmax;
  sl.w = p; p += (size_t)s * nmax;
  sl.dp = p; p += (size_t)nmax * nmax;
  sl.dm = p;
  return sl;
}

struct CheckArgs {
  const double* log;  // coefficient log of this operator
  double* slots;      // slot array for this operator
  int s;
  int nmax;
  int m_lo;           // slot c <-> m = m_lo + c
  int nchk;
  int every;          // check period d
  int* flags;
};

__device__ inline bool checked(const CheckArgs& g, int m) { return (m % g.every) == 0; }

// lower band (with one extra diagonal for the bulge) of T_m in shared memory
__device__ inline double& TB(double* tb, int N, int i, int c) { return tb[(size_t)(i - c) * N + c]; }

__global__ void __launch_bounds__(kBandThreads) k_band_reduce(CheckArgs g) {
  extern __shared__ double smem[];
  const int c_idx = blockIdx.x;
  const int m = g.m_lo + c_idx;
  if (!checked(g, m)) return;
  const int s = g.s, b = s, N = s * m;
  const int SS = s * s;
  Slot sl = get_slot(g.slots, s, g.nmax, c_idx);
  double* tb = smem;                        // (b + 2) x N
  const int nrows_tr = 2 * s;
  const bool rows_in_smem = ((size_t)(b + 2 + nrows_tr) * N * sizeof(double)) <= (size_t)200 * 1024;
  double* rows = rows_in_smem ? smem + (size_t)(b + 2) * N : sl.rows;
  // assemble the band of T_m: symmetric part of tau_jj on the diagonal blocks,
  // tau_{j+1,j} below them (Sec. 2); extra diagonal b+1 starts at zero
  for (size_t t = threadIdx.x; t < (size_t)(b + 2) * N; t += blockDim.x) {
    const int dd = (int)(t / N), c = (int)(t % N);
    const int i = c + dd;
    double v = 0.0;
    if (dd <= b && i < N) {
      const int J = i / s, Jc = c / s;
      if (J == Jc) {
        const double* D = g.log + (size_t)(J + 1) * LOG_NREC * SS + REC_TDIAG * SS;
        v = 0.5 * (D[(i % s) * s + (c % s)] + D[(c % s) * s + (i % s)]);
      } else if (J == Jc + 1) {
        const double* Tn = g.log + (size_t)(Jc + 1) * LOG_NREC * SS + REC_TNEXT * SS;
        v = Tn[(i % s) * s + (c % s)];
      }
    }
    tb[t] = v;
  }
  for (size_t t = threadIdx.x; t < (size_t)nrows_tr * N; t += blockDim.x) {
    const int r = (int)(t / N), c = (int)(t % N);
    const int target = r < s ? r : N - s + (r - s);
    rows[t] = (c == target) ? 1.0 : 0.0;
  }
  __syncthreads();
  if (b >= 2 && N >= 3) {
    const int lane = threadIdx.x & 31;
    const int glane = lane & (kGroup - 1);
    const int group = threadIdx.x / kGroup;
    const int ngroups = blockDim.x / kGroup;
    const int nsweeps = (N - 2) * (b - 1);
    const int maxlen = (N + b - 1) / b + 1;
    const long nstages = (long)kDelta * (nsweeps - 1) + maxlen + 1;
    for (long st = 0; st < nstages; ++st) {
      long lo = (st - maxlen) / kDelta;
      if (lo < 0) lo = 0;
      long hi = st / kDelta;
      if (hi > nsweeps - 1) hi = nsweeps - 1;
      for (long base = lo; base <= hi; base += ngroups) {
        const long idx = base + group;
        bool valid = idx <= hi;
        int p = 0, kc = 0;
        if (valid) {
          const int k = (int)(idx / (b - 1));
          const int d = b - (int)(idx % (b - 1));
          const long t = st - (long)kDelta * idx;
          if (t < 0) valid = false;
          else if (t == 0) {
            p = k + d - 1;
            kc = k;
            if (k + d > N - 1) valid = false;
          } else {
            p = k + d - 1 + (int)t * b;
            kc = p - b;
            if (p + 1 > N - 1) valid = false;
          }
        }
        const int q = p + 1;
        double cs = 1.0, sn = 0.0;
        if (valid && glane == 0) {
          const double x = TB(tb, N, p, kc);
          const double y = TB(tb, N, q, kc);
          const double r2 = x * x + y * y;
          if (r2 > 0.0) {
            const double r = sqrt(r2);
            const double inv = 1.0 / r;
            cs = x * inv;
            sn = y * inv;
            TB(tb, N, p, kc) = r;
            TB(tb, N, q, kc) = 0.0;
          }
        }
        const int src = lane & ~(kGroup - 1);
        cs = __shfl_sync(0xffffffffu, cs, src);
        sn = __shfl_sync(0xffffffffu, sn, src);
        if (valid && sn != 0.0) {
          // items: columns kc+1..p-1, the 2x2 block, rows q+1..min(N-1, p+b+1), tracked rows
          const int ncols = p - kc - 1;
          const int rlast = min(N - 1, p + b + 1);
          const int nbelow = rlast - q;
          const int nitems = ncols + 1 + (nbelow > 0 ? nbelow : 0) + nrows_tr;
          for (int it = glane; it < nitems; it += kGroup) {
            if (it < ncols) {
              const int j = kc + 1 + it;
              double& u = TB(tb, N, p, j);
              double& v = TB(tb, N, q, j);
              const double uu = u, vv = v;
              u = cs * uu + sn * vv;
              v = -sn * uu + cs * vv;
            } else if (it == ncols) {
              double& app = TB(tb, N, p, p);
              double& aqp = TB(tb, N, q, p);
              double& aqq = TB(tb, N, q, q);
              const double A = app, B = aqp, D = aqq;
              // rows then columns of the symmetric 2x2 block
              const double r0 = cs * A + sn * B, r1 = cs * B + sn * D;    // new row p (cols p, q)
              const double s0 = -sn * A + cs * B, s1 = -sn * B + cs * D;  // new row q
              app = cs * r0 + sn * r1;
              aqp = cs * s0 + sn * s1;
              aqq = -sn * s0 + cs * s1;
            } else if (it < ncols + 1 + (nbelow > 0 ? nbelow : 0)) {
              const int i = q + 1 + (it - ncols - 1);
              double& u = TB(tb, N, i, p);
              double& v = TB(tb, N, i, q);
              const double uu = u, vv = v;
              u = cs * uu + sn * vv;
              v = -sn * uu + cs * vv;
            } else {
              const int r = it - ncols - 1 - (nbelow > 0 ? nbelow : 0);
              double& u = rows[(size_t)r * N + p];
              double& v = rows[(size_t)r * N + q];
              const double uu = u, vv = v;
              u = cs * uu + sn * vv;
              v = -sn * uu + cs * vv;
            }
          }
        }
        __syncwarp();
      }
      __syncthreads();
    }
  }
  // tridiagonal out, Gershgorin bounds
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    sl.d[i] = TB(tb, N, i, i);
    const double ei = (i + 1 < N) ? TB(tb, N, i + 1, i) : 0.0;
    sl.e[i] = ei;
    sl.e2[i] = ei * ei;
  }
  if (rows_in_smem)
    for (size_t t = threadIdx.x; t < (size_t)nrows_tr * N; t += blockDim.x) sl.rows[(size_t)(t / N) * N + t % N] = rows[t];
  __syncthreads();
  if (threadIdx.x == 0) {
    double lo = INFINITY, hi = -INFINITY, emax = 0.0;
    for (int i = 0; i < N; ++i) {
      const double r = (i > 0 ? fabs(sl.e[i - 1]) : 0.0) + (i + 1 < N ? fabs(sl.e[i]) : 0.0);
      lo = fmin(lo, sl.d[i] - r);
      hi = fmax(hi, sl.d[i] + r);
      emax = fmax(emax, sl.e2[i]);
    }
    const double span = fmax(fabs(lo), fabs(hi));
    sl.hdr[0] = lo - 4.0 * DBL_EPSILON * span - DBL_MIN;
    sl.hdr[1] = hi + 4.0 * DBL_EPSILON * span + DBL_MIN;
    sl.hdr[2] = emax;
  }
}

__device__ inline int sturm_count(const double* __restrict__ d, const double* __restrict__ e2, int N, double x,
                                  double pivmin) {
  int cnt = 0;
  double q = d[0] - x;
  if (fabs(q) <= pivmin) q = -pivmin;
  cnt += q < 0.0;
  for (int i = 1; i < N; ++i) {
    q = (d[i] - x) - e2[i - 1] / q;
    if (fabs(q) <= pivmin) q = -pivmin;
    cnt += q < 0.0;
  }
  return cnt;
}

__global__ void k_eigvals(CheckArgs g) {
  const int c_idx = blockIdx.y;
  const int m = g.m_lo + c_idx;
  if (!checked(g, m)) return;
  const int N = g.s * m;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  Slot sl = get_slot(g.slots, g.s, g.nmax, c_idx);
  const double pivmin = DBL_MIN * fmax(1.0, sl.hdr[2]);
  double lo = sl.hdr[0], hi = sl.hdr[1];
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (!(hi - lo > DBL_EPSILON * (fabs(lo) + fabs(hi)) + pivmin) || mid <= lo || mid >= hi) break;
    if (sturm_count(sl.d, sl.e2, N, mid, pivmin) <= i) lo = mid;
    else hi = mid;
  }
  sl.lam[i] = 0.5 * (lo + hi);
}

__global__ void k_eigvecs(CheckArgs g) {
  const int c_idx = blockIdx.y;
  const int m = g.m_lo + c_idx;
  if (!checked(g, m)) return;
  const int s = g.s, N = s * m, SS = s * s;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  Slot sl = get_slot(g.slots, s, g.nmax, c_idx);
  const size_t ld = (size_t)g.nmax;
  const double lam = sl.lam[i];
  const double tiny = DBL_EPSILON * fmax(fabs(sl.hdr[0]), fabs(sl.hdr[1])) * 1e-3 + DBL_MIN;
  // stationary (top-down) factorisation pivots D+_k
  double dk = sl.d[0] - lam;
  if (fabs(dk) < tiny) dk = tiny;
  sl.dp[i] = dk;
  for (int k = 1; k < N; ++k) {
    dk = (sl.d[k] - lam) - sl.e2[k - 1] / dk;
    if (fabs(dk) < tiny) dk = tiny;
    sl.dp[(size_t)k * ld + i] = dk;
  }
  // progressive (bottom-up) pivots D-_k and the twist index r = argmin |gamma_k|
  double dmk = sl.d[N - 1] - lam;
  if (fabs(dmk) < tiny) dmk = tiny;
  sl.dm[(size_t)(N - 1) * ld + i] = dmk;
  int r = N - 1;
  double gbest = fabs(sl.dp[(size_t)(N - 1) * ld + i]);  // gamma_{N-1} = D+_{N-1}
  for (int k = N - 2; k >= 0; --k) {
    dmk = (sl.d[k] - lam) - sl.e2[k] / dmk;
    if (fabs(dmk) < tiny) dmk = tiny;
    sl.dm[(size_t)k * ld + i] = dmk;
    const double gam = sl.dp[(size_t)k * ld + i] + dmk - (sl.d[k] - lam);
    if (fabs(gam) < gbest) {
      gbest = fabs(gam);
      r = k;
    }
  }
  // eigenvector z of F_m with z_r = 1, projected on the tracked rows of P
  double y[2 * LYAP_MAX_S];
  for (int t = 0; t < 2 * s; ++t) y[t] = sl.rows[(size_t)t * N + r];
  double nrm2 = 1.0;
  double z = 1.0;
  for (int k = r - 1; k >= 0; --k) {
    z = -(sl.e[k] / sl.dp[(size_t)k * ld + i]) * z;
    nrm2 += z * z;
    for (int t = 0; t < 2 * s; ++t) y[t] += sl.rows[(size_t)t * N + k] * z;
  }
  z = 1.0;
  for (int k = r; k < N - 1; ++k) {
    z = -(sl.e[k] / sl.dm[(size_t)(k + 1) * ld + i]) * z;
    nrm2 += z * z;
    for (int t = 0; t < 2 * s; ++t) y[t] += sl.rows[(size_t)t * N + k + 1] * z;
  }
  const double inv = 1.0 / sqrt(nrm2);
  const double* gam = g.log + REC_TNEXT * SS;                                 // gamma (record 0)
  const double* tau = g.log + (size_t)m * LOG_NREC * SS + REC_TNEXT * SS;    // tau_{m+1,m}
  for (int c = 0; c < s; ++c) {
    double av = 0.0, wv = 0.0;
    for (int t = 0; t < s; ++t) {
      av += y[t] * inv * gam[t * s + c];        // (Q^T E_1 gamma)_{i,c}
      wv += y[s + t] * inv * tau[c * s + t];    // (Q^T E_m tau^T)_{i,c}
    }
    sl.a[(size_t)i * s + c] = av;
    sl.w[(size_t)i * s + c] = wv;
  }
}

// one warp per row i of Y~ W: ||sum_j (a_i.a_j)/(lam_i+lam_j) w_j||^2
__global__ void k_cauchy_lyap(CheckArgs g) {
  const int c_idx = blockIdx.y;
  const int m = g.m_lo + c_idx;
  if (!checked(g, m)) return;
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
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(g.flags, DERR_NOTNEGDEF);
  if (lane == 0) sl.part[i] = tot;
}

// Sylvester: one warp per row i (rows of Y~ G, A side) or column j (Y~^T F, B side)
__global__ void k_cauchy_sylv(CheckArgs ga, CheckArgs gb, int side) {
  const int c_idx = blockIdx.y;
  const int m = ga.m_lo + c_idx;
  if (!checked(ga, m)) return;
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
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(ga.flags, DERR_NOTNEGDEF);
  if (lane == 0) me.part[i] = tot;
}

// sum of the per-row parts in a fixed order; history entry and convergence flag
__global__ void k_finalize(CheckArgs ga, CheckArgs gb, int sylv, double* hist, double tol, int* first_conv) {
  const int c_idx = blockIdx.x;
  const int m = ga.m_lo + c_idx;
  if (!checked(ga, m)) {
    if (threadIdx.x == 0) hist[m - 1] = __longlong_as_double(0x7ff8000000000000LL);
    return;
  }
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
    if (!isfinite(rel)) atomicOr(ga.flags, DERR_NONFINITE);
    else if (rel <= tol) atomicMin(first_conv, m);
  }
}

CheckArgs make_args(lyap_handle* h, int opi, int m_lo, int nchk, int every, int slot_base) {
  CheckArgs g;
  g.log = h->op[opi].log;
  g.s = h->s;
  g.nmax = h->plan.nmax;
  const size_t sd = slot_doubles(h->s, h->plan.nmax);
  g.slots = reinterpret_cast<double*>(h->check_ws) + sd * (size_t)(opi * h->plan.check_batch + slot_base);
  g.m_lo = m_lo;
  g.nchk = nchk;
  g.every = every;
  g.flags = h->flags;
  return g;
}

size_t band_smem_bytes(int s, int N) {
  const size_t band = (size_t)(s + 2) * N * sizeof(double);
  const size_t rows = (size_t)2 * s * N * sizeof(double);
  return (band + rows) <= (size_t)200 * 1024 ? band + rows : band;
}

void eigen_pipeline(const CheckArgs& g, int nmax_batch, cudaStream_t st) {
  const size_t smem = band_smem_bytes(g.s, nmax_batch);
  cudaFuncSetAttribute(k_band_reduce, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_band_reduce<<<g.nchk, kBandThreads, smem, st>>>(g);
  dim3 gv((nmax_batch + 31) / 32, g.nchk);
  k_eigvals<<<gv, 32, 0, st>>>(g);
  k_eigvecs<<<gv, 32, 0, st>>>(g);
}

}  // namespace

size_t check_slot_bytes(int s, int nmax) { return slot_doubles(s, nmax) * sizeof(double); }

// Evaluates the checks for m = m_lo..m_hi (at most plan.check_batch of them).
void launch_check_batch(lyap_handle* h, int m_lo, int m_hi, cudaStream_t st) {
  const int nchk = m_hi - m_lo + 1;
  const int every = h->opt.check_every > 0 ? h->opt.check_every : 1;
  const int nmax_batch = h->s * m_hi;
  CheckArgs ga = make_args(h, 0, m_lo, nchk, every, 0);
  eigen_pipeline(ga, nmax_batch, st);
  CheckArgs gb = ga;
  const int wpb = 8;
  dim3 gc((nmax_batch + wpb - 1) / wpb, nchk);
  if (h->plan.sylv) {
    gb = make_args(h, 1, m_lo, nchk, every, 0);
    eigen_pipeline(gb, nmax_batch, st);
    k_cauchy_sylv<<<gc, wpb * 32, 0, st>>>(ga, gb, 0);
    k_cauchy_sylv<<<gc, wpb * 32, 0, st>>>(ga, gb, 1);
  } else {
    k_cauchy_lyap<<<gc, wpb * 32, 0, st>>>(ga);
  }
  k_finalize<<<nchk, 256, 0, st>>>(ga, gb, h->plan.sylv, h->hist, h->tol, h->flags + 1);
}

// Eigenvalues and a, w rows of T_m (slot 0 of operator opi) for the factor step.
void launch_eigen_for_factor(lyap_handle* h, int opi, int m, cudaStream_t st) {
  CheckArgs g = make_args(h, opi, m, 1, 1, 0);
  eigen_pipeline(g, h->s * m, st);
}

// device pointers of slot 0 of operator opi (factor step reads lam and a)
void check_slot0(lyap_handle* h, int opi, double** lam, double** a, double** w) {
  const size_t sd = slot_doubles(h->s, h->plan.nmax);
  double* p = reinterpret_cast<double*>(h->check_ws) + sd * (size_t)(opi * h->plan.check_batch);
  const int nmax = h->plan.nmax, s = h->s;
  p += 8;
  p += 3 * (size_t)nmax;  // d, e, e2
  *lam = p;
  p += 2 * (size_t)nmax;  // lam, part
  p += 2 * (size_t)s * nmax;  // rows
  *a = p;
  p += (size_t)s * nmax;
  *w = p;
}
