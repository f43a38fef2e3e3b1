// Block Lanczos sweeps (Alg. 2 with CholQR2 normalisation) and the second pass (Sec. 3.3).
//
// One iteration j of pass 1 is four row sweeps over n rows, each followed by a
// fixed-order reduction of per-CTA s x s partial sums done by the last CTA:
//
//   S1  W = A V_j (SELL-C-sigma SpMM)            partials V_{j-1}^T W, V_j^T W, V_j^T V_{j-1}
//       -> alpha_{j-1} = V_{j-1}^T W,  alpha_j = V_j^T W - (V_j^T V_{j-1}) alpha_{j-1}
//          (the first block MGS sweep of Alg. 2 in fused form: algebraically
//           identical to subtracting V_{j-1} alpha_{j-1} before projecting on V_j)
//   S2  w1 = W - V_{j-1} alpha_{j-1} - V_j alpha_j   partials V_{j-1}^T w1, V_j^T w1, w1^T w1
//       -> beta_{j-1}, beta_j (second MGS sweep), G1 = w1^T w1 - beta^T beta, R1 = chol(G1)
//   S3  w2 = w1 - V_{j-1} beta_{j-1} - V_j beta_j, x = w2 R1^{-1}   partial x^T x
//       -> R2 = chol(x^T x), tau_{j+1,j} = R2 R1
//   S4  V_{j+1} = x R2^{-1}
//
// The rows w1, w2, x are recomputed from W, V_{j-1}, V_j in every sweep instead
// of being stored; the second pass (S1's SpMM fused with S4's row recipe and the
// logged coefficients) therefore regenerates V_{j+1} bit for bit.
#include "common.cuh"

#include <math.h>

#include <algorithm>

namespace {

constexpr int kThreads = 256;
// CTAs per SM the sweeps are compiled for: enough warps for HBM latency without spilling
// the per-thread s x s accumulators (3 for fp32 rows, 2 for fp64)
template <typename T>
struct MinBlocks { static constexpr int value = 3; };
template <>
struct MinBlocks<double> { static constexpr int value = 2; };
constexpr int kWarps = kThreads / 32;

template <typename T>
struct AccT { using type = double; };
template <>
struct AccT<float> { using type = float; };

// ---- row loads/stores -------------------------------------------------------
template <typename T, int S>
__device__ __forceinline__ void load_row(const T* __restrict__ X, int64_t ld, int64_t i, T (&r)[S]) {
  const T* p = X + i * ld;
#pragma unroll
  for (int a = 0; a < S; ++a) r[a] = p[a];
}
template <int S>
__device__ __forceinline__ void load_row(const float* __restrict__ X, int64_t ld, int64_t i, float (&r)[S]) {
  const float* p = X + i * ld;
  if constexpr (S % 4 == 0) {
#pragma unroll
    for (int a = 0; a < S; a += 4) {
      float4 v = *reinterpret_cast<const float4*>(p + a);
      r[a] = v.x; r[a + 1] = v.y; r[a + 2] = v.z; r[a + 3] = v.w;
    }
  } else if constexpr (S == 2) {
    float2 v = *reinterpret_cast<const float2*>(p);
    r[0] = v.x; r[1] = v.y;
  } else {
#pragma unroll
    for (int a = 0; a < S; ++a) r[a] = p[a];
  }
}
template <int S>
__device__ __forceinline__ void load_row(const double* __restrict__ X, int64_t ld, int64_t i, double (&r)[S]) {
  const double* p = X + i * ld;
  if constexpr (S % 2 == 0) {
#pragma unroll
    for (int a = 0; a < S; a += 2) {
      double2 v = *reinterpret_cast<const double2*>(p + a);
      r[a] = v.x; r[a + 1] = v.y;
    }
  } else {
#pragma unroll
    for (int a = 0; a < S; ++a) r[a] = p[a];
  }
}
template <typename T, int S>
__device__ __forceinline__ void store_row(T* __restrict__ X, int64_t ld, int64_t i, const T (&r)[S]) {
  T* p = X + i * ld;
#pragma unroll
  for (int a = 0; a < S; ++a) p[a] = r[a];
}
template <int S>
__device__ __forceinline__ void store_row(float* __restrict__ X, int64_t ld, int64_t i, const float (&r)[S]) {
  float* p = X + i * ld;
  if constexpr (S % 4 == 0) {
#pragma unroll
    for (int a = 0; a < S; a += 4) *reinterpret_cast<float4*>(p + a) = make_float4(r[a], r[a + 1], r[a + 2], r[a + 3]);
  } else if constexpr (S == 2) {
    *reinterpret_cast<float2*>(p) = make_float2(r[0], r[1]);
  } else {
#pragma unroll
    for (int a = 0; a < S; ++a) p[a] = r[a];
  }
}
template <int S>
__device__ __forceinline__ void store_row(double* __restrict__ X, int64_t ld, int64_t i, const double (&r)[S]) {
  double* p = X + i * ld;
  if constexpr (S % 2 == 0) {
#pragma unroll
    for (int a = 0; a < S; a += 2) *reinterpret_cast<double2*>(p + a) = make_double2(r[a], r[a + 1]);
  } else {
#pragma unroll
    for (int a = 0; a < S; ++a) p[a] = r[a];
  }
}

// ---- SELL-C-sigma row product: w = (A V)[row] -----------------------------------
// Entries are taken kUnroll at a time: all column indices and values first, then all
// gathers of V rows, then the FMAs, so a row has kUnroll independent gathers in flight
// instead of waiting one DRAM round trip per nonzero.  The summation order is the
// entry order of the row in every case (identical bits in both passes).
constexpr int kUnroll = 8;
template <typename T, int S>
__device__ __forceinline__ void sell_row_at(const OpDev& op, int64_t slice_ptr, int width, int lane,
                                            const T* __restrict__ Vc, int64_t ldc, T (&w)[S]) {
#pragma unroll
  for (int a = 0; a < S; ++a) w[a] = T(0);
  const int64_t base = slice_ptr + lane;
  const T* __restrict__ val = static_cast<const T*>(op.sell_val);
  for (int j0 = 0; j0 < width; j0 += kUnroll) {
    int32_t c[kUnroll];
    T v[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const bool in = j0 + u < width;
      const int64_t e = base + (int64_t)(in ? j0 + u : 0) * LYAP_SLICE;
      c[u] = __ldg(op.sell_col + e);
      v[u] = in ? __ldg(val + e) : T(0);
    }
    T x[kUnroll][S];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) load_row<S>(Vc, ldc, c[u], x[u]);
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int a = 0; a < S; ++a) w[a] = fma(v[u], x[u][a], w[a]);
  }
}

template <typename T, int S>
__device__ __forceinline__ void sell_row(const OpDev& op, int64_t slice, int lane, const T* __restrict__ Vc,
                                         int64_t ldc, T (&w)[S]) {
  sell_row_at<T, S>(op, op.slice_ptr[slice], op.slice_w[slice], lane, Vc, ldc, w);
}


// loads through L2 only (ld.global.cg): rows written earlier in the same launch by other SMs
template <int S>
__device__ __forceinline__ void load_row_cg(const float* __restrict__ X, int64_t ld, int64_t i, float (&r)[S]) {
  const float* p = X + i * ld;
  if constexpr (S % 4 == 0) {
#pragma unroll
    for (int a = 0; a < S; a += 4) {
      const float4 v = __ldcg(reinterpret_cast<const float4*>(p + a));
      r[a] = v.x; r[a + 1] = v.y; r[a + 2] = v.z; r[a + 3] = v.w;
    }
  } else if constexpr (S == 2) {
    const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
    r[0] = v.x; r[1] = v.y;
  } else {
#pragma unroll
    for (int a = 0; a < S; ++a) r[a] = __ldcg(p + a);
  }
}
template <int S>
__device__ __forceinline__ void load_row_cg(const double* __restrict__ X, int64_t ld, int64_t i, double (&r)[S]) {
  const double* p = X + i * ld;
  if constexpr (S % 2 == 0) {
#pragma unroll
    for (int a = 0; a < S; a += 2) {
      const double2 v = __ldcg(reinterpret_cast<const double2*>(p + a));
      r[a] = v.x; r[a + 1] = v.y;
    }
  } else {
#pragma unroll
    for (int a = 0; a < S; ++a) r[a] = __ldcg(p + a);
  }
}

// sell_row with the V rows loaded through L2 (same entry order, same bits)
template <typename T, int S>
__device__ __forceinline__ void sell_row_cg(const OpDev& op, int64_t slice, int lane, const T* __restrict__ Vc,
                                            int64_t ldc, T (&w)[S]) {
#pragma unroll
  for (int a = 0; a < S; ++a) w[a] = T(0);
  const int64_t base = op.slice_ptr[slice] + lane;
  const int width = op.slice_w[slice];
  const T* __restrict__ val = static_cast<const T*>(op.sell_val);
  for (int j0 = 0; j0 < width; j0 += kUnroll) {
    int32_t c[kUnroll];
    T v[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const bool in = j0 + u < width;
      const int64_t e = base + (int64_t)(in ? j0 + u : 0) * LYAP_SLICE;
      c[u] = __ldg(op.sell_col + e);
      v[u] = in ? __ldg(val + e) : T(0);
    }
    T x[kUnroll][S];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) load_row_cg<S>(Vc, ldc, c[u], x[u]);
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int a = 0; a < S; ++a) w[a] = fma(v[u], x[u][a], w[a]);
  }
}

// ---- coefficient blocks in shared memory ---------------------------------------
// co[k][a][b]: k-th s x s coefficient block, converted to the bulk type.
template <typename T, int S>
struct Coefs {
  T ap[S][S], ad[S][S];  // first MGS sweep: alpha_{j-1}, alpha_j
  T tp[S][S], td[S][S];  // both sweeps combined: tau_{j-1,j}, tau_jj
  T r1[S][S], tn[S][S];  // first CholQR factor, tau_{j+1,j} = R2 R1 (upper)
  T r1i[S], tni[S];      // reciprocals of their diagonals
};

// w1 = W - Vp ap - Vc ad ; w2 = w1 - Vp bp - Vc bd (row vectors times s x s blocks)
template <typename T, int S>
__device__ __forceinline__ void mgs_row(const T (&p)[S], const T (&q)[S], const T (&M1)[S][S], const T (&M2)[S][S],
                                        T (&w)[S], bool has_prev) {
#pragma unroll
  for (int b = 0; b < S; ++b) {
    T t = w[b];
    if (has_prev) {
#pragma unroll
      for (int a = 0; a < S; ++a) t = fma(-p[a], M1[a][b], t);
    }
#pragma unroll
    for (int a = 0; a < S; ++a) t = fma(-q[a], M2[a][b], t);
    w[b] = t;
  }
}

// x R = w  (R upper triangular): forward substitution with precomputed 1/R_bb
template <typename T, int S>
__device__ __forceinline__ void trsm_row(const T (&R)[S][S], const T (&Ri)[S], T (&w)[S]) {
#pragma unroll
  for (int b = 0; b < S; ++b) {
    T t = w[b];
#pragma unroll
    for (int a = 0; a < b; ++a) t = fma(-w[a], R[a][b], t);
    w[b] = t * Ri[b];
  }
}

// row recipe of S4 and of the second pass: v = (w - p tau_{j-1,j} - q tau_jj) tau_{j+1,j}^{-1}
// (both MGS sweeps and both CholQR factors applied at once, as in the recurrence of eq. 2.6)
template <typename T, int S>
__device__ __forceinline__ void next_row(const Coefs<T, S>& co, const T (&p)[S], const T (&q)[S], T (&w)[S],
                                         bool has_prev) {
  mgs_row<T, S>(p, q, co.tp, co.td, w, has_prev);
  trsm_row<T, S>(co.tn, co.tni, w);
}

template <typename T, int S>
__device__ void load_coefs(Coefs<T, S>& co, const double* __restrict__ rec, int stage) {
  // stage: records available (1: alpha; 2: + tau_{j-1,j}, tau_jj, R1; 3: + tau_{j+1,j})
  const int SS = S * S;
  for (int k = threadIdx.x; k < SS; k += blockDim.x) {
    const int a = k / S, b = k % S;
    co.ap[a][b] = T(rec[REC_APREV * SS + k]);
    co.ad[a][b] = T(rec[REC_ADIAG * SS + k]);
    if (stage >= 2) {
      co.tp[a][b] = T(rec[REC_TPREV * SS + k]);
      co.td[a][b] = T(rec[REC_TDIAG * SS + k]);
      co.r1[a][b] = T(rec[REC_R1 * SS + k]);
    }
    if (stage >= 3) co.tn[a][b] = T(rec[REC_TNEXT * SS + k]);
  }
  for (int b = threadIdx.x; b < S; b += blockDim.x) {
    if (stage >= 2) co.r1i[b] = T(1.0 / rec[REC_R1 * SS + b * S + b]);
    if (stage >= 3) co.tni[b] = T(1.0 / rec[REC_TNEXT * SS + b * S + b]);
  }
  __syncthreads();
}

// ---- deterministic two-stage reductions ----------------------------------------------
// Stage 1 (every CTA): the threads' accumulators are summed by warp shuffles in a fixed order,
// then over the warps in order, into the CTA's slot of the partials array.  Stage 2 (one CTA):
// warp w sums coefficients w, w + kWarps, ...; its lanes stride over the slots and combine in a
// fixed shuffle order, so the result does not depend on timing.
//
// GB300 runs fp64 at a small fraction of its fp32 rate (a warp instruction holds the SM's fp64
// pipe for about 16 cycles whatever its active lanes), so with fp32 accumulators both stages
// stay on the fp32 pipe: a partial is an unevaluated pair hi + lo of floats, and pairs are
// added with Knuth's TwoSum, which yields the exact rounding error of each addition (about 44
// significant bits, far below the fp32 rounding of the sweep data).  A slot holds the pair in
// the 8 bytes of a double.  fp64 accumulators keep fp64 throughout.
struct FF {
  float hi, lo;
};
__device__ __forceinline__ FF ff_add(FF a, FF b) {
  const float s = a.hi + b.hi;
  const float v = s - a.hi;
  float e = (a.hi - (s - v)) + (b.hi - v);
  e += a.lo + b.lo;
  const float hi = s + e;
  return FF{hi, e - (hi - s)};
}

// Slots are stored coefficient-major, P[k * count + slot], so stage 2 reads each coefficient's
// slots with coalesced loads.
//
// stage 1: this CTA's sums of acc -> P[k * count + slot] (a float pair for fp32 accumulators);
// scratch holds kWarps * NACC doubles (shared memory).  Ends with the sums written by the
// threads k < NACC (no barrier after the writes).
template <typename Acc, int NACC>
__device__ void cta_partial(Acc (&acc)[NACC], double* __restrict__ P, unsigned int slot, unsigned int count,
                            double* __restrict__ scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  Acc* sc = reinterpret_cast<Acc*>(scratch);
#pragma unroll
  for (int k = 0; k < NACC; ++k) {
    Acc v = acc[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sc[warp * NACC + k] = v;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < NACC; k += blockDim.x) {
    if constexpr (sizeof(Acc) == sizeof(float)) {
      FF t{0.f, 0.f};
      for (int w = 0; w < kWarps; ++w) t = ff_add(t, FF{sc[w * NACC + k], 0.f});
      reinterpret_cast<float2*>(P)[(size_t)k * count + slot] = make_float2(t.hi, t.lo);
    } else {
      double t = 0.0;
      for (int w = 0; w < kWarps; ++w) t += sc[w * NACC + k];
      P[(size_t)k * count + slot] = t;
    }
  }
}

// stage 2: tot[k] = sum over slots b < count of P[k * count + b]; lane l adds the slots
// l, l + 32, ... in order, loading eight at a time (independent loads in flight together);
// ends with a barrier
template <typename Acc, int NACC>
__device__ void sum_slots(const double* __restrict__ P, unsigned int count, double* __restrict__ tot) {
  constexpr int kB = 8;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = warp; k < NACC; k += kWarps) {
    if constexpr (sizeof(Acc) == sizeof(float)) {
      const float2* col = reinterpret_cast<const float2*>(P) + (size_t)k * count;
      FF t{0.f, 0.f};
      for (unsigned int b0 = 0; b0 < count; b0 += 32 * kB) {
        float2 v[kB];
#pragma unroll
        for (int u = 0; u < kB; ++u) {
          const unsigned int b = b0 + 32 * u + lane;
          v[u] = b < count ? __ldcg(col + b) : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < kB; ++u) t = ff_add(t, FF{v[u].x, v[u].y});
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const FF u{__shfl_xor_sync(0xffffffffu, t.hi, o), __shfl_xor_sync(0xffffffffu, t.lo, o)};
        t = ff_add(t, u);
      }
      if (lane == 0) tot[k] = (double)t.hi + (double)t.lo;
    } else {
      const double* col = P + (size_t)k * count;
      double t = 0.0;
      for (unsigned int b0 = 0; b0 < count; b0 += 32 * kB) {
        double v[kB];
#pragma unroll
        for (int u = 0; u < kB; ++u) {
          const unsigned int b = b0 + 32 * u + lane;
          v[u] = b < count ? __ldcg(col + b) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < kB; ++u) t += v[u];
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (lane == 0) tot[k] = t;
    }
  }
  __syncthreads();
}

// stage 1 into this CTA's slot, then stage 2 by the last CTA to arrive (returns true there)
template <typename Acc, int NACC>
__device__ bool reduce_partials(Acc (&acc)[NACC], double* __restrict__ partials, unsigned int* counter,
                                double* __restrict__ tot /*smem NACC*/, double* __restrict__ scratch /*smem kWarps*NACC*/,
                                unsigned int slot, unsigned int count) {
  cta_partial<Acc, NACC>(acc, partials, slot, count, scratch);
  __threadfence();
  __shared__ unsigned int ticket;
  __syncthreads();
  if (threadIdx.x == 0) ticket = atomicAdd(counter, 1u);
  __syncthreads();
  if (ticket != count - 1) return false;
  __threadfence();
  sum_slots<Acc, NACC>(partials, count, tot);
  if (threadIdx.x == 0) *counter = 0u;
  return true;
}

// small dense helpers on one thread (fp64, S <= 8)
template <int S>
__device__ bool chol_upper(const double* G, double* R) {
  // G = R^T R, R upper triangular with positive diagonal
  for (int i = 0; i < S * S; ++i) R[i] = 0.0;
  for (int j = 0; j < S; ++j) {
    double d = G[j * S + j];
    for (int k = 0; k < j; ++k) d -= R[k * S + j] * R[k * S + j];
    if (!(d > 0.0) || !isfinite(d)) return false;
    const double rjj = sqrt(d);
    R[j * S + j] = rjj;
    for (int i = j + 1; i < S; ++i) {
      double t = G[j * S + i];
      for (int k = 0; k < j; ++k) t -= R[k * S + j] * R[k * S + i];
      R[j * S + i] = t / rjj;
    }
  }
  return true;
}
template <int S>
__device__ void matmul(const double* A, const double* B, double* C) {  // C = A B
  for (int i = 0; i < S; ++i)
    for (int j = 0; j < S; ++j) {
      double t = 0.0;
      for (int k = 0; k < S; ++k) t += A[i * S + k] * B[k * S + j];
      C[i * S + j] = t;
    }
}
template <int S>
__device__ bool all_finite(const double* A, int n) {
  for (int i = 0; i < n; ++i)
    if (!isfinite(A[i])) return false;
  return true;
}

// ---- per-iteration finalisations (one thread, after the reduction) -------------
// S1: alpha_{j-1} = V_{j-1}^T W, alpha_j = V_j^T W - (V_j^T V_{j-1}) alpha_{j-1}
template <int S>
__device__ void finalize_s1(double* rec, const double* tot, int has_prev, int* flags) {
  constexpr int SS = S * S;
  double ap[SS], ad[SS], cr[SS], t[SS];
  for (int k = 0; k < SS; ++k) {
    ap[k] = has_prev ? tot[k] : 0.0;
    cr[k] = has_prev ? tot[2 * SS + k] : 0.0;
  }
  matmul<S>(cr, ap, t);
  for (int k = 0; k < SS; ++k) ad[k] = tot[SS + k] - t[k];
  for (int k = 0; k < SS; ++k) {
    rec[REC_APREV * SS + k] = ap[k];
    rec[REC_ADIAG * SS + k] = ad[k];
    rec[REC_CROSS * SS + k] = cr[k];
  }
  if (!all_finite<S>(ad, SS) || !all_finite<S>(ap, SS)) atomicOr(flags, DERR_NONFINITE);
}

// S2: second MGS coefficients, combined tau_{j-1,j}, tau_jj, and R1 = chol(G1)
template <int S>
__device__ void finalize_s2(double* rw, const double* tot, int hp, int* flags) {
  constexpr int SS = S * S;
  double bp[SS], bd[SS], cr[SS], t[SS], G[SS], R1[SS];
  for (int k = 0; k < SS; ++k) {
    bp[k] = hp ? tot[k] : 0.0;
    cr[k] = rw[REC_CROSS * SS + k];
  }
  matmul<S>(cr, bp, t);
  for (int k = 0; k < SS; ++k) bd[k] = tot[SS + k] - t[k];
  // G1 = w1^T w1 - bp^T bp - bd^T bd: Gram of w2 = w1 - V beta (V orthonormal up to rounding)
  for (int a = 0, e = 2 * SS; a < S; ++a)
    for (int b = a; b < S; ++b, ++e) {
      double v = tot[e];
      for (int k = 0; k < S; ++k) v -= bp[k * S + a] * bp[k * S + b] + bd[k * S + a] * bd[k * S + b];
      G[a * S + b] = v;
      G[b * S + a] = v;
    }
  for (int k = 0; k < SS; ++k) {
    rw[REC_BPREV * SS + k] = bp[k];
    rw[REC_BDIAG * SS + k] = bd[k];
    rw[REC_TPREV * SS + k] = rw[REC_APREV * SS + k] + bp[k];
    rw[REC_TDIAG * SS + k] = rw[REC_ADIAG * SS + k] + bd[k];
  }
  const bool finite = all_finite<S>(G, SS);
  if (!finite) atomicOr(flags, DERR_NONFINITE);
  if (!chol_upper<S>(G, R1)) {
    if (finite) atomicOr(flags, DERR_BREAKDOWN);
    for (int k = 0; k < SS; ++k) R1[k] = (k % (S + 1) == 0) ? 1.0 : 0.0;
  }
  for (int k = 0; k < SS; ++k) rw[REC_R1 * SS + k] = R1[k];
}

// S3: R2 = chol(x^T x), tau_{j+1,j} = R2 R1
template <int S>
__device__ void finalize_s3(double* rw, const double* tot, int* flags) {
  constexpr int SS = S * S;
  double G[SS], R2[SS], R1[SS], Tn[SS];
  for (int a = 0; a < S; ++a)
    for (int b = 0; b < S; ++b) G[a * S + b] = 0.5 * (tot[a * S + b] + tot[b * S + a]);
  if (!chol_upper<S>(G, R2)) {
    atomicOr(flags, all_finite<S>(G, SS) ? DERR_BREAKDOWN : DERR_NONFINITE);
    for (int k = 0; k < SS; ++k) R2[k] = (k % (S + 1) == 0) ? 1.0 : 0.0;
  }
  for (int k = 0; k < SS; ++k) R1[k] = rw[REC_R1 * SS + k];
  matmul<S>(R2, R1, Tn);
  for (int k = 0; k < SS; ++k) {
    rw[REC_R2 * SS + k] = R2[k];
    rw[REC_TNEXT * SS + k] = Tn[k];
  }
  if (!all_finite<S>(Tn, SS)) atomicOr(flags, DERR_NONFINITE);
}

// rows of W, V_j and V_{j-1} (zero without a previous block)
template <typename T, int S>
__device__ __forceinline__ void load3(const T* __restrict__ W, const T* __restrict__ Vc, int64_t ldc,
                                      const T* __restrict__ Vp, int64_t ldp, bool hp, int64_t row, T (&w)[S],
                                      T (&q)[S], T (&p)[S]) {
  load_row<S>(W, (int64_t)S, row, w);
  load_row<S>(Vc, ldc, row, q);
  if (hp) load_row<S>(Vp, ldp, row, p);
  else {
#pragma unroll
    for (int a = 0; a < S; ++a) p[a] = T(0);
  }
}

// ---- sweep kernels -----------------------------------------------------------
struct SweepArgs {
  OpDev op;
  int j;           // iteration index (1-based); its log record is op.log + j*LOG_NREC*S*S
  int has_prev;    // j > 1
  const void* Vp;  // V_{j-1}
  const void* Vc;  // V_j
  void* Vn;        // V_{j+1} (S4) or W (S1)
  int64_t ldp, ldc, ldn;
  int* flags;
};

// S1: SpMM + first MGS projections
template <typename T, int S>
__global__ void __launch_bounds__(kThreads, MinBlocks<T>::value) k_spmm_proj(SweepArgs g) {
  using Acc = typename AccT<T>::type;
  constexpr int NACC = 3 * S * S;
  Acc acc[NACC];
#pragma unroll
  for (int k = 0; k < NACC; ++k) acc[k] = Acc(0);
  const T* Vp = static_cast<const T*>(g.Vp);
  const T* Vc = static_cast<const T*>(g.Vc);
  T* W = static_cast<T*>(g.Vn);
  const int lane = threadIdx.x & 31;
  const int64_t gwarp = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
  const int64_t nwarps = (int64_t)gridDim.x * kWarps;
  // the next slice's metadata is loaded one slice ahead, so a slice starts with its column
  // indices and values instead of a round trip for its offset and width
  int64_t nptr = 0;
  int nwid = 0;
  if (gwarp < g.op.nslices) {
    nptr = g.op.slice_ptr[gwarp];
    nwid = g.op.slice_w[gwarp];
  }
  for (int64_t sl = gwarp; sl < g.op.nslices; sl += nwarps) {
    const int64_t cptr = nptr;
    const int cwid = nwid;
    if (sl + nwarps < g.op.nslices) {
      nptr = g.op.slice_ptr[sl + nwarps];
      nwid = g.op.slice_w[sl + nwarps];
    }
    const int64_t rs = sl * LYAP_SLICE + lane;
    const int64_t row = g.op.perm ? (rs < g.op.n ? (int64_t)g.op.perm[rs] : g.op.n) : rs;
    if (row < g.op.n) {
      T w[S];
      sell_row_at<T, S>(g.op, cptr, cwid, lane, Vc, g.ldc, w);
      store_row<S>(W, (int64_t)S, row, w);
      T q[S], p[S];
      load_row<S>(Vc, g.ldc, row, q);
      if (g.has_prev) load_row<S>(Vp, g.ldp, row, p);
      else {
#pragma unroll
        for (int a = 0; a < S; ++a) p[a] = T(0);
      }
#pragma unroll
      for (int a = 0; a < S; ++a)
#pragma unroll
        for (int b = 0; b < S; ++b) {
          acc[a * S + b] = fma((Acc)p[a], (Acc)w[b], acc[a * S + b]);
          acc[S * S + a * S + b] = fma((Acc)q[a], (Acc)w[b], acc[S * S + a * S + b]);
          acc[2 * S * S + a * S + b] = fma((Acc)q[a], (Acc)p[b], acc[2 * S * S + a * S + b]);
        }
    }
  }
  __shared__ double tot[NACC];
  __shared__ double scratch[kWarps * NACC];
  if (!reduce_partials<Acc, NACC>(acc, g.op.partials, g.op.counter, tot, scratch, blockIdx.x, gridDim.x)) return;
  if (threadIdx.x == 0) finalize_s1<S>(g.op.log + (size_t)g.j * LOG_NREC * S * S, tot, g.has_prev, g.flags);
}

// S2: second MGS projections + first Gram
template <typename T, int S>
__global__ void __launch_bounds__(kThreads, MinBlocks<T>::value) k_proj2_gram1(SweepArgs g) {
  using Acc = typename AccT<T>::type;
  constexpr int SS = S * S;
  constexpr int NSYM = S * (S + 1) / 2;  // upper triangle of the Gram block
  constexpr int NACC = 2 * SS + NSYM;
  __shared__ Coefs<T, S> co;
  const double* rec = g.op.log + (size_t)g.j * LOG_NREC * SS;
  load_coefs<T, S>(co, rec, 1);
  Acc acc[NACC];
#pragma unroll
  for (int k = 0; k < NACC; ++k) acc[k] = Acc(0);
  const T* Vp = static_cast<const T*>(g.Vp);
  const T* Vc = static_cast<const T*>(g.Vc);
  const T* W = static_cast<const T*>(g.Vn);
  const bool hp = g.has_prev;
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < g.op.n; row += (int64_t)gridDim.x * blockDim.x) {
    T w[S], p[S], q[S];
    load_row<S>(W, (int64_t)S, row, w);
    load_row<S>(Vc, g.ldc, row, q);
    if (hp) load_row<S>(Vp, g.ldp, row, p);
    else {
#pragma unroll
      for (int a = 0; a < S; ++a) p[a] = T(0);
    }
    mgs_row<T, S>(p, q, co.ap, co.ad, w, hp);
#pragma unroll
    for (int a = 0; a < S; ++a)
#pragma unroll
      for (int b = 0; b < S; ++b) {
        acc[a * S + b] = fma((Acc)p[a], (Acc)w[b], acc[a * S + b]);
        acc[SS + a * S + b] = fma((Acc)q[a], (Acc)w[b], acc[SS + a * S + b]);
      }
    int e = 2 * SS;
#pragma unroll
    for (int a = 0; a < S; ++a)
#pragma unroll
      for (int b = a; b < S; ++b, ++e) acc[e] = fma((Acc)w[a], (Acc)w[b], acc[e]);
  }
  __shared__ double tot[NACC];
  __shared__ double scratch[kWarps * NACC];
  if (!reduce_partials<Acc, NACC>(acc, g.op.partials, g.op.counter, tot, scratch, blockIdx.x, gridDim.x)) return;
  if (threadIdx.x == 0) finalize_s2<S>(g.op.log + (size_t)g.j * LOG_NREC * SS, tot, hp, g.flags);
}

// S3: second Gram (CholQR2's second pass)
template <typename T, int S>
__global__ void __launch_bounds__(kThreads, MinBlocks<T>::value) k_gram2(SweepArgs g) {
  using Acc = typename AccT<T>::type;
  constexpr int SS = S * S;
  constexpr int NACC = SS;
  __shared__ Coefs<T, S> co;
  const double* rec = g.op.log + (size_t)g.j * LOG_NREC * SS;
  load_coefs<T, S>(co, rec, 2);
  Acc acc[NACC];
#pragma unroll
  for (int k = 0; k < NACC; ++k) acc[k] = Acc(0);
  const T* Vp = static_cast<const T*>(g.Vp);
  const T* Vc = static_cast<const T*>(g.Vc);
  const T* W = static_cast<const T*>(g.Vn);
  const bool hp = g.has_prev;
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < g.op.n; row += (int64_t)gridDim.x * blockDim.x) {
    T w[S], p[S], q[S];
    load3<T, S>(W, Vc, g.ldc, Vp, g.ldp, hp, row, w, q, p);
    mgs_row<T, S>(p, q, co.tp, co.td, w, hp);
    trsm_row<T, S>(co.r1, co.r1i, w);
#pragma unroll
    for (int a = 0; a < S; ++a)
#pragma unroll
      for (int b = 0; b < S; ++b) acc[a * S + b] = fma((Acc)w[a], (Acc)w[b], acc[a * S + b]);
  }
  __shared__ double tot[NACC];
  __shared__ double scratch[kWarps * NACC];
  if (!reduce_partials<Acc, NACC>(acc, g.op.partials, g.op.counter, tot, scratch, blockIdx.x, gridDim.x)) return;
  if (threadIdx.x == 0) finalize_s3<S>(g.op.log + (size_t)g.j * LOG_NREC * SS, tot, g.flags);
}

// S4: write V_{j+1}
template <typename T, int S>
__global__ void __launch_bounds__(kThreads, MinBlocks<T>::value) k_write_next(SweepArgs g) {
  constexpr int SS = S * S;
  __shared__ Coefs<T, S> co;
  const double* rec = g.op.log + (size_t)g.j * LOG_NREC * SS;
  load_coefs<T, S>(co, rec, 3);
  const T* Vp = static_cast<const T*>(g.Vp);
  const T* Vc = static_cast<const T*>(g.Vc);
  const T* W = static_cast<const T*>(g.op.W);
  T* Vn = static_cast<T*>(g.Vn);
  const bool hp = g.has_prev;
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < g.op.n; row += (int64_t)gridDim.x * blockDim.x) {
    T w[S], p[S], q[S];
    load3<T, S>(W, Vc, g.ldc, Vp, g.ldp, hp, row, w, q, p);
    next_row<T, S>(co, p, q, w, hp);
    store_row<S>(Vn, g.ldn, row, w);
  }
}

// Second pass: V_{j+1} = recipe(A V_j, V_{j-1}, V_j) in one sweep (no reductions).
// Same SpMM and row recipe as pass 1, hence the same bits.
template <typename T, int S>
__global__ void __launch_bounds__(kThreads, MinBlocks<T>::value) k_pass2(SweepArgs g) {
  constexpr int SS = S * S;
  __shared__ Coefs<T, S> co;
  const double* rec = g.op.log + (size_t)g.j * LOG_NREC * SS;
  load_coefs<T, S>(co, rec, 3);
  const T* Vp = static_cast<const T*>(g.Vp);
  const T* Vc = static_cast<const T*>(g.Vc);
  T* Vn = static_cast<T*>(g.Vn);
  const bool hp = g.has_prev;
  const int lane = threadIdx.x & 31;
  const int64_t gwarp = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
  const int64_t nwarps = (int64_t)gridDim.x * kWarps;
  for (int64_t sl = gwarp; sl < g.op.nslices; sl += nwarps) {
    const int64_t rs = sl * LYAP_SLICE + lane;
    const int64_t row = g.op.perm ? (rs < g.op.n ? (int64_t)g.op.perm[rs] : g.op.n) : rs;
    if (row < g.op.n) {
      T w[S], p[S], q[S];
      sell_row<T, S>(g.op, sl, lane, Vc, g.ldc, w);
      load_row<S>(Vc, g.ldc, row, q);
      if (hp) load_row<S>(Vp, g.ldp, row, p);
      else {
#pragma unroll
        for (int a = 0; a < S; ++a) p[a] = T(0);
      }
      next_row<T, S>(co, p, q, w, hp);
      store_row<S>(Vn, g.ldn, row, w);
    }
  }
}

// ---- initial block: C = V_1 gamma by CholQR2 on the fp64 right-hand side --------
// log record 0 holds R1, R2, gamma = R2 R1 (in REC_TNEXT) and beta = ||C||_F in REC_TDIAG[0].
template <int S>
__global__ void __launch_bounds__(kThreads) k_init_gram(SweepArgs g, int stage) {
  constexpr int SS = S * S;
  __shared__ double r1[S][S];
  __shared__ double r1i[S];
  double* rec = g.op.log;
  if (stage == 2) {
    for (int k = threadIdx.x; k < SS; k += blockDim.x) r1[k / S][k % S] = rec[REC_R1 * SS + k];
    for (int b = threadIdx.x; b < S; b += blockDim.x) r1i[b] = 1.0 / rec[REC_R1 * SS + b * S + b];
    __syncthreads();
  }
  double acc[SS];
#pragma unroll
  for (int k = 0; k < SS; ++k) acc[k] = 0.0;
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < g.op.n; row += (int64_t)gridDim.x * blockDim.x) {
    double w[S];
    load_row<S>(g.op.C, (int64_t)S, row, w);
    if (stage == 2) trsm_row<double, S>(r1, r1i, w);
#pragma unroll
    for (int a = 0; a < S; ++a)
#pragma unroll
      for (int b = 0; b < S; ++b) acc[a * S + b] = fma(w[a], w[b], acc[a * S + b]);
  }
  __shared__ double tot[SS];
  __shared__ double scratch[kWarps * SS];
  if (!reduce_partials<double, SS>(acc, g.op.partials, g.op.counter, tot, scratch, blockIdx.x, gridDim.x)) return;
  if (threadIdx.x == 0) {
    double G[SS], R[SS];
    for (int a = 0; a < S; ++a)
      for (int b = 0; b < S; ++b) G[a * S + b] = 0.5 * (tot[a * S + b] + tot[b * S + a]);
    const bool finite = all_finite<S>(G, SS);
    if (!finite) atomicOr(g.flags, DERR_NONFINITE);
    if (!chol_upper<S>(G, R)) {
      if (finite) atomicOr(g.flags, DERR_BREAKDOWN);
      for (int k = 0; k < SS; ++k) R[k] = (k % (S + 1) == 0) ? 1.0 : 0.0;
    }
    if (stage == 1) {
      double tr = 0.0;
      for (int a = 0; a < S; ++a) tr += G[a * S + a];
      for (int k = 0; k < SS; ++k) rec[REC_R1 * SS + k] = R[k];
      rec[REC_TDIAG * SS] = sqrt(tr);
    } else {
      double R1[SS], Gm[SS];
      for (int k = 0; k < SS; ++k) R1[k] = rec[REC_R1 * SS + k];
      matmul<S>(R, R1, Gm);
      for (int k = 0; k < SS; ++k) {
        rec[REC_R2 * SS + k] = R[k];
        rec[REC_TNEXT * SS + k] = Gm[k];
      }
    }
  }
}

template <typename T, int S>
__global__ void __launch_bounds__(kThreads) k_init_write(SweepArgs g) {
  constexpr int SS = S * S;
  __shared__ double r1[S][S], r2[S][S];
  __shared__ double r1i[S], r2i[S];
  const double* rec = g.op.log;
  for (int k = threadIdx.x; k < SS; k += blockDim.x) {
    r1[k / S][k % S] = rec[REC_R1 * SS + k];
    r2[k / S][k % S] = rec[REC_R2 * SS + k];
  }
  for (int b = threadIdx.x; b < S; b += blockDim.x) {
    r1i[b] = 1.0 / rec[REC_R1 * SS + b * S + b];
    r2i[b] = 1.0 / rec[REC_R2 * SS + b * S + b];
  }
  __syncthreads();
  T* Vn = static_cast<T*>(g.Vn);
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < g.op.n; row += (int64_t)gridDim.x * blockDim.x) {
    double w[S];
    load_row<S>(g.op.C, (int64_t)S, row, w);
    trsm_row<double, S>(r1, r1i, w);
    trsm_row<double, S>(r2, r2i, w);
    T v[S];
#pragma unroll
    for (int a = 0; a < S; ++a) v[a] = T(w[a]);
    store_row<S>(Vn, g.ldn, row, v);
  }
}


// ---- batched sweeps: many independent instances of one block size per launch ---------
// A persistent grid walks a list of row tiles (instance, rows [lo, hi)); each tile's CTA
// reduces its s x s partial sums into the instance's partials slot `local`, and the last tile
// of an instance to finish (per-instance counter) finalises that instance's coefficients,
// exactly as the last CTA does for a single instance.  Instances that stopped are skipped.
struct BatchArgs {
  const BInst* inst;
  const BTile* tiles;
  int ntiles;
};

template <typename T, int S>
__device__ __forceinline__ void ring(const BInst& in, int j, const T*& Vp, const T*& Vc, T*& Vn) {
  Vp = static_cast<const T*>(in.op.V[(j + 1) % 3]);
  Vc = static_cast<const T*>(in.op.V[(j + 2) % 3]);
  Vn = static_cast<T*>(in.op.V[j % 3]);
}

template <typename T, int S>
__global__ void __launch_bounds__(kThreads, MinBlocks<T>::value) kb_spmm_proj(BatchArgs b) {
  using Acc = typename AccT<T>::type;
  constexpr int NACC = 3 * S * S;
  __shared__ double tot[NACC];
  __shared__ double scratch[kWarps * NACC];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int t = blockIdx.x; t < b.ntiles; t += gridDim.x) {
    const BTile tile = b.tiles[t];
    const BInst& in = b.inst[tile.inst];
    const int j = in.step[0];
    if (!in.step[1]) continue;
    const bool hp = j > 1;
    const T *Vp, *Vc;
    T* Vn;
    ring<T, S>(in, j, Vp, Vc, Vn);
    T* W = static_cast<T*>(in.op.W);
    Acc acc[NACC];
#pragma unroll
    for (int k = 0; k < NACC; ++k) acc[k] = Acc(0);
    const int64_t s_lo = tile.lo / LYAP_SLICE, s_hi = (tile.hi + LYAP_SLICE - 1) / LYAP_SLICE;
    for (int64_t sl = s_lo + warp; sl < s_hi; sl += kWarps) {
      const int64_t row = sl * LYAP_SLICE + lane;
      if (row < in.op.n) {
        T w[S];
        sell_row<T, S>(in.op, sl, lane, Vc, (int64_t)S, w);
        store_row<S>(W, (int64_t)S, row, w);
        T q[S], p[S];
        load_row<S>(Vc, (int64_t)S, row, q);
        if (hp) load_row<S>(Vp, (int64_t)S, row, p);
        else {
#pragma unroll
          for (int a = 0; a < S; ++a) p[a] = T(0);
        }
#pragma unroll
        for (int a = 0; a < S; ++a)
#pragma unroll
          for (int c = 0; c < S; ++c) {
            acc[a * S + c] = fma((Acc)p[a], (Acc)w[c], acc[a * S + c]);
            acc[S * S + a * S + c] = fma((Acc)q[a], (Acc)w[c], acc[S * S + a * S + c]);
            acc[2 * S * S + a * S + c] = fma((Acc)q[a], (Acc)p[c], acc[2 * S * S + a * S + c]);
          }
      }
    }
    if (reduce_partials<Acc, NACC>(acc, in.op.partials, in.op.counter, tot, scratch, tile.local, in.ntiles) &&
        threadIdx.x == 0)
      finalize_s1<S>(in.op.log + (size_t)j * LOG_NREC * S * S, tot, hp, in.flags);
    __syncthreads();
  }
}

template <typename T, int S>
__global__ void __launch_bounds__(kThreads, MinBlocks<T>::value) kb_proj2_gram1(BatchArgs b) {
  using Acc = typename AccT<T>::type;
  constexpr int SS = S * S;
  constexpr int NSYM = S * (S + 1) / 2;
  constexpr int NACC = 2 * SS + NSYM;
  __shared__ Coefs<T, S> co;
  __shared__ double tot[NACC];
  __shared__ double scratch[kWarps * NACC];
  for (int t = blockIdx.x; t < b.ntiles; t += gridDim.x) {
    const BTile tile = b.tiles[t];
    const BInst& in = b.inst[tile.inst];
    const int j = in.step[0];
    if (!in.step[1]) continue;
    const bool hp = j > 1;
    const T *Vp, *Vc;
    T* Vn;
    ring<T, S>(in, j, Vp, Vc, Vn);
    const T* W = static_cast<const T*>(in.op.W);
    double* rec = in.op.log + (size_t)j * LOG_NREC * SS;
    load_coefs<T, S>(co, rec, 1);
    Acc acc[NACC];
#pragma unroll
    for (int k = 0; k < NACC; ++k) acc[k] = Acc(0);
    const int64_t hi = tile.hi < in.op.n ? tile.hi : in.op.n;
    for (int64_t row = tile.lo + threadIdx.x; row < hi; row += blockDim.x) {
      T w[S], p[S], q[S];
      load_row<S>(W, (int64_t)S, row, w);
      load_row<S>(Vc, (int64_t)S, row, q);
      if (hp) load_row<S>(Vp, (int64_t)S, row, p);
      else {
#pragma unroll
        for (int a = 0; a < S; ++a) p[a] = T(0);
      }
      mgs_row<T, S>(p, q, co.ap, co.ad, w, hp);
#pragma unroll
      for (int a = 0; a < S; ++a)
#pragma unroll
        for (int c = 0; c < S; ++c) {
          acc[a * S + c] = fma((Acc)p[a], (Acc)w[c], acc[a * S + c]);
          acc[SS + a * S + c] = fma((Acc)q[a], (Acc)w[c], acc[SS + a * S + c]);
        }
      int e = 2 * SS;
#pragma unroll
      for (int a = 0; a < S; ++a)
#pragma unroll
        for (int c = a; c < S; ++c, ++e) acc[e] = fma((Acc)w[a], (Acc)w[c], acc[e]);
    }
    if (reduce_partials<Acc, NACC>(acc, in.op.partials, in.op.counter, tot, scratch, tile.local, in.ntiles) &&
        threadIdx.x == 0)
      finalize_s2<S>(rec, tot, hp, in.flags);
    __syncthreads();
  }
}

template <typename T, int S>
__global__ void __launch_bounds__(kThreads, MinBlocks<T>::value) kb_gram2(BatchArgs b) {
  using Acc = typename AccT<T>::type;
  constexpr int SS = S * S;
  constexpr int NACC = SS;
  __shared__ Coefs<T, S> co;
  __shared__ double tot[NACC];
  __shared__ double scratch[kWarps * NACC];
  for (int t = blockIdx.x; t < b.ntiles; t += gridDim.x) {
    const BTile tile = b.tiles[t];
    const BInst& in = b.inst[tile.inst];
    const int j = in.step[0];
    if (!in.step[1]) continue;
    const bool hp = j > 1;
    const T *Vp, *Vc;
    T* Vn;
    ring<T, S>(in, j, Vp, Vc, Vn);
    const T* W = static_cast<const T*>(in.op.W);
    double* rec = in.op.log + (size_t)j * LOG_NREC * SS;
    load_coefs<T, S>(co, rec, 2);
    Acc acc[NACC];
#pragma unroll
    for (int k = 0; k < NACC; ++k) acc[k] = Acc(0);
    const int64_t hi = tile.hi < in.op.n ? tile.hi : in.op.n;
    for (int64_t row = tile.lo + threadIdx.x; row < hi; row += blockDim.x) {
      T w[S], p[S], q[S];
      load_row<S>(W, (int64_t)S, row, w);
      load_row<S>(Vc, (int64_t)S, row, q);
      if (hp) load_row<S>(Vp, (int64_t)S, row, p);
      else {
#pragma unroll
        for (int a = 0; a < S; ++a) p[a] = T(0);
      }
      mgs_row<T, S>(p, q, co.tp, co.td, w, hp);
      trsm_row<T, S>(co.r1, co.r1i, w);
#pragma unroll
      for (int a = 0; a < S; ++a)
#pragma unroll
        for (int c = 0; c < S; ++c) acc[a * S + c] = fma((Acc)w[a], (Acc)w[c], acc[a * S + c]);
    }
    if (reduce_partials<Acc, NACC>(acc, in.op.partials, in.op.counter, tot, scratch, tile.local, in.ntiles) &&
        threadIdx.x == 0)
      finalize_s3<S>(rec, tot, in.flags);
    __syncthreads();
  }
}

// writes V_{j+1}; the last tile of an instance advances its iteration counter (and stops it
// after maxit iterations)
template <typename T, int S>
__global__ void __launch_bounds__(kThreads, MinBlocks<T>::value) kb_write_next(BatchArgs b) {
  constexpr int SS = S * S;
  __shared__ Coefs<T, S> co;
  __shared__ unsigned int ticket;
  for (int t = blockIdx.x; t < b.ntiles; t += gridDim.x) {
    const BTile tile = b.tiles[t];
    const BInst& in = b.inst[tile.inst];
    const int j = in.step[0];
    if (!in.step[1]) continue;
    const bool hp = j > 1;
    const T *Vp, *Vc;
    T* Vn;
    ring<T, S>(in, j, Vp, Vc, Vn);
    const T* W = static_cast<const T*>(in.op.W);
    load_coefs<T, S>(co, in.op.log + (size_t)j * LOG_NREC * SS, 3);
    const int64_t hi = tile.hi < in.op.n ? tile.hi : in.op.n;
    for (int64_t row = tile.lo + threadIdx.x; row < hi; row += blockDim.x) {
      T w[S], p[S], q[S];
      load_row<S>(W, (int64_t)S, row, w);
      load_row<S>(Vc, (int64_t)S, row, q);
      if (hp) load_row<S>(Vp, (int64_t)S, row, p);
      else {
#pragma unroll
        for (int a = 0; a < S; ++a) p[a] = T(0);
      }
      next_row<T, S>(co, p, q, w, hp);
      store_row<S>(Vn, (int64_t)S, row, w);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      ticket = atomicAdd(in.op.counter, 1u);
      if (ticket == (unsigned int)in.ntiles - 1) {
        *in.op.counter = 0u;
        in.step[0] = j + 1;
        if (j + 1 > in.maxit) in.step[1] = 0;
      }
    }
    __syncthreads();
  }
}

template <typename T, int S>
void batch_step_impl(const BInst* d_inst, const BTile* d_tiles, int ntiles, int grid, cudaStream_t st) {
  BatchArgs b{d_inst, d_tiles, ntiles};
  kb_spmm_proj<T, S><<<grid, kThreads, 0, st>>>(b);
  kb_proj2_gram1<T, S><<<grid, kThreads, 0, st>>>(b);
  kb_gram2<T, S><<<grid, kThreads, 0, st>>>(b);
  kb_write_next<T, S><<<grid, kThreads, 0, st>>>(b);
}


// ---- fused persistent steps: the four sweeps of several iterations in one cooperative launch ----
// Every CTA owns a fixed range of SELL slices for all four sweeps, so the rows of W it computes
// in the first sweep stay in its shared memory for the other three (W never goes to DRAM).  The
// sweeps are separated by a grid barrier; after each barrier every CTA sums all CTAs' partials
// in the same fixed order, so all CTAs hold bit-identical coefficients without another barrier,
// and CTA 0 writes them to the log.  The rows of V_{j+1} come from the same row recipe as the
// second pass, which therefore still regenerates them bit for bit.
constexpr long long kSpinCycles = 2000000000LL;  // ~1 s of SM clock, then the launch gives up

struct FusedArgs {
  OpDev op;
  int j0, nsteps;
  int* flags;
  unsigned int* bar;  // [0] arrivals, [16] generation, [32] abort
  int64_t spc;        // slices per CTA
};

// grid barrier with a bounded wait: on timeout it raises DERR_TIMEOUT and tells every CTA to stop
__device__ bool grid_sync(unsigned int* bar, unsigned int nblocks, int* flags) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* gen = bar + 16;
    volatile unsigned int* stop = bar + 32;
    int ok = *stop == 0u;
    if (ok) {
      const unsigned int g = *gen;
      __threadfence();
      const unsigned int arrived = atomicAdd(bar, 1u) + 1u;
      if (arrived == nblocks) {
        atomicExch(bar, 0u);
        __threadfence();
        atomicAdd(const_cast<unsigned int*>(gen), 1u);
      } else {
        const long long t0 = clock64();
        while (*gen == g) {
          if (*stop != 0u) {
            ok = 0;
            break;
          }
          if (clock64() - t0 > kSpinCycles) {
            atomicOr(flags, DERR_TIMEOUT);
            atomicExch(const_cast<unsigned int*>(stop), 1u);
            ok = 0;
            break;
          }
        }
      }
      __threadfence();
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// this CTA's sums of the per-thread accumulators -> its slot of P, exactly as the sweeps' stage 1
template <typename Acc, int NACC>
__device__ void cta_reduce_to(Acc (&acc)[NACC], double* __restrict__ P, unsigned int G, double* __restrict__ scratch) {
  cta_partial<Acc, NACC>(acc, P, blockIdx.x, G, scratch);
  __syncthreads();
}

// tot[k] = sum over CTAs b of P[b][k], exactly as the sweeps' stage 2
template <typename Acc, int NACC>
__device__ void reduce_all(const double* __restrict__ P, unsigned int G, double* __restrict__ tot) {
  sum_slots<Acc, NACC>(P, G, tot);
}

template <typename T, int S>
__global__ void __launch_bounds__(kThreads, MinBlocks<T>::value) k_fused_steps(FusedArgs g) {
  using Acc = typename AccT<T>::type;
  constexpr int SS = S * S;
  constexpr int NSYM = S * (S + 1) / 2;
  constexpr int N1 = 3 * SS, N2 = 2 * SS + NSYM, N3 = SS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Ws = reinterpret_cast<T*>(smem_raw);  // this CTA's rows of W, S values per row
  __shared__ Coefs<T, S> co;
  __shared__ double tot[N1];
  __shared__ double scratch[kWarps * N1];
  __shared__ double rec[LOG_NREC * SS];
  __shared__ int dummy_flags;
  const OpDev& op = g.op;
  const unsigned int G = gridDim.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t s_lo = (int64_t)blockIdx.x * g.spc;
  const int64_t s_hi = s_lo + g.spc < op.nslices ? s_lo + g.spc : op.nslices;
  const int64_t r_lo = s_lo * LYAP_SLICE;
  const int64_t r_hi = s_hi * LYAP_SLICE < op.n ? s_hi * LYAP_SLICE : op.n;
  double* P1 = op.partials;
  double* P2 = P1 + (size_t)G * N1;
  double* P3 = P2 + (size_t)G * N2;
  int* fl = blockIdx.x == 0 ? g.flags : &dummy_flags;
  for (int step = 0; step < g.nsteps; ++step) {
    const int j = g.j0 + step;
    const bool hp = j > 1;
    const T* Vp = static_cast<const T*>(op.V[(j + 1) % 3]);
    const T* Vc = static_cast<const T*>(op.V[(j + 2) % 3]);
    T* Vn = static_cast<T*>(op.V[j % 3]);
    // S1: W = A V_j (own slices, kept in shared memory) and the first projections
    {
      Acc acc[N1];
#pragma unroll
      for (int k = 0; k < N1; ++k) acc[k] = Acc(0);
      for (int64_t sl = s_lo + warp; sl < s_hi; sl += kWarps) {
        const int64_t row = sl * LYAP_SLICE + lane;
        if (row < op.n) {
          T w[S];
          sell_row_cg<T, S>(op, sl, lane, Vc, (int64_t)S, w);
#pragma unroll
          for (int a = 0; a < S; ++a) Ws[(row - r_lo) * S + a] = w[a];
          T q[S], p[S];
          load_row_cg<S>(Vc, (int64_t)S, row, q);
          if (hp) load_row_cg<S>(Vp, (int64_t)S, row, p);
          else {
#pragma unroll
            for (int a = 0; a < S; ++a) p[a] = T(0);
          }
#pragma unroll
          for (int a = 0; a < S; ++a)
#pragma unroll
            for (int c = 0; c < S; ++c) {
              acc[a * S + c] = fma((Acc)p[a], (Acc)w[c], acc[a * S + c]);
              acc[SS + a * S + c] = fma((Acc)q[a], (Acc)w[c], acc[SS + a * S + c]);
              acc[2 * SS + a * S + c] = fma((Acc)q[a], (Acc)p[c], acc[2 * SS + a * S + c]);
            }
        }
      }
      cta_reduce_to<Acc, N1>(acc, P1, G, scratch);
    }
    if (!grid_sync(g.bar, G, g.flags)) return;
    reduce_all<Acc, N1>(P1, G, tot);
    if (threadIdx.x == 0) finalize_s1<S>(rec, tot, hp, fl);
    __syncthreads();
    load_coefs<T, S>(co, rec, 1);
    // S2: second projections and the first Gram matrix
    {
      Acc acc[N2];
#pragma unroll
      for (int k = 0; k < N2; ++k) acc[k] = Acc(0);
      for (int64_t row = r_lo + threadIdx.x; row < r_hi; row += blockDim.x) {
        T w[S], p[S], q[S];
#pragma unroll
        for (int a = 0; a < S; ++a) w[a] = Ws[(row - r_lo) * S + a];
        load_row_cg<S>(Vc, (int64_t)S, row, q);
        if (hp) load_row_cg<S>(Vp, (int64_t)S, row, p);
        else {
#pragma unroll
          for (int a = 0; a < S; ++a) p[a] = T(0);
        }
        mgs_row<T, S>(p, q, co.ap, co.ad, w, hp);
#pragma unroll
        for (int a = 0; a < S; ++a)
#pragma unroll
          for (int c = 0; c < S; ++c) {
            acc[a * S + c] = fma((Acc)p[a], (Acc)w[c], acc[a * S + c]);
            acc[SS + a * S + c] = fma((Acc)q[a], (Acc)w[c], acc[SS + a * S + c]);
          }
        int e = 2 * SS;
#pragma unroll
        for (int a = 0; a < S; ++a)
#pragma unroll
          for (int c = a; c < S; ++c, ++e) acc[e] = fma((Acc)w[a], (Acc)w[c], acc[e]);
      }
      cta_reduce_to<Acc, N2>(acc, P2, G, scratch);
    }
    if (!grid_sync(g.bar, G, g.flags)) return;
    reduce_all<Acc, N2>(P2, G, tot);
    if (threadIdx.x == 0) finalize_s2<S>(rec, tot, hp, fl);
    __syncthreads();
    load_coefs<T, S>(co, rec, 2);
    // S3: second Gram matrix (CholQR2)
    {
      Acc acc[N3];
#pragma unroll
      for (int k = 0; k < N3; ++k) acc[k] = Acc(0);
      for (int64_t row = r_lo + threadIdx.x; row < r_hi; row += blockDim.x) {
        T w[S], p[S], q[S];
#pragma unroll
        for (int a = 0; a < S; ++a) w[a] = Ws[(row - r_lo) * S + a];
        load_row_cg<S>(Vc, (int64_t)S, row, q);
        if (hp) load_row_cg<S>(Vp, (int64_t)S, row, p);
        else {
#pragma unroll
          for (int a = 0; a < S; ++a) p[a] = T(0);
        }
        mgs_row<T, S>(p, q, co.tp, co.td, w, hp);
        trsm_row<T, S>(co.r1, co.r1i, w);
#pragma unroll
        for (int a = 0; a < S; ++a)
#pragma unroll
          for (int c = 0; c < S; ++c) acc[a * S + c] = fma((Acc)w[a], (Acc)w[c], acc[a * S + c]);
      }
      cta_reduce_to<Acc, N3>(acc, P3, G, scratch);
    }
    if (!grid_sync(g.bar, G, g.flags)) return;
    reduce_all<Acc, N3>(P3, G, tot);
    if (threadIdx.x == 0) finalize_s3<S>(rec, tot, fl);
    __syncthreads();
    load_coefs<T, S>(co, rec, 3);
    // S4: V_{j+1} for the own rows; CTA 0 logs the iteration's coefficients
    for (int64_t row = r_lo + threadIdx.x; row < r_hi; row += blockDim.x) {
      T w[S], p[S], q[S];
#pragma unroll
      for (int a = 0; a < S; ++a) w[a] = Ws[(row - r_lo) * S + a];
      load_row_cg<S>(Vc, (int64_t)S, row, q);
      if (hp) load_row_cg<S>(Vp, (int64_t)S, row, p);
      else {
#pragma unroll
        for (int a = 0; a < S; ++a) p[a] = T(0);
      }
      next_row<T, S>(co, p, q, w, hp);
      store_row<S>(Vn, (int64_t)S, row, w);
    }
    if (blockIdx.x == 0)
      for (int k = threadIdx.x; k < LOG_NREC * SS; k += blockDim.x) op.log[(size_t)j * LOG_NREC * SS + k] = rec[k];
    if (!grid_sync(g.bar, G, g.flags)) return;
  }
}

template <typename T, int S>
int fused_impl(OpDev& op, int j0, int nsteps, int* flags, cudaStream_t st) {
  if (op.perm != nullptr || S > 4) return 0;  // s = 8 would spill its accumulators
  int dev = 0, sms = 0, coop = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (!coop || sms <= 0) return 0;
  const void* fn = (const void*)k_fused_steps<T, S>;
  // shared memory for W rows: try the grid that gives every SM MinBlocks CTAs first
  for (int bps = MinBlocks<T>::value; bps >= 1; --bps) {
    const int G = std::min(sms * bps, kMaxSweepGrid);
    const int64_t spc = (op.nslices + G - 1) / G;
    const size_t smem = (size_t)spc * LYAP_SLICE * S * sizeof(T);
    if (smem > (size_t)160 * 1024) continue;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) continue;
    int fit = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, fn, kThreads, smem) != cudaSuccess || fit < bps) continue;
    FusedArgs a;
    a.op = op;
    a.j0 = j0;
    a.nsteps = nsteps;
    a.flags = flags;
    a.bar = op.counter + 16;
    a.spc = spc;
    void* args[] = {&a};
    if (cudaMemsetAsync(op.counter + 48, 0, sizeof(unsigned int), st) != cudaSuccess) return 0;
    if (cudaLaunchCooperativeKernel(fn, dim3(G), dim3(kThreads), args, smem, st) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    return 1;
  }
  return 0;
}

// ---- dispatch ---------------------------------------------------------------
template <typename T, int S>
void step_impl(OpDev& op, int grid, int j, int* flags, cudaStream_t st) {
  SweepArgs g;
  g.op = op;
  g.j = j;
  g.has_prev = j > 1;
  g.Vp = op.V[(j + 1) % 3];  // V_{j-1}
  g.Vc = op.V[(j + 2) % 3];  // V_j   (V_1 lives in V[0])
  g.ldp = g.ldc = S;
  g.flags = flags;
  g.Vn = op.W;
  g.ldn = S;
  k_spmm_proj<T, S><<<grid, kThreads, 0, st>>>(g);
  k_proj2_gram1<T, S><<<grid, kThreads, 0, st>>>(g);
  k_gram2<T, S><<<grid, kThreads, 0, st>>>(g);
  g.Vn = op.V[j % 3];        // V_{j+1}
  k_write_next<T, S><<<grid, kThreads, 0, st>>>(g);
}

template <typename T, int S>
void init_impl(OpDev& op, int grid, int* flags, cudaStream_t st) {
  SweepArgs g;
  g.op = op;
  g.j = 0;
  g.has_prev = 0;
  g.flags = flags;
  g.Vn = op.V[0];
  g.ldn = S;
  k_init_gram<S><<<grid, kThreads, 0, st>>>(g, 1);
  k_init_gram<S><<<grid, kThreads, 0, st>>>(g, 2);
  k_init_write<T, S><<<grid, kThreads, 0, st>>>(g);
}

template <typename T, int S>
void pass2_impl(OpDev& op, int grid, int j, const void* vp, int64_t ldp, const void* vc, int64_t ldc, void* vn,
                int64_t ldn, cudaStream_t st) {
  SweepArgs g;
  g.op = op;
  g.j = j;
  g.has_prev = j > 1;
  g.Vp = vp;
  g.Vc = vc;
  g.Vn = vn;
  g.ldp = ldp;
  g.ldc = ldc;
  g.ldn = ldn;
  g.flags = nullptr;
  k_pass2<T, S><<<grid, kThreads, 0, st>>>(g);
}

template <typename T>
void init_T(OpDev& op, int s, int grid, int* flags, cudaStream_t st) {
  switch (s) {
    case 1: init_impl<T, 1>(op, grid, flags, st); break;
    case 2: init_impl<T, 2>(op, grid, flags, st); break;
    case 3: init_impl<T, 3>(op, grid, flags, st); break;
    case 4: init_impl<T, 4>(op, grid, flags, st); break;
    case 8: init_impl<T, 8>(op, grid, flags, st); break;
  }
}
template <typename T>
void step_T(OpDev& op, int s, int grid, int j, int* flags, cudaStream_t st) {
  switch (s) {
    case 1: step_impl<T, 1>(op, grid, j, flags, st); break;
    case 2: step_impl<T, 2>(op, grid, j, flags, st); break;
    case 3: step_impl<T, 3>(op, grid, j, flags, st); break;
    case 4: step_impl<T, 4>(op, grid, j, flags, st); break;
    case 8: step_impl<T, 8>(op, grid, j, flags, st); break;
  }
}
template <typename T>
void pass2_T(OpDev& op, int s, int grid, int j, const void* vp, int64_t ldp, const void* vc, int64_t ldc, void* vn,
             int64_t ldn, cudaStream_t st) {
  switch (s) {
    case 1: pass2_impl<T, 1>(op, grid, j, vp, ldp, vc, ldc, vn, ldn, st); break;
    case 2: pass2_impl<T, 2>(op, grid, j, vp, ldp, vc, ldc, vn, ldn, st); break;
    case 3: pass2_impl<T, 3>(op, grid, j, vp, ldp, vc, ldc, vn, ldn, st); break;
    case 4: pass2_impl<T, 4>(op, grid, j, vp, ldp, vc, ldc, vn, ldn, st); break;
    case 8: pass2_impl<T, 8>(op, grid, j, vp, ldp, vc, ldc, vn, ldn, st); break;
  }
}

}  // namespace

int max_nacc(int s) { return 3 * s * s; }

// CTAs of the sweep kernels that fit on one SM together (the smallest over the four)
int sweep_blocks_per_sm(int s, int bulk_f32) {
  int best = 1 << 30;
  auto q = [&](const void* f) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, f, kThreads, 0) == cudaSuccess && b > 0) best = std::min(best, b);
  };
#define LYAP_OCC(TT, SS_)                                                                    \
  q((const void*)k_spmm_proj<TT, SS_>); q((const void*)k_proj2_gram1<TT, SS_>);           \
  q((const void*)k_gram2<TT, SS_>); q((const void*)k_write_next<TT, SS_>)
  if (bulk_f32) {
    switch (s) { case 1: LYAP_OCC(float, 1); break; case 2: LYAP_OCC(float, 2); break; case 3: LYAP_OCC(float, 3); break;
                 case 4: LYAP_OCC(float, 4); break; case 8: LYAP_OCC(float, 8); break; }
  } else {
    switch (s) { case 1: LYAP_OCC(double, 1); break; case 2: LYAP_OCC(double, 2); break; case 3: LYAP_OCC(double, 3); break;
                 case 4: LYAP_OCC(double, 4); break; case 8: LYAP_OCC(double, 8); break; }
  }
#undef LYAP_OCC
  return best == (1 << 30) ? 1 : best;
}

int launch_init_block(OpDev& op, int s, int bulk_f32, int grid, int* d_flags, cudaStream_t st) {
  if (bulk_f32) init_T<float>(op, s, grid, d_flags, st);
  else init_T<double>(op, s, grid, d_flags, st);
  return 3;
}

int launch_batch_step(int s, int bulk_f32, const BInst* d_inst, const BTile* d_tiles, int ntiles, int grid,
                      cudaStream_t st) {
#define LYAP_BS(TT, SS_) batch_step_impl<TT, SS_>(d_inst, d_tiles, ntiles, grid, st)
  if (bulk_f32) {
    switch (s) { case 1: LYAP_BS(float, 1); break; case 2: LYAP_BS(float, 2); break; case 3: LYAP_BS(float, 3); break;
                 case 4: LYAP_BS(float, 4); break; case 8: LYAP_BS(float, 8); break; default: return 0; }
  } else {
    switch (s) { case 1: LYAP_BS(double, 1); break; case 2: LYAP_BS(double, 2); break; case 3: LYAP_BS(double, 3); break;
                 case 4: LYAP_BS(double, 4); break; case 8: LYAP_BS(double, 8); break; default: return 0; }
  }
#undef LYAP_BS
  return 4;
}

// CTAs of the batched sweep kernels that fit on one SM together
int batch_blocks_per_sm(int s, int bulk_f32) {
  int best = 1 << 30;
  auto q = [&](const void* f) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, f, kThreads, 0) == cudaSuccess && b > 0) best = std::min(best, b);
  };
#define LYAP_OCC(TT, SS_)                                                                    \
  q((const void*)kb_spmm_proj<TT, SS_>); q((const void*)kb_proj2_gram1<TT, SS_>);         \
  q((const void*)kb_gram2<TT, SS_>); q((const void*)kb_write_next<TT, SS_>)
  if (bulk_f32) {
    switch (s) { case 1: LYAP_OCC(float, 1); break; case 2: LYAP_OCC(float, 2); break; case 3: LYAP_OCC(float, 3); break;
                 case 4: LYAP_OCC(float, 4); break; case 8: LYAP_OCC(float, 8); break; }
  } else {
    switch (s) { case 1: LYAP_OCC(double, 1); break; case 2: LYAP_OCC(double, 2); break; case 3: LYAP_OCC(double, 3); break;
                 case 4: LYAP_OCC(double, 4); break; case 8: LYAP_OCC(double, 8); break; }
  }
#undef LYAP_OCC
  return best == (1 << 30) ? 1 : best;
}

// nsteps iterations from j0 in one cooperative launch; returns 1, or 0 when the fused kernel
// cannot run here (the caller then uses launch_lanczos_step)
int launch_fused_steps(OpDev& op, int s, int bulk_f32, int j0, int nsteps, int* d_flags, cudaStream_t st) {
#define LYAP_FS(TT, SS_) return fused_impl<TT, SS_>(op, j0, nsteps, d_flags, st)
  if (bulk_f32) {
    switch (s) { case 1: LYAP_FS(float, 1); case 2: LYAP_FS(float, 2); case 3: LYAP_FS(float, 3);
                 case 4: LYAP_FS(float, 4); }
  } else {
    switch (s) { case 1: LYAP_FS(double, 1); case 2: LYAP_FS(double, 2); case 3: LYAP_FS(double, 3);
                 case 4: LYAP_FS(double, 4); }
  }
#undef LYAP_FS
  return 0;
}

int launch_lanczos_step(OpDev& op, int s, int bulk_f32, int grid, int j, int* d_flags, cudaStream_t st) {
  if (bulk_f32) step_T<float>(op, s, grid, j, d_flags, st);
  else step_T<double>(op, s, grid, j, d_flags, st);
  return 4;
}

// Second pass, step j: writes V_{j+1} from V_{j-1} (vp), V_j (vc).
void launch_pass2(OpDev& op, int s, int bulk_f32, int grid, int j, const void* vp, int64_t ldp, const void* vc,
                  int64_t ldc, void* vn, int64_t ldn, cudaStream_t st) {
  if (bulk_f32) pass2_T<float>(op, s, grid, j, vp, ldp, vc, ldc, vn, ldn, st);
  else pass2_T<double>(op, s, grid, j, vp, ldp, vc, ldc, vn, ldn, st);
}

// Second pass, V_1 from C with the logged CholQR2 factors of the first pass.
void launch_pass2_v1(OpDev& op, int s, int bulk_f32, int grid, void* vn, int64_t ldn, cudaStream_t st) {
  SweepArgs g;
  g.op = op;
  g.j = 0;
  g.has_prev = 0;
  g.flags = nullptr;
  g.Vn = vn;
  g.ldn = ldn;
#define LYAP_V1(TT, SS_)                                     \
  k_init_write<TT, SS_><<<grid, kThreads, 0, st>>>(g)
  if (bulk_f32) {
    switch (s) { case 1: LYAP_V1(float, 1); break; case 2: LYAP_V1(float, 2); break; case 3: LYAP_V1(float, 3); break;
                 case 4: LYAP_V1(float, 4); break; case 8: LYAP_V1(float, 8); break; }
  } else {
    switch (s) { case 1: LYAP_V1(double, 1); break; case 2: LYAP_V1(double, 2); break; case 3: LYAP_V1(double, 3); break;
                 case 4: LYAP_V1(double, 4); break; case 8: LYAP_V1(double, 8); break; }
  }
#undef LYAP_V1
}
