// Batched block Lanczos sweeps (Alg. 2 with CholQR2 normalisation): many independent instances
// of one block size per launch, four row sweeps per iteration over a list of row tiles of all
// instances, each followed by a fixed-order reduction of per-tile s x s partial sums done by the
// instance's last tile:
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
// The rows w1, w2, x are recomputed from W, V_{j-1}, V_j in every sweep instead of being stored.
// V_{j+1} is written by the same SpMM and row recipe as the second pass (step.cu), which
// therefore regenerates the instances' bases bit for bit.
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
        sell_row_at<T, S>(in.op, in.op.slice_ptr[sl], in.op.slice_w[sl], lane, Vc, (int64_t)S, w);
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


}  // namespace

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
