// Block Lanczos step of one operator (Alg. 2: block MGS done twice, then a Cholesky QR done
// twice), and the second pass of Sec. 3.3.  One step is four row sweeps, each followed by a
// fixed-order reduction of per-CTA s x s sums done by the last CTA to finish:
//
//   S1  W = A V_j (SELL-C-sigma SpMM)         sums V_{j-1}^T W, V_j^T W, V_j^T V_{j-1}
//       -> alpha_{j-1}, alpha_j (the first MGS sweep in fused form)
//   S2  w1 = W - V_{j-1} alpha_{j-1} - V_j alpha_j   sums V_{j-1}^T w1, V_j^T w1, w1^T w1
//       -> beta_{j-1}, beta_j (the second MGS sweep), R1 = chol(w2^T w2), w2 = w1 - V beta
//   S3  x = w2 R1^{-1}                         sum x^T x -> R2 = chol(x^T x), tau_{j+1,j} = R2 R1
//   S4  V_{j+1} = (W - V_{j-1} tau_{j-1,j} - V_j tau_jj) tau_{j+1,j}^{-1}
//
// Every Gram matrix is measured on the rows actually formed, so the step keeps CholQR2's
// orthogonality even when the new block is ill-conditioned (block Lanczos near a converged
// Ritz vector), which a Gram matrix formed from W^T W by cancellation does not.  The rows w1,
// w2, x are recomputed from W, V_{j-1}, V_j in every sweep instead of being stored.
//
// Three bulk number types share the code: fp64; fp32 (per-thread fp32 sums, cross-CTA sums as
// float pairs); and float pairs throughout (values, sums and row arithmetic on the fp32 pipe,
// about 48 bits, see ff.cuh).  The second pass runs the same SpMM and the row recipe of S4 from
// the logged coefficients and therefore regenerates V_{j+1} bit for bit.
#include "common.cuh"
#include "ff.cuh"

#include <math.h>

#include <algorithm>
#include <type_traits>

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

// ---- bulk number types ------------------------------------------------------------------
// V: stored element; R: a value in registers; Acc: per-thread sum; kUnroll: SELL entries
// gathered at once; kMinBlocks: CTAs per SM
struct NumD {
  using V = double;
  using R = double;
  using Acc = double;
  static constexpr int kUnroll = 8;
  static constexpr int kMinBlocks = 1;
};
struct NumF {
  using V = float;
  using R = float;
  using Acc = float;
  static constexpr int kUnroll = 8;
  static constexpr int kMinBlocks = 2;
};
#ifndef LYAP_FF_UNROLL
#define LYAP_FF_UNROLL 4
#endif
#ifndef LYAP_FF_MINB
#define LYAP_FF_MINB 1
#endif
struct NumFF {
  using V = float;  // a row of S pairs is 2S floats: the S high parts, then the S low parts
  using R = ff;
  using Acc = ff;
  static constexpr int kUnroll = LYAP_FF_UNROLL;
  static constexpr int kMinBlocks = LYAP_FF_MINB;
};

// ---- row loads and stores (row i of a block with leading dimension ld, in values) ----------
template <int S>
__device__ __forceinline__ void ld_row(const double* __restrict__ X, int64_t ld, int64_t i, double (&r)[S]) {
  const double* p = X + i * ld;
  if constexpr (S % 2 == 0) {
#pragma unroll
    for (int a = 0; a < S; a += 2) {
      const double2 v = *reinterpret_cast<const double2*>(p + a);
      r[a] = v.x;
      r[a + 1] = v.y;
    }
  } else {
#pragma unroll
    for (int a = 0; a < S; ++a) r[a] = p[a];
  }
}
template <int S>
__device__ __forceinline__ void ld_row(const float* __restrict__ X, int64_t ld, int64_t i, float (&r)[S]) {
  const float* p = X + i * ld;
  if constexpr (S % 4 == 0) {
#pragma unroll
    for (int a = 0; a < S; a += 4) {
      const float4 v = *reinterpret_cast<const float4*>(p + a);
      r[a] = v.x; r[a + 1] = v.y; r[a + 2] = v.z; r[a + 3] = v.w;
    }
  } else if constexpr (S == 2) {
    const float2 v = *reinterpret_cast<const float2*>(p);
    r[0] = v.x;
    r[1] = v.y;
  } else {
#pragma unroll
    for (int a = 0; a < S; ++a) r[a] = p[a];
  }
}
template <int S>
__device__ __forceinline__ void ld_row(const float* __restrict__ X, int64_t ld, int64_t i, ff (&r)[S]) {
  const float* p = X + 2 * i * ld;
  if constexpr (S % 4 == 0) {
#pragma unroll
    for (int a = 0; a < S; a += 4) {
      const float4 h = *reinterpret_cast<const float4*>(p + a);
      const float4 l = *reinterpret_cast<const float4*>(p + S + a);
      r[a] = ff_make(h.x, l.x); r[a + 1] = ff_make(h.y, l.y);
      r[a + 2] = ff_make(h.z, l.z); r[a + 3] = ff_make(h.w, l.w);
    }
  } else if constexpr (S == 2) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    r[0] = ff_make(v.x, v.z);
    r[1] = ff_make(v.y, v.w);
  } else {
#pragma unroll
    for (int a = 0; a < S; ++a) {
      const float2 v = make_float2(p[a], p[S + a]);
      r[a] = ff_make(v.x, v.y);
    }
  }
}
template <int S>
__device__ __forceinline__ void st_row(double* __restrict__ X, int64_t ld, int64_t i, const double (&r)[S]) {
  double* p = X + i * ld;
  if constexpr (S % 2 == 0) {
#pragma unroll
    for (int a = 0; a < S; a += 2) *reinterpret_cast<double2*>(p + a) = make_double2(r[a], r[a + 1]);
  } else {
#pragma unroll
    for (int a = 0; a < S; ++a) p[a] = r[a];
  }
}
template <int S>
__device__ __forceinline__ void st_row(float* __restrict__ X, int64_t ld, int64_t i, const float (&r)[S]) {
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
__device__ __forceinline__ void st_row(float* __restrict__ X, int64_t ld, int64_t i, const ff (&r)[S]) {
  float* p = X + 2 * i * ld;
  if constexpr (S % 4 == 0) {
#pragma unroll
    for (int a = 0; a < S; a += 4) {
      *reinterpret_cast<float4*>(p + a) = make_float4(r[a].hi, r[a + 1].hi, r[a + 2].hi, r[a + 3].hi);
      *reinterpret_cast<float4*>(p + S + a) = make_float4(r[a].lo, r[a + 1].lo, r[a + 2].lo, r[a + 3].lo);
    }
  } else if constexpr (S == 2) {
    *reinterpret_cast<float4*>(p) = make_float4(r[0].hi, r[1].hi, r[0].lo, r[1].lo);
  } else {
#pragma unroll
    for (int a = 0; a < S; ++a) {
      p[a] = r[a].hi;
      p[S + a] = r[a].lo;
    }
  }
}

// ---- scalar arithmetic of the three types --------------------------------------------------
__device__ __forceinline__ void zero(double& x) { x = 0.0; }
__device__ __forceinline__ void zero(float& x) { x = 0.f; }
__device__ __forceinline__ void zero(ff& x) { x = ff_make(0.f, 0.f); }
// w += a x, a an operator entry
__device__ __forceinline__ void acc_a(double& w, double a, double x) { w = fma(a, x, w); }
__device__ __forceinline__ void acc_a(float& w, float a, float x) { w = fmaf(a, x, w); }
__device__ __forceinline__ void acc_a(ff& w, float a, ff x) { ff_acc(w, a, x); }
__device__ __forceinline__ void acc_a(ff& w, float2 a, ff x) { ff_acc(w, ff_make(a.x, a.y), x); }
// g += x y (per-thread sums)
__device__ __forceinline__ void gram(double& g, double x, double y) { g = fma(x, y, g); }
__device__ __forceinline__ void gram(float& g, float x, float y) { g = fmaf(x, y, g); }
__device__ __forceinline__ void gram(ff& g, ff x, ff y) { ff_acc(g, x, y); }
// w -= x c
__device__ __forceinline__ void msub(double& w, double x, double c) { w = fma(-x, c, w); }
__device__ __forceinline__ void msub(float& w, float x, float c) { w = fmaf(-x, c, w); }
__device__ __forceinline__ void msub(ff& w, ff x, ff c) { ff_sub_acc(w, x, c); }
// x c
__device__ __forceinline__ double mulc(double x, double c) { return x * c; }
__device__ __forceinline__ float mulc(float x, float c) { return x * c; }
__device__ __forceinline__ ff mulc(ff x, ff c) { return ff_mul(ff_norm(x), c); }
// the end of an accumulation (float pairs are renormalised)
__device__ __forceinline__ void settle(double&) {}
__device__ __forceinline__ void settle(float&) {}
__device__ __forceinline__ void settle(ff& x) { x = ff_norm(x); }
// a logged fp64 coefficient in the row arithmetic's type
template <typename R>
__device__ __forceinline__ R coef(double d);
template <>
__device__ __forceinline__ double coef<double>(double d) { return d; }
template <>
__device__ __forceinline__ float coef<float>(double d) { return (float)d; }
template <>
__device__ __forceinline__ ff coef<ff>(double d) { return ff_from_double(d); }

// ---- SELL-C-sigma row product: w = (A V)[row] ---------------------------------------------
// Entries are taken kUnroll at a time: first all column indices and values, then the gathers
// of V rows, then the products, so a row has kUnroll independent gathers in flight.  The
// summation order is the row's entry order in every case (identical bits in both passes).
template <class Num, typename AV, int S>
__device__ __forceinline__ void spmm_row(const OpDev& op, int64_t sptr, int width, int lane,
                                         const typename Num::V* __restrict__ Vc, int64_t ldc,
                                         typename Num::R (&w)[S]) {
  using R = typename Num::R;
  constexpr int U = Num::kUnroll;
#pragma unroll
  for (int a = 0; a < S; ++a) zero(w[a]);
  const int64_t base = sptr + lane;
  const AV* __restrict__ val = static_cast<const AV*>(op.sell_val);
  for (int j0 = 0; j0 < width; j0 += U) {
    int32_t c[U];
    AV v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const bool in = j0 + u < width;
      const int64_t e = base + (int64_t)(in ? j0 + u : 0) * LYAP_SLICE;
      c[u] = __ldg(op.sell_col + e);
      if (in) v[u] = __ldg(val + e);
      else v[u] = AV{};
    }
    R x[U][S];
#pragma unroll
    for (int u = 0; u < U; ++u) ld_row<S>(Vc, ldc, c[u], x[u]);
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int a = 0; a < S; ++a) acc_a(w[a], v[u], x[u][a]);
  }
#pragma unroll
  for (int a = 0; a < S; ++a) settle(w[a]);
}

// ---- coefficients of a step in shared memory -------------------------------------------------
template <typename R, int S>
struct Co {
  R ap[S][S], ac[S][S];  // tau_{j-1,j}, tau_jj
  R tn[S][S];            // tau_{j+1,j} (upper)
  R tni[S];              // reciprocals of its diagonal
};

template <typename R, int S>
__device__ void load_co(Co<R, S>& co, const double* __restrict__ rec) {
  constexpr int SS = S * S;
  for (int k = threadIdx.x; k < SS; k += blockDim.x) {
    const int a = k / S, b = k % S;
    co.ap[a][b] = coef<R>(rec[REC_TPREV * SS + k]);
    co.ac[a][b] = coef<R>(rec[REC_TDIAG * SS + k]);
    co.tn[a][b] = coef<R>(rec[REC_TNEXT * SS + k]);
  }
  for (int b = threadIdx.x; b < S; b += blockDim.x) co.tni[b] = coef<R>(1.0 / rec[REC_TNEXT * SS + b * S + b]);
  __syncthreads();
}

// v = (w - p tau_{j-1,j} - q tau_jj) tau_{j+1,j}^{-1}: the row recipe of sweep B and of the
// second pass (forward substitution with the reciprocal diagonal)
template <typename R, int S>
__device__ __forceinline__ void recipe(const Co<R, S>& co, const R (&p)[S], const R (&q)[S], R (&w)[S], bool hp) {
#pragma unroll
  for (int b = 0; b < S; ++b) {
    R t = w[b];
    if (hp) {
#pragma unroll
      for (int a = 0; a < S; ++a) msub(t, p[a], co.ap[a][b]);
    }
#pragma unroll
    for (int a = 0; a < S; ++a) msub(t, q[a], co.ac[a][b]);
    w[b] = t;
  }
#pragma unroll
  for (int b = 0; b < S; ++b) {
    R t = w[b];
#pragma unroll
    for (int a = 0; a < b; ++a) msub(t, w[a], co.tn[a][b]);
    w[b] = mulc(t, co.tni[b]);
  }
}

// ---- deterministic two-stage reduction ------------------------------------------------------
// Stage 1 (every CTA): fixed shuffle tree per warp, then the warps in order, into the CTA's slot
// of the partials (coefficient-major: P[k * count + slot]).  Stage 2 (the last CTA to arrive):
// warp w sums coefficients w, w + kWarps, ...; its lanes run over the slots in order and
// combine in a fixed shuffle order.  fp64 sums stay fp64; fp32 and float-pair sums are carried
// as float pairs (hi, lo in the 8 bytes of a slot), added with TwoSum.
template <typename Acc>
constexpr bool kPairSlots = !std::is_same<Acc, double>::value;
__device__ __forceinline__ ff to_ff(float x) { return ff_make(x, 0.f); }
__device__ __forceinline__ ff to_ff(ff x) { return ff_norm(x); }
__device__ __forceinline__ ff shfl_ff(ff v, int o) {
  return ff_make(__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o));
}

template <typename Acc, int NACC>
__device__ void stage1(Acc (&acc)[NACC], double* __restrict__ P, unsigned int slot, unsigned int count,
                       double* __restrict__ scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if constexpr (!kPairSlots<Acc>) {
#pragma unroll
    for (int k = 0; k < NACC; ++k) {
      double v = acc[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) scratch[warp * NACC + k] = v;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < NACC; k += blockDim.x) {
      double t = 0.0;
      for (int w = 0; w < kWarps; ++w) t += scratch[w * NACC + k];
      P[(size_t)k * count + slot] = t;
    }
  } else {
    float2* sc = reinterpret_cast<float2*>(scratch);
#pragma unroll
    for (int k = 0; k < NACC; ++k) {
      ff v = to_ff(acc[k]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v = ff_add(v, shfl_ff(v, o));
      if (lane == 0) sc[warp * NACC + k] = make_float2(v.hi, v.lo);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < NACC; k += blockDim.x) {
      ff t = ff_make(0.f, 0.f);
      for (int w = 0; w < kWarps; ++w) t = ff_add(t, ff_make(sc[w * NACC + k].x, sc[w * NACC + k].y));
      reinterpret_cast<float2*>(P)[(size_t)k * count + slot] = make_float2(t.hi, t.lo);
    }
  }
}

template <bool kPair, int NACC>
__device__ void stage2(const double* __restrict__ P, unsigned int count, double* __restrict__ tot) {
  constexpr int kB = 8;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = warp; k < NACC; k += kWarps) {
    if constexpr (kPair) {
      const float2* col = reinterpret_cast<const float2*>(P) + (size_t)k * count;
      ff t = ff_make(0.f, 0.f);
      for (unsigned int b0 = 0; b0 < count; b0 += 32 * kB) {
        float2 v[kB];
#pragma unroll
        for (int u = 0; u < kB; ++u) {
          const unsigned int b = b0 + 32 * u + lane;
          v[u] = b < count ? __ldcg(col + b) : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < kB; ++u) t = ff_add(t, ff_make(v[u].x, v[u].y));
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t = ff_add(t, shfl_ff(t, o));
      if (lane == 0) tot[k] = ff_to_double(t);
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
__device__ bool reduce_step(Acc (&acc)[NACC], double* __restrict__ partials, unsigned int* counter,
                            double* __restrict__ tot, double* __restrict__ scratch) {
  constexpr bool kPair = kPairSlots<Acc>;
  stage1<Acc, NACC>(acc, partials, blockIdx.x, gridDim.x, scratch);
  __threadfence();
  __shared__ unsigned int ticket;
  __syncthreads();
  if (threadIdx.x == 0) ticket = atomicAdd(counter, 1u);
  __syncthreads();
  if (ticket != gridDim.x - 1) return false;
  __threadfence();
  stage2<kPair, NACC>(partials, gridDim.x, tot);
  if (threadIdx.x == 0) *counter = 0u;
  return true;
}

// G = R^T R with R upper triangular and a positive diagonal; false if a pivot is not positive
template <int S>
__device__ bool chol_up(const double* G, double* R) {
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

// ---- kernels -------------------------------------------------------------------------------
struct StepArgs {
  OpDev op;
  int j;           // iteration (1-based); its record is op.log + j * LOG_NREC * S * S
  int has_prev;    // j > 1
  const void* Vp;  // V_{j-1}
  const void* Vc;  // V_j
  void* Vn;        // V_{j+1} (S4, pass 2) or W (S1)
  int64_t ldp, ldc, ldn;  // leading dimensions in values
  int* flags;
};

// coefficients of the sweeps S2 and S3, converted to the row arithmetic's type
template <typename R, int S>
struct CoMid {
  R ap[S][S], ac[S][S];  // S2: the first MGS sweep
  R tp[S][S], td[S][S];  // S3: both MGS sweeps combined
  R r1[S][S], r1i[S];    // S3: the first Cholesky QR factor and its reciprocal diagonal
};

template <typename R, int S>
__device__ void load_mid(CoMid<R, S>& co, const double* __restrict__ rec, int stage) {
  constexpr int SS = S * S;
  for (int k = threadIdx.x; k < SS; k += blockDim.x) {
    const int a = k / S, b = k % S;
    if (stage == 2) {
      co.ap[a][b] = coef<R>(rec[REC_APREV * SS + k]);
      co.ac[a][b] = coef<R>(rec[REC_ADIAG * SS + k]);
    } else {
      co.tp[a][b] = coef<R>(rec[REC_TPREV * SS + k]);
      co.td[a][b] = coef<R>(rec[REC_TDIAG * SS + k]);
      co.r1[a][b] = coef<R>(rec[REC_R1 * SS + k]);
    }
  }
  if (stage == 3)
    for (int b = threadIdx.x; b < S; b += blockDim.x) co.r1i[b] = coef<R>(1.0 / rec[REC_R1 * SS + b * S + b]);
  __syncthreads();
}

// w -= p M1 + q M2 (rows times s x s blocks), M1 skipped without a previous block
template <typename R, int S>
__device__ __forceinline__ void project(const R (&p)[S], const R (&q)[S], const R (&M1)[S][S], const R (&M2)[S][S],
                                        R (&w)[S], bool hp) {
#pragma unroll
  for (int b = 0; b < S; ++b) {
    R t = w[b];
    if (hp) {
#pragma unroll
      for (int a = 0; a < S; ++a) msub(t, p[a], M1[a][b]);
    }
#pragma unroll
    for (int a = 0; a < S; ++a) msub(t, q[a], M2[a][b]);
    settle(t);
    w[b] = t;
  }
}

// one sweep's rows: W, V_j and V_{j-1} (zero without a previous block)
template <class Num, int S>
__device__ __forceinline__ void load3(const StepArgs& g, int64_t row, typename Num::R (&w)[S],
                                      typename Num::R (&q)[S], typename Num::R (&p)[S]) {
  using V = typename Num::V;
  ld_row<S>(static_cast<const V*>(g.op.W), (int64_t)S, row, w);
  ld_row<S>(static_cast<const V*>(g.Vc), g.ldc, row, q);
  if (g.has_prev) ld_row<S>(static_cast<const V*>(g.Vp), g.ldp, row, p);
  else {
#pragma unroll
    for (int a = 0; a < S; ++a) zero(p[a]);
  }
}

__device__ __forceinline__ bool all_fin(const double* x, int n) {
  bool f = true;
  for (int i = 0; i < n; ++i) f = f && isfinite(x[i]);
  return f;
}

// S1: W = A V_j (SELL SpMM) and the first block MGS projections of Alg. 2 in fused form:
//   alpha_{j-1} = V_{j-1}^T W,  alpha_j = V_j^T W - (V_j^T V_{j-1}) alpha_{j-1}
// (the same as projecting V_j out of W - V_{j-1} alpha_{j-1}).  CTA b owns a contiguous range of
// slices, so rows its warps gather from the same plane of the operator are often still in its L1.
template <class Num, typename AV, int S>
__global__ void __launch_bounds__(kThreads, Num::kMinBlocks) k_s1(StepArgs g) {
  using V = typename Num::V;
  using R = typename Num::R;
  using Acc = typename Num::Acc;
  constexpr int SS = S * S;
  constexpr int NACC = 3 * SS;
  Acc acc[NACC];
#pragma unroll
  for (int k = 0; k < NACC; ++k) zero(acc[k]);
  const V* Vp = static_cast<const V*>(g.Vp);
  const V* Vc = static_cast<const V*>(g.Vc);
  V* W = static_cast<V*>(g.Vn);
  const bool hp = g.has_prev;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t nsl = g.op.nslices;
  const int64_t lo = nsl * blockIdx.x / gridDim.x, hi = nsl * (blockIdx.x + 1) / gridDim.x;
  for (int64_t sl = lo + warp; sl < hi; sl += kWarps) {
    const int64_t rs = sl * LYAP_SLICE + lane;
    const int64_t row = g.op.perm ? (rs < g.op.n ? (int64_t)g.op.perm[rs] : g.op.n) : rs;
    if (row >= g.op.n) continue;
    R w[S], q[S], p[S];
    spmm_row<Num, AV, S>(g.op, g.op.slice_ptr[sl], g.op.slice_w[sl], lane, Vc, g.ldc, w);
    st_row<S>(W, (int64_t)S, row, w);
    ld_row<S>(Vc, g.ldc, row, q);
    if (hp) ld_row<S>(Vp, g.ldp, row, p);
    else {
#pragma unroll
      for (int a = 0; a < S; ++a) zero(p[a]);
    }
#pragma unroll
    for (int a = 0; a < S; ++a)
#pragma unroll
      for (int b = 0; b < S; ++b) {
        gram(acc[a * S + b], p[a], w[b]);
        gram(acc[SS + a * S + b], q[a], w[b]);
        gram(acc[2 * SS + a * S + b], q[a], p[b]);
      }
  }
  __shared__ double tot[NACC];
  __shared__ double scratch[kWarps * NACC];
  if (!reduce_step<Acc, NACC>(acc, g.op.partials, g.op.counter, tot, scratch)) return;
  double* rec = g.op.log + (size_t)g.j * LOG_NREC * SS;
  const int k = threadIdx.x;
  if (k < SS) {
    const int a = k / S, b = k % S;
    double ap = hp ? tot[k] : 0.0, t = tot[SS + k];
    if (hp)
      for (int u = 0; u < S; ++u) t -= tot[2 * SS + a * S + u] * tot[u * S + b];
    rec[REC_APREV * SS + k] = ap;
    rec[REC_ADIAG * SS + k] = t;
    rec[REC_CROSS * SS + k] = hp ? tot[2 * SS + k] : 0.0;
    if (!isfinite(ap) || !isfinite(t)) atomicOr(g.flags, DERR_NONFINITE);
  }
}

// S2: w1 = W - V_{j-1} alpha_{j-1} - V_j alpha_j; the second MGS projections and G1 = w1^T w1 ->
//   beta_{j-1} = V_{j-1}^T w1, beta_j = V_j^T w1 - (V_j^T V_{j-1}) beta_{j-1},
//   tau_{j-1,j} = alpha_{j-1} + beta_{j-1}, tau_jj = alpha_j + beta_j,
//   R1 = chol(G1 - beta^T beta)  (the Gram matrix of w2 = w1 - V beta)
template <class Num, int S>
__global__ void __launch_bounds__(kThreads, Num::kMinBlocks) k_s2(StepArgs g) {
  using R = typename Num::R;
  using Acc = typename Num::Acc;
  constexpr int SS = S * S;
  constexpr int NSYM = S * (S + 1) / 2;
  constexpr int NACC = 2 * SS + NSYM;
  __shared__ CoMid<R, S> co;
  double* rec = g.op.log + (size_t)g.j * LOG_NREC * SS;
  load_mid<R, S>(co, rec, 2);
  Acc acc[NACC];
#pragma unroll
  for (int k = 0; k < NACC; ++k) zero(acc[k]);
  const bool hp = g.has_prev;
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < g.op.n;
       row += (int64_t)gridDim.x * blockDim.x) {
    R w[S], q[S], p[S];
    load3<Num, S>(g, row, w, q, p);
    project<R, S>(p, q, co.ap, co.ac, w, hp);
#pragma unroll
    for (int a = 0; a < S; ++a)
#pragma unroll
      for (int b = 0; b < S; ++b) {
        gram(acc[a * S + b], p[a], w[b]);
        gram(acc[SS + a * S + b], q[a], w[b]);
      }
    int e = 2 * SS;
#pragma unroll
    for (int a = 0; a < S; ++a)
#pragma unroll
      for (int b = a; b < S; ++b, ++e) gram(acc[e], w[a], w[b]);
  }
  __shared__ double tot[NACC];
  __shared__ double scratch[kWarps * NACC];
  if (!reduce_step<Acc, NACC>(acc, g.op.partials, g.op.counter, tot, scratch)) return;
  __shared__ double bp[SS], bd[SS], G[SS];
  const int k = threadIdx.x;
  const int a = k / S, b = k % S;
  if (k < SS) {
    bp[k] = hp ? tot[k] : 0.0;
    double t = tot[SS + k];
    if (hp)
      for (int u = 0; u < S; ++u) t -= rec[REC_CROSS * SS + a * S + u] * tot[u * S + b];
    bd[k] = t;
  }
  __syncthreads();
  if (k < SS) {
    const int lo = a < b ? a : b, hi = a < b ? b : a;
    double v = tot[2 * SS + lo * S - lo * (lo - 1) / 2 + (hi - lo)];
    for (int u = 0; u < S; ++u) v -= bp[u * S + a] * bp[u * S + b] + bd[u * S + a] * bd[u * S + b];
    G[k] = v;
    rec[REC_BPREV * SS + k] = bp[k];
    rec[REC_BDIAG * SS + k] = bd[k];
    rec[REC_TPREV * SS + k] = rec[REC_APREV * SS + k] + bp[k];
    rec[REC_TDIAG * SS + k] = rec[REC_ADIAG * SS + k] + bd[k];
  }
  __syncthreads();
  if (k == 0) {
    double R1[SS];
    const bool finite = all_fin(G, SS) && all_fin(bp, SS) && all_fin(bd, SS);
    if (!finite) atomicOr(g.flags, DERR_NONFINITE);
    if (!chol_up<S>(G, R1)) {
      if (finite) atomicOr(g.flags, DERR_BREAKDOWN);
      for (int e = 0; e < SS; ++e) R1[e] = (e % (S + 1) == 0) ? 1.0 : 0.0;
    }
    for (int e = 0; e < SS; ++e) rec[REC_R1 * SS + e] = R1[e];
  }
}

// S3: x = (W - V_{j-1} tau_{j-1,j} - V_j tau_jj) R1^{-1}; R2 = chol(x^T x), tau_{j+1,j} = R2 R1
// (the second pass of Cholesky QR measures the Gram matrix of the rows actually formed)
template <class Num, int S>
__global__ void __launch_bounds__(kThreads, Num::kMinBlocks) k_s3(StepArgs g) {
  using R = typename Num::R;
  using Acc = typename Num::Acc;
  constexpr int SS = S * S;
  constexpr int NSYM = S * (S + 1) / 2;
  constexpr int NACC = NSYM;
  __shared__ CoMid<R, S> co;
  double* rec = g.op.log + (size_t)g.j * LOG_NREC * SS;
  load_mid<R, S>(co, rec, 3);
  Acc acc[NACC];
#pragma unroll
  for (int k = 0; k < NACC; ++k) zero(acc[k]);
  const bool hp = g.has_prev;
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < g.op.n;
       row += (int64_t)gridDim.x * blockDim.x) {
    R w[S], q[S], p[S];
    load3<Num, S>(g, row, w, q, p);
    project<R, S>(p, q, co.tp, co.td, w, hp);
#pragma unroll
    for (int b = 0; b < S; ++b) {
      R t = w[b];
#pragma unroll
      for (int a = 0; a < b; ++a) msub(t, w[a], co.r1[a][b]);
      w[b] = mulc(t, co.r1i[b]);
    }
    int e = 0;
#pragma unroll
    for (int a = 0; a < S; ++a)
#pragma unroll
      for (int b = a; b < S; ++b, ++e) gram(acc[e], w[a], w[b]);
  }
  __shared__ double tot[NACC];
  __shared__ double scratch[kWarps * NACC];
  if (!reduce_step<Acc, NACC>(acc, g.op.partials, g.op.counter, tot, scratch)) return;
  if (threadIdx.x == 0) {
    double G[SS], R2[SS], Tn[SS];
    int e = 0;
    for (int a = 0; a < S; ++a)
      for (int b = a; b < S; ++b, ++e) G[a * S + b] = G[b * S + a] = tot[e];
    if (!chol_up<S>(G, R2)) {
      atomicOr(g.flags, all_fin(G, SS) ? DERR_BREAKDOWN : DERR_NONFINITE);
      for (int f = 0; f < SS; ++f) R2[f] = (f % (S + 1) == 0) ? 1.0 : 0.0;
    }
    for (int a = 0; a < S; ++a)
      for (int b = 0; b < S; ++b) {
        double t = 0.0;
        for (int u = 0; u < S; ++u) t += R2[a * S + u] * rec[REC_R1 * SS + u * S + b];
        Tn[a * S + b] = t;
      }
    for (int f = 0; f < SS; ++f) {
      rec[REC_R2 * SS + f] = R2[f];
      rec[REC_TNEXT * SS + f] = Tn[f];
    }
    if (!all_fin(Tn, SS)) atomicOr(g.flags, DERR_NONFINITE);
  }
}

// S4: V_{j+1} = (W - V_{j-1} tau_{j-1,j} - V_j tau_jj) tau_{j+1,j}^{-1}, the row recipe of the
// second pass (both MGS sweeps and both Cholesky QR factors applied at once: eq. 2.6)
template <class Num, int S>
__global__ void __launch_bounds__(kThreads) k_s4(StepArgs g) {
  using V = typename Num::V;
  using R = typename Num::R;
  constexpr int SS = S * S;
  __shared__ Co<R, S> co;
  load_co<R, S>(co, g.op.log + (size_t)g.j * LOG_NREC * SS);
  V* Vn = static_cast<V*>(g.Vn);
  const bool hp = g.has_prev;
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < g.op.n;
       row += (int64_t)gridDim.x * blockDim.x) {
    R w[S], q[S], p[S];
    load3<Num, S>(g, row, w, q, p);
    recipe<R, S>(co, p, q, w, hp);
    st_row<S>(Vn, g.ldn, row, w);
  }
}

// second pass, step j: V_{j+1} = recipe(A V_j, V_{j-1}, V_j) in one sweep, the same SpMM and row
// recipe as the first pass (hence the same bits)
template <class Num, typename AV, int S>
__global__ void __launch_bounds__(kThreads, Num::kMinBlocks) k_pass2(StepArgs g) {
  using V = typename Num::V;
  using R = typename Num::R;
  constexpr int SS = S * S;
  __shared__ Co<R, S> co;
  load_co<R, S>(co, g.op.log + (size_t)g.j * LOG_NREC * SS);
  const V* Vp = static_cast<const V*>(g.Vp);
  const V* Vc = static_cast<const V*>(g.Vc);
  V* Vn = static_cast<V*>(g.Vn);
  const bool hp = g.has_prev;
  const int lane = threadIdx.x & 31;
  const int64_t gwarp = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
  const int64_t nwarps = (int64_t)gridDim.x * kWarps;
  for (int64_t sl = gwarp; sl < g.op.nslices; sl += nwarps) {
    const int64_t rs = sl * LYAP_SLICE + lane;
    const int64_t row = g.op.perm ? (rs < g.op.n ? (int64_t)g.op.perm[rs] : g.op.n) : rs;
    if (row >= g.op.n) continue;
    R w[S], q[S], p[S];
    spmm_row<Num, AV, S>(g.op, g.op.slice_ptr[sl], g.op.slice_w[sl], lane, Vc, g.ldc, w);
    ld_row<S>(Vc, g.ldc, row, q);
    if (hp) ld_row<S>(Vp, g.ldp, row, p);
    else {
#pragma unroll
      for (int a = 0; a < S; ++a) zero(p[a]);
    }
    recipe<R, S>(co, p, q, w, hp);
    st_row<S>(Vn, g.ldn, row, w);
  }
}

// ---- the initial block: C = V_1 gamma by Cholesky QR twice on the fp64 right-hand side -------
// log record 0 holds R1, R2, gamma = R2 R1 (in REC_TNEXT) and beta = ||C||_F in REC_TDIAG[0]
template <int S>
__global__ void __launch_bounds__(kThreads) k_init_gram(StepArgs g, int stage) {
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
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < g.op.n;
       row += (int64_t)gridDim.x * blockDim.x) {
    double w[S];
    ld_row<S>(g.op.C, (int64_t)S, row, w);
    if (stage == 2) {
#pragma unroll
      for (int b = 0; b < S; ++b) {
        double t = w[b];
#pragma unroll
        for (int a = 0; a < b; ++a) t = fma(-w[a], r1[a][b], t);
        w[b] = t * r1i[b];
      }
    }
#pragma unroll
    for (int a = 0; a < S; ++a)
#pragma unroll
      for (int b = 0; b < S; ++b) acc[a * S + b] = fma(w[a], w[b], acc[a * S + b]);
  }
  __shared__ double tot[SS];
  __shared__ double scratch[kWarps * SS];
  if (!reduce_step<double, SS>(acc, g.op.partials, g.op.counter, tot, scratch)) return;
  if (threadIdx.x == 0) {
    double G[SS], R[SS];
    for (int a = 0; a < S; ++a)
      for (int b = 0; b < S; ++b) G[a * S + b] = 0.5 * (tot[a * S + b] + tot[b * S + a]);
    bool finite = true;
    for (int e = 0; e < SS; ++e) finite = finite && isfinite(G[e]);
    if (!finite) atomicOr(g.flags, DERR_NONFINITE);
    if (!chol_up<S>(G, R)) {
      if (finite) atomicOr(g.flags, DERR_BREAKDOWN);
      for (int e = 0; e < SS; ++e) R[e] = (e % (S + 1) == 0) ? 1.0 : 0.0;
    }
    if (stage == 1) {
      double tr = 0.0;
      for (int a = 0; a < S; ++a) tr += G[a * S + a];
      for (int e = 0; e < SS; ++e) rec[REC_R1 * SS + e] = R[e];
      rec[REC_TDIAG * SS] = sqrt(tr);
    } else {
      for (int a = 0; a < S; ++a)
        for (int b = 0; b < S; ++b) {
          double t = 0.0;
          for (int u = 0; u < S; ++u) t += R[a * S + u] * rec[REC_R1 * SS + u * S + b];
          rec[REC_TNEXT * SS + a * S + b] = t;  // gamma = R2 R1
        }
      for (int e = 0; e < SS; ++e) rec[REC_R2 * SS + e] = R[e];
    }
  }
}

// V_1 = C R1^{-1} R2^{-1} in fp64, stored in the bulk type
template <class Num, int S>
__global__ void __launch_bounds__(kThreads) k_init_write(StepArgs g) {
  using V = typename Num::V;
  using R = typename Num::R;
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
  V* Vn = static_cast<V*>(g.Vn);
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < g.op.n;
       row += (int64_t)gridDim.x * blockDim.x) {
    double w[S];
    ld_row<S>(g.op.C, (int64_t)S, row, w);
#pragma unroll
    for (int b = 0; b < S; ++b) {
      double t = w[b];
#pragma unroll
      for (int a = 0; a < b; ++a) t = fma(-w[a], r1[a][b], t);
      w[b] = t * r1i[b];
    }
#pragma unroll
    for (int b = 0; b < S; ++b) {
      double t = w[b];
#pragma unroll
      for (int a = 0; a < b; ++a) t = fma(-w[a], r2[a][b], t);
      w[b] = t * r2i[b];
    }
    R v[S];
#pragma unroll
    for (int a = 0; a < S; ++a) v[a] = coef<R>(w[a]);
    st_row<S>(Vn, g.ldn, row, v);
  }
}

// ---- dispatch over (bulk type, operator value type, block size) ------------------------------
// bulk: LYAP_PREC_F64, LYAP_PREC_MIXED (fp32) or LYAP_PREC_F32X2 (float pairs); the float-pair
// path stores operator values as fp32 when they are exact in fp32 (op.val_pair == 0), else as
// pairs.  Block sizes 1, 2, 3, 4 and 8 (float pairs: up to 4).
template <template <class, typename, int> class F, typename... Args>
int dispatch(int bulk, int pair, int s, Args&&... args) {
#define LYAP_DS(NUM, AV)                                            \
  switch (s) {                                                      \
    case 1: F<NUM, AV, 1>::run(args...); return 1;                  \
    case 2: F<NUM, AV, 2>::run(args...); return 1;                  \
    case 3: F<NUM, AV, 3>::run(args...); return 1;                  \
    case 4: F<NUM, AV, 4>::run(args...); return 1;                  \
    default: break;                                                 \
  }
  if (bulk == LYAP_PREC_F32X2) {
    if (pair) { LYAP_DS(NumFF, float2) }
    else { LYAP_DS(NumFF, float) }
    return 0;
  }
  if (bulk == LYAP_PREC_MIXED) {
    LYAP_DS(NumF, float)
    if (s == 8) { F<NumF, float, 8>::run(args...); return 1; }
    return 0;
  }
  LYAP_DS(NumD, double)
  if (s == 8) { F<NumD, double, 8>::run(args...); return 1; }
  return 0;
#undef LYAP_DS
}

template <class Num, typename AV, int S>
struct RunStep {
  static void run(OpDev& op, int grid_a, int grid_b, int j, int* flags, cudaStream_t st) {
    StepArgs g;
    g.op = op;
    g.j = j;
    g.has_prev = j > 1;
    g.Vp = op.V[(j + 1) % 3];  // V_{j-1}
    g.Vc = op.V[(j + 2) % 3];  // V_j   (V_1 lives in V[0])
    g.ldp = g.ldc = S;
    g.flags = flags;
    g.Vn = op.W;
    g.ldn = S;
    k_s1<Num, AV, S><<<grid_a, kThreads, 0, st>>>(g);
    k_s2<Num, S><<<grid_b, kThreads, 0, st>>>(g);
    k_s3<Num, S><<<grid_b, kThreads, 0, st>>>(g);
    g.Vn = op.V[j % 3];  // V_{j+1}
    k_s4<Num, S><<<grid_b, kThreads, 0, st>>>(g);
  }
};

template <class Num, typename AV, int S>
struct RunInit {
  static void run(OpDev& op, int grid, int* flags, void* vn, int64_t ldn, int gram, cudaStream_t st) {
    StepArgs g;
    g.op = op;
    g.j = 0;
    g.has_prev = 0;
    g.flags = flags;
    g.Vn = vn;
    g.ldn = ldn;
    if (gram) {
      k_init_gram<S><<<grid, kThreads, 0, st>>>(g, 1);
      k_init_gram<S><<<grid, kThreads, 0, st>>>(g, 2);
    }
    k_init_write<Num, S><<<grid, kThreads, 0, st>>>(g);
  }
};

template <class Num, typename AV, int S>
struct RunPass2 {
  static void run(OpDev& op, int grid, int j, const void* vp, int64_t ldp, const void* vc, int64_t ldc, void* vn,
                  int64_t ldn, cudaStream_t st) {
    StepArgs g;
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
    k_pass2<Num, AV, S><<<grid, kThreads, 0, st>>>(g);
  }
};

template <class Num, typename AV, int S>
struct Occ {
  static void run(int* a, int* b) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(a, k_s1<Num, AV, S>, kThreads, 0) != cudaSuccess) *a = 1;
    int b2 = 1, b3 = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b2, k_s2<Num, S>, kThreads, 0) != cudaSuccess) b2 = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b3, k_s3<Num, S>, kThreads, 0) != cudaSuccess) b3 = 1;
    *b = b2 < b3 ? b2 : b3;
  }
};

}  // namespace

int max_nacc(int s) { return 3 * s * s; }

int step_supported(int bulk, int s) {
  if (bulk == LYAP_PREC_F32X2) return s >= 1 && s <= 4;
  return s == 1 || s == 2 || s == 3 || s == 4 || s == 8;
}

// CTAs per SM of the two sweep kernels
void step_blocks_per_sm(int s, int bulk, int pair, int* per_sm_a, int* per_sm_b) {
  *per_sm_a = *per_sm_b = 1;
  dispatch<Occ>(bulk, pair, s, per_sm_a, per_sm_b);
  if (*per_sm_a < 1) *per_sm_a = 1;
  if (*per_sm_b < 1) *per_sm_b = 1;
}

int launch_init_block(OpDev& op, int s, int bulk, int grid, int* d_flags, cudaStream_t st) {
  dispatch<RunInit>(bulk, op.val_pair, s, op, grid, d_flags, op.V[0], (int64_t)s, 1, st);
  return 3;
}

int launch_lanczos_step(OpDev& op, int s, int bulk, int grid_a, int grid_b, int j, int* d_flags, cudaStream_t st) {
  dispatch<RunStep>(bulk, op.val_pair, s, op, grid_a, grid_b, j, d_flags, st);
  return 4;
}

// Second pass, step j: writes V_{j+1} from V_{j-1} (vp), V_j (vc).
void launch_pass2(OpDev& op, int s, int bulk, int grid, int j, const void* vp, int64_t ldp, const void* vc,
                  int64_t ldc, void* vn, int64_t ldn, cudaStream_t st) {
  dispatch<RunPass2>(bulk, op.val_pair, s, op, grid, j, vp, ldp, vc, ldc, vn, ldn, st);
}

// Second pass, V_1 from C with the logged Cholesky QR factors of the first pass.
void launch_pass2_v1(OpDev& op, int s, int bulk, int grid, void* vn, int64_t ldn, cudaStream_t st) {
  dispatch<RunInit>(bulk, op.val_pair, s, op, grid, (int*)nullptr, vn, ldn, 0, st);
}
