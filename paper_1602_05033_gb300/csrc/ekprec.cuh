// Preconditioners of the inner solves M x = b, M = -A, of the extended Krylov path, for a
// 5-point operator on an nx x ny grid (x fastest).  Included by ek.cu inside its anonymous
// namespace (it uses Csr, cta_partials, k_sum_partials, kT and kTile from there).
//
//  * IC(0) (Meijerink and van der Vorst): L = D + N with the pattern of tril(M).  For a 5-point
//    operator the pivots p_i = L_ii^2 obey p_i = M_ii - M_{i,i-1}^2 / p_{i-1} - M_{i,i-nx}^2 / p_{i-nx},
//    and L_{i,i-1} = M_{i,i-1} / L_{i-1,i-1}, L_{i,i-nx} = M_{i,i-nx} / L_{i-nx,i-nx}: one pass along
//    the anti-diagonals x + y = t of the grid (one CTA, a thread per grid column).
//  * Application by a truncated Neumann series, products only: with T = -D^{-1} N (nilpotent),
//    B_q = sum_{t=0}^{q} T^t D^{-1} ~ L^{-1}, evaluated by Horner steps y <- D^{-1} (r - N y), and
//    P_q = B_q^T B_q, symmetric positive definite for any positive d.  q = kQ.
//  * Learned values: a network of three 3x3 convolutions (5 -> 16 -> 16 -> 3 channels, ReLU, bf16
//    activations and weights, fp32 accumulation) maps the stencil row over its diagonal to
//    corrections of the IC(0) values, d = d0 exp(y0), lw = lw0 (1 + y1), ls = ls0 (1 + y2) (a zero
//    last layer is IC(0)).  It is trained with Adam on the energy-norm error of one application,
//    (1/K) sum_k ||P_q r_k - x_k||_M^2 / ||x_k||_M^2, over solve pairs of the method.  The gradient
//    with respect to the values runs the Horner recurrences backwards (reverse mode).  The 16 -> 16
//    convolution, which holds most of the arithmetic, runs forward, data-backward and
//    weight-backward on the tensor cores (mma.sync m16n8k16, bf16 in, fp32 accumulate); the
//    5 -> 16 and 16 -> 3 layers are small and run on the CUDA cores.
#pragma once

// (cuda_bf16.h and the integer types come from the including file)

constexpr int kQ = 3;         // Neumann terms beyond the first
constexpr int kCh = 16;       // hidden channels
constexpr int kNin = 5;       // input channels: 1, west, east, south, north over the diagonal
constexpr int kNout = 3;      // corrections of d, lw, ls
// parameters: w1 [16][5][9], b1 [16], w2 [16][16][9], b2 [16], w3 [3][16][9], b3 [3]
constexpr int oW1 = 0, oB1 = oW1 + kCh * kNin * 9, oW2 = oB1 + kCh, oB2 = oW2 + kCh * kCh * 9, oW3 = oB2 + kCh,
              oB3 = oW3 + kNout * kCh * 9, kNW = oB3 + kNout;
constexpr int kNW1 = kCh * kNin * 9 + kCh, kNW2 = kCh * kCh * 9 + kCh, kNW3 = kNout * kCh * 9 + kNout;
constexpr int kWarpsW = 8;    // warps per CTA of the tensor-core weight-gradient kernel

struct Grid {
  int nx, ny;
};

__device__ __forceinline__ int64_t gnode(const Grid g, int x, int y) { return (int64_t)y * g.nx + x; }
// grid coordinates of node p in 32-bit arithmetic (nx * ny < 2^31, checked at sizing)
__device__ __forceinline__ int grid_x(const Grid g, int64_t p) { return (int)p % g.nx; }
__device__ __forceinline__ int grid_y(const Grid g, int64_t p) { return (int)p / g.nx; }
__device__ __forceinline__ bool ginside(const Grid g, int x, int y) { return x >= 0 && x < g.nx && y >= 0 && y < g.ny; }

// ---- the operator's stencil --------------------------------------------------------------
// sten[i] = (M_ii, M_{i,i-1}, M_{i,i+1}, M_{i,i-nx}, M_{i,i+nx}) (zero outside the grid) and the
// network's input features (5 x n fp32: 1 and the four neighbours over the diagonal); *bad != 0
// when a row has an entry outside the 5-point pattern or a non-positive diagonal.
__global__ void k_stencil(Csr A, Grid g, double* __restrict__ sten, float* __restrict__ feats, int* __restrict__ bad) {
  const int64_t n = (int64_t)g.nx * g.ny;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int x = grid_x(g, i), y = grid_y(g, i);
    double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int64_t e = A.rowptr[i]; e < A.rowptr[i + 1]; ++e) {
      const int64_t j = A.col[e];
      const double m = -A.val[e];
      if (j == i) v[0] += m;
      else if (x > 0 && j == i - 1) v[1] += m;
      else if (x + 1 < g.nx && j == i + 1) v[2] += m;
      else if (y > 0 && j == i - g.nx) v[3] += m;
      else if (y + 1 < g.ny && j == i + g.nx) v[4] += m;
      else if (m != 0.0) atomicOr(bad, 1);
    }
    if (!(v[0] > 0.0)) atomicOr(bad, 2);
#pragma unroll
    for (int k = 0; k < 5; ++k) sten[i * 5 + k] = v[k];
    const double inv = v[0] > 0.0 ? 1.0 / v[0] : 0.0;
    feats[i] = 1.f;
#pragma unroll
    for (int k = 1; k < 5; ++k) feats[(int64_t)k * n + i] = (float)(v[k] * inv);
  }
}

// ---- IC(0): pivots along the anti-diagonals (one CTA, blockDim.x >= nx) ------------------------
__global__ void __launch_bounds__(1024) k_ic0_wave(const double* __restrict__ sten, Grid g, double* __restrict__ piv,
                                                   int* __restrict__ bad) {
  __shared__ double prow[2][1024];
  const int x = threadIdx.x;
  double below = 0.0;  // p(x, y - 1), this thread's previous pivot
  // coefficients of this thread's node on the current anti-diagonal, loaded one step ahead
  double c = 0.0, w = 0.0, s = 0.0;
  if (x < g.nx && 0 - x >= 0) {
    const int64_t i = gnode(g, x, 0);
    c = sten[i * 5];
    w = sten[i * 5 + 1];
    s = sten[i * 5 + 3];
  }
  const int steps = g.nx + g.ny - 1;
  for (int t = 0; t < steps; ++t) {
    const int y = t - x;
    double pv = 0.0;
    const bool mine = x < g.nx && y >= 0 && y < g.ny;
    const double cc = c, ww = w, ss = s;
    // prefetch the next step's node (x, y + 1)
    if (x < g.nx && y + 1 >= 0 && y + 1 < g.ny) {
      const int64_t i = gnode(g, x, y + 1);
      c = sten[i * 5];
      w = sten[i * 5 + 1];
      s = sten[i * 5 + 3];
    }
    if (mine) {
      double v = cc;
      if (x > 0) v -= ww * ww / prow[(t + 1) & 1][x - 1];  // p(x - 1, y), written at step t - 1
      if (y > 0) v -= ss * ss / below;
      if (!(v > 0.0)) {  // IC(0) does not exist for this operator; keep the sweep finite
        atomicOr(bad, 4);
        v = cc > 0.0 ? cc : 1.0;
      }
      piv[gnode(g, x, y)] = v;
      below = v;
      pv = v;
    }
    prow[t & 1][x] = pv;
    __syncthreads();
  }
}

// d = sqrt(p), lw = M_{i,i-1} / d_{i-1}, ls = M_{i,i-nx} / d_{i-nx}
__global__ void k_ic0_vals(const double* __restrict__ sten, const double* __restrict__ piv, Grid g,
                           double* __restrict__ d, double* __restrict__ lw, double* __restrict__ ls) {
  const int64_t n = (int64_t)g.nx * g.ny;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int x = grid_x(g, i), y = grid_y(g, i);
    d[i] = sqrt(piv[i]);
    lw[i] = x > 0 ? sten[i * 5 + 1] / sqrt(piv[i - 1]) : 0.0;
    ls[i] = y > 0 ? sten[i * 5 + 3] / sqrt(piv[i - g.nx]) : 0.0;
  }
}

// ---- Horner steps of B_q and B_q^T on C columns (blocks n x C, interleaved) --------------------
struct Vals {
  const double *d, *lw, *ls;
};

// U = Y0 = R / d (R with leading dimension ldr)
template <int C>
__global__ void k_h_first(const double* __restrict__ R, int ldr, const double* __restrict__ d, double* __restrict__ U,
                          double* __restrict__ Y0, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double inv = 1.0 / d[i];
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const double u = R[i * ldr + c] * inv;
      U[i * C + c] = u;
      Y0[i * C + c] = u;
    }
  }
}

// Y1 = U - (lw_i Y0(i-1) + ls_i Y0(i-nx)) / d_i
template <int C>
__global__ void k_h_fwd(const double* __restrict__ U, const double* __restrict__ Y0, Vals v, Grid g,
                        double* __restrict__ Y1) {
  const int64_t n = (int64_t)g.nx * g.ny;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int x = grid_x(g, i), y = grid_y(g, i);
    const double inv = 1.0 / v.d[i];
    const double a = x > 0 ? v.lw[i] : 0.0, b = y > 0 ? v.ls[i] : 0.0;
#pragma unroll
    for (int c = 0; c < C; ++c) {
      double t = 0.0;
      if (x > 0) t = a * Y0[(i - 1) * C + c];
      if (y > 0) t = fma(b, Y0[(i - g.nx) * C + c], t);
      Y1[i * C + c] = fma(-t, inv, U[i * C + c]);
    }
  }
}

// W1 = Y - (lw_{i+1} W0(i+1) / d_{i+1} + ls_{i+nx} W0(i+nx) / d_{i+nx})
template <int C>
__global__ void k_h_bwd(const double* __restrict__ Y, const double* __restrict__ W0, Vals v, Grid g,
                        double* __restrict__ W1) {
  const int64_t n = (int64_t)g.nx * g.ny;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int x = grid_x(g, i), y = grid_y(g, i);
    const bool e = x + 1 < g.nx, nn = y + 1 < g.ny;
    const double a = e ? v.lw[i + 1] / v.d[i + 1] : 0.0;
    const double b = nn ? v.ls[i + g.nx] / v.d[i + g.nx] : 0.0;
#pragma unroll
    for (int c = 0; c < C; ++c) {
      double t = 0.0;
      if (e) t = a * W0[(i + 1) * C + c];
      if (nn) t = fma(b, W0[(i + g.nx) * C + c], t);
      W1[i * C + c] = Y[i * C + c] - t;
    }
  }
}

// Z = W / d (Z with leading dimension ldz)
template <int C>
__global__ void k_h_last(const double* __restrict__ W, const double* __restrict__ d, double* __restrict__ Z, int ldz,
                         int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double inv = 1.0 / d[i];
#pragma unroll
    for (int c = 0; c < C; ++c) Z[i * ldz + c] = W[i * C + c] * inv;
  }
}

// reverse step j of sum_c a_c^T B_q c_c (forward iterates Y_j, Y_{j+1}; adjoint lam1 = lambda_{j+1}):
//   gd -= lam1 y_{j+1} / d,  gw -= lam1 y_j(i-1) / d,  gs -= lam1 y_j(i-nx) / d  (summed over columns)
//   lambda_j(i) = -(lw_{i+1} lam1(i+1) / d_{i+1} + ls_{i+nx} lam1(i+nx) / d_{i+nx})
template <int C>
__global__ void k_h_rev(const double* __restrict__ lam1, const double* __restrict__ Yj, const double* __restrict__ Yj1,
                        Vals v, Grid g, double* __restrict__ lam0, double* __restrict__ gd, double* __restrict__ gw,
                        double* __restrict__ gs) {
  const int64_t n = (int64_t)g.nx * g.ny;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int x = grid_x(g, i), y = grid_y(g, i);
    const double inv = 1.0 / v.d[i];
    double sd = 0.0, sw = 0.0, ss = 0.0;
    const bool e = x + 1 < g.nx, nn = y + 1 < g.ny;
    const double a = e ? v.lw[i + 1] / v.d[i + 1] : 0.0;
    const double b = nn ? v.ls[i + g.nx] / v.d[i + g.nx] : 0.0;
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const double l = lam1[i * C + c];
      sd = fma(l, Yj1[i * C + c], sd);
      if (x > 0) sw = fma(l, Yj[(i - 1) * C + c], sw);
      if (y > 0) ss = fma(l, Yj[(i - g.nx) * C + c], ss);
      double t = 0.0;
      if (e) t = a * lam1[(i + 1) * C + c];
      if (nn) t = fma(b, lam1[(i + g.nx) * C + c], t);
      lam0[i * C + c] = -t;
    }
    gd[i] -= sd * inv;
    if (x > 0) gw[i] -= sw * inv;
    if (y > 0) gs[i] -= ss * inv;
  }
}

// the first Horner value y_0 = D^{-1} r: gd -= lambda_0 y_0 / d
template <int C>
__global__ void k_h_rev_last(const double* __restrict__ lam0, const double* __restrict__ Y0, const double* __restrict__ d,
                             int64_t n, double* __restrict__ gd) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double sd = 0.0;
#pragma unroll
    for (int c = 0; c < C; ++c) sd = fma(lam0[i * C + c], Y0[i * C + c], sd);
    gd[i] -= sd / d[i];
  }
}

// per-column dot products sum_i U[i][c] V[i][c] -> partials
template <int C>
__global__ void k_coldots(const double* __restrict__ U, const double* __restrict__ V, int64_t n,
                          double* __restrict__ partials) {
  double acc[C];
#pragma unroll
  for (int c = 0; c < C; ++c) acc[c] = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
#pragma unroll
    for (int c = 0; c < C; ++c) acc[c] = fma(U[i * C + c], V[i * C + c], acc[c]);
  cta_partials<C>(acc, partials);
}

// Y[i][c] = a[c] * X[i][c] + b * Y[i][c] (a on the device)
__global__ void k_scale_cols(const double* __restrict__ X, const double* __restrict__ a, double b, int C, int64_t n,
                             double* __restrict__ Y) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * C; t += (int64_t)gridDim.x * blockDim.x)
    Y[t] = a[t % C] * X[t] + (b != 0.0 ? b * Y[t] : 0.0);
}

// energy loss terms: eMe[c], den[c] -> coef[0] = (1/K) sum_c eMe/den, coef[1 + c] = 2 / (K den_c)
__global__ void k_energy_terms(const double* __restrict__ eMe, const double* __restrict__ den, int K,
                               double* __restrict__ coef) {
  if (threadIdx.x) return;
  double L = 0.0;
  for (int c = 0; c < K; ++c) {
    L += eMe[c] / den[c];
    coef[1 + c] = 2.0 / (K * den[c]);
  }
  coef[0] = L / K;
}

// ---- the network's values and the gradient that flows into it -------------------------------
__global__ void k_net_vals(const float* __restrict__ y, Vals v0, int64_t n, double* __restrict__ d,
                           double* __restrict__ lw, double* __restrict__ ls) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    d[i] = v0.d[i] * exp((double)y[i * 3]);
    lw[i] = v0.lw[i] * (1.0 + (double)y[i * 3 + 1]);
    ls[i] = v0.ls[i] * (1.0 + (double)y[i * 3 + 2]);
  }
}

// gy = (g_d d, g_lw lw0, g_ls ls0)
__global__ void k_net_gy(const double* __restrict__ gd, const double* __restrict__ gw, const double* __restrict__ gs,
                         const double* __restrict__ d, Vals v0, int64_t n, float* __restrict__ gy) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    gy[i * 3] = (float)(gd[i] * d[i]);
    gy[i * 3 + 1] = (float)(gw[i] * v0.lw[i]);
    gy[i * 3 + 2] = (float)(gs[i] * v0.ls[i]);
  }
}

// ---- convolutions: activations are pixel-major (n x 16 bf16), taps k = dy * 3 + dx read the
// input at (x + dx - 1, y + dy - 1), zero outside the grid ------------------------------------
__device__ __forceinline__ float bfv(const __nv_bfloat16 v) { return __bfloat162float(v); }

__device__ __forceinline__ uint32_t pack_bf2(float lo, float hi) {
  const __nv_bfloat162 p = __floats2bfloat162_rn(lo, hi);  // .x = lo (low half), .y = hi
  return *reinterpret_cast<const uint32_t*>(&p);
}

__device__ __forceinline__ uint32_t pack_raw(uint16_t lo, uint16_t hi) { return (uint32_t)lo | ((uint32_t)hi << 16); }

// D += A B for one m16n8k16 tile (A row-major 16 x 16, B column-major 16 x 8, bf16; D fp32)
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// layer 1 (5 -> 16, ReLU) on the CUDA cores: feats 5 x n fp32 -> a1 n x 16 bf16
__global__ void k_l1_fwd(const float* __restrict__ feats, const __nv_bfloat16* __restrict__ wq,
                         const float* __restrict__ bias, Grid g, __nv_bfloat16* __restrict__ a1) {
  __shared__ float w[kCh * kNin * 9];
  __shared__ float b[kCh];
  for (int k = threadIdx.x; k < kCh * kNin * 9; k += blockDim.x) w[k] = bfv(wq[k]);
  for (int k = threadIdx.x; k < kCh; k += blockDim.x) b[k] = bias[k];
  __syncthreads();
  const int64_t n = (int64_t)g.nx * g.ny;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const int x = grid_x(g, p), y = grid_y(g, p);
    float acc[kCh];
#pragma unroll
    for (int co = 0; co < kCh; ++co) acc[co] = b[co];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const int xx = x + k % 3 - 1, yy = y + k / 3 - 1;
      if (!ginside(g, xx, yy)) continue;
      const int64_t q = gnode(g, xx, yy);
#pragma unroll
      for (int ci = 0; ci < kNin; ++ci) {
        const float f = feats[(int64_t)ci * n + q];
#pragma unroll
        for (int co = 0; co < kCh; ++co) acc[co] = fmaf(w[(co * kNin + ci) * 9 + k], f, acc[co]);
      }
    }
    uint32_t out[8];
#pragma unroll
    for (int h = 0; h < 8; ++h) out[h] = pack_bf2(fmaxf(acc[2 * h], 0.f), fmaxf(acc[2 * h + 1], 0.f));
    uint4* dst = reinterpret_cast<uint4*>(a1 + p * kCh);
    dst[0] = make_uint4(out[0], out[1], out[2], out[3]);
    dst[1] = make_uint4(out[4], out[5], out[6], out[7]);
  }
}

// 16 channels of pixel p (bf16) as floats
__device__ __forceinline__ void load16(const __nv_bfloat16* __restrict__ a, int64_t p, float (&v)[kCh]) {
  const uint4* s = reinterpret_cast<const uint4*>(a + p * kCh);
  const uint4 u0 = s[0], u1 = s[1];
  const uint32_t w[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
#pragma unroll
  for (int h = 0; h < 8; ++h) {
    const __nv_bfloat162 b2 = *reinterpret_cast<const __nv_bfloat162*>(&w[h]);
    v[2 * h] = __low2float(b2);
    v[2 * h + 1] = __high2float(b2);
  }
}

// layer 3 (16 -> 3, linear) on the CUDA cores: a2 n x 16 bf16 -> y n x 3 fp32
__global__ void k_l3_fwd(const __nv_bfloat16* __restrict__ a2, const __nv_bfloat16* __restrict__ wq,
                         const float* __restrict__ bias, Grid g, float* __restrict__ yout) {
  __shared__ float w[kNout * kCh * 9];
  for (int k = threadIdx.x; k < kNout * kCh * 9; k += blockDim.x) w[k] = bfv(wq[k]);
  __syncthreads();
  const int64_t n = (int64_t)g.nx * g.ny;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const int x = grid_x(g, p), y = grid_y(g, p);
    float acc[kNout];
#pragma unroll
    for (int co = 0; co < kNout; ++co) acc[co] = bias[co];
    for (int k = 0; k < 9; ++k) {
      const int xx = x + k % 3 - 1, yy = y + k / 3 - 1;
      if (!ginside(g, xx, yy)) continue;
      float v[kCh];
      load16(a2, gnode(g, xx, yy), v);
#pragma unroll
      for (int ci = 0; ci < kCh; ++ci)
#pragma unroll
        for (int co = 0; co < kNout; ++co) acc[co] = fmaf(w[(co * kCh + ci) * 9 + k], v[ci], acc[co]);
    }
#pragma unroll
    for (int co = 0; co < kNout; ++co) yout[p * kNout + co] = acc[co];
  }
}

// layer 3 data gradient: g2[p][ci] = [a2[p][ci] > 0] sum_k sum_co w3[co][ci][k] gy[q][co], where the
// output q = p - (dx - 1, dy - 1) read p through tap k
__global__ void k_l3_bwd_data(const float* __restrict__ gy, const __nv_bfloat16* __restrict__ wq,
                              const __nv_bfloat16* __restrict__ a2, Grid g, __nv_bfloat16* __restrict__ g2) {
  __shared__ float w[kNout * kCh * 9];
  for (int k = threadIdx.x; k < kNout * kCh * 9; k += blockDim.x) w[k] = bfv(wq[k]);
  __syncthreads();
  const int64_t n = (int64_t)g.nx * g.ny;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const int x = grid_x(g, p), y = grid_y(g, p);
    float acc[kCh];
#pragma unroll
    for (int ci = 0; ci < kCh; ++ci) acc[ci] = 0.f;
    for (int k = 0; k < 9; ++k) {
      const int xx = x - (k % 3 - 1), yy = y - (k / 3 - 1);
      if (!ginside(g, xx, yy)) continue;
      const int64_t q = gnode(g, xx, yy);
#pragma unroll
      for (int co = 0; co < kNout; ++co) {
        const float gq = gy[q * kNout + co];
#pragma unroll
        for (int ci = 0; ci < kCh; ++ci) acc[ci] = fmaf(w[(co * kCh + ci) * 9 + k], gq, acc[ci]);
      }
    }
    float a[kCh];
    load16(a2, p, a);
    uint32_t out[8];
#pragma unroll
    for (int h = 0; h < 8; ++h)
      out[h] = pack_bf2(a[2 * h] > 0.f ? acc[2 * h] : 0.f, a[2 * h + 1] > 0.f ? acc[2 * h + 1] : 0.f);
    uint4* dst = reinterpret_cast<uint4*>(g2 + p * kCh);
    dst[0] = make_uint4(out[0], out[1], out[2], out[3]);
    dst[1] = make_uint4(out[4], out[5], out[6], out[7]);
  }
}

// weight and bias gradients of a CUDA-core layer, per tile of kTile pixels (thread per weight):
//   layer 3: gw3[co][ci][k] = sum_p gy[p][co] a2[p + tap][ci],   gb3[co] = sum_p gy[p][co]
//   layer 1: gw1[co][ci][k] = sum_p g1[p][co] feats[ci][p + tap], gb1[co] = sum_p g1[p][co]
__global__ void k_l3_bwd_w(const float* __restrict__ gy, const __nv_bfloat16* __restrict__ a2, Grid g,
                           double* __restrict__ partials) {
  const int64_t n = (int64_t)g.nx * g.ny;
  const int64_t p0 = (int64_t)blockIdx.x * kTile;
  const int64_t p1 = p0 + kTile < n ? p0 + kTile : n;
  for (int wi = threadIdx.x; wi < kNW3; wi += blockDim.x) {
    double acc = 0.0;
    if (wi < kNout * kCh * 9) {
      const int co = wi / (kCh * 9), ci = (wi / 9) % kCh, k = wi % 9;
      float part = 0.f;
      for (int64_t p = p0; p < p1; ++p) {
        const int xx = grid_x(g, p) + k % 3 - 1, yy = grid_y(g, p) + k / 3 - 1;
        if (!ginside(g, xx, yy)) continue;
        part = fmaf(gy[p * kNout + co], bfv(a2[gnode(g, xx, yy) * kCh + ci]), part);
      }
      acc = part;
    } else {
      const int co = wi - kNout * kCh * 9;
      for (int64_t p = p0; p < p1; ++p) acc += gy[p * kNout + co];
    }
    partials[(size_t)blockIdx.x * kNW3 + wi] = acc;
  }
}

__global__ void k_l1_bwd_w(const __nv_bfloat16* __restrict__ g1, const float* __restrict__ feats, Grid g,
                           double* __restrict__ partials) {
  const int64_t n = (int64_t)g.nx * g.ny;
  const int64_t p0 = (int64_t)blockIdx.x * kTile;
  const int64_t p1 = p0 + kTile < n ? p0 + kTile : n;
  for (int wi = threadIdx.x; wi < kNW1; wi += blockDim.x) {
    double acc = 0.0;
    if (wi < kCh * kNin * 9) {
      const int co = wi / (kNin * 9), ci = (wi / 9) % kNin, k = wi % 9;
      float part = 0.f;
      for (int64_t p = p0; p < p1; ++p) {
        const int xx = grid_x(g, p) + k % 3 - 1, yy = grid_y(g, p) + k / 3 - 1;
        if (!ginside(g, xx, yy)) continue;
        part = fmaf(bfv(g1[p * kCh + co]), feats[(int64_t)ci * n + gnode(g, xx, yy)], part);
      }
      acc = part;
    } else {
      const int co = wi - kCh * kNin * 9;
      for (int64_t p = p0; p < p1; ++p) acc += bfv(g1[p * kCh + co]);
    }
    partials[(size_t)blockIdx.x * kNW1 + wi] = acc;
  }
}

// ---- layer 2 (16 -> 16) on the tensor cores -------------------------------------------------
// A warp owns chunks of 16 consecutive pixels.  Fragment ownership of mma.m16n8k16 (g = lane / 4,
// t = lane % 4): A rows g and g + 8, columns 2t, 2t + 1 (+ 8); B column g, rows 2t, 2t + 1 (+ 8);
// D rows g and g + 8, columns 2t, 2t + 1.

// word h (bf16 pair 2h, 2h + 1) of the 16 channels of pixel (x, y), zero outside the grid
__device__ __forceinline__ uint32_t ld_pair(const uint32_t* __restrict__ a, Grid g, int x, int y, bool ok, int h) {
  return ok && ginside(g, x, y) ? a[gnode(g, x, y) * 8 + h] : 0u;
}

// forward: a2[p][co] = relu(b2[co] + sum_k sum_ci w2[co][ci][k] a1[p + tap][ci]); GEMM per tap with
// M = 16 pixels, N = 16 output channels (two n8 tiles), K = 16 input channels
__global__ void __launch_bounds__(256) k_l2_fwd(const __nv_bfloat16* __restrict__ a1, const __nv_bfloat16* __restrict__ wq,
                                                const float* __restrict__ bias, Grid g, __nv_bfloat16* __restrict__ a2) {
  __shared__ uint16_t w[kCh * kCh * 9];
  const uint16_t* wraw = reinterpret_cast<const uint16_t*>(wq);
  for (int k = threadIdx.x; k < kCh * kCh * 9; k += blockDim.x) w[k] = wraw[k];
  __syncthreads();
  const int lane = threadIdx.x & 31, gq = lane >> 2, tq = lane & 3;
  // B fragments: B[k = ci][n = co] = w2[co][ci][tap]
  uint32_t bf[9][2][2];
#pragma unroll
  for (int k = 0; k < 9; ++k)
#pragma unroll
    for (int nb = 0; nb < 2; ++nb) {
      const int co = nb * 8 + gq;
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const int ci = 2 * tq + 8 * r;
        bf[k][nb][r] = pack_raw(w[(co * kCh + ci) * 9 + k], w[(co * kCh + ci + 1) * 9 + k]);
      }
    }
  float bb[2][2];
#pragma unroll
  for (int nb = 0; nb < 2; ++nb) {
    bb[nb][0] = bias[nb * 8 + 2 * tq];
    bb[nb][1] = bias[nb * 8 + 2 * tq + 1];
  }
  const int64_t n = (int64_t)g.nx * g.ny;
  const int64_t nchunks = (n + 15) / 16;
  const uint32_t* src = reinterpret_cast<const uint32_t*>(a1);
  uint32_t* dst = reinterpret_cast<uint32_t*>(a2);
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t ch = wid; ch < nchunks; ch += nw) {
    const int64_t pA = ch * 16 + gq, pB = pA + 8;
    const bool okA = pA < n, okB = pB < n;
    const int xA = grid_x(g, pA), yA = grid_y(g, pA), xB = grid_x(g, pB), yB = grid_y(g, pB);
    float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const int dx = k % 3 - 1, dy = k / 3 - 1;
      uint32_t a[4];
      a[0] = ld_pair(src, g, xA + dx, yA + dy, okA, tq);
      a[1] = ld_pair(src, g, xB + dx, yB + dy, okB, tq);
      a[2] = ld_pair(src, g, xA + dx, yA + dy, okA, tq + 4);
      a[3] = ld_pair(src, g, xB + dx, yB + dy, okB, tq + 4);
      mma_bf16(acc[0], a, bf[k][0]);
      mma_bf16(acc[1], a, bf[k][1]);
    }
#pragma unroll
    for (int nb = 0; nb < 2; ++nb) {
      if (okA) dst[pA * 8 + nb * 4 + tq] = pack_bf2(fmaxf(acc[nb][0] + bb[nb][0], 0.f), fmaxf(acc[nb][1] + bb[nb][1], 0.f));
      if (okB) dst[pB * 8 + nb * 4 + tq] = pack_bf2(fmaxf(acc[nb][2] + bb[nb][0], 0.f), fmaxf(acc[nb][3] + bb[nb][1], 0.f));
    }
  }
}

// data gradient: g1[p][ci] = [a1[p][ci] > 0] sum_k sum_co w2[co][ci][k] g2[p - tap][co]; GEMM per tap
// with M = 16 pixels, N = 16 input channels, K = 16 output channels
__global__ void __launch_bounds__(256) k_l2_bwd_data(const __nv_bfloat16* __restrict__ g2,
                                                     const __nv_bfloat16* __restrict__ wq,
                                                     const __nv_bfloat16* __restrict__ a1, Grid g,
                                                     __nv_bfloat16* __restrict__ g1) {
  __shared__ uint16_t w[kCh * kCh * 9];
  const uint16_t* wraw = reinterpret_cast<const uint16_t*>(wq);
  for (int k = threadIdx.x; k < kCh * kCh * 9; k += blockDim.x) w[k] = wraw[k];
  __syncthreads();
  const int lane = threadIdx.x & 31, gq = lane >> 2, tq = lane & 3;
  // B[k = co][n = ci] = w2[co][ci][tap]
  uint32_t bf[9][2][2];
#pragma unroll
  for (int k = 0; k < 9; ++k)
#pragma unroll
    for (int nb = 0; nb < 2; ++nb) {
      const int ci = nb * 8 + gq;
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const int co = 2 * tq + 8 * r;
        bf[k][nb][r] = pack_raw(w[(co * kCh + ci) * 9 + k], w[((co + 1) * kCh + ci) * 9 + k]);
      }
    }
  const int64_t n = (int64_t)g.nx * g.ny;
  const int64_t nchunks = (n + 15) / 16;
  const uint32_t* src = reinterpret_cast<const uint32_t*>(g2);
  const uint32_t* act = reinterpret_cast<const uint32_t*>(a1);
  uint32_t* dst = reinterpret_cast<uint32_t*>(g1);
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t ch = wid; ch < nchunks; ch += nw) {
    const int64_t pA = ch * 16 + gq, pB = pA + 8;
    const bool okA = pA < n, okB = pB < n;
    const int xA = grid_x(g, pA), yA = grid_y(g, pA), xB = grid_x(g, pB), yB = grid_y(g, pB);
    float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const int dx = k % 3 - 1, dy = k / 3 - 1;
      uint32_t a[4];
      a[0] = ld_pair(src, g, xA - dx, yA - dy, okA, tq);
      a[1] = ld_pair(src, g, xB - dx, yB - dy, okB, tq);
      a[2] = ld_pair(src, g, xA - dx, yA - dy, okA, tq + 4);
      a[3] = ld_pair(src, g, xB - dx, yB - dy, okB, tq + 4);
      mma_bf16(acc[0], a, bf[k][0]);
      mma_bf16(acc[1], a, bf[k][1]);
    }
#pragma unroll
    for (int nb = 0; nb < 2; ++nb) {
      const int h = nb * 4 + tq;
      if (okA) {
        const __nv_bfloat162 m = *reinterpret_cast<const __nv_bfloat162*>(&act[pA * 8 + h]);
        dst[pA * 8 + h] = pack_bf2(__low2float(m) > 0.f ? acc[nb][0] : 0.f, __high2float(m) > 0.f ? acc[nb][1] : 0.f);
      }
      if (okB) {
        const __nv_bfloat162 m = *reinterpret_cast<const __nv_bfloat162*>(&act[pB * 8 + h]);
        dst[pB * 8 + h] = pack_bf2(__low2float(m) > 0.f ? acc[nb][2] : 0.f, __high2float(m) > 0.f ? acc[nb][3] : 0.f);
      }
    }
  }
}

// bf16 value of channel c at pixel (x, y), zero outside the grid or past the last pixel
__device__ __forceinline__ uint16_t ld_ch(const uint16_t* __restrict__ a, Grid g, int64_t p, int64_t n, int dx, int dy,
                                          int c) {
  if (p >= n) return 0;
  const int x = grid_x(g, p) + dx, y = grid_y(g, p) + dy;
  return ginside(g, x, y) ? a[gnode(g, x, y) * kCh + c] : (uint16_t)0;
}

// weight gradient: gw2[co][ci][k] = sum_p g2[p][co] a1[p + tap][ci]; GEMM per tap with M = 16 output
// channels, N = 16 input channels, K = 16 pixels.  Each warp writes its own partial sums (one row of
// kNW2 values per warp, bias gradients last).
__global__ void __launch_bounds__(kWarpsW * 32, 1) k_l2_bwd_w(const __nv_bfloat16* __restrict__ g2,
                                                           const __nv_bfloat16* __restrict__ a1, Grid g,
                                                           double* __restrict__ partials) {
  const int lane = threadIdx.x & 31, gq = lane >> 2, tq = lane & 3;
  const int64_t n = (int64_t)g.nx * g.ny;
  const int64_t nchunks = (n + 15) / 16;
  const uint16_t* gr = reinterpret_cast<const uint16_t*>(g2);
  const uint16_t* ar = reinterpret_cast<const uint16_t*>(a1);
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  float acc[9][2][4];
#pragma unroll
  for (int k = 0; k < 9; ++k)
#pragma unroll
    for (int nb = 0; nb < 2; ++nb)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[k][nb][r] = 0.f;
  float bsum[2] = {0.f, 0.f};
  for (int64_t ch = wid; ch < nchunks; ch += nw) {
    const int64_t p0 = ch * 16;
    // pixels of this lane's K columns: 2t, 2t + 1, 2t + 8, 2t + 9
    const int64_t pk[4] = {p0 + 2 * tq, p0 + 2 * tq + 1, p0 + 2 * tq + 8, p0 + 2 * tq + 9};
    // A[m = co][k = pixel] = g2[pixel][co]
    uint16_t ga[2][4];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int j = 0; j < 4; ++j) ga[r][j] = pk[j] < n ? gr[pk[j] * kCh + gq + 8 * r] : (uint16_t)0;
    uint32_t a[4];
    a[0] = pack_raw(ga[0][0], ga[0][1]);
    a[1] = pack_raw(ga[1][0], ga[1][1]);
    a[2] = pack_raw(ga[0][2], ga[0][3]);
    a[3] = pack_raw(ga[1][2], ga[1][3]);
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const uint32_t u = (uint32_t)ga[r][j] << 16;
        bsum[r] += __uint_as_float(u);
      }
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const int dx = k % 3 - 1, dy = k / 3 - 1;
#pragma unroll
      for (int nb = 0; nb < 2; ++nb) {
        const int ci = nb * 8 + gq;
        // B[k = pixel][n = ci] = a1[pixel + tap][ci]
        uint32_t b[2];
        b[0] = pack_raw(ld_ch(ar, g, pk[0], n, dx, dy, ci), ld_ch(ar, g, pk[1], n, dx, dy, ci));
        b[1] = pack_raw(ld_ch(ar, g, pk[2], n, dx, dy, ci), ld_ch(ar, g, pk[3], n, dx, dy, ci));
        mma_bf16(acc[k][nb], a, b);
      }
    }
  }
  // bias sums: lanes with the same g hold the four pixels' shares of channels g and g + 8
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    bsum[r] += __shfl_xor_sync(0xffffffffu, bsum[r], 1);
    bsum[r] += __shfl_xor_sync(0xffffffffu, bsum[r], 2);
  }
  double* row = partials + (size_t)wid * kNW2;
#pragma unroll
  for (int k = 0; k < 9; ++k)
#pragma unroll
    for (int nb = 0; nb < 2; ++nb) {
      const int ci = nb * 8 + 2 * tq;
      row[(gq * kCh + ci) * 9 + k] = acc[k][nb][0];
      row[(gq * kCh + ci + 1) * 9 + k] = acc[k][nb][1];
      row[((gq + 8) * kCh + ci) * 9 + k] = acc[k][nb][2];
      row[((gq + 8) * kCh + ci + 1) * 9 + k] = acc[k][nb][3];
    }
  if (tq == 0) {
    row[kCh * kCh * 9 + gq] = bsum[0];
    row[kCh * kCh * 9 + gq + 8] = bsum[1];
  }
}

// grad[k] += sum over rows of partials[.][k] (fixed order)
__global__ void k_rows_sum(const double* __restrict__ partials, int nrows, int nv, double* __restrict__ grad) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nv; k += gridDim.x * blockDim.x) {
    double t = 0.0;
    for (int b = 0; b < nrows; ++b) t += partials[(size_t)b * nv + k];
    grad[k] += t;
  }
}

// Adam (Kingma and Ba) on the fp32 master parameters; the bf16 copy is what the kernels read
__global__ void k_adam(float* __restrict__ th, const double* __restrict__ gr, float* __restrict__ m1,
                       float* __restrict__ m2, __nv_bfloat16* __restrict__ thq, int nw, float lr, float b1, float b2,
                       float eps, int t) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nw) return;
  const float gk = (float)gr[k];
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
