// FIRLS_L1 with a dense sensing matrix (Sec. 5.2-5.3: random projections).
//
// The hot operator is S d = A^T (A d) + lambda W d.  A is streamed once per
// application: a CTA takes a chunk of rows, and for every group of R rows it
// forms the row products A_i . d (each thread over its own columns, then one
// block-wide reduction), then scatters them back, q += (A_i . d) A_i, from the
// same registers.  The chunk's partial q goes to qpart; one CTA per problem
// then sums the partials in a fixed order and runs the whole PCG step on the
// problem's short vectors (alpha, the x / r update, z = P^{-1} r, beta, the
// next direction), including the end of the outer step.  FP32 operators,
// FP64 inner products and PCG scalars (the SliceState helpers shared with the
// Fourier path).
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "firls.h"
#include "firls_common.cuh"

using namespace firls;

namespace {

constexpr int RT = 256;   // threads of the row kernel
constexpr int PT = 1024;  // threads of the per-problem PCG kernel

// Which problems a row pass serves and what it multiplies.
enum DenseRows {
  DR_X = 0,    // problems at the start of an outer step (PH_BOUNDARY): v = x
  DR_D = 1,    // problems in PCG (PH_PCG): v = d
  DR_ATB = 2,  // every problem, coefficients b_i instead of row products: A^T b
  DR_ALL = 3   // every problem, v = d (operator-level A^T A d)
};

template <int K4>
struct RowsPerIter {
  static constexpr int R = K4 >= 8 ? 2 : 4;
};

// qpart[p][c][:] = sum over the rows i of chunk c of coef_i A_i, coef_i =
// A_i . v_p (or b_i).  Thread t owns the float4 columns t + RT k, k < K4.
template <int K4>
__global__ void __launch_bounds__(RT) k_dense_rows(int M, int N, int CH, int shared, int mode,
                                                   const SliceState* __restrict__ st, const float* __restrict__ A,
                                                   const float* __restrict__ v, const float* __restrict__ b,
                                                   float* __restrict__ qpart) {
  constexpr int R = RowsPerIter<K4>::R;
  const int p = blockIdx.y, c = blockIdx.x, t = threadIdx.x;
  if (mode == DR_X || mode == DR_D) {
    if (!slice_running(st, p)) return;
    if (st[p].phase != (mode == DR_X ? PH_BOUNDARY : PH_PCG)) return;
  }
  const int N4 = N >> 2;
  const float4* A4 = reinterpret_cast<const float4*>(A + (shared ? (size_t)0 : (size_t)p * M * N));
  const float4* v4 = reinterpret_cast<const float4*>(v + (size_t)p * N);
  const int per = (M + CH - 1) / CH;
  const int r0 = c * per, r1 = min(M, r0 + per);
  float4 vr[K4], qr[K4];
#pragma unroll
  for (int k = 0; k < K4; ++k) {
    const int f = t + RT * k;
    vr[k] = (mode != DR_ATB && f < N4) ? v4[f] : make_float4(0.f, 0.f, 0.f, 0.f);
    qr[k] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  __shared__ float red[2][R][RT / 32];
  const int lane = t & 31, warp = t >> 5;
  int it = 0;
  for (int i = r0; i < r1; i += R, ++it) {
    float4 a[R][K4];
    float coef[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int row = i + r;
      float dot = 0.f;
#pragma unroll
      for (int k = 0; k < K4; ++k) {
        const int f = t + RT * k;
        if (row < r1 && f < N4) {
          // a private matrix is read once per application: stream it past L1
          a[r][k] = shared ? __ldg(A4 + (size_t)row * N4 + f) : __ldcs(A4 + (size_t)row * N4 + f);
        } else {
          a[r][k] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        dot = fmaf(a[r][k].x, vr[k].x, dot);
        dot = fmaf(a[r][k].y, vr[k].y, dot);
        dot = fmaf(a[r][k].z, vr[k].z, dot);
        dot = fmaf(a[r][k].w, vr[k].w, dot);
      }
      coef[r] = dot;
    }
    if (mode == DR_ATB) {
#pragma unroll
      for (int r = 0; r < R; ++r) coef[r] = (i + r < r1) ? b[(size_t)p * M + i + r] : 0.f;
    } else {
      // block-wide sums of the R row products (red alternates by iteration,
      // so one barrier per iteration keeps writes and reads apart)
#pragma unroll
      for (int r = 0; r < R; ++r) {
        float s = coef[r];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) red[it & 1][r][warp] = s;
      }
      __syncthreads();
#pragma unroll
      for (int r = 0; r < R; ++r) {
        float s = 0.f;
#pragma unroll
        for (int w = 0; w < RT / 32; ++w) s += red[it & 1][r][w];
        coef[r] = s;
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int k = 0; k < K4; ++k) {
        qr[k].x = fmaf(coef[r], a[r][k].x, qr[k].x);
        qr[k].y = fmaf(coef[r], a[r][k].y, qr[k].y);
        qr[k].z = fmaf(coef[r], a[r][k].z, qr[k].z);
        qr[k].w = fmaf(coef[r], a[r][k].w, qr[k].w);
      }
  }
  float4* out = reinterpret_cast<float4*>(qpart + ((size_t)p * CH + c) * N);
#pragma unroll
  for (int k = 0; k < K4; ++k) {
    const int f = t + RT * k;
    if (f < N4) out[f] = qr[k];
  }
}

typedef void (*RowsKernel)(int, int, int, int, int, const SliceState*, const float*, const float*, const float*,
                           float*);
RowsKernel rows_kernel(int N) {
  const int k4 = ((N >> 2) + RT - 1) / RT;
  if (k4 <= 1) return k_dense_rows<1>;
  if (k4 <= 2) return k_dense_rows<2>;
  if (k4 <= 4) return k_dense_rows<4>;
  return k_dense_rows<8>;
}

// Sum of the chunk partials of element i of problem p, in chunk order.
FI float qsum(const float* qpart, int p, int CH, int N, int i) {
  const float* q = qpart + (size_t)p * CH * N + i;
  float s = 0.f;
  for (int c = 0; c < CH; ++c) s += q[(size_t)c * N];
  return s;
}

// Block-wide FP64 sum broadcast to every thread.
FI double bsum(double v, double* red, double* out) {
  const double s = block_sum(v, red);
  if (threadIdx.x == 0) *out = s;
  __syncthreads();
  return *out;
}

// A^T A d = the summed partials (operator-level entry point).
__global__ void k_dense_reduce(int N, int CH, const float* __restrict__ qpart, float* __restrict__ q) {
  const int p = blockIdx.y;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
    q[(size_t)p * N + i] = qsum(qpart, p, CH, N, i);
}

// A^T b, ||A^T b||^2 and the initial state of every problem.
__global__ void __launch_bounds__(PT) k_dense_setup(int N, int CH, const float* __restrict__ qpart,
                                                    float* __restrict__ atb, float* __restrict__ x, int set_x,
                                                    SliceState* __restrict__ st, const float* __restrict__ lam,
                                                    const float* __restrict__ abar, int shared, float eps,
                                                    int outer_max) {
  const int p = blockIdx.x;
  __shared__ double red[32];
  __shared__ double bc;
  double s2 = 0.0;
  for (int i = threadIdx.x; i < N; i += PT) {
    const float v = qsum(qpart, p, CH, N, i);
    atb[(size_t)p * N + i] = v;
    if (set_x) x[(size_t)p * N + i] = v;
    s2 += (double)v * v;
  }
  const double rhs2 = bsum(s2, red, &bc);
  if (threadIdx.x == 0) {
    SliceState v;
    memset(&v, 0, sizeof v);
    v.rhs2 = rhs2;
    v.rr = rhs2;
    v.rr0 = rhs2;
    const bool bad = !isfinite(rhs2);
    v.active = bad ? 0 : 1;
    v.done = bad ? 1 : 0;
    v.breakdown = bad ? 1 : 0;
    v.lam = lam[p];
    v.abar = abar[shared ? 0 : p];
    v.eps = eps;
    v.phase = PH_BOUNDARY;
    v.outer_max = outer_max;
    st[p] = v;
  }
}

enum DensePcg { DP_INIT = 0, DP_STEP = 1 };

// One PCG step of problem p (or the start of its outer step), on its whole
// vectors; ends the outer step in place when its PCG stops.
__global__ void __launch_bounds__(PT) k_dense_pcg(int N, int CH, int mode, SliceState* __restrict__ st,
                                                  const float* __restrict__ qpart, float* __restrict__ x,
                                                  float* __restrict__ dx, float* __restrict__ r,
                                                  float* __restrict__ z, float* __restrict__ d,
                                                  float* __restrict__ q, float* __restrict__ w,
                                                  float* __restrict__ pinv, const float* __restrict__ atb,
                                                  const float* __restrict__ dAtA, int shared, int precond,
                                                  PcgSched ps, float outer_tol) {
  const int p = blockIdx.x;
  if (!slice_running(st, p)) return;
  const int ph = st[p].phase;
  if (ph != (mode == DP_INIT ? PH_BOUNDARY : PH_PCG)) return;
  __shared__ double red[32];
  __shared__ double bc;
  __shared__ int phase_s;
  SliceState* v = st + p;
  const size_t o = (size_t)p * N;
  const float lam = v->lam, eps = v->eps, abar = v->abar;
  const float* dg = dAtA + (shared ? (size_t)0 : o);
  if (mode == DP_INIT) {
    // W and P from x^k, r_0 = A^T b - S x^k, z_0 = P^{-1} r_0, d_0 = z_0
    double rz = 0.0, rr = 0.0;
    for (int i = threadIdx.x; i < N; i += PT) {
      const float xi = x[o + i];
      const float wi = rsqrtf(fmaf(xi, xi, eps));
      const float pd = precond == FIRLS_PRECOND_JACOBI ? dg[i] + lam * wi
                       : precond == FIRLS_PRECOND_NONE ? 1.f
                                                       : abar + lam * wi;
      const float pi = 1.f / pd;
      w[o + i] = wi;
      pinv[o + i] = pi;
      const float ri = atb[o + i] - (qsum(qpart, p, CH, N, i) + lam * wi * xi);
      const float zi = pi * ri;
      r[o + i] = ri;
      z[o + i] = zi;
      d[o + i] = zi;
      rz += (double)ri * zi;
      rr += (double)ri * ri;
    }
    rz = bsum(rz, red, &bc);
    rr = bsum(rr, red, &bc);
    if (threadIdx.x == 0) pcg_rho_init_from(v, rz, rr);
    return;
  }
  // q = S d, alpha = rho / <d, q>
  double dq = 0.0;
  for (int i = threadIdx.x; i < N; i += PT) {
    const float di = d[o + i];
    const float qi = qsum(qpart, p, CH, N, i) + lam * w[o + i] * di;
    q[o + i] = qi;
    dq += (double)di * qi;
  }
  dq = bsum(dq, red, &bc);
  if (threadIdx.x == 0) {
    pcg_alpha_from(v, dq);
    phase_s = v->done ? -1 : v->phase;
  }
  __syncthreads();
  if (phase_s < 0) return;  // breakdown: x keeps x^k
  if (phase_s == PH_PCG) {
    const float alpha = (float)v->alpha;
    double rz = 0.0, rr = 0.0;
    for (int i = threadIdx.x; i < N; i += PT) {
      dx[o + i] = fmaf(alpha, d[o + i], dx[o + i]);
      const float ri = fmaf(-alpha, q[o + i], r[o + i]);
      const float zi = pinv[o + i] * ri;
      r[o + i] = ri;
      z[o + i] = zi;
      rz += (double)ri * zi;
      rr += (double)ri * ri;
    }
    rz = bsum(rz, red, &bc);
    rr = bsum(rr, red, &bc);
    if (threadIdx.x == 0) {
      pcg_beta_from(v, rz, rr, ps);
      phase_s = v->phase;
    }
    __syncthreads();
    if (phase_s == PH_PCG) {
      const float beta = (float)v->beta;
      for (int i = threadIdx.x; i < N; i += PT) d[o + i] = fmaf(beta, d[o + i], z[o + i]);
      return;
    }
  }
  // end of the outer step: x^{k+1} = x^k + dx, relative change, stop
  double xx = 0.0, dd = 0.0;
  for (int i = threadIdx.x; i < N; i += PT) {
    const float xi = x[o + i], di = dx[o + i];
    xx += (double)xi * xi;
    dd += (double)di * di;
    x[o + i] = xi + di;
    dx[o + i] = 0.f;
  }
  xx = bsum(xx, red, &bc);
  dd = bsum(dd, red, &bc);
  if (threadIdx.x == 0) {
    const double rel = xx > 0.0 ? sqrt(dd / xx) : INFINITY;
    v->relchg = rel;
    v->outer_done += 1;
    if ((outer_tol > 0.f && rel <= (double)outer_tol) || v->outer_done >= v->outer_max) v->done = 1;
    else v->phase = PH_BOUNDARY;
  }
}

// diag(A^T A)_j = sum_i A_ij^2 per matrix (thread per column, rows in order).
__global__ void k_dense_colsq(int M, int N, const float* __restrict__ A, float* __restrict__ dAtA) {
  const int m = blockIdx.y;
  const float* Am = A + (size_t)m * M * N;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int i = 0; i < M; ++i) {
      const double a = Am[(size_t)i * N + j];
      s += a * a;
    }
    dAtA[(size_t)m * N + j] = (float)s;
  }
}

// abar = tr(A^T A) / N per matrix (Eq. ps).
__global__ void k_dense_abar(int N, const float* __restrict__ dAtA, float* __restrict__ abar, double* __restrict__ abar64) {
  const int m = blockIdx.x;
  __shared__ double red[32];
  double s = 0.0;
  for (int j = threadIdx.x; j < N; j += blockDim.x) s += dAtA[(size_t)m * N + j];
  s = block_sum(s, red);
  if (threadIdx.x == 0) {
    abar64[m] = s / N;
    abar[m] = (float)(s / N);
  }
}

// ---- shared matrix: S d for all problems as two register-tiled GEMMs ----
// With one A for every problem, A^T A d_p for all p is T = D A^T (P x M)
// then Q = T A (P x N): dense contractions in which a loaded tile of A serves
// 128 problems.  C[m][n] = sum_k X[m][k] Y(k, n) over one split of K, X
// row-major with K contiguous; Y(k, n) = B[n ldb + k] (YT) or B[k ldb + n].
// A CTA computes a 128 x 128 tile (each thread 8 rows x 8 columns: columns
// 4 tx .. 4 tx + 3 and 64 + 4 tx .. 64 + 4 tx + 3, so that the eight threads
// of a quarter warp read 128 consecutive bytes of the Y slab, free of bank
// conflicts) from 8-deep slabs staged in shared memory, the next slab's loads
// in flight while the current one is used.  FP32 throughout; the split
// partials are summed in split order by the next stage.
constexpr int GM = 128, GN = 128, GK = 8, GT = 256;

template <bool YT>
__global__ void __launch_bounds__(GT, 2) k_dense_gemm(int Mg, int Ng, int K, int kper, const float* __restrict__ X,
                                                      int ldx, const float* __restrict__ B, int ldb,
                                                      float* __restrict__ C, int ldc, size_t split_stride) {
  __shared__ __align__(16) float Xs[2][GK][GM + 4];
  __shared__ __align__(16) float Ys[2][GK][GN + 4];
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int bm = blockIdx.y * GM, bn = blockIdx.x * GN, sp = blockIdx.z;
  const int k0 = sp * kper, k1 = min(K, k0 + kper);
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
  float4 px, py;
  // X slab: 128 rows x 8 k, one float4 (4 k) per thread
  const int xr = tid / 2, xk = (tid % 2) * 4;
  auto load_x = [&](int k) {
    px = (bm + xr < Mg && k + xk < k1) ? *reinterpret_cast<const float4*>(X + (size_t)(bm + xr) * ldx + k + xk)
                                       : make_float4(0.f, 0.f, 0.f, 0.f);
  };
  auto store_x = [&](int buf) {
    Xs[buf][xk][xr] = px.x;
    Xs[buf][xk + 1][xr] = px.y;
    Xs[buf][xk + 2][xr] = px.z;
    Xs[buf][xk + 3][xr] = px.w;
  };
  // Y slab: 8 k x 128 n, one float4 per thread
  auto load_y = [&](int k) {
    if (YT) {
      const int n = tid / 2, kq = (tid % 2) * 4;
      py = (bn + n < Ng && k + kq < k1) ? *reinterpret_cast<const float4*>(B + (size_t)(bn + n) * ldb + k + kq)
                                        : make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
      const int kk = tid / 32, nq = (tid % 32) * 4;
      py = (k + kk < k1 && bn + nq < Ng) ? *reinterpret_cast<const float4*>(B + (size_t)(k + kk) * ldb + bn + nq)
                                         : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  };
  auto store_y = [&](int buf) {
    if (YT) {
      const int n = tid / 2, kq = (tid % 2) * 4;
      Ys[buf][kq][n] = py.x;
      Ys[buf][kq + 1][n] = py.y;
      Ys[buf][kq + 2][n] = py.z;
      Ys[buf][kq + 3][n] = py.w;
    } else {
      const int kk = tid / 32, nq = (tid % 32) * 4;
      *reinterpret_cast<float4*>(&Ys[buf][kk][nq]) = py;
    }
  };
  int buf = 0;
  if (k0 < k1) {
    load_x(k0);
    load_y(k0);
    store_x(0);
    store_y(0);
  }
  __syncthreads();
  for (int k = k0; k < k1; k += GK) {
    const bool more = k + GK < k1;
    if (more) {  // the next slab's loads fly while this one is multiplied
      load_x(k + GK);
      load_y(k + GK);
    }
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&Xs[buf][kk][ty * 8]);
      const float4 a1 = *reinterpret_cast<const float4*>(&Xs[buf][kk][ty * 8 + 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Ys[buf][kk][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Ys[buf][kk][64 + tx * 4]);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    if (more) {
      store_x(buf ^ 1);
      store_y(buf ^ 1);
    }
    __syncthreads();
    buf ^= 1;
  }
  // Ng, ldc and split_stride are multiples of 4 (M % 4 = N % 4 = 0 on this
  // path), so each group of four columns is one aligned float4, whole or out.
  float* Cs = C + (size_t)sp * split_stride;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int m = bm + ty * 8 + i;
    if (m >= Mg) continue;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int n = bn + h * 64 + tx * 4;
      if (n < Ng)
        *reinterpret_cast<float4*>(Cs + (size_t)m * ldc + n) =
            make_float4(acc[i][4 * h], acc[i][4 * h + 1], acc[i][4 * h + 2], acc[i][4 * h + 3]);
    }
  }
}

// Splits of K for a product of `tiles` output tiles with `slots` resident
// CTAs on the device: the count that minimises (waves of CTAs) x (slabs per
// CTA + 2), the 2 standing for a CTA's epilogue and the partial its split
// adds to the sum; at least 4 slabs per split, fewest splits on ties.
int gemm_splits(int tiles, int K, int slots) {
  int best = 1;
  long best_cost = -1;
  for (int S = 1; S <= std::max(1, K / (4 * GK)); ++S) {
    const int kper = ((K + S - 1) / S + GK - 1) / GK * GK;
    const long waves = ((long)tiles * S + slots - 1) / slots;
    const long cost = waves * (kper / GK + 2);
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      best = S;
    }
  }
  return best;
}

// T[p][i] = sum over the splits of Tpart[s][p][i] (split order).
__global__ void k_dense_sum_splits(int count, int S, const float* __restrict__ part, float* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    float a = 0.f;
    for (int sp = 0; sp < S; ++sp) a += part[(size_t)sp * count + i];
    out[i] = a;
  }
}

}  // namespace

struct firls_dense_ctx {
  int M = 0, N = 0, P = 0, shared = 0, nA = 0, CH = 1;
  // shared matrix with M % 4 == 0: the GEMM form (S1 splits of K = N in the
  // first product; CH splits of K = M in the second, the partials of q)
  bool gemm = false;
  int S1 = 1;
  float *tpart = nullptr, *tmat = nullptr;
  cudaStream_t stream = nullptr;
  bool matrix_set = false;
  float *A = nullptr, *dAtA = nullptr, *abar = nullptr;
  double* abar64 = nullptr;
  float *atb = nullptr, *x = nullptr, *dx = nullptr, *r = nullptr, *z = nullptr, *d = nullptr, *q = nullptr;
  float *w = nullptr, *pinv = nullptr, *qpart = nullptr, *lam = nullptr;
  SliceState* st = nullptr;
  std::vector<void*> allocs;
  std::string err;
  cudaGraphExec_t graph = nullptr;
  int graph_J = -1, graph_precond = -1;
  float graph_tol = -1.f, graph_otol = -1.f;
};

namespace {

firls_status dfail(firls_dense_ctx* c, firls_status s, const std::string& m) {
  if (c) c->err = m;
  return s;
}

firls_status dcheck(firls_dense_ctx* c, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return FIRLS_OK;
  return dfail(c, FIRLS_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define DTRY(expr)                       \
  do {                                   \
    const firls_status s_ = (expr);      \
    if (s_ != FIRLS_OK) return s_;       \
  } while (0)
#define DCU(expr) DTRY(dcheck(c, (expr), #expr))

template <typename T> firls_status dalloc(firls_dense_ctx* c, T** p, size_t count) {
  if (cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * (count ? count : 1)) != cudaSuccess) {
    cudaGetLastError();
    return dfail(c, FIRLS_E_NOMEM, "device allocation failed");
  }
  c->allocs.push_back(*p);
  return FIRLS_OK;
}

// Row chunks per problem: enough CTAs for several per SM, each with a few
// row groups to stream.
int chunks_for(int M, int P) {
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int want = (4 * sms + P - 1) / P;
  const int cap = M / 16 > 1 ? M / 16 : 1;
  return want < 1 ? 1 : (want > cap ? cap : want);
}

// q partials of A^T A v (or A^T b) per problem.  The GEMM form computes them
// for every problem (the PCG kernel reads only the problems it serves).
void launch_rows(firls_dense_ctx* c, int mode, const float* v, const float* b) {
  if (!c->gemm) {
    rows_kernel(c->N)<<<dim3(c->CH, c->P), RT, 0, c->stream>>>(c->M, c->N, c->CH, c->shared, mode, c->st, c->A,
                                                                 v, b, c->qpart);
    return;
  }
  const int M = c->M, N = c->N, P = c->P;
  const float* t = c->tmat;
  if (mode == DR_ATB) {
    cudaMemcpyAsync(c->tmat, b, sizeof(float) * (size_t)P * M, cudaMemcpyDeviceToDevice, c->stream);
  } else {
    // T = V A^T over S1 splits of N, then their sum
    const int kper1 = ((N + c->S1 - 1) / c->S1 + GK - 1) / GK * GK;
    k_dense_gemm<true><<<dim3((M + GN - 1) / GN, (P + GM - 1) / GM, c->S1), GT, 0, c->stream>>>(
        P, M, N, kper1, v, N, c->A, N, c->tpart, M, (size_t)P * M);
    const int cnt = P * M;
    k_dense_sum_splits<<<(cnt + 255) / 256 < 1024 ? (cnt + 255) / 256 : 1024, 256, 0, c->stream>>>(cnt, c->S1,
                                                                                                    c->tpart, c->tmat);
  }
  // q partials = T A over CH splits of M: partial s of problem p at qpart[(p CH + s) N]
  const int kper2 = ((M + c->CH - 1) / c->CH + GK - 1) / GK * GK;
  k_dense_gemm<false><<<dim3((N + GN - 1) / GN, (P + GM - 1) / GM, c->CH), GT, 0, c->stream>>>(
      P, N, M, kper2, t, M, c->A, N, c->qpart, c->CH * N, (size_t)N);
}

void launch_pcg(firls_dense_ctx* c, int mode, int precond, const PcgSched& ps, float outer_tol) {
  k_dense_pcg<<<c->P, PT, 0, c->stream>>>(c->N, c->CH, mode, c->st, c->qpart, c->x, c->dx, c->r, c->z, c->d, c->q,
                                           c->w, c->pinv, c->atb, c->dAtA, c->shared, precond, ps, outer_tol);
}

// One outer step: the start (S x^k, r_0, z_0) and J PCG steps; problems
// whose PCG has stopped skip the rest of the launches.
void enqueue_outer(firls_dense_ctx* c, int J, int precond, const PcgSched& ps, float outer_tol) {
  launch_rows(c, DR_X, c->x, nullptr);
  launch_pcg(c, DP_INIT, precond, ps, outer_tol);
  for (int j = 0; j < J; ++j) {
    launch_rows(c, DR_D, c->d, nullptr);
    launch_pcg(c, DP_STEP, precond, ps, outer_tol);
  }
}

firls_status dense_params_ok(firls_dense_ctx* c, const firls_params* p) {
  if (!p) return dfail(c, FIRLS_E_INVALID_ARG, "params is null");
  if (p->outer_iters < 1 || p->pcg_iters < 1) return dfail(c, FIRLS_E_INVALID_ARG, "iteration counts must be >= 1");
  if (!(p->pcg_tol >= 0.f) || !(p->outer_tol >= 0.f)) return dfail(c, FIRLS_E_INVALID_ARG, "tolerances must be >= 0");
  if (p->precond != FIRLS_PRECOND_PAPER && p->precond != FIRLS_PRECOND_JACOBI && p->precond != FIRLS_PRECOND_NONE)
    return dfail(c, FIRLS_E_INVALID_ARG, "dense A takes the PAPER, JACOBI or NONE preconditioner");
  if (p->lambda_tv != 0.f || p->lambda_tv_per_slice || p->outer_tol_kind || p->outer_stall_tol != 0.f ||
      p->pcg_tol_kind || p->pcg_iters_late || p->outer_late || p->boundary_period > 1)
    return dfail(c, FIRLS_E_INVALID_ARG, "a field the dense solver does not take is set");
  for (int s = 0; s < c->P; ++s) {
    const float l = p->lambda_per_slice ? p->lambda_per_slice[s] : p->lambda;
    if (!(l >= 0.f) || !std::isfinite(l)) return dfail(c, FIRLS_E_INVALID_ARG, "lambda must be finite and >= 0");
  }
  return FIRLS_OK;
}

}  // namespace

extern "C" firls_status firls_dense_create(firls_dense_ctx** out, int M, int N, int problems, int shared_matrix,
                                           void* cuda_stream) {
  if (!out) return FIRLS_E_INVALID_ARG;
  *out = nullptr;
  // problems index a grid dimension (<= 65535); P M and P N stay int-sized
  if (M < 1 || N < 4 || N > 8192 || N % 4 || problems < 1 || problems > 65535 ||
      (long long)problems * M > INT_MAX || (long long)problems * N > INT_MAX)
    return FIRLS_E_SHAPE;
  firls_dense_ctx* c = new firls_dense_ctx();
  c->M = M;
  c->N = N;
  c->P = problems;
  c->shared = shared_matrix ? 1 : 0;
  c->nA = c->shared ? 1 : problems;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  c->CH = chunks_for(M, problems);
  c->gemm = c->shared && M % 4 == 0;
  if (c->gemm) {  // splits of K sized to whole waves of resident CTAs
    int dev = 0, sms = 152, per_sm = 2;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int per_sm2 = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dense_gemm<true>, GT, 0) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm2, k_dense_gemm<false>, GT, 0) != cudaSuccess) {
      cudaGetLastError();
      per_sm = per_sm2 = 1;
    }
    per_sm = std::max(1, std::min(per_sm, per_sm2));
    const int tiles1 = ((M + GN - 1) / GN) * ((problems + GM - 1) / GM);
    const int tiles2 = ((N + GN - 1) / GN) * ((problems + GM - 1) / GM);
    c->S1 = gemm_splits(tiles1, N, per_sm * sms);
    c->CH = gemm_splits(tiles2, M, per_sm * sms);
  }
  const size_t PN = (size_t)problems * N;
  firls_status s = FIRLS_OK;
  auto al = [&](auto** p, size_t n) {
    if (s == FIRLS_OK) s = dalloc(c, p, n);
  };
  al(&c->A, (size_t)c->nA * M * N);
  al(&c->dAtA, (size_t)c->nA * N);
  al(&c->abar, (size_t)c->nA);
  al(&c->abar64, (size_t)c->nA);
  for (float** v : {&c->atb, &c->x, &c->dx, &c->r, &c->z, &c->d, &c->q, &c->w, &c->pinv}) al(v, PN);
  al(&c->qpart, PN * c->CH);
  if (c->gemm) {
    al(&c->tpart, (size_t)c->S1 * problems * M);
    al(&c->tmat, (size_t)problems * M);
  }
  al(&c->lam, (size_t)problems);
  al(&c->st, (size_t)problems);
  if (s != FIRLS_OK) {
    firls_dense_destroy(c);
    return s;
  }
  // problems never solved read as stopped
  if (cudaMemset(c->st, 0, sizeof(SliceState) * problems) != cudaSuccess ||
      cudaMemset(c->dx, 0, sizeof(float) * PN) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
    firls_dense_destroy(c);
    return FIRLS_E_CUDA;
  }
  *out = c;
  return FIRLS_OK;
}

extern "C" firls_status firls_dense_set_matrix(firls_dense_ctx* c, const float* A) {
  if (!c) return FIRLS_E_INVALID_ARG;
  if (!A) return dfail(c, FIRLS_E_INVALID_ARG, "A is null");
  if (reinterpret_cast<uintptr_t>(A) % 16) return dfail(c, FIRLS_E_INVALID_ARG, "A must be 16-byte aligned");
  c->matrix_set = false;
  DCU(cudaMemcpyAsync(c->A, A, sizeof(float) * (size_t)c->nA * c->M * c->N, cudaMemcpyDeviceToDevice, c->stream));
  k_dense_colsq<<<dim3((c->N + 255) / 256, c->nA), 256, 0, c->stream>>>(c->M, c->N, c->A, c->dAtA);
  k_dense_abar<<<c->nA, 256, 0, c->stream>>>(c->N, c->dAtA, c->abar, c->abar64);
  DCU(cudaGetLastError());
  DCU(cudaStreamSynchronize(c->stream));
  c->matrix_set = true;
  return FIRLS_OK;
}

extern "C" firls_status firls_dense_abar(firls_dense_ctx* c, double* out) {
  if (!c || !out) return FIRLS_E_INVALID_ARG;
  if (!c->matrix_set) return dfail(c, FIRLS_E_STATE, "matrix not set");
  DCU(cudaMemcpyAsync(out, c->abar64, sizeof(double) * c->nA, cudaMemcpyDeviceToHost, c->stream));
  DCU(cudaStreamSynchronize(c->stream));
  return FIRLS_OK;
}

extern "C" firls_status firls_dense_apply_AtA(firls_dense_ctx* c, const float* d, float* q) {
  if (!c || !d || !q) return FIRLS_E_INVALID_ARG;
  if (!c->matrix_set) return dfail(c, FIRLS_E_STATE, "matrix not set");
  if (reinterpret_cast<uintptr_t>(d) % 16) return dfail(c, FIRLS_E_INVALID_ARG, "d must be 16-byte aligned");
  launch_rows(c, DR_ALL, d, nullptr);
  k_dense_reduce<<<dim3((c->N + 255) / 256, c->P), 256, 0, c->stream>>>(c->N, c->CH, c->qpart, q);
  return dcheck(c, cudaGetLastError(), "apply_AtA");
}

extern "C" firls_status firls_dense_solve(firls_dense_ctx* c, const float* b, const firls_params* p,
                                          const float* x0, float* x_out, firls_stats* stats) {
  if (!c || !b || !x_out) return FIRLS_E_INVALID_ARG;
  if (!c->matrix_set) return dfail(c, FIRLS_E_STATE, "matrix not set");
  DTRY(dense_params_ok(c, p));
  const size_t PN = (size_t)c->P * c->N;
  std::vector<float> l(c->P);
  for (int s = 0; s < c->P; ++s) l[s] = p->lambda_per_slice ? p->lambda_per_slice[s] : p->lambda;
  DCU(cudaMemcpyAsync(c->lam, l.data(), sizeof(float) * c->P, cudaMemcpyHostToDevice, c->stream));
  DCU(cudaStreamSynchronize(c->stream));  // the host vector goes out of scope
  // A^T b (and x^1 = A^T b), ||A^T b||^2, the problems' states
  launch_rows(c, DR_ATB, c->x, b);
  const float eps = p->eps > 0.f ? p->eps : 1e-10f;
  k_dense_setup<<<c->P, PT, 0, c->stream>>>(c->N, c->CH, c->qpart, c->atb, c->x, x0 ? 0 : 1, c->st, c->lam, c->abar,
                                            c->shared, eps, p->outer_iters);
  if (x0) DCU(cudaMemcpyAsync(c->x, x0, sizeof(float) * PN, cudaMemcpyDeviceToDevice, c->stream));
  DCU(cudaMemsetAsync(c->dx, 0, sizeof(float) * PN, c->stream));
  DCU(cudaGetLastError());
  const PcgSched ps{p->pcg_tol, 0, p->pcg_iters, 0, 0};
  // one outer step as a graph, replayed (captured again when the schedule
  // changes); the legacy default stream cannot be captured: eager launches
  const bool use_graph = c->stream != nullptr;
  if (use_graph && (!c->graph || c->graph_J != p->pcg_iters || c->graph_precond != p->precond || c->graph_tol != p->pcg_tol ||
      c->graph_otol != p->outer_tol)) {
    if (c->graph) cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
    cudaGraph_t g = nullptr;
    DCU(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    enqueue_outer(c, p->pcg_iters, p->precond, ps, p->outer_tol);
    const cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    if (e != cudaSuccess) return dcheck(c, e, "capture");
    const cudaError_t e2 = cudaGraphInstantiate(&c->graph, g, 0);
    cudaGraphDestroy(g);
    if (e2 != cudaSuccess) {
      c->graph = nullptr;
      return dcheck(c, e2, "instantiate");
    }
    c->graph_J = p->pcg_iters;
    c->graph_precond = p->precond;
    c->graph_tol = p->pcg_tol;
    c->graph_otol = p->outer_tol;
  }
  std::vector<SliceState> h(c->P);
  auto read_states = [&]() -> firls_status {
    DCU(cudaMemcpyAsync(h.data(), c->st, sizeof(SliceState) * c->P, cudaMemcpyDeviceToHost, c->stream));
    DCU(cudaStreamSynchronize(c->stream));
    return FIRLS_OK;
  };
  const int poll = p->outer_tol > 0.f ? 8 : p->outer_iters;
  for (int k = 0; k < p->outer_iters;) {
    const int n = std::min(poll, p->outer_iters - k);
    for (int i = 0; i < n; ++i) {
      if (use_graph) DCU(cudaGraphLaunch(c->graph, c->stream));
      else enqueue_outer(c, p->pcg_iters, p->precond, ps, p->outer_tol);
    }
    DCU(cudaGetLastError());
    k += n;
    if (k < p->outer_iters) {
      DTRY(read_states());
      bool all = true;
      for (const SliceState& v : h) all = all && (v.done || !v.active);
      if (all) break;
    }
  }
  DCU(cudaMemcpyAsync(x_out, c->x, sizeof(float) * PN, cudaMemcpyDeviceToDevice, c->stream));
  DTRY(read_states());
  int nb = 0;
  firls_stats sv{};
  for (const SliceState& v : h) {
    nb += v.breakdown;
    sv.outer_done = std::max(sv.outer_done, v.outer_done);
    sv.pcg_steps += v.pcg_steps;
    sv.max_rel_change = std::max(sv.max_rel_change, v.relchg);
    if (v.rhs2 > 0.0) sv.max_rel_residual = std::max(sv.max_rel_residual, std::sqrt(v.rr / v.rhs2));
  }
  sv.n_breakdown = nb;
  if (stats) *stats = sv;
  if (nb) return dfail(c, FIRLS_E_BREAKDOWN, "PCG breakdown in " + std::to_string(nb) + " problem(s)");
  return FIRLS_OK;
}

extern "C" const char* firls_dense_last_error(const firls_dense_ctx* c) { return c ? c->err.c_str() : ""; }

extern "C" firls_status firls_dense_destroy(firls_dense_ctx* c) {
  if (!c) return FIRLS_E_INVALID_ARG;
  if (c->graph) cudaGraphExecDestroy(c->graph);
  for (void* v : c->allocs)
    if (v) cudaFree(v);
  delete c;
  return FIRLS_OK;
}
