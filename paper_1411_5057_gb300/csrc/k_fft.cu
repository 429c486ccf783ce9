// FFT-based kernels of A^H A = F^H R^T R F (Sec. 5.4: A = RF) and A^H b.
//
// A 2-D unitary FFT is a row pass and a column pass.  A^H A d runs as
//   row FFT of d  ->  column FFT, mask, column IFFT (one kernel)  ->
//   row IFFT fused with the rest of S d (TV stencil, wavelet term) and the
//   partial inner product Re<d, S d>.
// The unnormalised transforms are scaled once: 1/N for F^H R F, 1/n for
// F^H R b.  Rows: T threads of one warp per row (coalesced loads of
// t + T*s).  Columns: tiles of 16 columns x n rows staged in shared memory
// with 128-byte row segments.
#include "fft.cuh"
#include "launch.h"
#include "per_device.h"

namespace firls {

constexpr int COLS = 16;  // columns per column-pass CTA

template <int N> __host__ __device__ constexpr int rows_per_cta() {
  int r = 256 / FftCfg<N>::T;
  if (r > N) r = N;
  while (N % r) --r;
  return r;
}

// tv: staged d rows and TV weight rows; aniso (l1 TV): a second weight array
template <int N> constexpr int row_smem_bytes(bool tv, bool aniso = false) {
  constexpr int R = rows_per_cta<N>();
  int b = tw_bytes<N>() + R * 2 * fft_line_words<N>() * 4;
  if (tv) b += (R + 2) * N * 8 + (R + 1) * N * 4;
  if (tv && aniso) b += (R + 1) * N * 4;
  return b;
}

// Shared memory of a column-pass CTA: twiddles (padded table) | region | mask
// tile transposed ([COLS][N] bytes).  The region holds the N x COLS complex
// tile (rows of 16 float2, XOR-swizzled: element (r, c) at r*COLS + (c ^ (r
// mod COLS)), so that row-major fills and 16-row column reads are both free
// of bank conflicts) or, while the FFT runs, the per-column exchange lines.
template <int N> __host__ __device__ constexpr int col_region_bytes() {
  return N * COLS * 8 > COLS * 2 * fft_line_words<N>() * 4 ? N * COLS * 8 : COLS * 2 * fft_line_words<N>() * 4;
}
template <int N> __host__ __device__ constexpr int col_smem_bytes() {
  return tw_bytes<N>() + col_region_bytes<N>() + N * COLS;
}
FI int tslot(int r, int c) { return r * COLS + (c ^ (r & (COLS - 1))); }

FI void cp_async16_fft(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}

// The per-pass twiddle tables (see fft.cuh) from the global table
// twg[j] = exp(-2 pi i j / N).
template <int N> FI void load_twiddles(float2* tw, const float2* __restrict__ twg) {
  using C = FftCfg<N>;
  int P = C::radix(0);
#pragma unroll
  for (int p = 1; p < C::NP; ++p) {
    const int R = C::radix(p), step = N / (P * R), off = P - C::radix(0);
    for (int i = threadIdx.x; i < (R - 1) * P; i += blockDim.x) {
      const int q = i / P + 1, k = i % P;
      tw[off + i] = twg[q * k * step];
    }
    P *= R;
  }
}

// d = z (mode 0) | d = z + beta d (mode 1) | use d as is (mode 2) | per slice
// (mode < 0): d = x at the start of its outer step (S x^k), else d = z on the
// first PCG step and z + beta d after it; t = rowFFT(d)
template <int N>
__global__ void __launch_bounds__(256) k_row_fwd(const float2* __restrict__ z, float2* __restrict__ d,
                                                 float2* __restrict__ t_out,
                                                 const SliceState* __restrict__ st,
                                                 const float2* __restrict__ twg, int mode_arg,
                                                 const float2* __restrict__ x) {
  using C = FftCfg<N>;
  constexpr int R = rows_per_cta<N>(), E = C::E, T = C::T, LW = fft_line_words<N>();
  const int s = blockIdx.y;
  if (!slice_running(st, s)) return;
  int mode = mode_arg;
  if (mode_arg < 0) {
    const int ph = st[s].phase;
    if (ph != PH_START && ph != PH_PCG) return;  // waiting for its outer-step transition
    mode = ph == PH_START ? 3 : (st[s].pcg_j == 0 ? 0 : 1);
  }
  extern __shared__ __align__(16) unsigned char smem[];
  float2* tw = reinterpret_cast<float2*>(smem);
  float* lines = reinterpret_cast<float*>(smem + tw_bytes<N>());
  load_twiddles<N>(tw, twg);
  const int lr = threadIdx.x / T, t = threadIdx.x % T;
  const int row = blockIdx.x * R + lr;
  const size_t base = (size_t)s * N * N + (size_t)row * N;
  const float beta = (float)st[s].beta;
  float2 v[E];
  // one loop per mode, so that each touches only its own arrays
  if (mode == 1) {
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const size_t i = base + t + T * e;
      v[e] = cfma(beta, d[i], z[i]);
      d[i] = v[e];
    }
  } else if (mode == 0 || mode == 3) {
    const float2* __restrict__ src = mode == 0 ? z : x;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const size_t i = base + t + T * e;
      v[e] = src[i];
      d[i] = v[e];
    }
  } else {
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = d[base + t + T * e];
  }
  __syncthreads();
  fft_line<N, -1>(v, lines + lr * 2 * LW, lines + lr * 2 * LW + LW, tw, t);
#pragma unroll
  for (int e = 0; e < E; ++e) t_out[base + t + T * e] = v[e];
}

// t = rowIFFT(mask * b)
template <int N>
__global__ void __launch_bounds__(256) k_row_ahb(const float2* __restrict__ b, const uint8_t* __restrict__ mask,
                                                 float2* __restrict__ t_out,
                                                 const float2* __restrict__ twg) {
  using C = FftCfg<N>;
  constexpr int R = rows_per_cta<N>(), E = C::E, T = C::T, LW = fft_line_words<N>();
  const int s = blockIdx.y;
  extern __shared__ __align__(16) unsigned char smem[];
  float2* tw = reinterpret_cast<float2*>(smem);
  float* lines = reinterpret_cast<float*>(smem + tw_bytes<N>());
  load_twiddles<N>(tw, twg);
  const int lr = threadIdx.x / T, t = threadIdx.x % T;
  const int row = blockIdx.x * R + lr;
  const size_t base = (size_t)s * N * N + (size_t)row * N;
  float2 v[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const size_t i = base + t + T * e;
    v[e] = mask[i] ? b[i] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  fft_line<N, +1>(v, lines + lr * 2 * LW, lines + lr * 2 * LW + LW, tw, t);
#pragma unroll
  for (int e = 0; e < E; ++e) t_out[base + t + T * e] = v[e];
}

// Load a 16-column tile of t into shared memory (SoA, row stride COLS+1).
template <int N>
FI void load_col_tile(const float2* __restrict__ src, float2* tile, size_t sbase, int c0) {
  // every thread issues all its 16-byte loads (two columns each) before the
  // first shared-memory store, so a whole tile is in flight at once
  constexpr int NT = COLS * FftCfg<N>::T, HC = COLS / 2, K = N * HC / NT;
  static_assert(N * HC % NT == 0, "column tile split");
  float4 g[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int idx = threadIdx.x + NT * k, r = idx / HC, cp = idx % HC;
    g[k] = *reinterpret_cast<const float4*>(src + sbase + (size_t)r * N + c0 + 2 * cp);
  }
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int idx = threadIdx.x + NT * k, r = idx / HC, cp = idx % HC;
    tile[tslot(r, 2 * cp)] = make_float2(g[k].x, g[k].y);
    tile[tslot(r, 2 * cp + 1)] = make_float2(g[k].z, g[k].w);
  }
}

template <int N>
FI void store_col_tile(float2* __restrict__ dst, const float2* tile, size_t sbase, int c0) {
  constexpr int NT = COLS * FftCfg<N>::T, HC = COLS / 2, K = N * HC / NT;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int idx = threadIdx.x + NT * k, r = idx / HC, cp = idx % HC;
    const float2 a = tile[tslot(r, 2 * cp)], b = tile[tslot(r, 2 * cp + 1)];
    *reinterpret_cast<float4*>(dst + sbase + (size_t)r * N + c0 + 2 * cp) = make_float4(a.x, a.y, b.x, b.y);
  }
}

// The 16 mask bytes of each row of a column tile (one 16-byte load per row),
// stored transposed: mskt[c * N + r].
template <int N>
FI void load_mask_tile(const uint8_t* __restrict__ mask, uint8_t* mskt, size_t sbase, int c0) {
  constexpr int NT = COLS * FftCfg<N>::T;
  for (int r = threadIdx.x; r < N; r += NT) {
    const uint4 m = *reinterpret_cast<const uint4*>(mask + sbase + (size_t)r * N + c0);
    const unsigned w[4] = {m.x, m.y, m.z, m.w};
#pragma unroll
    for (int c = 0; c < COLS; ++c) mskt[c * N + r] = (uint8_t)(w[c >> 2] >> (8 * (c & 3)));
  }
}

// In place on t: t = colIFFT(mask * colFFT(t)) for a 16-column tile.
template <int N>
__global__ void __launch_bounds__(512) k_col_mask(float2* __restrict__ tbuf, const uint8_t* __restrict__ mask,
                                                  const SliceState* __restrict__ st,
                                                  const float2* __restrict__ twg) {
  using C = FftCfg<N>;
  constexpr int E = C::E, T = C::T, LW = fft_line_words<N>();
  const int s = blockIdx.y;
  if (st != nullptr && !slice_running(st, s)) return;
  extern __shared__ __align__(16) unsigned char smem[];
  float2* tw = reinterpret_cast<float2*>(smem);
  float2* tile = reinterpret_cast<float2*>(smem + tw_bytes<N>());
  uint8_t* mskt = smem + tw_bytes<N>() + col_region_bytes<N>();
  const int c0 = blockIdx.x * COLS;
  const size_t sbase = (size_t)s * N * N;
  load_twiddles<N>(tw, twg);
  load_mask_tile<N>(mask, mskt, sbase, c0);
  load_col_tile<N>(tbuf, tile, sbase, c0);
  __syncthreads();
  const int c = threadIdx.x / T, t = threadIdx.x % T;
  float2 v[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int r = t + T * e;
    v[e] = tile[tslot(r, c)];
  }
  __syncthreads();
  float* bre = reinterpret_cast<float*>(tile) + c * 2 * LW;
  float* bim = bre + LW;
  fft_line<N, -1>(v, bre, bim, tw, t);
#pragma unroll
  for (int e = 0; e < E; ++e)
    if (!mskt[c * N + t + T * e]) v[e] = make_float2(0.f, 0.f);
  fft_line<N, +1>(v, bre, bim, tw, t);
  __syncthreads();
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int r = t + T * e;
    tile[tslot(r, c)] = v[e];
  }
  __syncthreads();
  store_col_tile<N>(tbuf, tile, sbase, c0);
}

// atb = (1/n) colIFFT(t)  [real: imaginary part dropped]; x = atb if x != null;
// partial ||atb||^2.
template <int N>
__global__ void __launch_bounds__(512) k_col_inv(const float2* __restrict__ tbuf, float2* __restrict__ atb,
                                                 float2* __restrict__ x, int real,
                                                 double* __restrict__ part,
                                                 const float2* __restrict__ twg) {
  using C = FftCfg<N>;
  constexpr int E = C::E, T = C::T, LW = fft_line_words<N>();
  const int s = blockIdx.y;
  extern __shared__ __align__(16) unsigned char smem[];
  float2* tw = reinterpret_cast<float2*>(smem);
  float2* tile = reinterpret_cast<float2*>(smem + tw_bytes<N>());
  __shared__ double red[32];
  const int c0 = blockIdx.x * COLS;
  const size_t sbase = (size_t)s * N * N;
  load_twiddles<N>(tw, twg);
  load_col_tile<N>(tbuf, tile, sbase, c0);
  __syncthreads();
  const int c = threadIdx.x / T, t = threadIdx.x % T;
  float2 v[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int r = t + T * e;
    v[e] = tile[tslot(r, c)];
  }
  __syncthreads();
  fft_line<N, +1>(v, reinterpret_cast<float*>(tile) + c * 2 * LW, reinterpret_cast<float*>(tile) + c * 2 * LW + LW, tw, t);
  const float sc = 1.0f / (float)N;
  float acc = 0.f;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    v[e] = make_float2(v[e].x * sc, real ? 0.f : v[e].y * sc);
    acc += cabs2(v[e]);
  }
  __syncthreads();
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int r = t + T * e;
    tile[tslot(r, c)] = v[e];
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < N * COLS; idx += blockDim.x) {
    const int r = idx / COLS, cc = idx % COLS;
    const float2 o = tile[tslot(r, cc)];
    const size_t gi = sbase + (size_t)r * N + c0 + cc;
    atb[gi] = o;
    if (x) x[gi] = o;
  }
  const double tot = block_sum((double)acc, red);
  if (threadIdx.x == 0) part[((size_t)s * NSLOT + SLOT_RHS) * MAXPART + blockIdx.x] = tot;
}

// Data consistency of a warm start, column part: t = colIFFT((1 - R) colFFT(t) + R n b)
// (t = rowFFT(x); followed by the row IFFT with the 1/N scale this gives
// F^H((1 - R) F x + R b)).
template <int N>
__global__ void __launch_bounds__(512) k_col_dc(float2* __restrict__ tbuf, const float2* __restrict__ b,
                                                const uint8_t* __restrict__ mask, const float2* __restrict__ twg) {
  using C = FftCfg<N>;
  constexpr int E = C::E, T = C::T, LW = fft_line_words<N>();
  const int s = blockIdx.y;
  extern __shared__ __align__(16) unsigned char smem[];
  float2* tw = reinterpret_cast<float2*>(smem);
  float2* tile = reinterpret_cast<float2*>(smem + tw_bytes<N>());
  const int c0 = blockIdx.x * COLS;
  const size_t sbase = (size_t)s * N * N;
  load_twiddles<N>(tw, twg);
  load_col_tile<N>(tbuf, tile, sbase, c0);
  __syncthreads();
  const int c = threadIdx.x / T, t = threadIdx.x % T;
  float2 v[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int r = t + T * e;
    v[e] = tile[tslot(r, c)];
  }
  __syncthreads();
  fft_line<N, -1>(v, reinterpret_cast<float*>(tile) + c * 2 * LW, reinterpret_cast<float*>(tile) + c * 2 * LW + LW, tw, t);
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const size_t gi = sbase + (size_t)(t + T * e) * N + c0 + c;
    if (mask[gi]) v[e] = cscale(b[gi], (float)N);
  }
  fft_line<N, +1>(v, reinterpret_cast<float*>(tile) + c * 2 * LW, reinterpret_cast<float*>(tile) + c * 2 * LW + LW, tw, t);
  __syncthreads();
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int r = t + T * e;
    tile[tslot(r, c)] = v[e];
  }
  __syncthreads();
  store_col_tile<N>(tbuf, tile, sbase, c0);
}

// Data term of F: partial sum over sampled entries of |(1/n) colFFT(t) - b|^2,
// t = rowFFT(x), i.e. ||R F x - b||^2 with the unitary F (Eq. anapro).
template <int N>
__global__ void __launch_bounds__(512) k_col_resid(const float2* __restrict__ tbuf, const float2* __restrict__ b,
                                                   const uint8_t* __restrict__ mask, double* __restrict__ part,
                                                   int slot, const float2* __restrict__ twg) {
  using C = FftCfg<N>;
  constexpr int E = C::E, T = C::T, LW = fft_line_words<N>();
  const int s = blockIdx.y;
  extern __shared__ __align__(16) unsigned char smem[];
  float2* tw = reinterpret_cast<float2*>(smem);
  float2* tile = reinterpret_cast<float2*>(smem + tw_bytes<N>());
  __shared__ double red[32];
  const int c0 = blockIdx.x * COLS;
  const size_t sbase = (size_t)s * N * N;
  load_twiddles<N>(tw, twg);
  load_col_tile<N>(tbuf, tile, sbase, c0);
  __syncthreads();
  const int c = threadIdx.x / T, t = threadIdx.x % T;
  float2 v[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int r = t + T * e;
    v[e] = tile[tslot(r, c)];
  }
  __syncthreads();
  fft_line<N, -1>(v, reinterpret_cast<float*>(tile) + c * 2 * LW, reinterpret_cast<float*>(tile) + c * 2 * LW + LW, tw, t);
  const float sc = 1.0f / (float)N;
  float acc = 0.f;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const size_t gi = sbase + (size_t)(t + T * e) * N + c0 + c;
    if (mask[gi]) {
      const float2 bv = b[gi];
      acc += cabs2(make_float2(v[e].x * sc - bv.x, v[e].y * sc - bv.y));
    }
  }
  const double tot = block_sum((double)acc, red);
  if (threadIdx.x == 0) part[((size_t)s * NSLOT + slot) * MAXPART + blockIdx.x] = tot;
}

// q = (1/N) rowIFFT(t) [Re if real] + lam_tv (D1^T W1 D1 + D2^T W2 D2) d + lam u
// (W1 = W2 = wtv for isotropic TV; wtv2 holds W2 for l1 TV); partial
// Re<d, q>.
template <int N>
__global__ void __launch_bounds__(256) k_row_inv(const float2* __restrict__ tbuf, const float2* __restrict__ d,
                                                 const float2* __restrict__ u, const float* __restrict__ wtv,
                                                 float2* __restrict__ q, const SliceState* __restrict__ st,
                                                 double* __restrict__ part, int real,
                                                 const float2* __restrict__ twg, const float* __restrict__ wtv2) {
  using C = FftCfg<N>;
  constexpr int R = rows_per_cta<N>(), E = C::E, T = C::T, LW = fft_line_words<N>();
  const int s = blockIdx.y;
  if (!slice_running(st, s)) return;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[32];
  float2* tw = reinterpret_cast<float2*>(smem);
  float* lines = reinterpret_cast<float*>(smem + tw_bytes<N>());
  float2* ds = reinterpret_cast<float2*>(smem + tw_bytes<N>() + R * 2 * LW * 4);  // rows r0-1 .. r0+R
  float* ws = reinterpret_cast<float*>(ds + (R + 2) * N);                 // rows r0 .. r0+R
  float* ws2 = ws + (R + 1) * N;                                          // W2 rows (l1 TV)
  const int r0 = blockIdx.x * R;
  const size_t sbase = (size_t)s * N * N;
  const bool tv = (wtv != nullptr), aniso = tv && wtv2 != nullptr;
  if (tv) {
    // halo rows straight to shared memory, all copies in flight at once
    constexpr int NT = R * T, KD = (R + 2) * N / 2, KW = (R + 1) * N / 4;
    static_assert((tw_bytes<N>() + R * 2 * LW * 4) % 16 == 0 && N % 4 == 0, "16-byte staging");
    for (int idx = threadIdx.x; idx < KD; idx += NT) {
      const int rr = r0 - 1 + (2 * idx) / N, cc = (2 * idx) % N;
      if (rr >= 0 && rr < N)
        cp_async16_fft(ds + 2 * idx, d + sbase + (size_t)rr * N + cc);
      else
        *reinterpret_cast<float4*>(ds + 2 * idx) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    for (int idx = threadIdx.x; idx < KW; idx += NT) {
      const int rr = r0 + (4 * idx) / N, cc = (4 * idx) % N;
      if (rr < N)
        cp_async16_fft(ws + 4 * idx, wtv + sbase + (size_t)rr * N + cc);
      else
        *reinterpret_cast<float4*>(ws + 4 * idx) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (aniso) {
      for (int idx = threadIdx.x; idx < KW; idx += NT) {
        const int rr = r0 + (4 * idx) / N, cc = (4 * idx) % N;
        if (rr < N)
          cp_async16_fft(ws2 + 4 * idx, wtv2 + sbase + (size_t)rr * N + cc);
        else
          *reinterpret_cast<float4*>(ws2 + 4 * idx) = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  }
  load_twiddles<N>(tw, twg);
  const int lr = threadIdx.x / T, t = threadIdx.x % T;
  const int row = r0 + lr;
  const size_t base = sbase + (size_t)row * N;
  float2 v[E], uv[E];
#pragma unroll
  for (int e = 0; e < E; ++e) v[e] = tbuf[base + t + T * e];
  if (u) {  // in flight during the FFT
#pragma unroll
    for (int e = 0; e < E; ++e) uv[e] = u[base + t + T * e];
  }
  if (tv) asm volatile("cp.async.wait_all;\n" ::: "memory");
  __syncthreads();
  fft_line<N, +1>(v, lines + lr * 2 * LW, lines + lr * 2 * LW + LW, tw, t);
  const float sc = 1.0f / ((float)N * (float)N);
  const float lam = st[s].lam, lam_tv = st[s].lam_tv;
  float acc = 0.f;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int col = t + T * e;
    float2 a = make_float2(v[e].x * sc, real ? 0.f : v[e].y * sc);
    float2 dc;
    if (tv) {
      const float2* dr = ds + (lr + 1) * N;  // this row
      dc = dr[col];
      const float2 dl = col > 0 ? dr[col - 1] : make_float2(0.f, 0.f);
      const float2 du = (ds + lr * N)[col];  // row - 1 (zero above the image)
      const float2 g1 = csub(dc, dl), g2 = csub(dc, du);
      const float wc = ws[lr * N + col];
      float2 tvv;
      if (!aniso) {
        tvv = cscale(cadd(g1, g2), wc);
      } else {
        tvv = cadd(cscale(g1, wc), cscale(g2, ws2[lr * N + col]));
      }
      const float* wv = aniso ? ws2 : ws;  // vertical couplings: W2 (W for isotropic TV)
      if (col < N - 1) tvv = csub(tvv, cscale(csub(dr[col + 1], dc), ws[lr * N + col + 1]));
      if (row < N - 1) tvv = csub(tvv, cscale(csub((ds + (lr + 2) * N)[col], dc), wv[(lr + 1) * N + col]));
      a = cfma(lam_tv, tvv, a);
    } else {
      dc = d[base + col];
    }
    if (u) a = cfma(lam, uv[e], a);
    q[base + col] = a;
    acc += rdot2(dc, a);
  }
  const double tot = block_sum((double)acc, red);
  if (threadIdx.x == 0) part[((size_t)s * NSLOT + SLOT_DQ) * MAXPART + blockIdx.x] = tot;
}

// ------------------------------------------------------------------ launch --

// Dynamic shared-memory limits of one size's kernels, set once per device.
template <int N> static void set_smem_attrs() {
  static PerDeviceOnce once;
  once.run([] {
    const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
    bool ok = cudaFuncSetAttribute(k_row_fwd<N>, A, row_smem_bytes<N>(false)) == cudaSuccess;
    ok = cudaFuncSetAttribute(k_row_ahb<N>, A, row_smem_bytes<N>(false)) == cudaSuccess && ok;
    ok = cudaFuncSetAttribute(k_row_inv<N>, A, row_smem_bytes<N>(true, true)) == cudaSuccess && ok;
    ok = cudaFuncSetAttribute(k_col_mask<N>, A, col_smem_bytes<N>()) == cudaSuccess && ok;
    ok = cudaFuncSetAttribute(k_col_inv<N>, A, col_smem_bytes<N>()) == cudaSuccess && ok;
    ok = cudaFuncSetAttribute(k_col_resid<N>, A, col_smem_bytes<N>()) == cudaSuccess && ok;
    ok = cudaFuncSetAttribute(k_col_dc<N>, A, col_smem_bytes<N>()) == cudaSuccess && ok;
    return ok;
  });
}

template <int N> struct FftLaunch {
  static constexpr int R = rows_per_cta<N>();
  static void row_fwd(const FftArgs& a) {
    set_smem_attrs<N>();
    k_row_fwd<N><<<dim3(N / R, a.batch), R * FftCfg<N>::T, row_smem_bytes<N>(false), a.stream>>>(
        a.z, a.d, a.t, a.st, a.tw, a.mode, a.xs);
  }
  static void row_ahb(const FftArgs& a) {
    set_smem_attrs<N>();
    k_row_ahb<N><<<dim3(N / R, a.batch), R * FftCfg<N>::T, row_smem_bytes<N>(false), a.stream>>>(
        a.b, a.mask, a.t, a.tw);
  }
  static void col_mask(const FftArgs& a) {
    set_smem_attrs<N>();
    k_col_mask<N><<<dim3(N / COLS, a.batch), COLS * FftCfg<N>::T, col_smem_bytes<N>(), a.stream>>>(
        a.t, a.mask, a.st, a.tw);
  }
  static void col_inv(const FftArgs& a) {
    set_smem_attrs<N>();
    k_col_inv<N><<<dim3(N / COLS, a.batch), COLS * FftCfg<N>::T, col_smem_bytes<N>(), a.stream>>>(
        a.t, a.atb, a.x, a.real, a.part, a.tw);
  }
  static void col_resid(const FftArgs& a) {
    set_smem_attrs<N>();
    k_col_resid<N><<<dim3(N / COLS, a.batch), COLS * FftCfg<N>::T, col_smem_bytes<N>(), a.stream>>>(
        a.t, a.b, a.mask, a.part, a.mode, a.tw);
  }
  static void col_dc(const FftArgs& a) {
    set_smem_attrs<N>();
    k_col_dc<N><<<dim3(N / COLS, a.batch), COLS * FftCfg<N>::T, col_smem_bytes<N>(), a.stream>>>(a.t, a.b, a.mask,
                                                                                                  a.tw);
  }
  static void row_inv(const FftArgs& a) {
    set_smem_attrs<N>();
    k_row_inv<N><<<dim3(N / R, a.batch), R * FftCfg<N>::T,
                   row_smem_bytes<N>(a.wtv != nullptr, a.wtv2 != nullptr), a.stream>>>(
        a.t, a.d, a.u, a.wtv, a.q, a.st, a.part, a.real, a.tw, a.wtv2);
  }
};

#define FIRLS_FOR_SIZES(X) X(16) X(32) X(48) X(64) X(80) X(96) X(128) X(160) X(192) X(256) X(320) X(384) X(512)

#define FIRLS_DISPATCH(fn)                              \
  void fft_##fn(int n, const FftArgs& a) {              \
    switch (n) {                                        \
      FIRLS_FOR_SIZES(FIRLS_CASE_##fn)                  \
      default: break;                                   \
    }                                                   \
  }
#define FIRLS_CASE_row_fwd(n) case n: FftLaunch<n>::row_fwd(a); break;
#define FIRLS_CASE_row_ahb(n) case n: FftLaunch<n>::row_ahb(a); break;
#define FIRLS_CASE_col_mask(n) case n: FftLaunch<n>::col_mask(a); break;
#define FIRLS_CASE_col_inv(n) case n: FftLaunch<n>::col_inv(a); break;
#define FIRLS_CASE_row_inv(n) case n: FftLaunch<n>::row_inv(a); break;
#define FIRLS_CASE_col_resid(n) case n: FftLaunch<n>::col_resid(a); break;
#define FIRLS_CASE_col_dc(n) case n: FftLaunch<n>::col_dc(a); break;
FIRLS_DISPATCH(row_fwd)
FIRLS_DISPATCH(row_ahb)
FIRLS_DISPATCH(col_mask)
FIRLS_DISPATCH(col_inv)
FIRLS_DISPATCH(row_inv)
FIRLS_DISPATCH(col_resid)
FIRLS_DISPATCH(col_dc)

bool fft_size_supported(int n) {
  switch (n) {
#define FIRLS_CASE_SUP(n) case n: return true;
    FIRLS_FOR_SIZES(FIRLS_CASE_SUP)
#undef FIRLS_CASE_SUP
    default: return false;
  }
}

int fft_row_ctas(int n) {
  switch (n) {
#define FIRLS_CASE_RC(n) case n: return n / rows_per_cta<n>();
    FIRLS_FOR_SIZES(FIRLS_CASE_RC)
#undef FIRLS_CASE_RC
    default: return 0;
  }
}

int fft_col_ctas(int n) { return n / COLS; }

void fft_prepare(int n) {
  switch (n) {
#define FIRLS_CASE_PREP(n) case n: set_smem_attrs<n>(); break;
    FIRLS_FOR_SIZES(FIRLS_CASE_PREP)
#undef FIRLS_CASE_PREP
    default: break;
  }
}

}  // namespace firls
