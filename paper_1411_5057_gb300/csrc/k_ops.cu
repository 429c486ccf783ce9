// Non-FFT kernels of the FIRLS hot path: lifting wavelets (Phi, Phi^T),
// weights (Eq. gw, Eq. Wog, Eq. wi), preconditioner set-up and application
// (Eq. pog, Eq. ptv with the L U factors of Sec. 4.2), PCG vector updates
// and the FP64 PCG scalars.
#include "launch.h"

namespace firls {

// ============================================================ wavelets =====
// Lifting factorisation (Daubechies & Sweldens) arranged to reproduce the
// periodic filter bank a_k = sum_t h_t x_{2k+t}, d_k = sum_t g_t x_{2k+t},
// g_t = (-1)^t h_{3-t}, h the Daubechies-4 taps.  For output pair k, with
// s1_l = x_{2l} + sqrt3 x_{2l+1}:
//   D_k  = x_{2k+3} - (sqrt3/4) s1_{k+1} - ((sqrt3-2)/4) s1_k
//   a_k  = cs (s1_k - D_k),   d_k = -cd D_k,
// cs = (sqrt3-1)/sqrt2, cd = (sqrt3+1)/sqrt2.  The inverse solves these for
// x_{2l}, x_{2l+1} from pairs l-1 and l.  Haar: a = (x0+x1)/sqrt2,
// d = (x0-x1)/sqrt2.
namespace lift {
constexpr float S3 = 1.7320508075688772f;
constexpr float K1 = 0.43301270189221932f;   // sqrt3 / 4
constexpr float K2 = -0.066987298107780677f; // (sqrt3 - 2) / 4
constexpr float CS = 0.51763809020504152f;   // (sqrt3 - 1) / sqrt2
constexpr float CD = 1.9318516525781366f;    // (sqrt3 + 1) / sqrt2
constexpr float ICS = 1.9318516525781366f;   // 1 / CS
constexpr float ICD = 0.51763809020504152f;  // 1 / CD
constexpr float RS2 = 0.70710678118654752f;  // 1 / sqrt2

FI void fwd_db4(float2 x0, float2 x1, float2 x2, float2 x3, float2& a, float2& d) {
  const float2 s1k = cfma(S3, x1, x0);
  const float2 s1n = cfma(S3, x3, x2);
  const float2 D = make_float2(x3.x - K1 * s1n.x - K2 * s1k.x, x3.y - K1 * s1n.y - K2 * s1k.y);
  a = cscale(csub(s1k, D), CS);
  d = cscale(D, -CD);
}
FI void fwd_haar(float2 x0, float2 x1, float2& a, float2& d) {
  a = cscale(cadd(x0, x1), RS2);
  d = cscale(csub(x0, x1), RS2);
}
// from (a_{l-1}, d_{l-1}) and (a_l, d_l) to (x_{2l}, x_{2l+1})
FI void inv_db4(float2 am, float2 dm, float2 al, float2 dl, float2& x0, float2& x1) {
  const float2 Dm = cscale(dm, -ICD);
  const float2 s1m = cfma(ICS, am, Dm);
  const float2 Dl = cscale(dl, -ICD);
  const float2 s1l = cfma(ICS, al, Dl);
  x1 = make_float2(Dm.x + K1 * s1l.x + K2 * s1m.x, Dm.y + K1 * s1l.y + K2 * s1m.y);
  x0 = cfma(-S3, x1, s1l);
}
FI void inv_haar(float2 a, float2 d, float2& x0, float2& x1) {
  x0 = cscale(cadd(a, d), RS2);
  x1 = cscale(csub(a, d), RS2);
}
}  // namespace lift

constexpr int WAV_SMEM = 96 * 1024;
constexpr int WAV_THREADS = 256;

static int wav_fwd_rb(int m) {
  int half = m / 2;
  int rb = (WAV_SMEM / (m * 16) - 2) / 2;
  if (rb > 8) rb = 8;
  if (rb < 1) rb = 1;
  if (rb > half) rb = half;
  return rb;
}
static int wav_inv_rb(int m) {
  int half = m / 2;
  int rb = (WAV_SMEM / (m * 8) - 2) / 4;
  if (rb > 8) rb = 8;
  if (rb < 1) rb = 1;
  if (rb > half) rb = half;
  return rb;
}

// One analysis level on the m x m block `in` (row stride ld_in).
__global__ void __launch_bounds__(WAV_THREADS)
k_wav_fwd(const float2* __restrict__ in, size_t in_ss, int ld_in, float2* __restrict__ llo, size_t ll_ss,
          int ld_ll, float2* __restrict__ c, float* __restrict__ w, int n, int m, int rb, int kind,
          int mode, int last, const SliceState* __restrict__ st) {
  const int s = blockIdx.y;
  if (st != nullptr && !slice_running(st, s)) return;
  extern __shared__ __align__(16) unsigned char smem[];
  const int half = m / 2;
  const int k0 = blockIdx.x * rb;
  const int nrow = 2 * rb + (kind == 2 ? 2 : 0);
  float2* xs = reinterpret_cast<float2*>(smem);  // [nrow][m] input rows
  float2* rt = xs + nrow * m;                    // [nrow][m] row-transformed
  const float2* src = in + (size_t)s * in_ss;
  for (int idx = threadIdx.x; idx < nrow * m; idx += blockDim.x) {
    const int i = idx / m, col = idx % m;
    const int gr = (2 * k0 + i) % m;
    xs[idx] = src[(size_t)gr * ld_in + col];
  }
  __syncthreads();
  // horizontal step: [lo | hi] per row
  for (int idx = threadIdx.x; idx < nrow * half; idx += blockDim.x) {
    const int i = idx / half, k = idx % half;
    const float2* xr = xs + i * m;
    float2 a, d;
    if (kind == 2) {
      lift::fwd_db4(xr[2 * k], xr[2 * k + 1], xr[(2 * k + 2) % m], xr[(2 * k + 3) % m], a, d);
    } else {
      lift::fwd_haar(xr[2 * k], xr[2 * k + 1], a, d);
    }
    rt[i * m + k] = a;
    rt[i * m + half + k] = d;
  }
  __syncthreads();
  // vertical step and store
  const float lam = st ? st[s].lam : 0.f, abar = st ? st[s].abar : 0.f, eps = st ? st[s].eps : 1e-10f;
  float2* cs = c + (size_t)s * n * n;
  float* ws = w ? w + (size_t)s * n * n : nullptr;
  float2* lls = llo + (size_t)s * ll_ss;
  const int nout = min(rb, half - k0);
  for (int idx = threadIdx.x; idx < nout * m; idx += blockDim.x) {
    const int kk = idx / m, j = idx % m;
    float2 a, d;
    if (kind == 2) {
      lift::fwd_db4(rt[(2 * kk) * m + j], rt[(2 * kk + 1) * m + j], rt[(2 * kk + 2) * m + j],
                    rt[(2 * kk + 3) * m + j], a, d);
    } else {
      lift::fwd_haar(rt[(2 * kk) * m + j], rt[(2 * kk + 1) * m + j], a, d);
    }
    const int row = k0 + kk;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int orow = h ? half + row : row;
      const float2 v = h ? d : a;
      if (!h && j < half && !last) {  // intermediate LL: raw, to the ping-pong buffer
        lls[(size_t)row * ld_ll + j] = v;
        continue;
      }
      const size_t p = (size_t)orow * n + j;
      if (mode == WAV_RAW) {
        cs[p] = v;
      } else if (mode == WAV_MUL_W) {
        cs[p] = cscale(v, ws[p]);
      } else if (mode == WAV_MUL_PINV) {
        cs[p] = cscale(v, 1.0f / (abar + lam * ws[p]));
      } else {
        ws[p] = rsqrtf(cabs2(v) + eps);
      }
    }
  }
}

// One synthesis level: coefficients of the m x m block (LL from ll_in,
// details from c at stride n) to the m x m output block.
__global__ void __launch_bounds__(WAV_THREADS)
k_wav_inv(const float2* __restrict__ lli, size_t ll_ss, int ld_ll, const float2* __restrict__ c,
          float2* __restrict__ out, size_t out_ss, int ld_out, int n, int m, int rb, int kind,
          const float2* __restrict__ r, double* __restrict__ part, int real,
          const SliceState* __restrict__ st) {
  const int s = blockIdx.y;
  if (st != nullptr && !slice_running(st, s)) return;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[32];
  const int half = m / 2;
  const int k0 = blockIdx.x * rb;
  const int nout = min(rb, half - k0);
  float2* lo = reinterpret_cast<float2*>(smem);  // [rb+1][m]: [LL | LH] rows k0-1 .. k0+rb-1
  float2* hi = lo + (rb + 1) * m;                // [rb+1][m]: [HL | HH]
  float2* vs = hi + (rb + 1) * m;                // [2 rb][m]
  const float2* cs = c + (size_t)s * n * n;
  const float2* ls = lli + (size_t)s * ll_ss;
  for (int idx = threadIdx.x; idx < (nout + 1) * m; idx += blockDim.x) {
    const int i = idx / m, j = idx % m;
    const int kr = (k0 - 1 + i + half) % half;
    lo[idx] = j < half ? ls[(size_t)kr * ld_ll + j] : cs[(size_t)kr * n + j];
    hi[idx] = cs[(size_t)(half + kr) * n + j];
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < nout * m; idx += blockDim.x) {
    const int kk = idx / m, j = idx % m;
    float2 x0, x1;
    if (kind == 2) {
      lift::inv_db4(lo[kk * m + j], hi[kk * m + j], lo[(kk + 1) * m + j], hi[(kk + 1) * m + j], x0, x1);
    } else {
      lift::inv_haar(lo[(kk + 1) * m + j], hi[(kk + 1) * m + j], x0, x1);
    }
    vs[(2 * kk) * m + j] = x0;
    vs[(2 * kk + 1) * m + j] = x1;
  }
  __syncthreads();
  float2* os = out + (size_t)s * out_ss;
  const float2* rs = r ? r + (size_t)s * n * n : nullptr;
  float acc = 0.f;
  for (int idx = threadIdx.x; idx < 2 * nout * half; idx += blockDim.x) {
    const int i = idx / half, l = idx % half;
    const float2* vr = vs + i * m;
    float2 x0, x1;
    if (kind == 2) {
      const int lm = (l - 1 + half) % half;
      lift::inv_db4(vr[lm], vr[half + lm], vr[l], vr[half + l], x0, x1);
    } else {
      lift::inv_haar(vr[l], vr[half + l], x0, x1);
    }
    if (real) {
      x0.y = 0.f;
      x1.y = 0.f;
    }
    const int orow = 2 * k0 + i;
    const size_t p = (size_t)orow * ld_out + 2 * l;
    os[p] = x0;
    os[p + 1] = x1;
    if (rs) acc += rdot2(rs[(size_t)orow * n + 2 * l], x0) + rdot2(rs[(size_t)orow * n + 2 * l + 1], x1);
  }
  if (part) {
    const double tot = block_sum((double)acc, red);
    if (threadIdx.x == 0) part[((size_t)s * NSLOT + SLOT_RZ) * MAXPART + blockIdx.x] = tot;
  }
}

static void set_wav_attrs() {
  static bool done = false;
  if (done) return;
  done = true;
  cudaFuncSetAttribute(k_wav_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, WAV_SMEM);
  cudaFuncSetAttribute(k_wav_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, WAV_SMEM);
}

void wav_prepare() { set_wav_attrs(); }

void wavelet_forward(const WavArgs& a, const float2* x, float2* c, float* w, int mode) {
  set_wav_attrs();
  const int n = a.n;
  const size_t hh = (size_t)(n / 2) * (n / 2);
  const float2* src = x;
  size_t src_ss = (size_t)n * n;
  int src_ld = n;
  for (int l = 1; l <= a.levels; ++l) {
    const int m = n >> (l - 1), half = m / 2;
    const bool last = (l == a.levels);
    float2* dst = last ? c : ((l & 1) ? a.tmpA : a.tmpB);
    const size_t dst_ss = last ? (size_t)n * n : hh;
    const int dst_ld = last ? n : half;
    const int rb = wav_fwd_rb(m);
    const int nrow = 2 * rb + (a.kind == 2 ? 2 : 0);
    const int smem = 2 * nrow * m * 8;
    k_wav_fwd<<<dim3((half + rb - 1) / rb, a.batch), WAV_THREADS, smem, a.stream>>>(
        src, src_ss, src_ld, dst, dst_ss, dst_ld, c, w, n, m, rb, a.kind, mode, last ? 1 : 0, a.st);
    src = dst;
    src_ss = dst_ss;
    src_ld = dst_ld;
  }
}

int wavelet_inverse_ctas(int n) {
  const int rb = wav_inv_rb(n);
  return (n / 2 + rb - 1) / rb;
}

void wavelet_inverse(const WavArgs& a, const float2* c, float2* x, const float2* r, int real) {
  set_wav_attrs();
  const int n = a.n;
  const size_t hh = (size_t)(n / 2) * (n / 2);
  const float2* lli = c;
  size_t ll_ss = (size_t)n * n;
  int ll_ld = n;
  for (int l = a.levels; l >= 1; --l) {
    const int m = n >> (l - 1), half = m / 2;
    const bool final_level = (l == 1);
    float2* out = final_level ? x : ((l & 1) ? a.tmpA : a.tmpB);
    const size_t out_ss = final_level ? (size_t)n * n : hh;
    const int out_ld = final_level ? n : m;
    const int rb = wav_inv_rb(m);
    const int smem = (4 * rb + 2) * m * 8;
    k_wav_inv<<<dim3((half + rb - 1) / rb, a.batch), WAV_THREADS, smem, a.stream>>>(
        lli, ll_ss, ll_ld, c, out, out_ss, out_ld, n, m, rb, a.kind, final_level ? r : nullptr,
        final_level && r ? a.part : nullptr, real, a.st);
    lli = out;
    ll_ss = out_ss;
    ll_ld = out_ld;
  }
}

// ================================================================== TV =====

// W_i = (|grad_1 x_i|^2 + |grad_2 x_i|^2 + eps)^(-1/2), zero extension (Eq. wi)
__global__ void k_tv_weights(int n, const SliceState* __restrict__ st, const float2* __restrict__ x,
                             float* __restrict__ wtv) {
  const int s = blockIdx.y;
  if (!slice_running(st, s)) return;
  const float eps = st[s].eps;
  const size_t base = (size_t)s * n * n;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n * n; i += gridDim.x * blockDim.x) {
    const int r = i / n, c = i % n;
    const float2 xc = x[base + i];
    const float2 g1 = c > 0 ? csub(xc, x[base + i - 1]) : xc;
    const float2 g2 = r > 0 ? csub(xc, x[base + i - n]) : xc;
    wtv[base + i] = rsqrtf(cabs2(g1) + cabs2(g2) + eps);
  }
}

void tv_weights(int batch, int n, cudaStream_t s, const SliceState* st, const float2* x, float* wtv) {
  const int N = n * n;
  const int blocks = (N + 255) / 256 < 64 ? (N + 255) / 256 : 64;
  k_tv_weights<<<dim3(blocks, batch), 256, 0, s>>>(n, st, x, wtv);
}

// Exact diag(Phi^T diag(w) Phi): each 2-D basis function is an outer product
// of 1-D level-l functions f_{l,type}(i - 2^l p) whose squares are tabulated
// (sqtab[(l-1)*2 + type][0..len)), so the diagonal is a separable sum.
__global__ void k_wavelet_diag(int n, int levels, const SliceState* __restrict__ st,
                               const float* __restrict__ w, float* __restrict__ out,
                               const float* __restrict__ sqtab, const int* __restrict__ sqlen) {
  const int s = blockIdx.y;
  if (!slice_running(st, s)) return;
  const size_t base = (size_t)s * n * n;
  const float* ws = w + base;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n * n; i += gridDim.x * blockDim.x) {
    const int r = i / n, c = i % n;
    float acc = 0.f;
    for (int l = 1; l <= levels; ++l) {
      const int h = n >> l, step = 1 << l;
      const int nb = (l == levels) ? 4 : 3;
      for (int b = 0; b < nb; ++b) {
        // bands: (0,1) low/high, (1,0) high/low, (1,1) high/high, (0,0) low/low
        const int br = (b == 1 || b == 2) ? 1 : 0;
        const int bc = (b == 0 || b == 2) ? 1 : 0;
        const float* fr = sqtab + (size_t)((l - 1) * 2 + br) * n;
        const float* fc = sqtab + (size_t)((l - 1) * 2 + bc) * n;
        const int lr = sqlen[(l - 1) * 2 + br], lc = sqlen[(l - 1) * 2 + bc];
        for (int sr = r & (step - 1); sr < lr; sr += step) {
          const int p = ((r - sr + n) % n) >> l;
          const float vr = fr[sr];
          const float* wrow = ws + (size_t)(br * h + p) * n + bc * h;
          for (int sc = c & (step - 1); sc < lc; sc += step) {
            const int qq = ((c - sc + n) % n) >> l;
            acc = fmaf(vr * fc[sc], wrow[qq], acc);
          }
        }
      }
    }
    out[base + i] = acc;
  }
}

void wavelet_diag(int batch, int n, int levels, cudaStream_t s, const SliceState* st, const float* w,
                  float* out, const float* sqtab, const int* sqlen) {
  const int N = n * n;
  const int blocks = (N + 255) / 256 < 256 ? (N + 255) / 256 : 256;
  k_wavelet_diag<<<dim3(blocks, batch), 256, 0, s>>>(n, levels, st, w, out, sqtab, sqlen);
}

// P = abar I + lam_tv (D1^T W D1 + D2^T W D2) [+ lam diag(Phi^T W Phi)] (Eq. ptv):
// ia = 1/a_i, pb = b_i (coupling i, i+1), pc = c_i (coupling i, i+n).
__global__ void k_penta(int n, const SliceState* __restrict__ st, const float* __restrict__ wtv,
                        const float* __restrict__ wdiag, float* __restrict__ ia, float* __restrict__ pb,
                        float* __restrict__ pc) {
  const int s = blockIdx.y;
  if (!slice_running(st, s)) return;
  const float abar = st[s].abar, lt = st[s].lam_tv, lw = st[s].lam;
  const size_t base = (size_t)s * n * n;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n * n; i += gridDim.x * blockDim.x) {
    const int r = i / n, c = i % n;
    const float wc = wtv[base + i];
    const float wr = c < n - 1 ? wtv[base + i + 1] : 0.f;
    const float wd = r < n - 1 ? wtv[base + i + n] : 0.f;
    float a = abar + lt * (2.f * wc + wr + wd);
    if (wdiag) a = fmaf(lw, wdiag[base + i], a);
    ia[base + i] = 1.0f / a;
    pb[base + i] = -lt * wr;
    pc[base + i] = -lt * wd;
  }
}

void penta_setup(int batch, int n, cudaStream_t s, const SliceState* st, const float* wtv,
                 const float* wdiag, float* ia, float* pb, float* pc) {
  const int N = n * n;
  const int blocks = (N + 255) / 256 < 64 ? (N + 255) / 256 : 64;
  k_penta<<<dim3(blocks, batch), 256, 0, s>>>(n, st, wtv, wdiag, ia, pb, pc);
}

// ------------------------------------------------ ILU solves (Sec. 4.2) -----
// z = U^{-1} L^{-1} r with L = I + L_P diag(a)^{-1}, U = diag(a) + U_P:
//   forward  y_i = r_i - (b_{i-1}/a_{i-1}) y_{i-1} - (c_{i-n}/a_{i-n}) y_{i-n}
//   backward z_i = (y_i - b_i z_{i+1} - c_i z_{i+n}) / a_i
// One CTA per slice sweeps the rows; within a row the first-order
// recurrence is an affine scan across threads (4 columns per thread).

// Inclusive scan of affine maps y -> A y + B in thread order (forward) or
// reverse thread order; returns, per thread, B of the exclusive prefix
// (the value entering this thread's segment when the boundary value is 0).
template <bool REV>
FI float2 affine_exclusive(float A, float2 B, float* sA, float2* sB) {
  const int nt = blockDim.x;
  const int t = REV ? (nt - 1 - (int)threadIdx.x) : (int)threadIdx.x;  // logical index
  const int lane = threadIdx.x & 31;
  // warp-level inclusive scan in logical order
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const float Ap = REV ? __shfl_down_sync(0xffffffffu, A, off) : __shfl_up_sync(0xffffffffu, A, off);
    const float bx = REV ? __shfl_down_sync(0xffffffffu, B.x, off) : __shfl_up_sync(0xffffffffu, B.x, off);
    const float by = REV ? __shfl_down_sync(0xffffffffu, B.y, off) : __shfl_up_sync(0xffffffffu, B.y, off);
    const bool ok = REV ? (lane + off < 32) : (lane >= off);
    if (ok) {
      B = make_float2(fmaf(A, bx, B.x), fmaf(A, by, B.y));
      A = A * Ap;
    }
  }
  // warp totals: physical warp w holds logical block (REV: reversed)
  const int w = threadIdx.x >> 5, nw = nt >> 5;
  const bool tail = REV ? (lane == 0) : (lane == 31);
  if (tail) {
    sA[w] = A;
    sB[w] = B;
  }
  __syncthreads();
  // prefix of the logically preceding warps
  float Ap = 1.f;
  float2 Bp = make_float2(0.f, 0.f);
  if (!REV) {
    for (int v = 0; v < w; ++v) {
      Bp = make_float2(fmaf(sA[v], Bp.x, sB[v].x), fmaf(sA[v], Bp.y, sB[v].y));
      Ap *= sA[v];
    }
  } else {
    for (int v = nw - 1; v > w; --v) {
      Bp = make_float2(fmaf(sA[v], Bp.x, sB[v].x), fmaf(sA[v], Bp.y, sB[v].y));
      Ap *= sA[v];
    }
  }
  // inclusive value of this thread including earlier warps (boundary 0)
  const float2 inc = make_float2(fmaf(A, Bp.x, B.x), fmaf(A, Bp.y, B.y));
  __syncthreads();
  sB[32 + t] = inc;  // indexed by logical position
  __syncthreads();
  const float2 ex = t > 0 ? sB[32 + t - 1] : make_float2(0.f, 0.f);
  __syncthreads();
  (void)Ap;
  return ex;
}

constexpr int ILU_E = 4;

__global__ void __launch_bounds__(512) k_ilu(int n, int mode, const SliceState* __restrict__ st,
                                             double* __restrict__ part, float2* __restrict__ x,
                                             const float2* __restrict__ d, float2* __restrict__ r,
                                             const float2* __restrict__ q, const float2* __restrict__ atb,
                                             float2* __restrict__ y, float2* __restrict__ z,
                                             const float* __restrict__ ia, const float* __restrict__ pb,
                                             const float* __restrict__ pc) {
  const int s = blockIdx.x;
  if (!slice_running(st, s)) return;
  __shared__ float sA[32];
  __shared__ float2 sB[32 + 512];
  __shared__ double red[32];
  const int t = threadIdx.x;
  const int c0 = ILU_E * t;
  const bool own = c0 < n;
  const float alpha = (float)st[s].alpha;
  const size_t base = (size_t)s * n * n;
  float2 yprev[ILU_E];
  float mprev[ILU_E];
#pragma unroll
  for (int e = 0; e < ILU_E; ++e) {
    yprev[e] = make_float2(0.f, 0.f);
    mprev[e] = 0.f;
  }
  float rr = 0.f;
  for (int row = 0; row < n; ++row) {
    const size_t i0 = base + (size_t)row * n + c0;
    float A = 1.f;
    float2 B = make_float2(0.f, 0.f);
    float2 tv[ILU_E];
    float iav[ILU_E], pbv[ILU_E], pcv[ILU_E];
    if (own) {
#pragma unroll
      for (int e = 0; e < ILU_E; ++e) {
        float2 rv;
        if (mode == ILU_INIT) {
          rv = csub(atb[i0 + e], q[i0 + e]);
        } else {
          rv = cfma(-alpha, q[i0 + e], r[i0 + e]);
          x[i0 + e] = cfma(alpha, d[i0 + e], x[i0 + e]);
        }
        r[i0 + e] = rv;
        rr += cabs2(rv);
        iav[e] = ia[i0 + e];
        pbv[e] = pb[i0 + e];
        pcv[e] = pc[i0 + e];
        tv[e] = cfma(-mprev[e], yprev[e], rv);
      }
      float l = c0 > 0 ? pb[i0 - 1] * ia[i0 - 1] : 0.f;
#pragma unroll
      for (int e = 0; e < ILU_E; ++e) {
        if (e > 0) l = pbv[e - 1] * iav[e - 1];
        B = cfma(-l, B, tv[e]);
        A = -l * A;
      }
    }
    float2 yin = affine_exclusive<false>(A, B, sA, sB);
    if (own) {
      float l = c0 > 0 ? pb[i0 - 1] * ia[i0 - 1] : 0.f;
#pragma unroll
      for (int e = 0; e < ILU_E; ++e) {
        if (e > 0) l = pbv[e - 1] * iav[e - 1];
        yin = cfma(-l, yin, tv[e]);
        y[i0 + e] = yin;
        yprev[e] = yin;
        mprev[e] = pcv[e] * iav[e];
      }
    }
  }
  float2 znext[ILU_E];
#pragma unroll
  for (int e = 0; e < ILU_E; ++e) znext[e] = make_float2(0.f, 0.f);
  float rz = 0.f;
  for (int row = n - 1; row >= 0; --row) {
    const size_t i0 = base + (size_t)row * n + c0;
    float A = 1.f;
    float2 B = make_float2(0.f, 0.f);
    float2 tv[ILU_E];
    float iav[ILU_E], pbv[ILU_E];
    if (own) {
#pragma unroll
      for (int e = 0; e < ILU_E; ++e) {
        iav[e] = ia[i0 + e];
        pbv[e] = pb[i0 + e];
        tv[e] = cfma(-pc[i0 + e], znext[e], y[i0 + e]);
      }
#pragma unroll
      for (int e = ILU_E - 1; e >= 0; --e) {
        const float Ae = -iav[e] * pbv[e];
        B = cfma(Ae, B, cscale(tv[e], iav[e]));
        A = Ae * A;
      }
    }
    float2 zr = affine_exclusive<true>(A, B, sA, sB);
    if (own) {
#pragma unroll
      for (int e = ILU_E - 1; e >= 0; --e) {
        zr = cfma(-iav[e] * pbv[e], zr, cscale(tv[e], iav[e]));
        z[i0 + e] = zr;
        znext[e] = zr;
        rz += rdot2(r[i0 + e], zr);
      }
    }
  }
  const double trz = block_sum((double)rz, red);
  __syncthreads();
  const double trr = block_sum((double)rr, red);
  if (threadIdx.x == 0) {
    part[((size_t)s * NSLOT + SLOT_RZ) * MAXPART] = trz;
    part[((size_t)s * NSLOT + SLOT_RR) * MAXPART] = trr;
  }
}

void ilu_step(int batch, int n, cudaStream_t s, const SliceState* st, double* part, int mode, float2* x,
              const float2* d, float2* r, const float2* q, const float2* atb, float2* y, float2* z,
              const float* ia, const float* pb, const float* pc) {
  int threads = (n / ILU_E + 31) / 32 * 32;
  k_ilu<<<batch, threads, 0, s>>>(n, mode, st, part, x, d, r, q, atb, y, z, ia, pb, pc);
}

// =========================================================== PCG vectors ==

int axpy_ctas(int n) {
  const int N = n * n;
  int c = N / 2048;
  if (c < 1) c = 1;
  if (c > MAXPART) c = MAXPART;
  return c;
}

__global__ void k_axpy(int N, int mode, const SliceState* __restrict__ st, double* __restrict__ part,
                       float2* __restrict__ x, const float2* __restrict__ d, float2* __restrict__ r,
                       const float2* __restrict__ q, const float2* __restrict__ atb) {
  const int s = blockIdx.y;
  if (!slice_running(st, s)) return;
  __shared__ double red[32];
  const float alpha = (float)st[s].alpha;
  const size_t base = (size_t)s * N;
  const int chunk = (N + gridDim.x - 1) / gridDim.x;
  const int lo = blockIdx.x * chunk, hi = min(N, lo + chunk);
  float acc = 0.f;
  for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const size_t g = base + i;
    if (mode == AXPY_INIT) {
      const float2 rv = csub(atb[g], q[g]);
      r[g] = rv;
      acc += cabs2(rv);
    } else {
      x[g] = cfma(alpha, d[g], x[g]);
      if (mode == AXPY_STEP) {
        const float2 rv = cfma(-alpha, q[g], r[g]);
        r[g] = rv;
        acc += cabs2(rv);
      }
    }
  }
  const double tot = block_sum((double)acc, red);
  if (threadIdx.x == 0) part[((size_t)s * NSLOT + SLOT_RR) * MAXPART + blockIdx.x] = tot;
}

void axpy_step(int batch, int n, cudaStream_t s, const SliceState* st, double* part, int mode, float2* x,
               const float2* d, float2* r, const float2* q, const float2* atb) {
  k_axpy<<<dim3(axpy_ctas(n), batch), 256, 0, s>>>(n * n, mode, st, part, x, d, r, q, atb);
}

// partial ||x - xprev||^2 (SLOT_DX) and ||xprev||^2 (SLOT_XX)
__global__ void k_relchange(int N, const SliceState* __restrict__ st, const float2* __restrict__ x,
                            const float2* __restrict__ xp, double* __restrict__ part) {
  const int s = blockIdx.y;
  if (st[s].done) return;
  __shared__ double red[32];
  const size_t base = (size_t)s * N;
  const int chunk = (N + gridDim.x - 1) / gridDim.x;
  const int lo = blockIdx.x * chunk, hi = min(N, lo + chunk);
  float a = 0.f, b = 0.f;
  for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const float2 xv = x[base + i], pv = xp[base + i];
    a += cabs2(csub(xv, pv));
    b += cabs2(pv);
  }
  const double ta = block_sum((double)a, red);
  __syncthreads();
  const double tb = block_sum((double)b, red);
  if (threadIdx.x == 0) {
    part[((size_t)s * NSLOT + SLOT_DX) * MAXPART + blockIdx.x] = ta;
    part[((size_t)s * NSLOT + SLOT_XX) * MAXPART + blockIdx.x] = tb;
  }
}

void relchange_parts(int batch, int n, cudaStream_t s, const SliceState* st, const float2* x,
                     const float2* xprev, double* part) {
  k_relchange<<<dim3(axpy_ctas(n), batch), 256, 0, s>>>(n * n, st, x, xprev, part);
}

// ================================================================ groups ===

// W_g = (sum_{j in g} |c_j|^2 + eps)^(-1/2)   (Eq. gw)
__global__ void k_group_norms(int n, int G, const SliceState* __restrict__ st, const int* __restrict__ gidx,
                              const int* __restrict__ goff, int gsize, const float2* __restrict__ c,
                              float* __restrict__ wg) {
  const int s = blockIdx.y;
  if (!slice_running(st, s)) return;
  const float eps = st[s].eps;
  const float2* cs = c + (size_t)s * n * n;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
    const int b = goff ? goff[g] : g * gsize;
    const int e = goff ? goff[g + 1] : b + gsize;
    float acc = 0.f;
    for (int k = b; k < e; ++k) acc += cabs2(cs[gidx[k]]);
    wg[(size_t)s * G + g] = rsqrtf(acc + eps);
  }
}

void group_norms(int batch, int n, int G, cudaStream_t s, const SliceState* st, const int* gidx,
                 const int* goff, int gsize, const float2* c, float* wg, float) {
  const int blocks = (G + 255) / 256 < 256 ? (G + 255) / 256 : 256;
  k_group_norms<<<dim3(blocks, batch), 256, 0, s>>>(n, G, st, gidx, goff, gsize, c, wg);
}

// w_j = sum_{g containing j} W_g = diag(G^T W G)_j  (Eq. Wog), ascending g
__global__ void k_group_gather(int n, int G, const SliceState* __restrict__ st, const int* __restrict__ ioff,
                               const int* __restrict__ iids, const float* __restrict__ wg,
                               float* __restrict__ w) {
  const int s = blockIdx.y;
  if (!slice_running(st, s)) return;
  const float* wgs = wg + (size_t)s * G;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n * n; j += gridDim.x * blockDim.x) {
    float acc = 0.f;
    for (int k = ioff[j]; k < ioff[j + 1]; ++k) acc += wgs[iids[k]];
    w[(size_t)s * n * n + j] = acc;
  }
}

void group_gather(int batch, int n, int G, cudaStream_t s, const SliceState* st, const int* inv_off,
                  const int* inv_ids, const float* wg, float* w) {
  const int N = n * n;
  const int blocks = (N + 255) / 256 < 256 ? (N + 255) / 256 : 256;
  k_group_gather<<<dim3(blocks, batch), 256, 0, s>>>(n, G, st, inv_off, inv_ids, wg, w);
}

__global__ void k_gm_count(int N, int G, int gsize, const int* __restrict__ gidx, const int* __restrict__ goff,
                           int* __restrict__ counts, int* __restrict__ err) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
    const int b = goff ? goff[g] : g * gsize;
    const int e = goff ? goff[g + 1] : b + gsize;
    if (e < b) {
      atomicExch(err, 1);
      continue;
    }
    for (int k = b; k < e; ++k) {
      const int j = gidx[k];
      if (j < 0 || j >= N) {
        atomicExch(err, 1);
      } else {
        atomicAdd(&counts[j], 1);
      }
    }
  }
}

// Exclusive scan of counts[0..N) into off[0..N], one block.
__global__ void k_scan_counts(int N, const int* __restrict__ counts, int* __restrict__ off) {
  __shared__ int sums[1024];
  const int t = threadIdx.x, nt = blockDim.x;
  const int chunk = (N + nt - 1) / nt;
  const int lo = min(N, t * chunk), hi = min(N, lo + chunk);
  int acc = 0;
  for (int i = lo; i < hi; ++i) acc += counts[i];
  sums[t] = acc;
  __syncthreads();
  for (int o = 1; o < nt; o <<= 1) {
    const int v = t >= o ? sums[t - o] : 0;
    __syncthreads();
    sums[t] += v;
    __syncthreads();
  }
  int run = t > 0 ? sums[t - 1] : 0;
  for (int i = lo; i < hi; ++i) {
    off[i] = run;
    run += counts[i];
  }
  if (t == nt - 1) off[N] = sums[nt - 1];
}

__global__ void k_gm_fill(int N, int G, int gsize, const int* __restrict__ gidx, const int* __restrict__ goff,
                          const int* __restrict__ ioff, int* __restrict__ cursor, int* __restrict__ iids,
                          const int* __restrict__ err) {
  if (*err) return;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
    const int b = goff ? goff[g] : g * gsize;
    const int e = goff ? goff[g + 1] : b + gsize;
    for (int k = b; k < e; ++k) {
      const int j = gidx[k];
      const int pos = atomicAdd(&cursor[j], 1);
      iids[ioff[j] + pos] = g;
    }
  }
}

__global__ void k_gm_sort(int N, const int* __restrict__ ioff, int* __restrict__ iids, const int* __restrict__ err) {
  if (*err) return;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += gridDim.x * blockDim.x) {
    const int b = ioff[j], e = ioff[j + 1];
    for (int a = b + 1; a < e; ++a) {
      const int v = iids[a];
      int k = a - 1;
      while (k >= b && iids[k] > v) {
        iids[k + 1] = iids[k];
        --k;
      }
      iids[k + 1] = v;
    }
  }
}

void group_inverse_build(int n, int G, int gsize, cudaStream_t s, const int* gidx, const int* goff,
                         int* counts, int* inv_off, int* inv_ids, int* cursor, int* err) {
  const int N = n * n;
  const int gb = (G + 255) / 256 < 1024 ? (G + 255) / 256 : 1024;
  const int nb = (N + 255) / 256 < 1024 ? (N + 255) / 256 : 1024;
  k_gm_count<<<gb, 256, 0, s>>>(N, G, gsize, gidx, goff, counts, err);
  k_scan_counts<<<1, 1024, 0, s>>>(N, counts, inv_off);
  k_gm_fill<<<gb, 256, 0, s>>>(N, G, gsize, gidx, goff, inv_off, cursor, inv_ids, err);
  k_gm_sort<<<nb, 256, 0, s>>>(N, inv_off, inv_ids, err);
}

__global__ void k_popcount(int N, const uint8_t* __restrict__ mask, int* __restrict__ counts) {
  const int s = blockIdx.y;
  __shared__ int red[32];
  int acc = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
    acc += mask[(size_t)s * N + i] ? 1 : 0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    atomicAdd(&counts[s], t);
  }
}

void mask_popcount(int batch, int n, cudaStream_t s, const uint8_t* mask, int* counts) {
  const int N = n * n;
  const int blocks = (N + 255) / 256 < 64 ? (N + 255) / 256 : 64;
  k_popcount<<<dim3(blocks, batch), 256, 0, s>>>(N, mask, counts);
}

// ========================================================== PCG scalars ===

FI double sum_parts(const double* part, int s, int slot, int np) {
  const double* p = part + ((size_t)s * NSLOT + slot) * MAXPART;
  double a = 0.0;
  for (int i = 0; i < np; ++i) a += p[i];
  return a;
}

__global__ void k_state_init(int B, SliceState* st, const double* part, int np, const int* counts, int N,
                             const float* lam, const float* lam_tv, float eps) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= B) return;
  SliceState v;
  v.rho = 0.0;
  v.alpha = 0.0;
  v.beta = 0.0;
  v.rhs2 = sum_parts(part, s, SLOT_RHS, np);
  v.rr = v.rhs2;
  v.relchg = 0.0;
  v.active = 1;
  v.done = 0;
  v.breakdown = 0;
  v.pcg_steps = 0;
  v.outer_done = 0;
  v.pad_ = 0;
  v.lam = lam[s];
  v.lam_tv = lam_tv[s];
  v.abar = (float)((double)counts[s] / (double)N);
  v.eps = eps;
  st[s] = v;
}

void state_init(int batch, cudaStream_t s, SliceState* st, const double* part, int np, const int* counts,
                int n, const float* lam, const float* lam_tv, float eps) {
  k_state_init<<<(batch + 127) / 128, 128, 0, s>>>(batch, st, part, np, counts, n * n, lam, lam_tv, eps);
}

__global__ void k_outer_begin(int B, SliceState* st) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= B) return;
  st[s].active = st[s].done ? 0 : 1;
}

void outer_begin(int batch, cudaStream_t s, SliceState* st) {
  k_outer_begin<<<(batch + 127) / 128, 128, 0, s>>>(batch, st);
}

__global__ void k_alpha(int B, SliceState* st, const double* part, int np) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= B || !slice_running(st, s)) return;
  const double dq = sum_parts(part, s, SLOT_DQ, np);
  const double rho = st[s].rho;
  if (rho == 0.0) {  // exact solution reached: nothing left to do
    st[s].alpha = 0.0;
    st[s].active = 0;
    return;
  }
  if (!(dq > 0.0) || !isfinite(dq) || !isfinite(rho)) {
    st[s].active = 0;
    st[s].breakdown = 1;
    return;
  }
  st[s].alpha = rho / dq;
  st[s].pcg_steps += 1;
}

void pcg_alpha(int batch, cudaStream_t s, SliceState* st, const double* part, int np) {
  k_alpha<<<(batch + 127) / 128, 128, 0, s>>>(batch, st, part, np);
}

__global__ void k_rho_init(int B, SliceState* st, const double* part, int np_rz, int np_rr) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= B || !slice_running(st, s)) return;
  st[s].rho = sum_parts(part, s, SLOT_RZ, np_rz);
  st[s].rr = sum_parts(part, s, SLOT_RR, np_rr);
  st[s].beta = 0.0;
}

void pcg_rho_init(int batch, cudaStream_t s, SliceState* st, const double* part, int np_rz, int np_rr) {
  k_rho_init<<<(batch + 127) / 128, 128, 0, s>>>(batch, st, part, np_rz, np_rr);
}

__global__ void k_beta(int B, SliceState* st, const double* part, int np_rz, int np_rr, float tol) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= B || !slice_running(st, s)) return;
  const double rz = sum_parts(part, s, SLOT_RZ, np_rz);
  const double rr = sum_parts(part, s, SLOT_RR, np_rr);
  st[s].rr = rr;
  if (tol > 0.f && sqrt(rr) <= (double)tol * sqrt(st[s].rhs2)) {
    st[s].active = 0;
    return;
  }
  st[s].beta = rz / st[s].rho;
  st[s].rho = rz;
}

void pcg_beta(int batch, cudaStream_t s, SliceState* st, const double* part, int np_rz, int np_rr,
              float tol) {
  k_beta<<<(batch + 127) / 128, 128, 0, s>>>(batch, st, part, np_rz, np_rr, tol);
}

__global__ void k_outer_end(int B, SliceState* st, const double* part, int np, float tol) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= B || st[s].done) return;
  const double dx = sum_parts(part, s, SLOT_DX, np);
  const double xx = sum_parts(part, s, SLOT_XX, np);
  const double rel = xx > 0.0 ? sqrt(dx / xx) : INFINITY;
  st[s].relchg = rel;
  st[s].outer_done += 1;
  if (tol > 0.f && rel <= (double)tol) st[s].done = 1;
}

void outer_end(int batch, cudaStream_t s, SliceState* st, const double* part, int np, float tol) {
  k_outer_end<<<(batch + 127) / 128, 128, 0, s>>>(batch, st, part, np, tol);
}

}  // namespace firls
