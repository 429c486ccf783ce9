// Mixed-radix (2/3/4/5/8/16) Stockham FFT of one length-N line held by T
// threads of one warp, E = N / T elements per thread in registers.
//
// Thread t holds elements t + T*s (s = 0..E-1) on entry and exit (natural
// order, so global loads/stores of a row are coalesced).  A pass of radix R
// with p = product of the radices already applied runs butterflies
// i = t + T*m (m < E/R); butterfly i reads inputs i + q*N/R (which are this
// thread's own registers in slot m + q*E/R), multiplies input q by
// w_{pR}^{q*(i mod p)}, takes an R-point DFT and writes output q to
// (i / p) * p * R + (i mod p) + q * p.  Between passes the outputs go
// through shared memory (structure-of-arrays floats, one padding word per 32
// to spread banks); after the last pass they are already in natural order
// in the thread's registers.  Unnormalised; DIR = -1 forward, +1 inverse.
#pragma once

#include "firls_common.cuh"

namespace firls {

template <int N> struct FftCfg;
#define FIRLS_FFT_CFG(n, e, np, r0, r1, r2, r3, r4)                                   \
  template <> struct FftCfg<n> {                                                      \
    static constexpr int E = e, T = n / e, NP = np;                                   \
    static constexpr __host__ __device__ int radix(int p) {                           \
      return p == 0 ? r0 : p == 1 ? r1 : p == 2 ? r2 : p == 3 ? r3 : r4;             \
    }                                                                                 \
  };
FIRLS_FFT_CFG(16, 4, 2, 4, 4, 1, 1, 1)
FIRLS_FFT_CFG(32, 4, 3, 2, 4, 4, 1, 1)
FIRLS_FFT_CFG(48, 12, 3, 3, 4, 4, 1, 1)
FIRLS_FFT_CFG(64, 8, 2, 8, 8, 1, 1, 1)
FIRLS_FFT_CFG(80, 20, 3, 5, 4, 4, 1, 1)
FIRLS_FFT_CFG(96, 12, 4, 3, 4, 4, 2, 1)
FIRLS_FFT_CFG(128, 16, 2, 16, 8, 1, 1, 1)
FIRLS_FFT_CFG(160, 20, 4, 5, 4, 4, 2, 1)
FIRLS_FFT_CFG(192, 12, 4, 3, 4, 4, 4, 1)
FIRLS_FFT_CFG(256, 16, 2, 16, 16, 1, 1, 1)
FIRLS_FFT_CFG(320, 20, 4, 5, 4, 4, 4, 1)
FIRLS_FFT_CFG(384, 12, 5, 3, 4, 4, 4, 2)
FIRLS_FFT_CFG(512, 16, 3, 8, 8, 8, 1, 1)
#undef FIRLS_FFT_CFG

// Shared-memory words per line buffer (re or im plane): one padding word per
// 16, so that a radix-16 pass of 16 threads stores word 17 t + q and reads
// word t + 17 s, both on 16 distinct banks; the plane length is 8 mod 16, so
// the two lines that share a warp (their buffers 2 planes apart, 16 banks
// apart) never meet on a bank either.
template <int N> __host__ __device__ constexpr int fft_line_words() {
  return N + (N >> 4) + ((8 - (N + (N >> 4)) % 16) + 16) % 16;
}
FI int fpad(int a) { return a + (a >> 4); }

// Shared twiddle tables, one per pass after the first: the pass with radix R
// applied after P points (P > 1) multiplies input q of butterfly k by
// w_N^(q k N / (P R)); its table holds those factors as [q - 1][k]
// (q = 1..R-1, k < P), so the threads of a line, whose k are consecutive,
// read consecutive entries.  The tables of all passes together hold N - R0
// entries (R0 the first radix); the table of the pass after P points starts
// at entry P - R0.
template <int N> __host__ __device__ constexpr int tw_words() { return (N + 1) & ~1; }
template <int N> __host__ __device__ constexpr int tw_bytes() { return tw_words<N>() * 8; }

// ---- small DFTs in registers (DIR = -1 forward, +1 inverse) ----
template <int DIR> FI float2 mul_i(float2 a) {  // a * (DIR * i)
  return DIR < 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
}

template <int R, int DIR> struct Dft;

template <int DIR> struct Dft<2, DIR> {
  static FI void run(float2* a) {
    float2 t = a[1];
    a[1] = csub(a[0], t);
    a[0] = cadd(a[0], t);
  }
};

template <int DIR> struct Dft<4, DIR> {
  static FI void run(float2* a) {
    float2 t0 = cadd(a[0], a[2]), t1 = csub(a[0], a[2]);
    float2 t2 = cadd(a[1], a[3]), t3 = mul_i<DIR>(csub(a[1], a[3]));
    a[0] = cadd(t0, t2);
    a[2] = csub(t0, t2);
    a[1] = cadd(t1, t3);
    a[3] = csub(t1, t3);
  }
};

template <int DIR> struct Dft<8, DIR> {
  static FI void run(float2* a) {
    float2 e[4] = {a[0], a[2], a[4], a[6]};
    float2 o[4] = {a[1], a[3], a[5], a[7]};
    Dft<4, DIR>::run(e);
    Dft<4, DIR>::run(o);
    const float h = 0.70710678118654752f;  // 1/sqrt(2)
    // w8^k = exp(DIR * i * pi * k / 4)
    float2 o1 = make_float2(h * (o[1].x - DIR * o[1].y), h * (o[1].y + DIR * o[1].x));
    float2 o2 = mul_i<DIR>(o[2]);
    float2 o3 = make_float2(h * (-o[3].x - DIR * o[3].y), h * (-o[3].y + DIR * o[3].x));
    a[0] = cadd(e[0], o[0]);
    a[4] = csub(e[0], o[0]);
    a[1] = cadd(e[1], o1);
    a[5] = csub(e[1], o1);
    a[2] = cadd(e[2], o2);
    a[6] = csub(e[2], o2);
    a[3] = cadd(e[3], o3);
    a[7] = csub(e[3], o3);
  }
};

template <int DIR> struct Dft<3, DIR> {
  static FI void run(float2* a) {
    const float s = 0.86602540378443865f;  // sin(2 pi / 3)
    float2 t = cadd(a[1], a[2]);
    float2 u = csub(a[1], a[2]);
    float2 m = make_float2(a[0].x - 0.5f * t.x, a[0].y - 0.5f * t.y);
    // DIR * i * s * u
    float2 v = make_float2(-DIR * s * u.y, DIR * s * u.x);
    a[0] = cadd(a[0], t);
    a[1] = cadd(m, v);
    a[2] = csub(m, v);
  }
};

template <int DIR> struct Dft<5, DIR> {
  static FI void run(float2* a) {
    const float c1 = 0.30901699437494742f;   // cos(2 pi / 5)
    const float c2 = -0.80901699437494742f;  // cos(4 pi / 5)
    const float s1 = 0.95105651629515357f;   // sin(2 pi / 5)
    const float s2 = 0.58778525229247313f;   // sin(4 pi / 5)
    float2 t1 = cadd(a[1], a[4]), t3 = csub(a[1], a[4]);
    float2 t2 = cadd(a[2], a[3]), t4 = csub(a[2], a[3]);
    float2 b1 = make_float2(a[0].x + c1 * t1.x + c2 * t2.x, a[0].y + c1 * t1.y + c2 * t2.y);
    float2 b2 = make_float2(a[0].x + c2 * t1.x + c1 * t2.x, a[0].y + c2 * t1.y + c1 * t2.y);
    float2 g1 = make_float2(s1 * t3.x + s2 * t4.x, s1 * t3.y + s2 * t4.y);
    float2 g2 = make_float2(s2 * t3.x - s1 * t4.x, s2 * t3.y - s1 * t4.y);
    // forward: A1 = b1 - i g1, A4 = b1 + i g1, A2 = b2 - i g2, A3 = b2 + i g2
    float2 ig1 = mul_i<DIR>(g1), ig2 = mul_i<DIR>(g2);  // DIR * i * g
    a[0] = cadd(a[0], cadd(t1, t2));
    a[1] = cadd(b1, ig1);
    a[4] = csub(b1, ig1);
    a[2] = cadd(b2, ig2);
    a[3] = csub(b2, ig2);
  }
};

// 16 = 4 x 4: four 4-point DFTs over n1 (stride 4), twiddles w16^(n2 k1),
// four 4-point DFTs over n2; output k1 + 4 k2.
template <int DIR> struct Dft<16, DIR> {
  static FI void run(float2* a) {
    const float c1 = 0.92387953251128674f;  // cos(pi/8)
    const float s1 = 0.38268343236508977f;  // sin(pi/8)
    const float h = 0.70710678118654752f;
    float2 b[4][4];
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
      float2 t[4] = {a[n2], a[4 + n2], a[8 + n2], a[12 + n2]};
      Dft<4, DIR>::run(t);
#pragma unroll
      for (int k1 = 0; k1 < 4; ++k1) b[n2][k1] = t[k1];
    }
    // w16^j = (cos(2 pi j/16), DIR sin(2 pi j/16)) for j = n2 * k1
    const float2 w1 = make_float2(c1, DIR * s1), w2 = make_float2(h, DIR * h), w3 = make_float2(s1, DIR * c1);
    const float2 w6 = make_float2(-h, DIR * h), w9 = make_float2(-c1, -DIR * s1);
    b[1][1] = cmul(b[1][1], w1);
    b[1][2] = cmul(b[1][2], w2);
    b[1][3] = cmul(b[1][3], w3);
    b[2][1] = cmul(b[2][1], w2);
    b[2][2] = mul_i<DIR>(b[2][2]);  // w16^4 = DIR i
    b[2][3] = cmul(b[2][3], w6);
    b[3][1] = cmul(b[3][1], w3);
    b[3][2] = cmul(b[3][2], w6);
    b[3][3] = cmul(b[3][3], w9);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      float2 t[4] = {b[0][k1], b[1][k1], b[2][k1], b[3][k1]};
      Dft<4, DIR>::run(t);
#pragma unroll
      for (int k2 = 0; k2 < 4; ++k2) a[k1 + 4 * k2] = t[k2];
    }
  }
};

template <int R, int DIR> struct Dft {
  static FI void run(float2*) {}
};

// Twiddle table in shared memory: tw[j] = exp(-2 pi i j / N).
template <int DIR> FI float2 twiddle(const float2* tw, int j) {
  float2 w = tw[j];
  return DIR < 0 ? w : make_float2(w.x, -w.y);
}

template <int N, int PASS, int P, int DIR>
FI void fft_pass(float2 (&v)[FftCfg<N>::E], float* bre, float* bim, const float2* tw, int t) {
  using C = FftCfg<N>;
  constexpr int R = C::radix(PASS);
  constexpr int E = C::E, T = C::T, M = E / R;
  constexpr bool LAST = (PASS == C::NP - 1);
  static_assert(E % R == 0, "radix must divide the per-thread element count");
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const int i = t + T * m;
    const int k = (P == 1) ? 0 : (i % P);
    float2 a[R];
#pragma unroll
    for (int q = 0; q < R; ++q) a[q] = v[m + q * M];
    if (P > 1) {
      const float2* twp = tw + (P - C::radix(0)) + k;
#pragma unroll
      for (int q = 1; q < R; ++q) a[q] = cmul(a[q], twiddle<DIR>(twp, (q - 1) * P));
    }
    Dft<R, DIR>::run(a);
    if (LAST) {
#pragma unroll
      for (int q = 0; q < R; ++q) v[m + q * M] = a[q];
    } else {
      const int j = (i / P) * P * R + k;
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const int ad = fpad(j + q * P);
        bre[ad] = a[q].x;
        bim[ad] = a[q].y;
      }
    }
  }
  if constexpr (!LAST) {
    __syncwarp();
#pragma unroll
    for (int s = 0; s < E; ++s) {
      const int ad = fpad(t + T * s);
      v[s] = make_float2(bre[ad], bim[ad]);
    }
    __syncwarp();
    fft_pass<N, PASS + 1, P * R, DIR>(v, bre, bim, tw, t);
  }
}

// In-register FFT of one line; bre/bim: this line's exchange buffers
// (fft_line_words<N>() floats each), tw: shared twiddle table.
template <int N, int DIR>
FI void fft_line(float2 (&v)[FftCfg<N>::E], float* bre, float* bim, const float2* tw, int t) {
  fft_pass<N, 0, 1, DIR>(v, bre, bim, tw, t);
}

}  // namespace firls
