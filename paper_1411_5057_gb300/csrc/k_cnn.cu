// Learned warm start: a 6-layer 3x3 CNN (3 -> 32 -> 32 -> 32 -> 32 -> 32 -> 2,
// ReLU between layers) that maps [Re A^H b, Im A^H b, mask] to a correction,
// x1 = A^H b + CNN(.).  BF16 weights and activations (NHWC), FP32 accumulation
// on the tensor cores, FP32 master weights and Adam.
//
// Forward and data-gradient convolutions run on tcgen05 (TMEM accumulators,
// k_conv3x3_tc) when n is a multiple of 128; otherwise, and for the weight
// gradient, on mma.m16n8k16.  The mma.sync form is an implicit GEMM per tile
// of 8 x 32 output pixels: the input
// tile with a one-pixel halo sits in shared memory; each of the 9 taps is a
// shifted view of it (the A operand, pixels x input channels) times the tap's
// weights (input x output channels).  The same kernel runs the backward data
// pass with the taps flipped and the channel roles swapped; the weight
// gradient sums X[p + tap]^T dZ[p] over all pixels with per-CTA partials and a
// fixed-order reduction (deterministic).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_bf16.h>

#include "firls.h"
#include "firls_common.cuh"
#include "per_device.h"

using namespace firls;

namespace {

constexpr int NL = 6;
constexpr int CH[NL + 1] = {3, 32, 32, 32, 32, 32, 2};
constexpr int CINP[NL] = {16, 32, 32, 32, 32, 32};   // padded input channels
constexpr int COUTP[NL] = {32, 32, 32, 32, 32, 16};  // padded output channels
constexpr int TH = 8, TW = 32;                       // output tile
constexpr int HH = TH + 2, HW = TW + 2;              // halo tile
constexpr int CONV_THREADS = 256;
constexpr int WG_CTAS = 296;                         // weight-gradient partials

FI uint32_t ld_u32(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }

FI void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

enum { MODE_HIDDEN = 0, MODE_LAST = 1, MODE_DGRAD = 2 };

// in:  bf16 [B][n][n][CIN]; wt: bf16 [9][COUT][CIN] (tap, out, in); bias f32 [COUT]
// HIDDEN: out bf16 [B][n][n][COUT] = relu(conv + bias)
// LAST:   x1 complex64 = atb + (conv + bias)[0..1]
// DGRAD:  out bf16 [B][n][n][COUT] = conv (no bias) * (gate > 0), gate bf16 [..][COUT]
template <int CIN, int COUT, int MODE>
__global__ void __launch_bounds__(CONV_THREADS) k_conv3x3(int n, const __nv_bfloat16* __restrict__ in,
                                                          const __nv_bfloat16* __restrict__ wt,
                                                          const float* __restrict__ bias,
                                                          __nv_bfloat16* __restrict__ out,
                                                          const __nv_bfloat16* __restrict__ gate,
                                                          const float2* __restrict__ atb, float2* __restrict__ x1) {
  constexpr int PS = CIN + 8;   // padded pixel stride (bf16) in shared memory
  constexpr int WS = CIN + 8;   // padded weight row stride
  constexpr int NT = COUT / 8;  // n-tiles
  extern __shared__ __align__(16) unsigned char smem[];
  __nv_bfloat16* xs = reinterpret_cast<__nv_bfloat16*>(smem);  // [HH*HW][PS]
  __nv_bfloat16* ws = xs + HH * HW * PS;                        // [9*COUT][WS]
  const int tiles_x = n / TW;
  const int ty0 = (blockIdx.x / tiles_x) * TH, tx0 = (blockIdx.x % tiles_x) * TW;
  const int img = blockIdx.y;
  const size_t ibase = (size_t)img * n * n;
  // halo tile, 16-byte chunks
  constexpr int CPP = CIN / 8;
  for (int idx = threadIdx.x; idx < HH * HW * CPP; idx += blockDim.x) {
    const int px = idx / CPP, ch = idx % CPP;
    const int y = ty0 - 1 + px / HW, x = tx0 - 1 + px % HW;
    uint4 v = make_uint4(0, 0, 0, 0);
    if (y >= 0 && y < n && x >= 0 && x < n)
      v = reinterpret_cast<const uint4*>(in + (ibase + (size_t)y * n + x) * CIN)[ch];
    *reinterpret_cast<uint4*>(xs + px * PS + ch * 8) = v;
  }
  for (int idx = threadIdx.x; idx < 9 * COUT * CPP; idx += blockDim.x) {
    const int row = idx / CPP, ch = idx % CPP;
    *reinterpret_cast<uint4*>(ws + row * WS + ch * 8) = reinterpret_cast<const uint4*>(wt + (size_t)row * CIN)[ch];
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, tg = lane & 3;
  float acc[2][NT][4];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int j = 0; j < NT; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[mt][j][e] = 0.f;
#pragma unroll
  for (int t = 0; t < 9; ++t) {
    const int dy = t / 3, dx = t % 3;
#pragma unroll
    for (int kc = 0; kc < CIN / 16; ++kc) {
      const int c0 = kc * 16 + 2 * tg;
      uint32_t a[2][4];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        const int p0 = (warp + dy) * HW + mt * 16 + g + dx;
        a[mt][0] = ld_u32(xs + p0 * PS + c0);
        a[mt][1] = ld_u32(xs + (p0 + 8) * PS + c0);
        a[mt][2] = ld_u32(xs + p0 * PS + c0 + 8);
        a[mt][3] = ld_u32(xs + (p0 + 8) * PS + c0 + 8);
      }
#pragma unroll
      for (int j = 0; j < NT; ++j) {
        const __nv_bfloat16* wr = ws + (t * COUT + j * 8 + g) * WS + c0;
        const uint32_t b0 = ld_u32(wr), b1 = ld_u32(wr + 8);
        mma_bf16(acc[0][j], a[0], b0, b1);
        mma_bf16(acc[1][j], a[1], b0, b1);
      }
    }
  }
  // epilogue: acc[mt][j][e] -> pixel (warp, mt*16 + g + 8*(e>>1)), channel j*8 + 2*tg + (e&1)
#pragma unroll
  for (int mt = 0; mt < 2; ++mt) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int y = ty0 + warp, x = tx0 + mt * 16 + g + 8 * h;
      const size_t p = ibase + (size_t)y * n + x;
#pragma unroll
      for (int j = 0; j < NT; ++j) {
        const int co = j * 8 + 2 * tg;
        float v0 = acc[mt][j][2 * h], v1 = acc[mt][j][2 * h + 1];
        if (MODE == MODE_LAST) {
          if (j == 0 && tg == 0) {  // channels 0, 1 = Re, Im of the correction
            const float2 ab = atb[p];
            x1[p] = make_float2(ab.x + v0 + bias[0], ab.y + v1 + bias[1]);
          }
        } else {
          if (MODE == MODE_HIDDEN) {
            v0 = fmaxf(v0 + bias[co], 0.f);
            v1 = fmaxf(v1 + bias[co + 1], 0.f);
          } else {
            const __nv_bfloat162 gt = *reinterpret_cast<const __nv_bfloat162*>(gate + p * COUT + co);
            if (!(__bfloat162float(gt.x) > 0.f)) v0 = 0.f;
            if (!(__bfloat162float(gt.y) > 0.f)) v1 = 0.f;
          }
          *reinterpret_cast<__nv_bfloat162*>(out + p * COUT + co) = __floats2bfloat162_rn(v0, v1);
        }
      }
    }
  }
}

template <int CIN, int COUT> constexpr int conv_smem() { return (HH * HW * (CIN + 8) + 9 * COUT * (CIN + 8)) * 2; }

// ---- the same convolution on the 5th-generation tensor cores (tcgen05) ----
// A CTA computes TC_R image rows x TC_W pixels.  Per output row r the GEMM
// D_r[pixel][co] = sum_tap sum_ci X[row r + dy][pixel + dx][ci] W[tap][co][ci]
// runs as 9 * CIN/16 tcgen05.mma (M = 128 pixels, N = COUT, K = 16) with its
// FP32 accumulator in TMEM (columns 32 r ..).  Operands sit in shared memory
// in the canonical K-major layout without swizzle: 8-channel planes of
// 16-byte pixel (or weight-row) records, so the A operand of tap (dy, dx) is
// the halo row r + dy starting at pixel dx: core matrices 128 bytes apart
// along M (SBO), planes one plane apart along K (LBO).  One thread issues the
// MMAs and commits them to an mbarrier; after the (bounded) wait each warp
// reads its 32 pixel lanes with tcgen05.ld and runs the epilogue.
constexpr int TC_W = 128, TC_R = 4, TC_HW = TC_W + 2, TC_HR = TC_R + 2;
constexpr int TC_THREADS = 128;

FI unsigned cnn_su32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// tcgen05 shared-memory matrix descriptor: start, leading (K) and stride (M/N)
// byte offsets, fixed version bits 46-48 = 1, no swizzle.
FI uint64_t umma_desc(const void* p, unsigned lbo, unsigned sbo) {
  uint64_t d = (uint64_t)((cnn_su32(p) & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Operand bytes, but at least 64 KB so that at most 3 CTAs share an SM and
// their 3 x 128 TMEM columns fit the SM's 512.
template <int CIN, int COUT> constexpr int tc_smem() {
  return TC_HR * TC_HW * CIN * 2 + 9 * COUT * CIN * 2 > 64 * 1024 ? TC_HR * TC_HW * CIN * 2 + 9 * COUT * CIN * 2
                                                                   : 64 * 1024;
}

template <int CIN, int COUT, int MODE>
__global__ void __launch_bounds__(TC_THREADS, 1) k_conv3x3_tc(int n, const __nv_bfloat16* __restrict__ in,
                                                              const __nv_bfloat16* __restrict__ wt,
                                                              const float* __restrict__ bias,
                                                              __nv_bfloat16* __restrict__ out,
                                                              const __nv_bfloat16* __restrict__ gate,
                                                              const float2* __restrict__ atb, float2* __restrict__ x1,
                                                              int* __restrict__ err) {
  constexpr int KP = CIN / 8;                  // 8-channel planes
  constexpr int XPL = TC_HR * TC_HW * 16;      // bytes per activation plane
  constexpr int WPL = COUT * 16;               // bytes per weight plane
  static_assert(COUT % 16 == 0 && COUT <= 32 && CIN % 16 == 0, "tcgen05 conv shape");
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char* xs = smem;                    // [KP][TC_HR * TC_HW pixels][16 B]
  unsigned char* wsm = smem + KP * XPL;        // [9][KP][COUT][16 B]
  __shared__ uint32_t tmem_base;
  __shared__ __align__(8) uint64_t bar;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int segs = n / TC_W;
  const int y0 = (blockIdx.x / segs) * TC_R, x0 = (blockIdx.x % segs) * TC_W;
  const int img = blockIdx.y;
  const size_t ibase = (size_t)img * n * n;
  // halo rows y0-1 .. y0+TC_R, pixels x0-1 .. x0+TC_W (zero outside the
  // image) and the weights: asynchronous 16-byte copies, all in flight at once
  for (int idx = t; idx < TC_HR * TC_HW * KP; idx += TC_THREADS) {
    const int px = idx / KP, ch = idx % KP;
    const int y = y0 - 1 + px / TC_HW, x = x0 - 1 + px % TC_HW;
    unsigned char* dst = xs + (size_t)ch * XPL + px * 16;
    if (y >= 0 && y < n && x >= 0 && x < n)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(cnn_su32(dst)),
                   "l"(reinterpret_cast<const uint4*>(in + (ibase + (size_t)y * n + x) * CIN) + ch)
                   : "memory");
    else
      *reinterpret_cast<uint4*>(dst) = make_uint4(0, 0, 0, 0);
  }
  for (int idx = t; idx < 9 * COUT * KP; idx += TC_THREADS) {
    const int row = idx / KP, ch = idx % KP;  // row = tap * COUT + co
    const int tap = row / COUT, co = row % COUT;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(
                     cnn_su32(wsm + ((size_t)(tap * KP + ch) * COUT + co) * 16)),
                 "l"(reinterpret_cast<const uint4*>(wt + (size_t)row * CIN) + ch)
                 : "memory");
  }
  asm volatile("cp.async.commit_group;\n cp.async.wait_all;\n" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // generic writes -> tensor core reads
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(cnn_su32(&tmem_base)),
                 "r"(TC_R * 32)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (t == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(cnn_su32(&bar)) : "memory");
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_base;
  // D f32, A and B bf16, both K-major, N >> 3 at bit 17, M >> 4 at bit 24
  constexpr uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(COUT >> 3) << 17) | ((uint32_t)(TC_W >> 4) << 24);
  if (t == 0) {
    for (int r = 0; r < TC_R; ++r) {
      const uint32_t d = tmem + (uint32_t)(r * 32);
      int k = 0;
      for (int tap = 0; tap < 9; ++tap) {
        const int dy = tap / 3, dx = tap % 3;
        for (int kk = 0; kk < CIN / 16; ++kk, ++k) {
          const uint64_t ad = umma_desc(xs + (size_t)(2 * kk) * XPL + ((r + dy) * TC_HW + dx) * 16, XPL, 128);
          const uint64_t bd = umma_desc(wsm + (size_t)(tap * KP + 2 * kk) * WPL, WPL, 128);
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
              "l"(ad), "l"(bd), "r"(idesc), "r"(k > 0 ? 1u : 0u)
              : "memory");
        }
      }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(cnn_su32(&bar))
                 : "memory");
  }
  bool done = false;
  for (int it = 0; it < 10000 && !done; ++it) {  // bounded (about a second): the MMAs take microseconds
    unsigned ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0, %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok)
                 : "r"(cnn_su32(&bar)), "r"(100000u)
                 : "memory");
    done = ok != 0;
  }
  done = __all_sync(0xffffffffu, done);
  if (!done && lane == 0) atomicExch(err, 1);
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  if (done) {
    for (int r = 0; r < TC_R; ++r) {
      uint32_t v[32];
      const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(r * 32);
      if (COUT == 32) {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
            "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
              "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
              "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
            : "r"(ta));
      } else {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(ta));
      }
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
      // this thread's pixel: row y0 + r, column x0 + 32 warp + lane
      const size_t p = ibase + (size_t)(y0 + r) * n + x0 + warp * 32 + lane;
      if (MODE == MODE_LAST) {
        const float2 ab = atb[p];
        x1[p] = make_float2(ab.x + __uint_as_float(v[0]) + bias[0], ab.y + __uint_as_float(v[1]) + bias[1]);
      } else {
        uint32_t pk[COUT / 2];
#pragma unroll
        for (int j = 0; j < COUT / 2; ++j) {
          float a = __uint_as_float(v[2 * j]), b = __uint_as_float(v[2 * j + 1]);
          if (MODE == MODE_HIDDEN) {
            a = fmaxf(a + bias[2 * j], 0.f);
            b = fmaxf(b + bias[2 * j + 1], 0.f);
          } else {
            const __nv_bfloat162 gt = *reinterpret_cast<const __nv_bfloat162*>(gate + p * COUT + 2 * j);
            if (!(__bfloat162float(gt.x) > 0.f)) a = 0.f;
            if (!(__bfloat162float(gt.y) > 0.f)) b = 0.f;
          }
          const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
          pk[j] = *reinterpret_cast<const uint32_t*>(&h);
        }
        uint4* o = reinterpret_cast<uint4*>(out + p * COUT);
#pragma unroll
        for (int q = 0; q < COUT / 8; ++q) o[q] = make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TC_R * 32) : "memory");
}

// dW[t][ci][co] = sum_p X[p + off(t)][ci] dZ[p][co]; db[co] = sum_p dZ[p][co].
// Per-CTA partials over a strided set of tiles: pw [cta][9][CIN][COUT], pb [cta][COUT].
template <int CIN, int COUT>
__global__ void __launch_bounds__(CONV_THREADS) k_wgrad(int n, int batch, const __nv_bfloat16* __restrict__ x,
                                                        const __nv_bfloat16* __restrict__ dz,
                                                        float* __restrict__ pw, float* __restrict__ pb) {
  constexpr int HP = HH * HW + 8;  // transposed halo row stride
  constexpr int ZP = TH * TW + 8;  // transposed dz row stride
  constexpr int MT = CIN / 16, NT = COUT / 8, NCOMBO = 9 * MT * NT;
  constexpr int PER_WARP = (NCOMBO + 7) / 8;
  extern __shared__ __align__(16) unsigned char smem[];
  __nv_bfloat16* xs = reinterpret_cast<__nv_bfloat16*>(smem);  // [CIN][HP]
  __nv_bfloat16* zs = xs + CIN * HP;                            // [COUT][ZP]
  float* bsum = reinterpret_cast<float*>(zs + COUT * ZP);       // [COUT]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, tg = lane & 3;
  float acc[PER_WARP][4];
#pragma unroll
  for (int i = 0; i < PER_WARP; ++i)
#pragma unroll
    for (int e = 0; e < 4; ++e) acc[i][e] = 0.f;
  float bacc = 0.f;  // thread co = threadIdx.x < COUT
  const int tiles_x = n / TW, tiles = tiles_x * (n / TH) * batch;
  for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int img = tile / (tiles_x * (n / TH)), r = tile % (tiles_x * (n / TH));
    const int ty0 = (r / tiles_x) * TH, tx0 = (r % tiles_x) * TW;
    const size_t ibase = (size_t)img * n * n;
    __syncthreads();
    for (int idx = threadIdx.x; idx < HH * HW * CIN; idx += blockDim.x) {
      const int px = idx / CIN, ci = idx % CIN;
      const int y = ty0 - 1 + px / HW, xx = tx0 - 1 + px % HW;
      __nv_bfloat16 v = __float2bfloat16(0.f);
      if (y >= 0 && y < n && xx >= 0 && xx < n) v = x[(ibase + (size_t)y * n + xx) * CIN + ci];
      xs[ci * HP + px] = v;
    }
    for (int idx = threadIdx.x; idx < TH * TW * COUT; idx += blockDim.x) {
      const int px = idx / COUT, co = idx % COUT;
      zs[co * ZP + px] = dz[(ibase + (size_t)(ty0 + px / TW) * n + tx0 + px % TW) * COUT + co];
    }
    __syncthreads();
    if (threadIdx.x < COUT) {
      float s = 0.f;
      for (int px = 0; px < TH * TW; ++px) s += __bfloat162float(zs[threadIdx.x * ZP + px]);
      bacc += s;
    }
#pragma unroll
    for (int i = 0; i < PER_WARP; ++i) {
      const int combo = warp * PER_WARP + i;
      if (combo >= NCOMBO) break;
      const int t = combo / (MT * NT), mt = (combo / NT) % MT, nt = combo % NT;
      const int dy = t / 3, dx = t % 3;
      for (int kc = 0; kc < TH * TW / 16; ++kc) {
        const int k0 = kc * 16 + 2 * tg;  // output pixel index (pairs stay in one tile row)
        const int hp0 = (k0 / TW + dy) * HW + k0 % TW + dx;
        const int hp1 = ((k0 + 8) / TW + dy) * HW + (k0 + 8) % TW + dx;
        const __nv_bfloat16* xr0 = xs + (mt * 16 + g) * HP;
        const __nv_bfloat16* xr1 = xs + (mt * 16 + g + 8) * HP;
        uint32_t a[4];
        auto pack = [](__nv_bfloat16 lo, __nv_bfloat16 hi) {
          return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
        };
        a[0] = pack(xr0[hp0], xr0[hp0 + 1]);
        a[1] = pack(xr1[hp0], xr1[hp0 + 1]);
        a[2] = pack(xr0[hp1], xr0[hp1 + 1]);
        a[3] = pack(xr1[hp1], xr1[hp1 + 1]);
        const __nv_bfloat16* zr = zs + (nt * 8 + g) * ZP;
        const uint32_t b0 = ld_u32(zr + k0), b1 = ld_u32(zr + k0 + 8);
        mma_bf16(acc[i], a, b0, b1);
      }
    }
  }
  float* pwc = pw + (size_t)blockIdx.x * 9 * CIN * COUT;
#pragma unroll
  for (int i = 0; i < PER_WARP; ++i) {
    const int combo = warp * PER_WARP + i;
    if (combo >= NCOMBO) break;
    const int t = combo / (MT * NT), mt = (combo / NT) % MT, nt = combo % NT;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int ci = mt * 16 + g + 8 * (e >> 1), co = nt * 8 + 2 * tg + (e & 1);
      pwc[((size_t)t * CIN + ci) * COUT + co] = acc[i][e];
    }
  }
  if (threadIdx.x < COUT) pb[(size_t)blockIdx.x * COUT + threadIdx.x] = bacc;
  (void)bsum;
}

template <int CIN, int COUT> constexpr int wgrad_smem() {
  return (CIN * (HH * HW + 8) + COUT * (TH * TW + 8)) * 2 + COUT * 4;
}

// Fixed-order sum of the per-CTA partials into the real-size FP32 gradients.
__global__ void k_wgrad_reduce(int ctas, int cinp, int coutp, int cin, int cout, const float* __restrict__ pw,
                               const float* __restrict__ pb, float* __restrict__ dw, float* __restrict__ db) {
  const int total = 9 * cin * cout;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total + cout; i += gridDim.x * blockDim.x) {
    double s = 0.0;
    if (i < total) {
      const int t = i / (cin * cout), ci = (i / cout) % cin, co = i % cout;
      for (int k = 0; k < ctas; ++k) s += pw[((size_t)k * 9 + t) * cinp * coutp + (size_t)ci * coutp + co];
      dw[i] = (float)s;
    } else {
      const int co = i - total;
      for (int k = 0; k < ctas; ++k) s += pb[(size_t)k * coutp + co];
      db[co] = (float)s;
    }
  }
}

// NHWC bf16 input [B][n][n][16]: Re A^H b, Im A^H b, mask, zeros.
__global__ void k_cnn_input(int total, const float2* __restrict__ atb, const uint8_t* __restrict__ mask,
                            __nv_bfloat16* __restrict__ in) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < total; p += gridDim.x * blockDim.x) {
    const float2 a = atb[p];
    __nv_bfloat16 v[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) v[c] = __float2bfloat16(0.f);
    v[0] = __float2bfloat16(a.x);
    v[1] = __float2bfloat16(a.y);
    v[2] = __float2bfloat16(mask[p] ? 1.f : 0.f);
    uint4* o = reinterpret_cast<uint4*>(in + (size_t)p * 16);
    o[0] = *reinterpret_cast<uint4*>(v);
    o[1] = *reinterpret_cast<uint4*>(v + 8);
  }
}

// dOut = 2 (x1 - target) as bf16 [B][n][n][16] (channels 0, 1) and partial
// sums of |x1 - target|^2.
__global__ void k_cnn_loss(int total, const float2* __restrict__ x1, const float2* __restrict__ tgt,
                           __nv_bfloat16* __restrict__ dout, double* __restrict__ part) {
  __shared__ double red[32];
  float acc = 0.f;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < total; p += gridDim.x * blockDim.x) {
    const float2 r = make_float2(x1[p].x - tgt[p].x, x1[p].y - tgt[p].y);
    acc += r.x * r.x + r.y * r.y;
    __nv_bfloat16 v[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) v[c] = __float2bfloat16(0.f);
    v[0] = __float2bfloat16(2.f * r.x);
    v[1] = __float2bfloat16(2.f * r.y);
    uint4* o = reinterpret_cast<uint4*>(dout + (size_t)p * 16);
    o[0] = *reinterpret_cast<uint4*>(v);
    o[1] = *reinterpret_cast<uint4*>(v + 8);
  }
  const double tot = block_sum((double)acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// Adam (Kingma & Ba) on the FP32 master copy.
__global__ void k_adam(int count, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// Pack FP32 master weights [9][cin][cout] into the bf16 forward layout
// [9][coutp][cinp] and the data-gradient layout [9][cinp][coutp] (taps flipped).
__global__ void k_pack(int cin, int cout, int cinp, int coutp, const float* __restrict__ w,
                       __nv_bfloat16* __restrict__ wf, __nv_bfloat16* __restrict__ wd) {
  const int total = 9 * cinp * coutp;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const int t = i / (cinp * coutp), ci = (i / coutp) % cinp, co = i % coutp;
    const float v = (ci < cin && co < cout) ? w[((size_t)t * cin + ci) * cout + co] : 0.f;
    wf[((size_t)t * coutp + co) * cinp + ci] = __float2bfloat16(v);
    if (wd) wd[((size_t)(8 - t) * cinp + ci) * coutp + co] = __float2bfloat16(v);
  }
}

__global__ void k_pad_bias(int cout, int coutp, const float* __restrict__ b, float* __restrict__ bp) {
  const int i = threadIdx.x;
  if (i < coutp) bp[i] = i < cout ? b[i] : 0.f;
}

}  // namespace

struct firls_cnn {
  int n = 0, batch = 0;
  cudaStream_t stream = nullptr;
  std::vector<void*> allocs;
  float *w[NL] = {}, *b[NL] = {}, *bp[NL] = {};           // FP32 master, padded bias
  float *mw[NL] = {}, *vw[NL] = {}, *mb[NL] = {}, *vb[NL] = {};
  float *gw[NL] = {}, *gb[NL] = {};
  __nv_bfloat16 *wf[NL] = {}, *wd[NL] = {};
  __nv_bfloat16* act[NL] = {};  // act[0] input (16 ch), act[l] output of layer l (32 ch)
  __nv_bfloat16 *dza = nullptr, *dzb = nullptr;
  float *pw = nullptr, *pb = nullptr;
  double* lpart = nullptr;
  int* err = nullptr;  // set by a tcgen05 convolution whose bounded wait ran out
  int adam_t = 0;
  bool params_set = false;
};

namespace {

template <typename T> firls_status cnn_alloc(firls_cnn* c, T** p, size_t count) {
  void* v = nullptr;
  if (cudaMalloc(&v, count * sizeof(T) + 16) != cudaSuccess) return FIRLS_E_NOMEM;
  c->allocs.push_back(v);
  *p = static_cast<T*>(v);
  return FIRLS_OK;
}

template <int CIN, int COUT, int MODE> void launch_conv(firls_cnn* c, const __nv_bfloat16* in, const __nv_bfloat16* wt,
                                                       const float* bias, __nv_bfloat16* out,
                                                       const __nv_bfloat16* gate, const float2* atb, float2* x1) {
  if (c->n % TC_W == 0 && c->n % TC_R == 0) {  // tcgen05 form
    static PerDeviceOnce tattr;
    tattr.run([] {
      return cudaFuncSetAttribute(k_conv3x3_tc<CIN, COUT, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  tc_smem<CIN, COUT>()) == cudaSuccess;
    });
    const dim3 grid((c->n / TC_W) * (c->n / TC_R), c->batch);
    k_conv3x3_tc<CIN, COUT, MODE><<<grid, TC_THREADS, tc_smem<CIN, COUT>(), c->stream>>>(c->n, in, wt, bias, out, gate,
                                                                                          atb, x1, c->err);
    return;
  }
  static PerDeviceOnce attr;
  attr.run([] {
    return cudaFuncSetAttribute(k_conv3x3<CIN, COUT, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                conv_smem<CIN, COUT>()) == cudaSuccess;
  });
  const dim3 grid((c->n / TW) * (c->n / TH), c->batch);
  k_conv3x3<CIN, COUT, MODE><<<grid, CONV_THREADS, conv_smem<CIN, COUT>(), c->stream>>>(c->n, in, wt, bias, out, gate,
                                                                                         atb, x1);
}

template <int CIN, int COUT> void launch_wgrad(firls_cnn* c, const __nv_bfloat16* x, const __nv_bfloat16* dz, int l) {
  static PerDeviceOnce attr;
  attr.run([] {
    return cudaFuncSetAttribute(k_wgrad<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                wgrad_smem<CIN, COUT>()) == cudaSuccess;
  });
  k_wgrad<CIN, COUT><<<WG_CTAS, CONV_THREADS, wgrad_smem<CIN, COUT>(), c->stream>>>(c->n, c->batch, x, dz, c->pw,
                                                                                   c->pb);
  k_wgrad_reduce<<<64, 256, 0, c->stream>>>(WG_CTAS, CIN, COUT, CH[l], CH[l + 1], c->pw, c->pb, c->gw[l], c->gb[l]);
}

void pack_all(firls_cnn* c) {
  for (int l = 0; l < NL; ++l) {
    k_pack<<<64, 256, 0, c->stream>>>(CH[l], CH[l + 1], CINP[l], COUTP[l], c->w[l], c->wf[l], c->wd[l]);
    k_pad_bias<<<1, 64, 0, c->stream>>>(CH[l + 1], COUTP[l], c->b[l], c->bp[l]);
  }
}

void forward(firls_cnn* c, const float2* atb, const uint8_t* mask, float2* x1) {
  const int total = c->batch * c->n * c->n;
  k_cnn_input<<<1024, 256, 0, c->stream>>>(total, atb, mask, c->act[0]);
  launch_conv<16, 32, MODE_HIDDEN>(c, c->act[0], c->wf[0], c->bp[0], c->act[1], nullptr, nullptr, nullptr);
  for (int l = 1; l < 5; ++l)
    launch_conv<32, 32, MODE_HIDDEN>(c, c->act[l], c->wf[l], c->bp[l], c->act[l + 1], nullptr, nullptr, nullptr);
  launch_conv<32, 16, MODE_LAST>(c, c->act[5], c->wf[5], c->bp[5], nullptr, nullptr, atb, x1);
}

}  // namespace

extern "C" firls_status firls_cnn_create(firls_cnn** out, int n, int batch, void* cuda_stream) {
  if (!out) return FIRLS_E_INVALID_ARG;
  *out = nullptr;
  if (n < TW || n % TW || n % TH || batch < 1 || batch > 65535) return FIRLS_E_SHAPE;
  firls_cnn* c = new firls_cnn();
  c->n = n;
  c->batch = batch;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  const size_t P = (size_t)batch * n * n;
  firls_status s = FIRLS_OK;
  auto A = [&](auto** p, size_t cnt) {
    if (s == FIRLS_OK) s = cnn_alloc(c, p, cnt);
  };
  for (int l = 0; l < NL; ++l) {
    const size_t nw = 9 * (size_t)CH[l] * CH[l + 1];
    A(&c->w[l], nw);
    A(&c->mw[l], nw);
    A(&c->vw[l], nw);
    A(&c->gw[l], nw);
    A(&c->b[l], (size_t)CH[l + 1]);
    A(&c->mb[l], (size_t)CH[l + 1]);
    A(&c->vb[l], (size_t)CH[l + 1]);
    A(&c->gb[l], (size_t)CH[l + 1]);
    A(&c->bp[l], (size_t)COUTP[l]);
    A(&c->wf[l], 9 * (size_t)CINP[l] * COUTP[l]);
    A(&c->wd[l], 9 * (size_t)CINP[l] * COUTP[l]);
    A(&c->act[l], P * (l == 0 ? 16 : 32));
  }
  A(&c->dza, P * 32);
  A(&c->dzb, P * 32);
  A(&c->pw, (size_t)WG_CTAS * 9 * 32 * 32);
  A(&c->pb, (size_t)WG_CTAS * 32);
  A(&c->lpart, 1024);
  A(&c->err, 1);
  if (s != FIRLS_OK) {
    firls_cnn_destroy(c);
    return s;
  }
  cudaMemset(c->err, 0, sizeof(int));
  *out = c;
  return FIRLS_OK;
}

extern "C" firls_status firls_cnn_set_params(firls_cnn* c, const float* const* w, const float* const* b) {
  if (!c || !w || !b) return FIRLS_E_INVALID_ARG;
  for (int l = 0; l < NL; ++l) {
    const size_t nw = 9 * (size_t)CH[l] * CH[l + 1];
    if (cudaMemcpyAsync(c->w[l], w[l], nw * 4, cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
        cudaMemcpyAsync(c->b[l], b[l], CH[l + 1] * 4, cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
      return FIRLS_E_CUDA;
    cudaMemsetAsync(c->mw[l], 0, nw * 4, c->stream);
    cudaMemsetAsync(c->vw[l], 0, nw * 4, c->stream);
    cudaMemsetAsync(c->mb[l], 0, CH[l + 1] * 4, c->stream);
    cudaMemsetAsync(c->vb[l], 0, CH[l + 1] * 4, c->stream);
  }
  c->adam_t = 0;
  pack_all(c);
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return FIRLS_E_CUDA;
  c->params_set = true;
  return FIRLS_OK;
}

extern "C" firls_status firls_cnn_get_params(firls_cnn* c, float* const* w, float* const* b) {
  if (!c || !w || !b) return FIRLS_E_INVALID_ARG;
  for (int l = 0; l < NL; ++l) {
    const size_t nw = 9 * (size_t)CH[l] * CH[l + 1];
    if (w[l] && cudaMemcpyAsync(w[l], c->w[l], nw * 4, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
      return FIRLS_E_CUDA;
    if (b[l] && cudaMemcpyAsync(b[l], c->b[l], CH[l + 1] * 4, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
      return FIRLS_E_CUDA;
  }
  return cudaStreamSynchronize(c->stream) == cudaSuccess ? FIRLS_OK : FIRLS_E_CUDA;
}

extern "C" firls_status firls_cnn_get_grads(firls_cnn* c, float* const* gw, float* const* gb) {
  if (!c || !gw || !gb) return FIRLS_E_INVALID_ARG;
  for (int l = 0; l < NL; ++l) {
    const size_t nw = 9 * (size_t)CH[l] * CH[l + 1];
    if (gw[l] && cudaMemcpyAsync(gw[l], c->gw[l], nw * 4, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
      return FIRLS_E_CUDA;
    if (gb[l] && cudaMemcpyAsync(gb[l], c->gb[l], CH[l + 1] * 4, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
      return FIRLS_E_CUDA;
  }
  return cudaStreamSynchronize(c->stream) == cudaSuccess ? FIRLS_OK : FIRLS_E_CUDA;
}

extern "C" firls_status firls_cnn_forward(firls_cnn* c, const void* atb, const uint8_t* mask, void* x1) {
  if (!c || !atb || !mask || !x1) return FIRLS_E_INVALID_ARG;
  if (!c->params_set) return FIRLS_E_STATE;
  forward(c, static_cast<const float2*>(atb), mask, static_cast<float2*>(x1));
  return cudaGetLastError() == cudaSuccess ? FIRLS_OK : FIRLS_E_CUDA;
}

extern "C" firls_status firls_cnn_train_step(firls_cnn* c, const void* atb, const uint8_t* mask, const void* target,
                                             void* x1, float lr, double* loss) {
  if (!c || !atb || !mask || !target || !x1) return FIRLS_E_INVALID_ARG;
  if (!c->params_set) return FIRLS_E_STATE;
  if (!(lr >= 0.f)) return FIRLS_E_INVALID_ARG;
  float2* xo = static_cast<float2*>(x1);
  forward(c, static_cast<const float2*>(atb), mask, xo);
  const int total = c->batch * c->n * c->n;
  const int lblocks = 1024;
  k_cnn_loss<<<lblocks, 256, 0, c->stream>>>(total, xo, static_cast<const float2*>(target), c->dza, c->lpart);
  // layer 6: dZ6 = dOut (16 channels)
  launch_wgrad<32, 16>(c, c->act[5], c->dza, 5);
  launch_conv<16, 32, MODE_DGRAD>(c, c->dza, c->wd[5], nullptr, c->dzb, c->act[5], nullptr, nullptr);
  __nv_bfloat16 *cur = c->dzb, *nxt = c->dza;
  for (int l = 4; l >= 1; --l) {
    launch_wgrad<32, 32>(c, c->act[l], cur, l);
    launch_conv<32, 32, MODE_DGRAD>(c, cur, c->wd[l], nullptr, nxt, c->act[l], nullptr, nullptr);
    __nv_bfloat16* t = cur;
    cur = nxt;
    nxt = t;
  }
  launch_wgrad<16, 32>(c, c->act[0], cur, 0);
  // Adam
  c->adam_t += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - (float)std::pow(0.9, c->adam_t), c2 = 1.f - (float)std::pow(0.999, c->adam_t);
  for (int l = 0; l < NL; ++l) {
    const int nw = 9 * CH[l] * CH[l + 1];
    k_adam<<<64, 256, 0, c->stream>>>(nw, c->w[l], c->gw[l], c->mw[l], c->vw[l], lr, b1, b2, 1e-8f, c1, c2);
    k_adam<<<1, 64, 0, c->stream>>>(CH[l + 1], c->b[l], c->gb[l], c->mb[l], c->vb[l], lr, b1, b2, 1e-8f, c1, c2);
  }
  pack_all(c);
  if (loss) {
    std::vector<double> h(lblocks);
    if (cudaMemcpyAsync(h.data(), c->lpart, sizeof(double) * lblocks, cudaMemcpyDeviceToHost, c->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
      return FIRLS_E_CUDA;
    double s = 0.0;
    for (double v : h) s += v;
    *loss = s;
    int e = 0;
    if (cudaMemcpy(&e, c->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return FIRLS_E_CUDA;
    if (e) return FIRLS_E_DEVICE_TIMEOUT;
  }
  return cudaGetLastError() == cudaSuccess ? FIRLS_OK : FIRLS_E_CUDA;
}

extern "C" void firls_cnn_destroy(firls_cnn* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  for (void* p : c->allocs)
    if (p) cudaFree(p);
  delete c;
}
