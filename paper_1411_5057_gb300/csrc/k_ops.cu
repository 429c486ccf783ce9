// Non-FFT kernels of the FIRLS hot path: lifting wavelets (Phi, Phi^T),
// weights (Eq. gw, Eq. Wog, Eq. wi), preconditioner set-up and application
// (Eq. pog, Eq. ptv with the L U factors of Sec. 4.2), PCG vector updates
// and the FP64 PCG scalars.
#include "launch.h"
#include "per_device.h"

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

constexpr int WAV_THREADS = 256;
constexpr int WAV_RB = 8;            // output row pairs per CTA of a tiled level
constexpr int COARSE_MAX = 64;       // default largest block kept whole in shared memory
constexpr int COARSE_LIMIT = 64;     // the in-shared-memory transform handles up to 64^2 (2 pairs per lane)
constexpr int COARSE_THREADS = 256;

static int wav_rb(int m, int want = 0) {
  const int rb = want > 0 ? want : WAV_RB;
  return m / 2 < rb ? m / 2 : rb;
}

// One tiled analysis level on the m x m block `in` (row stride ld_in).  The
// horizontal step reads the input rows straight from global memory (16-byte
// pairs), the vertical step works from shared memory.
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
  float2* rt = reinterpret_cast<float2*>(smem);  // [nrow][m] row-transformed
  const float2* src = in + (size_t)s * in_ss;
  for (int idx = threadIdx.x; idx < nrow * half; idx += blockDim.x) {
    const int i = idx / half, k = idx % half;
    const float4* xr = reinterpret_cast<const float4*>(src + (size_t)((2 * k0 + i) % m) * ld_in);
    const float4 p0 = xr[k];
    float2 a, d;
    if (kind == 2) {
      const float4 p1 = xr[k + 1 < half ? k + 1 : 0];
      lift::fwd_db4(make_float2(p0.x, p0.y), make_float2(p0.z, p0.w), make_float2(p1.x, p1.y),
                    make_float2(p1.z, p1.w), a, d);
    } else {
      lift::fwd_haar(make_float2(p0.x, p0.y), make_float2(p0.z, p0.w), a, d);
    }
    rt[i * m + k] = a;
    rt[i * m + half + k] = d;
  }
  __syncthreads();
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
      if (!h && j < half && !last) {  // LL of a non-final level: raw, to the ping-pong buffer
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

// One tiled synthesis level: LL from `lli` (row stride ld_ll), details from c
// (stride n) to the m x m output block.  Vertical step from global memory,
// horizontal step from shared memory; optional partial Re<r, out>.
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
  float2* vs = reinterpret_cast<float2*>(smem);  // [2 rb][m]
  const float2* cs = c + (size_t)s * n * n;
  const float2* ls = lli + (size_t)s * ll_ss;
  for (int idx = threadIdx.x; idx < nout * m; idx += blockDim.x) {
    const int kk = idx / m, j = idx % m;
    const int k = k0 + kk;
    const float2 al = j < half ? ls[(size_t)k * ld_ll + j] : cs[(size_t)k * n + j];
    const float2 dl = cs[(size_t)(half + k) * n + j];
    float2 x0, x1;
    if (kind == 2) {
      const int km = (k - 1 + half) % half;
      const float2 am = j < half ? ls[(size_t)km * ld_ll + j] : cs[(size_t)km * n + j];
      const float2 dm = cs[(size_t)(half + km) * n + j];
      lift::inv_db4(am, dm, al, dl, x0, x1);
    } else {
      lift::inv_haar(al, dl, x0, x1);
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
    reinterpret_cast<float4*>(os + (size_t)orow * ld_out)[l] = make_float4(x0.x, x0.y, x1.x, x1.y);
    if (rs) {
      const float4 rv = reinterpret_cast<const float4*>(rs + (size_t)orow * n)[l];
      acc += rdot2(make_float2(rv.x, rv.y), x0) + rdot2(make_float2(rv.z, rv.w), x1);
    }
  }
  if (part) {
    const double tot = block_sum((double)acc, red);
    if (threadIdx.x == 0) part[((size_t)s * NSLOT + SLOT_RZ) * MAXPART + blockIdx.x] = tot;
  }
}

// ---- coarse levels of one slice in shared memory ----
// In-place one-level analysis of the top-left m x m block of S (row stride
// ls): every lane reads the inputs of its pairs, the warp syncs, then writes
// [lo | hi].  m <= COARSE_MAX, so a lane holds at most two pairs.
FI void smem_fwd_level(float2* S, int ls, int m, int kind) {
  const int half = m / 2, lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int pass = 0; pass < 2; ++pass) {  // 0: rows, 1: columns
    const int es = pass ? ls : 1;         // element stride along the line
    for (int line = wid; line < m; line += nw) {
      float2* L = pass ? S + line : S + (size_t)line * ls;
      float2 a[2], d[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int k = lane + 32 * u;
        if (k < half) {
          if (kind == 2) {
            lift::fwd_db4(L[(2 * k) * es], L[(2 * k + 1) * es], L[((2 * k + 2) % m) * es],
                          L[((2 * k + 3) % m) * es], a[u], d[u]);
          } else {
            lift::fwd_haar(L[(2 * k) * es], L[(2 * k + 1) * es], a[u], d[u]);
          }
        }
      }
      __syncwarp();
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int k = lane + 32 * u;
        if (k < half) {
          L[k * es] = a[u];
          L[(half + k) * es] = d[u];
        }
      }
      __syncwarp();
    }
    __syncthreads();
  }
}

// In-place inverse of smem_fwd_level (columns first, then rows).
FI void smem_inv_level(float2* S, int ls, int m, int kind) {
  const int half = m / 2, lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int pass = 0; pass < 2; ++pass) {  // 0: columns, 1: rows
    const int es = pass ? 1 : ls;
    for (int line = wid; line < m; line += nw) {
      float2* L = pass ? S + (size_t)line * ls : S + line;
      float2 x0[2], x1[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int l = lane + 32 * u;
        if (l < half) {
          if (kind == 2) {
            const int lm = (l - 1 + half) % half;
            lift::inv_db4(L[lm * es], L[(half + lm) * es], L[l * es], L[(half + l) * es], x0[u], x1[u]);
          } else {
            lift::inv_haar(L[l * es], L[(half + l) * es], x0[u], x1[u]);
          }
        }
      }
      __syncwarp();
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int l = lane + 32 * u;
        if (l < half) {
          L[(2 * l) * es] = x0[u];
          L[(2 * l + 1) * es] = x1[u];
        }
      }
      __syncwarp();
    }
    __syncthreads();
  }
}

enum { COARSE_FWD = 1, COARSE_INV = 2 };

// Levels l0..L of one slice on the m0 x m0 block (m0 <= COARSE_MAX) held in
// shared memory.  FWD: analysis of `src`; without INV the coefficients are
// stored per `mode` at their Mallat positions (top-left block of c / w).
// FWD|INV: analysis, per-coefficient scaling (MUL_W or MUL_PINV), synthesis;
// the coarse coefficients never leave shared memory.  INV alone: synthesis
// of the coefficients read from c.  The synthesised block goes to `dst`.
__global__ void __launch_bounds__(COARSE_THREADS)
k_wav_coarse(const float2* __restrict__ src, size_t src_ss, int src_ld, float2* __restrict__ dst, size_t dst_ss,
             int dst_ld, float2* __restrict__ c, float* __restrict__ w, int n, int m0, int nlev, int kind,
             int mode, int flags, const float2* __restrict__ r, double* __restrict__ part, int real,
             const SliceState* __restrict__ st) {
  const int s = blockIdx.x;
  if (st != nullptr && !slice_running(st, s)) return;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[32];
  float2* S = reinterpret_cast<float2*>(smem);
  const int ls = m0 + 1;
  const size_t nn = (size_t)n * n;
  float2* cs = c + (size_t)s * nn;
  float* ws = w ? w + (size_t)s * nn : nullptr;
  const int cnt = m0 * m0;
  // the block goes to shared memory with asynchronous 8-byte copies, all in
  // flight at once (rows keep the odd stride ls that spreads column accesses)
  {
    const float2* sp = (flags & COARSE_FWD) ? src + (size_t)s * src_ss : cs;
    const size_t sld = (flags & COARSE_FWD) ? (size_t)src_ld : (size_t)n;
    for (int idx = threadIdx.x; idx < cnt; idx += blockDim.x) {
      const int rr = idx / m0, cc = idx % m0;
      asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(
                       (unsigned)__cvta_generic_to_shared(S + rr * ls + cc)),
                   "l"(sp + rr * sld + cc)
                   : "memory");
    }
    asm volatile("cp.async.commit_group;\n cp.async.wait_all;\n" ::: "memory");
  }
  __syncthreads();
  if (flags & COARSE_FWD) {
    // the coefficient weights this thread scales, fetched before the levels run
    constexpr int WMAX = COARSE_LIMIT * COARSE_LIMIT / COARSE_THREADS;
    float wv[WMAX];
    if ((flags & COARSE_INV) && ws) {
#pragma unroll
      for (int k = 0; k < WMAX; ++k) {
        const int idx = threadIdx.x + COARSE_THREADS * k;
        wv[k] = idx < cnt ? ws[(size_t)(idx / m0) * n + idx % m0] : 0.f;
      }
    }
    for (int lev = 0; lev < nlev; ++lev) smem_fwd_level(S, ls, m0 >> lev, kind);
    const float lam = st ? st[s].lam : 0.f, abar = st ? st[s].abar : 0.f, eps = st ? st[s].eps : 1e-10f;
    if (flags & COARSE_INV) {
#pragma unroll
      for (int k = 0; k < WMAX; ++k) {
        const int idx = threadIdx.x + COARSE_THREADS * k;
        if (idx < cnt) {
          float2& v = S[(idx / m0) * ls + idx % m0];
          v = cscale(v, mode == WAV_MUL_W ? wv[k] : 1.0f / (abar + lam * wv[k]));
        }
      }
    }
    for (int idx = threadIdx.x; idx < cnt && !(flags & COARSE_INV); idx += blockDim.x) {
      const int rr = idx / m0, cc = idx % m0;
      const size_t p = (size_t)rr * n + cc;
      float2& v = S[rr * ls + cc];
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
    __syncthreads();
  }
  if (!(flags & COARSE_INV)) return;
  for (int lev = nlev - 1; lev >= 0; --lev) smem_inv_level(S, ls, m0 >> lev, kind);
  float2* dp = dst + (size_t)s * dst_ss;
  const float2* rs = r ? r + (size_t)s * nn : nullptr;
  float acc = 0.f;
  for (int idx = threadIdx.x; idx < cnt; idx += blockDim.x) {
    const int rr = idx / m0, cc = idx % m0;
    float2 v = S[rr * ls + cc];
    if (real) v.y = 0.f;
    dp[(size_t)rr * dst_ld + cc] = v;
    if (rs) acc += rdot2(rs[(size_t)rr * n + cc], v);
  }
  if (part) {
    const double tot = block_sum((double)acc, red);
    if (threadIdx.x == 0) part[((size_t)s * NSLOT + SLOT_RZ) * MAXPART] = tot;
  }
}

// ---- every level of one slice on a thread-block cluster ----
// u = Phi^T (s o Phi x) in one launch: the C CTAs of a cluster own R = n/C
// consecutive rows of the slice each, so the whole slice lives in their
// shared memory and only x, the weights and u cross HBM.  All levels run in
// place.  Level l (side m = n >> (l-1), R_l = R >> (l-1) rows per CTA) keeps
// its row r at local row r << (l-1); the row step stores each row as
// [lowpass | highpass], the column step stores output pair k as rows 2k
// (lowpass) and 2k+1 (highpass), so the next level's block is the even rows'
// left halves, and every local position ends holding exactly one
// coefficient.  The column step scales each coefficient by its weight as
// soon as it is final, so no separate pass touches them.
// The Daubechies-4 column step of the last pair needs the next CTA's first
// two rows, the inverse column step of the first pair the previous CTA's last
// pair.  Each exchange e (forward level l: e = l - 1; inverse level l:
// e = 2L - l) has its own halo buffer and mbarrier in the receiving CTA: the
// sender writes the rows there with st.async, which counts the bytes on that
// mbarrier, and the receiver waits for them (bounded).  No buffer is written
// twice in a launch, so one cluster barrier at the start (every mbarrier
// armed before any remote write) is the only cluster-wide synchronisation;
// only the thread range whose pair reads a halo waits for it, just before
// that pair, so the exchange overlaps the rest of the column step.
constexpr int WCL_THREADS = 256;      // threads per CTA of the generic shape
constexpr int WCL_THREADS_256 = 512;  // and of the 256^2 four-level shape (a column's pairs split over 2-4 threads)
constexpr int WCL_NMAX = 256;
constexpr int WCL_LANE_PAIRS = WCL_NMAX / 64;  // pairs per lane of a row
constexpr int WCL_LMAX = 5;
constexpr int WCL_RMAX = 32;  // rows per CTA: two CTAs per SM fit with the weights mirrored

FI unsigned wcl_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
FI unsigned wcl_smem(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
// 16 bytes to the same shared-memory offset in CTA `rank`, counted on that
// CTA's mbarrier at the offset of `bar`
FI void wcl_st_async16(const void* dst, const uint64_t* bar, unsigned rank, float4 v) {
  unsigned ra, rb;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(wcl_smem(dst)), "r"(rank));
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(rb) : "r"(wcl_smem(bar)), "r"(rank));
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(
                   ra),
               "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "r"(rb)
               : "memory");
}
// bounded wait (about a second) for the first phase of `bar`, with
// cluster-scope acquire of the remote writes it counted
FI bool wcl_wait(const uint64_t* bar) {
  for (int it = 0; it < 20000; ++it) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], 0, %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(wcl_smem(bar)), "r"(50000u)
        : "memory");
    if (ok) return true;
  }
  return false;
}
FI void wcl_cp16(void* sdst, const void* gsrc) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(wcl_smem(sdst)), "l"(gsrc) : "memory");
}

// level of exchange e, and the offset (float2) of its halo buffer
__host__ __device__ inline int wcl_ex_level(int L, int e) { return e < L ? e + 1 : 2 * L - e; }
__host__ __device__ inline int wcl_halo_off(int n, int L, int e) {
  int off = 0;
  for (int q = 0; q < e; ++q) off += 2 * (n >> (wcl_ex_level(L, q) - 1));
  return off;
}

// Mallat row (in the n x n coefficient array) of the coefficient held at
// local row rho, column j of CTA `rank` after all L analysis levels.
FI int wcl_coef_row(int rho, int j, int n, int L, int R, int rank) {
  for (int l = 1; l <= L; ++l) {
    const int m = n >> (l - 1), r = rho >> (l - 1);
    const int k = rank * ((R >> (l - 1)) / 2) + (r >> 1);  // global pair index at level l
    if (r & 1) return m / 2 + k;                            // highpass row
    if (j >= m / 2 || l == L) return k;                     // lowpass row, final
  }
  return 0;  // not reached for L >= 1
}

struct WclScale {  // per-coefficient factor: w (MUL_W) or 1/(abar + lam w)
  const float* Wm;  // mirrored weights, or null: read from ws
  const float* ws;
  int n, L, R, rank, mode;
  float lam, abar;
  FI float2 apply(float2 v, int rho, int j) const {
    const float wv = Wm ? Wm[rho * n + j] : __ldg(ws + (size_t)wcl_coef_row(rho, j, n, L, R, rank) * n + j);
    return cscale(v, mode == WAV_MUL_W ? wv : 1.0f / (abar + lam * wv));
  }
};

// one level-l row step over the R_l rows (a warp per row); the inverse of
// level 1 (out != null) writes the samples straight to `out` (row stride n)
// with the optional real projection and partial Re<r, out>
FI float wcl_rows(float2* D, int n, int sr, int Rl, int m, int kind, bool inverse, int nth, float2* out = nullptr,
                  const float2* rr_ = nullptr, int real = 0) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, half = m / 2;
  float acc = 0.f;
  for (int rr = wid; rr < Rl; rr += nth / 32) {
    float2* L = D + rr * sr * n;
    float2 o0[WCL_LANE_PAIRS], o1[WCL_LANE_PAIRS];
#pragma unroll
    for (int u = 0; u < WCL_LANE_PAIRS; ++u) {
      const int k = lane + 32 * u;
      if (k >= half) continue;
      if (!inverse) {
        const float4 p0 = reinterpret_cast<const float4*>(L)[k];
        if (kind == 2) {
          const float4 p1 = reinterpret_cast<const float4*>(L)[k + 1 < half ? k + 1 : 0];
          lift::fwd_db4(make_float2(p0.x, p0.y), make_float2(p0.z, p0.w), make_float2(p1.x, p1.y),
                        make_float2(p1.z, p1.w), o0[u], o1[u]);
        } else {
          lift::fwd_haar(make_float2(p0.x, p0.y), make_float2(p0.z, p0.w), o0[u], o1[u]);
        }
      } else if (kind == 2) {
        const int km = k ? k - 1 : half - 1;
        lift::inv_db4(L[km], L[half + km], L[k], L[half + k], o0[u], o1[u]);
      } else {
        lift::inv_haar(L[k], L[half + k], o0[u], o1[u]);
      }
    }
    if (out) {
#pragma unroll
      for (int u = 0; u < WCL_LANE_PAIRS; ++u) {
        const int k = lane + 32 * u;
        if (k >= half) continue;
        float4 v = make_float4(o0[u].x, o0[u].y, o1[u].x, o1[u].y);
        if (real) v.y = v.w = 0.f;
        reinterpret_cast<float4*>(out + (size_t)rr * n)[k] = v;
        if (rr_) {
          const float4 q = reinterpret_cast<const float4*>(rr_ + (size_t)rr * n)[k];
          acc += q.x * v.x + q.y * v.y + q.z * v.z + q.w * v.w;
        }
      }
      continue;
    }
    __syncwarp();
#pragma unroll
    for (int u = 0; u < WCL_LANE_PAIRS; ++u) {
      const int k = lane + 32 * u;
      if (k >= half) continue;
      if (!inverse) {
        L[k] = o0[u];
        L[half + k] = o1[u];
      } else {
        reinterpret_cast<float4*>(L)[k] = make_float4(o0[u].x, o0[u].y, o1[u].x, o1[u].y);
      }
    }
    __syncwarp();
  }
  return acc;
}

// Pairs [k0, k1) of one column of a level-l column step, streaming down the
// column in place, two pairs per step with every load before the first
// store.  Forward: rows 2 k1 and 2 k1 + 1 (the next part's first rows, or the
// halo) are (e0, e1); the step scales the coefficients that are final after
// this level (highpass rows; lowpass rows right of m/2 or at the last
// level).  Inverse: (e0, e1) is pair k0 - 1 as it was before its update.
FI void wcl_col_pairs(float2* Dc, int rs, int sr, int j, int k0, int k1, float2 e0, float2 e1, int kind,
                      bool inverse, bool lo_final, const WclScale& sc) {
  if (kind != 2) {
    for (int kk = k0; kk < k1; ++kk) {
      float2 o0, o1;
      if (!inverse) {
        lift::fwd_haar(Dc[2 * kk * rs], Dc[(2 * kk + 1) * rs], o0, o1);
        if (lo_final) o0 = sc.apply(o0, 2 * kk * sr, j);
        o1 = sc.apply(o1, (2 * kk + 1) * sr, j);
      } else {
        lift::inv_haar(Dc[2 * kk * rs], Dc[(2 * kk + 1) * rs], o0, o1);
      }
      Dc[2 * kk * rs] = o0;
      Dc[(2 * kk + 1) * rs] = o1;
    }
  } else if (!inverse) {
    float2 r0 = Dc[2 * k0 * rs], r1 = Dc[(2 * k0 + 1) * rs];
    int kk = k0;
    for (; kk + 1 < k1; kk += 2) {
      const bool last = kk + 2 >= k1;
      const float2 r2 = Dc[(2 * kk + 2) * rs], r3 = Dc[(2 * kk + 3) * rs];
      const float2 r4 = last ? e0 : Dc[(2 * kk + 4) * rs];
      const float2 r5 = last ? e1 : Dc[(2 * kk + 5) * rs];
      float2 a0, d0, a1, d1;
      lift::fwd_db4(r0, r1, r2, r3, a0, d0);
      lift::fwd_db4(r2, r3, r4, r5, a1, d1);
      if (lo_final) {
        a0 = sc.apply(a0, 2 * kk * sr, j);
        a1 = sc.apply(a1, (2 * kk + 2) * sr, j);
      }
      Dc[2 * kk * rs] = a0;
      Dc[(2 * kk + 1) * rs] = sc.apply(d0, (2 * kk + 1) * sr, j);
      Dc[(2 * kk + 2) * rs] = a1;
      Dc[(2 * kk + 3) * rs] = sc.apply(d1, (2 * kk + 3) * sr, j);
      r0 = r4;
      r1 = r5;
    }
    if (kk < k1) {  // the last pair alone: its rows 2k+2, 2k+3 are (e0, e1)
      float2 a, d;
      lift::fwd_db4(r0, r1, e0, e1, a, d);
      if (lo_final) a = sc.apply(a, 2 * kk * sr, j);
      Dc[2 * kk * rs] = a;
      Dc[(2 * kk + 1) * rs] = sc.apply(d, (2 * kk + 1) * sr, j);
    }
  } else {
    float2 am = e0, dm = e1;
    int kk = k0;
    for (; kk + 1 < k1; kk += 2) {
      const float2 al = Dc[2 * kk * rs], dl = Dc[(2 * kk + 1) * rs];
      const float2 bl = Dc[(2 * kk + 2) * rs], el = Dc[(2 * kk + 3) * rs];
      float2 x0, x1, y0, y1;
      lift::inv_db4(am, dm, al, dl, x0, x1);
      lift::inv_db4(al, dl, bl, el, y0, y1);
      Dc[2 * kk * rs] = x0;
      Dc[(2 * kk + 1) * rs] = x1;
      Dc[(2 * kk + 2) * rs] = y0;
      Dc[(2 * kk + 3) * rs] = y1;
      am = bl;
      dm = el;
    }
    if (kk < k1) {
      const float2 al = Dc[2 * kk * rs], dl = Dc[(2 * kk + 1) * rs];
      float2 x0, x1;
      lift::inv_db4(am, dm, al, dl, x0, x1);
      Dc[2 * kk * rs] = x0;
      Dc[(2 * kk + 1) * rs] = x1;
    }
  }
}

// Pairs [k0, k1) of one column when the range touches the halo (forward:
// its last pair reads the next CTA's rows 0, 1; inverse: its first pair reads
// the previous CTA's last pair).  Every other pair is done first; the halo is
// waited for only before the pair that reads it, so the exchange overlaps the
// column work.  The inverse order is in-place safe: pairs k0+1.. need pair
// k0 as it was, and pair k0 is updated last.
FI void wcl_col_edge(float2* Dc, const float2* H, const uint64_t* bar, bool& ok, int rs, int sr, int j, int m,
                     int k0, int k1, int kind, bool inverse, bool lo_final, const WclScale& sc) {
  if (!inverse) {
    if (k1 - k0 >= 2)
      wcl_col_pairs(Dc, rs, sr, j, k0, k1 - 1, Dc[2 * (k1 - 1) * rs], Dc[(2 * (k1 - 1) + 1) * rs], kind, false,
                    lo_final, sc);
    ok = wcl_wait(bar) && ok;
    wcl_col_pairs(Dc, rs, sr, j, k1 - 1, k1, H[j], H[m + j], kind, false, lo_final, sc);
  } else {
    if (k1 - k0 >= 2)
      wcl_col_pairs(Dc, rs, sr, j, k0 + 1, k1, Dc[2 * k0 * rs], Dc[(2 * k0 + 1) * rs], kind, true, lo_final, sc);
    ok = wcl_wait(bar) && ok;
    wcl_col_pairs(Dc, rs, sr, j, k0, k0 + 1, H[j], H[m + j], kind, true, lo_final, sc);
  }
}

// One level-l column step over the m columns and R_l rows; H holds the halo
// rows (forward: the next CTA's rows 0, 1; inverse: the previous CTA's last
// pair), counted on `bar` (Daubechies-4 only; null for Haar).  With at least
// 2m threads the pairs of a column are split into `parts` ranges, one thread
// each: every part first reads the rows its neighbouring part will overwrite
// (forward: the next part's first two rows; inverse: the previous part's
// last pair), the CTA synchronises, then all parts stream in place.
FI void wcl_cols(float2* D, const float2* H, const uint64_t* bar, bool& ok, int n, int sr, int Rl, int m, int kind,
                 bool inverse, bool last_level, const WclScale& sc, int nth) {
  const int rs = sr * n, npair = Rl / 2;
  const bool halo = kind == 2;
  int parts = 1;
  while (parts * 2 * m <= nth && npair % (parts * 2) == 0) parts *= 2;  // equal ranges only
  if (parts == 1) {
    for (int j = threadIdx.x; j < m; j += nth) {
      const bool lo_final = last_level || j >= m / 2;
      if (halo)
        wcl_col_edge(D + j, H, bar, ok, rs, sr, j, m, 0, npair, kind, inverse, lo_final, sc);
      else
        wcl_col_pairs(D + j, rs, sr, j, 0, npair, H[j], H[m + j], kind, inverse, lo_final, sc);
    }
    return;
  }
  const int per = npair / parts, tid = threadIdx.x, j = tid % m, p = tid / m, k0 = p * per;
  const bool act = tid < m * parts;
  const bool edge = halo && (inverse ? p == 0 : p + 1 == parts);
  float2* Dc = D + j;
  float2 e0 = make_float2(0.f, 0.f), e1 = e0;
  if (act && !edge) {
    if (!inverse) {
      const bool last = p + 1 == parts;  // Haar: no row beyond the range is read
      e0 = last ? e0 : Dc[2 * (k0 + per) * rs];
      e1 = last ? e1 : Dc[(2 * (k0 + per) + 1) * rs];
    } else if (p > 0) {
      e0 = Dc[(2 * k0 - 2) * rs];
      e1 = Dc[(2 * k0 - 1) * rs];
    }
  }
  __syncthreads();
  if (!act) return;
  const bool lo_final = last_level || j >= m / 2;
  if (edge)
    wcl_col_edge(Dc, H, bar, ok, rs, sr, j, m, k0, k0 + per, kind, inverse, lo_final, sc);
  else
    wcl_col_pairs(Dc, rs, sr, j, k0, k0 + per, e0, e1, kind, inverse, lo_final, sc);
}

// rows row0, row1 (local) of width m to halo buffer Hb of CTA `to`
// (buffer rows of width m), counted on its mbarrier `bar`
FI void wcl_push(const float2* D, const float2* Hb, const uint64_t* bar, int n, int row0, int row1, int m,
                 unsigned to, int nth) {
  const int q4 = m / 2;  // float4 per row
  for (int q = threadIdx.x; q < 2 * q4; q += nth) {
    const int h = q / q4, jj = 2 * (q % q4);
    const float4 v = *reinterpret_cast<const float4*>(D + (h ? row1 : row0) * n + jj);
    wcl_st_async16(Hb + h * m + jj, bar, to, v);
  }
}

// NT, RT, LT, KT: side, rows per CTA, levels and wavelet kind fixed at
// compile time (0: taken from the arguments and the grid), so that the
// common shape runs with constant loop bounds, strides and offsets.
template <int NT, int RT, int LT, int KT, int TH>
__global__ void __launch_bounds__(TH, 2)
k_wav_cluster(const float2* x, float2* u, const float* __restrict__ w, int n_arg, int L_arg, int kind_arg,
              int mode, int mirror, const float2* __restrict__ r, double* __restrict__ part, int real,
              SliceState* __restrict__ st) {
  const int s = blockIdx.y;
  // the same slice for every CTA of the cluster: all of them leave or none
  if (st != nullptr && !slice_running(st, s)) return;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[32];
  const int n = NT ? NT : n_arg, L = LT ? LT : L_arg, kind = KT ? KT : kind_arg;
  const unsigned rank = wcl_rank();
  const unsigned C = RT ? (unsigned)(n / RT) : gridDim.x;
  const int R = RT ? RT : n / (int)C, tid = threadIdx.x;
  float2* D = reinterpret_cast<float2*>(smem);        // [R][n]
  float2* H = D + R * n;                              // halo buffers of the 2L exchanges
  uint64_t* mb = reinterpret_cast<uint64_t*>(H + wcl_halo_off(n, L, 2 * L));  // their mbarriers
  float* Wm = reinterpret_cast<float*>(mb + 2 * L);   // [R][n] weights (mirror)
  const size_t nn = (size_t)n * n;
  const float* ws = w + (size_t)s * nn;
  {
    const float2* xs = x + (size_t)s * nn + (size_t)rank * R * n;
    for (int q = tid; q < R * n / 2; q += TH) wcl_cp16(D + 2 * q, xs + 2 * q);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    if (mirror) {  // the weight of the coefficient each position will hold
      for (int q = tid; q < R * n / 4; q += TH) {
        const int rho = 4 * q / n, j = 4 * q % n;
        wcl_cp16(Wm + 4 * q, ws + (size_t)wcl_coef_row(rho, j, n, L, R, rank) * n + j);
      }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  }
  if (kind == 2 && tid == 0) {  // arm every exchange: two halo rows of its level
    for (int e = 0; e < 2 * L; ++e) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(wcl_smem(mb + e)) : "memory");
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    for (int e = 0; e < 2 * L; ++e) {
      const unsigned bytes = 2u * (unsigned)(n >> (wcl_ex_level(L, e) - 1)) * 8u;
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(wcl_smem(mb + e)), "r"(bytes)
                   : "memory");
    }
  }
  asm volatile("cp.async.wait_group 1;\n" ::: "memory");
  __syncthreads();
  if (kind == 2)  // every CTA's mbarriers armed before any remote write
    asm volatile("barrier.cluster.arrive.release.aligned;\n barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
  WclScale sc;
  sc.Wm = mirror ? Wm : nullptr;
  sc.ws = ws;
  sc.n = n;
  sc.L = L;
  sc.R = R;
  sc.rank = (int)rank;
  sc.mode = mode;
  sc.lam = st ? st[s].lam : 0.f;
  sc.abar = st ? st[s].abar : 0.f;
  bool ok = true;
#pragma unroll
  for (int l = 1; l <= (LT ? LT : WCL_LMAX); ++l) {
    if (l > L) break;
    const int m = n >> (l - 1), Rl = R >> (l - 1), sr = 1 << (l - 1), e = l - 1;
    wcl_rows(D, n, sr, Rl, m, kind, false, TH);
    __syncthreads();
    const float2* He = H + wcl_halo_off(n, L, e);
    if (kind == 2) {
      wcl_push(D, He, mb + e, n, 0, sr, m, (rank + C - 1) % C, TH);
    }
    if (l == 1) {
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");
      __syncthreads();
    }
    wcl_cols(D, He, mb + e, ok, n, sr, Rl, m, kind, false, l == L, sc, TH);
    __syncthreads();
  }
  float acc = 0.f;
#pragma unroll
  for (int lr = 0; lr < (LT ? LT : WCL_LMAX); ++lr) {
    const int l = L - lr;
    if (l < 1) break;
    const int m = n >> (l - 1), Rl = R >> (l - 1), sr = 1 << (l - 1), e = 2 * L - l;
    const float2* He = H + wcl_halo_off(n, L, e);
    if (kind == 2) {
      wcl_push(D, He, mb + e, n, (Rl - 2) * sr, (Rl - 1) * sr, m, (rank + 1) % C, TH);
      // the last remote write of this CTA is issued: arrive on the cluster
      // barrier that every CTA waits on before it exits
      if (l == 1) asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
    }
    wcl_cols(D, He, mb + e, ok, n, sr, Rl, m, kind, true, false, sc, TH);
    __syncthreads();
    if (l > 1) {
      wcl_rows(D, n, sr, Rl, m, kind, true, TH);
      __syncthreads();
    } else {  // the last row step writes u
      const size_t off = (size_t)s * nn + (size_t)rank * R * n;
      acc = wcl_rows(D, n, 1, R, n, kind, true, TH, u + off, r ? r + off : nullptr, real);
    }
  }
  if (!ok && st) st[s].fault = 1;  // a halo never arrived: results invalid
  if (part) {
    const double tot = block_sum((double)acc, red);
    if (tid == 0) part[((size_t)s * NSLOT + SLOT_RZ) * MAXPART + rank] = tot;
  }
  // no CTA leaves (releasing its shared memory) while a peer of the cluster
  // may still issue a write into it, even after a halo wait ran out; every
  // CTA reaches this point, so the wait ends
  if (kind == 2) asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

static int wcl_smem_bytes(int n, int R, int L, bool mirror) {
  return R * n * 8 + wcl_halo_off(n, L, 2 * L) * 8 + 2 * L * 8 + (mirror ? R * n * 4 : 0);
}

// Rows per CTA of the one-launch form (0 when it does not apply): the
// fewest rows (most CTAs, at most 8 per cluster) for which every level has an
// even number of rows per CTA.  choice: 0 default, 1 weights mirrored in
// shared memory, 2 read from HBM; *mirror receives which.
static int wcl_rows_per_cta(int n, int L, int kind, int choice, bool* mirror) {
  if (kind != 1 && kind != 2) return 0;
  if (choice != 0 && choice != 1 && choice != 2) return 0;
  if (n % 8 || n > WCL_NMAX || L < 1 || L > WCL_LMAX || (n >> L) % 4) return 0;
  for (int C = 8; C >= 1; --C) {
    if (n % (C << L) || n / C > WCL_RMAX) continue;
    if (mirror) *mirror = choice != 2;
    return n / C;
  }
  return 0;
}

static void wcl_launch(const WavArgs& a, int R, bool mirror, const float2* x, const float* w, int mode, float2* u,
                       const float2* r, int real) {
  const int C = a.n / R;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C, a.batch);
  cfg.blockDim = dim3(WCL_THREADS);
  cfg.dynamicSmemBytes = wcl_smem_bytes(a.n, R, a.levels, mirror);
  cfg.stream = a.stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  SliceState* st = const_cast<SliceState*>(a.st);
  double* pp = r ? a.part : nullptr;
  const int mi = mirror ? 1 : 0;
  if (a.n == 256 && R == 32 && a.levels == 4 && a.kind == 2) {  // the 256^2 four-level Daubechies-4 shape
    cfg.blockDim = dim3(WCL_THREADS_256);
    cudaLaunchKernelEx(&cfg, k_wav_cluster<256, 32, 4, 2, WCL_THREADS_256>, x, u, w, a.n, a.levels, a.kind, mode, mi, r,
                       pp, real, st);
  } else {
    cudaLaunchKernelEx(&cfg, k_wav_cluster<0, 0, 0, 0, WCL_THREADS>, x, u, w, a.n, a.levels, a.kind, mode, mi, r, pp,
                       real, st);
  }
}

static int coarse_smem(int m0) { return m0 * (m0 + 1) * 8; }

bool ilu_prepare();
bool wavelet_diag_prepare();

// Dynamic shared-memory limits of the wavelet, ILU and pseudo-diagonal
// kernels, set once per device.
static void set_wav_attrs() {
  static PerDeviceOnce once;
  once.run([] {
    const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
    bool ok = cudaFuncSetAttribute(k_wav_fwd, A, (2 * 16 + 2) * 512 * 8) == cudaSuccess;
    ok = cudaFuncSetAttribute(k_wav_inv, A, 2 * 16 * 512 * 8) == cudaSuccess && ok;
    ok = cudaFuncSetAttribute(k_wav_coarse, A, coarse_smem(COARSE_LIMIT)) == cudaSuccess && ok;
    ok = cudaFuncSetAttribute(k_wav_cluster<0, 0, 0, 0, WCL_THREADS>, A,
                              wcl_smem_bytes(WCL_NMAX, WCL_RMAX, WCL_LMAX, true)) == cudaSuccess && ok;
    ok = cudaFuncSetAttribute(k_wav_cluster<256, 32, 4, 2, WCL_THREADS_256>, A, wcl_smem_bytes(256, 32, 4, true)) ==
             cudaSuccess && ok;
    ok = ilu_prepare() && ok;
    ok = wavelet_diag_prepare() && ok;
    return ok;
  });
}

void wav_prepare() { set_wav_attrs(); }

// First level handled by the coarse kernel: its input side m <= cmax.
static int coarse_first_level(int n, int levels, int cmax = 0) {
  const int lim = cmax > 0 ? (cmax < COARSE_LIMIT ? cmax : COARSE_LIMIT) : COARSE_MAX;
  int l0 = 1;
  while (l0 <= levels && (n >> (l0 - 1)) > lim) ++l0;
  return l0;  // levels + 1 when no level fits
}

// Tiled analysis of levels 1 .. lend; returns the buffer holding LL_lend.
static const float2* tiled_forward(const WavArgs& a, const float2* x, float2* c, float* w, int mode, int lend,
                                   bool ll_final_to_c, size_t* ss, int* ld) {
  const int n = a.n;
  const size_t hh = (size_t)(n / 2) * (n / 2);
  const float2* src = x;
  size_t src_ss = (size_t)n * n;
  int src_ld = n;
  for (int l = 1; l <= lend; ++l) {
    const int m = n >> (l - 1), half = m / 2;
    const bool to_c = ll_final_to_c && l == lend;
    float2* dst = to_c ? c : ((l & 1) ? a.tmpA : a.tmpB);
    const size_t dst_ss = to_c ? (size_t)n * n : hh;
    const int dst_ld = to_c ? n : half;
    const int rb = wav_rb(m, a.rb);
    const int smem = (2 * rb + (a.kind == 2 ? 2 : 0)) * m * 8;
    k_wav_fwd<<<dim3((half + rb - 1) / rb, a.batch), WAV_THREADS, smem, a.stream>>>(
        src, src_ss, src_ld, dst, dst_ss, dst_ld, c, w, n, m, rb, a.kind, mode, to_c ? 1 : 0, a.st);
    src = dst;
    src_ss = dst_ss;
    src_ld = dst_ld;
  }
  *ss = src_ss;
  *ld = src_ld;
  return src;
}

// Tiled synthesis of levels lstart .. 1 with LL_lstart in (lli, ll_ss, ll_ld).
static void tiled_inverse(const WavArgs& a, const float2* lli, size_t ll_ss, int ll_ld, const float2* c,
                          float2* x, int lstart, const float2* r, int real) {
  const int n = a.n;
  const size_t hh = (size_t)(n / 2) * (n / 2);
  for (int l = lstart; l >= 1; --l) {
    const int m = n >> (l - 1), half = m / 2;
    const bool final_level = (l == 1);
    // write into the ping-pong buffer the input does not occupy
    float2* out = final_level ? x : (lli == a.tmpA ? a.tmpB : a.tmpA);
    const size_t out_ss = final_level ? (size_t)n * n : hh;
    const int out_ld = final_level ? n : m;
    const int rb = wav_rb(m, a.rb);
    k_wav_inv<<<dim3((half + rb - 1) / rb, a.batch), WAV_THREADS, 2 * rb * m * 8, a.stream>>>(
        lli, ll_ss, ll_ld, c, out, out_ss, out_ld, n, m, rb, a.kind, final_level ? r : nullptr,
        final_level && r ? a.part : nullptr, real, a.st);
    lli = out;
    ll_ss = out_ss;
    ll_ld = out_ld;
  }
}

void wavelet_forward(const WavArgs& a, const float2* x, float2* c, float* w, int mode) {
  set_wav_attrs();
  const int n = a.n, L = a.levels;
  const int l0 = coarse_first_level(n, L, a.coarse_max);
  size_t ss;
  int ld;
  const float2* ll = tiled_forward(a, x, c, w, mode, l0 - 1, l0 > L, &ss, &ld);
  if (l0 <= L) {
    const int m0 = n >> (l0 - 1);
    k_wav_coarse<<<a.batch, COARSE_THREADS, coarse_smem(m0), a.stream>>>(
        ll, ss, ld, nullptr, 0, 0, c, w, n, m0, L - l0 + 1, a.kind, mode, COARSE_FWD, nullptr, nullptr, 0, a.st);
  }
}

void wavelet_inverse(const WavArgs& a, const float2* c, float2* x, const float2* r, int real) {
  set_wav_attrs();
  const int n = a.n, L = a.levels;
  const int l0 = coarse_first_level(n, L, a.coarse_max);
  if (l0 <= L) {
    const int m0 = n >> (l0 - 1);
    const bool final_coarse = (l0 == 1);
    float2* dst = final_coarse ? x : ((l0 - 1) & 1 ? a.tmpA : a.tmpB);
    const size_t dss = final_coarse ? (size_t)n * n : (size_t)(n / 2) * (n / 2);
    const int dld = final_coarse ? n : m0;
    k_wav_coarse<<<a.batch, COARSE_THREADS, coarse_smem(m0), a.stream>>>(
        nullptr, 0, 0, dst, dss, dld, const_cast<float2*>(c), nullptr, n, m0, L - l0 + 1, a.kind, WAV_RAW,
        COARSE_INV, final_coarse ? r : nullptr, final_coarse && r ? a.part : nullptr, real, a.st);
    if (!final_coarse) tiled_inverse(a, dst, dss, dld, c, x, l0 - 1, r, real);
  } else {
    tiled_inverse(a, c, (size_t)n * n, n, c, x, L, r, real);
  }
}

// u = Phi^T (s o Phi x) with s = w (MUL_W) or 1/(abar + lam w) (MUL_PINV).
void wavelet_apply(const WavArgs& a, const float2* x, float2* c, float* w, int mode, float2* u,
                   const float2* r, int real) {
  set_wav_attrs();
  const int n = a.n, L = a.levels;
  bool mirror = false;
  const int R = wcl_rows_per_cta(n, L, a.kind, a.rb, &mirror);
  if (R > 0) {  // every level on chip, c untouched
    wcl_launch(a, R, mirror, x, w, mode, u, r, real);
    return;
  }
  const int l0 = coarse_first_level(n, L, a.coarse_max);
  if (l0 > L) {
    wavelet_forward(a, x, c, w, mode);
    wavelet_inverse(a, c, u, r, real);
    return;
  }
  size_t ss;
  int ld;
  const float2* ll = tiled_forward(a, x, c, w, mode, l0 - 1, false, &ss, &ld);
  const int m0 = n >> (l0 - 1);
  const bool final_coarse = (l0 == 1);
  float2* dst = final_coarse ? u : const_cast<float2*>(ll);  // LL' overwrites LL in place
  const size_t dss = final_coarse ? (size_t)n * n : ss;
  const int dld = final_coarse ? n : ld;
  k_wav_coarse<<<a.batch, COARSE_THREADS, coarse_smem(m0), a.stream>>>(
      ll, ss, ld, dst, dss, dld, c, w, n, m0, L - l0 + 1, a.kind, mode, COARSE_FWD | COARSE_INV,
      final_coarse ? r : nullptr, final_coarse && r ? a.part : nullptr, real, a.st);
  if (!final_coarse) tiled_inverse(a, dst, dss, dld, c, u, l0 - 1, r, real);
}

// CTAs per slice of the one-launch cluster form of wavelet_apply (0: tiled).
int wavelet_cluster_ctas(int n, int levels, int kind, int rb) {
  const int R = wcl_rows_per_cta(n, levels, kind, rb, nullptr);
  return R ? n / R : 0;
}

// Partial-sum count of the wavelet_apply stage that computes Re<r, Phi^T ...>.
int wavelet_apply_ctas(int n, int levels, int kind, int rb, int cmax) {
  const int C = wavelet_cluster_ctas(n, levels, kind, rb);
  if (C > 0) return C;
  if (coarse_first_level(n, levels, cmax) == 1) return 1;
  return (n / 2 + wav_rb(n, rb) - 1) / wav_rb(n, rb);
}

// Launches per wavelet_apply call (for the launch count).
int wavelet_apply_launches(int n, int levels, int kind, int rb, int cmax) {
  if (wavelet_cluster_ctas(n, levels, kind, rb) > 0) return 1;
  const int l0 = coarse_first_level(n, levels, cmax);
  if (l0 > levels) return 2 * levels;
  return 2 * (l0 - 1) + 1;
}

// ================================================================== TV =====

// Isotropic TV (wtv2 null): W_i = (|grad_1 x_i|^2 + |grad_2 x_i|^2 + eps)^(-1/2)
// (Eq. wi).  l1 TV (Eq. l1): W1_i = (|grad_1 x_i|^2 + eps)^(-1/2) into wtv and
// W2_i = (|grad_2 x_i|^2 + eps)^(-1/2) into wtv2.  Zero extension.  Joint TV
// (Sec. 5.6, C > 1 contrasts in consecutive slices, isotropic only): the
// squared gradients of all contrasts of the image are summed under the root,
// and every contrast gets the same W.
__global__ void k_tv_weights(int n, int C, const SliceState* __restrict__ st, const float2* __restrict__ x,
                             float* __restrict__ wtv, float* __restrict__ wtv2) {
  const int s = blockIdx.y;
  if (!slice_running(st, s)) return;
  const float eps = st[s].eps;
  const size_t base = (size_t)s * n * n;
  const size_t img = (size_t)(s - s % C) * n * n;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n * n; i += gridDim.x * blockDim.x) {
    const int r = i / n, c = i % n;
    if (C > 1) {
      float g = 0.f;
      for (int t = 0; t < C; ++t) {
        const size_t bt = img + (size_t)t * n * n;
        const float2 xc = x[bt + i];
        const float2 g1 = c > 0 ? csub(xc, x[bt + i - 1]) : xc;
        const float2 g2 = r > 0 ? csub(xc, x[bt + i - n]) : xc;
        g += cabs2(g1) + cabs2(g2);
      }
      wtv[base + i] = rsqrtf(g + eps);
      continue;
    }
    const float2 xc = x[base + i];
    const float2 g1 = c > 0 ? csub(xc, x[base + i - 1]) : xc;
    const float2 g2 = r > 0 ? csub(xc, x[base + i - n]) : xc;
    if (wtv2) {
      wtv[base + i] = rsqrtf(cabs2(g1) + eps);
      wtv2[base + i] = rsqrtf(cabs2(g2) + eps);
    } else {
      wtv[base + i] = rsqrtf(cabs2(g1) + cabs2(g2) + eps);
    }
  }
}

void tv_weights(int batch, int n, cudaStream_t s, const SliceState* st, const float2* x, float* wtv, float* wtv2,
                int channels) {
  const int N = n * n;
  const int blocks = (N + 255) / 256 < 64 ? (N + 255) / 256 : 64;
  k_tv_weights<<<dim3(blocks, batch), 256, 0, s>>>(n, channels, st, x, wtv, wtv2);
}

// Joint wavelet sparsity (Sec. 5.6, FIRLS_MT): coefficient j of the C
// contrasts of an image forms one non-overlapping group, W_j = (sum_t
// |(Phi x_t)_j|^2 + eps)^(-1/2) (Eq. gw), written to every contrast.  cw holds
// the raw coefficients of all slices.
__global__ void k_joint_wavelet_weights(int N, int C, const SliceState* __restrict__ st,
                                        const float2* __restrict__ cw, float* __restrict__ ww) {
  const int s = blockIdx.y;
  if (!slice_running(st, s)) return;
  const float eps = st[s].eps;
  const size_t img = (size_t)(s - s % C) * N;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += gridDim.x * blockDim.x) {
    float g = 0.f;
    for (int t = 0; t < C; ++t) g += cabs2(cw[img + (size_t)t * N + j]);
    ww[(size_t)s * N + j] = rsqrtf(g + eps);
  }
}

void joint_wavelet_weights(int batch, int n, int channels, cudaStream_t s, const SliceState* st, const float2* cw,
                           float* ww) {
  const int N = n * n;
  const int blocks = (N + 255) / 256 < 64 ? (N + 255) / 256 : 64;
  k_joint_wavelet_weights<<<dim3(blocks, batch), 256, 0, s>>>(N, channels, st, cw, ww);
}

// Exact diag(Phi^T diag(w) Phi).  Each 2-D basis function of level l is an
// outer product of 1-D level-l functions f_{l,type}(i - 2^l p) (type 0 low,
// 1 high) whose squares are tabulated (sqtab[(l-1)*2 + type][0 .. sqlen)),
// so the diagonal is a separable sum over levels and subbands:
//   diag(r, c) = sum_l sum_br sum_pr F_{l,br}(r - 2^l pr) T_{l,br}(pr, c),
//   T_{l,br}(pr, c) = sum_{bands (br, bc)} sum_pc F_{l,bc}(c - 2^l pc) w_band(pr, pc),
// indices periodic.  A CTA owns WD_RB output rows: per level it forms the
// T rows those outputs need in shared memory (both row types), then adds
// their row-filtered sums.  Bands at level l (h = n >> l, Mallat layout):
// (0,1) rows [0,h) cols [h,2h); (1,0) rows [h,2h) cols [0,h); (1,1) rows and
// cols [h,2h); at the last level also (0,0), rows and cols [0,h).
constexpr int WD_RB = 16;
constexpr int WD_PRMAX = WD_RB / 2 + 4;  // coarse rows a level needs (filters of <= 3 * 2^l taps)

// NT, LT: side and levels fixed at compile time (0: from the arguments), so
// that the common shape's row and column index arithmetic is shifts and masks.
template <int NT, int LT>
__global__ void __launch_bounds__(256) k_wavelet_diag(int n_arg, int levels_arg, const SliceState* __restrict__ st,
                                                      const float* __restrict__ w, float* __restrict__ out,
                                                      const float* __restrict__ sqtab,
                                                      const int* __restrict__ sqlen) {
  const int s = blockIdx.y;
  if (!slice_running(st, s)) return;
  const int n = NT ? NT : n_arg, levels = LT ? LT : levels_arg;
  extern __shared__ __align__(16) float tsm[];  // [2][WD_PRMAX][n]
  const int r0 = blockIdx.x * WD_RB;
  const int rows = min(WD_RB, n - r0);
  const size_t base = (size_t)s * n * n;
  const float* ws = w + base;
  constexpr int PER = WD_RB * 512 / 256;  // outputs per thread, n <= 512
  float acc[PER];
#pragma unroll
  for (int k = 0; k < PER; ++k) acc[k] = 0.f;
#pragma unroll
  for (int l = 1; l <= levels; ++l) {  // a constant trip count (unrolled) for LT > 0
    const int h = n >> l, step = 1 << l, msk = step - 1;
    const int len[2] = {sqlen[(l - 1) * 2], sqlen[(l - 1) * 2 + 1]};
    const float* F[2] = {sqtab + (size_t)((l - 1) * 2) * n, sqtab + (size_t)((l - 1) * 2 + 1) * n};
    const int lmax = len[0] > len[1] ? len[0] : len[1];
    // coarse rows pr = pr_lo + j (mod h), j < cnt, cover every r - sr with sr < lmax
    const int pr_lo = (r0 - (lmax - 1) - (step - 1)) >> l;  // floor division (arithmetic shift)
    int cnt = ((r0 + rows - 1) >> l) - pr_lo + 1;
    if (cnt > WD_PRMAX) cnt = WD_PRMAX;
    const int pr0 = ((pr_lo % h) + h) % h;
    __syncthreads();  // the previous level's T rows are no longer read
    for (int idx = threadIdx.x; idx < 2 * cnt * n; idx += blockDim.x) {
      const int br = idx / (cnt * n), j = (idx / n) % cnt, c = idx % n;
      const int pr = (pr0 + j) % h;
      float t = 0.f;
      for (int bc = 0; bc < 2; ++bc) {
        if (br == 0 && bc == 0 && l != levels) continue;  // LL is a band only at the last level
        const float* wrow = ws + (size_t)(br * h + pr) * n + bc * h;
        const float* fc = F[bc];
        for (int sc = c & msk; sc < len[bc]; sc += step) {
          int pc = c - sc;
          if (pc < 0) pc += n;
          t = fmaf(fc[sc], wrow[pc >> l], t);
        }
      }
      tsm[(size_t)(br * WD_PRMAX + j) * n + c] = t;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int idx = threadIdx.x + 256 * k;
      if (idx < rows * n) {
        const int r = r0 + idx / n, c = idx % n;
        float a = acc[k];
        for (int br = 0; br < 2; ++br) {
          const float* fr = F[br];
          for (int sr = r & msk; sr < len[br]; sr += step) {
            int pr = r - sr;
            if (pr < 0) pr += n;
            const int j = (((pr >> l) - pr0) % h + h) % h;
            a = fmaf(fr[sr], tsm[(size_t)(br * WD_PRMAX + j) * n + c], a);
          }
        }
        acc[k] = a;
      }
    }
  }
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int idx = threadIdx.x + 256 * k;
    if (idx < rows * n) out[base + (size_t)(r0 + idx / n) * n + idx % n] = acc[k];
  }
}

bool wavelet_diag_prepare() {
  const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
  bool ok = cudaFuncSetAttribute(k_wavelet_diag<0, 0>, A, 2 * WD_PRMAX * 512 * 4) == cudaSuccess;
  return cudaFuncSetAttribute(k_wavelet_diag<256, 4>, A, 2 * WD_PRMAX * 256 * 4) == cudaSuccess && ok;
}

void wavelet_diag(int batch, int n, int levels, cudaStream_t s, const SliceState* st, const float* w,
                  float* out, const float* sqtab, const int* sqlen) {
  const dim3 grid((n + WD_RB - 1) / WD_RB, batch);
  if (n == 256 && levels == 4)
    k_wavelet_diag<256, 4><<<grid, 256, 2 * WD_PRMAX * n * 4, s>>>(n, levels, st, w, out, sqtab, sqlen);
  else
    k_wavelet_diag<0, 0><<<grid, 256, 2 * WD_PRMAX * n * 4, s>>>(n, levels, st, w, out, sqtab, sqlen);
}

// P = abar I + lam_tv (D1^T W1 D1 + D2^T W2 D2) [+ lam diag(Phi^T W Phi)]
// (Eq. ptv; W1 = W2 = W for isotropic TV, wtv2 null): ia = 1 / a_i, the
// inverse diagonal, a_i = abar + lam_tv (W1_i + W1_{i+1} + W2_i + W2_{i+n}).
// The off-diagonals (-lam_tv W1_{i+1}, -lam_tv W2_{i+n}) are formed from the
// weights inside the ILU sweeps.
__global__ void k_penta(int n, const SliceState* __restrict__ st, const float* __restrict__ wtv,
                        const float* __restrict__ wtv2, const float* __restrict__ wdiag, float* __restrict__ ia) {
  const int s = blockIdx.y;
  if (!slice_running(st, s)) return;
  const float abar = st[s].abar, lt = st[s].lam_tv, lw = st[s].lam;
  const size_t base = (size_t)s * n * n;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n * n; i += gridDim.x * blockDim.x) {
    const int r = i / n, c = i % n;
    const float wc = wtv[base + i];
    const float wr = c < n - 1 ? wtv[base + i + 1] : 0.f;
    float a;
    if (wtv2) {
      const float wd = r < n - 1 ? wtv2[base + i + n] : 0.f;
      a = abar + lt * (wc + wr + wtv2[base + i] + wd);
    } else {
      const float wd = r < n - 1 ? wtv[base + i + n] : 0.f;
      a = abar + lt * (2.f * wc + wr + wd);
    }
    if (wdiag) a = fmaf(lw, wdiag[base + i], a);
    ia[base + i] = 1.0f / a;
  }
}

void penta_setup(int batch, int n, cudaStream_t s, const SliceState* st, const float* wtv, const float* wtv2,
                 const float* wdiag, float* ia) {
  const int N = n * n;
  const int blocks = (N + 255) / 256 < 64 ? (N + 255) / 256 : 64;
  k_penta<<<dim3(blocks, batch), 256, 0, s>>>(n, st, wtv, wtv2, wdiag, ia);
}

// ILU(0) pivots of the penta-diagonal P: d_i = a_i - (lam W1_i)^2 / d_{i-1}
// [col > 0] - (lam W2_i)^2 / d_{i-n} [row > 0] (the incomplete LU with zero
// fill of Sec. 4.2 with updated pivots; W1 = W2 = W for isotropic TV).
// In: ia = 1/a; out: ia = 1/d in place.  One warp per slice, a row at a time:
// with alpha_i = a_i - (lam W2_i)^2 / d_{i-n} the row recurrence
// d_i = alpha_i - (lam W1_i)^2 / d_{i-1} is a Moebius map of d_{i-1}, i.e.
// (p, q) -> M_i (p, q) with M_i = [[alpha_i, -(lam W1_i)^2], [1, 0]] and
// d = p / q, so the row is a scan of 2 x 2 matrix products: each lane folds
// its E columns, a warp shuffle scan combines the lanes (every product
// scaled by its largest entry: only the ratio p / q matters), and each lane
// then runs its own columns from the incoming ratio.
template <int E>
__global__ void __launch_bounds__(32) k_ilu0_pivots(int n, const SliceState* __restrict__ st,
                                                     const float* __restrict__ wtv, const float* __restrict__ wtv2,
                                                     float* __restrict__ ia) {
  const int s = blockIdx.x;
  if (!slice_running(st, s)) return;
  const int lane = threadIdx.x;
  const float lam = st[s].lam_tv;
  const float* w2 = wtv2 ? wtv2 : wtv;
  const size_t base = (size_t)s * n * n;
  float dprev[E];  // d of the row above in this lane's columns
#pragma unroll
  for (int e = 0; e < E; ++e) dprev[e] = 1.f;
  for (int r = 0; r < n; ++r) {
    const size_t rb = base + (size_t)r * n;
    float al[E], k2[E];
    // this lane's segment as a 2 x 2 matrix T = M_{last} ... M_{first}
    float t00 = 1.f, t01 = 0.f, t10 = 0.f, t11 = 1.f;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int c = lane * E + e;
      al[e] = 1.f;
      k2[e] = 0.f;
      if (c < n) {
        const float a = 1.0f / ia[rb + c];
        const float kv = r > 0 ? lam * w2[rb + c] : 0.f;
        const float kh = c > 0 ? lam * wtv[rb + c] : 0.f;
        al[e] = a - kv * kv / dprev[e];
        k2[e] = kh * kh;
      }
      // M_e * T
      const float n00 = al[e] * t00 - k2[e] * t10, n01 = al[e] * t01 - k2[e] * t11;
      t10 = t00;
      t11 = t01;
      t00 = n00;
      t01 = n01;
      const float m = fmaxf(fmaxf(fabsf(t00), fabsf(t01)), fmaxf(fabsf(t10), fabsf(t11)));
      if (m > 0.f) {
        const float im = 1.0f / m;
        t00 *= im;
        t01 *= im;
        t10 *= im;
        t11 *= im;
      }
    }
    // inclusive scan over the lanes: P_L = T_L ... T_0
    float p00 = t00, p01 = t01, p10 = t10, p11 = t11;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const float q00 = __shfl_up_sync(0xffffffffu, p00, off), q01 = __shfl_up_sync(0xffffffffu, p01, off);
      const float q10 = __shfl_up_sync(0xffffffffu, p10, off), q11 = __shfl_up_sync(0xffffffffu, p11, off);
      if (lane >= off) {  // P = P_mine * P_earlier
        const float n00 = p00 * q00 + p01 * q10, n01 = p00 * q01 + p01 * q11;
        const float n10 = p10 * q00 + p11 * q10, n11 = p10 * q01 + p11 * q11;
        const float m = fmaxf(fmaxf(fabsf(n00), fabsf(n01)), fmaxf(fabsf(n10), fabsf(n11)));
        const float im = m > 0.f ? 1.0f / m : 1.f;
        p00 = n00 * im;
        p01 = n01 * im;
        p10 = n10 * im;
        p11 = n11 * im;
      }
    }
    // the ratio entering this lane: the previous lane's prefix applied to
    // (1, 0) (no left neighbour for column 0)
    const float e00 = __shfl_up_sync(0xffffffffu, p00, 1), e10 = __shfl_up_sync(0xffffffffu, p10, 1);
    float d = lane == 0 ? 0.f : e00 / e10;  // lane 0: column 0 has k2 = 0, d_in unused
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int c = lane * E + e;
      if (c < n) {
        d = k2[e] > 0.f ? al[e] - k2[e] / d : al[e];
        dprev[e] = d;
        ia[rb + c] = 1.0f / d;
      }
    }
  }
}

void ilu0_pivots(int batch, int n, cudaStream_t s, const SliceState* st, const float* wtv, const float* wtv2,
                 float* ia) {
  const int E = (n + 31) / 32;
  switch (E) {
    case 1: k_ilu0_pivots<1><<<batch, 32, 0, s>>>(n, st, wtv, wtv2, ia); break;
    case 2: k_ilu0_pivots<2><<<batch, 32, 0, s>>>(n, st, wtv, wtv2, ia); break;
    case 3: k_ilu0_pivots<3><<<batch, 32, 0, s>>>(n, st, wtv, wtv2, ia); break;
    case 4: k_ilu0_pivots<4><<<batch, 32, 0, s>>>(n, st, wtv, wtv2, ia); break;
    case 5: k_ilu0_pivots<5><<<batch, 32, 0, s>>>(n, st, wtv, wtv2, ia); break;
    case 6: k_ilu0_pivots<6><<<batch, 32, 0, s>>>(n, st, wtv, wtv2, ia); break;
    case 8: k_ilu0_pivots<8><<<batch, 32, 0, s>>>(n, st, wtv, wtv2, ia); break;
    case 10: k_ilu0_pivots<10><<<batch, 32, 0, s>>>(n, st, wtv, wtv2, ia); break;
    case 12: k_ilu0_pivots<12><<<batch, 32, 0, s>>>(n, st, wtv, wtv2, ia); break;
    case 16: k_ilu0_pivots<16><<<batch, 32, 0, s>>>(n, st, wtv, wtv2, ia); break;
    default: break;
  }
}

// ------------------------------------------------ ILU solves (Sec. 4.2) -----
// z = U^{-1} L^{-1} r with L = I + L_P diag(a)^{-1}, U = diag(a) + U_P, where
// P = diag(a) + L_P + U_P is the TV penta-diagonal matrix.  Its off-diagonal
// entries are b_i = -lam_tv W_{i+1} (couples i, i+1; zero at a row end) and
// c_i = -lam_tv W_{i+n} (couples i, i+n; zero in the last row), so with
// ia = 1/a the sweeps need only W and ia:
//   forward  y_i = r_i + g_i y_{i-1} + h_i y_{i-n},
//            g_i = lam W_i ia_{i-1} [col > 0],  h_i = lam W_i ia_{i-n} [row > 0]
//   backward z_i = ia_i y_i + g_i z_{i+1} + h_i z_{i+n},
//            g_i = lam ia_i W_{i+1} [col < n-1],  h_i = lam ia_i W_{i+n} [row < n-1]
// P is symmetric, so U = diag(a) L^T and Re<r, z> = sum_i ia_i |y_i|^2.
//
// Kernel layout: one CTA per slice, five warps.
//  * Warp 1 (scan warp) runs only the row recurrences: a row is E columns
//    per lane, composed as affine maps and combined by a warp shuffle scan
//    (no block barrier); it stores y (z) itself.
//  * Warps 2-4 (helpers) own two-column chunks and process G rows at a time
//    (independent rows, so their latencies overlap): the residual update
//    r -= alpha q, x += alpha d, and per column (t, h, g) in the scan warp's
//    lane-major layout.
//  * Warp 0 (producer, one lane) fills a ring of S stages of G rows with
//    1-D bulk copies (TMA), one copy per array and stage.
// Handover per stage, with mbarriers: `full` (bytes landed), `empty`
// (helpers done with the natural rows), `ready` (helpers wrote the group's
// coefficients), `consumed` (scan warp done with them).  The scan warp waits
// once per group of G rows and prefetches the next row of the group while
// it scans the current one.  Every wait is bounded; a wait that runs out
// marks the slice faulted and the CTA finishes without hanging.

FI unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

FI void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
FI void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}
FI void mbar_arrive_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
FI bool mbar_test(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// try_wait suspends the thread until the phase completes or the hint
// (nanoseconds) runs out; the loop bounds the whole wait to about a second.
FI bool mbar_try(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(100000u)
      : "memory");
  return ok != 0;
}
// Bounded wait: `tries` suspended polls of about 100 us each after a first
// test (10000 tries: about a second).
FI bool mbar_wait(uint64_t* bar, unsigned parity, int tries = 10000) {
  if (mbar_test(bar, parity)) return true;
  for (int it = 0; it < tries; ++it)
    if (mbar_try(bar, parity)) return true;
  return false;
}
// 1-D bulk copy global -> shared (16-byte aligned, size a multiple of 16),
// completion counted in bytes on `bar`.
FI void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// The same with an L2 eviction policy (a hint: what the ILU reads again in
// its backward sweep stays, what it streams through goes first).
FI void bulk_g2s_hint(void* dst, const void* src, unsigned bytes, uint64_t* bar, uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;\n" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
      : "memory");
}
FI uint64_t l2_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(p));
  return p;
}
FI uint64_t l2_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;\n" : "=l"(p));
  return p;
}
FI void st_hint_f4(float2* dst, float4 v, uint64_t policy) {
  asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;\n" ::"l"(dst), "f"(v.x), "f"(v.y),
               "f"(v.z), "f"(v.w), "l"(policy)
               : "memory");
}
FI void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;\n" ::: "memory"); }
FI int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.cta.shared.b32 %0, [%1];\n" : "=r"(v) : "r"(smem_u32(p)) : "memory");
  return v;
}
FI void st_release(int* p, int v) {
  asm volatile("st.release.cta.shared.b32 [%0], %1;\n" ::"r"(smem_u32(p)), "r"(v) : "memory");
}
// Bounded poll until *p >= want (about a second at most); returns the value
// seen, or -1 when the wait ran out.
FI int poll_at_least(const int* p, int want, int tries = 1 << 24) {
  for (int it = 0; it < tries; ++it) {
    const int v = ld_acquire(p);
    if (v >= want) return v;
    if (it >= 256) __nanosleep(32);
  }
  return -1;
}

// Warp-wide exclusive scan of affine maps v -> A v + B in lane order
// (REV: from lane 31 down).  Returns the value entering this lane's segment
// for a zero value entering the row.
template <bool REV>
FI float2 warp_affine_exclusive(float A, float2 B) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const float Ap = REV ? __shfl_down_sync(0xffffffffu, A, off) : __shfl_up_sync(0xffffffffu, A, off);
    const float bx = REV ? __shfl_down_sync(0xffffffffu, B.x, off) : __shfl_up_sync(0xffffffffu, B.x, off);
    const float by = REV ? __shfl_down_sync(0xffffffffu, B.y, off) : __shfl_up_sync(0xffffffffu, B.y, off);
    if (REV ? (lane + off < 32) : (lane >= off)) {
      B = make_float2(fmaf(A, bx, B.x), fmaf(A, by, B.y));
      A = A * Ap;
    }
  }
  const float bx = REV ? __shfl_down_sync(0xffffffffu, B.x, 1) : __shfl_up_sync(0xffffffffu, B.x, 1);
  const float by = REV ? __shfl_down_sync(0xffffffffu, B.y, 1) : __shfl_up_sync(0xffffffffu, B.y, 1);
  if (lane == (REV ? 31 : 0)) return make_float2(0.f, 0.f);
  return make_float2(bx, by);
}

// Store E consecutive complex values of one lane (columns c0 .. c0+E-1 < n),
// with an L2 eviction policy.
template <int E>
FI void store_lane_row(float2* dst, int c0, int n, const float2 (&v)[E], uint64_t policy) {
  if ((E & 1) == 0 && c0 + E <= n) {
#pragma unroll
    for (int e = 0; e < E; e += 2)
      st_hint_f4(dst + c0 + e, make_float4(v[e].x, v[e].y, v[e + 1].x, v[e + 1].y), policy);
  } else {
#pragma unroll
    for (int e = 0; e < E; ++e)
      if (c0 + e < n) dst[c0 + e] = v[e];
  }
}

constexpr int IW_HWARPS = 3;                   // helper warps (warps 2-4)
constexpr int IW_HELPERS = 32 * IW_HWARPS;
constexpr int IW_THREADS = 32 + IW_HELPERS + 32;
constexpr int IW_MAXCH = 3;                    // chunks of two columns per helper thread (n <= 512)
constexpr int IW_MAXSTAGES = 8;

static int iw_cols_per_lane(int n) { return (n + 31) / 32; }
// Stage of G rows (bytes): R, Q, X, D (8nG each), W (W1 for l1 TV), IA
// (4nG each), W2 (4nG, l1 TV only), then SC: per row, float4 (t.x, t.y, h, g)
// per lane-major column slot.
struct IwLayout {
  int n, G, ns, oQ, oX, oD, oW, oIA, oW2, oSC, bytes;
};
static IwLayout iw_layout(int n, int G, bool aniso = false) {
  IwLayout L;
  L.n = n;
  L.G = G;
  L.ns = 32 * iw_cols_per_lane(n);
  L.oQ = 8 * n * G;
  L.oX = 16 * n * G;
  L.oD = 24 * n * G;
  L.oW = 32 * n * G;
  L.oIA = 36 * n * G;
  L.oW2 = 40 * n * G;
  L.oSC = (aniso ? 44 : 40) * n * G;
  L.bytes = (L.oSC + 16 * L.ns * G + 127) / 128 * 128;
  return L;
}

// Ring position: stage index and the parity of its current use.
struct RingPos {
  int s;
  unsigned ph;
  FI void next(int S) {
    if (++s == S) {
      s = 0;
      ph ^= 1u;
    }
  }
};

// Groups: forward group g holds rows gG .. gG+G-1; backward group g (after
// the NG = n/G forward ones) holds rows n-(g'+1)G .. n-g'G-1, g' = g - NG,
// processed from the bottom row up.  Row uses: forward row k is use k,
// backward step k (row n-1-k) is use n + k; use u sits in group u / G at
// row slot u % G.
template <int E, int G>
__global__ void __launch_bounds__(IW_THREADS, (G == 2 && E <= 10) ? 3 : 1)
    k_ilu(int n, int mode_arg, int S, IwLayout lay, SliceState* __restrict__ st, double* __restrict__ part,
          float2* __restrict__ x, const float2* __restrict__ d, float2* __restrict__ r,
          const float2* __restrict__ q, const float2* __restrict__ atb, float2* __restrict__ y,
          float2* __restrict__ z, const float* __restrict__ ia, const float* __restrict__ wtv, int fuse,
          PcgSched ps, int wait_test, const float* __restrict__ wtv2, int alpha_np) {
  const int s = blockIdx.x;
  if (!slice_running(st, s)) return;
  // ILU_PER_SLICE: the first residual for a slice at the start of its outer
  // step, a PCG step otherwise
  int ph = st[s].phase;
  if (alpha_np > 0 && mode_arg == ILU_PER_SLICE && ph == PH_PCG) {
    // alpha = rho / <d, S d> from the S apply's alpha_np partial sums, as the
    // scalar kernel forms it (same order); a slice that stops here (rho = 0
    // or a breakdown) does nothing more in this macro step
    __shared__ int ph_alpha;
    if (threadIdx.x == 0) {
      const double* pp = part + ((size_t)s * NSLOT + SLOT_DQ) * MAXPART;
      double dq = 0.0;
      for (int i = 0; i < alpha_np; ++i) dq += pp[i];
      pcg_alpha_from(st + s, dq);
      ph_alpha = st[s].done ? -1 : st[s].phase;
    }
    __syncthreads();
    if (ph_alpha < 0) return;
    ph = ph_alpha;
  }
  if (mode_arg == ILU_PER_SLICE && !slice_working(ph)) return;
  const int mode = mode_arg != ILU_PER_SLICE ? mode_arg : (ph == PH_START ? ILU_INIT : ILU_STEP);
  // wait_test (failure-detection test only): the producer issues no copy and
  // every wait gives up after its first poll, so the waits run out with
  // nothing in flight and the slice is reported faulted
  const int tries = wait_test ? 0 : 10000;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar_full[IW_MAXSTAGES], bar_empty[IW_MAXSTAGES];
  __shared__ __align__(8) uint64_t bar_ready[IW_MAXSTAGES], bar_used[IW_MAXSTAGES];
  __shared__ int y_stored;  // 1 once every y row is stored and fenced
  __shared__ volatile int abort_flag;
  __shared__ double red[32];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int NCH = n >> 1;
  const int NG = n / G;
  const float lam = st[s].lam_tv;
  const float alpha = (float)st[s].alpha;
  const size_t base = (size_t)s * n * n;
  // L2 policies: y, W and 1/a are read again by the backward sweep; the
  // rest passes through once
  const uint64_t pol_keep = l2_evict_last(), pol_stream = l2_evict_first();
  if (t == 0) {
    for (int i = 0; i < S; ++i) {
      mbar_init(&bar_full[i], 1);
      mbar_init(&bar_empty[i], IW_HWARPS);
      mbar_init(&bar_ready[i], IW_HWARPS);
      mbar_init(&bar_used[i], 1);
    }
    y_stored = 0;
    abort_flag = 0;
  }
  if (lay.ns > n) {  // slots of columns >= n are never written: make them zero, not garbage
    for (int i = t; i < S * G * lay.ns; i += IW_THREADS) {
      const int row = i / lay.ns;
      unsigned char* sp = smem + (size_t)(row / G) * lay.bytes + lay.oSC + (size_t)(row % G) * 16 * lay.ns;
      reinterpret_cast<float4*>(sp)[i % lay.ns] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  __syncthreads();
  auto fault = [&]() {
    abort_flag = 1;
    st[s].fault = 1;
  };
  // lane-major slot of column c (lane c / E, element c % E), XOR-swizzled so
  // that helper stores of neighbouring columns hit different banks
  auto slot_of = [&](int c) -> int {
    const int e = c % E;
    return e * 32 + ((c / E) ^ (e & 31));
  };
  auto sc_row = [&](int stg, int slot) -> float4* {
    return reinterpret_cast<float4*>(smem + (size_t)stg * lay.bytes + lay.oSC + (size_t)slot * 16 * lay.ns);
  };

  float rr = 0.f, rho = 0.f;

  if (warp == 1) {
    // ============================================================ scan warp
    // (alone on its SM sub-partition: of the five warps, 0 and 4 share one)
    float2 vab[E];  // y of the row above (forward) / z of the row below (backward)
    RingPos pos{0, 0u};
    bool ok = true;
    for (int sweep = 0; sweep < 2 && ok; ++sweep) {
      if (sweep == 1) {
        // y goes back to global memory and is re-read by bulk copies, so
        // order the generic stores before the async proxy
        fence_proxy_async_global();
        __syncwarp();
        if (lane == 0) st_release(&y_stored, 1);
      }
#pragma unroll
      for (int e = 0; e < E; ++e) vab[e] = make_float2(0.f, 0.f);
      for (int gg = 0; gg < NG; ++gg) {
        if (!__all_sync(0xffffffffu, mbar_wait(&bar_ready[pos.s], pos.ph, tries))) {
          ok = false;
          break;
        }
        float4 cA[E], cB[E];
        {
          const float4* sc = sc_row(pos.s, 0);
#pragma unroll
          for (int e = 0; e < E; ++e) cA[e] = sc[e * 32 + (lane ^ (e & 31))];
        }
#pragma unroll
        for (int i = 0; i < G; ++i) {
          float4(&cur)[E] = (i & 1) ? cB : cA;
          float4(&nxt)[E] = (i & 1) ? cA : cB;
          if (i + 1 < G) {  // the next row of this group, while this one is scanned
            const float4* sc = sc_row(pos.s, i + 1);
#pragma unroll
            for (int e = 0; e < E; ++e) nxt[e] = sc[e * 32 + (lane ^ (e & 31))];
          } else {
            __syncwarp();
            if (lane == 0) mbar_arrive(&bar_used[pos.s]);
          }
          float2 tv[E];
          float A = 1.f;
          float2 B = make_float2(0.f, 0.f);
          if (sweep == 0) {
#pragma unroll
            for (int e = 0; e < E; ++e) {
              tv[e] = make_float2(fmaf(cur[e].z, vab[e].x, cur[e].x), fmaf(cur[e].z, vab[e].y, cur[e].y));
              B = make_float2(fmaf(cur[e].w, B.x, tv[e].x), fmaf(cur[e].w, B.y, tv[e].y));
              A *= cur[e].w;
            }
            float2 v = warp_affine_exclusive<false>(A, B);
#pragma unroll
            for (int e = 0; e < E; ++e) {
              v = make_float2(fmaf(cur[e].w, v.x, tv[e].x), fmaf(cur[e].w, v.y, tv[e].y));
              vab[e] = v;
            }
            store_lane_row<E>(y + base + (size_t)(gg * G + i) * n, E * lane, n, vab, pol_keep);
          } else {
#pragma unroll
            for (int e = E - 1; e >= 0; --e) {
              tv[e] = make_float2(fmaf(cur[e].z, vab[e].x, cur[e].x), fmaf(cur[e].z, vab[e].y, cur[e].y));
              B = make_float2(fmaf(cur[e].w, B.x, tv[e].x), fmaf(cur[e].w, B.y, tv[e].y));
              A *= cur[e].w;
            }
            float2 v = warp_affine_exclusive<true>(A, B);
#pragma unroll
            for (int e = E - 1; e >= 0; --e) {
              v = make_float2(fmaf(cur[e].w, v.x, tv[e].x), fmaf(cur[e].w, v.y, tv[e].y));
              vab[e] = v;
            }
            store_lane_row<E>(z + base + (size_t)(n - 1 - gg * G - i) * n, E * lane, n, vab, pol_stream);
          }
        }
        pos.next(S);
      }
    }
    if (!ok) fault();
  } else if (warp == 0) {
    // ============================================================= producer
    if (lane == 0) {
      const float2* rsrc = (mode == ILU_INIT) ? atb : r;
      const bool init = mode == ILU_INIT;
      const unsigned c8 = 8u * n * G, c4 = 4u * n * G;
      RingPos pos{0, 0u};
      bool ok = true;
      for (int g = 0; g < 2 * NG && ok; ++g) {
        if (abort_flag) break;
        if (wait_test) {  // no copy is issued: the consumers' waits run out
          ok = false;
          break;
        }
        // the stage's previous group (g - S) has been left by every helper
        if (g >= S && !mbar_wait(&bar_empty[pos.s], pos.ph ^ 1u, tries)) {
          ok = false;
          break;
        }
        if (g == NG && poll_at_least(&y_stored, 1, tries ? 1 << 24 : 0) < 1) {  // backward copies read y
          ok = false;
          break;
        }
        unsigned char* sp = smem + (size_t)pos.s * lay.bytes;
        uint64_t* bar = &bar_full[pos.s];
        const unsigned cw2 = wtv2 ? c4 : 0u;
        if (g < NG) {
          const size_t go = base + (size_t)g * G * n;
          mbar_arrive_tx(bar, (init ? 2 * c8 + 2 * c4 : 4 * c8 + 2 * c4) + cw2);
          // streamed once: r, q, x, d; read again by the backward sweep: W, 1/a
          bulk_g2s_hint(sp, rsrc + go, c8, bar, pol_stream);
          bulk_g2s_hint(sp + lay.oQ, q + go, c8, bar, pol_stream);
          if (!init) {
            bulk_g2s_hint(sp + lay.oX, x + go, c8, bar, pol_stream);
            bulk_g2s_hint(sp + lay.oD, d + go, c8, bar, pol_stream);
          }
          bulk_g2s_hint(sp + lay.oW, wtv + go, c4, bar, pol_keep);
          bulk_g2s_hint(sp + lay.oIA, ia + go, c4, bar, pol_keep);
          if (wtv2) bulk_g2s_hint(sp + lay.oW2, wtv2 + go, c4, bar, pol_keep);
        } else {
          const size_t go = base + (size_t)(n - (g - NG + 1) * G) * n;
          mbar_arrive_tx(bar, c8 + 2 * c4 + cw2);
          // last uses
          bulk_g2s_hint(sp, y + go, c8, bar, pol_stream);
          bulk_g2s_hint(sp + lay.oW, wtv + go, c4, bar, pol_stream);
          bulk_g2s_hint(sp + lay.oIA, ia + go, c4, bar, pol_stream);
          if (wtv2) bulk_g2s_hint(sp + lay.oW2, wtv2 + go, c4, bar, pol_stream);
        }
        pos.next(S);
      }
      if (!ok) fault();
    }
  } else {
    // ============================================================== helpers
    const int hh = t - 64;
    float2 prev[IW_MAXCH];  // ia of the row above (forward) / W of the row below (backward)
    // sums per column chunk: each chunk meets its rows in the same order for
    // every ring shape, so the totals do not depend on G or S
    float rr_c[IW_MAXCH], rho_c[IW_MAXCH];
#pragma unroll
    for (int c = 0; c < IW_MAXCH; ++c) rr_c[c] = rho_c[c] = 0.f;
#pragma unroll
    for (int c = 0; c < IW_MAXCH; ++c) prev[c] = make_float2(0.f, 0.f);
    bool ok = true;
    RingPos pos{0, 0u};
    const size_t nG4 = (size_t)4 * n;  // bytes per float row
    for (int g = 0; g < 2 * NG && ok; ++g) {
      if (__any_sync(0xffffffffu, abort_flag != 0)) break;
      if (g == NG) {
#pragma unroll
        for (int c = 0; c < IW_MAXCH; ++c) prev[c] = make_float2(0.f, 0.f);
      }
      unsigned char* sp = smem + (size_t)pos.s * lay.bytes;
      bool got = mbar_wait(&bar_full[pos.s], pos.ph, tries);
      if (g >= S) got = got && mbar_wait(&bar_used[pos.s], pos.ph ^ 1u, tries);  // scan warp left group g - S
      if (!__all_sync(0xffffffffu, got)) {
        ok = false;
        break;
      }
      if (g < NG) {
#pragma unroll
        for (int ch = 0; ch < IW_MAXCH; ++ch) {
          const int j = hh + IW_HELPERS * ch;
          if (j < NCH) {
            const int c = 2 * j;
#pragma unroll
            for (int i = 0; i < G; ++i) {
              const size_t g0 = base + (size_t)(g * G + i) * n + c;
              const unsigned char* rowp = sp + (size_t)i * 8 * n;
              const float4 r4 = *reinterpret_cast<const float4*>(rowp + 16 * j);
              const float4 q4 = *reinterpret_cast<const float4*>(rowp + lay.oQ + 16 * j);
              float4 rn;
              if (mode == ILU_INIT) {
                rn = make_float4(r4.x - q4.x, r4.y - q4.y, r4.z - q4.z, r4.w - q4.w);
              } else {
                const float4 x4 = *reinterpret_cast<const float4*>(rowp + lay.oX + 16 * j);
                const float4 d4 = *reinterpret_cast<const float4*>(rowp + lay.oD + 16 * j);
                rn = make_float4(fmaf(-alpha, q4.x, r4.x), fmaf(-alpha, q4.y, r4.y), fmaf(-alpha, q4.z, r4.z),
                                 fmaf(-alpha, q4.w, r4.w));
                st_hint_f4(x + g0,
                           make_float4(fmaf(alpha, d4.x, x4.x), fmaf(alpha, d4.y, x4.y), fmaf(alpha, d4.z, x4.z),
                                       fmaf(alpha, d4.w, x4.w)),
                           pol_stream);
              }
              st_hint_f4(r + g0, rn, pol_stream);
              rr_c[ch] += rn.x * rn.x + rn.y * rn.y + rn.z * rn.z + rn.w * rn.w;
              const float* wrow = reinterpret_cast<const float*>(sp + lay.oW + i * nG4);
              const float* arow = reinterpret_cast<const float*>(sp + lay.oIA + i * nG4);
              const float2 w2 = *reinterpret_cast<const float2*>(wrow + c);
              const float2 a2 = *reinterpret_cast<const float2*>(arow + c);
              const float ial = c > 0 ? arow[c - 1] : 0.f;
              const float2 aab = prev[ch];  // ia of the row above
              const float lw0 = lam * w2.x, lw1 = lam * w2.y;
              // vertical couplings use W2 (l1 TV), else W
              float lv0 = lw0, lv1 = lw1;
              if (wtv2) {
                const float2 v2 = *reinterpret_cast<const float2*>(
                    reinterpret_cast<const float*>(sp + lay.oW2 + i * nG4) + c);
                lv0 = lam * v2.x;
                lv1 = lam * v2.y;
              }
              float4* sc = sc_row(pos.s, i);
              sc[slot_of(c)] = make_float4(rn.x, rn.y, lv0 * aab.x, lw0 * ial);
              sc[slot_of(c + 1)] = make_float4(rn.z, rn.w, lv1 * aab.y, lw1 * a2.x);
              prev[ch] = a2;
            }
          }
        }
      } else {
#pragma unroll
        for (int ch = 0; ch < IW_MAXCH; ++ch) {
          const int j = hh + IW_HELPERS * ch;
          if (j < NCH) {
            const int c = 2 * j;
#pragma unroll
            for (int i = 0; i < G; ++i) {
              const int o = G - 1 - i;  // memory row of processing slot i
              const float4 y4 = *reinterpret_cast<const float4*>(sp + (size_t)o * 8 * n + 16 * j);
              const float* wrow = reinterpret_cast<const float*>(sp + lay.oW + o * nG4);
              const float* arow = reinterpret_cast<const float*>(sp + lay.oIA + o * nG4);
              const float2 w2 = *reinterpret_cast<const float2*>(wrow + c);
              const float2 a2 = *reinterpret_cast<const float2*>(arow + c);
              const float w3 = c + 2 < n ? wrow[c + 2] : 0.f;
              const float2 wbl = prev[ch];  // W (W2 for l1 TV) of the row below
              const float la0 = lam * a2.x, la1 = lam * a2.y;
              const float2 t0 = make_float2(a2.x * y4.x, a2.x * y4.y), t1 = make_float2(a2.y * y4.z, a2.y * y4.w);
              rho_c[ch] = fmaf(t0.x, y4.x, fmaf(t0.y, y4.y, rho_c[ch]));
              rho_c[ch] = fmaf(t1.x, y4.z, fmaf(t1.y, y4.w, rho_c[ch]));
              float4* sc = sc_row(pos.s, i);
              sc[slot_of(c)] = make_float4(t0.x, t0.y, la0 * wbl.x, la0 * w2.y);
              sc[slot_of(c + 1)] = make_float4(t1.x, t1.y, la1 * wbl.y, la1 * w3);
              prev[ch] = wtv2 ? *reinterpret_cast<const float2*>(
                                    reinterpret_cast<const float*>(sp + lay.oW2 + o * nG4) + c)
                              : w2;
            }
          }
        }
      }
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&bar_empty[pos.s]);
        mbar_arrive(&bar_ready[pos.s]);
      }
      pos.next(S);
    }
    if (!ok) fault();
#pragma unroll
    for (int c = 0; c < IW_MAXCH; ++c) {
      rr += rr_c[c];
      rho += rho_c[c];
    }
  }
  __syncthreads();
  const double trz = block_sum((double)rho, red);
  __syncthreads();
  const double trr = block_sum((double)rr, red);
  if (t == 0) {
    part[((size_t)s * NSLOT + SLOT_RZ) * MAXPART] = trz;
    part[((size_t)s * NSLOT + SLOT_RR) * MAXPART] = trr;
    if (fuse && !abort_flag) {
      if (mode == ILU_INIT)
        pcg_rho_init_from(st + s, 0.0 + trz, 0.0 + trr);
      else
        pcg_beta_from(st + s, 0.0 + trz, 0.0 + trr, ps);
    }
  }
}

typedef void (*IluKernel)(int, int, int, IwLayout, SliceState*, double*, float2*, const float2*, float2*,
                          const float2*, const float2*, float2*, float2*, const float*, const float*, int, PcgSched,
                          int, const float*, int);
template <int G>
static IluKernel ilu_kernel_g(int E) {
  switch (E) {
    case 1: return k_ilu<1, G>;
    case 2: return k_ilu<2, G>;
    case 3: return k_ilu<3, G>;
    case 4: return k_ilu<4, G>;
    case 5: return k_ilu<5, G>;
    case 6: return k_ilu<6, G>;
    case 8: return k_ilu<8, G>;
    case 10: return k_ilu<10, G>;
    case 12: return k_ilu<12, G>;
    case 16: return k_ilu<16, G>;
    default: return nullptr;
  }
}
static IluKernel ilu_kernel(int n, int G) {
  const int E = iw_cols_per_lane(n);
  return G == 4 ? ilu_kernel_g<4>(E) : ilu_kernel_g<2>(E);
}

static constexpr int ILU_SMEM_MAX = 200 * 1024;

bool ilu_prepare() {
  bool ok = true;
  for (int e : {1, 2, 3, 4, 5, 6, 8, 10, 12, 16})
    for (int G : {2, 4})
      ok = cudaFuncSetAttribute(ilu_kernel(32 * e, G), cudaFuncAttributeMaxDynamicSharedMemorySize, ILU_SMEM_MAX) ==
               cudaSuccess && ok;
  return ok;
}

// Ring shape, encoded 10 * G + S: G rows per stage and S stages.  With one
// CTA per SM (batch <= 152) the ring takes 4-row stages, three of them as
// long as they fit; with more CTAs per SM, 2-row stages in the shared
// memory each CTA gets.
int ilu_default_shape(int n, int batch, bool aniso) {
  int per_sm = (batch + 151) / 152;
  if (per_sm > 3) per_sm = 3;
  const int budget = per_sm == 1 ? ILU_SMEM_MAX : (224 * 1024) / per_sm - 2048;
  for (int G : {4, 2}) {
    if (per_sm > 1 && G == 4) continue;
    int S = budget / iw_layout(n, G, aniso).bytes;
    if (S > 4) S = 4;
    if (S >= 2) return 10 * G + S;
  }
  return 10 * 2 + 2;
}

bool ilu_shape_fits(int n, int shape, bool aniso) {
  const int G = shape / 10, S = shape % 10;
  if ((G != 2 && G != 4) || S < 2 || S > IW_MAXSTAGES || n % G) return false;
  return (long)S * iw_layout(n, G, aniso).bytes <= ILU_SMEM_MAX;
}

void ilu_step(int batch, int n, cudaStream_t s, SliceState* st, double* part, int mode, float2* x,
              const float2* d, float2* r, const float2* q, const float2* atb, float2* y, float2* z,
              const float* ia, const float* wtv, int shape, int fuse_scalars, PcgSched ps, int wait_test,
              const float* wtv2, int alpha_np) {
  const bool aniso = wtv2 != nullptr;
  if (shape <= 0 || !ilu_shape_fits(n, shape, aniso)) shape = ilu_default_shape(n, batch, aniso);
  const int G = shape / 10, S = shape % 10;
  const IwLayout lay = iw_layout(n, G, aniso);
  ilu_kernel(n, G)<<<batch, IW_THREADS, (size_t)S * lay.bytes, s>>>(n, mode, S, lay, st, part, x, d, r, q, atb, y,
                                                                     z, ia, wtv, fuse_scalars, ps, wait_test, wtv2,
                                                                     alpha_np);
}

// =========================================================== PCG vectors ==

int axpy_ctas(int n) {
  const int N = n * n;
  int c = N / 2048;
  if (c < 1) c = 1;
  if (c > MAXPART) c = MAXPART;
  return c;
}

__global__ void k_axpy(int N, int mode_arg, const SliceState* __restrict__ st, double* __restrict__ part,
                       float2* __restrict__ x, const float2* __restrict__ d, float2* __restrict__ r,
                       const float2* __restrict__ q, const float2* __restrict__ atb) {
  const int s = blockIdx.y;
  if (!slice_running(st, s)) return;
  const int ph = st[s].phase;
  if (mode_arg == AXPY_PER_SLICE && !slice_working(ph)) return;
  const int mode = mode_arg != AXPY_PER_SLICE ? mode_arg : (ph == PH_START ? AXPY_INIT : AXPY_STEP);
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

// Residual update with a diagonal preconditioner (Jacobi PCG, sdiag = 1 /
// diag(S)) or none (standard CG, sdiag null), for the comparison of Sec. 5.2.
__global__ void k_axpy_diag(int N, int mode_arg, const SliceState* __restrict__ st, double* __restrict__ part,
                            float2* __restrict__ x, const float2* __restrict__ d, float2* __restrict__ r,
                            const float2* __restrict__ q, const float2* __restrict__ atb,
                            const float* __restrict__ sdiag, float2* __restrict__ z) {
  const int s = blockIdx.y;
  if (!slice_running(st, s)) return;
  const int ph = st[s].phase;
  if (mode_arg == AXPY_PER_SLICE && !slice_working(ph)) return;
  const int mode = mode_arg != AXPY_PER_SLICE ? mode_arg : (ph == PH_START ? AXPY_INIT : AXPY_STEP);
  __shared__ double red[32];
  const float alpha = (float)st[s].alpha;
  const size_t base = (size_t)s * N;
  const int chunk = (N + gridDim.x - 1) / gridDim.x;
  const int lo = blockIdx.x * chunk, hi = min(N, lo + chunk);
  float rz = 0.f, rr = 0.f;
  for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const size_t g = base + i;
    float2 rv;
    if (mode == AXPY_INIT) {
      rv = csub(atb[g], q[g]);
    } else {
      x[g] = cfma(alpha, d[g], x[g]);
      rv = cfma(-alpha, q[g], r[g]);
    }
    r[g] = rv;
    const float sc = sdiag ? sdiag[g] : 1.f;
    z[g] = cscale(rv, sc);
    const float r2 = cabs2(rv);
    rr += r2;
    rz = fmaf(sc, r2, rz);
  }
  const double trz = block_sum((double)rz, red);
  __syncthreads();
  const double trr = block_sum((double)rr, red);
  if (threadIdx.x == 0) {
    part[((size_t)s * NSLOT + SLOT_RZ) * MAXPART + blockIdx.x] = trz;
    part[((size_t)s * NSLOT + SLOT_RR) * MAXPART + blockIdx.x] = trr;
  }
}

void axpy_diag_step(int batch, int n, cudaStream_t s, const SliceState* st, double* part, int mode, float2* x,
                    const float2* d, float2* r, const float2* q, const float2* atb, const float* sdiag, float2* z) {
  k_axpy_diag<<<dim3(axpy_ctas(n), batch), 256, 0, s>>>(n * n, mode, st, part, x, d, r, q, atb, sdiag, z);
}

__global__ void k_jacobi_wavelet(int N, const SliceState* __restrict__ st, const float* __restrict__ wdiag,
                                 float* __restrict__ ia) {
  const int s = blockIdx.y;
  if (!slice_running(st, s)) return;
  const float abar = st[s].abar, lw = st[s].lam;
  const size_t base = (size_t)s * N;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
    ia[base + i] = 1.0f / fmaf(lw, wdiag[base + i], abar);
}

void jacobi_wavelet_setup(int batch, int n, cudaStream_t s, const SliceState* st, const float* wdiag, float* ia) {
  const int N = n * n;
  const int blocks = (N + 255) / 256 < 64 ? (N + 255) / 256 : 64;
  k_jacobi_wavelet<<<dim3(blocks, batch), 256, 0, s>>>(N, st, wdiag, ia);
}

// End of a slice's outer step (PH_END): x^{k+1} = x^k + dx, where
// dx = sum_j alpha_j d_j was accumulated from zero by the PCG steps (so its
// rounding is relative to the step, not to x), and dx is cleared for the next
// outer step; partial ||dx||^2 (SLOT_DX) and ||x^k||^2 (SLOT_XX) for the
// relative change.  Slices stopped by a breakdown are done and keep x^k.
__global__ void k_outer_apply(int N, const SliceState* __restrict__ st, float2* __restrict__ x,
                              float2* __restrict__ dx, double* __restrict__ part) {
  const int s = blockIdx.y;
  if (!slice_running(st, s) || st[s].phase != PH_END) return;
  __shared__ double red[32];
  const size_t base = (size_t)s * N;
  const int chunk = (N + gridDim.x - 1) / gridDim.x;
  const int lo = blockIdx.x * chunk, hi = min(N, lo + chunk);
  float a = 0.f, b = 0.f;
  for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const float2 xv = x[base + i], dv = dx[base + i];
    a += cabs2(dv);
    b += cabs2(xv);
    x[base + i] = cadd(xv, dv);
    dx[base + i] = make_float2(0.f, 0.f);
  }
  const double ta = block_sum((double)a, red);
  __syncthreads();
  const double tb = block_sum((double)b, red);
  if (threadIdx.x == 0) {
    part[((size_t)s * NSLOT + SLOT_DX) * MAXPART + blockIdx.x] = ta;
    part[((size_t)s * NSLOT + SLOT_XX) * MAXPART + blockIdx.x] = tb;
  }
}

void outer_apply(int batch, int n, cudaStream_t s, const SliceState* st, float2* x, float2* dx,
                 double* part) {
  k_outer_apply<<<dim3(axpy_ctas(n), batch), 256, 0, s>>>(n * n, st, x, dx, part);
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

// ======================================================== objective sums ===

// C > 1 (joint sparsity, no group map): the first slice of each image sums
// sqrt(sum_t |c_tj|^2 + eps) over its C contrasts, the others contribute 0.
__global__ void k_l21_sum(int n, int C, const float2* __restrict__ c, const int* __restrict__ gidx,
                          const int* __restrict__ goff, int G, int gsize, float eps, double* __restrict__ part,
                          int slot) {
  const int s = blockIdx.y;
  __shared__ double red[32];
  const size_t N = (size_t)n * n;
  const float2* cs = c + (size_t)s * N;
  const int count = gidx ? G : n * n;
  const int chunk = (count + gridDim.x - 1) / gridDim.x;
  const int lo = blockIdx.x * chunk, hi = min(count, lo + chunk);
  const int cc = s % C == 0 ? C : 0;
  float acc = 0.f;
  for (int g = lo + threadIdx.x; g < hi; g += blockDim.x) {
    float ss;
    if (C > 1) {
      if (!cc) break;
      ss = 0.f;
      for (int t = 0; t < cc; ++t) ss += cabs2(cs[(size_t)t * N + g]);
    } else if (!gidx) {
      ss = cabs2(cs[g]);
    } else {
      const int b = goff ? goff[g] : g * gsize;
      const int e = goff ? goff[g + 1] : b + gsize;
      ss = 0.f;
      for (int k = b; k < e; ++k) ss += cabs2(cs[gidx[k]]);
    }
    acc += sqrtf(ss + eps);
  }
  const double tot = block_sum((double)acc, red);
  if (threadIdx.x == 0) part[((size_t)s * NSLOT + slot) * MAXPART + blockIdx.x] = tot;
}

void l21_sum(int batch, int n, cudaStream_t s, const float2* c, const int* gidx, const int* goff, int G, int gsize,
             float eps, double* part, int slot, int channels) {
  k_l21_sum<<<dim3(axpy_ctas(n), batch), 256, 0, s>>>(n, channels, c, gidx, goff, G, gsize, eps, part, slot);
}

// C > 1 (joint TV): the first slice of each image sums sqrt(sum_t |grad
// x_t,i|^2 + eps) over its C contrasts, the others contribute 0.
__global__ void k_tv_sum(int n, int C, const float2* __restrict__ x, float eps, double* __restrict__ part, int slot,
                         int aniso) {
  const int s = blockIdx.y;
  __shared__ double red[32];
  const size_t base = (size_t)s * n * n;
  const int N = n * n;
  const int chunk = (N + gridDim.x - 1) / gridDim.x;
  const int lo = blockIdx.x * chunk, hi = min(N, lo + chunk);
  const int cc = (C == 1 || s % C == 0) ? C : 0;
  float acc = 0.f;
  for (int i = lo + threadIdx.x; i < hi && cc; i += blockDim.x) {
    const int r = i / n, col = i % n;
    float g = 0.f, ga = 0.f;
    for (int t = 0; t < cc; ++t) {
      const size_t bt = base + (size_t)t * N;
      const float2 xc = x[bt + i];
      const float2 g1 = col > 0 ? csub(xc, x[bt + i - 1]) : xc;
      const float2 g2 = r > 0 ? csub(xc, x[bt + i - n]) : xc;
      g += cabs2(g1) + cabs2(g2);
      if (aniso) ga = sqrtf(cabs2(g1) + eps) + sqrtf(cabs2(g2) + eps);
    }
    acc += aniso ? ga : sqrtf(g + eps);
  }
  const double tot = block_sum((double)acc, red);
  if (threadIdx.x == 0) part[((size_t)s * NSLOT + slot) * MAXPART + blockIdx.x] = tot;
}

void tv_sum(int batch, int n, cudaStream_t s, const float2* x, float eps, double* part, int slot, int aniso,
            int channels) {
  k_tv_sum<<<dim3(axpy_ctas(n), batch), 256, 0, s>>>(n, channels, x, eps, part, slot, aniso);
}

// ========================================================== PCG scalars ===

FI double sum_parts(const double* part, int s, int slot, int np) {
  const double* p = part + ((size_t)s * NSLOT + slot) * MAXPART;
  double a = 0.0;
  for (int i = 0; i < np; ++i) a += p[i];
  return a;
}

// The sum over the C contrasts (consecutive slices) of the image that slice s
// belongs to: multi-contrast PCG runs on the stacked unknown (Sec. 5.6), so
// its inner products, and the relative change of the outer step, are sums
// over the contrasts.  Every slice of the image sums in the same order and
// takes the same scalars and the same phase transitions.
FI double image_parts(const double* part, int s, int slot, int np, int C) {
  if (C == 1) return sum_parts(part, s, slot, np);
  const int s0 = s - s % C;
  double a = 0.0;
  for (int t = s0; t < s0 + C; ++t) a += sum_parts(part, t, slot, np);
  return a;
}

__global__ void k_state_init(int B, SliceState* st, const double* part, int np, const int* counts, int N,
                             const float* lam, const float* lam_tv, float eps, int outer_max, int phase, int C) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= B) return;
  SliceState v;
  v.rho = 0.0;
  v.alpha = 0.0;
  v.beta = 0.0;
  v.rhs2 = image_parts(part, s, SLOT_RHS, np, C);
  v.rr = v.rhs2;
  v.rr0 = v.rhs2;
  v.relchg = 0.0;
  v.stall = 0;
  v.phase = phase;
  v.pcg_j = 0;
  v.outer_max = outer_max;
  for (int i = 0; i < MU_WINDOW; ++i) v.hist[i] = 0.f;
  // non-finite k-space on the mask makes A^H b non-finite: the slice is not
  // iterated and counts as a breakdown (its x keeps the start)
  const bool bad = !isfinite(v.rhs2);
  v.active = bad ? 0 : 1;
  v.done = bad ? 1 : 0;
  v.breakdown = bad ? 1 : 0;
  v.pcg_steps = 0;
  v.outer_done = 0;
  v.fault = 0;
  v.lam = lam[s];
  v.lam_tv = lam_tv[s];
  v.abar = (float)((double)counts[s] / (double)N);
  v.eps = eps;
  st[s] = v;
}

void state_init(int batch, cudaStream_t s, SliceState* st, const double* part, int np, const int* counts,
                int n, const float* lam, const float* lam_tv, float eps, int outer_max, int phase, int channels) {
  k_state_init<<<(batch + 127) / 128, 128, 0, s>>>(batch, st, part, np, counts, n * n, lam, lam_tv, eps,
                                                   outer_max, phase, channels);
}

// The slices whose outer step is due (PH_BOUNDARY), as a copy of the state in
// which every other slice reads as done: the weight and preconditioner
// set-up kernels, which skip done slices and never write the state, then
// work on exactly those slices.  The slices themselves move to PH_START (this
// macro step's S apply and PCG update form their first residual, after the
// set-up kernels have run).
__global__ void k_boundary_view(int B, SliceState* __restrict__ st, SliceState* __restrict__ view) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= B) return;
  SliceState v = st[s];
  if (v.phase != PH_BOUNDARY) {
    v.done = 1;
  } else if (v.active && !v.done) {
    st[s].phase = PH_START;
  }
  view[s] = v;
}

void boundary_view(int batch, cudaStream_t s, SliceState* st, SliceState* view) {
  k_boundary_view<<<(batch + 127) / 128, 128, 0, s>>>(batch, st, view);
}

__global__ void k_alpha(int B, SliceState* st, const double* part, int np, int C) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= B || !slice_in_pcg(st, s)) return;
  pcg_alpha_from(st + s, image_parts(part, s, SLOT_DQ, np, C));
}

void pcg_alpha(int batch, cudaStream_t s, SliceState* st, const double* part, int np, int channels) {
  k_alpha<<<(batch + 127) / 128, 128, 0, s>>>(batch, st, part, np, channels);
}

// After z = P^{-1} r: rho (first residual, slices at the start of an outer
// step) or beta and the PCG stop (slices in PCG); mode INIT / STEP forces one
// of them for every running slice.
__global__ void k_pcg_scalars(int B, SliceState* st, const double* part, int np_rz, int np_rr, int mode,
                              PcgSched ps, int C) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= B || !slice_running(st, s) || st[s].fault) return;
  const int ph = st[s].phase;
  const bool init = mode == SCALARS_INIT || (mode == SCALARS_PER_SLICE && ph == PH_START);
  const bool step = mode == SCALARS_STEP || (mode == SCALARS_PER_SLICE && ph == PH_PCG);
  const double rz = image_parts(part, s, SLOT_RZ, np_rz, C), rr = image_parts(part, s, SLOT_RR, np_rr, C);
  if (init)
    pcg_rho_init_from(st + s, rz, rr);
  else if (step)
    pcg_beta_from(st + s, rz, rr, ps);
}

void pcg_scalars(int batch, cudaStream_t s, SliceState* st, const double* part, int np_rz, int np_rr, int mode,
                 const PcgSched& ps, int channels) {
  k_pcg_scalars<<<(batch + 127) / 128, 128, 0, s>>>(batch, st, part, np_rz, np_rr, mode, ps, channels);
}

// Outer-loop stop.  kind 0: relative change <= tol.  kind 1: estimated
// distance to the limit <= tol.  Under linear convergence x^k -> x* with
// contraction mu, ||x^k - x*|| ~ relchg_k mu / (1 - mu) (the sum of the
// remaining steps) relative to ||x^k||; mu is the geometric mean contraction
// over the last MU_WINDOW steps, (relchg_k / relchg_{k-W})^(1/W), capped at
// 0.999 (a long window: the rate drifts early on and FP32 rounding jitters
// single steps).  Either kind also stops a slice whose relative change has
// stayed at or below stall_tol for STALL_STEPS consecutive steps: the FP32
// rounding floor of the outer iteration, below which it cannot move.  Kind 1
// stops a slice on a plateau too: from outer step plateau_after on (a whole
// window in the phase of nearly exact inner solves, where the outer
// iteration contracts by far more than 20 % over the window), a relative
// change at or below tol that has not fallen by 20 % over the window is that
// slice's FP32 floor, whatever its level.
__global__ void k_outer_end(int B, SliceState* st, const double* part, int np, float tol, int kind,
                            float stall_tol, int plateau_after, int C) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= B || !slice_running(st, s) || st[s].phase != PH_END) return;
  SliceState* v = st + s;
  const double dx = image_parts(part, s, SLOT_DX, np, C);
  const double xx = image_parts(part, s, SLOT_XX, np, C);
  const double rel = xx > 0.0 ? sqrt(dx / xx) : INFINITY;
  const int k = v->outer_done;  // this step's index
  const float old = v->hist[k % MU_WINDOW];  // relchg of step k - MU_WINDOW
  v->hist[k % MU_WINDOW] = (float)rel;
  v->relchg = rel;
  v->outer_done = k + 1;
  v->stall = (stall_tol > 0.f && rel <= (double)stall_tol) ? v->stall + 1 : 0;
  if (v->stall >= STALL_STEPS) {
    v->done = 1;
    return;
  }
  if (tol > 0.f) {
    if (kind == 0) {
      if (rel <= (double)tol) v->done = 1;
    } else if (k >= MU_WINDOW && old > 0.f) {
      const double mu = fmin(pow(rel / (double)old, 1.0 / MU_WINDOW), 0.999);
      if (rel * mu / (1.0 - mu) <= (double)tol && rel <= (double)tol) v->done = 1;
      if (k >= plateau_after && rel <= (double)tol && rel >= 0.8 * (double)old) v->done = 1;
    }
  }
  if (v->outer_done >= v->outer_max) v->done = 1;
  if (!v->done) v->phase = PH_BOUNDARY;  // the next outer step starts
}

void outer_end(int batch, cudaStream_t s, SliceState* st, const double* part, int np, float tol, int kind,
               float stall_tol, int plateau_after, int channels) {
  k_outer_end<<<(batch + 127) / 128, 128, 0, s>>>(batch, st, part, np, tol, kind, stall_tol, plateau_after,
                                                  channels);
}

}  // namespace firls
