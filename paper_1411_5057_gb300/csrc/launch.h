// Host-side launch wrappers shared by the translation units of the library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "firls_common.cuh"

namespace firls {

struct FftArgs {
  int batch = 0;
  cudaStream_t stream = 0;
  const float2* tw = nullptr;     // twiddles exp(-2 pi i j / n), j < n
  const SliceState* st = nullptr;
  double* part = nullptr;
  const float2* z = nullptr;
  float2* d = nullptr;
  float2* t = nullptr;
  const float2* b = nullptr;
  const uint8_t* mask = nullptr;
  float2* atb = nullptr;
  float2* x = nullptr;
  const float2* u = nullptr;
  const float* wtv = nullptr;
  const float* wtv2 = nullptr;  // l1 TV: the vertical weights W2 (wtv then holds W1)
  float2* q = nullptr;
  const float2* xs = nullptr;   // row FFT, per-slice mode: x^k of slices starting an outer step
  int mode = 0;
  int real = 0;
};

bool fft_size_supported(int n);
int fft_row_ctas(int n);
int fft_col_ctas(int n);
void fft_row_fwd(int n, const FftArgs& a);
void fft_row_ahb(int n, const FftArgs& a);
void fft_col_mask(int n, const FftArgs& a);
void fft_col_inv(int n, const FftArgs& a);
void fft_row_inv(int n, const FftArgs& a);
// partial ||R F x - b||^2 (t = rowFFT(x), a.b, a.mask) into slot a.mode
void fft_col_resid(int n, const FftArgs& a);
// t = colIFFT((1 - R) colFFT(t) + R n b)  (data consistency, column part)
void fft_col_dc(int n, const FftArgs& a);
void fft_prepare(int n);  // set shared-memory limits (call outside capture)

// ---- wavelet (lifting) ----
enum WavMode { WAV_RAW = 0, WAV_MUL_W = 1, WAV_MUL_PINV = 2, WAV_SINGLETON_W = 3 };

struct WavArgs {
  int batch = 0, n = 0, levels = 0, kind = 0;
  cudaStream_t stream = 0;
  const SliceState* st = nullptr;   // slices not running are skipped (may be null)
  float2* tmpA = nullptr;           // [batch][n/2 * n/2] ping-pong LL buffers
  float2* tmpB = nullptr;
  double* part = nullptr;
  int rb = 0;          // rows per CTA of the tiled levels (0: default 8)
  int coarse_max = 0;  // largest side kept in shared memory (0: default 64)
};
// c = Phi x (Mallat, stride n) with the final store scaled per `mode`:
// RAW: c; MUL_W: w*c; MUL_PINV: c / (abar + lam w); SINGLETON_W: writes
// w = (|c|^2 + eps)^-1/2 into `w` instead of c.
void wavelet_forward(const WavArgs& a, const float2* x, float2* c, float* w, int mode);
// x = Phi^T c; if r != null also partial Re<r, x> into SLOT_RZ.
void wavelet_inverse(const WavArgs& a, const float2* c, float2* x, const float2* r, int real);
// u = Phi^T (s o Phi x), s = w (MUL_W) or 1/(abar + lam w) (MUL_PINV).
// Where a slice fits the shared memory of one thread-block cluster (rb 0, 1
// or 2) every level runs in one launch and c is not touched; otherwise
// (rb 4, 8, 16, or no fit) the fine levels are tiled, a launch per level,
// their scaled details going through c, and the levels that fit one CTA's
// shared memory are fused.  Optional partial Re<r, u>.
void wavelet_apply(const WavArgs& a, const float2* x, float2* c, float* w, int mode, float2* u,
                   const float2* r, int real);
int wavelet_cluster_ctas(int n, int levels, int kind, int rb);
int wavelet_apply_ctas(int n, int levels, int kind, int rb, int coarse_max);
int wavelet_apply_launches(int n, int levels, int kind, int rb, int coarse_max);
void wav_prepare();

// ---- TV, preconditioner, groups, PCG scalars ----
// wtv2 null: isotropic TV weights into wtv; else l1 TV: W1 into wtv, W2 into wtv2.
// channels C > 1: joint TV weights of each image of C consecutive slices
// (isotropic only), the same W into every contrast.
void tv_weights(int batch, int n, cudaStream_t s, const SliceState* st, const float2* x, float* wtv, float* wtv2,
                int channels = 1);
// Joint wavelet-sparsity weights from the raw coefficients cw of every slice:
// ww = (sum over the C contrasts of |c_j|^2 + eps)^(-1/2) for every contrast.
void joint_wavelet_weights(int batch, int n, int channels, cudaStream_t s, const SliceState* st, const float2* cw,
                           float* ww);
void wavelet_diag(int batch, int n, int levels, cudaStream_t s, const SliceState* st, const float* w,
                  float* out, const float* sqtab, const int* sqlen);
void penta_setup(int batch, int n, cudaStream_t s, const SliceState* st, const float* wtv, const float* wtv2,
                 const float* wdiag, float* ia);
// ia = 1/a -> 1/d, the ILU(0) pivots (updated pivots, zero fill)
void ilu0_pivots(int batch, int n, cudaStream_t s, const SliceState* st, const float* wtv, const float* wtv2,
                 float* ia);

// In the PCG-step kernels below, `x` is the vector that receives alpha d: the
// solver passes the outer step's update accumulator dx (added to the iterate
// once per outer step by outer_apply).
enum IluMode { ILU_INIT = 0, ILU_STEP = 1, ILU_LAST = 2, ILU_PER_SLICE = -1 };
// shape: shared-memory ring, 10 * rows per stage + stages (0: chosen from n and batch)
// fuse_scalars: the CTA finishes the PCG scalars itself from its sums (rho
// at ILU_INIT; rr, the residual test against pcg_tol, beta and rho at ILU_STEP)
// alpha_np > 0 (ILU_PER_SLICE): the CTA of a slice in PCG first forms alpha
// from the S apply's alpha_np partial sums of <d, S d> (pcg_alpha's work)
void ilu_step(int batch, int n, cudaStream_t s, SliceState* st, double* part, int mode,
              float2* x, const float2* d, float2* r, const float2* q, const float2* atb, float2* y,
              float2* z, const float* ia, const float* wtv, int shape, int fuse_scalars = 0,
              PcgSched ps = PcgSched{0.f, 0, 1 << 30, 0, 0}, int wait_test = 0, const float* wtv2 = nullptr,
              int alpha_np = 0);
// aniso: the ring stages also hold the second weight array of l1 TV
int ilu_default_shape(int n, int batch, bool aniso = false);
bool ilu_shape_fits(int n, int shape, bool aniso = false);

// AXPY_PER_SLICE (and ILU_PER_SLICE, SCALARS_PER_SLICE, mode < 0 of the row
// FFT): each slice's own phase picks the first residual (PH_BOUNDARY) or a
// PCG step (PH_PCG).
enum AxpyMode { AXPY_INIT = 0, AXPY_STEP = 1, AXPY_LAST = 2, AXPY_PER_SLICE = -1 };
// Residual update (INIT: r = A^H b - q; STEP: r -= alpha q, x += alpha d) with
// a diagonal preconditioner z = sdiag o r (sdiag null: z = r), partial
// Re<r, z> into SLOT_RZ and ||r||^2 into SLOT_RR (axpy_ctas parts).
void axpy_diag_step(int batch, int n, cudaStream_t s, const SliceState* st, double* part, int mode, float2* x,
                    const float2* d, float2* r, const float2* q, const float2* atb, const float* sdiag, float2* z);
// Jacobi scale of a wavelet-only system: ia = 1 / (abar + lam diag(Phi^T W Phi)).
void jacobi_wavelet_setup(int batch, int n, cudaStream_t s, const SliceState* st, const float* wdiag, float* ia);
void axpy_step(int batch, int n, cudaStream_t s, const SliceState* st, double* part, int mode,
               float2* x, const float2* d, float2* r, const float2* q, const float2* atb);
int axpy_ctas(int n);

void group_norms(int batch, int n, int n_groups, cudaStream_t s, const SliceState* st,
                 const int* gidx, const int* goff, int gsize, const float2* c, float* wg, float eps_unused);
void group_gather(int batch, int n, int n_groups, cudaStream_t s, const SliceState* st,
                  const int* inv_off, const int* inv_ids, const float* wg, float* w);
// Build the inverse map; returns via err (device int) 1 on bad index/offsets.
void group_inverse_build(int n, int n_groups, int gsize, cudaStream_t s, const int* gidx, const int* goff,
                         int* counts, int* inv_off, int* inv_ids, int* cursor, int* err);

void mask_popcount(int batch, int n, cudaStream_t s, const uint8_t* mask, int* counts);

// Partial sums of the regularisers of F_eps (one slot each, axpy_ctas parts):
// sum_j sqrt(|c_j|^2 + eps) (singleton groups) or sum_g sqrt(||c_g||^2 + eps),
// and sum_i sqrt(|D1 x|_i^2 + |D2 x|_i^2 + eps).  channels C > 1: the joint
// sums of each image in its first slice (the other slices' parts are 0).
void l21_sum(int batch, int n, cudaStream_t s, const float2* c, const int* gidx, const int* goff, int n_groups,
             int gsize, float eps, double* part, int slot, int channels = 1);
void tv_sum(int batch, int n, cudaStream_t s, const float2* x, float eps, double* part, int slot, int aniso,
            int channels = 1);

// PCG scalar updates (one thread per slice).  channels C > 1: the inner
// products are summed over the C consecutive slices of a multi-contrast
// image, whose slices then carry the same scalars (here, in outer_end and in
// state_init's ||A^H b||^2).
void pcg_alpha(int batch, cudaStream_t s, SliceState* st, const double* part, int nparts, int channels = 1);
enum ScalarsMode { SCALARS_INIT = 0, SCALARS_STEP = 1, SCALARS_PER_SLICE = -1 };
void pcg_scalars(int batch, cudaStream_t s, SliceState* st, const double* part, int nparts_rz, int nparts_rr,
                 int mode, const PcgSched& ps, int channels = 1);
// view = st with every slice not at the start of its outer step marked done
// (and the slices whose outer step is due move to PH_START)
void boundary_view(int batch, cudaStream_t s, SliceState* st, SliceState* view);
// x += dx (the outer step's accumulated update) with partial ||dx||^2 and
// ||x||^2 (before the update) for the relative change.
void outer_apply(int batch, int n, cudaStream_t s, const SliceState* st, float2* x, float2* dx,
                 double* part);
// plateau_after: first outer step at which kind 1 also stops on a plateau
void outer_end(int batch, cudaStream_t s, SliceState* st, const double* part, int nparts,
               float outer_tol, int tol_kind, float stall_tol, int plateau_after, int channels = 1);
// phase: PH_BOUNDARY for a solve (its first outer step is due), PH_START for
// the single operator applications (no outer step)
void state_init(int batch, cudaStream_t s, SliceState* st, const double* part, int nparts_rhs,
                const int* counts, int n, const float* lam, const float* lam_tv, float eps, int outer_max,
                int phase, int channels = 1);

}  // namespace firls
