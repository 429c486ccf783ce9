// Shared device-side definitions of the FIRLS CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define FI __device__ __forceinline__

namespace firls {

// Outer steps over which the contraction of the outer iteration is measured
// by the distance-to-the-limit stop (outer_tol_kind 1).
constexpr int MU_WINDOW = 24;
// Consecutive outer steps at or below the stall tolerance that stop a slice.
constexpr int STALL_STEPS = 4;

// Where a slice is in its own outer step.  Every slice advances on its own:
// one launch sequence (a macro step) does a PCG step for the slices in
// PH_PCG and the outer-step transition for the others.
//   PH_BOUNDARY: an outer step is due: the next macro step with a boundary
//                stage updates the weights and P from x^k.
//   PH_START:    weights and P are ready: S x^k, the first residual
//                r_0 = A^H b - S x^k, z_0 and rho.
//   PH_PCG:      PCG step pcg_j + 1 of the outer step.
//   PH_END:      the outer step's PCG has stopped; the next boundary stage
//                adds its update to x, measures the relative change, applies
//                the stopping rules and, if the slice goes on, sets
//                PH_BOUNDARY for its next outer step.
// Boundary stages (weights, transitions) may run only every few macro
// steps; slices in PH_BOUNDARY or PH_END wait for the next one.
enum { PH_BOUNDARY = 0, PH_PCG = 1, PH_END = 2, PH_START = 3 };

// Per-slice PCG / outer-loop state, FP64 scalars (the only FP64 steps:
// inner products, alpha, beta, rho, residual norms, relative change).
struct SliceState {
  double rho;        // Re<r, z> of the current PCG step
  double alpha;      // rho / Re<d, S d>
  double beta;       // rho_new / rho
  double rhs2;       // ||A^H b||^2
  double rr;         // ||r||^2 after the last update
  double rr0;        // ||r_0||^2, the first residual of the current outer step
  double relchg;     // ||x^{k+1} - x^k|| / ||x^k|| of the last outer step
  int active;        // PCG running in this outer step
  int done;          // outer loop stopped (outer_tol reached)
  int breakdown;     // PCG broke down at least once
  int pcg_steps;     // PCG steps taken (all outer steps)
  int outer_done;    // outer steps taken
  int fault;         // a bounded device wait ran out (results invalid)
  float lam;         // wavelet lambda
  float lam_tv;      // TV lambda
  float abar;        // mean(diag(A^H A)) = popcount / N
  float eps;         // smoothing eps
  int stall;         // consecutive outer steps with relchg <= the stall tolerance
  int phase;         // PH_*: where the slice is in its current outer step
  int pcg_j;         // PCG steps taken in the current outer step
  int outer_max;     // outer steps after which the slice stops
  float hist[MU_WINDOW];  // relchg of the last MU_WINDOW outer steps (ring, by outer_done)
};

// Partial-sum slots (double part[B][NSLOT][MAXPART]).
enum { SLOT_DQ = 0, SLOT_RZ = 1, SLOT_RR = 2, SLOT_RHS = 3, SLOT_DX = 4, SLOT_XX = 5, NSLOT = 6 };
constexpr int MAXPART = 128;

FI float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
FI float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
FI float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
FI float2 cfma(float s, float2 a, float2 b) { return make_float2(fmaf(s, a.x, b.x), fmaf(s, a.y, b.y)); }
FI float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
FI float cabs2(float2 a) { return fmaf(a.x, a.x, a.y * a.y); }
FI float rdot2(float2 a, float2 b) { return fmaf(a.x, b.x, a.y * b.y); }

FI bool slice_running(const SliceState* st, int s) { return st[s].active && !st[s].done; }
FI bool slice_in_pcg(const SliceState* st, int s) { return slice_running(st, s) && st[s].phase == PH_PCG; }
// A slice that takes part in this macro step's S apply and PCG update.
FI bool slice_working(int phase) { return phase == PH_START || phase == PH_PCG; }

// PCG scalar updates of one slice (FP64), shared by the scalar kernels and
// the kernels that finish them in place.
// alpha = rho / <d, S d>; a non-positive or non-finite <d, S d> is a breakdown.
FI void pcg_alpha_from(SliceState* v, double dq) {
  const double rho = v->rho;
  if (rho == 0.0) {  // exact solution reached: nothing left to do in this outer step
    v->alpha = 0.0;
    v->phase = PH_END;
    return;
  }
  if (!(dq > 0.0) || !isfinite(dq) || !isfinite(rho)) {  // breakdown: the slice stops, x keeps its last value
    v->active = 0;
    v->done = 1;
    v->breakdown = 1;
    return;
  }
  v->alpha = rho / dq;
  v->pcg_steps += 1;
}
// First residual: rho = Re<r, z>, rr = ||r||^2, no previous direction; the
// slice's PCG steps begin.
FI void pcg_rho_init_from(SliceState* v, double rz, double rr) {
  v->rho = rz;
  v->rr = rr;
  v->rr0 = rr;
  v->beta = 0.0;
  v->phase = PH_PCG;
  v->pcg_j = 0;
}
// Inner-solve schedule of the PCG steps: stop at ||r|| <= tol ||A^H b|| (rel
// = 0) or tol ||r_0|| (rel = 1), or after J steps per outer step, J_late
// from outer step k_late on (J_late <= 0: always J).
struct PcgSched {
  float tol;
  int rel, J, J_late, k_late;
  FI int cap(const SliceState* v) const { return (J_late > 0 && v->outer_done >= k_late) ? J_late : J; }
};
// After the residual update of PCG step pcg_j + 1: the outer step's PCG ends
// on ||r|| <= tol ||A^H b|| (or, with rel, ||r|| <= tol ||r_0||: the forcing
// term of an inexact inner solve) or after the schedule's steps for this outer
// step; otherwise beta = rho_new / rho.
FI void pcg_beta_from(SliceState* v, double rz, double rr, const PcgSched& ps) {
  v->rr = rr;
  v->pcg_j += 1;
  if ((ps.tol > 0.f && sqrt(rr) <= (double)ps.tol * sqrt(ps.rel ? v->rr0 : v->rhs2)) || v->pcg_j >= ps.cap(v)) {
    v->phase = PH_END;
    return;
  }
  v->beta = rz / v->rho;
  v->rho = rz;
}

// Block-wide FP64 sum; result valid in thread 0.  `red` holds >= 32 doubles.
FI double block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < nw; ++i) s += red[i];
  return s;
}

}  // namespace firls
