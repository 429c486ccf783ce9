// A^H A d without any device allocation, for callers that cannot allocate.
//
// Some callers must not allocate device memory at all: code that runs
// inside another framework's memory pool or a real-time loop where
// cudaMalloc/cudaFree would synchronise the device or fragment a budgeted
// heap, and plug-ins that are handed only their input and output buffers.
// firls_apply_AHA_noalloc serves them: it runs the same kernels as
// firls_apply_AHA, but the FFT intermediate, the twiddle table, the
// per-slice state and the partial sums live in file-scope __device__ arrays
// of fixed size that every GPU loading this library holds until exit.
#include <cmath>
#include <mutex>

#include "firls.h"
#include "launch.h"

using namespace firls;

namespace {

constexpr int kMaxDevices = 64;
constexpr int kMaxTw = 512;

// Fixed scratch: 8,792,064 bytes (8.4 MiB) per device.
__device__ __align__(256) float2 g_na_t[FIRLS_NOALLOC_MAX_ELEMS];
__device__ __align__(256) float2 g_na_tw[kMaxTw];
__device__ __align__(256) SliceState g_na_st[FIRLS_NOALLOC_MAX_BATCH];
__device__ __align__(256) double g_na_part[FIRLS_NOALLOC_MAX_BATCH * NSLOT * MAXPART];

struct NaPtrs {
  float2* t = nullptr;
  float2* tw = nullptr;
  SliceState* st = nullptr;
  double* part = nullptr;
  int tw_n = 0;  // size whose twiddles are in g_na_tw
};
NaPtrs g_ptrs[kMaxDevices];
bool g_ready[kMaxDevices];
// Guards g_ptrs / g_ready and the twiddle-table bookkeeping against host
// threads that make their first call (or change n) at the same time.
std::mutex g_mu;

__global__ void k_na_state(int B, SliceState* st) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= B) return;
  SliceState v{};
  v.active = 1;
  v.eps = 1e-10f;
  st[s] = v;
}

// Device addresses of the scratch arrays for the current device (taken once
// per device; the array names are host-side stand-ins, not addresses).
firls_status setup(int dev, NaPtrs** out) {
  if (dev < 0 || dev >= kMaxDevices) return FIRLS_E_INVALID_ARG;
  if (!g_ready[dev]) {
    NaPtrs p;
    if (cudaGetSymbolAddress((void**)&p.t, g_na_t) != cudaSuccess) return FIRLS_E_CUDA;
    if (cudaGetSymbolAddress((void**)&p.tw, g_na_tw) != cudaSuccess) return FIRLS_E_CUDA;
    if (cudaGetSymbolAddress((void**)&p.st, g_na_st) != cudaSuccess) return FIRLS_E_CUDA;
    if (cudaGetSymbolAddress((void**)&p.part, g_na_part) != cudaSuccess) return FIRLS_E_CUDA;
    p.tw_n = 0;
    g_ptrs[dev] = p;
    g_ready[dev] = true;
  }
  *out = &g_ptrs[dev];
  return FIRLS_OK;
}

}  // namespace

extern "C" firls_status firls_apply_AHA_noalloc(int n, int batch, const uint8_t* mask, const void* d, void* q,
                                                void* cuda_stream) {
  if (!mask || !d || !q) return FIRLS_E_INVALID_ARG;
  if (!fft_size_supported(n) || n > kMaxTw) return FIRLS_E_SHAPE;
  if (batch < 1 || batch > FIRLS_NOALLOC_MAX_BATCH || (size_t)batch * n * n > (size_t)FIRLS_NOALLOC_MAX_ELEMS)
    return FIRLS_E_SHAPE;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FIRLS_E_CUDA;
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  NaPtrs p;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    NaPtrs* pp = nullptr;
    const firls_status s0 = setup(dev, &pp);
    if (s0 != FIRLS_OK) return s0;
    if (pp->tw_n != n) {  // twiddles exp(-2 pi i j / n), written into the fixed table
      float2 tw[kMaxTw];
      for (int j = 0; j < n; ++j) {
        const double ang = -2.0 * 3.14159265358979323846 * (double)j / (double)n;
        tw[j] = make_float2((float)std::cos(ang), (float)std::sin(ang));
      }
      pp->tw_n = 0;
      if (cudaMemcpyAsync(pp->tw, tw, sizeof(float2) * n, cudaMemcpyHostToDevice, stream) != cudaSuccess ||
          cudaStreamSynchronize(stream) != cudaSuccess) {  // tw is a stack buffer
        g_ready[dev] = false;
        return FIRLS_E_CUDA;
      }
      pp->tw_n = n;
    }
    p = *pp;
  }
  fft_prepare(n);
  // the state of every slice is rewritten: lambdas 0, running
  k_na_state<<<(batch + 127) / 128, 128, 0, stream>>>(batch, p.st);
  FftArgs a;
  a.batch = batch;
  a.stream = stream;
  a.tw = p.tw;
  a.st = p.st;
  a.part = p.part;
  a.d = const_cast<float2*>(static_cast<const float2*>(d));
  a.t = p.t;
  a.mode = 2;
  fft_row_fwd(n, a);
  a.mask = mask;
  fft_col_mask(n, a);
  a.q = static_cast<float2*>(q);
  fft_row_inv(n, a);
  if (cudaGetLastError() != cudaSuccess) {
    // set up again at the next call (the table may not hold n's twiddles)
    std::lock_guard<std::mutex> lock(g_mu);
    g_ready[dev] = false;
    return FIRLS_E_CUDA;
  }
  return FIRLS_OK;
}
