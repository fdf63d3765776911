// ce_noalloc.cu -- ce_moments_noalloc: per-field mean and variance of field
// arrays the caller already holds in device memory, computed without any
// device allocation by the library.
//
// Scratch lives in one file-scope __device__ array (g_moments_scratch, 64 KiB)
// that every GPU loading the library keeps until the process exits.  Host code
// must not hand the array's name to a kernel (on the host it is only a
// stand-in for the symbol), so the device address is fetched once per device
// with cudaGetSymbolAddress and passed to the kernels explicitly.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>

#include "ce_internal.h"
#include "clusterlat.h"

namespace {

constexpr int kBlocks = 1024;          // blocks of the partial-sum pass (fixed)
constexpr int kThreads = 256;
constexpr int kMaxFields = 4;
constexpr int kMaxDevices = 64;
constexpr int64_t kMaxSites = int64_t(1) << 34;

// Partial sums, [block][field][2]: sum (f - f0) and sum (f - f0)^2 with
// f0 = the field's first value.  Every call overwrites the slots it reads, so
// nothing here has to start at zero.
static __device__ __align__(256) double g_moments_scratch[kBlocks * kMaxFields * 2];

std::mutex g_setup_mutex;
double* g_scratch_ptr[kMaxDevices] = {};

int noalloc_fail(int code, const std::string& msg) {
  ce::set_last_error(msg);
  return code;
}

// Device address of the scratch array for the current device (set-up once per device).
int scratch_for_device(int dev, double** out) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_moments_scratch);
    if (e != cudaSuccess || !p)
      return noalloc_fail(CE_ECUDA, std::string("ce_moments_noalloc: cudaGetSymbolAddress failed: ") +
                                        cudaGetErrorString(e));
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return CE_OK;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_moments_partial(const T* __restrict__ f, int64_t n, int nf,
                                                               double* __restrict__ scratch) {
  __shared__ double red[kThreads / 32][2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = 0; i < nf; ++i) {
    const T* fi = f + (int64_t)i * n;
    const double shift = (double)fi[0];
    double s1 = 0.0, s2 = 0.0;
    for (int64_t k = (int64_t)blockIdx.x * kThreads + threadIdx.x; k < n; k += (int64_t)kBlocks * kThreads) {
      const double d = (double)fi[k] - shift;
      s1 += d;
      s2 += d * d;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s1 += __shfl_down_sync(0xffffffffu, s1, o);
      s2 += __shfl_down_sync(0xffffffffu, s2, o);
    }
    if (lane == 0) {
      red[warp][0] = s1;
      red[warp][1] = s2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double a = 0.0, b = 0.0;
      for (int w = 0; w < kThreads / 32; ++w) {
        a += red[w][0];
        b += red[w][1];
      }
      scratch[((int64_t)blockIdx.x * kMaxFields + i) * 2] = a;
      scratch[((int64_t)blockIdx.x * kMaxFields + i) * 2 + 1] = b;
    }
    __syncthreads();
  }
}

template <typename T>
__global__ void k_moments_final(const T* __restrict__ f, int64_t n, int nf, const double* __restrict__ scratch,
                                double* __restrict__ mean, double* __restrict__ var) {
  const int i = threadIdx.x;
  if (i >= nf) return;
  double a = 0.0, b = 0.0;
  for (int blk = 0; blk < kBlocks; ++blk) {  // fixed order
    a += scratch[((int64_t)blk * kMaxFields + i) * 2];
    b += scratch[((int64_t)blk * kMaxFields + i) * 2 + 1];
  }
  const double m1 = a / (double)n, m2 = b / (double)n;
  mean[i] = (double)f[(int64_t)i * n] + m1;
  var[i] = m2 - m1 * m1;
}

}  // namespace

extern "C" int ce_moments_noalloc(const void* f, int precision, int64_t n, int nfields, void* stream,
                                  double* mean, double* var) {
  ce::set_last_error("");
  if (!f || !mean || !var) return noalloc_fail(CE_EINVAL, "ce_moments_noalloc: NULL pointer");
  if (precision != CE_F32 && precision != CE_F64)
    return noalloc_fail(CE_EINVAL, "ce_moments_noalloc: precision must be CE_F32 or CE_F64");
  if (nfields < 1 || nfields > kMaxFields)
    return noalloc_fail(CE_EINVAL, "ce_moments_noalloc: nfields must be 1..4 (the static scratch holds 4 fields)");
  if (n < 1 || n > kMaxSites)
    return noalloc_fail(CE_EINVAL, "ce_moments_noalloc: n must be 1..2^34 sites per field");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return noalloc_fail(CE_ECUDA, std::string("ce_moments_noalloc: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(CE_EINVAL, "ce_moments_noalloc: device index out of range");
  double* scratch = nullptr;
  int rc = scratch_for_device(dev, &scratch);
  if (rc != CE_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (precision == CE_F32) {
    k_moments_partial<float><<<kBlocks, kThreads, 0, st>>>(static_cast<const float*>(f), n, nfields, scratch);
    k_moments_final<float><<<1, 32, 0, st>>>(static_cast<const float*>(f), n, nfields, scratch, mean, var);
  } else {
    k_moments_partial<double><<<kBlocks, kThreads, 0, st>>>(static_cast<const double*>(f), n, nfields, scratch);
    k_moments_final<double><<<1, 32, 0, st>>>(static_cast<const double*>(f), n, nfields, scratch, mean, var);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return noalloc_fail(CE_ECUDA, std::string("ce_moments_noalloc: launch: ") + cudaGetErrorString(e));
  return CE_OK;
}
