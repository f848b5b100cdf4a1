// J = lambda^T A u over a CSR matrix without allocating anything.
//
// Who needs this: code that is not allowed to call cudaMalloc at the point where it wants
// the reduction, for example a solver running inside a memory pool it does not own, or a
// host callback that must not touch the allocator.  sfa_bilinear needs a mesh (which owns
// its scratch); this variant takes the CSR arrays directly and keeps its scratch, one
// partial sum per row, in a fixed array compiled into the library.
//
// The scratch array is shared by every call in the process and keeps the last call's
// contents.  Each call overwrites entries [0, n_rows) before reading them, so nothing has
// to be cleared first; calls that overlap on the GPU (different streams, or threads)
// write the same array and race.
#include <mutex>

#include "sfa_internal.cuh"

// Capacity of the scratch: one double per matrix row.
#define SFA_STATIC_SCRATCH_ROWS (1 << 20)

static __device__ __align__(256) double g_static_row_partials[SFA_STATIC_SCRATCH_ROWS];

namespace {

// Per-device address of the scratch array, looked up once per device with that device
// current (a host-side name of a __device__ variable is not a device address).  The cached
// address assumes the device's primary context lives until the process exits: after a
// cudaDeviceReset the array has a new context and the cached address is stale.
std::mutex g_static_mu;
double* g_static_ptr[128] = {nullptr};

template <typename R>
__global__ void k_row_partials(const int64_t* rowptr, const int32_t* colind, int64_t nrows, const R* values,
                               const double* lam, const double* u, double* partial) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < nrows; i += nw) {
    const int64_t a = rowptr[i], b = rowptr[i + 1];
    double s = 0.0;
    for (int64_t k = a + lane; k < b; k += 32) s += (double)values[k] * u[colind[k]];
    s = warp_sum(s);
    if (lane == 0) partial[i] = lam[i] * s;
  }
}

// Single block: fixed-order strided sums then a tree, so the result is deterministic.
__global__ void __launch_bounds__(1024) k_sum_partials(const double* partial, int64_t n, double* out) {
  __shared__ double sh[1024];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += partial[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

}  // namespace

namespace {
sfa_status static_fail(sfa_status st, const std::string& msg) {
  sfa_record_error("sfa_bilinear_static: " + msg);
  return st;
}
}  // namespace

extern "C" sfa_status sfa_bilinear_static(const int64_t* rowptr_dev, const int32_t* colind_dev, int64_t n_rows,
                                          sfa_precision prec, const void* values_dev, const double* lambda_dev,
                                          const double* u_dev, double* J_dev, void* stream) {
  if (!rowptr_dev || !colind_dev || !values_dev || !lambda_dev || !u_dev || !J_dev || n_rows < 0)
    return static_fail(SFA_ERR_INVALID_ARG, "null pointer or negative row count");
  if (!prec_valid(prec)) return static_fail(SFA_ERR_INVALID_ARG, "unknown precision");
  if (n_rows > SFA_STATIC_SCRATCH_ROWS)  // scratch holds one double per row
    return static_fail(SFA_ERR_INVALID_ARG, "n_rows exceeds the fixed scratch of 1048576 rows");
  // an error left pending by earlier, unrelated work on this thread is reported as such (and
  // not taken for a failure of the launches below)
  const cudaError_t pending = cudaPeekAtLastError();
  if (pending != cudaSuccess)
    return static_fail(SFA_ERR_CUDA, std::string("a CUDA error was pending before the call: ") +
                                         cudaGetErrorString(pending));
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 128) {
    cudaGetLastError();
    return static_fail(SFA_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  }
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_static_row_partials);
      if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return static_fail(SFA_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      }
      g_static_ptr[dev] = static_cast<double*>(p);
    }
    scratch = g_static_ptr[dev];
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (n_rows > 0) {
    if (prec == SFA_FP64)
      k_row_partials<double><<<1216, 256, 0, st>>>(rowptr_dev, colind_dev, n_rows, (const double*)values_dev,
                                                   lambda_dev, u_dev, scratch);
    else
      k_row_partials<float><<<1216, 256, 0, st>>>(rowptr_dev, colind_dev, n_rows, (const float*)values_dev,
                                                  lambda_dev, u_dev, scratch);
    SFA_LAUNCHED(1);
    if ((e = cudaGetLastError()) != cudaSuccess)
      return static_fail(SFA_ERR_CUDA, std::string("row partials launch: ") + cudaGetErrorString(e));
  }
  k_sum_partials<<<1, 1024, 0, st>>>(scratch, n_rows, J_dev);
  SFA_LAUNCHED(1);
  if ((e = cudaGetLastError()) != cudaSuccess)
    return static_fail(SFA_ERR_CUDA, std::string("sum launch: ") + cudaGetErrorString(e));
  return SFA_OK;
}
