// fm_mass_noalloc: the mass (rho || 1) = h^d sum rho of a caller-owned
// float64 device array, computed without allocating any device memory.
//
// Who needs this: callers that cannot call cudaMalloc -- for example a host
// application whose device memory is entirely reserved by its own allocator,
// or a time-critical loop in which the implicit device synchronisation of
// cudaMalloc/cudaFree is not acceptable.  fm_mass needs an fm_state, whose
// fm_create allocates; this entry point needs none.
//
// The reduction scratch (one float64 partial sum per thread block) lives in a
// file-scope __device__ array of FM_NOALLOC_MAX_BLOCKS doubles (32 KiB), which
// every GPU that loads libfm holds until the process exits.  Every call shares
// it and it keeps the last call's contents; each call writes every slot it
// later reads (stream order), so nothing has to start at zero.  Calls whose
// work overlaps on the GPU (different streams, no ordering) race on it.
//
// Host code cannot use the array's name as a device address (there it names a
// host-side stand-in), so the device address is looked up with
// cudaGetSymbolAddress once per device, on the first call made while that
// device is current, and passed to the kernels.  Make that first call before
// any stream capture.
#include <cuda_runtime.h>

#include "../../include/fm.h"

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_PER_THREAD = 4;
constexpr int NA_MAX_BLOCKS = 4096;
constexpr int NA_MAX_DEVICES = 64;

static __device__ __align__(256) double g_noalloc_partials[NA_MAX_BLOCKS];

static double* g_partials_addr[NA_MAX_DEVICES] = {nullptr};

// Block b sums the points [b * 1024, (b + 1) * 1024) in a fixed order and
// writes its partial sum to partials[b].
__global__ void __launch_bounds__(NA_THREADS) k_mass_partials_na(const double* rho, long long n,
                                                                 double* partials) {
  double acc = 0.0;
  const long long base = (long long)blockIdx.x * NA_THREADS * NA_PER_THREAD + threadIdx.x;
#pragma unroll
  for (int q = 0; q < NA_PER_THREAD; ++q) {
    const long long i = base + (long long)q * NA_THREADS;
    if (i < n) acc += rho[i];
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  __shared__ double sm[NA_THREADS / 32];
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < NA_THREADS / 32; ++w) s += sm[w];
    partials[blockIdx.x] = s;
  }
}

// out[0] = w * sum of the first nblk partials (fixed order).
__global__ void __launch_bounds__(NA_THREADS) k_mass_final_na(const double* partials, int nblk, double w,
                                                              double* out) {
  double acc = 0.0;
  for (int b = threadIdx.x; b < nblk; b += NA_THREADS) acc += partials[b];
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  __shared__ double sm[NA_THREADS / 32];
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < NA_THREADS / 32; ++k) s += sm[k];
    out[0] = w * s;
  }
}

}  // namespace

extern "C" int fm_mass_noalloc(const double* rho, int dim, const int* n, double h, double* out,
                               void* stream) {
  if (!rho || !n || !out || (dim != 2 && dim != 3) || !(h > 0.0)) return FM_EINVAL;
  long long npts = 1;
  for (int d = 0; d < dim; ++d) {
    if (n[d] < 1 || n[d] > FM_NOALLOC_MAX_POINTS) return FM_EINVAL;
    npts *= n[d];  // at most FM_NOALLOC_MAX_POINTS^2 < 2^63: no overflow
    if (npts > FM_NOALLOC_MAX_POINTS) return FM_EINVAL;  // checked before the next factor
  }
  const long long per_block = (long long)NA_THREADS * NA_PER_THREAD;
  const long long nblk = (npts + per_block - 1) / per_block;
  if (nblk > NA_MAX_BLOCKS) return FM_EINVAL;  // more than FM_NOALLOC_MAX_POINTS points
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return FM_ECUDA;
  }
  if (dev < 0 || dev >= NA_MAX_DEVICES) return FM_EINVAL;
  if (!g_partials_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_partials) != cudaSuccess || !p) {
      cudaGetLastError();
      return FM_ECUDA;
    }
    g_partials_addr[dev] = (double*)p;
  }
  cudaStream_t s = (cudaStream_t)stream;
  double w = h * h;
  if (dim == 3) w *= h;
  k_mass_partials_na<<<(int)nblk, NA_THREADS, 0, s>>>(rho, npts, g_partials_addr[dev]);
  k_mass_final_na<<<1, NA_THREADS, 0, s>>>(g_partials_addr[dev], (int)nblk, w, out);
  if (cudaPeekAtLastError() != cudaSuccess) {
    cudaGetLastError();
    return FM_ECUDA;
  }
  return FM_OK;
}
