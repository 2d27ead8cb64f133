// Periodic discrete convolution J * rho of Eq. (discrete_convolution),
// evaluated with a hand-written shared-memory radix-2 FFT (float64).
//
//   (J * rho)_p = h^d sum_q J_q rho_{p-q}  =  IDFT( DFT(h^d J) . DFT(rho) ) / N
//
// J is the kernel of Sec. 6, sampled with the minimum-image distance on the
// periodic box; J_e = -J where J <= 0, and c_e = (J_e * 1) = h^d sum J_e
// (Lemma 5.2).  Both are computed once per fm_create; DFT(h^d J)/N is stored.
//
// The transform of a d-dimensional array is d passes of 1-D transforms:
//  * along x (contiguous): one block per line, the line in shared memory;
//  * along y / z (strided): one block per tile of TC consecutive x-columns,
//    loaded row by row so that global accesses stay coalesced.
// Each 1-D transform is an iterative radix-2 decimation-in-time butterfly
// network on a bit-reversed load, with twiddles exp(-2 pi i k/n) from a table
// built once with sincospi.
#include <cuda_runtime.h>
#include <cmath>

#include "fm_state.h"

namespace fm {

constexpr int FT = 256;

__global__ void k_twiddles(double2* tw, int n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n / 2) return;
  double sv, cv;
  sincospi(2.0 * (double)k / (double)n, &sv, &cv);
  tw[k] = make_double2(cv, -sv);
}

// work = (J, 0); partial sums of J_e.
__global__ void k_sample_J(double2* work, Geo G, double h, double nu, double* partials) {
  double acc = 0.0;
  const double pi2 = M_PI * M_PI;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < G.N; idx += gridDim.x * blockDim.x) {
    const int i = idx % G.nx;
    const int t = idx / G.nx;
    const int j = t % G.ny;
    const int k = t / G.ny;
    const double dx = h * (double)min(i, G.nx - i);
    const double dy = h * (double)min(j, G.ny - j);
    const double dz = h * (double)min(k, G.nz - k);
    const double r2 = dx * dx + dy * dy + (G.nz > 1 ? dz * dz : 0.0);
    const double J = sqrt(2.0) * exp(-pi2 * r2 / (2.0 * nu * nu)) - exp(-pi2 * r2 / (4.0 * nu * nu));
    work[idx] = make_double2(J, 0.0);
    if (J <= 0.0) acc += -J;
  }
  __shared__ double sm[FT / 32];
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < FT / 32; ++w) s += sm[w];
    partials[blockIdx.x] = s;
  }
}

__global__ void k_sum_partials(const double* partials, int nb, double scale, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += partials[b];
    out[0] = s * scale;
  }
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// In-place radix-2 DIT on `ncols` lines of length n stored at a[c * n + j],
// already in bit-reversed order.  All threads of the block cooperate.
__device__ void butterflies(double2* a, int n, int ncols, const double2* tw, bool inverse) {
  const int half = n >> 1;
  const int total = half * ncols;
  for (int m = 2; m <= n; m <<= 1) {
    const int hm = m >> 1;
    const int tstride = n / m;
    for (int b = threadIdx.x; b < total; b += blockDim.x) {
      const int c = b / half;
      const int bb = b - c * half;
      const int grp = bb / hm;
      const int kk = bb - grp * hm;
      const int i0 = c * n + grp * m + kk;
      const int i1 = i0 + hm;
      double2 w = tw[kk * tstride];
      if (inverse) w.y = -w.y;
      const double2 t = cmul(w, a[i1]);
      const double2 u = a[i0];
      a[i0] = make_double2(u.x + t.x, u.y + t.y);
      a[i1] = make_double2(u.x - t.x, u.y - t.y);
    }
    __syncthreads();
  }
}

// 1-D transforms along x: one block per line.
__global__ void k_fft_x(double2* data, int n, int logn, const double2* tw, int inverse) {
  extern __shared__ double2 sh[];
  double2* line = data + (size_t)blockIdx.x * n;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const int rj = (int)(__brev((unsigned)j) >> (32 - logn));
    sh[rj] = line[j];
  }
  __syncthreads();
  butterflies(sh, n, 1, tw, inverse != 0);
  for (int j = threadIdx.x; j < n; j += blockDim.x) line[j] = sh[j];
}

// 1-D transforms along a strided axis of length n (stride `stride` elements):
// block (blockIdx.x, blockIdx.y) handles TC consecutive x-columns starting at
// x0 = blockIdx.x * TC of the outer slice blockIdx.y (offset ostride).
__global__ void k_fft_strided(double2* data, int n, int logn, int stride, int ostride, int TC,
                              const double2* tw, int inverse) {
  extern __shared__ double2 sh[];
  double2* base = data + (size_t)blockIdx.y * ostride + (size_t)blockIdx.x * TC;
  const int total = n * TC;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int j = t / TC;
    const int c = t - j * TC;
    const int rj = (int)(__brev((unsigned)j) >> (32 - logn));
    sh[c * n + rj] = base[(size_t)j * stride + c];
  }
  __syncthreads();
  butterflies(sh, n, TC, tw, inverse != 0);
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int j = t / TC;
    const int c = t - j * TC;
    base[(size_t)j * stride + c] = sh[c * n + j];
  }
}

__global__ void k_load_real(const double* rho, double2* w, int N) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) w[i] = make_double2(rho[i], 0.0);
}

__global__ void k_cmul_inplace(double2* w, const double2* Jh, int N) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) w[i] = cmul(w[i], Jh[i]);
}

__global__ void k_store_real(const double2* w, double* out, int N) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) out[i] = w[i].x;
}

__global__ void k_scale(double2* w, int N, double s) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) w[i] = make_double2(w[i].x * s, w[i].y * s);
}

static int ilog2(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}

static fm_state* g_cur = nullptr;  // state whose launches are being counted

static bool launch_ok() {
  if (g_cur) ++g_cur->launches;
  if (cudaPeekAtLastError() != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return true;
}

// Forward (inverse = 0) or unnormalised inverse transform of st->fft.work.
static int fft_all(fm_state* st, int inverse) {
  const Geo G = st->lv[0].g;
  cudaStream_t s = st->stream;
  const int ns[3] = {G.nx, G.ny, G.nz};
  // x
  {
    const int n = G.nx;
    const size_t smem = (size_t)n * sizeof(double2);
    const int thr = n / 2 < FT ? (n / 2 < 32 ? 32 : n / 2) : FT;
    k_fft_x<<<G.ny * G.nz, thr, smem, s>>>(st->fft.work, n, ilog2(n), st->fft.tw[0], inverse);
    if (!launch_ok()) return FM_ECUDA;
  }
  for (int ax = 1; ax < st->dim; ++ax) {
    const int n = ns[ax];
    const int stride = ax == 1 ? G.nx : G.nx * G.ny;
    const int outer = ax == 1 ? G.nz : G.ny;
    const int ostride = ax == 1 ? G.nx * G.ny : G.nx;
    // TC columns per block: as many as keep at least two blocks per SM (one
    // column per block when the lines are too few), at most 16 and 64 KB of
    // shared memory; a power of two, so it divides nx
    int TC = 16;
    while (TC > 1 && ((G.nx / TC) * outer < 2 * st->sms || (size_t)n * TC * sizeof(double2) > 65536)) TC >>= 1;
    if (TC > G.nx) TC = G.nx;
    const size_t smem = (size_t)n * TC * sizeof(double2);
    int thr = n * TC / 2;  // one butterfly per thread and stage
    thr = thr > FT ? FT : (thr < 32 ? 32 : thr);
    dim3 grid(G.nx / TC, outer);
    k_fft_strided<<<grid, thr, smem, s>>>(st->fft.work, n, ilog2(n), stride, ostride, TC, st->fft.tw[ax],
                                          inverse);
    if (!launch_ok()) return FM_ECUDA;
  }
  return FM_OK;
}

int fft_init(fm_state* st) {
  g_cur = st;
  const Geo G = st->lv[0].g;
  const double h = st->lv[0].h;
  cudaStream_t s = st->stream;
  const int ns[3] = {G.nx, G.ny, G.nz};
  for (int d = 0; d < st->dim; ++d) {
    const int n = ns[d];
    k_twiddles<<<(n / 2 + FT - 1) / FT + 1, FT, 0, s>>>(st->fft.tw[d], n);
    if (!launch_ok()) return FM_ECUDA;
  }
  // allow up to 64 KB of dynamic shared memory per transform block
  if (cudaFuncSetAttribute(k_fft_x, cudaFuncAttributeMaxDynamicSharedMemorySize, 65536) != cudaSuccess ||
      cudaFuncSetAttribute(k_fft_strided, cudaFuncAttributeMaxDynamicSharedMemorySize, 65536) != cudaSuccess) {
    cudaGetLastError();
    return FM_ECUDA;
  }
  k_sample_J<<<st->nblk, FT, 0, s>>>(st->fft.work, G, h, st->fn.nu, st->partials);
  if (!launch_ok()) return FM_ECUDA;
  const double w = st->dim == 3 ? h * h * h : h * h;
  k_sum_partials<<<1, 32, 0, s>>>(st->partials, st->nblk, w, st->dscal + 24);
  if (!launch_ok()) return FM_ECUDA;
  int rc = fft_all(st, 0);
  if (rc) return rc;
  // Jhat = DFT(h^d J) / N
  k_scale<<<(G.N + FT - 1) / FT, FT, 0, s>>>(st->fft.work, G.N, w / (double)G.N);
  if (!launch_ok()) return FM_ECUDA;
  if (cudaMemcpyAsync(st->fft.Jhat, st->fft.work, (size_t)G.N * sizeof(double2), cudaMemcpyDeviceToDevice, s) !=
          cudaSuccess ||
      cudaMemcpyAsync(st->hscal + 24, st->dscal + 24, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return FM_ECUDA;
  }
  st->ce = st->hscal[24];
  return FM_OK;
}

int fft_convolve(fm_state* st, const double* rho, double* out) {
  g_cur = st;
  const Geo G = st->lv[0].g;
  cudaStream_t s = st->stream;
  const int nb = (G.N + FT - 1) / FT;
  k_load_real<<<nb, FT, 0, s>>>(rho, st->fft.work, G.N);
  if (!launch_ok()) return FM_ECUDA;
  int rc = fft_all(st, 0);
  if (rc) return rc;
  k_cmul_inplace<<<nb, FT, 0, s>>>(st->fft.work, st->fft.Jhat, G.N);
  if (!launch_ok()) return FM_ECUDA;
  rc = fft_all(st, 1);
  if (rc) return rc;
  k_store_real<<<nb, FT, 0, s>>>(st->fft.work, out, G.N);
  if (!launch_ok()) return FM_ECUDA;
  return FM_OK;
}

}  // namespace fm
