// Periodic discrete convolution J * rho of Eq. (discrete_convolution),
// evaluated with a hand-written shared-memory radix-2 FFT (float64).
//
//   (J * rho)_p = h^d sum_q J_q rho_{p-q}  =  IDFT( DFT(h^d J) . DFT(rho) ) / N
//
// J is the kernel of Sec. 6, sampled with the minimum-image distance on the
// periodic box; J_e = -J where J <= 0, and c_e = (J_e * 1) = h^d sum J_e
// (Lemma 5.2).  Both are computed once per fm_create; DFT(h^d J)/N is stored.
//
// A real density is transformed in the real-input form (convolve_real): the
// x transforms of its real rows as complex transforms of half length and the
// remaining passes and the product on the half spectrum.  The complex form
// (all passes on the full complex array) serves the kernel's transform at
// fm_create, grids narrower than 8 points, and FM_FFT_COMPLEX=1 (measurement).
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
#include <cstdlib>

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

// Butterflies of length n with the twiddle table of length n * tmul (a
// table for a longer transform serves a shorter one at a multiple of its
// stride).
__device__ void butterflies_t(double2* a, int n, const double2* tw, bool inverse, int tmul) {
  const int half = n >> 1;
  for (int m = 2; m <= n; m <<= 1) {
    const int hm = m >> 1;
    const int tstride = (n / m) * tmul;
    for (int b = threadIdx.x; b < half; b += blockDim.x) {
      const int grp = b / hm;
      const int kk = b - grp * hm;
      const int i0 = grp * m + kk;
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

// Real-input transform along x, one block per row of n reals (n = nx >= 8):
// the row as n/2 complex values z_m = rho_2m + i rho_2m+1, an FFT of length
// n/2 (Z), then the half spectrum X_k = E_k + W^k O_k, k < n/2, with
// E_k = (Z_k + conj Z_{n/2-k}) / 2, O_k = (Z_k - conj Z_{n/2-k}) / 2i and
// W = exp(-2 pi i / n); X_0 and X_{n/2} are real and are stored together as
// H_0 = (X_0, X_{n/2}).  Output rows of n/2 complex values.
__global__ void k_rfft_x(const double* rho, double2* H, int n, int logh, const double2* tw) {
  extern __shared__ double2 sh[];
  const int h = n >> 1;
  const double* row = rho + (size_t)blockIdx.x * n;
  for (int m = threadIdx.x; m < h; m += blockDim.x) {
    const int rm = (int)(__brev((unsigned)m) >> (32 - logh));
    sh[rm] = make_double2(row[2 * m], row[2 * m + 1]);
  }
  __syncthreads();
  butterflies_t(sh, h, tw, false, 2);
  double2* out = H + (size_t)blockIdx.x * h;
  for (int k = threadIdx.x; k < h; k += blockDim.x) {
    const double2 z = sh[k];
    if (k == 0) {
      out[0] = make_double2(z.x + z.y, z.x - z.y);
    } else {
      const double2 zc = sh[h - k];  // conj taken below
      const double2 E = make_double2(0.5 * (z.x + zc.x), 0.5 * (z.y - zc.y));
      const double2 O = make_double2(0.5 * (z.y + zc.y), -0.5 * (z.x - zc.x));
      const double2 wo = cmul(tw[k], O);
      out[k] = make_double2(E.x + wo.x, E.y + wo.y);
    }
  }
}

// Inverse of k_rfft_x times n (unnormalised, as the complex inverse): from
// the half spectrum, Z_k = E'_k + i O'_k with E'_k = X_k + conj X_{n/2-k} and
// O'_k = W^-k (X_k - conj X_{n/2-k}), an inverse FFT of length n/2, and
// rho_2m = Re z_m, rho_2m+1 = Im z_m.
__global__ void k_irfft_x(const double2* H, double* out, int n, int logh, const double2* tw) {
  extern __shared__ double2 sh[];
  const int h = n >> 1;
  const double2* in = H + (size_t)blockIdx.x * h;
  for (int k = threadIdx.x; k < h; k += blockDim.x) {
    double2 Z;
    if (k == 0) {
      const double2 p = in[0];  // (X_0, X_{n/2})
      Z = make_double2(p.x + p.y, p.x - p.y);
    } else {
      const double2 x = in[k], xc = in[h - k];
      const double2 E = make_double2(x.x + xc.x, x.y - xc.y);
      const double2 D = make_double2(x.x - xc.x, x.y + xc.y);
      const double2 wc = make_double2(tw[k].x, -tw[k].y);
      const double2 O = cmul(wc, D);
      Z = make_double2(E.x - O.y, E.y + O.x);
    }
    const int rk = (int)(__brev((unsigned)k) >> (32 - logh));
    sh[rk] = Z;
  }
  __syncthreads();
  butterflies_t(sh, h, tw, true, 2);
  double* row = out + (size_t)blockIdx.x * n;
  for (int m = threadIdx.x; m < h; m += blockDim.x) {
    row[2 * m] = sh[m].x;
    row[2 * m + 1] = sh[m].y;
  }
}

// Half spectrum times DFT(h^d J)/N, which is real (J is real and even on the
// periodic grid; Jr holds its real part at kx = 0 .. n/2, rows of n/2 + 1).
// Column kx = 0 holds C = X_0 + i X_{n/2} (two real sequences packed
// together): its transform P splits into A = (P(k) + conj P(-k)) / 2 and
// B = (P(k) - conj P(-k)) / 2i, each is multiplied by its own column of Jr,
// and Q = Jr_0 A + i Jr_{n/2} B is stored back.  A thread takes an index of
// that column and its mirror -k together (the lower of the two), so nothing
// is read after it is overwritten.
__global__ void k_rmul(double2* H, const double* Jr, int h, int ny, int nz) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const int total = h * ny * nz;
  if (idx >= total) return;
  const int kx = idx % h;
  const int rest = idx / h;
  const int ky = rest % ny, kz = rest / ny;
  const int jrow = (kz * ny + ky) * (h + 1);
  if (kx != 0) {
    const double j = Jr[jrow + kx];
    const double2 v = H[idx];
    H[idx] = make_double2(v.x * j, v.y * j);
    return;
  }
  const int ky2 = ky == 0 ? 0 : ny - ky, kz2 = kz == 0 ? 0 : nz - kz;
  const int midx = (kz2 * ny + ky2) * h;
  if (idx > midx) return;
  const double2 p = H[idx], pm = H[midx];
  const double2 A = make_double2(0.5 * (p.x + pm.x), 0.5 * (p.y - pm.y));
  const double2 B = make_double2(0.5 * (p.y + pm.y), -0.5 * (p.x - pm.x));
  const double j0 = Jr[jrow], jn = Jr[jrow + h];
  H[idx] = make_double2(j0 * A.x - jn * B.y, j0 * A.y + jn * B.x);
  if (midx != idx) {  // A(-k) = conj A(k), B(-k) = conj B(k)
    const int jrow2 = (kz2 * ny + ky2) * (h + 1);
    const double j0m = Jr[jrow2], jnm = Jr[jrow2 + h];
    H[midx] = make_double2(j0m * A.x + jnm * B.y, -j0m * A.y + jnm * B.x);
  }
}

// Jr = Re DFT(h^d J)/N at kx = 0 .. nx/2 (rows of nx/2 + 1).
__global__ void k_extract_jr(const double2* Jhat, double* Jr, int nx, int ny, int nz) {
  const int h1 = nx / 2 + 1;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= h1 * ny * nz) return;
  const int kx = idx % h1, r = idx / h1;
  Jr[idx] = Jhat[(size_t)r * nx + kx].x;
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

// Transforms along y (and z) of `data`, rows of W complex values (W = nx for
// the full array, nx/2 for the half spectrum): forward or unnormalised inverse.
static int fft_cols(fm_state* st, double2* data, int W, int inverse) {
  const Geo G = st->lv[0].g;
  cudaStream_t s = st->stream;
  const int ns[3] = {G.nx, G.ny, G.nz};
  for (int ax = 1; ax < st->dim; ++ax) {
    const int n = ns[ax];
    const int stride = ax == 1 ? W : W * G.ny;
    const int outer = ax == 1 ? G.nz : G.ny;
    const int ostride = ax == 1 ? W * G.ny : W;
    // TC columns per block: as many as keep at least two blocks per SM (one
    // column per block when the lines are too few), at most 16 and 64 KB of
    // shared memory; a power of two, so it divides W
    int TC = 16;
    while (TC > 1 && ((W / TC) * outer < 2 * st->sms || (size_t)n * TC * sizeof(double2) > 65536)) TC >>= 1;
    if (TC > W) TC = W;
    const size_t smem = (size_t)n * TC * sizeof(double2);
    int thr = n * TC / 2;  // one butterfly per thread and stage
    thr = thr > FT ? FT : (thr < 32 ? 32 : thr);
    dim3 grid(W / TC, outer);
    k_fft_strided<<<grid, thr, smem, s>>>(data, n, ilog2(n), stride, ostride, TC, st->fft.tw[ax], inverse);
    if (!launch_ok()) return FM_ECUDA;
  }
  return FM_OK;
}

// Forward (inverse = 0) or unnormalised inverse transform of st->fft.work.
static int fft_all(fm_state* st, int inverse) {
  const Geo G = st->lv[0].g;
  cudaStream_t s = st->stream;
  {
    const int n = G.nx;
    const size_t smem = (size_t)n * sizeof(double2);
    const int thr = n / 2 < FT ? (n / 2 < 32 ? 32 : n / 2) : FT;
    k_fft_x<<<G.ny * G.nz, thr, smem, s>>>(st->fft.work, n, ilog2(n), st->fft.tw[0], inverse);
    if (!launch_ok()) return FM_ECUDA;
  }
  return fft_cols(st, st->fft.work, G.nx, inverse);
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
      cudaFuncSetAttribute(k_fft_strided, cudaFuncAttributeMaxDynamicSharedMemorySize, 65536) != cudaSuccess ||
      cudaFuncSetAttribute(k_rfft_x, cudaFuncAttributeMaxDynamicSharedMemorySize, 65536) != cudaSuccess ||
      cudaFuncSetAttribute(k_irfft_x, cudaFuncAttributeMaxDynamicSharedMemorySize, 65536) != cudaSuccess) {
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
  {
    const int nr = (G.nx / 2 + 1) * G.ny * G.nz;
    k_extract_jr<<<(nr + FT - 1) / FT, FT, 0, s>>>(st->fft.work, st->fft.Jr, G.nx, G.ny, G.nz);
    if (!launch_ok()) return FM_ECUDA;
  }
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

// Real-input form (nx >= 8): the x transforms of the real rows as complex
// transforms of half length, the y / z transforms and the product on the
// half spectrum -- half the work and half the data of the complex form.
static int convolve_real(fm_state* st, const double* rho, double* out) {
  const Geo G = st->lv[0].g;
  cudaStream_t s = st->stream;
  const int n = G.nx, h = n / 2, logh = ilog2(h);
  const int rows = G.ny * G.nz;
  const size_t smem = (size_t)h * sizeof(double2);
  const int thr = h / 2 < FT ? (h / 2 < 32 ? 32 : h / 2) : FT;
  k_rfft_x<<<rows, thr, smem, s>>>(rho, st->fft.work, n, logh, st->fft.tw[0]);
  if (!launch_ok()) return FM_ECUDA;
  int rc = fft_cols(st, st->fft.work, h, 0);
  if (rc) return rc;
  const int nh = h * rows;
  k_rmul<<<(nh + FT - 1) / FT, FT, 0, s>>>(st->fft.work, st->fft.Jr, h, G.ny, G.nz);
  if (!launch_ok()) return FM_ECUDA;
  rc = fft_cols(st, st->fft.work, h, 1);
  if (rc) return rc;
  k_irfft_x<<<rows, thr, smem, s>>>(st->fft.work, out, n, logh, st->fft.tw[0]);
  if (!launch_ok()) return FM_ECUDA;
  return FM_OK;
}

int fft_convolve(fm_state* st, const double* rho, double* out) {
  g_cur = st;
  const Geo G = st->lv[0].g;
  if (G.nx >= 8 && !getenv("FM_FFT_COMPLEX")) return convolve_real(st, rho, out);
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
