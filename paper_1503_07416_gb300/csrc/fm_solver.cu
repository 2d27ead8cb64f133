// libfm: FAS multigrid solve of one implicit convex-splitting time step of the
// hydrodynamic PFC / CDFT freezing models (Sec. 5, Sec. 6, App. G), sm_103a.
//
// Solver structure (GB300-first; the paper's own solver is prior art):
//  * Outer loop in float64 (Sec. 6 residual test): r = S - N(g) for the
//    current iterate g, its norm max_c sqrt(h^d sum r_c^2), stop at tol.
//  * Each outer iteration runs one FAS V(nu1, nu2) cycle on the correction
//    equation M(e) = N(g + e) - N(g) = r in precision T (float64 for the FP64
//    path, float32 for the mixed path) with the iterate g frozen as a
//    coefficient, then g += e in float64.  M is N rewritten exactly in terms
//    of e (|c+e|^2 - |c|^2 = e(2c+e), (p+e)^3 - p^3 = e(3p^2 + 3pe + e^2),
//    ln(c+e) - ln c = log1p(e/c)), so the float32 cycle carries the relative
//    precision of the correction and the outer float64 loop converges to the
//    float64 fixed point.
//  * Smoother: red-black point-block Gauss-Seidel (App. G.1/G.2).  The point
//    block is triangular: rho from continuity, then kappa, mu (PFC), then the
//    d x d velocity block a I + [b]_x, solved in closed form; damping of the
//    whole block (App. G.3); positive projection (Sec. 6) when rho <= 0.
//  * Transfers: nodal full weighting of r, injection of e and of the
//    coefficients, bilinear/trilinear prolongation of the coarse correction.
//  * Coarsest grid: one thread block runs ncoarse red-black iterations.
#include <cuda.h>
#include <cudaTypedefs.h>  // PFN_cuTensorMapEncodeTiled
#include <cuda_runtime.h>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <cmath>
#include <new>

#include "fm_state.h"
#include "fm_device.cuh"
#include "fm_stepper.cuh"
#include "fm_zmarch.cuh"
#include "fm_coop.cuh"

namespace fm {

__global__ void __launch_bounds__(TPB) k_mass(const double* rho, int N, double* partials) {
  double acc[1] = {0.0};
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += gridDim.x * blockDim.x)
    acc[0] += rho[idx];
  block_partials<1>(acc, partials, blockIdx.x);
}

// Standalone float64 transfers (row-level entry points).
// out = in, converted element by element.
template <typename A, typename B>
__global__ void __launch_bounds__(TPB) k_convert(const A* in, B* out, int N) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) out[i] = (B)in[i];
}

__global__ void __launch_bounds__(TPB) k_narrow(const double* in, float* out, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = narrow_rn(in[i]);
}

__global__ void __launch_bounds__(TPB) k_widen(const float* in, double* out, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = widen(in[i]);
}

__global__ void k_restrict_one(const double* fine, double* coarse, Geo F, Geo C, int dim) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= C.N) return;
  int I, J, K;
  coords(idx, C, I, J, K);
  const int fi = 2 * I, fj = 2 * J, fk = 2 * K;
  const double wt[3] = {1.0, 2.0, 1.0};
  double acc = 0;
  const int kz = dim == 3 ? 3 : 1;
  for (int c = 0; c < kz; ++c) {
    const int zz = dim == 3 ? (fk + c - 1 + F.nz) % F.nz : 0;
    const double wz = dim == 3 ? wt[c] : 1.0;
    for (int b = 0; b < 3; ++b) {
      const int yy = (fj + b - 1 + F.ny) % F.ny;
      for (int a = 0; a < 3; ++a) {
        const int xx = (fi + a - 1 + F.nx) % F.nx;
        acc += wz * wt[b] * wt[a] * fine[(zz * F.ny + yy) * F.nx + xx];
      }
    }
  }
  coarse[idx] = acc / (dim == 3 ? 64.0 : 16.0);
}

__global__ void k_prolong_one(const double* coarse, double* fine, Geo F, Geo C, int dim) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= F.N) return;
  int i, j, k;
  coords(idx, F, i, j, k);
  double acc = 0;
  const int kz = (dim == 3 && (k & 1)) ? 2 : 1;
  const int ky = (j & 1) ? 2 : 1, kx = (i & 1) ? 2 : 1;
  for (int c = 0; c < kz; ++c) {
    const int Z = dim == 3 ? ((k >> 1) + c) % C.nz : 0;
    const double wz = (dim == 3 && (k & 1)) ? 0.5 : 1.0;
    for (int b = 0; b < ky; ++b) {
      const int Y = ((j >> 1) + b) % C.ny;
      const double wy = (j & 1) ? 0.5 : 1.0;
      for (int a = 0; a < kx; ++a) {
        const int X = ((i >> 1) + a) % C.nx;
        const double wx = (i & 1) ? 0.5 : 1.0;
        acc += wz * wy * wx * coarse[(Z * C.ny + Y) * C.nx + X];
      }
    }
  }
  fine[idx] += acc;
}


// --------------------------------------------------------------------------
// Host driver
// --------------------------------------------------------------------------
static cudaMemcpyKind kind_in(int where) {
  return where == FM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
}
static cudaMemcpyKind kind_out(int where) {
  return where == FM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
}


// Launch variant (TX, TY, SF, PIPE) of the 2-D fused sweep on level L.
template <typename T, int KIND, int TX, int TY, bool SF, bool PIPE, int NS = 1>
static int launch_rb_v(fm_state* st, const Lvl<T>& L, const Phys<T>& P, cudaStream_t s, int dir) {
  constexpr size_t smem = rb_smem_bytes<T, KIND, TX, TY, SF, PIPE, NS>();
  if (smem + 4096 > (size_t)st->smem_optin) return FM_EINVAL;  // variant does not fit on this device
  if (!L.r[0]) return FM_EINVAL;                               // no second correction buffer
  static int per_sm = 0;
  if (!per_sm) {
    if (cudaFuncSetAttribute(k_smooth_rb2d<T, KIND, TX, TY, SF, PIPE, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_smooth_rb2d<T, KIND, TX, TY, SF, PIPE, NS>, rb_threads(TX, TY),
                                                      smem) != cudaSuccess) {
      cudaGetLastError();
      return FM_ECUDA;
    }
    if (per_sm < 1) per_sm = 1;
  }
  const int ntx = (L.g.nx + TX - 1) / TX;
  const int ntiles = ntx * ((L.g.ny + TY - 1) / TY);
  int grid = ntiles;
  if (PIPE && grid > per_sm * st->sms) grid = per_sm * st->sms;
  k_smooth_rb2d<T, KIND, TX, TY, SF, PIPE, NS><<<grid, rb_threads(TX, TY), smem, s>>>(L, P, ntx, ntiles, dir);
  return FM_OK;
}

// cuTensorMapEncodeTiled, taken from the driver through the runtime (libfm
// links only the runtime); null when the driver does not provide it.
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

// Tensor map of one level array (nx x ny values of T, rows contiguous) with
// a box of bw x bh values; false where a tensor copy cannot address it (a
// row that is not a whole number of 16 bytes, a base not on a 16-byte
// boundary) or the driver refuses it.
template <typename T>
static bool encode_box_map(CUtensorMap* m, const void* base, const Geo& g, int bw, int bh) {
  const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc || !base || g.nz != 1) return false;
  if ((reinterpret_cast<uintptr_t>(base) & 15) || ((size_t)g.nx * sizeof(T)) % 16) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny};
  const cuuint64_t strides[1] = {(cuuint64_t)g.nx * sizeof(T)};
  const cuuint32_t box[2] = {(cuuint32_t)bw, (cuuint32_t)bh};
  const cuuint32_t es[2] = {1, 1};
  return enc(m, sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2,
             const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Tile form (SF = PIPE = false) with the tile staged by tensor copies; on a
// level whose arrays a tensor copy cannot address, the same tile form staged
// by cp.async (the same updates).
template <typename T, int KIND, int TX, int TY, int NS>
static int launch_rb_tma(fm_state* st, const Lvl<T>& L, const Phys<T>& P, cudaStream_t s, int dir) {
  using Gm = RBGeom<TX, TY, NS>;
  constexpr int NU = Layout<KIND, 2>::NU;
  constexpr size_t smem = rb_smem_bytes<T, KIND, TX, TY, false, false, NS>() + 128;  // + alignment to 128 B
  if (smem + 4096 > (size_t)st->smem_optin) return FM_EINVAL;
  if (!L.r[0]) return FM_EINVAL;
  RbMaps maps;
  memset(&maps, 0, sizeof(maps));
  const void* src[NU + 4];
  for (int q = 0; q < NU; ++q) src[q] = dir ? L.r[q] : L.e[q];
  src[NU + 0] = L.rk;
  src[NU + 1] = L.cr;
  src[NU + 2] = L.cv[0];
  src[NU + 3] = L.cv[1];
  bool ok = true;
  for (int a = 0; a < NU + 4 && ok; ++a) ok = encode_box_map<T>(&maps.m[a], src[a], L.g, Gm::SW, TY + 2 * Gm::H);
  if (!ok) return launch_rb_v<T, KIND, TX, TY, false, false, NS>(st, L, P, s, dir);
  static bool attr = false;
  if (!attr) {
    FM_CUDA(cudaFuncSetAttribute(k_smooth_rb2d_tma<T, KIND, TX, TY, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
    attr = true;
  }
  const int ntx = (L.g.nx + TX - 1) / TX;
  const int ntiles = ntx * ((L.g.ny + TY - 1) / TY);
  k_smooth_rb2d_tma<T, KIND, TX, TY, NS><<<ntiles, rb_threads(TX, TY), smem, s>>>(
      L, P, ntx, ntiles, dir, maps, &static_cast<Ctl*>(st->ctl)->fault);
  return FM_OK;
}

// Launch the row-marching form (strip width TX, ly rows per block) on level L.
template <typename T, int KIND, int TX>
static int launch_march(fm_state* st, const Lvl<T>& L, const Phys<T>& P, cudaStream_t s, int dir, int ly) {
  constexpr size_t smem = march_smem_bytes<T, KIND, TX>();
  if (smem + 4096 > (size_t)st->smem_optin) return FM_EINVAL;
  if (!L.r[0]) return FM_EINVAL;
  static bool attr = false;
  if (!attr) {
    FM_CUDA(cudaFuncSetAttribute(k_smooth_march<T, KIND, TX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
    attr = true;
  }
  const int nstrips = (L.g.nx + TX - 1) / TX;
  const int nseg = (L.g.ny + ly - 1) / ly;
  k_smooth_march<T, KIND, TX><<<nstrips * nseg, march_threads(TX), smem, s>>>(L, P, nstrips, ly, dir);
  return FM_OK;
}

// Launch the two-sweep marching form (strip width TX, ly rows per block).
template <typename T, int KIND, int TX>
static int launch_march2(fm_state* st, const Lvl<T>& L, const Phys<T>& P, cudaStream_t s, int dir, int ly) {
  constexpr size_t smem = march2_smem_bytes<T, KIND, TX>();
  if (smem + 4096 > (size_t)st->smem_optin) return FM_EINVAL;
  if (!L.r[0]) return FM_EINVAL;
  static bool attr = false;
  if (!attr) {
    FM_CUDA(cudaFuncSetAttribute(k_smooth_march2<T, KIND, TX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
    attr = true;
  }
  const int nstrips = (L.g.nx + TX - 1) / TX;
  const int nseg = (L.g.ny + ly - 1) / ly;
  k_smooth_march2<T, KIND, TX><<<nstrips * nseg, march_threads(TX), smem, s>>>(L, P, nstrips, ly, dir);
  return FM_OK;
}

// One launch of fused-sweep variant v on level L: sweeps_per_launch(v)
// sweeps, the correction read from L.e and written to L.r (dir = 0) or the
// reverse (dir = 1).
template <typename T, int KIND>
static int launch_coop(fm_state* st, const Lvl<T>& L, const Phys<T>& P, cudaStream_t s, int nsweeps);

template <typename T, int KIND>
static int launch_rb(fm_state* st, int v, const Lvl<T>& L, const Phys<T>& P, cudaStream_t s, int dir = 0) {
  switch (v) {
    case 0: return launch_rb_v<T, KIND, 32, 16, false, false>(st, L, P, s, dir);
    case 1: return launch_rb_v<T, KIND, 32, 16, false, true>(st, L, P, s, dir);
    case 2: return launch_rb_v<T, KIND, 32, 16, true, false>(st, L, P, s, dir);
    case 3: return launch_rb_v<T, KIND, 32, 16, true, true>(st, L, P, s, dir);
    case 4: return launch_rb_v<T, KIND, 64, 8, false, false>(st, L, P, s, dir);
    case 5: return launch_rb_v<T, KIND, 64, 8, false, true>(st, L, P, s, dir);
    case 6: return launch_rb_v<T, KIND, 64, 8, true, false>(st, L, P, s, dir);
    case 7: return launch_rb_v<T, KIND, 64, 8, true, true>(st, L, P, s, dir);
    case 8: return launch_rb_v<T, KIND, 32, 32, false, false>(st, L, P, s, dir);
    case 9: return launch_rb_v<T, KIND, 32, 32, false, true>(st, L, P, s, dir);
    case 10: return launch_rb_v<T, KIND, 32, 32, true, false>(st, L, P, s, dir);
    case 11: return launch_rb_v<T, KIND, 32, 32, true, true>(st, L, P, s, dir);
    case 12: return launch_march<T, KIND, 64>(st, L, P, s, dir, 16);
    case 13: return launch_march<T, KIND, 64>(st, L, P, s, dir, 32);
    case 14: return launch_march<T, KIND, 64>(st, L, P, s, dir, 64);
    case 15: return launch_march<T, KIND, 128>(st, L, P, s, dir, 16);
    case 16: return launch_march<T, KIND, 128>(st, L, P, s, dir, 32);
    case 17: return launch_march<T, KIND, 128>(st, L, P, s, dir, 64);
    case 18: return launch_march2<T, KIND, 64>(st, L, P, s, dir, 16);
    case 19: return launch_march2<T, KIND, 64>(st, L, P, s, dir, 32);
    case 20: return launch_march2<T, KIND, 64>(st, L, P, s, dir, 64);
    case 21: return launch_march2<T, KIND, 128>(st, L, P, s, dir, 16);
    case 22: return launch_march2<T, KIND, 128>(st, L, P, s, dir, 32);
    case 23: return launch_march2<T, KIND, 128>(st, L, P, s, dir, 64);
    case 24: return launch_rb_v<T, KIND, 32, 16, false, false, 2>(st, L, P, s, dir);
    case 25: return launch_rb_v<T, KIND, 64, 8, false, false, 2>(st, L, P, s, dir);
    case 26: return launch_rb_v<T, KIND, 32, 32, false, false, 2>(st, L, P, s, dir);
    case 27: return launch_rb_tma<T, KIND, 32, 16, 2>(st, L, P, s, dir);
    case 28: return launch_rb_tma<T, KIND, 32, 16, 1>(st, L, P, s, dir);
    case 29: return launch_rb_tma<T, KIND, 32, 32, 2>(st, L, P, s, dir);
    case 30: return launch_rb_v<T, KIND, 16, 16, false, false>(st, L, P, s, dir);
    case 31: return launch_rb_v<T, KIND, 16, 16, false, false, 2>(st, L, P, s, dir);
    case 32: return launch_rb_v<T, KIND, 16, 8, false, false>(st, L, P, s, dir);
    case 33: return launch_rb_v<T, KIND, 16, 8, false, false, 2>(st, L, P, s, dir);
    case 35: return launch_rb_v<T, KIND, 32, 14, false, false, 2>(st, L, P, s, dir);
    default: return launch_coop<T, KIND>(st, L, P, s, 2);  // in place (dir does not apply)
  }
}

// Launch the 3-D z-marching sweep (tiles 32 x TY) on level L: one block per
// tile and z-chunk, as many blocks as there are resident slots (at most nz / 2
// chunks a tile): nchunks = slots / ntile chunks for the first nlong tiles,
// one more for the others.  FM_EINVAL where it does not apply (sides not
// multiples of the tile, no second correction buffer, shared memory too
// small).
template <typename T, int KIND, int TY>
static bool zm3_applies_v(const fm_state* st, const Lvl<T>& L) {
  constexpr size_t smem = zm_smem_bytes<T, KIND, TY>();
  return smem + 1024 <= (size_t)st->smem_optin && L.r[0] && L.g.nx % ZmGeom<TY>::TX == 0 && L.g.ny % TY == 0 &&
         L.g.nz >= 2 && (L.g.nz & 1) == 0;
}

template <typename T, int KIND>
static bool zm3_applies(const fm_state* st, int v, const Lvl<T>& L) {
  return v == SM3_ZM ? zm3_applies_v<T, KIND, 8>(st, L) : zm3_applies_v<T, KIND, 16>(st, L);
}

template <typename T, int KIND, int TY>
static int launch_zm3_v(fm_state* st, const Lvl<T>& L, const Phys<T>& P, cudaStream_t s, int dir) {
  constexpr size_t smem = zm_smem_bytes<T, KIND, TY>();
  if constexpr (smem > 232448) {  // beyond any device's shared memory per block: not instantiated
    return FM_EINVAL;
  } else {
  if (!zm3_applies_v<T, KIND, TY>(st, L)) return FM_EINVAL;
  static int per_sm = 0;
  if (!per_sm) {
    if (cudaFuncSetAttribute(k_smooth_zm3<T, KIND, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_smooth_zm3<T, KIND, TY>, ZmGeom<TY>::THREADS,
                                                      smem) != cudaSuccess) {
      cudaGetLastError();
      per_sm = 0;
      return FM_ECUDA;
    }
    if (per_sm < 1) per_sm = 1;
  }
  const int ntile = (L.g.nx / ZmGeom<TY>::TX) * (L.g.ny / TY);
  long long nblk = (long long)per_sm * st->sms;
  if (nblk > (long long)ntile * (L.g.nz / 2)) nblk = (long long)ntile * (L.g.nz / 2);
  if (nblk < ntile) nblk = ntile;
  const int nchunks = (int)(nblk / ntile), nlong = ntile - (int)(nblk % ntile);
  k_smooth_zm3<T, KIND, TY><<<(int)nblk, ZmGeom<TY>::THREADS, smem, s>>>(L, P, dir, nchunks, nlong);
  return FM_OK;
  }
}

// Launch nsweeps red-black sweeps of 2-D level L in place as one cooperative
// launch (variant 34): as many blocks as are resident at once, at most one
// thread per point of a colour.  FM_EINVAL where it does not apply (odd
// rows, 3-D).
template <typename T, int KIND>
static bool coop_applies(const Lvl<T>& L) {
  return L.g.nz == 1 && (L.g.nx & 1) == 0 && L.g.N >= 2;
}

template <typename T, int KIND>
static int launch_coop(fm_state* st, const Lvl<T>& L, const Phys<T>& P, cudaStream_t s, int nsweeps) {
  if (!coop_applies<T, KIND>(L) || nsweeps < 1) return FM_EINVAL;
  static int per_sm = 0;
  if (!per_sm) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_smooth_coop<T, KIND>, TPB, 0) != cudaSuccess) {
      cudaGetLastError();
      per_sm = 0;
      return FM_ECUDA;
    }
    if (per_sm < 1) return FM_EINVAL;
  }
  const int half = L.g.N / 2;
  int grid = per_sm * st->sms;
  if (grid > (half + TPB - 1) / TPB) grid = (half + TPB - 1) / TPB;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(TPB);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  Ctl* ctl = static_cast<Ctl*>(st->ctl);
  if (cudaLaunchKernelEx(&cfg, k_smooth_coop<T, KIND>, L, P, nsweeps, &ctl->gbar[0], &ctl->fault) != cudaSuccess) {
    cudaGetLastError();
    return FM_ECUDA;
  }
  return FM_OK;
}

template <typename T, int KIND>
static int launch_zm3(fm_state* st, int v, const Lvl<T>& L, const Phys<T>& P, cudaStream_t s, int dir) {
  return v == SM3_ZM ? launch_zm3_v<T, KIND, 8>(st, L, P, s, dir) : launch_zm3_v<T, KIND, 16>(st, L, P, s, dir);
}

// The sweep variants FM_RB_VARIANT fixes (a measurement switch): one number
// for every level, or a comma-separated list, one per level from the finest
// (the last one repeats); numbers outside 0 .. nvar - 1 give 0.
static void fixed_variants(fm_state* st, const char* spec, int nvar) {
  const char* p = spec;
  int v = 0;
  for (int l = 0; l < MAXLEV; ++l) {
    if (*p) {
      v = atoi(p);
      if (v < 0 || v >= nvar) v = 0;
      while (*p && *p != ',') ++p;
      if (*p == ',') ++p;
    }
    st->rbv[l] = v;
  }
}

// Element-wise conversions of up to CONV_MAX arrays in one launch: array a
// (n[a] values) from src[a] to dst[a], block row blockIdx.y taking array a.
constexpr int CONV_MAX = 96;
// the coarse solve's conversions: the entry level's f and e, and rk, cr, omega
// (3) and the coefficient velocity (3) of up to MAXSMALL levels
static_assert(CONV_MAX >= 2 * MAXU + MAXSMALL * 8, "room for every array the coarse-solve conversions copy");
template <typename A, typename B>
struct ConvSet {
  const A* src[CONV_MAX];
  B* dst[CONV_MAX];
  int n[CONV_MAX];
  int count;
  int maxn;
};
template <typename A, typename B>
__global__ void __launch_bounds__(TPB) k_convert_set(const __grid_constant__ ConvSet<A, B> C) {
  const int a = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < C.n[a]) C.dst[a][i] = static_cast<B>(C.src[a][i]);
}

// e = r on every point of a level (the correction back in e).
template <typename T, int NU>
__global__ void __launch_bounds__(TPB) k_copy_back(Lvl<T> L) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= L.g.N) return;
  T v[NU];
#pragma unroll
  for (int q = 0; q < NU; ++q) v[q] = L.r[q][idx];
#pragma unroll
  for (int q = 0; q < NU; ++q) L.e[q][idx] = v[q];
}

// View of a level with the roles of the correction and residual buffers
// exchanged (the correction in r).
template <typename T>
static Lvl<T> swap_er(Lvl<T> L) {
  for (int q = 0; q < MAXU; ++q) {
    T* t = L.e[q];
    L.e[q] = L.r[q];
    L.r[q] = t;
  }
  return L;
}


// FM_ETIMEOUT if a kernel of this state gave up a bounded wait (the control
// block's fault flag; synchronises the stream).
static int read_fault(fm_state* st) {
  int fault = 0;
  FM_CUDA(cudaMemcpyAsync(&fault, &static_cast<Ctl*>(st->ctl)->fault, sizeof(int), cudaMemcpyDeviceToHost,
                          st->stream));
  FM_CUDA(cudaStreamSynchronize(st->stream));
  return fault ? FM_ETIMEOUT : FM_OK;
}

// The step is issued in three parts:
//   pre  : omega^k, (J * rho^k), S, g^0, coefficients rho^k/omega^k down the
//          hierarchy, the float64 residual of g^0 and its norm;
//   body : coefficients g down the hierarchy, one FAS V-cycle on the
//          correction equation, g += e, the float64 residual and its norm;
//   post : closure and commit of the new time level (skipped on failure),
//          the control block copied to pinned host memory.
// Graph mode captures pre, a WHILE conditional node around body, and post
// into one CUDA graph (one launch and one host synchronisation per step);
// host-loop mode (used while profiling) launches the parts directly and
// reads the control block after each norm.
template <typename T, int KIND, int DIM>
struct Solver {
  using LY = Layout<KIND, DIM>;
  static constexpr int NVEL = DIM;  // velocity arrays of the state (copied by step_host)

  static int inject_all(fm_state* st, bool coefficients_only) {
    if (st->nlev < 2) return FM_OK;
    InjAll<T> A;
    memset(&A, 0, sizeof(A));
    A.nl = st->nlev;
    A.g0 = st->lv[0].g;
    A.off[0] = A.off[1] = 0;
    for (int l = 1; l < st->nlev; ++l) {
      A.g[l] = st->lv[l].g;
      A.off[l + 1] = A.off[l] + st->lv[l].g.N;
    }
    int q = 0;
    if (coefficients_only) {
      A.src[q] = (const T*)st->lv[0].cr;
      for (int l = 1; l < st->nlev; ++l) A.dst[l][q] = (T*)st->lv[l].cr;
      ++q;
      for (int d = 0; d < DIM; ++d, ++q) {
        A.src[q] = (const T*)st->lv[0].cv[d];
        for (int l = 1; l < st->nlev; ++l) A.dst[l][q] = (T*)st->lv[l].cv[d];
      }
    } else {
      A.src[q] = (const T*)st->lv[0].rk;
      for (int l = 1; l < st->nlev; ++l) A.dst[l][q] = (T*)st->lv[l].rk;
      ++q;
      for (int d = 0; d < LY::NOM; ++d, ++q) {
        A.src[q] = (const T*)st->lv[0].om[d];
        for (int l = 1; l < st->nlev; ++l) A.dst[l][q] = (T*)st->lv[l].om[d];
      }
    }
    A.nsrc = q;
    k_inject_all<T><<<nblocks(A.off[st->nlev]), TPB, 0, st->stream>>>(A);
    FM_LAUNCHED();
    return FM_OK;
  }

  // Choose, per multi-kernel level, the fastest variant of the fused 2-D
  // sweep: each variant is timed with CUDA events (one warm-up and TUNE_REPS
  // timed launches) on the level itself and compared per sweep; a later
  // variant replaces the choice only if it is 2% faster.  The sweeps only
  // touch solver scratch.
  // One 3-D sweep in z-chunks of Z planes (variant 2): red over planes
  // [cZ, (c+1)Z), then black over the planes whose neighbours are all red by
  // then -- [max(1, cZ - 1), (c+1)Z - 1), the last chunk through nz - 1 and
  // plane 0.  Every black plane is swept once, after the red planes beside it.
  static int chunked_sweep(fm_state* st, const Lvl<T>& L, const Phys<T>& P, int Z, cudaStream_t s) {
    const int ny = L.g.ny, nz = L.g.nz, half = L.g.nx >> 1;
    const int nch = nz / Z;
    for (int c = 0; c < nch; ++c) {
      int rows = Z * ny;
      k_smooth_rows<T, KIND, DIM><<<nblocks((long long)rows * half), TPB, 0, s>>>(L, P, 0, c * Z * ny, rows);
      FM_LAUNCHED();
      const int b0 = c == 0 ? 1 : c * Z - 1;
      const int b1 = c == nch - 1 ? nz + 1 : (c + 1) * Z - 1;  // nz + 1: through nz - 1 and plane 0
      rows = (b1 - b0) * ny;
      if (rows > 0) {
        k_smooth_rows<T, KIND, DIM><<<nblocks((long long)rows * half), TPB, 0, s>>>(L, P, 1, b0 * ny, rows);
        FM_LAUNCHED();
      }
    }
    return FM_OK;
  }

  // Launch one sweep (a red and a black colour pass) of variant v (3-D) on level L.
  static int launch_colour_pair(fm_state* st, int v, const Lvl<T>& L, const Phys<T>& P) {
    const int half = L.g.N / 2;
    if (v >= SM3_ZM) {
      if constexpr (DIM == 3) {
        const int rc = launch_zm3<T, KIND>(st, v, L, P, st->stream, 0);
        if (rc == FM_OK) FM_LAUNCHED();
        return rc;
      }
      return FM_EINVAL;
    }
    if (v == 2) {
      const int Z = z_chunk_planes(L.g);
      return Z ? chunked_sweep(st, L, P, Z, st->stream) : FM_EINVAL;  // no chunking at this size
    }
    for (int color = 0; color < 2; ++color) {
      if (v == 1)
        k_smooth_occ<T, KIND, DIM><<<nblocks(half), TPB, 0, st->stream>>>(L, P, color);
      else
        k_smooth<T, KIND, DIM><<<nblocks(half), TPB, 0, st->stream>>>(L, P, color);
      FM_LAUNCHED();
    }
    return FM_OK;
  }

  // 3-D: time the colour-sweep variants per multi-kernel level (one warm-up
  // pair, TUNE_REPS timed pairs); a later variant replaces the choice only if
  // it is 2% faster.  FM_RB_VARIANT fixes it (0 or 1).
  static int autotune3(fm_state* st) {
    const char* fixed = getenv("FM_RB_VARIANT");
    for (int l = 0; l < MAXLEV; ++l) st->rbv[l] = 0;
    if (fixed && fixed[0]) {
      fixed_variants(st, fixed, SM3_NVAR);
      return FM_OK;
    }
    Phys<T> P = make_phys<T>(st);
    cudaEvent_t e0, e1;
    FM_CUDA(cudaEventCreate(&e0));
    FM_CUDA(cudaEventCreate(&e1));
    int rc = FM_OK;
    const int ntuned = st->small_from + (st->coarse_fused ? 1 : 0);
    for (int l = 0; l < ntuned && rc == FM_OK; ++l) {
      const Lvl<T> L = make_lvl<T>(st, l);
      float best = 1e30f;
      for (int v = 0; v < SM3_NVAR && rc == FM_OK; ++v) {
        rc = launch_colour_pair(st, v, L, P);
        if (rc == FM_EINVAL) {  // not applicable at this size
          rc = FM_OK;
          continue;
        }
        if (rc) break;
        if (cudaEventRecord(e0, st->stream) != cudaSuccess) { rc = FM_ECUDA; break; }
        for (int k = 0; k < TUNE_REPS && rc == FM_OK; ++k) rc = launch_colour_pair(st, v, L, P);
        if (rc) break;
        float ms = 0.f;
        if (cudaEventRecord(e1, st->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
          rc = FM_ECUDA;
          break;
        }
        st->rbt[l][v] = ms / TUNE_REPS;
        if (ms < best * 0.98f) {
          best = ms;
          st->rbv[l] = v;
        }
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaGetLastError();
    return rc;
  }

  static int autotune(fm_state* st) {
    if constexpr (DIM != 2) {
      return st->fused_rb ? autotune3(st) : FM_OK;
    } else {
      const char* fixed = getenv("FM_RB_VARIANT");
      for (int l = 0; l < MAXLEV; ++l) st->rbv[l] = 0;
      if (fixed && fixed[0]) {
        fixed_variants(st, fixed, RB_NVAR);
        return FM_OK;
      }
      if (!st->fused_rb) return FM_OK;
      Phys<T> P = make_phys<T>(st);
      cudaEvent_t e0, e1;
      FM_CUDA(cudaEventCreate(&e0));
      FM_CUDA(cudaEventCreate(&e1));
      int rc = FM_OK;
      const int ntuned = st->small_from + (st->coarse_fused ? 1 : 0);
      for (int l = 0; l < ntuned && rc == FM_OK; ++l) {
        Lvl<T> L = make_lvl<T>(st, l);
        float best = 1e30f;
        for (int v = 0; v < RB_NVAR && rc == FM_OK; ++v) {
          rc = launch_rb<T, KIND>(st, v, L, P, st->stream);
          if (rc == FM_EINVAL) {  // does not fit in shared memory: skip
            rc = FM_OK;
            continue;
          }
          if (rc) break;
          if (cudaEventRecord(e0, st->stream) != cudaSuccess) { rc = FM_ECUDA; break; }
          for (int k = 0; k < TUNE_REPS && rc == FM_OK; ++k) rc = launch_rb<T, KIND>(st, v, L, P, st->stream);
          if (rc) break;
          if (cudaEventRecord(e1, st->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
            rc = FM_ECUDA;
            break;
          }
          float ms = 0.f;
          if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) { rc = FM_ECUDA; break; }
          ms /= sweeps_per_launch(v);  // compared per sweep
          st->rbt[l][v] = ms / TUNE_REPS;
          if (ms < best * 0.98f) {  // a later variant must be clearly faster
            best = ms;
            st->rbv[l] = v;
          }
        }
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      cudaGetLastError();
      return rc ? rc : read_fault(st);
    }
  }

  static int enqueue_prepare(fm_state* st) {
    const Geo G = st->lv[0].g;
    const double h = st->lv[0].h;
    Phys<double> P = make_phys<double>(st);
    cudaStream_t s = st->stream;
    if (st->prm.init == FM_INIT_EXTRAPOLATE) {
      Ptr6 g, gp;
      for (int q = 0; q < MAXU; ++q) {
        g.p[q] = st->g[q];
        gp.p[q] = st->gp[q];
      }
      k_extrapolate<LY::NU><<<nblocks(G.N), TPB, 0, s>>>(g, gp, G.N, (const Ctl*)st->ctl);
      FM_LAUNCHED();
    }
    if (KIND == KCDFT) {
      FM_CUDA(cudaMemsetAsync(&static_cast<Ctl*>(st->ctl)->nonpos, 0, sizeof(int), s));
      int rc = fft_convolve(st, st->rho, st->conv);
      if (rc) return rc;
    }
    Fields64 F = make_fields(st);
    const Step64 K = make_step64(P, 1.0 / h);
    k_prepare<KIND, DIM><<<nblocks(G.N), TPB, 0, s>>>(F, G, K, P);
    FM_LAUNCHED();
    if (KIND == KPFC) {
      k_prepare_mu<DIM><<<nblocks(G.N), TPB, 0, s>>>(F, G, K, P);
      FM_LAUNCHED();
    }
    return inject_all(st, false);
  }

  static int prepare(fm_state* st) {
    int rc = enqueue_prepare(st);
    if (rc) return rc;
    FM_CUDA(cudaStreamSynchronize(st->stream));
    st->prepared = true;
    return FM_OK;
  }

  static Resid64Out resid_out(fm_state* st, bool cycle, double* const* r64) {
    Resid64Out O;
    for (int q = 0; q < MAXU; ++q) {
      O.f0[q] = (cycle && q < LY::NU) ? st->lv[0].f[q] : nullptr;
      O.e0[q] = (cycle && q < LY::NU) ? st->lv[0].e[q] : nullptr;
      O.r64[q] = (r64 && q < LY::NU) ? r64[q] : nullptr;
    }
    O.cr32 = nullptr;
    for (int d = 0; d < 3; ++d) O.cv32[d] = nullptr;
    if (cycle && st->prm.precision == FM_MIXED) {
      O.cr32 = (float*)st->lv[0].cr;
      for (int d = 0; d < DIM; ++d) O.cv32[d] = (float*)st->lv[0].cv[d];
    }
    return O;
  }

  // Float64 residual: 2-D tiled kernel; 3-D shared quantities then residual.
  // update (3-D, after a cycle): the float64 update g += e is made by the
  // shared-quantity pass (2-D makes it in k_update64 before this).
  static int launch_resid64(fm_state* st, const Fields64& F, const Resid64Out& O, const Geo& G, double h,
                            const Phys<double>& P, bool update = false) {
    cudaStream_t s = st->stream;
    if constexpr (DIM == 2) {
      k_resid64_tile<KIND, T><<<st->nblk, TPB, 0, s>>>(F, O, G, make_step64(P, 1.0 / h), P, st->partials);
      FM_LAUNCHED();
    } else {
      Shared64 X;
      for (int q = 0; q < 5; ++q) X.x[q] = st->x64[q];
      if (update)
        k_update_shared64<KIND, DIM, T><<<nblocks(G.N), TPB, 0, s>>>(F, O, X, G.N, P.ce, st->prm.delta);
      else
        k_shared64<KIND, DIM><<<nblocks(G.N), TPB, 0, s>>>(F, X, G.N, P.ce);
      FM_LAUNCHED();
      k_resid64_x<KIND, DIM, T><<<st->nblk, TPB, 0, s>>>(F, X, O, G, make_step64(P, 1.0 / h), P,
                                                           st->partials);
      FM_LAUNCHED();
    }
    return FM_OK;
  }

  // float64 residual of the current iterate, the level-0 set-up of a cycle
  // and the control-block update (in_body: this follows a cycle).
  static int enqueue_resid_norm(fm_state* st, int in_body, cudaGraphConditionalHandle hdl, int use_handle) {
    const Geo G = st->lv[0].g;
    const double h = st->lv[0].h;
    Phys<double> P = make_phys<double>(st);
    cudaStream_t s = st->stream;
    Fields64 F = make_fields(st);
    Resid64Out O = resid_out(st, true, nullptr);
    int rc = launch_resid64(st, F, O, G, h, P, DIM == 3 && in_body);
    if (rc) return rc;
    const double w = (DIM == 3) ? h * h * h : h * h;
    k_norm_ctl<LY::NU><<<1, TPB, 0, s>>>(st->partials, st->nblk, w, (Ctl*)st->ctl, st->prm.tol,
                                         st->prm.max_cycles, in_body, hdl, use_handle);
    FM_LAUNCHED();
    return FM_OK;
  }

  // Standalone float64 residual for fm_residual (synchronous).
  static int residual64(fm_state* st, double* const* r64, double* norm_host) {
    const Geo G = st->lv[0].g;
    const double h = st->lv[0].h;
    Phys<double> P = make_phys<double>(st);
    cudaStream_t s = st->stream;
    Fields64 F = make_fields(st);
    Resid64Out O = resid_out(st, false, r64);
    int rc = launch_resid64(st, F, O, G, h, P);
    if (rc) return rc;
    const double w = (DIM == 3) ? h * h * h : h * h;
    k_norm_final<LY::NU><<<1, TPB, 0, s>>>(st->partials, st->nblk, w, st->dscal);
    FM_LAUNCHED();
    FM_CUDA(cudaMemcpyAsync(st->hscal, st->dscal, sizeof(double), cudaMemcpyDeviceToHost, s));
    FM_CUDA(cudaStreamSynchronize(s));
    *norm_host = st->hscal[0];
    return FM_OK;
  }

  // Smoother row: sweeps on level 0 for caller-supplied e and f (float64,
  // staged through the float64 scratch r64 and rounded to T).
  static int smooth_row(fm_state* st, double* const* e, const double* const* f, int sweeps, int variant,
                        int where) {
    if (variant < FM_SWEEP_TWO_COLOUR || variant >= (DIM == 3 ? SM3_NVAR : RB_NVAR)) return FM_EINVAL;
    const Geo G = st->lv[0].g;
    cudaStream_t s = st->stream;
    // coefficient copies of the iterate (mixed path), as at the start of a cycle
    Fields64 F = make_fields(st);
    Resid64Out O = resid_out(st, true, nullptr);
    int rc = launch_resid64(st, F, O, G, st->lv[0].h, make_phys<double>(st));
    if (rc) return rc;
    Lvl<T> L = make_lvl<T>(st, 0);
    const size_t bytes = (size_t)G.N * sizeof(double);
    for (int q = 0; q < LY::NU; ++q) {
      FM_CUDA(cudaMemcpyAsync(st->r64[q], e[q], bytes, kind_in(where), s));
      k_convert<double, T><<<nblocks(G.N), TPB, 0, s>>>(st->r64[q], L.e[q], G.N);
      FM_LAUNCHED();
      FM_CUDA(cudaMemcpyAsync(st->r64[q], f[q], bytes, kind_in(where), s));
      k_convert<double, T><<<nblocks(G.N), TPB, 0, s>>>(st->r64[q], L.f[q], G.N);
      FM_LAUNCHED();
    }
    const Phys<T> P = make_phys<T>(st);
    int v = (DIM == 2 && variant != FM_SWEEP_TWO_COLOUR && (st->fused_rb || variant >= 0))
                ? (variant >= 0 ? variant : st->rbv[0])
                : -1;
    if (DIM == 3 && variant != FM_SWEEP_TWO_COLOUR) v = variant >= 0 ? variant : st->rbv[0];
    int in_r = 0;
    rc = run_sweeps(st, L, v, P, sweeps, &in_r, false);
    if (rc) return rc;
    const Lvl<T> E = in_r ? swap_er(L) : L;
    for (int q = 0; q < LY::NU; ++q) {
      k_convert<T, double><<<nblocks(G.N), TPB, 0, s>>>(E.e[q], st->r64[q], G.N);
      FM_LAUNCHED();
      FM_CUDA(cudaMemcpyAsync(e[q], st->r64[q], bytes, kind_out(where), s));
    }
    return read_fault(st);
  }

  // `iters` sweeps on level L (its physical buffers; the correction is in
  // L.r if *in_r, else in L.e; *in_r is updated).  v >= 0: fused variant v,
  // each launch reading the correction from one buffer and writing it to the
  // other, over the largest even number of sweeps; the rest (and all sweeps
  // for v < 0) in place as a red and a black launch.  prof: CUDA events
  // around each launch.
  static int run_sweeps(fm_state* st, const Lvl<T>& L, int v, const Phys<T>& P, int iters, int* in_r, bool prof) {
    cudaStream_t s = st->stream;
    const int half = L.g.N / 2;
    const int nfused = (DIM == 2 && v >= 0) ? (iters & ~1) : 0;
    const int per = v >= 0 ? sweeps_per_launch(v) : 1;
    if (DIM == 2 && v == RB_COOP && !coop_applies<T, KIND>(L)) v = -1;  // odd rows: two-colour launches
    if (DIM == 2 && v == RB_COOP) {  // all sweeps in one cooperative launch, in place
      if (prof && st->npev + 2 <= MAXEV) FM_CUDA(cudaEventRecord(st->pev[st->npev], s));
      if (iters > 0) {
        if constexpr (DIM == 2) {
          const int rc = launch_coop<T, KIND>(st, *in_r ? swap_er(L) : L, P, s, iters);
          if (rc) return rc;
        }
        FM_LAUNCHED();
      }
      if (prof && st->npev + 2 <= MAXEV) {
        FM_CUDA(cudaEventRecord(st->pev[st->npev + 1], s));
        st->npev += 2;
      }
      return FM_OK;
    }
    if (DIM == 3 && v >= SM3_ZM && !zm3_applies<T, KIND>(st, v, L)) v = 1;  // not at this level's size
    if (DIM == 3 && v >= SM3_ZM) {  // fused z-marching sweeps, one launch each, e and r alternating
      for (int it = 0; it < iters; ++it) {
        if (prof && st->npev + 2 <= MAXEV) FM_CUDA(cudaEventRecord(st->pev[st->npev], s));
        if constexpr (DIM == 3) {
          const int rc = launch_zm3<T, KIND>(st, v, L, P, s, *in_r);
          if (rc) return rc;
        }
        FM_LAUNCHED();
        if (prof && st->npev + 2 <= MAXEV) {
          FM_CUDA(cudaEventRecord(st->pev[st->npev + 1], s));
          st->npev += 2;
        }
        *in_r ^= 1;
      }
      return FM_OK;
    }
    if (DIM == 3 && v == 2) {  // z-chunked sweeps (in place, like the colour launches)
      const int Z = z_chunk_planes(L.g);
      if (Z) {
        const Lvl<T> E = *in_r ? swap_er(L) : L;
        for (int it = 0; it < iters; ++it) {
          if (prof && st->npev + 2 <= MAXEV) FM_CUDA(cudaEventRecord(st->pev[st->npev], s));
          const int rc = chunked_sweep(st, E, P, Z, s);
          if (rc) return rc;
          if (prof && st->npev + 2 <= MAXEV) {
            FM_CUDA(cudaEventRecord(st->pev[st->npev + 1], s));
            st->npev += 2;
          }
        }
        return FM_OK;
      }
      v = 1;  // no chunking at this size
    }
    for (int it = 0; it < iters;) {
      const bool fused = it < nfused;
      const int nlaunch = fused ? 1 : 2;
      for (int color = 0; color < nlaunch; ++color) {
        if (prof && st->npev + 2 <= MAXEV) FM_CUDA(cudaEventRecord(st->pev[st->npev], s));
        if (fused) {
          if constexpr (DIM == 2) {
            const int rc = launch_rb<T, KIND>(st, v, L, P, s, *in_r);
            if (rc) return rc;
          }
        } else if (DIM == 3 && v == 1) {  // 3-D: v is the colour-sweep variant
          k_smooth_occ<T, KIND, DIM><<<nblocks(half), TPB, 0, s>>>(*in_r ? swap_er(L) : L, P, color);
        } else {
          k_smooth<T, KIND, DIM><<<nblocks(half), TPB, 0, s>>>(*in_r ? swap_er(L) : L, P, color);
        }
        FM_LAUNCHED();
        if (prof && st->npev + 2 <= MAXEV) {
          FM_CUDA(cudaEventRecord(st->pev[st->npev + 1], s));
          st->npev += 2;
        }
      }
      if (fused) {
        *in_r ^= 1;
        it += per;
      } else {
        it += 1;
      }
    }
    return FM_OK;
  }

  static int smooth(fm_state* st, int l, const Phys<T>& P, int iters, int* in_r) {
    const bool prof = st->prof && !st->capturing && l == 0;
    const int v = DIM == 3 ? st->rbv[l] : (st->fused_rb ? st->rbv[l] : -1);
    return run_sweeps(st, make_lvl<T>(st, l), v, P, iters, in_r, prof);
  }

  // One V-cycle from level l down; *out_in_r: on return the correction of
  // level l is in its r buffer (1) or in e (0).
  // The V-cycle of the small levels S (each of at most SMALL_N points) in
  // one block: shared memory when they fit, else global memory.
  static int small_cycle(fm_state* st, const SmallLv<T>& S, const Phys<T>& P) {
    cudaStream_t s = st->stream;
    SmallSmem<T> M;
    const size_t smem = small_layout<T, KIND, DIM>(S, M, SMALL_SMEM_MAX);
    if (smem <= SMALL_SMEM_MAX && S.lv[0].g.N <= SMALL_SMEM_N) {
      static bool attr = false;
      if (!attr) {
        FM_CUDA(cudaFuncSetAttribute(k_vcycle_small_smem<T, KIND, DIM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)SMALL_SMEM_MAX));
        attr = true;
      }
      k_vcycle_small_smem<T, KIND, DIM><<<1, SMALL_TPB, smem, s>>>(S, M, P, st->prm.nu1, st->prm.nu2,
                                                                    st->prm.ncoarse);
    } else {
      k_vcycle_small<T, KIND, DIM><<<1, SMALL_TPB, 0, s>>>(S, P, st->prm.nu1, st->prm.nu2, st->prm.ncoarse);
    }
    FM_LAUNCHED();
    return FM_OK;
  }

  // Conversions between the coarse levels and their float64 copies (lv64):
  // to64 copies the entry level l's right-hand side and correction and the
  // coefficients of levels l .. nlev - 1; from64 copies the entry level's
  // float64 correction (in r when in_r) back.  One launch each.
  static int coarse_to64(fm_state* st, int l) {
    ConvSet<T, double> C{};
    auto add = [&](const void* src, void* dst, int n) {
      if (src && dst && C.count < CONV_MAX) {
        C.src[C.count] = static_cast<const T*>(src);
        C.dst[C.count] = static_cast<double*>(dst);
        C.n[C.count] = n;
        C.count++;
        if (n > C.maxn) C.maxn = n;
      }
    };
    const int n0 = st->lv[l].g.N;
    for (int q = 0; q < LY::NU; ++q) {
      add(st->lv[l].f[q], st->lv64[l].f[q], n0);
      add(st->lv[l].e[q], st->lv64[l].e[q], n0);
    }
    for (int k = l; k < st->nlev; ++k) {
      const int n = st->lv[k].g.N;
      add(st->lv[k].rk, st->lv64[k].rk, n);
      add(st->lv[k].cr, st->lv64[k].cr, n);
      for (int d = 0; d < LY::NOM; ++d) add(st->lv[k].om[d], st->lv64[k].om[d], n);
      for (int d = 0; d < DIM; ++d) add(st->lv[k].cv[d], st->lv64[k].cv[d], n);
    }
    k_convert_set<T, double><<<dim3((C.maxn + TPB - 1) / TPB, C.count), TPB, 0, st->stream>>>(C);
    FM_LAUNCHED();
    return FM_OK;
  }
  static int coarse_from64(fm_state* st, int l, int in_r) {
    ConvSet<double, T> C{};
    const int n0 = st->lv[l].g.N;
    for (int q = 0; q < LY::NU; ++q) {
      C.src[q] = static_cast<const double*>(in_r ? st->lv64[l].r[q] : st->lv64[l].e[q]);
      C.dst[q] = static_cast<T*>(st->lv[l].e[q]);
      C.n[q] = n0;
    }
    C.count = LY::NU;
    C.maxn = n0;
    k_convert_set<double, T><<<dim3((n0 + TPB - 1) / TPB, C.count), TPB, 0, st->stream>>>(C);
    FM_LAUNCHED();
    return FM_OK;
  }

  // The coarsest-grid solve in float64 (mixed path): the coarse levels from
  // l down on their float64 copies -- the single-block V-cycle, or the
  // coarsest level's ncoarse sweeps as colour launches -- between the two
  // conversions.
  static int coarse_solve64(fm_state* st, int l) {
    int rc = coarse_to64(st, l);
    if (rc) return rc;
    const Phys<double> P64 = make_phys<double>(st);
    int in_r = 0;
    if (st->coarse_fused) {
      // colour launches of 32-thread blocks: the float64 point updates of a
      // small level spread over all multiprocessors (GB300 issues few float64
      // operations per multiprocessor and clock)
      const Lvl<double> L64 = make_lvl_bufs<double>(st->lv64[l]);
      const int half = L64.g.N / 2;
      // CDFT: the chemical-potential part of the points a launch updates is
      // kept in M (the level's float64 r[0], unused by these sweeps) for the
      // next launch
      double* M = static_cast<double*>(st->lv64[l].r[0]);
      for (int it = 0; it < st->prm.ncoarse; ++it)
        for (int color = 0; color < 2; ++color) {
          if constexpr (KIND == KCDFT) {
            if (it == 0 && color == 0)
              k_smooth_cdft64_mc<DIM, false><<<(half + 31) / 32, 32, 0, st->stream>>>(L64, P64, color, M);
            else
              k_smooth_cdft64_mc<DIM, true><<<(half + 31) / 32, 32, 0, st->stream>>>(L64, P64, color, M);
          } else {
            k_smooth<double, KIND, DIM><<<(half + 31) / 32, 32, 0, st->stream>>>(L64, P64, color);
          }
          FM_LAUNCHED();
        }
    } else {
      SmallLv<double> S;
      S.count = st->nlev - l;
      for (int q = 0; q < S.count; ++q) S.lv[q] = make_lvl_bufs<double>(st->lv64[l + q]);
      rc = Solver<double, KIND, DIM>::small_cycle(st, S, P64);
    }
    if (rc) return rc;
    return coarse_from64(st, l, in_r);
  }

  static int vcycle(fm_state* st, int l, const Phys<T>& P, int* out_in_r) {
    cudaStream_t s = st->stream;
    *out_in_r = 0;
    if constexpr (sizeof(T) == 4) {
      if (l >= st->small_from && st->coarse64) return coarse_solve64(st, l);
    }
    if (l >= st->small_from && st->coarse_fused) {  // the coarsest level: ncoarse fused sweeps
      return smooth(st, l, P, st->prm.ncoarse, out_in_r);
    }
    if (l >= st->small_from) {
      SmallLv<T> S;
      S.count = st->nlev - l;
      for (int q = 0; q < S.count; ++q) S.lv[q] = make_lvl<T>(st, l + q);
      return small_cycle(st, S, P);
    }
    // The correction of level l may sit in its r buffer between the pre- and
    // the post-smoothing (after an odd number of fused launches); the
    // residual, restriction and prolongation then use the exchanged view.
    int in_r = 0;
    int rc = smooth(st, l, P, st->prm.nu1, &in_r);
    if (rc) return rc;
    Lvl<T> F = make_lvl<T>(st, l);
    if (in_r) F = swap_er(F);
    Lvl<T> C = make_lvl<T>(st, l + 1);
    if constexpr (DIM == 2) {
      const int ntx = (C.g.nx + RR_TX - 1) / RR_TX, nty = (C.g.ny + RR_TY - 1) / RR_TY;
      k_resid_restrict2<T, KIND><<<ntx * nty, TPB, 0, s>>>(F, C, P, ntx);
      FM_LAUNCHED();
    } else {
      k_resid<T, KIND, DIM><<<nblocks(F.g.N), TPB, 0, s>>>(F, P);
      FM_LAUNCHED();
      k_restrict_rhs<T, KIND, DIM><<<nblocks(C.g.N), TPB, 0, s>>>(F, C, P);
      FM_LAUNCHED();
    }
    int c_in_r = 0;
    rc = vcycle(st, l + 1, P, &c_in_r);
    if (rc) return rc;
    k_prolong<T, LY::NU, DIM><<<nblocks(F.g.N), TPB, 0, s>>>(F, c_in_r ? swap_er(C) : C, P);
    FM_LAUNCHED();
    rc = smooth(st, l, P, st->prm.nu2, &in_r);
    if (rc) return rc;
    *out_in_r = in_r;
    return FM_OK;
  }

  static int enqueue_body(fm_state* st, cudaGraphConditionalHandle hdl, int use_handle) {
    int rc = inject_all(st, true);
    if (rc) return rc;
    Phys<T> P = make_phys<T>(st);
    int in_r = 0;
    rc = vcycle(st, 0, P, &in_r);
    if (rc) return rc;
    if (in_r) {  // the float64 update reads the level-0 correction from e
      k_copy_back<T, LY::NU><<<nblocks(st->lv[0].g.N), TPB, 0, st->stream>>>(make_lvl<T>(st, 0));
      FM_LAUNCHED();
    }
    if constexpr (DIM == 2) {  // (3-D: the residual's first pass makes the update)
      const Geo G = st->lv[0].g;
      Fields64 F = make_fields(st);
      Resid64Out O = resid_out(st, true, nullptr);
      k_update64<LY::NU, T><<<nblocks(G.N), TPB, 0, st->stream>>>(F, O, G.N, st->prm.delta);
      FM_LAUNCHED();
    }
    return enqueue_resid_norm(st, 1, hdl, use_handle);
  }

  static int enqueue_post(fm_state* st) {
    const Geo G = st->lv[0].g;
    Fields64 F = make_fields(st);
    Phys<double> P64 = make_phys<double>(st);
    const Ctl* ctl = (const Ctl*)st->ctl;
    k_closure<DIM><<<nblocks(G.N), TPB, 0, st->stream>>>(F, G, make_step64(P64, 1.0 / st->lv[0].h), P64, st->tmp,
                                                         ctl);
    FM_LAUNCHED();
    Vel3W vw{{st->vel[0], st->vel[1], st->vel[2]}};
    Vel3 gv{{st->g[1], st->g[2], DIM == 3 ? st->g[3] : nullptr}};
    k_commit<DIM><<<nblocks(G.N), TPB, 0, st->stream>>>(st->rho, vw, st->tmp, gv, G.N, ctl);
    FM_LAUNCHED();
    if (st->prm.init == FM_INIT_EXTRAPOLATE) {
      k_hist_advance<<<1, 32, 0, st->stream>>>((Ctl*)st->ctl);
      FM_LAUNCHED();
    }
    FM_CUDA(cudaMemcpyAsync(st->hscal + 32, st->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st->stream));
    return FM_OK;
  }

  static int step(fm_state* st, fm_step_info* info) { return Stepper<Solver>::step(st, info); }
  static int step_host(fm_state* st, const double* rho_in, const double* const* vel_in, double* rho_out,
                       double* const* vel_out, fm_step_info* info) {
    return Stepper<Solver>::step_host(st, rho_in, vel_in, rho_out, vel_out, info);
  }
};

template <typename T>
static int dispatch_step(fm_state* st, fm_step_info* info) {
  if (st->kind == FM_PFC) {
    return st->dim == 2 ? Solver<T, KPFC, 2>::step(st, info) : Solver<T, KPFC, 3>::step(st, info);
  }
  return st->dim == 2 ? Solver<T, KCDFT, 2>::step(st, info) : Solver<T, KCDFT, 3>::step(st, info);
}

template <typename T>
static int dispatch_step_host(fm_state* st, const double* ri, const double* const* vi, double* ro,
                              double* const* vo, fm_step_info* info) {
  if (st->kind == FM_PFC) {
    return st->dim == 2 ? Solver<T, KPFC, 2>::step_host(st, ri, vi, ro, vo, info)
                        : Solver<T, KPFC, 3>::step_host(st, ri, vi, ro, vo, info);
  }
  return st->dim == 2 ? Solver<T, KCDFT, 2>::step_host(st, ri, vi, ro, vo, info)
                      : Solver<T, KCDFT, 3>::step_host(st, ri, vi, ro, vo, info);
}

template <typename T>
static int dispatch_autotune(fm_state* st) {
  if (st->kind == FM_PFC)
    return st->dim == 2 ? Solver<T, KPFC, 2>::autotune(st) : Solver<T, KPFC, 3>::autotune(st);
  return st->dim == 2 ? Solver<T, KCDFT, 2>::autotune(st) : Solver<T, KCDFT, 3>::autotune(st);
}

template <typename T>
static int dispatch_prepare(fm_state* st) {
  if (st->kind == FM_PFC)
    return st->dim == 2 ? Solver<T, KPFC, 2>::prepare(st) : Solver<T, KPFC, 3>::prepare(st);
  return st->dim == 2 ? Solver<T, KCDFT, 2>::prepare(st) : Solver<T, KCDFT, 3>::prepare(st);
}

template <typename T>
static int dispatch_smooth_row(fm_state* st, double* const* e, const double* const* f, int sweeps, int variant,
                               int where) {
  if (st->kind == FM_PFC)
    return st->dim == 2 ? Solver<T, KPFC, 2>::smooth_row(st, e, f, sweeps, variant, where)
                        : Solver<T, KPFC, 3>::smooth_row(st, e, f, sweeps, variant, where);
  return st->dim == 2 ? Solver<T, KCDFT, 2>::smooth_row(st, e, f, sweeps, variant, where)
                      : Solver<T, KCDFT, 3>::smooth_row(st, e, f, sweeps, variant, where);
}

template <typename T>
static int dispatch_resid(fm_state* st, double* const* r, double* nr) {
  if (st->kind == FM_PFC)
    return st->dim == 2 ? Solver<T, KPFC, 2>::residual64(st, r, nr) : Solver<T, KPFC, 3>::residual64(st, r, nr);
  return st->dim == 2 ? Solver<T, KCDFT, 2>::residual64(st, r, nr) : Solver<T, KCDFT, 3>::residual64(st, r, nr);
}

// --------------------------------------------------------------------------
// Set-up
// --------------------------------------------------------------------------
static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Carver {
  char* base;
  size_t off;
  void* take(size_t bytes) {
    void* p = base ? (void*)(base + off) : nullptr;
    off += align256(bytes);
    return p;
  }
};

// Lay out every buffer; with base == nullptr only measures.
static size_t carve(fm_state* st, char* base) {
  Carver C{base, 0};
  const int N0 = st->lv[0].g.N;
  const size_t d8 = sizeof(double);
  const size_t es = (size_t)st->elem;
  st->rho = (double*)C.take(N0 * d8);
  for (int d = 0; d < 3; ++d) st->vel[d] = d < st->dim ? (double*)C.take(N0 * d8) : nullptr;
  for (int q = 0; q < MAXU; ++q) {
    st->g[q] = q < st->nu ? (double*)C.take(N0 * d8) : nullptr;
    st->S[q] = q < st->nu ? (double*)C.take(N0 * d8) : nullptr;
    st->gp[q] = (q < st->nu && st->prm.init == FM_INIT_EXTRAPOLATE) ? (double*)C.take(N0 * d8) : nullptr;
  }
  for (int d = 0; d < 3; ++d) st->om[d] = d < st->nom ? (double*)C.take(N0 * d8) : nullptr;
  st->conv = st->kind == FM_CDFT ? (double*)C.take(N0 * d8) : nullptr;
  st->emu = (st->kind == FM_CDFT && st->model == FM_GRADFLOW) ? (double*)C.take(N0 * d8) : nullptr;
  st->tmp = (double*)C.take(N0 * d8);
  for (int q = 0; q < MAXU; ++q) st->r64[q] = q < st->nu ? (double*)C.take(N0 * d8) : nullptr;
  for (int q = 0; q < 5; ++q)
    st->x64[q] = (st->model == FM_HYDRO && st->dim == 3 && (q < 4 || st->kind == FM_CDFT))
                     ? (double*)C.take(N0 * d8)
                     : nullptr;
  st->partials = (double*)C.take((size_t)st->nblk * 8 * d8);
  st->dscal = (double*)C.take(64 * d8);
  st->ctl = C.take(64);
  for (int l = 0; l < st->nlev; ++l) {
    LevelBufs& B = st->lv[l];
    const size_t N = B.g.N;
    for (int q = 0; q < MAXU; ++q) {
      B.e[q] = q < st->nu ? C.take(N * es) : nullptr;
      B.f[q] = q < st->nu ? C.take(N * es) : nullptr;
      B.r[q] = q < st->nu ? C.take(N * es) : nullptr;  // also the second buffer of the fused sweep
      B.eh[q] = (q < st->nu && l > 0) ? C.take(N * es) : nullptr;
    }
    const bool alias = (l == 0 && st->prm.precision == FM_FP64);
    const int nvel = st->model == FM_HYDRO ? st->dim : 0;  // velocity coefficients
    if (alias) {
      B.rk = st->rho;
      B.cr = st->g[0];
      for (int d = 0; d < 3; ++d) {
        B.om[d] = st->om[d];
        B.cv[d] = d < nvel ? st->g[1 + d] : nullptr;
      }
    } else {
      B.rk = st->model == FM_HYDRO ? C.take(N * es) : nullptr;
      B.cr = C.take(N * es);
      for (int d = 0; d < 3; ++d) {
        B.om[d] = d < st->nom ? C.take(N * es) : nullptr;
        B.cv[d] = d < nvel ? C.take(N * es) : nullptr;
      }
    }
  }
  // float64 copies of the coarse levels (mixed path, coarsest solve in
  // float64): e, f, r, eh and the coefficients of levels small_from ..
  // nlev - 1 (the entry level's eh stays in the float32 level: the
  // prolongation reads it; a multi-block coarsest level's r[0] holds the
  // CDFT chemical-potential parts of its colour launches)
  for (int l = 0; l < MAXLEV; ++l) st->lv64[l] = LevelBufs{};
  if (st->coarse64) {
    for (int l = st->small_from; l < st->nlev; ++l) {
      LevelBufs& B = st->lv64[l];
      B.g = st->lv[l].g;
      B.h = st->lv[l].h;
      const size_t N = B.g.N;
      for (int q = 0; q < MAXU; ++q) {
        B.e[q] = q < st->nu ? C.take(N * d8) : nullptr;
        B.f[q] = q < st->nu ? C.take(N * d8) : nullptr;
        B.r[q] = q < st->nu ? C.take(N * d8) : nullptr;
        B.eh[q] = (q < st->nu && l > st->small_from) ? C.take(N * d8) : nullptr;
      }
      B.rk = C.take(N * d8);
      B.cr = C.take(N * d8);
      for (int d = 0; d < 3; ++d) {
        B.om[d] = d < st->nom ? C.take(N * d8) : nullptr;
        B.cv[d] = d < st->dim ? C.take(N * d8) : nullptr;
      }
    }
  }
  if (st->kind == FM_CDFT) {
    st->fft.Jhat = (double2*)C.take(N0 * sizeof(double2));
    st->fft.work = (double2*)C.take(N0 * sizeof(double2));
    const int ns[3] = {st->lv[0].g.nx, st->lv[0].g.ny, st->lv[0].g.nz};
    st->fft.Jr = (double*)C.take((size_t)(ns[0] / 2 + 1) * ns[1] * ns[2] * sizeof(double));
    for (int d = 0; d < 3; ++d)
      st->fft.tw[d] = d < st->dim ? (double2*)C.take((size_t)(ns[d] / 2 + 1) * sizeof(double2)) : nullptr;
  }
  return C.off;
}

}  // namespace fm

using namespace fm;

// Forget the converged iterates kept for FM_INIT_EXTRAPOLATE (stream-ordered).
static int reset_history(fm_state* st) {
  if (st->prm.init != FM_INIT_EXTRAPOLATE) return FM_OK;
  FM_CUDA(cudaMemsetAsync(&static_cast<Ctl*>(st->ctl)->hist, 0, sizeof(int), st->stream));
  return FM_OK;
}

// A step of another size than the kept iterates' starts without them.
static int check_history_dt(fm_state* st, double dt) {
  if (st->prm.init != FM_INIT_EXTRAPOLATE || st->hist_dt == dt) return FM_OK;
  st->hist_dt = dt;
  return reset_history(st);
}

extern "C" {

void fm_default_params(fm_params* p) {
  if (!p) return;
  p->gamma = 2.0;
  p->w_damp = 0.5;
  p->delta = 0.0;
  p->tol = 1e-10;
  p->sigma = 1.0;
  p->nu1 = 2;
  p->nu2 = 2;
  p->max_cycles = 50;
  p->coarsest = 16;
  p->ncoarse = 4;
  p->precision = FM_FP64;
  p->model = FM_HYDRO;
  p->walls = FM_WALLS_NONE;
  p->u_wall[0] = p->u_wall[1] = 0.0;
  p->init = FM_INIT_PREVIOUS;
  p->coarse_precision = FM_FP64;
}

const char* fm_strerror(int code) {
  switch (code) {
    case FM_OK: return "ok";
    case FM_EINVAL: return "invalid argument";
    case FM_ENOMEM: return "device allocation failed";
    case FM_ECUDA: return "CUDA runtime error";
    case FM_ENOCONV: return "no convergence within max_cycles";
    case FM_ENONPOS: return "non-positive density";
    case FM_ENAN: return "non-finite residual";
    case FM_ETIMEOUT: return "a bounded wait inside a kernel ran out";
    default: return "unknown error";
  }
}

int fm_create(const fm_grid* grid, const fm_params* prm, const fm_functional* fn, fm_state** out) {
  if (!grid || !prm || !fn || !out) return FM_EINVAL;
  *out = nullptr;
  if (grid->dim != 2 && grid->dim != 3) return FM_EINVAL;
  if (!(grid->h > 0.0)) return FM_EINVAL;
  if (fn->kind != FM_PFC && fn->kind != FM_CDFT) return FM_EINVAL;
  if (fn->kind == FM_CDFT && !(fn->nu > 0.0)) return FM_EINVAL;
  if (prm->precision != FM_FP64 && prm->precision != FM_MIXED) return FM_EINVAL;
  if (prm->model != FM_HYDRO && prm->model != FM_GRADFLOW) return FM_EINVAL;
  if (prm->walls != FM_WALLS_NONE && prm->walls != FM_WALLS_Y) return FM_EINVAL;
  if (prm->walls == FM_WALLS_Y &&
      (grid->dim != 2 || fn->kind != FM_PFC || prm->model != FM_HYDRO ||
       !(prm->u_wall[0] == prm->u_wall[0]) || !(prm->u_wall[1] == prm->u_wall[1])))
    return FM_EINVAL;  // walls: the 2-D hydrodynamic PFC channel only
  if (prm->init != FM_INIT_PREVIOUS && prm->init != FM_INIT_EXTRAPOLATE) return FM_EINVAL;
  if (prm->coarse_precision != FM_FP64 && prm->coarse_precision != FM_MIXED) return FM_EINVAL;
  if (prm->init == FM_INIT_EXTRAPOLATE && (prm->model != FM_HYDRO || prm->walls != FM_WALLS_NONE))
    return FM_EINVAL;  // the periodic hydrodynamic solver only
  if (prm->nu1 < 0 || prm->nu2 < 0 || prm->nu1 + prm->nu2 < 1 || prm->ncoarse < 1 || prm->max_cycles < 0)
    return FM_EINVAL;
  if (!(prm->w_damp >= 0.0 && prm->w_damp < 1.0) || !(prm->gamma >= 0.0) || !(prm->tol > 0.0) ||
      !(prm->delta >= 0.0) || prm->coarsest < 2)
    return FM_EINVAL;
  long long N = 1;
  for (int d = 0; d < grid->dim; ++d) {
    const int n = grid->n[d];
    if (n < 2 || (n & 1)) return FM_EINVAL;
    N *= n;
  }
  if (N > (1LL << 30)) return FM_EINVAL;
  if (fn->kind == FM_CDFT) {
    for (int d = 0; d < grid->dim; ++d) {
      const int n = grid->n[d];
      if ((n & (n - 1)) != 0 || n > 4096) return FM_EINVAL;  // power-of-two FFT
    }
  }
  fm_state* st = new (std::nothrow) fm_state();
  if (!st) return FM_ENOMEM;
  st->grid = *grid;
  st->prm = *prm;
  st->fn = *fn;
  st->kind = fn->kind;
  st->model = prm->model;
  st->dim = grid->dim;
  if (st->model == FM_GRADFLOW) {
    st->nu = fn->kind == FM_PFC ? 3 : 1;  // (rho, mu, kappa) or rho
    st->nom = 0;
  } else {
    st->nu = 1 + grid->dim + (fn->kind == FM_PFC ? 2 : 0);
    st->nom = grid->dim == 2 ? 1 : 3;
  }
  st->elem = prm->precision == FM_MIXED ? (int)sizeof(float) : (int)sizeof(double);
  st->stream = 0;
  // hierarchy
  int nlev = 0;
  Geo g{grid->n[0], grid->n[1], grid->dim == 3 ? grid->n[2] : 1, 0};
  double h = grid->h;
  for (;;) {
    g.N = g.nx * g.ny * g.nz;
    st->lv[nlev].g = g;
    st->lv[nlev].h = h;
    ++nlev;
    bool can = nlev < MAXLEV;
    const int ns[3] = {g.nx, g.ny, g.nz};
    for (int d = 0; d < grid->dim; ++d) {
      const int hn = ns[d] / 2;
      if ((ns[d] & 1) || hn < prm->coarsest || (hn & 1)) can = false;
    }
    if (!can) break;
    g.nx /= 2;
    g.ny /= 2;
    if (grid->dim == 3) g.nz /= 2;
    h *= 2.0;
  }
  st->nlev = nlev;
  st->small_from = nlev - 1;
  for (int l = 0; l < nlev; ++l)
    if (st->lv[l].g.N <= SMALL_N && nlev - l <= MAXSMALL) {
      st->small_from = l;
      break;
    }
  {
    const char* eg = getenv("FM_GRAPH");
    st->use_graph = !(eg && eg[0] == '0');
    const char* ef = getenv("FM_FUSED_RB");
    st->fused_rb = !(ef && ef[0] == '0');
  }
  // A coarsest level that is the only level of the single-block part and
  // larger than SMALL_N points is smoothed by multi-block sweeps instead (the
  // fused sweeps in 2-D, a red and a black launch per sweep in 3-D or without
  // fusion); one block would run its points serially.
  st->coarse_fused = st->small_from == nlev - 1 && st->lv[nlev - 1].g.N > SMALL_N;
  st->coarse64 = st->prm.precision == FM_MIXED && st->prm.coarse_precision == FM_FP64 &&
                 st->model == FM_HYDRO && st->prm.walls == FM_WALLS_NONE;
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    delete st;
    return FM_ECUDA;
  }
  st->sms = sms;
  if (cudaDeviceGetAttribute(&st->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    cudaGetLastError();
    delete st;
    return FM_ECUDA;
  }
  const int need = (int)((st->lv[0].g.N + TPB - 1) / TPB);
  st->nblk = need < 4 * sms ? need : 4 * sms;
  const size_t bytes = carve(st, nullptr);
  void* arena = nullptr;
  if (cudaMalloc(&arena, bytes) != cudaSuccess) {
    cudaGetLastError();
    delete st;
    return FM_ENOMEM;
  }
  st->arena = arena;
  st->arena_bytes = bytes;
  carve(st, (char*)arena);
  if (cudaMallocHost((void**)&st->hscal, 64 * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(arena);
    delete st;
    return FM_ENOMEM;
  }
  if (cudaMemset(arena, 0, bytes) != cudaSuccess) {
    cudaGetLastError();
    fm_destroy(st);
    return FM_ECUDA;
  }
  if (cudaStreamCreateWithFlags(&st->cap[0], cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&st->cap[1], cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    fm_destroy(st);
    return FM_ECUDA;
  }
  st->ce = 0.0;
  if (st->kind == FM_CDFT) {
    const int rc = fft_init(st);
    if (rc) {
      fm_destroy(st);
      return rc;
    }
  }
  if (st->model == FM_HYDRO && prm->walls == FM_WALLS_NONE) {
    const int rc = prm->precision == FM_MIXED ? dispatch_autotune<float>(st) : dispatch_autotune<double>(st);
    if (rc) {
      fm_destroy(st);
      return rc;
    }
  }
  if (cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    fm_destroy(st);
    return FM_ECUDA;
  }
  st->prepared = false;
  st->dt = 0.0;
  *out = st;
  return FM_OK;
}

void fm_destroy(fm_state* st) {
  if (!st) return;
  if (st->gexec) cudaGraphExecDestroy(st->gexec);
  if (st->graph) cudaGraphDestroy(st->graph);
  for (int i = 0; i < 2; ++i)
    if (st->cap[i]) cudaStreamDestroy(st->cap[i]);
  if (st->pev_ready)
    for (int i = 0; i < MAXEV; ++i) cudaEventDestroy(st->pev[i]);
  if (st->arena) cudaFree(st->arena);
  if (st->hscal) cudaFreeHost(st->hscal);
  delete st;
}

int fm_set_stream(fm_state* st, void* stream) {
  if (!st) return FM_EINVAL;
  st->stream = (cudaStream_t)stream;
  return FM_OK;
}

int fm_levels(const fm_state* st) { return st ? st->nlev : FM_EINVAL; }

int fm_tuning(const fm_state* st, int level, int* variant, float* ms_per_variant) {
  if (!st || level < 0 || level >= st->nlev) return FM_EINVAL;
  if (variant) *variant = st->rbv[level];
  if (ms_per_variant)
    for (int v = 0; v < RB_NVAR; ++v) ms_per_variant[v] = st->rbt[level][v];
  return FM_OK;
}

int fm_profile(fm_state* st, int enable) {
  if (!st) return FM_EINVAL;
  if (enable && !st->pev_ready) {
    for (int i = 0; i < MAXEV; ++i) FM_CUDA(cudaEventCreate(&st->pev[i]));
    st->pev_ready = true;
  }
  st->prof = enable != 0;
  st->npev = 0;
  st->prof_ms = 0.0;
  st->prof_count = 0;
  return FM_OK;
}

int fm_profile_read(const fm_state* st, double* smoother_ms, long long* smoother_launches,
                    long long* launches) {
  if (!st) return FM_EINVAL;
  if (smoother_ms) *smoother_ms = st->prof_ms;
  if (smoother_launches) *smoother_launches = st->prof_count;
  if (launches) *launches = st->launches;
  return FM_OK;
}

int fm_set_fields(fm_state* st, const double* rho, const double* const* vel, int where) {
  if (!st || !rho || (!vel && st->model == FM_HYDRO) || (where != FM_HOST && where != FM_DEVICE)) return FM_EINVAL;
  const size_t bytes = (size_t)st->lv[0].g.N * sizeof(double);
  {
    const int rc = reset_history(st);
    if (rc) return rc;
  }
  FM_CUDA(cudaMemcpyAsync(st->rho, rho, bytes, kind_in(where), st->stream));
  for (int d = 0; d < st->dim && st->model == FM_HYDRO; ++d) {  // the gradient flow keeps u = 0
    if (!vel[d]) return FM_EINVAL;
    FM_CUDA(cudaMemcpyAsync(st->vel[d], vel[d], bytes, kind_in(where), st->stream));
  }
  if (where == FM_HOST) FM_CUDA(cudaStreamSynchronize(st->stream));
  st->prepared = false;
  return FM_OK;
}

int fm_get_fields(fm_state* st, double* rho, double* const* vel, int where) {
  if (!st || (where != FM_HOST && where != FM_DEVICE)) return FM_EINVAL;
  const size_t bytes = (size_t)st->lv[0].g.N * sizeof(double);
  if (rho) FM_CUDA(cudaMemcpyAsync(rho, st->rho, bytes, kind_out(where), st->stream));
  if (vel)
    for (int d = 0; d < st->dim; ++d)
      if (vel[d]) FM_CUDA(cudaMemcpyAsync(vel[d], st->vel[d], bytes, kind_out(where), st->stream));
  if (where == FM_HOST) FM_CUDA(cudaStreamSynchronize(st->stream));
  return FM_OK;
}

int fm_step_host(fm_state* st, double dt, const double* rho_in, const double* const* vel_in, double* rho_out,
                 double* const* vel_out, fm_step_info* info) {
  if (st && st->model == FM_GRADFLOW) {
    if (!(dt > 0.0) || !rho_in || !rho_out) return FM_EINVAL;
    st->dt = dt;
    return gf_step_host(st, rho_in, rho_out, info);
  }
  if (!st || !(dt > 0.0) || !rho_in || !vel_in || !rho_out || !vel_out) return FM_EINVAL;
  if (st->prm.walls == FM_WALLS_Y) {
    for (int d = 0; d < 2; ++d)
      if (!vel_in[d] || !vel_out[d]) return FM_EINVAL;
    st->dt = dt;
    return ch_step_host(st, rho_in, vel_in, rho_out, vel_out, info);
  }
  {
    const int rc = check_history_dt(st, dt);
    if (rc) return rc;
  }
  for (int d = 0; d < st->dim; ++d)
    if (!vel_in[d] || !vel_out[d]) return FM_EINVAL;
  st->dt = dt;
  return st->prm.precision == FM_MIXED ? dispatch_step_host<float>(st, rho_in, vel_in, rho_out, vel_out, info)
                                       : dispatch_step_host<double>(st, rho_in, vel_in, rho_out, vel_out, info);
}

int fm_prepare(fm_state* st, double dt) {
  if (!st || !(dt > 0.0)) return FM_EINVAL;
  st->dt = dt;
  if (st->model == FM_GRADFLOW) return gf_prepare(st);
  if (st->prm.walls == FM_WALLS_Y) return ch_prepare(st);
  {
    const int rc = reset_history(st);  // the row call replaces the step's iterate
    if (rc) return rc;
  }
  return st->prm.precision == FM_MIXED ? dispatch_prepare<float>(st) : dispatch_prepare<double>(st);
}

int fm_step(fm_state* st, double dt, fm_step_info* info) {
  if (!st || !(dt > 0.0)) return FM_EINVAL;
  st->dt = dt;
  if (st->model == FM_GRADFLOW) return gf_step(st, info);
  if (st->prm.walls == FM_WALLS_Y) return ch_step(st, info);
  {
    const int rc = check_history_dt(st, dt);
    if (rc) return rc;
  }
  return st->prm.precision == FM_MIXED ? dispatch_step<float>(st, info) : dispatch_step<double>(st, info);
}

int fm_get_aux(fm_state* st, int what, int comp, double* out, int where) {
  if (!st || !out || (where != FM_HOST && where != FM_DEVICE)) return FM_EINVAL;
  const double* src = nullptr;
  switch (what) {
    case FM_AUX_OMEGA: if (comp >= 0 && comp < st->nom) src = st->om[comp]; break;
    case FM_AUX_SOURCE: if (comp >= 0 && comp < st->nu) src = st->S[comp]; break;
    case FM_AUX_CONV: if (comp == 0 && st->kind == FM_CDFT) src = st->conv; break;
    case FM_AUX_ITERATE: if (comp >= 0 && comp < st->nu) src = st->g[comp]; break;
    default: break;
  }
  if (!src) return FM_EINVAL;
  const size_t bytes = (size_t)st->lv[0].g.N * sizeof(double);
  FM_CUDA(cudaMemcpyAsync(out, src, bytes, kind_out(where), st->stream));
  FM_CUDA(cudaStreamSynchronize(st->stream));
  return FM_OK;
}

int fm_residual(fm_state* st, const double* const* g, double* const* r, double* norm, int where) {
  if (!st || !g || !norm || (where != FM_HOST && where != FM_DEVICE)) return FM_EINVAL;
  if (!st->prepared) return FM_EINVAL;
  const size_t bytes = (size_t)st->lv[0].g.N * sizeof(double);
  for (int q = 0; q < st->nu; ++q) {
    if (!g[q]) return FM_EINVAL;
    FM_CUDA(cudaMemcpyAsync(st->g[q], g[q], bytes, kind_in(where), st->stream));
  }
  {
    const int rc = reset_history(st);  // the caller's iterate replaced the converged one
    if (rc) return rc;
  }
  int rc = st->model == FM_GRADFLOW           ? gf_residual(st, st->r64, norm)
           : st->prm.walls == FM_WALLS_Y     ? ch_residual(st, st->r64, norm)
           : st->prm.precision == FM_MIXED   ? dispatch_resid<float>(st, st->r64, norm)
                                             : dispatch_resid<double>(st, st->r64, norm);
  if (rc == FM_OK && r) {
    for (int q = 0; q < st->nu; ++q)
      if (r[q]) FM_CUDA(cudaMemcpyAsync(r[q], st->r64[q], bytes, kind_out(where), st->stream));
    FM_CUDA(cudaStreamSynchronize(st->stream));
  }
  return rc;
}

int fm_smooth(fm_state* st, double* const* e, const double* const* f, int sweeps, int variant, int where) {
  if (!st || !e || !f || sweeps < 0 || (where != FM_HOST && where != FM_DEVICE)) return FM_EINVAL;
  if (st->model != FM_HYDRO || st->prm.walls != FM_WALLS_NONE) return FM_EINVAL;
  if (!st->prepared) return FM_EINVAL;
  for (int q = 0; q < st->nu; ++q)
    if (!e[q] || !f[q]) return FM_EINVAL;
  return st->prm.precision == FM_MIXED ? dispatch_smooth_row<float>(st, e, f, sweeps, variant, where)
                                       : dispatch_smooth_row<double>(st, e, f, sweeps, variant, where);
}

int fm_narrow(const double* in, float* out, long long n, void* stream) {
  if (!in || !out || n < 0) return FM_EINVAL;
  if (n == 0) return FM_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const long long nb = (n + TPB - 1) / TPB;
  if (nb > 0x7fffffffLL) return FM_EINVAL;
  k_narrow<<<(int)nb, TPB, 0, s>>>(in, out, n);
  if (cudaGetLastError() != cudaSuccess) return FM_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return FM_ECUDA;
  return FM_OK;
}

int fm_widen(const float* in, double* out, long long n, void* stream) {
  if (!in || !out || n < 0) return FM_EINVAL;
  if (n == 0) return FM_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const long long nb = (n + TPB - 1) / TPB;
  if (nb > 0x7fffffffLL) return FM_EINVAL;
  k_widen<<<(int)nb, TPB, 0, s>>>(in, out, n);
  if (cudaGetLastError() != cudaSuccess) return FM_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return FM_ECUDA;
  return FM_OK;
}

// Status word of fm_wait_selftest.
__device__ int g_wait_status;

// One block: an mbarrier of one arrival, completed by thread 0 or by nobody,
// then the bounded wait of the tensor-copy smoother in every thread.
__global__ void k_wait_selftest(int complete, unsigned long long limit_ns) {
  __shared__ __align__(8) unsigned long long bar;
  const unsigned b = smem_u32(&bar);
  if (threadIdx.x == 0) mbar_init(b, 1);
  __syncthreads();
  if (complete && threadIdx.x == 0) mbar_arrive(b);
  const bool ok = __syncthreads_and(mbar_wait(b, 0, limit_ns));
  if (threadIdx.x == 0) g_wait_status = ok ? FM_OK : FM_ETIMEOUT;
}

int fm_wait_selftest(int complete, int limit_us, void* stream) {
  if (limit_us < 1 || limit_us > 1000000) return FM_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const int unset = FM_ECUDA;
  if (cudaMemcpyToSymbolAsync(g_wait_status, &unset, sizeof(int), 0, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return FM_ECUDA;
  k_wait_selftest<<<1, 64, 0, s>>>(complete ? 1 : 0, 1000ull * (unsigned long long)limit_us);
  if (cudaGetLastError() != cudaSuccess) return FM_ECUDA;
  int status = FM_ECUDA;
  if (cudaMemcpyFromSymbolAsync(&status, g_wait_status, sizeof(int), 0, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return FM_ECUDA;
  return status;
}

// Grid barrier of fm_grid_barrier_selftest: counters, fault flag and status.
__device__ unsigned g_gbar_test[2];
__device__ int g_gbar_fault;
__device__ int g_gbar_status;

// A cooperative launch of every resident block of k_smooth_coop's size; each
// arrives once at the barrier of the cooperative sweep and waits for one
// arrival of every block (complete = 1, reached) or for two (never reached).
__global__ void __launch_bounds__(TPB) k_grid_barrier_selftest(int complete, unsigned long long limit_ns) {
  const bool ok = grid_barrier(g_gbar_test, complete ? 1u : 2u, &g_gbar_fault, limit_ns);
  if (!ok) {
    if (threadIdx.x == 0) atomicExch(&g_gbar_status, FM_ETIMEOUT);
    return;
  }
  grid_barrier_leave(g_gbar_test);
}

int fm_grid_barrier_selftest(int complete, int limit_us, void* stream) {
  if (limit_us < 1 || limit_us > 1000000) return FM_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_grid_barrier_selftest, TPB, 0) != cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    return FM_ECUDA;
  }
  const unsigned zero2[2] = {0u, 0u};
  const int zero = 0, ok = FM_OK;
  if (cudaMemcpyToSymbolAsync(g_gbar_test, zero2, sizeof(zero2), 0, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyToSymbolAsync(g_gbar_fault, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyToSymbolAsync(g_gbar_status, &ok, sizeof(int), 0, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return FM_ECUDA;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(per_sm * sms);
  cfg.blockDim = dim3(TPB);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (cudaLaunchKernelEx(&cfg, k_grid_barrier_selftest, complete ? 1 : 0, 1000ull * (unsigned long long)limit_us) !=
      cudaSuccess) {
    cudaGetLastError();
    return FM_ECUDA;
  }
  int status = FM_ECUDA;
  if (cudaMemcpyFromSymbolAsync(&status, g_gbar_status, sizeof(int), 0, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return FM_ECUDA;
  return status;
}

// Weighted energy sums of the current state into q[0..4]: KE, then the PFC
// terms or F_id, F_ex (CDFT; q[3] = q[4] = 0).
static int energy_sums(fm_state* st, double* q) {
  const Geo G = st->lv[0].g;
  const double h = st->lv[0].h;
  cudaStream_t s = st->stream;
  if (st->kind == FM_CDFT) {
    const int rc = fft_convolve(st, st->rho, st->tmp);
    if (rc) return rc;
  }
  Vel3 v3{{st->vel[0], st->vel[1], st->vel[2]}};
  const double a = st->fn.alpha;
  if (st->prm.walls == FM_WALLS_Y) {
    const int rc = ch_energy_launch(st);
    if (rc) return rc;
    ++st->launches;
  } else if (st->kind == FM_PFC && st->dim == 2)
    k_energy<KPFC, 2><<<st->nblk, TPB, 0, s>>>(st->rho, v3, nullptr, G, h, a, st->partials);
  else if (st->kind == FM_PFC)
    k_energy<KPFC, 3><<<st->nblk, TPB, 0, s>>>(st->rho, v3, nullptr, G, h, a, st->partials);
  else if (st->dim == 2)
    k_energy<KCDFT, 2><<<st->nblk, TPB, 0, s>>>(st->rho, v3, st->tmp, G, h, a, st->partials);
  else
    k_energy<KCDFT, 3><<<st->nblk, TPB, 0, s>>>(st->rho, v3, st->tmp, G, h, a, st->partials);
  if (st->prm.walls != FM_WALLS_Y) FM_LAUNCHED();
  k_final_sum<5><<<1, TPB, 0, s>>>(st->partials, st->nblk, st->dscal + 8);
  FM_LAUNCHED();
  FM_CUDA(cudaMemcpyAsync(st->hscal + 8, st->dscal + 8, 5 * sizeof(double), cudaMemcpyDeviceToHost, s));
  FM_CUDA(cudaStreamSynchronize(s));
  const double w = st->dim == 3 ? h * h * h : h * h;
  for (int t = 0; t < 5; ++t) q[t] = w * st->hscal[8 + t];
  return FM_OK;
}

int fm_energy(fm_state* st, double* E, double* F, double* KE) {
  if (!st) return FM_EINVAL;
  double q[5];
  const int rc = energy_sums(st, q);
  if (rc) return rc;
  const double f = q[1] + q[2] + q[3] + q[4];
  if (E) *E = q[0] + f;
  if (F) *F = f;
  if (KE) *KE = q[0];
  return FM_OK;
}

int fm_energy_terms(fm_state* st, double* terms) {
  if (!st || !terms) return FM_EINVAL;
  return energy_sums(st, terms);
}

int fm_mass(fm_state* st, double* M) {
  if (!st || !M) return FM_EINVAL;
  const Geo G = st->lv[0].g;
  const double h = st->lv[0].h;
  cudaStream_t s = st->stream;
  k_mass<<<st->nblk, TPB, 0, s>>>(st->rho, G.N, st->partials);
  FM_LAUNCHED();
  k_final_sum<1><<<1, TPB, 0, s>>>(st->partials, st->nblk, st->dscal + 16);
  FM_LAUNCHED();
  FM_CUDA(cudaMemcpyAsync(st->hscal + 16, st->dscal + 16, sizeof(double), cudaMemcpyDeviceToHost, s));
  FM_CUDA(cudaStreamSynchronize(s));
  const double w = st->dim == 3 ? h * h * h : h * h;
  *M = w * st->hscal[16];
  return FM_OK;
}

int fm_convolve(fm_state* st, const double* rho, double* out, int where) {
  if (!st || !rho || !out || st->kind != FM_CDFT || (where != FM_HOST && where != FM_DEVICE))
    return FM_EINVAL;
  const size_t bytes = (size_t)st->lv[0].g.N * sizeof(double);
  FM_CUDA(cudaMemcpyAsync(st->tmp, rho, bytes, kind_in(where), st->stream));
  const int rc = fft_convolve(st, st->tmp, st->r64[0]);
  if (rc) return rc;
  FM_CUDA(cudaMemcpyAsync(out, st->r64[0], bytes, kind_out(where), st->stream));
  FM_CUDA(cudaStreamSynchronize(st->stream));
  return FM_OK;
}

int fm_restrict(fm_state* st, const double* fine, double* coarse, int where) {
  if (!st || !fine || !coarse || st->nlev < 2 || (where != FM_HOST && where != FM_DEVICE)) return FM_EINVAL;
  const Geo F = st->lv[0].g, C = st->lv[1].g;
  FM_CUDA(cudaMemcpyAsync(st->tmp, fine, (size_t)F.N * sizeof(double), kind_in(where), st->stream));
  k_restrict_one<<<nblocks(C.N), TPB, 0, st->stream>>>(st->tmp, st->r64[0], F, C, st->dim);
  FM_LAUNCHED();
  FM_CUDA(cudaMemcpyAsync(coarse, st->r64[0], (size_t)C.N * sizeof(double), kind_out(where), st->stream));
  FM_CUDA(cudaStreamSynchronize(st->stream));
  return FM_OK;
}

int fm_prolong_add(fm_state* st, const double* coarse, double* fine, int where) {
  if (!st || !fine || !coarse || st->nlev < 2 || (where != FM_HOST && where != FM_DEVICE)) return FM_EINVAL;
  const Geo F = st->lv[0].g, C = st->lv[1].g;
  FM_CUDA(cudaMemcpyAsync(st->r64[0], coarse, (size_t)C.N * sizeof(double), kind_in(where), st->stream));
  FM_CUDA(cudaMemcpyAsync(st->tmp, fine, (size_t)F.N * sizeof(double), kind_in(where), st->stream));
  k_prolong_one<<<nblocks(F.N), TPB, 0, st->stream>>>(st->r64[0], st->tmp, F, C, st->dim);
  FM_LAUNCHED();
  FM_CUDA(cudaMemcpyAsync(fine, st->tmp, (size_t)F.N * sizeof(double), kind_out(where), st->stream));
  FM_CUDA(cudaStreamSynchronize(st->stream));
  return FM_OK;
}

}  // extern "C"
