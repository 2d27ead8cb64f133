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
#include <cuda_runtime.h>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <cmath>
#include <new>

#include "fm_state.h"

namespace fm {

constexpr int TPB = 256;

static inline int nblocks(long long work) { return (int)((work + TPB - 1) / TPB); }

// --------------------------------------------------------------------------
// Smoother point update (correction form)
// --------------------------------------------------------------------------
template <typename T, int KIND, int DIM>
__device__ __forceinline__ void smooth_point(const Lvl<T>& L, const Phys<T>& P, const Nb& n) {
  using LY = Layout<KIND, DIM>;
  T* const* E = L.e;
  const T ih = T(1) / L.h;
  const T ih2 = ih * ih;
  const int c = n.c;
  const T rkc = L.rk[c];
  const T crc = L.cr[c];
  T eo[LY::NU];
#pragma unroll
  for (int q = 0; q < LY::NU; ++q) eo[q] = E[q][c];

  // rho from the continuity row (neighbour velocities only)
  T div = 0;
#pragma unroll
  for (int d = 0; d < DIM; ++d)
    div += L.rk[n.p[d]] * E[1 + d][n.p[d]] - L.rk[n.m[d]] * E[1 + d][n.m[d]];
  T er = L.f[0][c] - P.s * T(0.25) * ih * div;
  {
    const T x = crc + er;
    if (x <= T(0)) er = sqrt_t(x * x + P.delta * P.delta) - crc;  // Sec. 6 projection
  }
  T eg[LY::NU];
  eg[0] = er;

  if constexpr (KIND == KPFC) {
    // kappa = f5 + Lap_h e_rho with the new centre value
    const T ek = L.f[LY::IKA][c] + (nbsum<T, DIM>(E[0], n) - T(2 * DIM) * er) * ih2;
    // mu = f4 + [(p+e)^3 - p^3]/3 + alpha e + Lap_h e_kappa (exact: the block is triangular)
    const T psi = crc - T(1.5);
    const T em = L.f[LY::IMU][c] + er * (psi * psi + psi * er + er * er / T(3)) + P.alpha * er
               + (nbsum<T, DIM>(E[LY::IKA], n) - T(2 * DIM) * ek) * ih2;
    eg[LY::IKA] = ek;
    eg[LY::IMU] = em;
  }

  // velocity block: (a I + [b]_x) e_u = rhs
  T rhs[3];
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    const T dq = qcorr<T, DIM>(E, L.cv, n.p[a]) - qcorr<T, DIM>(E, L.cv, n.m[a]);
    const T dm = mcorr<T, KIND, DIM>(E, L.cr, n.p[a], P.ce) - mcorr<T, KIND, DIM>(E, L.cr, n.m[a], P.ce);
    rhs[a] = L.f[1 + a][c] - P.s * rkc * ih * (T(0.25) * dq + T(0.5) * dm)
           + T(0.5) * P.s * P.gamma * ih2 * nbsum<T, DIM>(E[1 + a], n);
  }
  const T A = rkc + P.s * P.gamma * T(DIM) * ih2;
  const T bs = T(0.5) * P.sigma * P.s * rkc;
  if constexpr (DIM == 2) {
    const T b = bs * L.om[0][c];
    const T inv = T(1) / (A * A + b * b);
    eg[1] = (A * rhs[0] + b * rhs[1]) * inv;
    eg[2] = (A * rhs[1] - b * rhs[0]) * inv;
  } else {
    T b[3], bx[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) b[d] = bs * L.om[d][c];
    cross<T, 3>(b, rhs, bx);
    const T bdy = b[0] * rhs[0] + b[1] * rhs[1] + b[2] * rhs[2];
    const T inv = T(1) / (A * (A * A + b[0] * b[0] + b[1] * b[1] + b[2] * b[2]));
#pragma unroll
    for (int d = 0; d < 3; ++d) eg[1 + d] = (A * A * rhs[d] - A * bx[d] + bdy * b[d]) * inv;
  }
  // damping of the whole point block (App. G.3)
  const T w = P.w;
#pragma unroll
  for (int q = 0; q < LY::NU; ++q) E[q][c] = (T(1) - w) * eg[q] + w * eo[q];
}

// --------------------------------------------------------------------------
// Point operations of one level (shared by the per-level kernels and the
// single-block small-level V-cycle)
// --------------------------------------------------------------------------
template <typename T, int KIND, int DIM>
__device__ __forceinline__ void resid_point(const Lvl<T>& L, const Phys<T>& P, int idx) {
  using LY = Layout<KIND, DIM>;
  int i, j, k;
  coords(idx, L.g, i, j, k);
  const Nb n = neighbours(i, j, k, L.g);
  T M[LY::NU];
  applyM<T, KIND, DIM>(L, P, n, L.e, M);
#pragma unroll
  for (int q = 0; q < LY::NU; ++q) L.r[q][idx] = L.f[q][idx] - M[q];
}

// coarse point idx: f_C = FW(r_F); e_C = eh_C = inject(e_F)
template <typename T, int NU, int DIM>
__device__ __forceinline__ void restrict_point(const Lvl<T>& F, const Lvl<T>& C, int idx) {
  int I, J, K;
  coords(idx, C.g, I, J, K);
  const int fi = 2 * I, fj = 2 * J, fk = 2 * K;
  const int ctr = (fk * F.g.ny + fj) * F.g.nx + fi;
  int xs[3], ys[3], zs[3];
  xs[0] = (fi == 0 ? F.g.nx - 1 : fi - 1); xs[1] = fi; xs[2] = (fi + 1 == F.g.nx ? 0 : fi + 1);
  ys[0] = (fj == 0 ? F.g.ny - 1 : fj - 1); ys[1] = fj; ys[2] = (fj + 1 == F.g.ny ? 0 : fj + 1);
  if constexpr (DIM == 3) {
    zs[0] = (fk == 0 ? F.g.nz - 1 : fk - 1); zs[1] = fk; zs[2] = (fk + 1 == F.g.nz ? 0 : fk + 1);
  } else {
    zs[0] = zs[1] = zs[2] = 0;
  }
  constexpr int KZ = (DIM == 3) ? 3 : 1;
  const T norm = (DIM == 3) ? T(1.0 / 64.0) : T(1.0 / 16.0);
#pragma unroll
  for (int q = 0; q < NU; ++q) {
    T acc = 0;
#pragma unroll
    for (int c = 0; c < KZ; ++c) {
      const int zz = (DIM == 3) ? zs[c] : 0;
      const T wz = (DIM == 3) ? (c == 1 ? T(2) : T(1)) : T(1);
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const int rowb = (zz * F.g.ny + ys[b]) * F.g.nx;
        const T wy = wz * (b == 1 ? T(2) : T(1));
        acc += wy * (F.r[q][rowb + xs[0]] + T(2) * F.r[q][rowb + xs[1]] + F.r[q][rowb + xs[2]]);
      }
    }
    C.f[q][idx] = acc * norm;
    const T ev = F.e[q][ctr];
    C.e[q][idx] = ev;
    C.eh[q][idx] = ev;
  }
}

// f_C += M_C(eh_C)
template <typename T, int KIND, int DIM>
__device__ __forceinline__ void coarse_rhs_point(const Lvl<T>& L, const Phys<T>& P, int idx) {
  using LY = Layout<KIND, DIM>;
  int i, j, k;
  coords(idx, L.g, i, j, k);
  const Nb n = neighbours(i, j, k, L.g);
  T M[LY::NU];
  applyM<T, KIND, DIM>(L, P, n, L.eh, M);
#pragma unroll
  for (int q = 0; q < LY::NU; ++q) L.f[q][idx] += M[q];
}

// fine point idx: e_F += P(e_C - eh_C)  (bilinear / trilinear)
template <typename T, int NU, int DIM>
__device__ __forceinline__ void prolong_point(const Lvl<T>& F, const Lvl<T>& C, int idx) {
  int i, j, k;
  coords(idx, F.g, i, j, k);
  int xi[2], yi[2], zi[2];
  T xw, yw, zw;
  const int X = i >> 1, Y = j >> 1, Z = k >> 1;
  xi[0] = X; xi[1] = (X + 1 == C.g.nx) ? 0 : X + 1;
  yi[0] = Y; yi[1] = (Y + 1 == C.g.ny) ? 0 : Y + 1;
  const int nxp = (i & 1) ? 2 : 1, nyp = (j & 1) ? 2 : 1;
  xw = (i & 1) ? T(0.5) : T(1);
  yw = (j & 1) ? T(0.5) : T(1);
  int nzp = 1;
  zi[0] = zi[1] = 0;
  zw = T(1);
  if constexpr (DIM == 3) {
    zi[0] = Z; zi[1] = (Z + 1 == C.g.nz) ? 0 : Z + 1;
    nzp = (k & 1) ? 2 : 1;
    zw = (k & 1) ? T(0.5) : T(1);
  }
  const T w = xw * yw * zw;
#pragma unroll
  for (int q = 0; q < NU; ++q) {
    T acc = 0;
    for (int c = 0; c < nzp; ++c)
      for (int b = 0; b < nyp; ++b)
        for (int a = 0; a < nxp; ++a) {
          const int ci = (zi[c] * C.g.ny + yi[b]) * C.g.nx + xi[a];
          acc += C.e[q][ci] - C.eh[q][ci];
        }
    F.e[q][idx] += w * acc;
  }
}

template <typename T, int KIND, int DIM>
__global__ void __launch_bounds__(TPB) k_smooth(Lvl<T> L, Phys<T> P, int color) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  int i, j, k;
  if (!colour_point(t, color, L.g, i, j, k)) return;
  const Nb n = neighbours(i, j, k, L.g);
  smooth_point<T, KIND, DIM>(L, P, n);
}

template <typename T, int KIND, int DIM>
__global__ void __launch_bounds__(TPB) k_resid(Lvl<T> L, Phys<T> P) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < L.g.N) resid_point<T, KIND, DIM>(L, P, idx);
}

template <typename T, int NU, int DIM>
__global__ void __launch_bounds__(TPB) k_restrict(Lvl<T> F, Lvl<T> C) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < C.g.N) restrict_point<T, NU, DIM>(F, C, idx);
}

template <typename T, int KIND, int DIM>
__global__ void __launch_bounds__(TPB) k_coarse_rhs(Lvl<T> L, Phys<T> P) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < L.g.N) coarse_rhs_point<T, KIND, DIM>(L, P, idx);
}

template <typename T, int NU, int DIM>
__global__ void __launch_bounds__(TPB) k_prolong(Lvl<T> F, Lvl<T> C) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < F.g.N) prolong_point<T, NU, DIM>(F, C, idx);
}

// Fused red-black sweep of a 2-D level: one thread block per RB_TX x RB_TY
// tile.  The tile and a halo of two points of every array the point update
// reads are staged in shared memory; red points are updated on the tile and
// its first halo ring (their black neighbours are all staged), then black
// points on the tile, and the tile's corrections are written back.  Red
// values on the ring are recomputed identically by the neighbouring tiles, so
// the result equals a red launch followed by a black launch.
constexpr int RB_TX = 32, RB_TY = 16, RB_H = 2;
constexpr int RB_SW = RB_TX + 2 * RB_H;
constexpr int RB_SN = RB_SW * (RB_TY + 2 * RB_H);
constexpr int RB_THREADS = 256;

template <int KIND>
constexpr int rb_arrays() {
  return 2 * Layout<KIND, 2>::NU + 5;  // e, f, rk, om, cr, cv0, cv1
}

__device__ __forceinline__ int wrapi(int x, int n) {
  x %= n;
  return x < 0 ? x + n : x;
}

template <typename T, int KIND>
__global__ void __launch_bounds__(RB_THREADS) k_smooth_rb2d(Lvl<T> G, Phys<T> P) {
  using LY = Layout<KIND, 2>;
  constexpr int NU = LY::NU;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  const int nx = G.g.nx, ny = G.g.ny;
  const int x0 = blockIdx.x * RB_TX, y0 = blockIdx.y * RB_TY;
  for (int t = threadIdx.x; t < RB_SN; t += blockDim.x) {
    const int ly = t / RB_SW, lx = t - ly * RB_SW;
    const int gidx = wrapi(y0 + ly - RB_H, ny) * nx + wrapi(x0 + lx - RB_H, nx);
#pragma unroll
    for (int q = 0; q < NU; ++q) {
      sm[q * RB_SN + t] = G.e[q][gidx];
      sm[(NU + q) * RB_SN + t] = G.f[q][gidx];
    }
    sm[(2 * NU) * RB_SN + t] = G.rk[gidx];
    sm[(2 * NU + 1) * RB_SN + t] = G.om[0][gidx];
    sm[(2 * NU + 2) * RB_SN + t] = G.cr[gidx];
    sm[(2 * NU + 3) * RB_SN + t] = G.cv[0][gidx];
    sm[(2 * NU + 4) * RB_SN + t] = G.cv[1][gidx];
  }
  Lvl<T> L;
  L.g = G.g;
  L.h = G.h;
#pragma unroll
  for (int q = 0; q < MAXU; ++q) {
    L.e[q] = q < NU ? sm + q * RB_SN : nullptr;
    L.f[q] = q < NU ? sm + (NU + q) * RB_SN : nullptr;
    L.r[q] = L.eh[q] = nullptr;
  }
  L.rk = sm + (2 * NU) * RB_SN;
  L.om[0] = sm + (2 * NU + 1) * RB_SN;
  L.om[1] = L.om[2] = nullptr;
  L.cr = sm + (2 * NU + 2) * RB_SN;
  L.cv[0] = sm + (2 * NU + 3) * RB_SN;
  L.cv[1] = sm + (2 * NU + 4) * RB_SN;
  L.cv[2] = nullptr;
  __syncthreads();
#pragma unroll 1
  for (int pass = 0; pass < 2; ++pass) {
    const int color = pass;              // red (i + j even) first, then black
    const int ring = pass == 0 ? 1 : 0;  // red also on the first halo ring
    const int w = RB_TX + 2 * ring;      // even
    const int hw = w >> 1;
    const int npts = hw * (RB_TY + 2 * ring);
    for (int t = threadIdx.x; t < npts; t += blockDim.x) {
      const int ry = t / hw;
      const int gy = y0 - ring + ry;
      const int rx = 2 * (t - ry * hw) + ((color + x0 + ring + gy) & 1);
      const int lx = RB_H - ring + rx, ly = RB_H - ring + ry;
      Nb n;
      n.c = ly * RB_SW + lx;
      n.m[0] = n.c - 1;
      n.p[0] = n.c + 1;
      n.m[1] = n.c - RB_SW;
      n.p[1] = n.c + RB_SW;
      n.m[2] = n.p[2] = n.c;
      smooth_point<T, KIND, 2>(L, P, n);
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < RB_TX * RB_TY; t += blockDim.x) {
    const int ty = t / RB_TX, tx = t - ty * RB_TX;
    const int gx = x0 + tx, gy = y0 + ty;
    if (gx < nx && gy < ny) {
      const int sidx = (ty + RB_H) * RB_SW + tx + RB_H;
#pragma unroll
      for (int q = 0; q < NU; ++q) G.e[q][gy * nx + gx] = L.e[q][sidx];
    }
  }
}

// The whole V-cycle of the small levels (each at most SMALL_N points) in one
// thread block: phases separated by __syncthreads, data in L1/L2.
constexpr int SMALL_N = 1024;           // levels of at most this many points run in one block
constexpr int SMALL_SMEM_N = 1024;
constexpr size_t SMALL_SMEM_MAX = 200 * 1024;
constexpr int SMALL_TPB = 512;
constexpr int MAXSMALL = 8;

template <typename T>
struct SmallLv {
  Lvl<T> lv[MAXSMALL];
  int count;
};

template <typename T, int KIND, int DIM>
__device__ __forceinline__ void block_smooth(const Lvl<T>& L, const Phys<T>& P, int iters) {
  const int half = L.g.N / 2;
  for (int it = 0; it < iters; ++it)
    for (int color = 0; color < 2; ++color) {
      for (int t = threadIdx.x; t < half; t += blockDim.x) {
        int i, j, k;
        colour_point(t, color, L.g, i, j, k);
        const Nb n = neighbours(i, j, k, L.g);
        smooth_point<T, KIND, DIM>(L, P, n);
      }
      __syncthreads();
    }
}

template <typename T, int KIND, int DIM>
__global__ void __launch_bounds__(SMALL_TPB) k_vcycle_small(SmallLv<T> S, Phys<T> P, int nu1, int nu2,
                                                            int ncoarse) {
  using LY = Layout<KIND, DIM>;
  const int nl = S.count;
  for (int l = 0; l + 1 < nl; ++l) {
    const Lvl<T>& F = S.lv[l];
    const Lvl<T>& C = S.lv[l + 1];
    block_smooth<T, KIND, DIM>(F, P, nu1);
    for (int idx = threadIdx.x; idx < F.g.N; idx += blockDim.x) resid_point<T, KIND, DIM>(F, P, idx);
    __syncthreads();
    for (int idx = threadIdx.x; idx < C.g.N; idx += blockDim.x) restrict_point<T, LY::NU, DIM>(F, C, idx);
    __syncthreads();
    for (int idx = threadIdx.x; idx < C.g.N; idx += blockDim.x) coarse_rhs_point<T, KIND, DIM>(C, P, idx);
    __syncthreads();
  }
  block_smooth<T, KIND, DIM>(S.lv[nl - 1], P, ncoarse);
  for (int l = nl - 2; l >= 0; --l) {
    const Lvl<T>& F = S.lv[l];
    const Lvl<T>& C = S.lv[l + 1];
    for (int idx = threadIdx.x; idx < F.g.N; idx += blockDim.x) prolong_point<T, LY::NU, DIM>(F, C, idx);
    __syncthreads();
    block_smooth<T, KIND, DIM>(F, P, nu2);
  }
}

// Same V-cycle with the corrections, right-hand sides and residuals of the
// small levels held in shared memory (coefficients are read through L1).
// On entry the first small level's e and f are in global memory; on exit its
// e is written back.  `layout` gives each level's shared-memory offsets.
template <typename T>
struct SmallSmem {
  int off_e[MAXSMALL][MAXU];
  int off_f[MAXSMALL][MAXU];
  int off_r[MAXSMALL][MAXU];
  int off_eh[MAXSMALL][MAXU];
};

template <typename T, int KIND, int DIM>
__global__ void __launch_bounds__(SMALL_TPB) k_vcycle_small_smem(SmallLv<T> S, SmallSmem<T> M, Phys<T> P,
                                                                 int nu1, int nu2, int ncoarse) {
  using LY = Layout<KIND, DIM>;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  __shared__ Lvl<T> SL[MAXSMALL];
  const int nl = S.count;
  if (threadIdx.x == 0) {
    for (int l = 0; l < nl; ++l) {
      SL[l] = S.lv[l];
      for (int q = 0; q < MAXU; ++q) {
        SL[l].e[q] = q < LY::NU ? sm + M.off_e[l][q] : nullptr;
        SL[l].f[q] = q < LY::NU ? sm + M.off_f[l][q] : nullptr;
        SL[l].r[q] = (q < LY::NU && l + 1 < nl) ? sm + M.off_r[l][q] : nullptr;
        SL[l].eh[q] = (q < LY::NU && l > 0) ? sm + M.off_eh[l][q] : nullptr;
      }
    }
  }
  __syncthreads();
  {
    const Lvl<T>& G = S.lv[0];
    for (int idx = threadIdx.x; idx < G.g.N; idx += blockDim.x)
#pragma unroll
      for (int q = 0; q < LY::NU; ++q) {
        SL[0].e[q][idx] = G.e[q][idx];
        SL[0].f[q][idx] = G.f[q][idx];
      }
  }
  __syncthreads();
  for (int l = 0; l + 1 < nl; ++l) {
    const Lvl<T>& F = SL[l];
    const Lvl<T>& C = SL[l + 1];
    block_smooth<T, KIND, DIM>(F, P, nu1);
    for (int idx = threadIdx.x; idx < F.g.N; idx += blockDim.x) resid_point<T, KIND, DIM>(F, P, idx);
    __syncthreads();
    for (int idx = threadIdx.x; idx < C.g.N; idx += blockDim.x) restrict_point<T, LY::NU, DIM>(F, C, idx);
    __syncthreads();
    for (int idx = threadIdx.x; idx < C.g.N; idx += blockDim.x) coarse_rhs_point<T, KIND, DIM>(C, P, idx);
    __syncthreads();
  }
  block_smooth<T, KIND, DIM>(SL[nl - 1], P, ncoarse);
  for (int l = nl - 2; l >= 0; --l) {
    const Lvl<T>& F = SL[l];
    const Lvl<T>& C = SL[l + 1];
    for (int idx = threadIdx.x; idx < F.g.N; idx += blockDim.x) prolong_point<T, LY::NU, DIM>(F, C, idx);
    __syncthreads();
    block_smooth<T, KIND, DIM>(F, P, nu2);
  }
  {
    const Lvl<T>& G = S.lv[0];
    for (int idx = threadIdx.x; idx < G.g.N; idx += blockDim.x)
#pragma unroll
      for (int q = 0; q < LY::NU; ++q) G.e[q][idx] = SL[0].e[q][idx];
  }
}

// Injection of up to 6 coefficient fields from the finest grid to every
// coarser level at once (injection of an injection samples every 2^l-th
// point of the finest grid).
template <typename T>
struct InjAll {
  const T* src[6];
  T* dst[MAXLEV][6];
  Geo g[MAXLEV];
  int off[MAXLEV + 1];
  int nsrc;
  int nl;      // levels 1..nl-1 are written
  Geo g0;
};

template <typename T>
__global__ void __launch_bounds__(TPB) k_inject_all(InjAll<T> A) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= A.off[A.nl]) return;
  int l = 1;
  while (t >= A.off[l + 1]) ++l;
  const int idx = t - A.off[l];
  int I, J, K;
  coords(idx, A.g[l], I, J, K);
  const int sc = 1 << l;
  const int fidx = ((K * sc) * A.g0.ny + J * sc) * A.g0.nx + I * sc;
  for (int q = 0; q < A.nsrc; ++q) A.dst[l][q][idx] = A.src[q][fidx];
}

// --------------------------------------------------------------------------
// float64 kernels of the finest level
// --------------------------------------------------------------------------
struct Vel3 {
  const double* p[3];
};
struct Vel3W {
  double* p[3];
};

struct Fields64 {
  const double* rho;          // rho^k
  const double* vel[3];       // u^k
  const double* conv;         // J * rho^k (CDFT)
  double* om[3];              // omega^k (out)
  double* S[MAXU];            // source (out)
  double* g[MAXU];            // iterate
  float* rk32;                // float copies for the mixed path (or null)
  float* om32[3];
};

// omega^k, S and the initial iterate g^0 (kappa^0 = Lap_h rho^k for PFC).
template <int KIND, int DIM>
__global__ void __launch_bounds__(TPB) k_prepare(Fields64 F, Geo G, double h, Phys<double> P) {
  using LY = Layout<KIND, DIM>;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= G.N) return;
  int i, j, k;
  coords(idx, G, i, j, k);
  const Nb n = neighbours(i, j, k, G);
  const double ih = 1.0 / h, ih2 = ih * ih;
  const double* u = F.vel[0];
  const double* v = F.vel[1];
  double w[3];
  if constexpr (DIM == 2) {
    w[0] = 0.5 * ih * ((v[n.p[0]] - v[n.m[0]]) - (u[n.p[1]] - u[n.m[1]]));
  } else {
    const double* ww = F.vel[2];
    w[0] = 0.5 * ih * ((ww[n.p[1]] - ww[n.m[1]]) - (v[n.p[2]] - v[n.m[2]]));
    w[1] = 0.5 * ih * ((u[n.p[2]] - u[n.m[2]]) - (ww[n.p[0]] - ww[n.m[0]]));
    w[2] = 0.5 * ih * ((v[n.p[0]] - v[n.m[0]]) - (u[n.p[1]] - u[n.m[1]]));
  }
  const double rkc = F.rho[n.c];
  double div = 0;
#pragma unroll
  for (int d = 0; d < DIM; ++d)
    div += F.rho[n.p[d]] * F.vel[d][n.p[d]] - F.rho[n.m[d]] * F.vel[d][n.m[d]];
  F.S[0][idx] = rkc - P.s * 0.25 * ih * div;
  double uc[3], wx[3];
#pragma unroll
  for (int d = 0; d < DIM; ++d) uc[d] = F.vel[d][n.c];
  cross<double, DIM>(w, uc, wx);
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    double sa = rkc * uc[a] - 0.5 * P.sigma * P.s * rkc * wx[a]
              + 0.5 * P.s * P.gamma * (nbsum<double, DIM>(F.vel[a], n) - 2.0 * DIM * uc[a]) * ih2;
    if constexpr (KIND == KCDFT) {
      const double Ep = 2.0 * P.ce * F.rho[n.p[a]] + F.conv[n.p[a]];
      const double Em = 2.0 * P.ce * F.rho[n.m[a]] + F.conv[n.m[a]];
      sa += P.s * rkc * 0.5 * ih * (Ep - Em);
    }
    F.S[1 + a][idx] = sa;
    F.g[1 + a][idx] = uc[a];
  }
  F.g[0][idx] = rkc;
  if constexpr (KIND == KPFC) {
    const double lapr = (nbsum<double, DIM>(F.rho, n) - 2.0 * DIM * rkc) * ih2;
    F.S[LY::IMU][idx] = 2.0 * lapr;
    F.S[LY::IKA][idx] = 0.0;
    F.g[LY::IKA][idx] = lapr;
  }
#pragma unroll
  for (int d = 0; d < LY::NOM; ++d) F.om[d][idx] = w[d];
  if (F.rk32) {
    F.rk32[idx] = (float)rkc;
#pragma unroll
    for (int d = 0; d < LY::NOM; ++d) F.om32[d][idx] = (float)w[d];
  }
}

// PFC: mu^0 = psi^3/3 + alpha psi + Lap_h kappa^0 + S_mu (value of the mu row at rho^k).
template <int DIM>
__global__ void __launch_bounds__(TPB) k_prepare_mu(Fields64 F, Geo G, double h, Phys<double> P) {
  using LY = Layout<KPFC, DIM>;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= G.N) return;
  int i, j, k;
  coords(idx, G, i, j, k);
  const Nb n = neighbours(i, j, k, G);
  const double psi = F.rho[idx] - 1.5;
  const double* ka = F.g[LY::IKA];
  const double lapk = (nbsum<double, DIM>(ka, n) - 2.0 * DIM * ka[idx]) / (h * h);
  F.g[LY::IMU][idx] = psi * psi * psi / 3.0 + P.alpha * psi + lapk + F.S[LY::IMU][idx];
}

template <int NQ>
__device__ __forceinline__ void block_partials(double (&v)[NQ], double* partials) {
  __shared__ double sm[NQ][TPB / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q)
    for (int off = 16; off > 0; off >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], off);
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < NQ; ++q) sm[q][warp] = v[q];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      double x = (lane < TPB / 32) ? sm[q][lane] : 0.0;
      for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
      if (lane == 0) partials[blockIdx.x * NQ + q] = x;
    }
  }
}

// Fixed-order reduction of per-block partials: out[q] = sum_b partials[b][q].
template <int NQ>
__global__ void __launch_bounds__(TPB) k_final_sum(const double* partials, int nblk, double* out) {
  double v[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) v[q] = 0.0;
  for (int b = threadIdx.x; b < nblk; b += TPB)
#pragma unroll
    for (int q = 0; q < NQ; ++q) v[q] += partials[b * NQ + q];
  __shared__ double sm[NQ][TPB / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q)
    for (int off = 16; off > 0; off >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], off);
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < NQ; ++q) sm[q][warp] = v[q];
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      double x = 0.0;
      for (int w = 0; w < TPB / 32; ++w) x += sm[q][w];
      out[q] = x;
    }
  }
}

// out[0] = max_q sqrt(w * sum_q); out[1 + q] = sums
template <int NQ>
__global__ void k_norm_final(const double* partials, int nblk, double w, double* out) {
  double v[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) v[q] = 0.0;
  for (int b = threadIdx.x; b < nblk; b += TPB)
#pragma unroll
    for (int q = 0; q < NQ; ++q) v[q] += partials[b * NQ + q];
  __shared__ double sm[NQ][TPB / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q)
    for (int off = 16; off > 0; off >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], off);
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < NQ; ++q) sm[q][warp] = v[q];
  __syncthreads();
  if (threadIdx.x == 0) {
    double mx = 0.0;
    bool finite = true;
    for (int q = 0; q < NQ; ++q) {
      double x = 0.0;
      for (int ww = 0; ww < TPB / 32; ++ww) x += sm[q][ww];
      out[1 + q] = x;
      const double nq = sqrt(w * x);
      if (!(nq == nq) || isinf(nq)) finite = false;
      mx = fmax(mx, nq);
    }
    out[0] = finite ? mx : NAN;
  }
}

struct Resid64Out {
  void* f0[MAXU];   // precision-T rhs of level 0 (or null)
  void* e0[MAXU];   // precision-T correction of level 0, zeroed (or null)
  float* cr32;      // float coefficient copies (mixed path) or null
  float* cv32[3];
  double* r64[MAXU];  // optional float64 residual output
};

// r = S - N(g) in float64 (App. G operator N, full form), block partials of r^2.
template <int KIND, int DIM, typename T>
__global__ void __launch_bounds__(TPB) k_resid64(Fields64 F, Resid64Out O, Geo G, double h,
                                                 Phys<double> P, double* partials) {
  using LY = Layout<KIND, DIM>;
  double acc[LY::NU];
#pragma unroll
  for (int q = 0; q < LY::NU; ++q) acc[q] = 0.0;
  const double ih = 1.0 / h, ih2 = ih * ih;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < G.N; idx += gridDim.x * blockDim.x) {
    int i, j, k;
    coords(idx, G, i, j, k);
    const Nb n = neighbours(i, j, k, G);
    const double* const* g = F.g;
    const double rkc = F.rho[n.c];
    double N[LY::NU];
    double div = 0;
#pragma unroll
    for (int d = 0; d < DIM; ++d)
      div += F.rho[n.p[d]] * g[1 + d][n.p[d]] - F.rho[n.m[d]] * g[1 + d][n.m[d]];
    N[0] = g[0][n.c] + P.s * 0.25 * ih * div;
    double uc[3], w[3], wx[3];
#pragma unroll
    for (int d = 0; d < DIM; ++d) uc[d] = g[1 + d][n.c];
#pragma unroll
    for (int d = 0; d < LY::NOM; ++d) w[d] = F.om[d][n.c];
    cross<double, DIM>(w, uc, wx);
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      double qp = 0, qm = 0;
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        const double up = g[1 + d][n.p[a]], um = g[1 + d][n.m[a]];
        qp += up * up;
        qm += um * um;
      }
      double mp, mm;
      if constexpr (KIND == KPFC) {
        mp = g[LY::IMU][n.p[a]];
        mm = g[LY::IMU][n.m[a]];
      } else {
        const double rp = g[0][n.p[a]], rm = g[0][n.m[a]];
        mp = log(rp) + 2.0 * P.ce * rp;
        mm = log(rm) + 2.0 * P.ce * rm;
      }
      const double lapa = (nbsum<double, DIM>(g[1 + a], n) - 2.0 * DIM * uc[a]) * ih2;
      N[1 + a] = rkc * uc[a] + 0.5 * P.sigma * P.s * rkc * wx[a]
               + P.s * rkc * ih * (0.25 * (qp - qm) + 0.5 * (mp - mm))
               - 0.5 * P.s * P.gamma * lapa;
    }
    if constexpr (KIND == KPFC) {
      const double rc = g[0][n.c];
      const double psi = rc - 1.5;
      const double kc = g[LY::IKA][n.c];
      const double lapk = (nbsum<double, DIM>(g[LY::IKA], n) - 2.0 * DIM * kc) * ih2;
      const double lapr = (nbsum<double, DIM>(g[0], n) - 2.0 * DIM * rc) * ih2;
      N[LY::IMU] = g[LY::IMU][n.c] - psi * psi * psi / 3.0 - P.alpha * psi - lapk;
      N[LY::IKA] = kc - lapr;
    }
#pragma unroll
    for (int q = 0; q < LY::NU; ++q) {
      const double r = F.S[q][idx] - N[q];
      acc[q] += r * r;
      if (O.f0[q]) static_cast<T*>(O.f0[q])[idx] = (T)r;
      if (O.e0[q]) static_cast<T*>(O.e0[q])[idx] = T(0);
      if (O.r64[q]) O.r64[q][idx] = r;
    }
    if (O.cr32) {
      O.cr32[idx] = (float)g[0][idx];
#pragma unroll
      for (int d = 0; d < DIM; ++d) O.cv32[d][idx] = (float)g[1 + d][idx];
    }
  }
  block_partials<LY::NU>(acc, partials);
}

// g += e (float64), then the projection of Sec. 6 on rho.
template <int NU, typename T>
__global__ void __launch_bounds__(TPB) k_update64(Fields64 F, Resid64Out O, int N, double delta) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= N) return;
#pragma unroll
  for (int q = 0; q < NU; ++q) F.g[q][idx] += (double)static_cast<const T*>(O.e0[q])[idx];
  const double r = F.g[0][idx];
  F.g[0][idx] = (delta > 0.0) ? sqrt(r * r + delta * delta) : fabs(r);
}

// Device-side control block of one step: residual norms, cycle count and
// status; read by the host once per step (graph mode) or per cycle.
struct Ctl {
  double norm;
  double norm0;
  int cycles;
  int status;
  int pad[2];
};

// Finishes the residual norm max_q sqrt(w * sum_q), updates the control
// block (cycles += in_body) and, in graph mode, sets the WHILE condition:
// continue while the norm is finite, above tol and cycles < max_cycles.
template <int NQ>
__global__ void k_norm_ctl(const double* partials, int nblk, double w, Ctl* ctl, double tol, int max_cycles,
                           int in_body, cudaGraphConditionalHandle handle, int use_handle) {
  double v[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) v[q] = 0.0;
  for (int b = threadIdx.x; b < nblk; b += TPB)
#pragma unroll
    for (int q = 0; q < NQ; ++q) v[q] += partials[b * NQ + q];
  __shared__ double sm[NQ][TPB / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q)
    for (int off = 16; off > 0; off >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], off);
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < NQ; ++q) sm[q][warp] = v[q];
  __syncthreads();
  if (threadIdx.x == 0) {
    double mx = 0.0;
    bool finite = true;
    for (int q = 0; q < NQ; ++q) {
      double x = 0.0;
      for (int ww = 0; ww < TPB / 32; ++ww) x += sm[q][ww];
      const double nq = sqrt(w * x);
      if (!(nq == nq) || isinf(nq)) finite = false;
      mx = fmax(mx, nq);
    }
    const double nrm = finite ? mx : NAN;
    int cycles = in_body ? ctl->cycles + 1 : 0;
    ctl->cycles = cycles;
    ctl->norm = nrm;
    if (!in_body) ctl->norm0 = nrm;
    int status = FM_OK;
    if (!finite) status = FM_ENAN;
    else if (nrm > tol && cycles >= max_cycles) status = FM_ENOCONV;
    ctl->status = status;
    const bool cont = status == FM_OK && nrm > tol;
    if (use_handle) cudaGraphSetConditional(handle, cont ? 1u : 0u);
  }
}

// rho^{k+1} = S1 - (s/4h) sum_d ([rho^k u_d]_{+d} - [rho^k u_d]_{-d}), projected,
// into `out`; skipped unless the solve succeeded.
template <int DIM>
__global__ void __launch_bounds__(TPB) k_closure(Fields64 F, Geo G, double h, Phys<double> P, double* out,
                                                 const Ctl* ctl) {
  if (ctl->status != FM_OK) return;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= G.N) return;
  int i, j, k;
  coords(idx, G, i, j, k);
  const Nb n = neighbours(i, j, k, G);
  double div = 0;
#pragma unroll
  for (int d = 0; d < DIM; ++d)
    div += F.rho[n.p[d]] * F.g[1 + d][n.p[d]] - F.rho[n.m[d]] * F.g[1 + d][n.m[d]];
  const double r = F.S[0][idx] - P.s * 0.25 / h * div;
  out[idx] = (P.delta > 0.0) ? sqrt(r * r + P.delta * P.delta) : fabs(r);
}

// New time level: rho <- closure result, u <- converged velocity (if the
// solve succeeded).
template <int DIM>
__global__ void __launch_bounds__(TPB) k_commit(double* rho, Vel3W vel, const double* rnew, Vel3 gvel, int N,
                                                const Ctl* ctl) {
  if (ctl->status != FM_OK) return;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= N) return;
  rho[idx] = rnew[idx];
#pragma unroll
  for (int d = 0; d < DIM; ++d) vel.p[d][idx] = gvel.p[d][idx];
}

// Energy densities: q0 = KE, then PFC: psi^4/12, alpha psi^2/2, (Lap rho)^2/2,
// rho Lap rho; CDFT: rho (ln rho - 1), -rho (J*rho)/2.
template <int KIND, int DIM>
__global__ void __launch_bounds__(TPB) k_energy(const double* rho, Vel3 vel3,
                                                const double* conv, Geo G, double h, double alpha,
                                                double* partials) {
  constexpr int NQ = 5;
  double acc[NQ] = {0, 0, 0, 0, 0};
  const double ih2 = 1.0 / (h * h);
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < G.N; idx += gridDim.x * blockDim.x) {
    const double rc = rho[idx];
    double u2 = 0;
#pragma unroll
    for (int d = 0; d < DIM; ++d) u2 += vel3.p[d][idx] * vel3.p[d][idx];
    acc[0] += 0.5 * rc * u2;
    if constexpr (KIND == KPFC) {
      int i, j, k;
      coords(idx, G, i, j, k);
      const Nb n = neighbours(i, j, k, G);
      const double psi = rc - 1.5;
      const double L = (nbsum<double, DIM>(rho, n) - 2.0 * DIM * rc) * ih2;
      acc[1] += psi * psi * psi * psi / 12.0;
      acc[2] += 0.5 * alpha * psi * psi;
      acc[3] += 0.5 * L * L;
      acc[4] += rc * L;
    } else {
      acc[1] += rc * (log(rc) - 1.0);
      acc[2] += -0.5 * rc * conv[idx];
    }
  }
  block_partials<NQ>(acc, partials);
}

__global__ void __launch_bounds__(TPB) k_mass(const double* rho, int N, double* partials) {
  double acc[1] = {0.0};
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += gridDim.x * blockDim.x)
    acc[0] += rho[idx];
  block_partials<1>(acc, partials);
}

// Standalone float64 transfers (row-level entry points).
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
#define FM_CUDA(call)                                   \
  do {                                                  \
    cudaError_t err__ = (call);                         \
    if (err__ != cudaSuccess) return FM_ECUDA;          \
  } while (0)

#define FM_LAUNCHED()                                   \
  do {                                                  \
    ++st->launches;                                     \
    if (cudaPeekAtLastError() != cudaSuccess) {         \
      cudaGetLastError();                               \
      return FM_ECUDA;                                  \
    }                                                   \
  } while (0)

template <typename T>
static Lvl<T> make_lvl(const fm_state* st, int l) {
  const LevelBufs& B = st->lv[l];
  Lvl<T> L;
  L.g = B.g;
  L.h = (T)B.h;
  for (int q = 0; q < MAXU; ++q) {
    L.e[q] = (T*)B.e[q];
    L.f[q] = (T*)B.f[q];
    L.r[q] = (T*)B.r[q];
    L.eh[q] = (T*)B.eh[q];
  }
  L.rk = (const T*)B.rk;
  L.cr = (const T*)B.cr;
  for (int d = 0; d < 3; ++d) {
    L.om[d] = (const T*)B.om[d];
    L.cv[d] = (const T*)B.cv[d];
  }
  return L;
}

template <typename T>
static Phys<T> make_phys(const fm_state* st) {
  Phys<T> P;
  P.s = (T)st->dt;
  P.gamma = (T)st->prm.gamma;
  P.alpha = (T)st->fn.alpha;
  P.ce = (T)st->ce;
  P.sigma = (T)st->prm.sigma;
  P.w = (T)st->prm.w_damp;
  P.delta = (T)st->prm.delta;
  return P;
}

static Fields64 make_fields(fm_state* st) {
  Fields64 F;
  F.rho = st->rho;
  for (int d = 0; d < 3; ++d) {
    F.vel[d] = st->vel[d];
    F.om[d] = st->om[d];
    F.om32[d] = nullptr;
  }
  F.conv = st->conv;
  for (int q = 0; q < MAXU; ++q) {
    F.S[q] = st->S[q];
    F.g[q] = st->g[q];
  }
  F.rk32 = nullptr;
  if (st->prm.precision == FM_MIXED) {
    F.rk32 = (float*)st->lv[0].rk;
    for (int d = 0; d < st->nom; ++d) F.om32[d] = (float*)st->lv[0].om[d];
  }
  return F;
}

// Sum the durations of the recorded (start, end) event pairs; call only after
// the stream has been synchronised.
static int harvest_profile(fm_state* st) {
  for (int i = 0; i + 1 < st->npev; i += 2) {
    float ms = 0.f;
    FM_CUDA(cudaEventElapsedTime(&ms, st->pev[i], st->pev[i + 1]));
    st->prof_ms += ms;
    st->prof_count += 1;
  }
  st->npev = 0;
  return FM_OK;
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

  static int enqueue_prepare(fm_state* st) {
    const Geo G = st->lv[0].g;
    const double h = st->lv[0].h;
    Phys<double> P = make_phys<double>(st);
    cudaStream_t s = st->stream;
    if (KIND == KCDFT) {
      int rc = fft_convolve(st, st->rho, st->conv);
      if (rc) return rc;
    }
    Fields64 F = make_fields(st);
    k_prepare<KIND, DIM><<<nblocks(G.N), TPB, 0, s>>>(F, G, h, P);
    FM_LAUNCHED();
    if (KIND == KPFC) {
      k_prepare_mu<DIM><<<nblocks(G.N), TPB, 0, s>>>(F, G, h, P);
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

  // float64 residual of the current iterate, the level-0 set-up of a cycle
  // and the control-block update (in_body: this follows a cycle).
  static int enqueue_resid_norm(fm_state* st, int in_body, cudaGraphConditionalHandle hdl, int use_handle) {
    const Geo G = st->lv[0].g;
    const double h = st->lv[0].h;
    Phys<double> P = make_phys<double>(st);
    cudaStream_t s = st->stream;
    Fields64 F = make_fields(st);
    Resid64Out O = resid_out(st, true, nullptr);
    k_resid64<KIND, DIM, T><<<st->nblk, TPB, 0, s>>>(F, O, G, h, P, st->partials);
    FM_LAUNCHED();
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
    k_resid64<KIND, DIM, T><<<st->nblk, TPB, 0, s>>>(F, O, G, h, P, st->partials);
    FM_LAUNCHED();
    const double w = (DIM == 3) ? h * h * h : h * h;
    k_norm_final<LY::NU><<<1, TPB, 0, s>>>(st->partials, st->nblk, w, st->dscal);
    FM_LAUNCHED();
    FM_CUDA(cudaMemcpyAsync(st->hscal, st->dscal, sizeof(double), cudaMemcpyDeviceToHost, s));
    FM_CUDA(cudaStreamSynchronize(s));
    *norm_host = st->hscal[0];
    return FM_OK;
  }

  static int smooth(fm_state* st, int l, const Phys<T>& P, int iters) {
    cudaStream_t s = st->stream;
    Lvl<T> L = make_lvl<T>(st, l);
    const int half = L.g.N / 2;
    const bool prof = st->prof && !st->capturing && l == 0;
    const bool fused = DIM == 2 && st->fused_rb;
    const size_t smem = (size_t)rb_arrays<KIND>() * RB_SN * sizeof(T);
    if (fused) {
      static bool attr = false;
      if (!attr) {
        FM_CUDA(cudaFuncSetAttribute(k_smooth_rb2d<T, KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
        attr = true;
      }
    }
    const dim3 tiles((L.g.nx + RB_TX - 1) / RB_TX, (L.g.ny + RB_TY - 1) / RB_TY);
    for (int it = 0; it < iters; ++it) {
      const int nlaunch = fused ? 1 : 2;
      for (int color = 0; color < nlaunch; ++color) {
        if (prof && st->npev + 2 <= MAXEV) FM_CUDA(cudaEventRecord(st->pev[st->npev], s));
        if (fused)
          k_smooth_rb2d<T, KIND><<<tiles, RB_THREADS, smem, s>>>(L, P);
        else
          k_smooth<T, KIND, DIM><<<nblocks(half), TPB, 0, s>>>(L, P, color);
        FM_LAUNCHED();
        if (prof && st->npev + 2 <= MAXEV) {
          FM_CUDA(cudaEventRecord(st->pev[st->npev + 1], s));
          st->npev += 2;
        }
      }
    }
    return FM_OK;
  }

  static int vcycle(fm_state* st, int l, const Phys<T>& P) {
    cudaStream_t s = st->stream;
    if (l >= st->small_from) {
      SmallLv<T> S;
      S.count = st->nlev - l;
      for (int q = 0; q < S.count; ++q) S.lv[q] = make_lvl<T>(st, l + q);
      // shared-memory layout of the small levels' e, f, r, eh
      SmallSmem<T> M;
      memset(&M, 0, sizeof(M));
      int off = 0;
      for (int q = 0; q < S.count; ++q) {
        const int N = S.lv[q].g.N;
        for (int u = 0; u < LY::NU; ++u) {
          M.off_e[q][u] = off; off += N;
          M.off_f[q][u] = off; off += N;
          if (q + 1 < S.count) { M.off_r[q][u] = off; off += N; }
          if (q > 0) { M.off_eh[q][u] = off; off += N; }
        }
      }
      const size_t smem = (size_t)off * sizeof(T);
      if (smem <= SMALL_SMEM_MAX && S.lv[0].g.N <= SMALL_SMEM_N) {
        static bool attr = false;
        if (!attr) {
          FM_CUDA(cudaFuncSetAttribute(k_vcycle_small_smem<T, KIND, DIM>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMALL_SMEM_MAX));
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
    int rc = smooth(st, l, P, st->prm.nu1);
    if (rc) return rc;
    Lvl<T> F = make_lvl<T>(st, l);
    Lvl<T> C = make_lvl<T>(st, l + 1);
    k_resid<T, KIND, DIM><<<nblocks(F.g.N), TPB, 0, s>>>(F, P);
    FM_LAUNCHED();
    k_restrict<T, LY::NU, DIM><<<nblocks(C.g.N), TPB, 0, s>>>(F, C);
    FM_LAUNCHED();
    k_coarse_rhs<T, KIND, DIM><<<nblocks(C.g.N), TPB, 0, s>>>(C, P);
    FM_LAUNCHED();
    rc = vcycle(st, l + 1, P);
    if (rc) return rc;
    k_prolong<T, LY::NU, DIM><<<nblocks(F.g.N), TPB, 0, s>>>(F, C);
    FM_LAUNCHED();
    return smooth(st, l, P, st->prm.nu2);
  }

  static int enqueue_body(fm_state* st, cudaGraphConditionalHandle hdl, int use_handle) {
    int rc = inject_all(st, true);
    if (rc) return rc;
    Phys<T> P = make_phys<T>(st);
    rc = vcycle(st, 0, P);
    if (rc) return rc;
    const Geo G = st->lv[0].g;
    Fields64 F = make_fields(st);
    Resid64Out O = resid_out(st, true, nullptr);
    k_update64<LY::NU, T><<<nblocks(G.N), TPB, 0, st->stream>>>(F, O, G.N, st->prm.delta);
    FM_LAUNCHED();
    return enqueue_resid_norm(st, 1, hdl, use_handle);
  }

  static int enqueue_post(fm_state* st) {
    const Geo G = st->lv[0].g;
    Fields64 F = make_fields(st);
    Phys<double> P64 = make_phys<double>(st);
    const Ctl* ctl = (const Ctl*)st->ctl;
    k_closure<DIM><<<nblocks(G.N), TPB, 0, st->stream>>>(F, G, st->lv[0].h, P64, st->tmp, ctl);
    FM_LAUNCHED();
    Vel3W vw{{st->vel[0], st->vel[1], st->vel[2]}};
    Vel3 gv{{st->g[1], st->g[2], DIM == 3 ? st->g[3] : nullptr}};
    k_commit<DIM><<<nblocks(G.N), TPB, 0, st->stream>>>(st->rho, vw, st->tmp, gv, G.N, ctl);
    FM_LAUNCHED();
    FM_CUDA(cudaMemcpyAsync(st->hscal + 32, st->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st->stream));
    return FM_OK;
  }

  static int read_ctl(fm_state* st, Ctl* out) {
    FM_CUDA(cudaMemcpyAsync(st->hscal + 32, st->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st->stream));
    FM_CUDA(cudaStreamSynchronize(st->stream));
    memcpy(out, st->hscal + 32, sizeof(Ctl));
    return harvest_profile(st);
  }

  static int finish(fm_state* st, fm_step_info* info) {
    Ctl c;
    memcpy(&c, st->hscal + 32, sizeof(Ctl));
    st->prepared = false;
    if (info) {
      info->cycles = c.cycles;
      info->res0 = c.norm0;
      info->res = c.norm;
    }
    return c.status;
  }

  static int step_hostloop(fm_state* st, fm_step_info* info) {
    int rc = enqueue_prepare(st);
    if (rc) return rc;
    rc = enqueue_resid_norm(st, 0, 0, 0);
    if (rc) return rc;
    Ctl c;
    for (;;) {
      rc = read_ctl(st, &c);
      if (rc) return rc;
      if (c.status != FM_OK || !(c.norm > st->prm.tol)) break;
      rc = enqueue_body(st, 0, 0);
      if (rc) return rc;
    }
    rc = enqueue_post(st);
    if (rc) return rc;
    FM_CUDA(cudaStreamSynchronize(st->stream));
    return finish(st, info);
  }

  static int build_graph(fm_state* st) {
    if (st->gexec) {
      cudaGraphExecDestroy(st->gexec);
      st->gexec = nullptr;
    }
    if (st->graph) {
      cudaGraphDestroy(st->graph);
      st->graph = nullptr;
    }
    cudaStream_t saved = st->stream;
    cudaStream_t s0 = st->cap[0], s1 = st->cap[1];
    st->capturing = true;
    st->stream = s0;
    int rc = FM_OK;
    cudaGraph_t g = nullptr;
    do {
      if (cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal) != cudaSuccess) { rc = FM_ECUDA; break; }
      const long long l0 = st->launches;
      rc = enqueue_prepare(st);
      if (rc) break;
      cudaStreamCaptureStatus cs;
      const cudaGraphNode_t* deps = nullptr;
      size_t nd = 0;
      cudaGraph_t cg = nullptr;
      if (cudaStreamGetCaptureInfo(s0, &cs, nullptr, &cg, nullptr, nullptr, nullptr) != cudaSuccess) { rc = FM_ECUDA; break; }
      cudaGraphConditionalHandle hdl;
      if (cudaGraphConditionalHandleCreate(&hdl, cg, 0, cudaGraphCondAssignDefault) != cudaSuccess) { rc = FM_ECUDA; break; }
      rc = enqueue_resid_norm(st, 0, hdl, 1);
      if (rc) break;
      st->cnt_pre = st->launches - l0;
      if (cudaStreamGetCaptureInfo(s0, &cs, nullptr, &cg, &deps, nullptr, &nd) != cudaSuccess) { rc = FM_ECUDA; break; }
      cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
      cp.conditional.handle = hdl;
      cp.conditional.type = cudaGraphCondTypeWhile;
      cp.conditional.size = 1;
      cudaGraphNode_t wnode;
      if (cudaGraphAddNode(&wnode, cg, deps, nullptr, nd, &cp) != cudaSuccess) { rc = FM_ECUDA; break; }
      cudaGraph_t body = cp.conditional.phGraph_out[0];
      if (cudaStreamUpdateCaptureDependencies(s0, &wnode, nullptr, 1, cudaStreamSetCaptureDependencies) != cudaSuccess) { rc = FM_ECUDA; break; }
      st->stream = s1;
      if (cudaStreamBeginCaptureToGraph(s1, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) != cudaSuccess) { rc = FM_ECUDA; break; }
      const long long l1 = st->launches;
      rc = enqueue_body(st, hdl, 1);
      st->cnt_body = st->launches - l1;
      cudaGraph_t bodyout = nullptr;
      if (cudaStreamEndCapture(s1, &bodyout) != cudaSuccess && rc == FM_OK) rc = FM_ECUDA;
      if (rc) break;
      st->stream = s0;
      const long long l2 = st->launches;
      rc = enqueue_post(st);
      st->cnt_post = st->launches - l2;
      st->launches = l0;
    } while (0);
    st->stream = s0;
    if (cudaStreamEndCapture(s0, &g) != cudaSuccess && rc == FM_OK) rc = FM_ECUDA;
    st->stream = saved;
    st->capturing = false;
    if (rc) {
      cudaGetLastError();
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (cudaGraphInstantiate(&st->gexec, g, 0) != cudaSuccess) {
      cudaGetLastError();
      cudaGraphDestroy(g);
      return FM_ECUDA;
    }
    st->graph = g;
    st->graph_dt = st->dt;
    return FM_OK;
  }

  static int step(fm_state* st, fm_step_info* info) {
    if (st->prof || !st->use_graph) return step_hostloop(st, info);
    if (!st->gexec || st->graph_dt != st->dt) {
      int rc = build_graph(st);
      if (rc) return rc;
    }
    FM_CUDA(cudaGraphLaunch(st->gexec, st->stream));
    FM_CUDA(cudaStreamSynchronize(st->stream));
    Ctl c;
    memcpy(&c, st->hscal + 32, sizeof(Ctl));
    st->launches += st->cnt_pre + (long long)c.cycles * st->cnt_body + st->cnt_post;
    return finish(st, info);
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
static int dispatch_prepare(fm_state* st) {
  if (st->kind == FM_PFC)
    return st->dim == 2 ? Solver<T, KPFC, 2>::prepare(st) : Solver<T, KPFC, 3>::prepare(st);
  return st->dim == 2 ? Solver<T, KCDFT, 2>::prepare(st) : Solver<T, KCDFT, 3>::prepare(st);
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
  }
  for (int d = 0; d < 3; ++d) st->om[d] = d < st->nom ? (double*)C.take(N0 * d8) : nullptr;
  st->conv = st->kind == FM_CDFT ? (double*)C.take(N0 * d8) : nullptr;
  st->tmp = (double*)C.take(N0 * d8);
  for (int q = 0; q < MAXU; ++q) st->r64[q] = q < st->nu ? (double*)C.take(N0 * d8) : nullptr;
  st->partials = (double*)C.take((size_t)st->nblk * 8 * d8);
  st->dscal = (double*)C.take(64 * d8);
  st->ctl = C.take(64);
  for (int l = 0; l < st->nlev; ++l) {
    LevelBufs& B = st->lv[l];
    const size_t N = B.g.N;
    for (int q = 0; q < MAXU; ++q) {
      B.e[q] = q < st->nu ? C.take(N * es) : nullptr;
      B.f[q] = q < st->nu ? C.take(N * es) : nullptr;
      B.r[q] = (q < st->nu && l + 1 < st->nlev) ? C.take(N * es) : nullptr;
      B.eh[q] = (q < st->nu && l > 0) ? C.take(N * es) : nullptr;
    }
    const bool alias = (l == 0 && st->prm.precision == FM_FP64);
    if (alias) {
      B.rk = st->rho;
      B.cr = st->g[0];
      for (int d = 0; d < 3; ++d) {
        B.om[d] = st->om[d];
        B.cv[d] = d < st->dim ? st->g[1 + d] : nullptr;
      }
    } else {
      B.rk = C.take(N * es);
      B.cr = C.take(N * es);
      for (int d = 0; d < 3; ++d) {
        B.om[d] = d < st->nom ? C.take(N * es) : nullptr;
        B.cv[d] = d < st->dim ? C.take(N * es) : nullptr;
      }
    }
  }
  if (st->kind == FM_CDFT) {
    st->fft.Jhat = (double2*)C.take(N0 * sizeof(double2));
    st->fft.work = (double2*)C.take(N0 * sizeof(double2));
    const int ns[3] = {st->lv[0].g.nx, st->lv[0].g.ny, st->lv[0].g.nz};
    for (int d = 0; d < 3; ++d)
      st->fft.tw[d] = d < st->dim ? (double2*)C.take((size_t)(ns[d] / 2 + 1) * sizeof(double2)) : nullptr;
  }
  return C.off;
}

}  // namespace fm

using namespace fm;

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
  p->coarsest = 4;
  p->ncoarse = 16;
  p->precision = FM_FP64;
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
  st->dim = grid->dim;
  st->nu = 1 + grid->dim + (fn->kind == FM_PFC ? 2 : 0);
  st->nom = grid->dim == 2 ? 1 : 3;
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
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
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

static cudaMemcpyKind kind_in(int where) {
  return where == FM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
}
static cudaMemcpyKind kind_out(int where) {
  return where == FM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
}

int fm_set_fields(fm_state* st, const double* rho, const double* const* vel, int where) {
  if (!st || !rho || !vel || (where != FM_HOST && where != FM_DEVICE)) return FM_EINVAL;
  const size_t bytes = (size_t)st->lv[0].g.N * sizeof(double);
  FM_CUDA(cudaMemcpyAsync(st->rho, rho, bytes, kind_in(where), st->stream));
  for (int d = 0; d < st->dim; ++d) {
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

int fm_prepare(fm_state* st, double dt) {
  if (!st || !(dt > 0.0)) return FM_EINVAL;
  st->dt = dt;
  return st->prm.precision == FM_MIXED ? dispatch_prepare<float>(st) : dispatch_prepare<double>(st);
}

int fm_step(fm_state* st, double dt, fm_step_info* info) {
  if (!st || !(dt > 0.0)) return FM_EINVAL;
  st->dt = dt;
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
  int rc = st->prm.precision == FM_MIXED ? dispatch_resid<float>(st, st->r64, norm)
                                         : dispatch_resid<double>(st, st->r64, norm);
  if (rc == FM_OK && r) {
    for (int q = 0; q < st->nu; ++q)
      if (r[q]) FM_CUDA(cudaMemcpyAsync(r[q], st->r64[q], bytes, kind_out(where), st->stream));
    FM_CUDA(cudaStreamSynchronize(st->stream));
  }
  return rc;
}

int fm_energy(fm_state* st, double* E, double* F, double* KE) {
  if (!st) return FM_EINVAL;
  const Geo G = st->lv[0].g;
  const double h = st->lv[0].h;
  cudaStream_t s = st->stream;
  if (st->kind == FM_CDFT) {
    const int rc = fft_convolve(st, st->rho, st->tmp);
    if (rc) return rc;
  }
  Vel3 v3{{st->vel[0], st->vel[1], st->vel[2]}};
  const double a = st->fn.alpha;
  if (st->kind == FM_PFC && st->dim == 2)
    k_energy<KPFC, 2><<<st->nblk, TPB, 0, s>>>(st->rho, v3, nullptr, G, h, a, st->partials);
  else if (st->kind == FM_PFC)
    k_energy<KPFC, 3><<<st->nblk, TPB, 0, s>>>(st->rho, v3, nullptr, G, h, a, st->partials);
  else if (st->dim == 2)
    k_energy<KCDFT, 2><<<st->nblk, TPB, 0, s>>>(st->rho, v3, st->tmp, G, h, a, st->partials);
  else
    k_energy<KCDFT, 3><<<st->nblk, TPB, 0, s>>>(st->rho, v3, st->tmp, G, h, a, st->partials);
  FM_LAUNCHED();
  k_final_sum<5><<<1, TPB, 0, s>>>(st->partials, st->nblk, st->dscal + 8);
  FM_LAUNCHED();
  FM_CUDA(cudaMemcpyAsync(st->hscal + 8, st->dscal + 8, 5 * sizeof(double), cudaMemcpyDeviceToHost, s));
  FM_CUDA(cudaStreamSynchronize(s));
  const double w = st->dim == 3 ? h * h * h : h * h;
  const double* q = st->hscal + 8;
  const double ke = w * q[0];
  const double f = w * (q[1] + q[2] + q[3] + q[4]);
  if (E) *E = ke + f;
  if (F) *F = f;
  if (KE) *KE = ke;
  return FM_OK;
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
