// Device code of libfm shared by the single-instance driver (fm_solver.cu)
// and the batched driver (fm_batch.cu): per-point operations of the FAS
// cycle on the correction equation, the fused 2-D red-black tile sweep, the
// single-block small-level V-cycle and the float64 kernels of the finest
// level, each as a device function with a thin kernel wrapper.
#pragma once

#include <cuda.h>  // CUtensorMap (the descriptor type only; no driver calls here)
#include <cuda_runtime.h>
#include <cmath>
#include <cstring>
#include <cstdlib>
#include <type_traits>
#include <utility>

#include "fm_state.h"

namespace fm {

constexpr int TPB = 256;

static inline int nblocks(long long work) { return (int)((work + TPB - 1) / TPB); }

// --------------------------------------------------------------------------
// Smoother point update (correction form)
// --------------------------------------------------------------------------
// Constants of the point update on one level (grid spacing h), formed once
// per thread outside the point loops.
template <typename T>
struct PtK {
  T ih2;    // 1/h^2
  T c_div;  // s/(4h): continuity flux difference
  T c_sih;  // s/h: kinetic-energy and chemical-potential gradients (times rho^k)
  T c_v;    // s gamma/(2h^2): viscous neighbour sum
  T c_ad;   // s gamma d/h^2: viscous diagonal (reading R2)
  T c_b;    // sigma s/2: vorticity coupling (times rho^k omega^k)
  T proj;   // positive projection applied where rho <= proj (see proj_threshold)
};

// The positive projection rho <- sqrt(rho^2 + delta^2) of Sec. 6 changes a
// density x >= delta * sqrt(2 / eps_T) by less than a quarter of its last
// bit, so above that threshold it is the identity in precision T; below it
// (and wherever x <= 0) it is applied.  This gives the projection applied at
// every density update, up to rounding, while the correction e keeps its
// full relative precision where the projection cannot show.
template <typename T>
__host__ __device__ __forceinline__ T proj_threshold(T delta) {
  return delta * (sizeof(T) == 4 ? T(8192) : T(134217728));  // 2^13 ~ sqrt(2/2^-24), 2^27 ~ sqrt(2/2^-53)
}

template <typename T, int DIM>
__device__ __forceinline__ PtK<T> make_ptk(const Phys<T>& P, T h) {
  PtK<T> K;
  const T ih = T(1) / h;
  K.ih2 = ih * ih;
  K.c_div = P.s * T(0.25) * ih;
  K.c_sih = P.s * ih;
  K.c_v = T(0.5) * P.s * P.gamma * K.ih2;
  K.c_ad = P.s * P.gamma * T(DIM) * K.ih2;
  K.c_b = T(0.5) * P.sigma * P.s;
  K.proj = proj_threshold<T>(P.delta);
  return K;
}

// Reciprocal of the point block's velocity determinant: the float32 smoother
// uses the hardware approximate division (its errors only change how fast
// the float64 outer iteration converges); float64 divides exactly.
__device__ __forceinline__ float rcp_blk(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double rcp_blk(double x) { return 1.0 / x; }

// CDFT chemical-potential part of the correction form at a point with
// correction e and coefficient density cr: ln(1 + e / cr) + 2 c_e e (the
// change of ln rho + 2 c_e rho from rho = cr to cr + e).
template <typename T>
__device__ __forceinline__ T cdft_mc(T e, T cr, T ce) {
  return log1p_t(e / cr) + T(2) * ce * e;
}

// An accessor that also provides mcv(i), cdft_mc of point i's current
// correction kept by the launch that last changed it.
template <class A, class = void>
struct HasMcv : std::false_type {};
template <class A>
struct HasMcv<A, std::void_t<decltype(std::declval<const A&>().mcv(0))>> : std::true_type {};

// Point-block update of one point, written against an accessor A that
// provides e(q, i) / set_e(q, i, v), rk(i), cr(i), cv(d, i), f(q, fc) and
// om(d, fc) (A is a level descriptor in any memory, or a shared-memory tile
// with compile-time strides), and optionally mcv(i); K holds the level
// constants.  Neighbours are at n.m / n.p; the right-hand side and omega^k
// are read at index fc.
template <typename T, int KIND, int DIM, class A>
__device__ __forceinline__ void smooth_point_a(const A& a, const Phys<T>& P, const PtK<T>& K, const Nb& n,
                                               int fc) {
  using LY = Layout<KIND, DIM>;
  const T ih2 = K.ih2;
  const int c = n.c;
  const T rkc = a.rk(c);
  const T crc = a.cr(c);
  T eo[LY::NU];
#pragma unroll
  for (int q = 0; q < LY::NU; ++q) eo[q] = a.e(q, c);

  // rho from the continuity row (neighbour velocities only)
  T div = 0;
#pragma unroll
  for (int d = 0; d < DIM; ++d)
    div += a.rk(n.p[d]) * a.e(1 + d, n.p[d]) - a.rk(n.m[d]) * a.e(1 + d, n.m[d]);
  T er = a.f(0, fc) - K.c_div * div;
  {
    const T x = crc + er;
    if (x <= K.proj) er = sqrt_t(x * x + P.delta * P.delta) - crc;  // Sec. 6 projection
  }
  T eg[LY::NU];
  eg[0] = er;

  auto nbs = [&](int q) {
    T s = a.e(q, n.m[0]) + a.e(q, n.p[0]) + a.e(q, n.m[1]) + a.e(q, n.p[1]);
    if constexpr (DIM == 3) s += a.e(q, n.m[2]) + a.e(q, n.p[2]);
    return s;
  };
  auto qc = [&](int idx) {
    T q = 0;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      const T e = a.e(1 + d, idx);
      q += e * (T(2) * a.cv(d, idx) + e);
    }
    return q;
  };
  auto mc = [&](int idx) {
    if constexpr (KIND == KPFC) {
      return a.e(LY::IMU, idx);
    } else if constexpr (HasMcv<A>::value) {
      return a.mcv(idx);
    } else {
      return cdft_mc<T>(a.e(0, idx), a.cr(idx), P.ce);
    }
  };

  if constexpr (KIND == KPFC) {
    // kappa = f5 + Lap_h e_rho with the new centre value
    const T ek = a.f(LY::IKA, fc) + (nbs(0) - T(2 * DIM) * er) * ih2;
    // mu = f4 + [(p+e)^3 - p^3]/3 + alpha e + Lap_h e_kappa (exact: the block is triangular)
    const T psi = crc - T(1.5);
    const T em = a.f(LY::IMU, fc) + er * (psi * psi + psi * er + er * er * T(1.0 / 3.0)) + P.alpha * er
               + (nbs(LY::IKA) - T(2 * DIM) * ek) * ih2;
    eg[LY::IKA] = ek;
    eg[LY::IMU] = em;
  }

  // velocity block: (a I + [b]_x) e_u = rhs
  T rhs[3];
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    const T dq = qc(n.p[d]) - qc(n.m[d]);
    const T dm = mc(n.p[d]) - mc(n.m[d]);
    rhs[d] = a.f(1 + d, fc) - K.c_sih * rkc * (T(0.25) * dq + T(0.5) * dm) + K.c_v * nbs(1 + d);
  }
  const T Ad = rkc + K.c_ad;
  const T bs = K.c_b * rkc;
  if constexpr (DIM == 2) {
    const T b = bs * a.om(0, fc);
    const T inv = rcp_blk(Ad * Ad + b * b);
    eg[1] = (Ad * rhs[0] + b * rhs[1]) * inv;
    eg[2] = (Ad * rhs[1] - b * rhs[0]) * inv;
  } else {
    T b[3], bx[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) b[d] = bs * a.om(d, fc);
    cross<T, 3>(b, rhs, bx);
    const T bdy = b[0] * rhs[0] + b[1] * rhs[1] + b[2] * rhs[2];
    const T inv = rcp_blk(Ad * (Ad * Ad + b[0] * b[0] + b[1] * b[1] + b[2] * b[2]));
#pragma unroll
    for (int d = 0; d < 3; ++d) eg[1 + d] = (Ad * Ad * rhs[d] - Ad * bx[d] + bdy * b[d]) * inv;
  }
  // damping of the whole point block (App. G.3)
  const T w = P.w;
#pragma unroll
  for (int q = 0; q < LY::NU; ++q) a.set_e(q, c, (T(1) - w) * eg[q] + w * eo[q]);
}

// Accessor through a level descriptor; f and omega through (Fr, Om).
template <typename T>
struct LvlAcc {
  const Lvl<T>& L;
  T* const* Fr;
  const T* const* Om;
  __device__ __forceinline__ T h() const { return L.h; }
  __device__ __forceinline__ T e(int q, int i) const { return L.e[q][i]; }
  __device__ __forceinline__ void set_e(int q, int i, T v) const { L.e[q][i] = v; }
  __device__ __forceinline__ T rk(int i) const { return L.rk[i]; }
  __device__ __forceinline__ T cr(int i) const { return L.cr[i]; }
  __device__ __forceinline__ T cv(int d, int i) const { return L.cv[d][i]; }
  __device__ __forceinline__ T f(int q, int i) const { return Fr[q][i]; }
  __device__ __forceinline__ T om(int d, int i) const { return Om[d][i]; }
};

template <typename T, int KIND, int DIM>
__device__ __forceinline__ void smooth_point_ex(const Lvl<T>& L, const Phys<T>& P, const PtK<T>& K, const Nb& n,
                                                T* const* Fr, const T* const* Om, int fc) {
  LvlAcc<T> a{L, Fr, Om};
  smooth_point_a<T, KIND, DIM>(a, P, K, n, fc);
}

template <typename T, int KIND, int DIM>
__device__ __forceinline__ void smooth_point(const Lvl<T>& L, const Phys<T>& P, const PtK<T>& K, const Nb& n) {
  smooth_point_ex<T, KIND, DIM>(L, P, K, n, L.f, L.om, n.c);
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
  T M[LY::NU], fv[LY::NU];
  // all loads before the first store: the arrays may alias as far as the
  // compiler knows, so interleaving would serialise them
#pragma unroll
  for (int q = 0; q < LY::NU; ++q) fv[q] = L.f[q][idx];
  applyM<T, KIND, DIM>(L, P, n, L.e, M);
#pragma unroll
  for (int q = 0; q < LY::NU; ++q) L.r[q][idx] = fv[q] - M[q];
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
  T fr[NU], ev[NU];  // all loads before the first store
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
    fr[q] = acc * norm;
    ev[q] = F.e[q][ctr];
  }
#pragma unroll
  for (int q = 0; q < NU; ++q) {
    C.f[q][idx] = fr[q];
    C.e[q][idx] = ev[q];
    C.eh[q][idx] = ev[q];
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
// e_F += P(e_C - eh_C) at fine point idx; for delta > 0 (the CDFT case,
// where ln rho needs a positive argument) the corrected density c + e is then
// projected as in the smoother (Sec. 6, item 1).
template <typename T, int NU, int DIM>
__device__ __forceinline__ void prolong_point(const Lvl<T>& F, const Lvl<T>& C, const Phys<T>& P, int idx) {
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
  T ev[NU];  // all loads before the first store
#pragma unroll
  for (int q = 0; q < NU; ++q) {
    T acc = 0;
    for (int c = 0; c < nzp; ++c)
      for (int b = 0; b < nyp; ++b)
        for (int a = 0; a < nxp; ++a) {
          const int ci = (zi[c] * C.g.ny + yi[b]) * C.g.nx + xi[a];
          acc += C.e[q][ci] - C.eh[q][ci];
        }
    ev[q] = F.e[q][idx] + w * acc;
  }
  if (P.delta > T(0)) {
    const T c = F.cr[idx];
    const T x = c + ev[0];
    if (x <= proj_threshold<T>(P.delta)) ev[0] = sqrt_t(x * x + P.delta * P.delta) - c;
  }
#pragma unroll
  for (int q = 0; q < NU; ++q) F.e[q][idx] = ev[q];
}

// Coarse point idx: f_C = FW(r_F) + M_C(eh_C), e_C = eh_C = inject(e_F), in
// one pass.  Every coarse coefficient is the injection of the fine one, so
// M_C(eh) at the coarse point is evaluated on the fine arrays at the fine
// indices 2I and 2I +- 2 with the coarse spacing.
template <typename T, int KIND, int DIM>
__device__ __forceinline__ void coarse_m_on_fine(const Lvl<T>& F, const Lvl<T>& C, const Phys<T>& P, int idx);

template <typename T, int KIND, int DIM>
__device__ __forceinline__ void restrict_rhs_point(const Lvl<T>& F, const Lvl<T>& C, const Phys<T>& P, int idx) {
  using LY = Layout<KIND, DIM>;
  restrict_point<T, LY::NU, DIM>(F, C, idx);
  coarse_m_on_fine<T, KIND, DIM>(F, C, P, idx);
}

// f_C += M_C(eh_C) at coarse point idx, evaluated on the fine arrays (see
// restrict_rhs_point).
template <typename T, int KIND, int DIM>
__device__ __forceinline__ void coarse_m_on_fine(const Lvl<T>& F, const Lvl<T>& C, const Phys<T>& P, int idx) {
  using LY = Layout<KIND, DIM>;
  int I, J, K;
  coords(idx, C.g, I, J, K);
  const int fnx = F.g.nx, fny = F.g.ny, fnz = F.g.nz;
  const int fi = 2 * I, fj = 2 * J, fk = 2 * K;
  Nb n;
  const int row = (fk * fny + fj) * fnx;
  n.c = row + fi;
  n.m[0] = row + (fi == 0 ? fnx - 2 : fi - 2);
  n.p[0] = row + (fi + 2 >= fnx ? fi + 2 - fnx : fi + 2);
  n.m[1] = n.c + (fj == 0 ? (fny - 2) * fnx : -2 * fnx);
  n.p[1] = n.c + (fj + 2 >= fny ? (2 - fny) * fnx : 2 * fnx);
  if constexpr (DIM == 3) {
    const int pl = fnx * fny;
    n.m[2] = n.c + (fk == 0 ? (fnz - 2) * pl : -2 * pl);
    n.p[2] = n.c + (fk + 2 >= fnz ? (2 - fnz) * pl : 2 * pl);
  } else {
    n.m[2] = n.p[2] = n.c;
  }
  Lvl<T> V = F;
  V.h = C.h;
  T M[LY::NU];
  T fv[LY::NU];
#pragma unroll
  for (int q = 0; q < LY::NU; ++q) fv[q] = C.f[q][idx];
  applyM<T, KIND, DIM>(V, P, n, F.e, M);
#pragma unroll
  for (int q = 0; q < LY::NU; ++q) C.f[q][idx] = fv[q] + M[q];
}

template <typename T, int KIND, int DIM>
__global__ void __launch_bounds__(TPB) k_restrict_rhs(Lvl<T> F, Lvl<T> C, Phys<T> P) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < C.g.N) restrict_rhs_point<T, KIND, DIM>(F, C, P, idx);
}

// 2-D, one launch in place of k_resid + k_restrict_rhs: a block takes a
// tile of RR_TX x RR_TY coarse points, computes the fine residual
// r = f - M(e) on the (2 RR_TX + 1) x (2 RR_TY + 1) fine points their full
// weighting reads into shared memory (r is not written to the level), then
// f_C = FW(r) + M_C(eh_C) and e_C = eh_C = inject(e_F) on the tile.
constexpr int RR_TX = 16, RR_TY = 8;

constexpr int RR_FN = (2 * RR_TX + 1) * (2 * RR_TY + 1);  // fine points per tile

// Coarse tile (I0, J0); sr: shared memory for NU x RR_FN values.
template <typename T, int KIND>
__device__ __forceinline__ void resid_restrict2_tile(const Lvl<T>& F, const Lvl<T>& C, const Phys<T>& P, int I0,
                                                     int J0, T* sr) {
  constexpr int NU = Layout<KIND, 2>::NU;
  constexpr int FW = 2 * RR_TX + 1, FN = RR_FN;
  for (int t = threadIdx.x; t < FN; t += blockDim.x) {
    const int ly = t / FW, lx = t - ly * FW;
    const int x = wrapi(2 * I0 - 1 + lx, F.g.nx), y = wrapi(2 * J0 - 1 + ly, F.g.ny);
    const Nb n = neighbours(x, y, 0, F.g);
    T M[NU];
    applyM<T, KIND, 2>(F, P, n, F.e, M);
#pragma unroll
    for (int q = 0; q < NU; ++q) sr[q * FN + t] = F.f[q][n.c] - M[q];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < RR_TX * RR_TY; t += blockDim.x) {
    const int ty = t / RR_TX, tx = t - ty * RR_TX;
    const int I = I0 + tx, J = J0 + ty;
    if (I >= C.g.nx || J >= C.g.ny) continue;
    const int cidx = J * C.g.nx + I;
    const int c = (2 * ty + 1) * FW + 2 * tx + 1;
    const int ctr = 2 * J * F.g.nx + 2 * I;
    T ev[NU];
#pragma unroll
    for (int q = 0; q < NU; ++q) ev[q] = F.e[q][ctr];
#pragma unroll
    for (int q = 0; q < NU; ++q) {
      const T* r = sr + q * FN;
      T acc = T(0);
      acc += r[c - FW - 1] + T(2) * r[c - FW] + r[c - FW + 1];
      acc += T(2) * (r[c - 1] + T(2) * r[c] + r[c + 1]);
      acc += r[c + FW - 1] + T(2) * r[c + FW] + r[c + FW + 1];
      C.f[q][cidx] = acc * T(1.0 / 16.0);
      C.e[q][cidx] = ev[q];
      C.eh[q][cidx] = ev[q];
    }
    coarse_m_on_fine<T, KIND, 2>(F, C, P, cidx);
  }
}

template <typename T, int KIND>
__global__ void __launch_bounds__(TPB) k_resid_restrict2(Lvl<T> F, Lvl<T> C, Phys<T> P, int ntx) {
  __shared__ T sr[Layout<KIND, 2>::NU * RR_FN];
  resid_restrict2_tile<T, KIND>(F, C, P, (blockIdx.x % ntx) * RR_TX, (blockIdx.x / ntx) * RR_TY, sr);
}

template <typename T, int KIND, int DIM>
__global__ void __launch_bounds__(TPB) k_smooth(Lvl<T> L, Phys<T> P, int color) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  int i, j, k;
  if (!colour_point(t, color, L.g, i, j, k)) return;
  const Nb n = neighbours(i, j, k, L.g);
  smooth_point<T, KIND, DIM>(L, P, make_ptk<T, DIM>(P, L.h), n);
}

// Level accessor whose neighbours' CDFT chemical-potential parts come from M.
struct McAcc64 {
  const Lvl<double>& L;
  const double* M;
  __device__ __forceinline__ double e(int q, int i) const { return L.e[q][i]; }
  __device__ __forceinline__ void set_e(int q, int i, double v) const { L.e[q][i] = v; }
  __device__ __forceinline__ double rk(int i) const { return L.rk[i]; }
  __device__ __forceinline__ double cr(int i) const { return L.cr[i]; }
  __device__ __forceinline__ double cv(int d, int i) const { return L.cv[d][i]; }
  __device__ __forceinline__ double f(int q, int i) const { return L.f[q][i]; }
  __device__ __forceinline__ double om(int d, int i) const { return L.om[d][i]; }
  __device__ __forceinline__ double mcv(int i) const { return M[i]; }
};

// A CDFT colour launch of the float64 coarsest-level sweeps that keeps
// M[i] = cdft_mc of every point it updates: the next launch (the other
// colour) reads its neighbours' values from M instead of evaluating the
// logarithm at each of them (2 DIM evaluations a point on GB300's slow
// float64 pipe become one).  The first launch of a solve (USE_M false)
// evaluates its neighbours' values itself, as k_smooth does; M of a colour is
// read only by the launch after the one that wrote it, so values and order
// are those of k_smooth.
template <int DIM, bool USE_M>
__global__ void __launch_bounds__(TPB) k_smooth_cdft64_mc(Lvl<double> L, Phys<double> P, int color, double* M) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  int i, j, k;
  if (!colour_point(t, color, L.g, i, j, k)) return;
  const Nb n = neighbours(i, j, k, L.g);
  const PtK<double> K = make_ptk<double, DIM>(P, L.h);
  if constexpr (USE_M) {
    const McAcc64 a{L, M};
    smooth_point_a<double, KCDFT, DIM>(a, P, K, n, n.c);
  } else {
    smooth_point<double, KCDFT, DIM>(L, P, K, n);
  }
  M[n.c] = cdft_mc<double>(L.e[0][n.c], L.cr[n.c], P.ce);
}

// The same colour sweep compiled for six resident blocks per SM (at most 40
// registers a thread instead of 64): the 3-D point update waits on its many
// cached loads, and more warps in flight hide that latency.  The 3-D
// autotuner times it against k_smooth per level (it spills in float64).
template <typename T, int KIND, int DIM>
__global__ void __launch_bounds__(TPB, 6) k_smooth_occ(Lvl<T> L, Phys<T> P, int color) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  int i, j, k;
  if (!colour_point(t, color, L.g, i, j, k)) return;
  const Nb n = neighbours(i, j, k, L.g);
  smooth_point<T, KIND, DIM>(L, P, make_ptk<T, DIM>(P, L.h), n);
}

// One colour of a sweep over the rows [row0, row0 + nrows) of a 3-D level
// (a row is one (j, k); rows past the last wrap to the first), bounded to six
// blocks per SM like k_smooth_occ.  Used to sweep the level in z-chunks.
template <typename T, int KIND, int DIM>
__global__ void __launch_bounds__(TPB, 6) k_smooth_rows(Lvl<T> L, Phys<T> P, int color, int row0, int nrows) {
  const int half = L.g.nx >> 1;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)nrows * half) return;
  const int nr = L.g.ny * L.g.nz;
  int rowid = row0 + (int)(t / half);
  if (rowid >= nr) rowid -= nr;
  const int j = rowid % L.g.ny, k = rowid / L.g.ny;
  const int i = 2 * (int)(t % half) + ((j + k + color) & 1);
  const Nb n = neighbours(i, j, k, L.g);
  smooth_point<T, KIND, DIM>(L, P, make_ptk<T, DIM>(P, L.h), n);
}

// 3-D sweep variants: 0 k_smooth, 1 k_smooth_occ, 2 the same sweep in
// z-chunks (z_chunk_planes): red over a chunk, then black over the planes
// whose z-neighbours are all red by then, so the black launch finds the
// chunk's arrays in L2; the same updates in the same order of dependence as
// a red and a black launch over the whole level; 3 and 4 the fused
// z-marching sweep (fm_zmarch.cuh) with 32 x 8 and 32 x 16 tiles, one launch
// per sweep, reading the correction from one buffer and writing the other.
constexpr int SM3_NVAR = 5;
constexpr int SM3_ZM = 3;  // first z-marching variant

// Planes per chunk: the largest divisor of nz whose arrays (about 20 float
// words a point) stay within 48 MB, at least 2; 0 (no chunking) when the
// whole level does.
static inline int z_chunk_planes(const Geo& g) {
  const double plane = 80.0 * g.nx * (double)g.ny;
  if (plane * g.nz <= 48e6 || g.nz < 4) return 0;
  const char* fixed = getenv("FM_ZCHUNK");  // planes per chunk, for measurements (a divisor of nz)
  if (fixed && fixed[0]) {
    const int z = atoi(fixed);
    if (z >= 2 && z <= g.nz / 2 && g.nz % z == 0) return z;
  }
  int best = 0;
  for (int z = 2; z <= g.nz / 2; ++z)
    if (g.nz % z == 0 && plane * z <= 48e6) best = z;
  return best;
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
__global__ void __launch_bounds__(TPB) k_prolong(Lvl<T> F, Lvl<T> C, Phys<T> P) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < F.g.N) prolong_point<T, NU, DIM>(F, C, P, idx);
}

// Fused red-black sweep of a 2-D level in TX x TY tiles.  The tile and a
// halo of two points of every array the point update reads are staged in
// shared memory; red points are updated on the tile and its first halo ring
// (their black neighbours are all staged), then black points on the tile, and
// the tile's corrections are written back.  Red values on the ring are
// recomputed identically by the neighbouring tiles, so a sweep equals a red
// launch followed by a black launch.  Blocks are persistent: each walks a
// strided sequence of tiles with two shared-memory buffers, copying the next
// tile in with cp.async (global -> shared, no register staging) while it
// computes the current one.  The two-sweep form (NS = 2) stages a halo of
// four and runs both sweeps on the tile in one launch.
constexpr int RB_H = 2;
// Threads of a tile block: enough whole warps for the red pass over the tile
// and its first halo ring ((tx + 2)/2 x (ty + 2) points) in one round.
__host__ __device__ constexpr int rb_threads(int tx, int ty) { return ((tx + 2) / 2 * (ty + 2) + 31) / 32 * 32; }
// Minimum resident blocks per SM the float32 tile kernels are compiled for
// (caps their registers so that four blocks fit; measured best on GB300).
template <typename T>
__host__ __device__ constexpr int rb_minb(int tx, int ty) {
  return sizeof(T) == 4 ? (2048 / rb_threads(tx, ty) < 4 ? 2048 / rb_threads(tx, ty) : 4) : 1;
}

// The dynamic shared memory of the tile kernels (every extern __shared__
// array of a kernel starts at the same address).
extern __shared__ __align__(16) unsigned char fm_dyn_smem[];

// Accessor of a staged tile: arrays e[NU], rk, cr, cv0, cv1 and (SF) f[NU],
// omega at compile-time strides SN from element `base` of the dynamic shared
// memory, so every access is a shared-memory load; without SF the right-hand
// side and omega are read from the level in global memory.
template <typename T, int KIND, int SN, bool SF>
struct TileAcc {
  static constexpr int NU = Layout<KIND, 2>::NU;
  int base;
  T hh;
  const Lvl<T>* G;
  __device__ __forceinline__ T* sm() const { return reinterpret_cast<T*>(fm_dyn_smem) + base; }
  __device__ __forceinline__ T h() const { return hh; }
  __device__ __forceinline__ T e(int q, int i) const { return sm()[q * SN + i]; }
  __device__ __forceinline__ void set_e(int q, int i, T v) const { sm()[q * SN + i] = v; }
  __device__ __forceinline__ T rk(int i) const { return sm()[NU * SN + i]; }
  __device__ __forceinline__ T cr(int i) const { return sm()[(NU + 1) * SN + i]; }
  __device__ __forceinline__ T cv(int d, int i) const { return sm()[(NU + 2 + d) * SN + i]; }
  __device__ __forceinline__ T f(int q, int i) const {
    if constexpr (SF) return sm()[(NU + 4 + q) * SN + i];
    else return G->f[q][i];
  }
  __device__ __forceinline__ T om(int d, int i) const {
    if constexpr (SF) return sm()[(2 * NU + 4) * SN + i];
    else return G->om[d][i];
  }
};

// Shared-memory tile: rows of SW = TX + 2*XO values (the tile starts at
// column XO = 4 so that every row begins on a 16-byte boundary in global and
// shared memory), TY + 2*RB_H rows.
constexpr int RB_XO = 4;

template <int TX, int TY, int NS = 1>
struct RBGeom {
  static constexpr int H = RB_H * NS;  // halo rows: two per sweep of the pass
  static constexpr int SW = TX + 2 * RB_XO;
  static constexpr int SN = SW * (TY + 2 * H);
};

// Arrays staged per tile: e (NU), rk, cr, cv0, cv1, and with SF also f (NU)
// and omega (otherwise f and omega are read from global memory).
template <int KIND, bool SF>
__host__ __device__ constexpr int rb_arrays() {
  return Layout<KIND, 2>::NU + 4 + (SF ? Layout<KIND, 2>::NU + 1 : 0);
}

template <typename T, int KIND, int TX, int TY, bool SF, bool PIPE, int NS = 1>
__host__ __device__ constexpr size_t rb_smem_bytes() {
  return (PIPE ? 2 : 1) * (size_t)rb_arrays<KIND, SF>() * RBGeom<TX, TY, NS>::SN * sizeof(T);
}


template <typename T>
__device__ __forceinline__ void cp_async_elem(T* smem, const T* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  if constexpr (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
template <typename T>
__device__ __forceinline__ void cp_async_16(T* smem, const T* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_one() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
// Wait until at most N of this thread's most recent copy groups are pending.
template <int N>
__device__ __forceinline__ void cp_async_wait_n() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Start the copies of tile (x0, y0) of level G into buf: 16-byte chunks when
// the row length is a multiple of the chunk (chunks then never straddle the
// periodic wrap), single elements otherwise.  The correction is read from G.e
// (dir = 0) or from G.r (dir = 1).
template <typename T, int KIND, int TX, int TY, bool SF, int NS = 1>
__device__ __forceinline__ void rb2d_issue(const Lvl<T>& G, T* buf, int x0, int y0, int dir) {
  using Gm = RBGeom<TX, TY, NS>;
  constexpr int NU = Layout<KIND, 2>::NU;
  constexpr int NA = rb_arrays<KIND, SF>();
  constexpr int V = 16 / sizeof(T);
  const int nx = G.g.nx, ny = G.g.ny;
  const T* src[NA];
#pragma unroll
  for (int q = 0; q < NU; ++q) src[q] = dir ? G.r[q] : G.e[q];
  src[NU + 0] = G.rk;
  src[NU + 1] = G.cr;
  src[NU + 2] = G.cv[0];
  src[NU + 3] = G.cv[1];
  if constexpr (SF) {
#pragma unroll
    for (int q = 0; q < NU; ++q) src[NU + 4 + q] = G.f[q];
    src[2 * NU + 4] = G.om[0];
  }
  if (nx % V == 0) {
    constexpr int CPR = Gm::SW / V;  // chunks per row
    constexpr int NCH = CPR * (TY + 2 * Gm::H);
    for (int t = threadIdx.x; t < NCH; t += blockDim.x) {
      const int ly = t / CPR, c = t - ly * CPR;
      const int gidx = wrapi(y0 + ly - Gm::H, ny) * nx + wrapi(x0 - RB_XO + c * V, nx);
      const int sidx = ly * Gm::SW + c * V;
#pragma unroll
      for (int a = 0; a < NA; ++a) cp_async_16(buf + a * Gm::SN + sidx, src[a] + gidx);
    }
  } else {
    for (int t = threadIdx.x; t < Gm::SN; t += blockDim.x) {
      const int ly = t / Gm::SW, lx = t - ly * Gm::SW;
      const int gidx = wrapi(y0 + ly - Gm::H, ny) * nx + wrapi(x0 + lx - RB_XO, nx);
#pragma unroll
      for (int a = 0; a < NA; ++a) cp_async_elem(buf + a * Gm::SN + t, src[a] + gidx);
    }
  }
}

// NS = 1: red pass on tile + ring 1, black pass on the tile.  NS = 2 (two
// sweeps, halo of four): red on tile + ring 3, black on ring 2, red on ring
// 1, black on the tile -- each pass reads only values the previous pass has
// finished on its wider ring.  Then the tile is written back to G.r (dir = 0)
// or G.e (dir = 1); the staged tile starts at element `base` of the dynamic
// shared memory.
template <typename T, int KIND, int TX, int TY, bool SF, int NS = 1>
__device__ __forceinline__ void rb2d_compute(const Lvl<T>& G, const Phys<T>& P, int base, int x0, int y0,
                                             int dir) {
  using Gm = RBGeom<TX, TY, NS>;
  constexpr int NU = Layout<KIND, 2>::NU;
  constexpr int SN = Gm::SN, SW = Gm::SW;
  const TileAcc<T, KIND, SN, SF> acc{base, G.h, &G};
  const PtK<T> K = make_ptk<T, 2>(P, G.h);
  const int nx = G.g.nx, ny = G.g.ny;
#pragma unroll
  for (int pass = 0; pass < 2 * NS; ++pass) {
    const int color = pass & 1;           // red (i + j even) first, then black
    const int ring = 2 * NS - 1 - pass;   // halo rings the pass also covers
    const int w = TX + 2 * ring;          // even
    const int hw = w >> 1;
    const int npts = hw * (TY + 2 * ring);
    for (int t = threadIdx.x; t < npts; t += blockDim.x) {
      const int ry = t / hw;
      const int gy = y0 - ring + ry;
      const int rx = 2 * (t - ry * hw) + ((color + x0 + ring + gy) & 1);
      const int lx = RB_XO - ring + rx, ly = Gm::H - ring + ry;
      Nb n;
      n.c = ly * SW + lx;
      n.m[0] = n.c - 1;
      n.p[0] = n.c + 1;
      n.m[1] = n.c - SW;
      n.p[1] = n.c + SW;
      n.m[2] = n.p[2] = n.c;
      const int fc = SF ? n.c : wrapi(gy, ny) * nx + wrapi(x0 - ring + rx, nx);
      smooth_point_a<T, KIND, 2>(acc, P, K, n, fc);
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < TX * TY; t += blockDim.x) {
    const int ty = t / TX, tx = t - ty * TX;
    const int gx = x0 + tx, gy = y0 + ty;
    if (gx < nx && gy < ny) {
      const int sidx = (ty + Gm::H) * SW + tx + RB_XO;
#pragma unroll
      for (int q = 0; q < NU; ++q) (dir ? G.e[q] : G.r[q])[gy * nx + gx] = acc.e(q, sidx);
    }
  }
}

// Single level.  PIPE: persistent blocks over tiles t = blockIdx.x,
// blockIdx.x + gridDim.x, ..., the next tile's copies in flight while the
// current one is computed; otherwise one tile per block.
//
// The sweep reads the correction from one buffer and writes it to the other
// (G.e -> G.r for dir = 0, G.r -> G.e for dir = 1; the residual buffer of a
// level is free while the level is smoothed).  A tile's halo therefore always
// holds values from before the sweep, whichever tiles have already been
// written, so the result is exactly one red-black sweep for any block
// schedule.
template <typename T, int KIND, int TX, int TY, bool SF, bool PIPE, int NS = 1>
__global__ void __launch_bounds__(rb_threads(TX, TY), rb_minb<T>(TX, TY)) k_smooth_rb2d(Lvl<T> G, Phys<T> P, int ntx, int ntiles,
                                                                    int dir) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* buf0 = reinterpret_cast<T*>(smraw);
  constexpr int BUFSTRIDE = rb_arrays<KIND, SF>() * RBGeom<TX, TY, NS>::SN;
  int t = blockIdx.x;
  if (t >= ntiles) return;
  if constexpr (!PIPE) {
    rb2d_issue<T, KIND, TX, TY, SF, NS>(G, buf0, (t % ntx) * TX, (t / ntx) * TY, dir);
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
    rb2d_compute<T, KIND, TX, TY, SF, NS>(G, P, 0, (t % ntx) * TX, (t / ntx) * TY, dir);
  } else {
    rb2d_issue<T, KIND, TX, TY, SF, NS>(G, buf0, (t % ntx) * TX, (t / ntx) * TY, dir);
    cp_async_commit();
    for (int k = 0;; ++k) {
      const int tn = t + gridDim.x;
      const bool next = tn < ntiles;
      if (next)
        rb2d_issue<T, KIND, TX, TY, SF, NS>(G, buf0 + ((k + 1) & 1) * BUFSTRIDE, (tn % ntx) * TX, (tn / ntx) * TY, dir);
      cp_async_commit();
      cp_async_wait_one();
      __syncthreads();
      rb2d_compute<T, KIND, TX, TY, SF, NS>(G, P, (k & 1) * BUFSTRIDE, (t % ntx) * TX, (t / ntx) * TY, dir);
      __syncthreads();
      if (!next) break;
      t = tn;
    }
  }
}

// --------------------------------------------------------------------------
// Tile staging by tensor copies (TMA)
// --------------------------------------------------------------------------
// The staged arrays of the two-sweep tile form are one box each: SW x (TY +
// 2H) values from (x0 - RB_XO, y0 - H), the layout the tile already has in
// shared memory.  One thread issues one cp.async.bulk.tensor per array onto
// an mbarrier that expects the bytes of all of them; every thread then waits
// on it, with a time limit.  A box that crosses the periodic boundary gets
// zeros there from the copy (the tensor map does not wrap), and those cells
// are then loaded with their wrapped values by plain loads.  The x coordinate
// x0 - RB_XO is a multiple of 4 elements (16 bytes) for every tile.
struct RbMaps {
  CUtensorMap m[MAXU + 4];  // staged arrays in rb2d_issue order: e (or r) [NU], rk, cr, cv0, cv1
};

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait for phase `parity` of the mbarrier for at most `limit_ns`; false when
// the limit ran out.
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity, unsigned long long limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait(bar, parity))
    if (global_ns() - t0 > limit_ns) return false;
  return true;
}
__device__ __forceinline__ void tma_load_2d(unsigned dst, const CUtensorMap* map, int x, int y, unsigned bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
      "[%4];\n" ::"r"(dst),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

constexpr unsigned long long TMA_WAIT_NS = 1000000000ull;  // 1 s: a tile's copies take microseconds

// One tile per block, staged by tensor copies, then the passes of
// rb2d_compute (the same updates, in the same order, as k_smooth_rb2d with
// SF = false and PIPE = false).  If the copies do not complete within the
// limit the block sets *fault, waits once more for them and returns without
// writing its tile (the step then reports FM_ETIMEOUT).
template <typename T, int KIND, int TX, int TY, int NS>
__global__ void __launch_bounds__(rb_threads(TX, TY), rb_minb<T>(TX, TY))
    k_smooth_rb2d_tma(Lvl<T> G, Phys<T> P, int ntx, int ntiles, int dir, const __grid_constant__ RbMaps maps,
                      int* fault) {
  using Gm = RBGeom<TX, TY, NS>;
  constexpr int NU = Layout<KIND, 2>::NU;
  constexpr int NA = rb_arrays<KIND, false>();
  constexpr int SN = Gm::SN, SW = Gm::SW;
  constexpr unsigned ABYTES = SN * sizeof(T);  // a multiple of 128 for the tiles instantiated
  static_assert(ABYTES % 128 == 0, "each staged array must start on a 128-byte boundary");
  __shared__ __align__(8) unsigned long long bar;
  const int t = blockIdx.x;
  if (t >= ntiles) return;
  const int x0 = (t % ntx) * TX, y0 = (t / ntx) * TY;
  const unsigned s0 = smem_u32(fm_dyn_smem);
  const unsigned sa = (s0 + 127u) & ~127u;  // the launch adds 128 bytes for this
  const int base = (int)((sa - s0) / sizeof(T));
  const unsigned b = smem_u32(&bar);
  if (threadIdx.x == 0) mbar_init(b, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_expect_tx(b, NA * ABYTES);
#pragma unroll
    for (int a = 0; a < NA; ++a) tma_load_2d(sa + a * ABYTES, &maps.m[a], x0 - RB_XO, y0 - Gm::H, b);
  }
  if (!__syncthreads_and(mbar_wait(b, 0, TMA_WAIT_NS))) {
    if (threadIdx.x == 0) atomicExch(fault, 1);
    mbar_wait(b, 0, TMA_WAIT_NS);  // the copies may still be in flight
    return;
  }
  const int nx = G.g.nx, ny = G.g.ny;
  if (x0 - RB_XO < 0 || x0 + TX + RB_XO > nx || y0 - Gm::H < 0 || y0 + TY + Gm::H > ny) {
    T* buf = reinterpret_cast<T*>(fm_dyn_smem) + base;
    const T* src[NA];
#pragma unroll
    for (int q = 0; q < NU; ++q) src[q] = dir ? G.r[q] : G.e[q];
    src[NU + 0] = G.rk;
    src[NU + 1] = G.cr;
    src[NU + 2] = G.cv[0];
    src[NU + 3] = G.cv[1];
    for (int c = threadIdx.x; c < SN; c += blockDim.x) {
      const int ly = c / SW, lx = c - ly * SW;
      const int gx = x0 - RB_XO + lx, gy = y0 - Gm::H + ly;
      if (gx < 0 || gx >= nx || gy < 0 || gy >= ny) {
        const int gi = wrapi(gy, ny) * nx + wrapi(gx, nx);
#pragma unroll
        for (int a = 0; a < NA; ++a) buf[a * SN + c] = src[a][gi];
      }
    }
    __syncthreads();
  }
  rb2d_compute<T, KIND, TX, TY, false, NS>(G, P, base, x0, y0, dir);
}

// --------------------------------------------------------------------------
// 2-D fused red-black sweep, row-marching form
// --------------------------------------------------------------------------
// A block owns the columns [x0, x0 + TX) of rows [y0, y1) of one level and
// marches down them two rows per step.  Step s (ya = y0 - 2 + 2 s) updates
// the red points of rows ya + 1 and ya + 2, then the black points of rows ya
// and ya + 1, after which rows ya and ya + 1 are final and are written out.
// Each thread owns one column (its red and its black point of every step),
// so a step needs one barrier, between its red and its black half.
//
// The arrays the point update reads at neighbours -- e, rho^k, the
// coefficient velocity and, for CDFT, the coefficient density -- are staged
// by cp.async into a ring of MR row slots, two steps ahead of their use.  The
// right-hand side, omega^k and (PFC) the coefficient density are read only
// at the point itself: they go to registers, one step ahead.  The red points
// of the columns x0 - 1 and x0 + TX (two lanes of an extra warp) and of the
// rows y0 - 1 and y1 are computed again by the blocks that own them; as in
// the tile form, e is read from one buffer and written to the other, so all
// staged values are from before the sweep and the result is exactly one
// red-black sweep.
constexpr int MR = 10;  // row slots: rows ya - 1 .. ya + 7 are live in step s

template <int KIND>
__host__ __device__ constexpr int march_arrays() {
  return Layout<KIND, 2>::NU + 3 + (KIND == KCDFT ? 1 : 0);  // e, rk, cv0, cv1 (, cr)
}
template <typename T, int KIND, int TX>
__host__ __device__ constexpr size_t march_smem_bytes() {
  return (size_t)MR * march_arrays<KIND>() * (TX + 2 * RB_XO) * sizeof(T);
}
__host__ __device__ constexpr int march_threads(int tx) { return tx + 32; }
// Minimum resident blocks the float32 128-wide marching kernel is compiled
// for (registers capped so that five blocks fit; measured best on GB300).
template <typename T>
__host__ __device__ constexpr int march_minb(int tx) { return (sizeof(T) == 4 && tx == 128) ? 5 : 1; }

// Values of one point read only at that point.
template <typename T, int KIND>
struct MarchPt {
  T fv[Layout<KIND, 2>::NU];
  T omv, crv;
};

template <typename T, int KIND>
__device__ __forceinline__ void march_load_pt(const Lvl<T>& G, int gidx, MarchPt<T, KIND>& p) {
#pragma unroll
  for (int q = 0; q < Layout<KIND, 2>::NU; ++q) p.fv[q] = G.f[q][gidx];
  p.omv = G.om[0][gidx];
  p.crv = KIND == KPFC ? G.cr[gidx] : T(0);
}

// Accessor of the point update over the row ring (index = slot * NA * SW +
// staged column, array a at offset a * SW) and one point's register values.
template <typename T, int KIND, int SW>
struct MarchAcc {
  static constexpr int NU = Layout<KIND, 2>::NU;
  T* sm;
  const MarchPt<T, KIND>& p;
  __device__ __forceinline__ T e(int q, int i) const { return sm[i + q * SW]; }
  __device__ __forceinline__ void set_e(int q, int i, T v) const { sm[i + q * SW] = v; }
  __device__ __forceinline__ T rk(int i) const { return sm[i + NU * SW]; }
  __device__ __forceinline__ T cv(int d, int i) const { return sm[i + (NU + 1 + d) * SW]; }
  __device__ __forceinline__ T cr(int i) const {
    if constexpr (KIND == KCDFT) return sm[i + (NU + 3) * SW];
    else return p.crv;  // the PFC update reads the coefficient density at the point only
  }
  __device__ __forceinline__ T f(int q, int) const { return p.fv[q]; }
  __device__ __forceinline__ T om(int, int) const { return p.omv; }
};

// Start the copies of rows row0 and row0 + 1 (local rows lrow0, lrow0 + 1,
// counted from y0 - 2) into their ring slots.
template <typename T, int KIND, int TX, int NR = MR>
__device__ __forceinline__ void march_issue2(const Lvl<T>& G, T* buf, int x0, int row0, int lrow0, int dir) {
  constexpr int NU = Layout<KIND, 2>::NU;
  constexpr int NA = march_arrays<KIND>();
  constexpr int SW = TX + 2 * RB_XO;
  constexpr int V = 16 / sizeof(T);
  const int nx = G.g.nx, ny = G.g.ny;
  const T* src[NA];
#pragma unroll
  for (int q = 0; q < NU; ++q) src[q] = dir ? G.r[q] : G.e[q];
  src[NU] = G.rk;
  src[NU + 1] = G.cv[0];
  src[NU + 2] = G.cv[1];
  if constexpr (KIND == KCDFT) src[NU + 3] = G.cr;
  if (nx % V == 0) {
    constexpr int CPR = SW / V;
    for (int t = threadIdx.x; t < 2 * CPR; t += blockDim.x) {
      const int k = t >= CPR, c = t - k * CPR;
      const int gi = wrapi(row0 + k, ny) * nx + wrapi(x0 - RB_XO + c * V, nx);
      T* d = buf + ((lrow0 + k) % NR) * NA * SW + c * V;
#pragma unroll
      for (int a = 0; a < NA; ++a) cp_async_16(d + a * SW, src[a] + gi);
    }
  } else {
    for (int t = threadIdx.x; t < 2 * SW; t += blockDim.x) {
      const int k = t >= SW, c = t - k * SW;
      const int gi = wrapi(row0 + k, ny) * nx + wrapi(x0 - RB_XO + c, nx);
      T* d = buf + ((lrow0 + k) % NR) * NA * SW + c;
#pragma unroll
      for (int a = 0; a < NA; ++a) cp_async_elem(d + a * SW, src[a] + gi);
    }
  }
}

// One fused sweep of the block's strip (see above); buf is the ring in
// dynamic shared memory.
template <typename T, int KIND, int TX>
__device__ __forceinline__ void march_sweep(const Lvl<T>& G, const Phys<T>& P, T* buf, int x0, int y0, int y1,
                                            int dir) {
  constexpr int NU = Layout<KIND, 2>::NU;
  constexpr int NA = march_arrays<KIND>();
  constexpr int SW = TX + 2 * RB_XO;
  constexpr int RS = NA * SW;  // stride of a row slot
  const int nx = G.g.nx, ny = G.g.ny;
  const int txe = min(TX, nx - x0);
  const PtK<T> K = make_ptk<T, 2>(P, G.h);
  // this thread's staged column: interior x0 + tid, or (lanes 0, 1 of the
  // last warp) the red-only columns x0 - 1 and x0 + txe
  const int tid = threadIdx.x;
  const bool interior = tid < txe;
  int lx = -1;
  if (interior) lx = RB_XO + tid;
  else if (tid == TX) lx = RB_XO - 1;
  else if (tid == TX + 1) lx = RB_XO + txe;
  const int gx = x0 - RB_XO + lx;  // unwrapped column: its parity is the colour's
  const int gxw = wrapi(gx, nx);
  T* const* dst = dir ? G.e : G.r;
  const int nsteps = (y1 - y0) / 2 + 1;
  auto slot = [&](int row) { return ((row - y0 + 2) % MR) * RS; };
  auto red_row = [&](int ya) { return ((gx + ya + 1) & 1) == 0 ? ya + 1 : ya + 2; };
  auto black_row = [&](int ya) { return ((gx + ya) & 1) ? ya : ya + 1; };
  auto update = [&](int row, const MarchPt<T, KIND>& pt) {
    const MarchAcc<T, KIND, SW> acc{buf, pt};
    Nb n;
    n.c = slot(row) + lx;
    n.m[0] = n.c - 1;
    n.p[0] = n.c + 1;
    n.m[1] = slot(row - 1) + lx;
    n.p[1] = slot(row + 1) + lx;
    n.m[2] = n.p[2] = n.c;
    smooth_point_a<T, KIND, 2>(acc, P, K, n, 0);
  };

  // rows y0 - 2 .. y0 + 3 (steps 0 and 1)
  for (int k = 0; k < 3; ++k) march_issue2<T, KIND, TX>(G, buf, x0, y0 - 2 + 2 * k, 2 * k, dir);
  cp_async_commit();
  MarchPt<T, KIND> pr, pb, nr, nbk;
  if (lx >= 0) march_load_pt<T, KIND>(G, wrapi(red_row(y0 - 2), ny) * nx + gxw, pr);
  cp_async_wait_all();
  __syncthreads();
#pragma unroll 1
  for (int s = 0; s < nsteps; ++s) {
    const int ya = y0 - 2 + 2 * s;
    if (lx >= 0) update(red_row(ya), pr);
    cp_async_wait_all();
    __syncthreads();
    if (s + 2 < nsteps) march_issue2<T, KIND, TX>(G, buf, x0, ya + 6, 2 * s + 6, dir);  // rows of step s + 2
    cp_async_commit();
    const int rb = black_row(ya);
    const bool do_black = interior && rb >= y0 && rb < y1;
    // next step's point values
    if (lx >= 0 && s + 1 < nsteps) march_load_pt<T, KIND>(G, wrapi(red_row(ya + 2), ny) * nx + gxw, nr);
    const int rbn = black_row(ya + 2);
    if (interior && s + 1 < nsteps && rbn >= y0 && rbn < y1) march_load_pt<T, KIND>(G, rbn * nx + gxw, nbk);
    if (do_black) update(rb, pb);
    if (interior) {
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const int row = ya + k;
        if (row >= y0 && row < y1) {
          const int si = slot(row) + lx;
#pragma unroll
          for (int q = 0; q < NU; ++q) dst[q][row * nx + gxw] = buf[si + q * SW];
        }
      }
    }
    pr = nr;
    pb = nbk;
  }
}

template <typename T, int KIND, int TX>
__global__ void __launch_bounds__(march_threads(TX), march_minb<T>(TX)) k_smooth_march(Lvl<T> G, Phys<T> P, int nstrips, int ly,
                                                                    int dir) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int strip = blockIdx.x % nstrips, seg = blockIdx.x / nstrips;
  const int y0 = seg * ly;
  march_sweep<T, KIND, TX>(G, P, reinterpret_cast<T*>(smraw), strip * TX, y0, min(y0 + ly, G.g.ny), dir);
}

// --------------------------------------------------------------------------
// 2-D fused red-black sweep, two sweeps per pass (row-marching form)
// --------------------------------------------------------------------------
// The marching form above with a second sweep following the first, four
// rows behind it, in the same pass.  Step s (ya = y0 - 4 + 2 s):
//   phase 1: red of sweep 1 on rows ya + 1, ya + 2 (one point per column)
//            and red of sweep 2 on rows ya - 3, ya - 2;
//   phase 2: black of sweep 1 on rows ya, ya + 1 and black of sweep 2 on
//            rows ya - 4, ya - 3, which are then final and written out.
// Sweep-2 red on row r reads sweep-1 values of rows r - 1 .. r + 1, all
// final after phase 2 of step s - 1; sweep-2 black reads sweep-2 red values
// of phase 1.  A point keeps one value in the ring (before the sweeps, after
// sweep 1, after sweep 2), and every read of an older value comes before the
// phase that overwrites it, so one barrier after each phase suffices.
//
// Because sweep 2 at the block's edge rows and columns needs sweep-1 values
// one point further out, the block computes sweep-1 red on rows y0 - 3 ..
// y1 + 2 and columns x0 - 3 .. x0 + TX + 2, sweep-1 black one row and column
// less, sweep-2 red one less again and sweep-2 black on its own points only
// (the lanes 0..5 of the extra warp take the six outer columns); the staged
// rows are y0 - 4 .. y1 + 3.  As in the one-sweep forms the correction is
// read from one buffer and written to the other, so the result is exactly two
// red-black sweeps.  The data are read once and written once for both sweeps.
constexpr int MR2 = 14;  // row slots: rows ya - 5 .. ya + 7 are live in step s (one slot spare)

template <typename T, int KIND, int TX>
__host__ __device__ constexpr size_t march2_smem_bytes() {
  return (size_t)MR2 * march_arrays<KIND>() * (TX + 2 * RB_XO) * sizeof(T);
}
template <typename T>
__host__ __device__ constexpr int march2_minb(int tx) { return (sizeof(T) == 4 && tx == 128) ? 4 : 1; }

template <typename T, int KIND, int TX>
__device__ __forceinline__ void march2_sweep(const Lvl<T>& G, const Phys<T>& P, T* buf, int x0, int y0, int y1,
                                             int dir) {
  static_assert(RB_XO >= 4, "the two-sweep pass stages four halo columns");
  constexpr int NU = Layout<KIND, 2>::NU;
  constexpr int NA = march_arrays<KIND>();
  constexpr int SW = TX + 2 * RB_XO;
  constexpr int RS = NA * SW;
  const int nx = G.g.nx, ny = G.g.ny;
  const int txe = min(TX, nx - x0);
  const PtK<T> K = make_ptk<T, 2>(P, G.h);
  // this thread's staged column and its distance from the block's columns
  // (0 inside; lanes 0..5 of the extra warp: x0 - 3 .. x0 - 1 at distance
  // 3, 2, 1 and x0 + txe .. x0 + txe + 2 at distance 1, 2, 3)
  const int tid = threadIdx.x;
  int lx = -1, dist = 4;
  if (tid < txe) {
    lx = RB_XO + tid;
    dist = 0;
  } else if (tid >= TX && tid < TX + 3) {
    lx = RB_XO - 3 + (tid - TX);
    dist = 3 - (tid - TX);
  } else if (tid >= TX + 3 && tid < TX + 6) {
    lx = RB_XO + txe + (tid - TX - 3);
    dist = 1 + (tid - TX - 3);
  }
  const int gx = x0 - RB_XO + lx;  // unwrapped column: its parity is the colour's
  const int gxw = wrapi(gx, nx);
  T* const* dst = dir ? G.e : G.r;
  const int ylo = y0 - 4;  // first staged row
  const int nsteps = (y1 - y0 + 7) / 2 + 1;
  auto slot = [&](int row) { return ((row - ylo) % MR2) * RS; };
  auto red_row = [&](int ya) { return ((gx + ya + 1) & 1) == 0 ? ya + 1 : ya + 2; };
  auto black_row = [&](int ya) { return ((gx + ya) & 1) ? ya : ya + 1; };
  // rows and columns each half-sweep covers
  auto red1 = [&](int row) { return dist <= 3 && row >= y0 - 3 && row <= y1 + 2; };
  auto black1 = [&](int row) { return dist <= 2 && row >= y0 - 2 && row <= y1 + 1; };
  auto red2 = [&](int row) { return dist <= 1 && row >= y0 - 1 && row <= y1; };
  auto black2 = [&](int row) { return dist == 0 && row >= y0 && row < y1; };
  auto update = [&](int row, const MarchPt<T, KIND>& pt) {
    const MarchAcc<T, KIND, SW> acc{buf, pt};
    Nb n;
    n.c = slot(row) + lx;
    n.m[0] = n.c - 1;
    n.p[0] = n.c + 1;
    n.m[1] = slot(row - 1) + lx;
    n.p[1] = slot(row + 1) + lx;
    n.m[2] = n.p[2] = n.c;
    smooth_point_a<T, KIND, 2>(acc, P, K, n, 0);
  };

  // rows y0 - 4 .. y0 + 1 (steps 0 and 1)
  for (int k = 0; k < 3; ++k) march_issue2<T, KIND, TX, MR2>(G, buf, x0, ylo + 2 * k, 2 * k, dir);
  cp_async_commit();
  // point values of the red and black point of this column in steps s, s - 1,
  // s - 2 (sweep 2 at step s updates the points sweep 1 updated at s - 2)
  MarchPt<T, KIND> r0{}, r1{}, r2{}, b0{}, b1{}, b2{}, rn{}, bn{};
  if (red1(red_row(ylo))) march_load_pt<T, KIND>(G, wrapi(red_row(ylo), ny) * nx + gxw, r0);
  if (black1(black_row(ylo))) march_load_pt<T, KIND>(G, wrapi(black_row(ylo), ny) * nx + gxw, b0);
  cp_async_wait_all();
  __syncthreads();
#pragma unroll 1
  for (int s = 0; s < nsteps; ++s) {
    const int ya = ylo + 2 * s;
    const int rr = red_row(ya), br = black_row(ya);
    if (red1(rr)) update(rr, r0);
    if (red2(rr - 4)) update(rr - 4, r2);
    cp_async_wait_all();
    __syncthreads();
    if (ya + 6 <= y1 + 3) march_issue2<T, KIND, TX, MR2>(G, buf, x0, ya + 6, 2 * s + 6, dir);  // step s + 2
    cp_async_commit();
    if (s + 1 < nsteps) {
      const int rrn = red_row(ya + 2), brn = black_row(ya + 2);
      if (red1(rrn)) march_load_pt<T, KIND>(G, wrapi(rrn, ny) * nx + gxw, rn);
      if (black1(brn)) march_load_pt<T, KIND>(G, wrapi(brn, ny) * nx + gxw, bn);
    }
    if (black1(br)) update(br, b0);
    if (black2(br - 4)) update(br - 4, b2);
    if (dist == 0) {
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const int row = ya - 4 + k;
        if (row >= y0 && row < y1) {
          const int si = slot(row) + lx;
#pragma unroll
          for (int q = 0; q < NU; ++q) dst[q][row * nx + gxw] = buf[si + q * SW];
        }
      }
    }
    __syncthreads();
    r2 = r1;
    r1 = r0;
    r0 = rn;
    b2 = b1;
    b1 = b0;
    b0 = bn;
  }
}

template <typename T, int KIND, int TX>
__global__ void __launch_bounds__(march_threads(TX), march2_minb<T>(TX)) k_smooth_march2(Lvl<T> G, Phys<T> P,
                                                                     int nstrips, int ly, int dir) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int strip = blockIdx.x % nstrips, seg = blockIdx.x / nstrips;
  const int y0 = seg * ly;
  march2_sweep<T, KIND, TX>(G, P, reinterpret_cast<T*>(smraw), strip * TX, y0, min(y0 + ly, G.g.ny), dir);
}

// Variants of the 2-D fused sweep, chosen per level by the autotuner:
// 0..11 tile form (bits 0-1: PIPE, SF; v >> 2: tile 32x16, 64x8, 32x32),
// 12..17 marching form (strip width 64 or 128; rows per block 16, 32, 64),
// 18..23 the two-sweep marching form with the same strips and rows, 24..26
// the two-sweep tile form (tiles 32x16, 64x8, 32x32; f and omega from global
// memory, one tile per block), 27..29 tiles staged by tensor copies (27: as
// 24, 28: as 0, 29: as 26; single-instance solver only -- the batch runs
// them as their cp.async twins), 30..33 the tile form on small tiles for the
// coarse levels (30: 16 x 16 one sweep, 31: 16 x 16 two sweeps, 32: 16 x 8
// one sweep, 33: 16 x 8 two sweeps; single-instance solver only, the batch
// runs them as 0 and 24), 34 all sweeps of a smoothing step in one
// cooperative launch with grid barriers between the colour passes
// (fm_coop.cuh; single-instance solver only, the batch runs it as 24), 35
// the two-sweep tile form on 32 x 14 tiles (single-instance solver only, the
// batch runs it as 24).
constexpr int RB_NVAR = FM_SWEEP_VARIANTS;
constexpr int RB_TMA0 = 27;  // first variant staged by tensor copies
constexpr int RB_SMALL0 = 30;  // first small-tile variant
constexpr int RB_COOP = 34;  // a level's sweeps in one cooperative launch (in place; single-instance solver)
constexpr int RB_T14 = 35;   // two-sweep tiles of 32 x 14 (single-instance solver)
constexpr int TUNE_REPS = 10;  // timed launches per variant and level in the autotuners
constexpr int RB_NTILE = 12;
constexpr int RB_NMARCH = 6;
constexpr int RB_TWO = RB_NTILE + RB_NMARCH;  // first two-sweep variant
constexpr int RB_TWO_TILE = RB_TWO + RB_NMARCH;  // first two-sweep tile variant
__host__ __device__ constexpr int march_tx(int v) { return (v - RB_NTILE) % RB_NMARCH < 3 ? 64 : 128; }
__host__ __device__ constexpr int march_ly(int v) { return 16 << ((v - RB_NTILE) % 3); }
// (variant 34 runs all the sweeps of a smoothing step in one launch; it is
// timed and reported with two, the pre- and post-smoothing count.)
__host__ __device__ constexpr int sweeps_per_launch(int v) {
  return (v == RB_COOP || v == RB_T14) ? 2
         : v >= RB_SMALL0              ? 1 + ((v - RB_SMALL0) & 1)
                                       : ((v >= RB_TWO && v != RB_TMA0 + 1) ? 2 : 1);
}
// The one-sweep variant with the same blocks as two-sweep variant v.
__host__ __device__ constexpr int one_sweep_twin(int v) {
  return (v == RB_COOP || v == RB_T14) ? 0
         : v >= RB_SMALL0 ? RB_SMALL0 + ((v - RB_SMALL0) & ~1)
         : v >= RB_TMA0 ? (v == RB_TMA0 ? RB_TMA0 + 1 : (v == RB_TMA0 + 2 ? 8 : v))
                        : (v >= RB_TWO_TILE ? (v - RB_TWO_TILE) * 4 : (v >= RB_TWO ? v - RB_NMARCH : v));
}

// The whole V-cycle of the small levels (each at most SMALL_N points) in one
// thread block: phases separated by __syncthreads, data in L1/L2.
constexpr int SMALL_N = 1024;           // levels of at most this many points run in one block
constexpr int SMALL_SMEM_N = 1024;      // larger coarse levels: the global-memory kernel (measured faster)
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
  const PtK<T> K = make_ptk<T, DIM>(P, L.h);
  for (int it = 0; it < iters; ++it)
    for (int color = 0; color < 2; ++color) {
      for (int t = threadIdx.x; t < half; t += blockDim.x) {
        int i, j, k;
        colour_point(t, color, L.g, i, j, k);
        const Nb n = neighbours(i, j, k, L.g);
        smooth_point<T, KIND, DIM>(L, P, K, n);
      }
      __syncthreads();
    }
}

template <typename T, int KIND, int DIM>
__device__ __forceinline__ void vcycle_small_body(const SmallLv<T>& S, const Phys<T>& P, int nu1, int nu2,
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
    for (int idx = threadIdx.x; idx < F.g.N; idx += blockDim.x) prolong_point<T, LY::NU, DIM>(F, C, P, idx);
    __syncthreads();
    block_smooth<T, KIND, DIM>(F, P, nu2);
  }
}

template <typename T, int KIND, int DIM>
__global__ void __launch_bounds__(SMALL_TPB) k_vcycle_small(SmallLv<T> S, Phys<T> P, int nu1, int nu2,
                                                            int ncoarse) {
  vcycle_small_body<T, KIND, DIM>(S, P, nu1, nu2, ncoarse);
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
  int off_rk[MAXSMALL];
  int off_cr[MAXSMALL];
  int off_om[MAXSMALL][3];
  int off_cv[MAXSMALL][3];
  int stage_coef;  // coefficients also in shared memory
};

// Levels of at most SMALL_WARP_N points are processed by warp 0 alone
// (phases separated by __syncwarp instead of __syncthreads).
constexpr int SMALL_WARP_N = 64;

// One smoothing iteration set of level L by a group of threads: the whole
// block (WARP = false) or warp 0 (WARP = true).
template <typename T, int KIND, int DIM, bool WARP>
__device__ __forceinline__ void group_sync() {
  if constexpr (WARP) __syncwarp();
  else __syncthreads();
}

template <typename T, int KIND, int DIM, bool WARP>
__device__ __forceinline__ void group_smooth(const Lvl<T>& L, const Phys<T>& P, int iters) {
  const int tid = WARP ? (threadIdx.x & 31) : threadIdx.x;
  const int nth = WARP ? 32 : blockDim.x;
  const int half = L.g.N / 2;
  const PtK<T> K = make_ptk<T, DIM>(P, L.h);
  for (int it = 0; it < iters; ++it)
    for (int color = 0; color < 2; ++color) {
      for (int t = tid; t < half; t += nth) {
        int i, j, k;
        colour_point(t, color, L.g, i, j, k);
        const Nb n = neighbours(i, j, k, L.g);
        smooth_point<T, KIND, DIM>(L, P, K, n);
      }
      group_sync<T, KIND, DIM, WARP>();
    }
}

// Down sweep of level l (smooth, residual, restriction, coarse right-hand side).
template <typename T, int KIND, int DIM, bool WARP>
__device__ __forceinline__ void group_down(const Lvl<T>& F, const Lvl<T>& C, const Phys<T>& P, int nu1) {
  using LY = Layout<KIND, DIM>;
  const int tid = WARP ? (threadIdx.x & 31) : threadIdx.x;
  const int nth = WARP ? 32 : blockDim.x;
  group_smooth<T, KIND, DIM, WARP>(F, P, nu1);
  for (int idx = tid; idx < F.g.N; idx += nth) resid_point<T, KIND, DIM>(F, P, idx);
  group_sync<T, KIND, DIM, WARP>();
  for (int idx = tid; idx < C.g.N; idx += nth) restrict_point<T, LY::NU, DIM>(F, C, idx);
  group_sync<T, KIND, DIM, WARP>();
  for (int idx = tid; idx < C.g.N; idx += nth) coarse_rhs_point<T, KIND, DIM>(C, P, idx);
  group_sync<T, KIND, DIM, WARP>();
}

template <typename T, int KIND, int DIM, bool WARP>
__device__ __forceinline__ void group_up(const Lvl<T>& F, const Lvl<T>& C, const Phys<T>& P, int nu2) {
  using LY = Layout<KIND, DIM>;
  const int tid = WARP ? (threadIdx.x & 31) : threadIdx.x;
  const int nth = WARP ? 32 : blockDim.x;
  for (int idx = tid; idx < F.g.N; idx += nth) prolong_point<T, LY::NU, DIM>(F, C, P, idx);
  group_sync<T, KIND, DIM, WARP>();
  group_smooth<T, KIND, DIM, WARP>(F, P, nu2);
}

template <typename T, int KIND, int DIM>
__device__ __forceinline__ void vcycle_small_smem_body(const SmallLv<T>& S, const SmallSmem<T>& M,
                                                       const Phys<T>& P, int nu1, int nu2, int ncoarse) {
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
      if (M.stage_coef) {
        SL[l].rk = sm + M.off_rk[l];
        SL[l].cr = sm + M.off_cr[l];
        for (int d = 0; d < 3; ++d) {
          SL[l].om[d] = d < LY::NOM ? sm + M.off_om[l][d] : nullptr;
          SL[l].cv[d] = d < DIM ? sm + M.off_cv[l][d] : nullptr;
        }
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
    if (M.stage_coef)
      for (int l = 0; l < nl; ++l) {
        const Lvl<T>& H = S.lv[l];
        for (int idx = threadIdx.x; idx < H.g.N; idx += blockDim.x) {
          sm[M.off_rk[l] + idx] = H.rk[idx];
          sm[M.off_cr[l] + idx] = H.cr[idx];
#pragma unroll
          for (int d = 0; d < LY::NOM; ++d) sm[M.off_om[l][d] + idx] = H.om[d][idx];
#pragma unroll
          for (int d = 0; d < DIM; ++d) sm[M.off_cv[l][d] + idx] = H.cv[d][idx];
        }
      }
  }
  __syncthreads();
  // first level handled by warp 0 alone
  int lw = nl;
  for (int l = 0; l < nl; ++l)
    if (SL[l].g.N <= SMALL_WARP_N) {
      lw = l;
      break;
    }
  if (lw == 0) lw = 1;  // the entry level is always block-wide
  const int nb = lw < nl - 1 ? lw : nl - 1;  // levels 0..nb-1 go down block-wide
  for (int l = 0; l < nb; ++l) group_down<T, KIND, DIM, false>(SL[l], SL[l + 1], P, nu1);
  if (lw >= nl) {
    group_smooth<T, KIND, DIM, false>(SL[nl - 1], P, ncoarse);
  } else {
    if ((threadIdx.x >> 5) == 0) {
      for (int l = lw; l + 1 < nl; ++l) group_down<T, KIND, DIM, true>(SL[l], SL[l + 1], P, nu1);
      group_smooth<T, KIND, DIM, true>(SL[nl - 1], P, ncoarse);
      for (int l = nl - 2; l >= lw; --l) group_up<T, KIND, DIM, true>(SL[l], SL[l + 1], P, nu2);
    }
    __syncthreads();
  }
  for (int l = nb - 1; l >= 0; --l) group_up<T, KIND, DIM, false>(SL[l], SL[l + 1], P, nu2);
  {
    const Lvl<T>& G = S.lv[0];
    for (int idx = threadIdx.x; idx < G.g.N; idx += blockDim.x)
#pragma unroll
      for (int q = 0; q < LY::NU; ++q) G.e[q][idx] = SL[0].e[q][idx];
  }
}

template <typename T, int KIND, int DIM>
__global__ void __launch_bounds__(SMALL_TPB) k_vcycle_small_smem(SmallLv<T> S, SmallSmem<T> M, Phys<T> P,
                                                                 int nu1, int nu2, int ncoarse) {
  vcycle_small_smem_body<T, KIND, DIM>(S, M, P, nu1, nu2, ncoarse);
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
__device__ __forceinline__ void inject_all_point(const InjAll<T>& A, int t) {
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

template <typename T>
__global__ void __launch_bounds__(TPB) k_inject_all(InjAll<T> A) {
  inject_all_point<T>(A, blockIdx.x * blockDim.x + threadIdx.x);
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

// float64 -> float32 rounded to nearest, ties to even, with integer
// instructions only (IEEE 754 binary64 -> binary32 narrowing written from the
// two formats' definitions).  The hardware conversion runs on the float64
// pipe, which bounds the residual kernels that write the float32 right-hand
// side; this one runs on the integer pipes.  Exact for every input: normal
// and subnormal results, overflow to infinity, signed zeros; NaN stays NaN.
__host__ __device__ inline float narrow_rn(double x) {
  unsigned long long b;
  memcpy(&b, &x, sizeof(b));
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const int ex = (int)((b >> 52) & 0x7FF);
  const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  unsigned r;
  if (ex == 0x7FF) {
    r = 0x7F800000u | (m ? (0x400000u | (unsigned)(m >> 29)) : 0u);  // infinity, or a quiet NaN
  } else {
    const int E = ex - 1023 + 127;  // biased binary32 exponent of a normal result
    unsigned long long mant;
    int sh;
    if (E > 0) {  // normal range: keep 23 of the 52 fraction bits
      mant = ((unsigned long long)E << 52 | m) >> 0;  // exponent travels with the fraction
      sh = 29;
    } else {      // subnormal result (or zero): the implicit bit becomes explicit
      mant = ex ? (m | (1ull << 52)) : m;
      sh = 30 - E;
    }
    if (sh >= 64) {
      r = 0u;  // below half the smallest subnormal
    } else {
      const unsigned long long keep = mant >> sh;
      const unsigned long long rem = mant & ((1ull << sh) - 1ull);
      const unsigned long long half = 1ull << (sh - 1);
      unsigned long long q = keep + ((rem > half || (rem == half && (keep & 1ull))) ? 1ull : 0ull);
      if (E > 0 && q >= (255ull << 23)) q = 255ull << 23;  // overflow: infinity
      r = (unsigned)q;
    }
  }
  r |= sign;
  float f;
  memcpy(&f, &r, sizeof(f));
  return f;
}

// float32 -> float64 (exact) with integer instructions only, for the same
// reason: every binary32 value is a binary64 value; subnormal inputs are
// normalised with a leading-zero count.
__device__ __forceinline__ double widen(float x) {
  const unsigned b = __float_as_uint(x);
  const unsigned long long sign = (unsigned long long)(b & 0x80000000u) << 32;
  const unsigned ex = (b >> 23) & 0xFFu;
  const unsigned m = b & 0x7FFFFFu;
  unsigned long long r;
  if (ex == 0xFFu) {
    r = 0x7FF0000000000000ull | ((unsigned long long)m << 29);  // infinity or NaN (payload kept)
  } else if (ex != 0u) {
    r = ((unsigned long long)(ex + 896u) << 52) | ((unsigned long long)m << 29);
  } else if (m == 0u) {
    r = 0ull;
  } else {  // subnormal: m * 2^-149 = 1.f * 2^(p - 149), p the position of m's leading one
    const int lz = __clz(m) - 8;  // 23 - p
    const unsigned mn = (m << lz) & 0x7FFFFFu;
    r = ((unsigned long long)(897 - lz) << 52) | ((unsigned long long)mn << 29);
  }
  return __longlong_as_double((long long)(sign | r));
}

template <typename T>
__device__ __forceinline__ double from_t(T x) {
  if constexpr (sizeof(T) == 4) return widen(x);
  else return (double)x;
}

template <typename T>
__device__ __forceinline__ T to_t(double x) {
  if constexpr (sizeof(T) == 4) return narrow_rn(x);
  else return (T)x;
}

// Step constants of the float64 kernels (grid spacing h, step s), formed once
// per step on the host (per instance for a batch) instead of per thread.
struct Step64 {
  double ih;     // 1/h
  double ih2;    // 1/h^2
  double hih;    // 1/(2h): centred differences of the vorticity
  double c_div;  // s/(4h): continuity flux difference, kinetic-energy gradient
  double c_w;    // sigma s/2: vorticity term
  double c_m;    // s/(2h): chemical-potential gradient (non-local source term)
  double c_v;    // s gamma/(2h^2): viscous Laplacian
};

__host__ __device__ inline Step64 make_step64(const Phys<double>& P, double ih) {
  Step64 K;
  K.ih = ih;
  K.ih2 = ih * ih;
  K.hih = 0.5 * ih;
  K.c_div = P.s * 0.25 * ih;
  K.c_w = 0.5 * P.sigma * P.s;
  K.c_m = 0.5 * P.s * ih;
  K.c_v = 0.5 * P.s * P.gamma * K.ih2;
  return K;
}

struct Fields64 {
  const double* rho;          // rho^k
  const double* vel[3];       // u^k
  const double* conv;         // J * rho^k (CDFT)
  double* om[3];              // omega^k (out)
  double* S[MAXU];            // source (out)
  double* g[MAXU];            // iterate
  float* rk32;                // float copies for the mixed path (or null)
  float* om32[3];
  int* nonpos;                // CDFT: set to 1 where a density <= 0 would reach ln (or null)
  const int* hist;            // extrapolated initial iterate: g already holds g^0 when *hist > 0 (or null)
};

// omega^k, S and the initial iterate g^0 (kappa^0 = Lap_h rho^k for PFC).
template <int KIND, int DIM>
__device__ __forceinline__ void prepare_point(const Fields64& F, const Geo& G, const Step64& K,
                                              const Phys<double>& P, int idx) {
  using LY = Layout<KIND, DIM>;
  if (idx >= G.N) return;
  int i, j, k;
  coords(idx, G, i, j, k);
  const Nb n = neighbours(i, j, k, G);
  const double ih2 = K.ih2;
  const double* u = F.vel[0];
  const double* v = F.vel[1];
  double w[3];
  if constexpr (DIM == 2) {
    w[0] = K.hih * ((v[n.p[0]] - v[n.m[0]]) - (u[n.p[1]] - u[n.m[1]]));
  } else {
    const double* ww = F.vel[2];
    w[0] = K.hih * ((ww[n.p[1]] - ww[n.m[1]]) - (v[n.p[2]] - v[n.m[2]]));
    w[1] = K.hih * ((u[n.p[2]] - u[n.m[2]]) - (ww[n.p[0]] - ww[n.m[0]]));
    w[2] = K.hih * ((v[n.p[0]] - v[n.m[0]]) - (u[n.p[1]] - u[n.m[1]]));
  }
  const double rkc = F.rho[n.c];
  if constexpr (KIND == KCDFT) {
    if (F.nonpos && rkc <= 0.0) atomicOr(F.nonpos, 1);  // ln rho^k undefined: FM_ENONPOS
  }
  double div = 0;
#pragma unroll
  for (int d = 0; d < DIM; ++d)
    div += F.rho[n.p[d]] * F.vel[d][n.p[d]] - F.rho[n.m[d]] * F.vel[d][n.m[d]];
  const double c_w = K.c_w, c_v = K.c_v, c_e = K.c_m;
  const double s0 = rkc - K.c_div * div;
  double uc[3], wx[3], sv[3];  // all loads before the first store
#pragma unroll
  for (int d = 0; d < DIM; ++d) uc[d] = F.vel[d][n.c];
  cross<double, DIM>(w, uc, wx);
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    double sa = rkc * (uc[a] - c_w * wx[a]) + c_v * (nbsum<double, DIM>(F.vel[a], n) - 2.0 * DIM * uc[a]);
    if constexpr (KIND == KCDFT) {
      const double Ep = 2.0 * P.ce * F.rho[n.p[a]] + F.conv[n.p[a]];
      const double Em = 2.0 * P.ce * F.rho[n.m[a]] + F.conv[n.m[a]];
      sa += c_e * rkc * (Ep - Em);
    }
    sv[a] = sa;
  }
  const double lapr = (KIND == KPFC) ? (nbsum<double, DIM>(F.rho, n) - 2.0 * DIM * rkc) * ih2 : 0.0;
  const bool keep = F.hist && *F.hist > 0;  // g^0 extrapolated in time already (k_extrapolate)
  F.S[0][idx] = s0;
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    F.S[1 + a][idx] = sv[a];
    if (!keep) F.g[1 + a][idx] = uc[a];
  }
  if (!keep) F.g[0][idx] = rkc;
  if constexpr (KIND == KPFC) {
    F.S[LY::IMU][idx] = 2.0 * lapr;
    F.S[LY::IKA][idx] = 0.0;
    if (!keep) F.g[LY::IKA][idx] = lapr;
  }
#pragma unroll
  for (int d = 0; d < LY::NOM; ++d) F.om[d][idx] = w[d];
  if (F.rk32) {
    F.rk32[idx] = narrow_rn(rkc);
#pragma unroll
    for (int d = 0; d < LY::NOM; ++d) F.om32[d][idx] = narrow_rn(w[d]);
  }
}

template <int KIND, int DIM>
__global__ void __launch_bounds__(TPB) k_prepare(Fields64 F, Geo G, Step64 K, Phys<double> P) {
  prepare_point<KIND, DIM>(F, G, K, P, blockIdx.x * blockDim.x + threadIdx.x);
}

// PFC: mu^0 = psi^3/3 + alpha psi + Lap_h kappa^0 + S_mu (value of the mu row at rho^k).
template <int DIM>
__device__ __forceinline__ void prepare_mu_point(const Fields64& F, const Geo& G, const Step64& K,
                                                 const Phys<double>& P, int idx) {
  using LY = Layout<KPFC, DIM>;
  if (idx >= G.N) return;
  if (F.hist && *F.hist > 0) return;  // mu^0 extrapolated with the rest of g^0
  int i, j, k;
  coords(idx, G, i, j, k);
  const Nb n = neighbours(i, j, k, G);
  const double psi = F.rho[idx] - 1.5;
  const double* ka = F.g[LY::IKA];
  const double lapk = (nbsum<double, DIM>(ka, n) - 2.0 * DIM * ka[idx]) * K.ih2;
  F.g[LY::IMU][idx] = psi * psi * psi * (1.0 / 3.0) + P.alpha * psi + lapk + F.S[LY::IMU][idx];
}

template <int DIM>
__global__ void __launch_bounds__(TPB) k_prepare_mu(Fields64 F, Geo G, Step64 K, Phys<double> P) {
  prepare_mu_point<DIM>(F, G, K, P, blockIdx.x * blockDim.x + threadIdx.x);
}

// Fixed-order block sum of NQ per-thread values into partials[blk][q]: a
// tree in shared memory down to one warp, then shuffles.  Few float64 warp
// instructions (the float64 pipe is the bound of the residual kernels), and
// the same order on every run.
template <int NQ>
__device__ __forceinline__ void block_partials(double (&v)[NQ], double* partials, int blk) {
  __shared__ double sm[NQ][TPB];
  const int tid = threadIdx.x, lane = tid & 31;
#pragma unroll
  for (int q = 0; q < NQ; ++q) sm[q][tid] = v[q];
  __syncthreads();
#pragma unroll
  for (int s = TPB / 2; s >= 32; s >>= 1) {
    if (tid < s)
#pragma unroll
      for (int q = 0; q < NQ; ++q) sm[q][tid] += sm[q][tid + s];
    __syncthreads();
  }
  if (tid < 32) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      double x = sm[q][lane];
      for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
      if (lane == 0) partials[blk * NQ + q] = x;
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


// Residual value r at point idx: store it in precision T for the cycle (f0,
// when given) and add r^2 to the sum of squares of the stopping test.  In the
// cycle of the mixed path the square is taken of the float32-rounded residual
// the cycle receives and summed in float32 (fa), off the float64 pipe: the
// sum only decides when to stop, and float32 carries it to ~1e-7 relative.
// Otherwise it is summed in float64 (acc).
template <typename T>
__device__ __forceinline__ void norm_add(void* f0, double r, double& acc, float& fa, int idx) {
  if (f0) {
    const T rt = to_t<T>(r);
    static_cast<T*>(f0)[idx] = rt;
    if constexpr (sizeof(T) == 4) {
      fa = fmaf(rt, rt, fa);
      return;
    }
  }
  acc += r * r;
}
// Block partial sums of the stopping test: from the float32 sums (fa) when
// the float32-rounded residual was summed (mixed cycle: f0 given, T float;
// the tree stays in float32 and each block's result is widened once),
// otherwise from the float64 sums (acc).  `f0` is the same for the whole
// launch, so the branch is uniform.
template <int NQ>
__device__ __forceinline__ void block_partials_f(float (&v)[NQ], double* partials, int blk) {
  __shared__ float sm[NQ][TPB];
  const int tid = threadIdx.x, lane = tid & 31;
#pragma unroll
  for (int q = 0; q < NQ; ++q) sm[q][tid] = v[q];
  __syncthreads();
#pragma unroll
  for (int s = TPB / 2; s >= 32; s >>= 1) {
    if (tid < s)
#pragma unroll
      for (int q = 0; q < NQ; ++q) sm[q][tid] += sm[q][tid + s];
    __syncthreads();
  }
  if (tid < 32) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      float x = sm[q][lane];
      for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
      if (lane == 0) partials[blk * NQ + q] = widen(x);
    }
  }
}
template <typename T, int NQ>
__device__ __forceinline__ void norm_partials(const void* f0, double (&acc)[NQ], float (&fa)[NQ], double* partials,
                                              int blk) {
  if constexpr (sizeof(T) == 4) {
    if (f0) {
      block_partials_f<NQ>(fa, partials, blk);
      return;
    }
  }
  block_partials<NQ>(acc, partials, blk);
}

struct Resid64Out {
  void* f0[MAXU];   // precision-T rhs of level 0 (or null)
  void* e0[MAXU];   // precision-T correction of level 0, zeroed (or null)
  float* cr32;      // float coefficient copies (mixed path) or null
  float* cv32[3];
  double* r64[MAXU];  // optional float64 residual output
};

// r = S - N(g) in float64 (App. G operator N, full form), block partials of r^2.
// Block `lb` of `nb` blocks: strided loop over the points, partial sums of
// r^2 into partials[lb][q].
template <int KIND, int DIM, typename T>
__device__ __forceinline__ void resid64_body(const Fields64& F, const Resid64Out& O, const Geo& G, const Step64& K,
                                             const Phys<double>& P, double* partials, int lb, int nb) {
  using LY = Layout<KIND, DIM>;
  double acc[LY::NU];
#pragma unroll
  for (int q = 0; q < LY::NU; ++q) acc[q] = 0.0;
  float fa[LY::NU];
#pragma unroll
  for (int q = 0; q < LY::NU; ++q) fa[q] = 0.0f;
  const double ih2 = K.ih2, c_div = K.c_div, c_w = K.c_w, c_q = K.c_div, c_m = K.c_m, c_v = K.c_v;
  const double third = 1.0 / 3.0;
  for (int idx = lb * blockDim.x + threadIdx.x; idx < G.N; idx += nb * blockDim.x) {
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
    N[0] = g[0][n.c] + c_div * div;
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
      N[1 + a] = rkc * (uc[a] + c_w * wx[a] + c_q * (qp - qm) + c_m * (mp - mm))
               - c_v * (nbsum<double, DIM>(g[1 + a], n) - 2.0 * DIM * uc[a]);
    }
    if constexpr (KIND == KPFC) {
      const double rc = g[0][n.c];
      const double psi = rc - 1.5;
      const double kc = g[LY::IKA][n.c];
      // h^2 Lap_h kappa and h^2 Lap_h rho; the 1/h^2 scale and the cubic (Horner form)
      // go into fused multiply-adds (fewer float64 instructions, the same rows)
      const double dk = nbsum<double, DIM>(g[LY::IKA], n) - 2.0 * DIM * kc;
      const double dr = nbsum<double, DIM>(g[0], n) - 2.0 * DIM * rc;
      N[LY::IMU] = fma(-ih2, dk, g[LY::IMU][n.c] - psi * fma(psi * psi, third, P.alpha));
      N[LY::IKA] = fma(-ih2, dr, kc);
    }
    double rv[LY::NU];  // all loads (S, rho) before the first store
#pragma unroll
    for (int q = 0; q < LY::NU; ++q) rv[q] = F.S[q][idx] - N[q];
    const double g0c = g[0][idx];
#pragma unroll
    for (int q = 0; q < LY::NU; ++q) {
      const double r = rv[q];
      norm_add<T>(O.f0[q], r, acc[q], fa[q], idx);
      if (O.e0[q]) static_cast<T*>(O.e0[q])[idx] = T(0);
      if (O.r64[q]) O.r64[q][idx] = r;
    }
    if (O.cr32) {
      O.cr32[idx] = narrow_rn(g0c);
#pragma unroll
      for (int d = 0; d < DIM; ++d) O.cv32[d][idx] = narrow_rn(uc[d]);
    }
  }
  norm_partials<T, LY::NU>(O.f0[0], acc, fa, partials, lb);
}

// 2-D float64 residual in 32 x 8 tiles: the quantities every point shares
// with its neighbours -- |u|^2, rho^k u, rho^k v and the implicit chemical
// potential (mu, or ln rho + 2 c_e rho) -- are computed once per point of the
// tile and its one-point halo in shared memory, then N is evaluated on the
// tile.  Block lb of nb walks tiles lb, lb + nb, ...; partial sums of r^2 as
// in resid64_body (same per-block accumulation order on every run).
constexpr int R64_TX = 32, R64_TY = 8;
constexpr int R64_SW = R64_TX + 2, R64_SN = R64_SW * (R64_TY + 2);

template <int KIND, typename T>
__device__ __forceinline__ void resid64_tile_body(const Fields64& F, const Resid64Out& O, const Geo& G,
                                                  const Step64& K,
                                                  const Phys<double>& P, double* partials, int lb, int nb) {
  using LY = Layout<KIND, 2>;
  __shared__ double sQ[R64_SN], sM[R64_SN], sRU[R64_SN], sRV[R64_SN];
  double acc[LY::NU];
#pragma unroll
  for (int q = 0; q < LY::NU; ++q) acc[q] = 0.0;
  float fa[LY::NU];
#pragma unroll
  for (int q = 0; q < LY::NU; ++q) fa[q] = 0.0f;
  const double ih2 = K.ih2, c_div = K.c_div, c_w = K.c_w, c_q = K.c_div, c_m = K.c_m, c_v = K.c_v;
  const double third = 1.0 / 3.0;
  const int nx = G.nx, ny = G.ny;
  const int ntx = (nx + R64_TX - 1) / R64_TX;
  const int ntiles = ntx * ((ny + R64_TY - 1) / R64_TY);
  const double* const* g = F.g;
  for (int tile = lb; tile < ntiles; tile += nb) {
    const int x0 = (tile % ntx) * R64_TX, y0 = (tile / ntx) * R64_TY;
    for (int t = threadIdx.x; t < R64_SN; t += blockDim.x) {
      const int ly = t / R64_SW, lx = t - ly * R64_SW;
      int gx = x0 + lx - 1, gy = y0 + ly - 1;
      gx = gx < 0 ? gx + nx : (gx >= nx ? gx - nx : gx);
      gy = gy < 0 ? gy + ny : (gy >= ny ? gy - ny : gy);
      gx = gx >= nx ? gx % nx : gx;
      gy = gy >= ny ? gy % ny : gy;
      const int gi = gy * nx + gx;
      const double u = g[1][gi], v = g[2][gi], rk = F.rho[gi];
      sQ[t] = u * u + v * v;
      sRU[t] = rk * u;
      sRV[t] = rk * v;
      if constexpr (KIND == KPFC) {
        sM[t] = g[LY::IMU][gi];
      } else {
        const double r = g[0][gi];
        sM[t] = log(r) + 2.0 * P.ce * r;
      }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < R64_TX * R64_TY; t += blockDim.x) {
      const int ty = t / R64_TX, tx = t - ty * R64_TX;
      const int i = x0 + tx, j = y0 + ty;
      if (i < nx && j < ny) {
        const int idx = j * nx + i;
        const Nb n = neighbours(i, j, 0, G);
        const int c = (ty + 1) * R64_SW + tx + 1;
        const int xm = c - 1, xp = c + 1, ym = c - R64_SW, yp = c + R64_SW;
        const double rkc = F.rho[idx];
        double N[LY::NU];
        N[0] = g[0][idx] + c_div * ((sRU[xp] - sRU[xm]) + (sRV[yp] - sRV[ym]));
        const double uc = g[1][idx], vc = g[2][idx];
        const double w = F.om[0][idx];
        N[1] = rkc * (uc - c_w * w * vc + c_q * (sQ[xp] - sQ[xm]) + c_m * (sM[xp] - sM[xm]))
             - c_v * (nbsum<double, 2>(g[1], n) - 4.0 * uc);
        N[2] = rkc * (vc + c_w * w * uc + c_q * (sQ[yp] - sQ[ym]) + c_m * (sM[yp] - sM[ym]))
             - c_v * (nbsum<double, 2>(g[2], n) - 4.0 * vc);
        if constexpr (KIND == KPFC) {
          const double rc = g[0][idx];
          const double psi = rc - 1.5;
          const double kc = g[LY::IKA][idx];
          // h^2 Lap_h kappa and h^2 Lap_h rho; the 1/h^2 scale and the cubic (Horner form)
          // go into fused multiply-adds (fewer float64 instructions, the same rows)
          const double dk = nbsum<double, 2>(g[LY::IKA], n) - 4.0 * kc;
          const double dr = nbsum<double, 2>(g[0], n) - 4.0 * rc;
          N[LY::IMU] = fma(-ih2, dk, g[LY::IMU][idx] - psi * fma(psi * psi, third, P.alpha));
          N[LY::IKA] = fma(-ih2, dr, kc);
        }
        double rv[LY::NU];  // all loads (S, rho) before the first store
#pragma unroll
        for (int q = 0; q < LY::NU; ++q) rv[q] = F.S[q][idx] - N[q];
        const double g0c = g[0][idx];
#pragma unroll
        for (int q = 0; q < LY::NU; ++q) {
          const double r = rv[q];
          norm_add<T>(O.f0[q], r, acc[q], fa[q], idx);
          if (O.e0[q]) static_cast<T*>(O.e0[q])[idx] = T(0);
          if (O.r64[q]) O.r64[q][idx] = r;
        }
        if (O.cr32) {
          O.cr32[idx] = narrow_rn(g0c);
          O.cv32[0][idx] = narrow_rn(uc);
          O.cv32[1][idx] = narrow_rn(vc);
        }
      }
    }
    __syncthreads();
  }
  norm_partials<T, LY::NU>(O.f0[0], acc, fa, partials, lb);
}

template <int KIND, typename T>
__global__ void __launch_bounds__(TPB) k_resid64_tile(Fields64 F, Resid64Out O, Geo G, Step64 K,
                                                      Phys<double> P, double* partials) {
  resid64_tile_body<KIND, T>(F, O, G, K, P, partials, blockIdx.x, gridDim.x);
}

// Per-point quantities every point shares with its neighbours in the
// float64 residual (used in 3-D): X[0] = |u|^2, X[1 + d] = rho^k u_d, and for
// CDFT X[4] = ln rho + 2 c_e rho.
struct Shared64 {
  double* x[5];
};

template <int KIND, int DIM>
__global__ void __launch_bounds__(TPB) k_shared64(Fields64 F, Shared64 X, int N, double ce) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= N) return;
  const double rk = F.rho[idx];
  double u[DIM];
#pragma unroll
  for (int d = 0; d < DIM; ++d) u[d] = F.g[1 + d][idx];
  const double r = F.g[0][idx];
  double q = 0;
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    q += u[d] * u[d];
    X.x[1 + d][idx] = rk * u[d];
  }
  X.x[0][idx] = q;
  if constexpr (KIND == KCDFT) X.x[4][idx] = log(r) + 2.0 * ce * r;
}

// After a cycle (3-D): the float64 update g += e of update64_point (with its
// projection and non-positive-density flag) and then k_shared64's quantities
// of the updated iterate, in one pass.  Each point reads and writes only its
// own values, so the update can be in place.
template <int KIND, int DIM, typename T>
__global__ void __launch_bounds__(TPB) k_update_shared64(Fields64 F, Resid64Out O, Shared64 X, int N, double ce,
                                                         double delta) {
  using LY = Layout<KIND, DIM>;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= N) return;
  double gv[LY::NU];
  T ev[LY::NU];  // all loads before the first store
#pragma unroll
  for (int q = 0; q < LY::NU; ++q) {
    gv[q] = F.g[q][idx];
    ev[q] = static_cast<const T*>(O.e0[q])[idx];
  }
  const double rk = F.rho[idx];
#pragma unroll
  for (int q = 0; q < LY::NU; ++q) gv[q] += from_t<T>(ev[q]);
  gv[0] = (delta > 0.0) ? sqrt(gv[0] * gv[0] + delta * delta) : fabs(gv[0]);
  if (F.nonpos && gv[0] <= 0.0) atomicOr(F.nonpos, 1);  // CDFT, delta = 0: ln 0 next
#pragma unroll
  for (int q = 0; q < LY::NU; ++q) F.g[q][idx] = gv[q];
  double q2 = 0;
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    q2 += gv[1 + d] * gv[1 + d];
    X.x[1 + d][idx] = rk * gv[1 + d];
  }
  X.x[0][idx] = q2;
  if constexpr (KIND == KCDFT) X.x[4][idx] = log(gv[0]) + 2.0 * ce * gv[0];
}

// Float64 residual reading the shared quantities of k_shared64.
template <int KIND, int DIM, typename T>
__global__ void __launch_bounds__(TPB) k_resid64_x(Fields64 F, Shared64 X, Resid64Out O, Geo G, Step64 K,
                                                   Phys<double> P, double* partials) {
  using LY = Layout<KIND, DIM>;
  double acc[LY::NU];
#pragma unroll
  for (int q = 0; q < LY::NU; ++q) acc[q] = 0.0;
  float fa[LY::NU];
#pragma unroll
  for (int q = 0; q < LY::NU; ++q) fa[q] = 0.0f;
  const double ih2 = K.ih2, c_div = K.c_div, c_w = K.c_w, c_q = K.c_div, c_m = K.c_m, c_v = K.c_v;
  const double third = 1.0 / 3.0;
  const double* const* g = F.g;
  const double* M = (KIND == KPFC) ? g[LY::IMU] : X.x[4];
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < G.N; idx += gridDim.x * blockDim.x) {
    int i, j, k;
    coords(idx, G, i, j, k);
    const Nb n = neighbours(i, j, k, G);
    const double rkc = F.rho[n.c];
    double N[LY::NU];
    double div = 0;
#pragma unroll
    for (int d = 0; d < DIM; ++d) div += X.x[1 + d][n.p[d]] - X.x[1 + d][n.m[d]];
    N[0] = g[0][n.c] + c_div * div;
    double uc[3], w[3], wx[3];
#pragma unroll
    for (int d = 0; d < DIM; ++d) uc[d] = g[1 + d][n.c];
#pragma unroll
    for (int d = 0; d < LY::NOM; ++d) w[d] = F.om[d][n.c];
    cross<double, DIM>(w, uc, wx);
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      N[1 + a] = rkc * (uc[a] + c_w * wx[a] + c_q * (X.x[0][n.p[a]] - X.x[0][n.m[a]]) + c_m * (M[n.p[a]] - M[n.m[a]]))
               - c_v * (nbsum<double, DIM>(g[1 + a], n) - 2.0 * DIM * uc[a]);
    }
    if constexpr (KIND == KPFC) {
      const double rc = g[0][n.c];
      const double psi = rc - 1.5;
      const double kc = g[LY::IKA][n.c];
      // h^2 Lap_h kappa and h^2 Lap_h rho; the 1/h^2 scale and the cubic (Horner form)
      // go into fused multiply-adds (fewer float64 instructions, the same rows)
      const double dk = nbsum<double, DIM>(g[LY::IKA], n) - 2.0 * DIM * kc;
      const double dr = nbsum<double, DIM>(g[0], n) - 2.0 * DIM * rc;
      N[LY::IMU] = fma(-ih2, dk, g[LY::IMU][n.c] - psi * fma(psi * psi, third, P.alpha));
      N[LY::IKA] = fma(-ih2, dr, kc);
    }
    double rv[LY::NU];  // all loads (S, rho) before the first store
#pragma unroll
    for (int q = 0; q < LY::NU; ++q) rv[q] = F.S[q][idx] - N[q];
    const double g0c = g[0][idx];
#pragma unroll
    for (int q = 0; q < LY::NU; ++q) {
      const double r = rv[q];
      norm_add<T>(O.f0[q], r, acc[q], fa[q], idx);
      if (O.e0[q]) static_cast<T*>(O.e0[q])[idx] = T(0);
      if (O.r64[q]) O.r64[q][idx] = r;
    }
    if (O.cr32) {
      O.cr32[idx] = narrow_rn(g0c);
#pragma unroll
      for (int d = 0; d < DIM; ++d) O.cv32[d][idx] = narrow_rn(uc[d]);
    }
  }
  norm_partials<T, LY::NU>(O.f0[0], acc, fa, partials, blockIdx.x);
}

template <int KIND, int DIM, typename T>
__global__ void __launch_bounds__(TPB) k_resid64(Fields64 F, Resid64Out O, Geo G, Step64 K,
                                                 Phys<double> P, double* partials) {
  resid64_body<KIND, DIM, T>(F, O, G, K, P, partials, blockIdx.x, gridDim.x);
}

// g += e (float64), then the projection of Sec. 6 on rho.
template <int NU, typename T>
__device__ __forceinline__ void update64_point(const Fields64& F, const Resid64Out& O, int N, double delta,
                                               int idx) {
  if (idx >= N) return;
  double gv[NU];
  T ev[NU];  // all loads before the first store
#pragma unroll
  for (int q = 0; q < NU; ++q) {
    gv[q] = F.g[q][idx];
    ev[q] = static_cast<const T*>(O.e0[q])[idx];
  }
#pragma unroll
  for (int q = 0; q < NU; ++q) gv[q] += from_t<T>(ev[q]);
  gv[0] = (delta > 0.0) ? sqrt(gv[0] * gv[0] + delta * delta) : fabs(gv[0]);
  if (F.nonpos && gv[0] <= 0.0) atomicOr(F.nonpos, 1);  // CDFT, delta = 0: ln 0 next
#pragma unroll
  for (int q = 0; q < NU; ++q) F.g[q][idx] = gv[q];
}

template <int NU, typename T>
__global__ void __launch_bounds__(TPB) k_update64(Fields64 F, Resid64Out O, int N, double delta) {
  update64_point<NU, T>(F, O, N, delta, blockIdx.x * blockDim.x + threadIdx.x);
}

// Device-side control block of one step: residual norms, cycle count and
// status; read by the host once per step (graph mode) or per cycle.
struct Ctl {
  double norm;
  double norm0;
  int cycles;
  int status;
  int active;   // batch: the instance still iterates
  int nonpos;   // CDFT: a density <= 0 reached ln this step (FM_ENONPOS)
  int hist;     // converged iterates kept for the extrapolated initial iterate (0, 1 or 2)
  int fault;    // a bounded wait inside a kernel ran out (FM_ETIMEOUT; never cleared)
  unsigned gbar[2];  // grid barrier of the cooperative sweep: arrivals, blocks that left (zero between launches)
};
static_assert(sizeof(Ctl) <= 64, "the control block's slot in the arena and its host mirror hold 64 bytes");

// Initial iterate extrapolated in time (fm_params.init = FM_INIT_EXTRAPOLATE),
// before the prepare of a step: with the converged iterate g^k of the last
// step still in g and the one before in gp, g^0 = 2 g^k - g^{k-1} when two
// are known (hist = 2), g^k when one is (hist = 1); gp <- g^k.  A density the
// extrapolation would make non-positive keeps g^k.  Nothing is done when no
// converged iterate is known (hist = 0): the prepare then writes the
// previous time level.
struct Ptr6 {
  double* p[MAXU];
};

template <int NU>
__global__ void __launch_bounds__(TPB) k_extrapolate(Ptr6 g, Ptr6 gp, int N, const Ctl* ctl) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const int h = ctl->hist;
  if (idx >= N || h == 0) return;
#pragma unroll
  for (int q = 0; q < NU; ++q) {
    const double gc = g.p[q][idx];
    double gn = gc;
    if (h >= 2) {
      gn = 2.0 * gc - gp.p[q][idx];
      if (q == 0 && !(gn > 0.0)) gn = gc;
    }
    gp.p[q][idx] = gc;
    g.p[q][idx] = gn;
  }
}

// After the step's commit: one more converged iterate kept (at most 2), or
// none after a failed step (its iterate is not a solution).
static __global__ void k_hist_advance(Ctl* ctl) {
  if (threadIdx.x == 0 && blockIdx.x == 0) ctl->hist = ctl->status == FM_OK ? min(ctl->hist + 1, 2) : 0;
}

// Finishes the residual norm max_q sqrt(w * sum_q), updates the control
// block (cycles += in_body) and, in graph mode, sets the WHILE condition:
// continue while the norm is finite, above tol and cycles < max_cycles.
// Block-level body: thread 0 returns whether the instance continues.
template <int NQ>
__device__ __forceinline__ bool norm_ctl_body(const double* partials, int nblk, double w, Ctl* ctl, double tol,
                                              int max_cycles, int in_body) {
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
    if (ctl->fault) status = FM_ETIMEOUT;
    else if (ctl->nonpos) status = FM_ENONPOS;
    else if (!finite) status = FM_ENAN;
    else if (nrm > tol && cycles >= max_cycles) status = FM_ENOCONV;
    ctl->status = status;
    return status == FM_OK && nrm > tol;
  }
  return false;
}

template <int NQ>
__global__ void k_norm_ctl(const double* partials, int nblk, double w, Ctl* ctl, double tol, int max_cycles,
                           int in_body, cudaGraphConditionalHandle handle, int use_handle) {
  const bool cont = norm_ctl_body<NQ>(partials, nblk, w, ctl, tol, max_cycles, in_body);
  if (threadIdx.x == 0 && use_handle) cudaGraphSetConditional(handle, cont ? 1u : 0u);
}

// rho^{k+1} = S1 - (s/4h) sum_d ([rho^k u_d]_{+d} - [rho^k u_d]_{-d}), projected,
// into `out`; skipped unless the solve succeeded.
template <int DIM>
__device__ __forceinline__ void closure_point(const Fields64& F, const Geo& G, const Step64& K, const Phys<double>& P,
                                              double* out, int idx) {
  if (idx >= G.N) return;
  int i, j, k;
  coords(idx, G, i, j, k);
  const Nb n = neighbours(i, j, k, G);
  double div = 0;
#pragma unroll
  for (int d = 0; d < DIM; ++d)
    div += F.rho[n.p[d]] * F.g[1 + d][n.p[d]] - F.rho[n.m[d]] * F.g[1 + d][n.m[d]];
  const double r = F.S[0][idx] - K.c_div * div;
  out[idx] = (P.delta > 0.0) ? sqrt(r * r + P.delta * P.delta) : fabs(r);
}

template <int DIM>
__global__ void __launch_bounds__(TPB) k_closure(Fields64 F, Geo G, Step64 K, Phys<double> P, double* out,
                                                 const Ctl* ctl) {
  if (ctl->status != FM_OK) return;
  closure_point<DIM>(F, G, K, P, out, blockIdx.x * blockDim.x + threadIdx.x);
}

// New time level: rho <- closure result, u <- converged velocity (if the
// solve succeeded).
template <int DIM>
__device__ __forceinline__ void commit_point(double* rho, const Vel3W& vel, const double* rnew, const Vel3& gvel,
                                             int N, int idx) {
  if (idx >= N) return;
  double v[DIM];
  const double r = rnew[idx];
#pragma unroll
  for (int d = 0; d < DIM; ++d) v[d] = gvel.p[d][idx];
  rho[idx] = r;
#pragma unroll
  for (int d = 0; d < DIM; ++d) vel.p[d][idx] = v[d];
}

template <int DIM>
__global__ void __launch_bounds__(TPB) k_commit(double* rho, Vel3W vel, const double* rnew, Vel3 gvel, int N,
                                                const Ctl* ctl) {
  if (ctl->status != FM_OK) return;
  commit_point<DIM>(rho, vel, rnew, gvel, N, blockIdx.x * blockDim.x + threadIdx.x);
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
  block_partials<NQ>(acc, partials, blockIdx.x);
}

// Shared-memory layout of the small-level V-cycle; returns the bytes needed.
template <typename T, int KIND, int DIM>
static size_t small_layout(const SmallLv<T>& S, SmallSmem<T>& M, size_t limit) {
  using LY = Layout<KIND, DIM>;
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
  const int base = off;
  for (int q = 0; q < S.count; ++q) {
    const int N = S.lv[q].g.N;
    M.off_rk[q] = off; off += N;
    M.off_cr[q] = off; off += N;
    for (int d = 0; d < LY::NOM; ++d) { M.off_om[q][d] = off; off += N; }
    for (int d = 0; d < DIM; ++d) { M.off_cv[q][d] = off; off += N; }
  }
  M.stage_coef = (size_t)off * sizeof(T) <= limit ? 1 : 0;
  return (size_t)(M.stage_coef ? off : base) * sizeof(T);
}

// --------------------------------------------------------------------------
// Host-side builders of the kernel argument structs from a state
// --------------------------------------------------------------------------
template <typename T>
static Lvl<T> make_lvl_bufs(const LevelBufs& B) {
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
static Lvl<T> make_lvl(const fm_state* st, int l) {
  return make_lvl_bufs<T>(st->lv[l]);
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
  F.nonpos = st->kind == FM_CDFT ? &static_cast<Ctl*>(st->ctl)->nonpos : nullptr;
  F.hist = st->prm.init == FM_INIT_EXTRAPOLATE ? &static_cast<Ctl*>(st->ctl)->hist : nullptr;
  if (st->prm.precision == FM_MIXED) {
    F.rk32 = (float*)st->lv[0].rk;
    for (int d = 0; d < st->nom; ++d) F.om32[d] = (float*)st->lv[0].om[d];
  }
  return F;
}


}  // namespace fm
