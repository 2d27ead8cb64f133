// Internal definitions shared by the CUDA translation units of libfm.
//
// Unknown ordering of an iterate g (App. G): 0 = rho, 1..dim = velocity,
// then for PFC dim+1 = mu and dim+2 = kappa.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cmath>

namespace fm {

enum { KPFC = 1, KCDFT = 2 };
constexpr int MAXU = 6;

template <int KIND, int DIM>
struct Layout {
  static constexpr int NU = 1 + DIM + (KIND == KPFC ? 2 : 0);
  static constexpr int IMU = 1 + DIM;
  static constexpr int IKA = 2 + DIM;
  static constexpr int NOM = (DIM == 2) ? 1 : 3;
};

struct Geo {
  int nx, ny, nz;   // nz = 1 in 2-D
  int N;            // nx*ny*nz
};

// One multigrid level in precision T (correction form, see fm_solver.cu).
template <typename T>
struct Lvl {
  Geo g;
  T h;
  T* e[MAXU];        // correction unknowns
  T* f[MAXU];        // right-hand side
  T* r[MAXU];        // residual
  T* eh[MAXU];       // injected correction (coarse levels)
  const T* rk;       // rho^k
  const T* om[3];    // omega^k
  const T* cr;       // coefficient iterate: rho
  const T* cv[3];    // coefficient iterate: velocity
};

template <typename T>
struct Phys {
  T s, gamma, alpha, ce, sigma, w, delta;
};

// Periodic neighbour indices of a point.
struct Nb {
  int c;
  int m[3], p[3];
};

__device__ __forceinline__ Nb neighbours(int i, int j, int k, const Geo& g) {
  Nb n;
  const int plane = g.nx * g.ny;
  const int row = (k * g.ny + j) * g.nx;
  n.c = row + i;
  n.m[0] = row + (i == 0 ? g.nx - 1 : i - 1);
  n.p[0] = row + (i == g.nx - 1 ? 0 : i + 1);
  n.m[1] = n.c + (j == 0 ? (g.ny - 1) * g.nx : -g.nx);
  n.p[1] = n.c + (j == g.ny - 1 ? -(g.ny - 1) * g.nx : g.nx);
  if (g.nz > 1) {
    n.m[2] = n.c + (k == 0 ? (g.nz - 1) * plane : -plane);
    n.p[2] = n.c + (k == g.nz - 1 ? -(g.nz - 1) * plane : plane);
  } else {
    n.m[2] = n.p[2] = n.c;
  }
  return n;
}

// x mod n for any int x (periodic index).
__device__ __forceinline__ int wrapi(int x, int n) {
  if (x < 0) x += n;
  else if (x >= n) x -= n;
  if ((unsigned)x >= (unsigned)n) {
    x %= n;
    if (x < 0) x += n;
  }
  return x;
}

__device__ __forceinline__ void coords(int idx, const Geo& g, int& i, int& j, int& k) {
  i = idx % g.nx;
  const int t = idx / g.nx;
  j = t % g.ny;
  k = t / g.ny;
}

// Thread t of a colour sweep -> point (i, j, k) with (i + j + k) % 2 == color.
__device__ __forceinline__ bool colour_point(int t, int color, const Geo& g, int& i, int& j, int& k) {
  const int half = g.nx >> 1;
  const int rowid = t / half;
  if (rowid >= g.ny * g.nz) return false;
  j = rowid % g.ny;
  k = rowid / g.ny;
  i = 2 * (t - rowid * half) + ((j + k + color) & 1);
  return true;
}

__device__ __forceinline__ float log1p_t(float x) { return log1pf(x); }
__device__ __forceinline__ double log1p_t(double x) { return log1p(x); }
__device__ __forceinline__ float sqrt_t(float x) { return sqrtf(x); }
__device__ __forceinline__ double sqrt_t(double x) { return sqrt(x); }

template <typename T, int DIM>
__device__ __forceinline__ T nbsum(const T* a, const Nb& n) {
  T s = a[n.m[0]] + a[n.p[0]] + a[n.m[1]] + a[n.p[1]];
  if constexpr (DIM == 3) s += a[n.m[2]] + a[n.p[2]];
  return s;
}

// omega x U (omega along z in 2-D).
template <typename T, int DIM>
__device__ __forceinline__ void cross(const T* w, const T* U, T* out) {
  if constexpr (DIM == 2) {
    out[0] = -w[0] * U[1];
    out[1] = w[0] * U[0];
  } else {
    out[0] = w[1] * U[2] - w[2] * U[1];
    out[1] = w[2] * U[0] - w[0] * U[2];
    out[2] = w[0] * U[1] - w[1] * U[0];
  }
}

// Correction-form momentum kinetic term |c + e|^2 - |c|^2 = e (2c + e).
template <typename T, int DIM>
__device__ __forceinline__ T qcorr(T* const* E, const T* const* cv, int idx) {
  T q = 0;
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    const T e = E[1 + d][idx];
    q += e * (T(2) * cv[d][idx] + e);
  }
  return q;
}

// Correction-form implicit chemical potential: e_mu (PFC) or
// ln(c + e) - ln(c) + 2 c_e e (CDFT).
template <typename T, int KIND, int DIM>
__device__ __forceinline__ T mcorr(T* const* E, const T* cr, int idx, T ce) {
  if constexpr (KIND == KPFC) {
    return E[Layout<KIND, DIM>::IMU][idx];
  } else {
    const T e = E[0][idx];
    return log1p_t(e / cr[idx]) + T(2) * ce * e;
  }
}

// M(e) = N(c + e) - N(c) at one point, all components (App. G operator N in
// correction form about the coefficient iterate c).
template <typename T, int KIND, int DIM>
__device__ __forceinline__ void applyM(const Lvl<T>& L, const Phys<T>& P, const Nb& n,
                                       T* const* E, T* M) {
  using LY = Layout<KIND, DIM>;
  const T ih = T(1) / L.h;
  const T ih2 = ih * ih;
  const T rkc = L.rk[n.c];
  T div = 0;
#pragma unroll
  for (int d = 0; d < DIM; ++d)
    div += L.rk[n.p[d]] * E[1 + d][n.p[d]] - L.rk[n.m[d]] * E[1 + d][n.m[d]];
  M[0] = E[0][n.c] + P.s * T(0.25) * ih * div;

  T ec[3], w[3], wx[3];
#pragma unroll
  for (int d = 0; d < DIM; ++d) ec[d] = E[1 + d][n.c];
#pragma unroll
  for (int d = 0; d < LY::NOM; ++d) w[d] = L.om[d][n.c];
  cross<T, DIM>(w, ec, wx);
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    const T dq = qcorr<T, DIM>(E, L.cv, n.p[a]) - qcorr<T, DIM>(E, L.cv, n.m[a]);
    const T dm = mcorr<T, KIND, DIM>(E, L.cr, n.p[a], P.ce) - mcorr<T, KIND, DIM>(E, L.cr, n.m[a], P.ce);
    const T lapa = (nbsum<T, DIM>(E[1 + a], n) - T(2 * DIM) * ec[a]) * ih2;
    M[1 + a] = rkc * ec[a] + T(0.5) * P.sigma * P.s * rkc * wx[a]
             + P.s * rkc * ih * (T(0.25) * dq + T(0.5) * dm)
             - T(0.5) * P.s * P.gamma * lapa;
  }
  if constexpr (KIND == KPFC) {
    const T er = E[0][n.c];
    const T psi = L.cr[n.c] - T(1.5);
    const T ek = E[LY::IKA][n.c];
    const T lapk = (nbsum<T, DIM>(E[LY::IKA], n) - T(2 * DIM) * ek) * ih2;
    const T lapr = (nbsum<T, DIM>(E[0], n) - T(2 * DIM) * er) * ih2;
    M[LY::IMU] = E[LY::IMU][n.c] - er * (psi * psi + psi * er + er * er * T(1.0 / 3.0)) - P.alpha * er - lapk;
    M[LY::IKA] = ek - lapr;
  }
}

}  // namespace fm
