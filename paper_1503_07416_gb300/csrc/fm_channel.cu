// libfm: the hydrodynamic PFC step in a channel (fm_params.walls = FM_WALLS_Y):
// periodic in x, no-slip walls at y = 0 and y = n_y h (Sec. 6.3), the walls
// moving along x at u_wall[0] (bottom) and u_wall[1] (top).
//
// Grid: the n_y rows are cells j = 0 .. n_y - 1 (centres at (j + 1/2) h), the
// walls half a cell beyond the first and last rows.  A neighbour across a
// wall is a ghost given by the rules of App. E.2: scalars (rho, rho^k, mu,
// kappa) mirror the wall row (no flux), the normal velocity is odd (no
// slip), the tangential velocity is 2 U_wall - u (no slip on a wall moving
// at U_wall); |u|^2 takes the ghosts of its factors.  In the correction form
// of the cycle (M(e) = N(c + e) - N(c)) the corrections carry homogeneous
// ghosts (odd velocity, mirrored scalars) and the coefficient velocity the
// wall speed.
//
// The same scheme and solver as fm_solver.cu otherwise: float64 outer
// residual, FAS V-cycles on the correction equation in precision T, the
// hydrodynamic point block (smooth_point_a) evaluated through an accessor
// that returns the ghost values, red and black launches per sweep, the
// coarsest level smoothed ncoarse times; the transfers are nodal in x and
// cell-centred in y (a coarse cell is two fine cells: restriction and
// injection average them, prolongation interpolates linearly between cell
// centres, weights 3/4 and 1/4).  One CUDA graph per step (fm_stepper.cuh).
#include <cuda_runtime.h>
#include <cstring>

#include "fm_state.h"
#include "fm_device.cuh"
#include "fm_stepper.cuh"

namespace fm {
namespace ch {

using LY = Layout<KPFC, 2>;  // rho, u, v, mu, kappa

// Neighbours of cell (i, j) of a channel level: x periodic; a neighbour
// across a wall is encoded as -1 - c (bottom) or -1 - c - N (top), c the wall
// row's own cell (the ghost mirrors it).
__device__ __forceinline__ Nb ch_neighbours(int i, int j, const Geo& g) {
  Nb n;
  const int row = j * g.nx;
  n.c = row + i;
  n.m[0] = row + (i == 0 ? g.nx - 1 : i - 1);
  n.p[0] = row + (i == g.nx - 1 ? 0 : i + 1);
  n.m[1] = j == 0 ? -1 - n.c : n.c - g.nx;
  n.p[1] = j == g.ny - 1 ? -1 - n.c - g.N : n.c + g.nx;
  n.m[2] = n.p[2] = n.c;
  return n;
}

__device__ __forceinline__ int cell_of(int i, int N) {
  if (i >= 0) return i;
  const int m = -1 - i;
  return m >= N ? m - N : m;
}

// Ghost of a value: 0 scalar (mirror), 1 tangential velocity (2U - x),
// 2 normal velocity (-x).
template <typename T>
__device__ __forceinline__ T ghost_of(T x, int type, T U) {
  return type == 0 ? x : (type == 2 ? -x : T(2) * U - x);
}

// Accessor of the correction-form point update over a channel level.
template <typename T>
struct ChAcc {
  const Lvl<T>& L;
  T ub, ut;  // wall speeds (of the coefficient velocity)
  __device__ __forceinline__ T e(int q, int i) const {
    const T v = L.e[q][cell_of(i, L.g.N)];
    return (i < 0 && (q == 1 || q == 2)) ? -v : v;  // corrections: odd velocity ghosts
  }
  __device__ __forceinline__ void set_e(int q, int i, T v) const { L.e[q][i] = v; }
  __device__ __forceinline__ T rk(int i) const { return L.rk[cell_of(i, L.g.N)]; }
  __device__ __forceinline__ T cr(int i) const { return L.cr[cell_of(i, L.g.N)]; }
  __device__ __forceinline__ T cv(int d, int i) const {
    const T v = L.cv[d][cell_of(i, L.g.N)];
    if (i >= 0) return v;
    return ghost_of(v, d == 0 ? 1 : 2, i < -L.g.N ? ut : ub);
  }
  __device__ __forceinline__ T f(int q, int i) const { return L.f[q][i]; }
  __device__ __forceinline__ T om(int d, int i) const { return L.om[d][i]; }
};

template <typename T>
struct WallsT {
  T ub, ut;
};

template <typename T>
__global__ void __launch_bounds__(TPB) k_ch_smooth(Lvl<T> L, Phys<T> P, WallsT<T> W, int color) {
  int i, j, k;
  if (!colour_point(blockIdx.x * blockDim.x + threadIdx.x, color, L.g, i, j, k)) return;
  ChAcc<T> a{L, W.ub, W.ut};
  const Nb n = ch_neighbours(i, j, L.g);
  smooth_point_a<T, KPFC, 2>(a, P, make_ptk<T, 2>(P, L.h), n, n.c);
}

// M(e) = N(c + e) - N(c) at one cell, through the accessor (App. G.2 operator
// in correction form, as applyM of the periodic solver).
template <typename T>
__device__ __forceinline__ void ch_applyM(const ChAcc<T>& a, const Phys<T>& P, T h, const Nb& n, T* M) {
  const T ih = T(1) / h, ih2 = ih * ih;
  const int c = n.c;
  const T rkc = a.rk(c);
  T div = 0;
#pragma unroll
  for (int d = 0; d < 2; ++d) div += a.rk(n.p[d]) * a.e(1 + d, n.p[d]) - a.rk(n.m[d]) * a.e(1 + d, n.m[d]);
  M[0] = a.e(0, c) + P.s * T(0.25) * ih * div;
  auto qc = [&](int idx) {
    T q = 0;
#pragma unroll
    for (int d = 0; d < 2; ++d) {
      const T e = a.e(1 + d, idx);
      q += e * (T(2) * a.cv(d, idx) + e);
    }
    return q;
  };
  const T ec[2] = {a.e(1, c), a.e(2, c)};
  const T w = a.om(0, c);
  const T wx[2] = {-w * ec[1], w * ec[0]};
#pragma unroll
  for (int d = 0; d < 2; ++d) {
    const T dq = qc(n.p[d]) - qc(n.m[d]);
    const T dm = a.e(LY::IMU, n.p[d]) - a.e(LY::IMU, n.m[d]);
    const T nb = a.e(1 + d, n.m[0]) + a.e(1 + d, n.p[0]) + a.e(1 + d, n.m[1]) + a.e(1 + d, n.p[1]);
    const T lapa = (nb - T(4) * ec[d]) * ih2;
    M[1 + d] = rkc * ec[d] + T(0.5) * P.sigma * P.s * rkc * wx[d] + P.s * rkc * ih * (T(0.25) * dq + T(0.5) * dm)
             - T(0.5) * P.s * P.gamma * lapa;
  }
  const T er = a.e(0, c), ek = a.e(LY::IKA, c);
  const T psi = a.cr(c) - T(1.5);
  const T nbk = a.e(LY::IKA, n.m[0]) + a.e(LY::IKA, n.p[0]) + a.e(LY::IKA, n.m[1]) + a.e(LY::IKA, n.p[1]);
  const T nbr = a.e(0, n.m[0]) + a.e(0, n.p[0]) + a.e(0, n.m[1]) + a.e(0, n.p[1]);
  M[LY::IMU] = a.e(LY::IMU, c) - er * (psi * psi + psi * er + er * er * T(1.0 / 3.0)) - P.alpha * er
             - (nbk - T(4) * ek) * ih2;
  M[LY::IKA] = ek - (nbr - T(4) * er) * ih2;
}

// r = f - M(e) on a level (out = L.r), or f += M(e) (coarse right-hand side).
template <typename T, bool RHS>
__global__ void __launch_bounds__(TPB) k_ch_resid(Lvl<T> L, Phys<T> P, WallsT<T> W) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= L.g.N) return;
  const int i = idx % L.g.nx, j = idx / L.g.nx;
  ChAcc<T> a{L, W.ub, W.ut};
  T M[LY::NU], fv[LY::NU];
#pragma unroll
  for (int q = 0; q < LY::NU; ++q) fv[q] = L.f[q][idx];
  ch_applyM<T>(a, P, L.h, ch_neighbours(i, j, L.g), M);
#pragma unroll
  for (int q = 0; q < LY::NU; ++q) {
    if (RHS) L.f[q][idx] = fv[q] + M[q];
    else L.r[q][idx] = fv[q] - M[q];
  }
}

// Coarse cell (I, J) of fine rows 2J, 2J + 1: f_C = R(r_F) (x full weighting
// about 2I, y the mean of the two rows), e_C = eh_C = the injection (the
// mean of the two cells at x = 2I).
template <typename T>
__global__ void __launch_bounds__(TPB) k_ch_restrict(Lvl<T> F, Lvl<T> C) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= C.g.N) return;
  const int I = idx % C.g.nx, J = idx / C.g.nx;
  const int x = 2 * I, xm = x == 0 ? F.g.nx - 1 : x - 1, xp = x + 1 == F.g.nx ? 0 : x + 1;
  const int r0 = 2 * J * F.g.nx, r1 = r0 + F.g.nx;
  T fr[LY::NU], ev[LY::NU];
#pragma unroll
  for (int q = 0; q < LY::NU; ++q) {
    const T* r = F.r[q];
    fr[q] = T(0.125) * (r[r0 + xm] + r[r1 + xm] + r[r0 + xp] + r[r1 + xp]) + T(0.25) * (r[r0 + x] + r[r1 + x]);
    ev[q] = T(0.5) * (F.e[q][r0 + x] + F.e[q][r1 + x]);
  }
#pragma unroll
  for (int q = 0; q < LY::NU; ++q) {
    C.f[q][idx] = fr[q];
    C.e[q][idx] = ev[q];
    C.eh[q][idx] = ev[q];
  }
}

// Coefficients of level F injected into level C (same averaging): rho^k and
// omega^k (which = 0) or the coefficient iterate rho, u, v (which = 1).
template <typename T>
__global__ void __launch_bounds__(TPB) k_ch_inject(Lvl<T> F, Lvl<T> C, int which) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= C.g.N) return;
  const int I = idx % C.g.nx, J = idx / C.g.nx;
  const int a = 2 * J * F.g.nx + 2 * I, b = a + F.g.nx;
  if (which == 0) {
    const_cast<T*>(C.rk)[idx] = T(0.5) * (F.rk[a] + F.rk[b]);
    const_cast<T*>(C.om[0])[idx] = T(0.5) * (F.om[0][a] + F.om[0][b]);
  } else {
    const_cast<T*>(C.cr)[idx] = T(0.5) * (F.cr[a] + F.cr[b]);
    const_cast<T*>(C.cv[0])[idx] = T(0.5) * (F.cv[0][a] + F.cv[0][b]);
    const_cast<T*>(C.cv[1])[idx] = T(0.5) * (F.cv[1][a] + F.cv[1][b]);
  }
}

// e_F += P(e_C - eh_C): x linear between nodes, y linear between cell
// centres (3/4 the own coarse cell, 1/4 the next one towards the fine cell),
// the coarse correction's ghost beyond a wall mirrored (scalars) or odd
// (velocity).
template <typename T>
__global__ void __launch_bounds__(TPB) k_ch_prolong(Lvl<T> F, Lvl<T> C) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= F.g.N) return;
  const int i = idx % F.g.nx, j = idx / F.g.nx;
  const int J = j >> 1;
  const int Jn = (j & 1) ? J + 1 : J - 1;
  const bool ghost = Jn < 0 || Jn >= C.g.ny;
  const int Jr = ghost ? J : Jn;
  const int I0 = i >> 1, I1 = (I0 + 1 == C.g.nx) ? 0 : I0 + 1;
  const bool odd = i & 1;
  T ev[LY::NU];
#pragma unroll
  for (int q = 0; q < LY::NU; ++q) {
    const T sg = (ghost && (q == 1 || q == 2)) ? T(-1) : T(1);
    auto dc = [&](int JJ, int II) { return C.e[q][JJ * C.g.nx + II] - C.eh[q][JJ * C.g.nx + II]; };
    T v0 = T(0.75) * dc(J, I0) + T(0.25) * sg * dc(Jr, I0);
    if (odd) v0 = T(0.5) * (v0 + T(0.75) * dc(J, I1) + T(0.25) * sg * dc(Jr, I1));
    ev[q] = F.e[q][idx] + v0;
  }
#pragma unroll
  for (int q = 0; q < LY::NU; ++q) F.e[q][idx] = ev[q];
}

// ---------------------------------------------------------------------------
// float64 kernels of the finest level
// ---------------------------------------------------------------------------
struct Walls64 {
  double ub, ut;
};

// value of array x at an encoded neighbour index with ghost type `type`
__device__ __forceinline__ double gv(const double* x, int i, int N, int type, const Walls64& W) {
  const double v = x[cell_of(i, N)];
  return i >= 0 ? v : ghost_of(v, type, i < -N ? W.ut : W.ub);
}

// omega^k, S, g^0 (kappa^0 = Lap_h rho^k) with the wall ghosts.
__global__ void __launch_bounds__(TPB) k_ch_prepare(Fields64 F, Geo G, Step64 K, Walls64 W) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= G.N) return;
  const int i = idx % G.nx, j = idx / G.nx;
  const Nb n = ch_neighbours(i, j, G);
  const double* u = F.vel[0];
  const double* v = F.vel[1];
  const int N = G.N;
  const double w = K.hih * ((gv(v, n.p[0], N, 2, W) - gv(v, n.m[0], N, 2, W)) -
                            (gv(u, n.p[1], N, 1, W) - gv(u, n.m[1], N, 1, W)));
  const double rkc = F.rho[idx];
  double div = 0.0;
#pragma unroll
  for (int d = 0; d < 2; ++d)
    div += gv(F.rho, n.p[d], N, 0, W) * gv(F.vel[d], n.p[d], N, d + 1, W) -
           gv(F.rho, n.m[d], N, 0, W) * gv(F.vel[d], n.m[d], N, d + 1, W);
  const double uc[2] = {u[idx], v[idx]};
  const double wx[2] = {-w * uc[1], w * uc[0]};
  double sv[2];
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    const double nb = gv(F.vel[a], n.m[0], N, a + 1, W) + gv(F.vel[a], n.p[0], N, a + 1, W) +
                      gv(F.vel[a], n.m[1], N, a + 1, W) + gv(F.vel[a], n.p[1], N, a + 1, W);
    sv[a] = rkc * (uc[a] - K.c_w * wx[a]) + K.c_v * (nb - 4.0 * uc[a]);
  }
  const double nbr = gv(F.rho, n.m[0], N, 0, W) + gv(F.rho, n.p[0], N, 0, W) + gv(F.rho, n.m[1], N, 0, W) +
                     gv(F.rho, n.p[1], N, 0, W);
  const double lapr = (nbr - 4.0 * rkc) * K.ih2;
  F.S[0][idx] = rkc - K.c_div * div;
  F.S[1][idx] = sv[0];
  F.S[2][idx] = sv[1];
  F.S[LY::IMU][idx] = 2.0 * lapr;
  F.S[LY::IKA][idx] = 0.0;
  F.g[0][idx] = rkc;
  F.g[1][idx] = uc[0];
  F.g[2][idx] = uc[1];
  F.g[LY::IKA][idx] = lapr;
  F.om[0][idx] = w;
  if (F.rk32) {
    F.rk32[idx] = narrow_rn(rkc);
    F.om32[0][idx] = narrow_rn(w);
  }
}

// mu^0 = psi^3/3 + alpha psi + Lap_h kappa^0 + S_mu.
__global__ void __launch_bounds__(TPB) k_ch_prepare_mu(Fields64 F, Geo G, Step64 K, double alpha, Walls64 W) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= G.N) return;
  const int i = idx % G.nx, j = idx / G.nx;
  const Nb n = ch_neighbours(i, j, G);
  const double* ka = F.g[LY::IKA];
  const int N = G.N;
  const double nbk = gv(ka, n.m[0], N, 0, W) + gv(ka, n.p[0], N, 0, W) + gv(ka, n.m[1], N, 0, W) +
                     gv(ka, n.p[1], N, 0, W);
  const double psi = F.rho[idx] - 1.5;
  F.g[LY::IMU][idx] = psi * psi * psi * (1.0 / 3.0) + alpha * psi + (nbk - 4.0 * ka[idx]) * K.ih2 + F.S[LY::IMU][idx];
}

// r = S - N(g) in float64 with the wall ghosts; the level-0 set-up of a
// cycle and the block partial sums of r^2 (as resid64_body).
template <typename T>
__global__ void __launch_bounds__(TPB) k_ch_resid64(Fields64 F, Resid64Out O, Geo G, Step64 K, Phys<double> P,
                                                    Walls64 W, double* partials) {
  double acc[LY::NU];
  float fa[LY::NU];
#pragma unroll
  for (int q = 0; q < LY::NU; ++q) {
    acc[q] = 0.0;
    fa[q] = 0.0f;
  }
  const int N = G.N;
  const double* const* g = F.g;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += gridDim.x * blockDim.x) {
    const int i = idx % G.nx, j = idx / G.nx;
    const Nb n = ch_neighbours(i, j, G);
    const double rkc = F.rho[idx];
    double Nv[LY::NU];
    double div = 0.0;
#pragma unroll
    for (int d = 0; d < 2; ++d)
      div += gv(F.rho, n.p[d], N, 0, W) * gv(g[1 + d], n.p[d], N, d + 1, W) -
             gv(F.rho, n.m[d], N, 0, W) * gv(g[1 + d], n.m[d], N, d + 1, W);
    Nv[0] = g[0][idx] + K.c_div * div;
    const double uc[2] = {g[1][idx], g[2][idx]};
    const double w = F.om[0][idx];
    const double wx[2] = {-w * uc[1], w * uc[0]};
    auto q_at = [&](int k) {
      const double a = gv(g[1], k, N, 1, W), b = gv(g[2], k, N, 2, W);
      return a * a + b * b;
    };
#pragma unroll
    for (int a = 0; a < 2; ++a) {
      const double dq = q_at(n.p[a]) - q_at(n.m[a]);
      const double dm = gv(g[LY::IMU], n.p[a], N, 0, W) - gv(g[LY::IMU], n.m[a], N, 0, W);
      const double nb = gv(g[1 + a], n.m[0], N, a + 1, W) + gv(g[1 + a], n.p[0], N, a + 1, W) +
                        gv(g[1 + a], n.m[1], N, a + 1, W) + gv(g[1 + a], n.p[1], N, a + 1, W);
      Nv[1 + a] = rkc * (uc[a] + K.c_w * wx[a] + K.c_div * dq + K.c_m * dm) - K.c_v * (nb - 4.0 * uc[a]);
    }
    const double rc = g[0][idx], psi = rc - 1.5, kc = g[LY::IKA][idx];
    const double nbk = gv(g[LY::IKA], n.m[0], N, 0, W) + gv(g[LY::IKA], n.p[0], N, 0, W) +
                       gv(g[LY::IKA], n.m[1], N, 0, W) + gv(g[LY::IKA], n.p[1], N, 0, W);
    const double nbr = gv(g[0], n.m[0], N, 0, W) + gv(g[0], n.p[0], N, 0, W) + gv(g[0], n.m[1], N, 0, W) +
                       gv(g[0], n.p[1], N, 0, W);
    Nv[LY::IMU] = g[LY::IMU][idx] - psi * (psi * psi * (1.0 / 3.0) + P.alpha) - (nbk - 4.0 * kc) * K.ih2;
    Nv[LY::IKA] = kc - (nbr - 4.0 * rc) * K.ih2;
    double rv[LY::NU];
#pragma unroll
    for (int q = 0; q < LY::NU; ++q) rv[q] = F.S[q][idx] - Nv[q];
#pragma unroll
    for (int q = 0; q < LY::NU; ++q) {
      norm_add<T>(O.f0[q], rv[q], acc[q], fa[q], idx);
      if (O.e0[q]) static_cast<T*>(O.e0[q])[idx] = T(0);
      if (O.r64[q]) O.r64[q][idx] = rv[q];
    }
    if (O.cr32) {
      O.cr32[idx] = narrow_rn(rc);
      O.cv32[0][idx] = narrow_rn(uc[0]);
      O.cv32[1][idx] = narrow_rn(uc[1]);
    }
  }
  norm_partials<T, LY::NU>(O.f0[0], acc, fa, partials, blockIdx.x);
}

// rho^{k+1} = S1 - (s/4h) sum_d ([rho^k u_d]_{+d} - [rho^k u_d]_{-d}) with the
// converged velocity (the explicit half is in S1), projected; skipped unless
// the solve succeeded.
__global__ void __launch_bounds__(TPB) k_ch_closure(Fields64 F, Geo G, Step64 K, double delta, Walls64 W, double* out,
                                                    const Ctl* ctl) {
  if (ctl->status != FM_OK) return;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= G.N) return;
  const int i = idx % G.nx, j = idx / G.nx;
  const Nb n = ch_neighbours(i, j, G);
  double div = 0.0;
#pragma unroll
  for (int d = 0; d < 2; ++d)
    div += gv(F.rho, n.p[d], G.N, 0, W) * gv(F.g[1 + d], n.p[d], G.N, d + 1, W) -
           gv(F.rho, n.m[d], G.N, 0, W) * gv(F.g[1 + d], n.m[d], G.N, d + 1, W);
  const double r = F.S[0][idx] - K.c_div * div;
  out[idx] = delta > 0.0 ? sqrt(r * r + delta * delta) : fabs(r);
}

// Energy densities of the PFC functional with the Neumann Laplacian, and KE.
__global__ void __launch_bounds__(TPB) k_ch_energy(const double* rho, const double* u, const double* v, Geo G,
                                                   double h, double alpha, double* partials) {
  double acc[5] = {0, 0, 0, 0, 0};
  const double ih2 = 1.0 / (h * h);
  const Walls64 W{0.0, 0.0};
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < G.N; idx += gridDim.x * blockDim.x) {
    const int i = idx % G.nx, j = idx / G.nx;
    const Nb n = ch_neighbours(i, j, G);
    const double rc = rho[idx];
    acc[0] += 0.5 * rc * (u[idx] * u[idx] + v[idx] * v[idx]);
    const double psi = rc - 1.5;
    const double L = (gv(rho, n.m[0], G.N, 0, W) + gv(rho, n.p[0], G.N, 0, W) + gv(rho, n.m[1], G.N, 0, W) +
                      gv(rho, n.p[1], G.N, 0, W) - 4.0 * rc) * ih2;
    acc[1] += psi * psi * psi * psi / 12.0;
    acc[2] += 0.5 * alpha * psi * psi;
    acc[3] += 0.5 * L * L;
    acc[4] += rc * L;
  }
  block_partials<5>(acc, partials, blockIdx.x);
}

// ---------------------------------------------------------------------------
// Host driver
// ---------------------------------------------------------------------------
template <typename T>
struct ChannelSolver {
  static constexpr int NVEL = 2;

  static Walls64 walls64(const fm_state* st) { return Walls64{st->prm.u_wall[0], st->prm.u_wall[1]}; }
  static WallsT<T> wallsT(const fm_state* st) { return WallsT<T>{(T)st->prm.u_wall[0], (T)st->prm.u_wall[1]}; }
  static Step64 step64(const fm_state* st) { return make_step64(make_phys<double>(st), 1.0 / st->lv[0].h); }

  static Resid64Out out0(fm_state* st, bool cycle, double* const* r64) {
    Resid64Out O;
    memset(&O, 0, sizeof(O));
    for (int q = 0; q < LY::NU; ++q) {
      O.f0[q] = cycle ? st->lv[0].f[q] : nullptr;
      O.e0[q] = cycle ? st->lv[0].e[q] : nullptr;
      O.r64[q] = r64 ? r64[q] : nullptr;
    }
    if (cycle && st->prm.precision == FM_MIXED) {
      O.cr32 = (float*)st->lv[0].cr;
      for (int d = 0; d < 2; ++d) O.cv32[d] = (float*)st->lv[0].cv[d];
    }
    return O;
  }

  static int inject(fm_state* st, int which) {
    for (int l = 0; l + 1 < st->nlev; ++l) {
      const Lvl<T> F = make_lvl<T>(st, l), C = make_lvl<T>(st, l + 1);
      k_ch_inject<T><<<nblocks(C.g.N), TPB, 0, st->stream>>>(F, C, which);
      FM_LAUNCHED();
    }
    return FM_OK;
  }

  static int enqueue_prepare(fm_state* st) {
    const Geo G = st->lv[0].g;
    const Fields64 F = make_fields(st);
    k_ch_prepare<<<nblocks(G.N), TPB, 0, st->stream>>>(F, G, step64(st), walls64(st));
    FM_LAUNCHED();
    k_ch_prepare_mu<<<nblocks(G.N), TPB, 0, st->stream>>>(F, G, step64(st), st->fn.alpha, walls64(st));
    FM_LAUNCHED();
    return inject(st, 0);
  }

  static int launch_resid64(fm_state* st, const Resid64Out& O) {
    k_ch_resid64<T><<<st->nblk, TPB, 0, st->stream>>>(make_fields(st), O, st->lv[0].g, step64(st),
                                                       make_phys<double>(st), walls64(st), st->partials);
    FM_LAUNCHED();
    return FM_OK;
  }

  static int enqueue_resid_norm(fm_state* st, int in_body, cudaGraphConditionalHandle hdl, int use_handle) {
    int rc = launch_resid64(st, out0(st, true, nullptr));
    if (rc) return rc;
    const double h = st->lv[0].h;
    k_norm_ctl<LY::NU><<<1, TPB, 0, st->stream>>>(st->partials, st->nblk, h * h, (Ctl*)st->ctl, st->prm.tol,
                                                  st->prm.max_cycles, in_body, hdl, use_handle);
    FM_LAUNCHED();
    return FM_OK;
  }

  static int smooth(fm_state* st, const Lvl<T>& L, const Phys<T>& P, int iters) {
    for (int it = 0; it < iters; ++it)
      for (int color = 0; color < 2; ++color) {
        k_ch_smooth<T><<<nblocks(L.g.N / 2), TPB, 0, st->stream>>>(L, P, wallsT(st), color);
        FM_LAUNCHED();
      }
    return FM_OK;
  }

  static int vcycle(fm_state* st, int l, const Phys<T>& P) {
    cudaStream_t s = st->stream;
    const Lvl<T> F = make_lvl<T>(st, l);
    if (l == st->nlev - 1) return smooth(st, F, P, st->prm.ncoarse);
    int rc = smooth(st, F, P, st->prm.nu1);
    if (rc) return rc;
    const Lvl<T> C = make_lvl<T>(st, l + 1);
    k_ch_resid<T, false><<<nblocks(F.g.N), TPB, 0, s>>>(F, P, wallsT(st));
    FM_LAUNCHED();
    k_ch_restrict<T><<<nblocks(C.g.N), TPB, 0, s>>>(F, C);
    FM_LAUNCHED();
    k_ch_resid<T, true><<<nblocks(C.g.N), TPB, 0, s>>>(C, P, wallsT(st));
    FM_LAUNCHED();
    rc = vcycle(st, l + 1, P);
    if (rc) return rc;
    k_ch_prolong<T><<<nblocks(F.g.N), TPB, 0, s>>>(F, C);
    FM_LAUNCHED();
    return smooth(st, F, P, st->prm.nu2);
  }

  static int enqueue_body(fm_state* st, cudaGraphConditionalHandle hdl, int use_handle) {
    int rc = inject(st, 1);
    if (rc) return rc;
    rc = vcycle(st, 0, make_phys<T>(st));
    if (rc) return rc;
    const Geo G = st->lv[0].g;
    k_update64<LY::NU, T><<<nblocks(G.N), TPB, 0, st->stream>>>(make_fields(st), out0(st, true, nullptr), G.N,
                                                                st->prm.delta);
    FM_LAUNCHED();
    return enqueue_resid_norm(st, 1, hdl, use_handle);
  }

  static int enqueue_post(fm_state* st) {
    const Geo G = st->lv[0].g;
    const Ctl* ctl = (const Ctl*)st->ctl;
    k_ch_closure<<<nblocks(G.N), TPB, 0, st->stream>>>(make_fields(st), G, step64(st), st->prm.delta, walls64(st),
                                                       st->tmp, ctl);
    FM_LAUNCHED();
    Vel3W vw{{st->vel[0], st->vel[1], nullptr}};
    Vel3 gv3{{st->g[1], st->g[2], nullptr}};
    k_commit<2><<<nblocks(G.N), TPB, 0, st->stream>>>(st->rho, vw, st->tmp, gv3, G.N, ctl);
    FM_LAUNCHED();
    FM_CUDA(cudaMemcpyAsync(st->hscal + 32, st->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st->stream));
    return FM_OK;
  }

  static int prepare(fm_state* st) {
    int rc = enqueue_prepare(st);
    if (rc) return rc;
    FM_CUDA(cudaStreamSynchronize(st->stream));
    st->prepared = true;
    return FM_OK;
  }

  static int residual64(fm_state* st, double* const* r64, double* norm_host) {
    int rc = launch_resid64(st, out0(st, false, r64));
    if (rc) return rc;
    const double h = st->lv[0].h;
    k_norm_final<LY::NU><<<1, TPB, 0, st->stream>>>(st->partials, st->nblk, h * h, st->dscal);
    FM_LAUNCHED();
    FM_CUDA(cudaMemcpyAsync(st->hscal, st->dscal, sizeof(double), cudaMemcpyDeviceToHost, st->stream));
    FM_CUDA(cudaStreamSynchronize(st->stream));
    *norm_host = st->hscal[0];
    return FM_OK;
  }
};

template <typename T>
static int dispatch(fm_state* st, int what, fm_step_info* info, const double* ri, const double* const* vi,
                    double* ro, double* const* vo, double* const* r64, double* nrm) {
  switch (what) {
    case 0: return Stepper<ChannelSolver<T>>::step(st, info);
    case 1: return Stepper<ChannelSolver<T>>::step_host(st, ri, vi, ro, vo, info);
    case 2: return ChannelSolver<T>::prepare(st);
    default: return ChannelSolver<T>::residual64(st, r64, nrm);
  }
}

static int run(fm_state* st, int what, fm_step_info* info, const double* ri, const double* const* vi, double* ro,
               double* const* vo, double* const* r64, double* nrm) {
  return st->prm.precision == FM_MIXED ? dispatch<float>(st, what, info, ri, vi, ro, vo, r64, nrm)
                                       : dispatch<double>(st, what, info, ri, vi, ro, vo, r64, nrm);
}

}  // namespace ch

int ch_step(fm_state* st, fm_step_info* info) {
  return ch::run(st, 0, info, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
}
int ch_step_host(fm_state* st, const double* rho_in, const double* const* vel_in, double* rho_out,
                 double* const* vel_out, fm_step_info* info) {
  return ch::run(st, 1, info, rho_in, vel_in, rho_out, vel_out, nullptr, nullptr);
}
int ch_prepare(fm_state* st) { return ch::run(st, 2, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr); }
int ch_residual(fm_state* st, double* const* r64, double* norm) {
  return ch::run(st, 3, nullptr, nullptr, nullptr, nullptr, nullptr, r64, norm);
}
int ch_energy_launch(fm_state* st) {
  const Geo G = st->lv[0].g;
  ch::k_ch_energy<<<st->nblk, TPB, 0, st->stream>>>(st->rho, st->vel[0], st->vel[1], G, st->lv[0].h, st->fn.alpha,
                                                    st->partials);
  return cudaPeekAtLastError() == cudaSuccess ? FM_OK : (cudaGetLastError(), FM_ECUDA);
}

}  // namespace fm
