// libfm: the conservative gradient-flow scheme of Sec. 3 (Thm 3.3, Eq.
// gradient_scheme) on the same multigrid machinery as the hydrodynamic step:
//
//   rho^{k+1} - rho^k = s Lap_h ( dF_c[rho^{k+1}] - dF_e[rho^k] ),
//
// with the PFC (Lemma 5.4) or CDFT (Lemma 5.2) splitting.  Unknowns per point:
//   PFC   g = (rho, mu, kappa):  N0 = rho - s Lap_h mu
//                                N1 = mu - psi^3/3 - alpha psi - Lap_h kappa
//                                N2 = kappa - Lap_h rho
//         S = (rho^k, 2 Lap_h rho^k, 0)
//   CDFT  g = (rho):             N0 = rho - s Lap_h (ln rho + 2 c_e rho)
//         S = rho^k + s Lap_h E,  E = -(2 c_e rho^k + J * rho^k)
// (J * rho^k by the FFT of fm_fft.cu).  As in fm_solver.cu: a float64 outer
// loop r = S - N(g), one FAS V-cycle per iteration on the correction
// equation M(e) = N(g + e) - N(g) = r in precision T with g frozen as the
// coefficient (float32 in the mixed path), then g += e in float64; the
// whole step is one CUDA graph (fm_stepper.cuh).
//
// Point block (red-black Gauss-Seidel, App. G.3 damping of the whole block):
//   PFC   the 3x3 system of (e_rho, e_mu, e_kappa) at the point, with the
//         cubic linearised about the current density,
//           e_rho + a e_mu = b1,  e_mu - q e_rho + c e_kappa = b2,
//           e_kappa + c e_rho = b3   (a = 2 d s / h^2, c = 2 d / h^2),
//         solved in closed form (determinant 1 + a (q + c^2) > 0);
//   CDFT  one Newton step on the scalar point equation about the current
//         density (the left side is increasing in rho).
// Then the positive projection of Sec. 6 on rho.  After the solve the new
// density is re-evaluated as rho^k + s Lap_h mu^{k+1} with the converged mu,
// so mass is conserved to round-off, and projected.
#include <cuda_runtime.h>
#include <cstring>

#include "fm_state.h"
#include "fm_device.cuh"
#include "fm_stepper.cuh"

namespace fm {
namespace gf {

template <int KIND>
struct GL {
  static constexpr int NU = KIND == KPFC ? 3 : 1;
};

// Constants of one level (spacing h).
template <typename T>
struct GK {
  T ih2;   // 1/h^2
  T c;     // 2 d / h^2: diagonal of -Lap_h
  T a;     // s c
  T sih2;  // s / h^2
  T proj;  // projection threshold (see proj_threshold)
};

template <typename T, int DIM>
__device__ __forceinline__ GK<T> make_gk(const Phys<T>& P, T h) {
  GK<T> K;
  K.ih2 = T(1) / (h * h);
  K.c = T(2 * DIM) * K.ih2;
  K.a = P.s * K.c;
  K.sih2 = P.s * K.ih2;
  K.proj = proj_threshold<T>(P.delta);
  return K;
}

// Correction-form chemical potential of CDFT at idx: ln(c + e) - ln c + 2 c_e e.
template <typename T>
__device__ __forceinline__ T mcorr_gf(const T* e, const T* c, int idx, T ce) {
  const T x = e[idx];
  return log1p_t(x / c[idx]) + T(2) * ce * x;
}

// M(e) = N(c + e) - N(c) at one point (all components).
template <typename T, int KIND, int DIM>
__device__ __forceinline__ void gf_applyM(const Lvl<T>& L, const Phys<T>& P, const GK<T>& K, const Nb& n, T* M) {
  if constexpr (KIND == KPFC) {
    const T er = L.e[0][n.c], em = L.e[1][n.c], ek = L.e[2][n.c];
    const T psi = L.cr[n.c] - T(1.5);
    M[0] = er + K.a * em - K.sih2 * nbsum<T, DIM>(L.e[1], n);
    M[1] = em - er * (psi * psi + psi * er + er * er * T(1.0 / 3.0)) - P.alpha * er + K.c * ek
         - K.ih2 * nbsum<T, DIM>(L.e[2], n);
    M[2] = ek + K.c * er - K.ih2 * nbsum<T, DIM>(L.e[0], n);
  } else {
    T sm = mcorr_gf(L.e[0], L.cr, n.m[0], P.ce) + mcorr_gf(L.e[0], L.cr, n.p[0], P.ce)
         + mcorr_gf(L.e[0], L.cr, n.m[1], P.ce) + mcorr_gf(L.e[0], L.cr, n.p[1], P.ce);
    if constexpr (DIM == 3) sm += mcorr_gf(L.e[0], L.cr, n.m[2], P.ce) + mcorr_gf(L.e[0], L.cr, n.p[2], P.ce);
    M[0] = L.e[0][n.c] + K.a * mcorr_gf(L.e[0], L.cr, n.c, P.ce) - K.sih2 * sm;
  }
}

// Point-block update of one point (see the file comment), projection, damping.
template <typename T, int KIND, int DIM>
__device__ __forceinline__ void gf_smooth_point(const Lvl<T>& L, const Phys<T>& P, const GK<T>& K, const Nb& n) {
  const int c = n.c;
  const T crc = L.cr[c];
  const T w = P.w;
  if constexpr (KIND == KPFC) {
    const T eo0 = L.e[0][c], eo1 = L.e[1][c], eo2 = L.e[2][c];
    const T b1 = L.f[0][c] + K.sih2 * nbsum<T, DIM>(L.e[1], n);
    const T b3 = L.f[2][c] + K.ih2 * nbsum<T, DIM>(L.e[0], n);
    const T psc = crc - T(1.5);
    const T p = psc + eo0;                                                  // current psi
    const T cub = eo0 * (psc * psc + psc * eo0 + eo0 * eo0 * T(1.0 / 3.0));  // [(psc+e)^3 - psc^3]/3
    const T q = p * p + P.alpha;
    const T b2 = L.f[1][c] + K.ih2 * nbsum<T, DIM>(L.e[2], n) + cub - p * p * eo0;
    const T qc = q + K.c * K.c;
    const T em = (b2 + qc * b1 - K.c * b3) * rcp_blk(T(1) + K.a * qc);
    T er = b1 - K.a * em;
    {
      const T x = crc + er;
      if (x <= K.proj) er = sqrt_t(x * x + P.delta * P.delta) - crc;  // Sec. 6 projection
    }
    const T ek = b3 - K.c * er;
    L.e[0][c] = (T(1) - w) * er + w * eo0;
    L.e[1][c] = (T(1) - w) * em + w * eo1;
    L.e[2][c] = (T(1) - w) * ek + w * eo2;
  } else {
    const T eo = L.e[0][c];
    T sm = mcorr_gf(L.e[0], L.cr, n.m[0], P.ce) + mcorr_gf(L.e[0], L.cr, n.p[0], P.ce)
         + mcorr_gf(L.e[0], L.cr, n.m[1], P.ce) + mcorr_gf(L.e[0], L.cr, n.p[1], P.ce);
    if constexpr (DIM == 3) sm += mcorr_gf(L.e[0], L.cr, n.m[2], P.ce) + mcorr_gf(L.e[0], L.cr, n.p[2], P.ce);
    const T b = L.f[0][c] + K.sih2 * sm;
    // one Newton step on e + a (log1p(e/c) + 2 c_e e) = b about the current e
    const T F = eo + K.a * (log1p_t(eo / crc) + T(2) * P.ce * eo) - b;
    const T dF = T(1) + K.a * (T(1) / (crc + eo) + T(2) * P.ce);
    T en = eo - F / dF;
    {
      const T x = crc + en;
      if (x <= K.proj) en = sqrt_t(x * x + P.delta * P.delta) - crc;
    }
    L.e[0][c] = (T(1) - w) * en + w * eo;
  }
}

template <typename T, int KIND, int DIM>
__global__ void __launch_bounds__(TPB) k_gf_smooth(Lvl<T> L, Phys<T> P, int color) {
  int i, j, k;
  if (!colour_point(blockIdx.x * blockDim.x + threadIdx.x, color, L.g, i, j, k)) return;
  gf_smooth_point<T, KIND, DIM>(L, P, make_gk<T, DIM>(P, L.h), neighbours(i, j, k, L.g));
}

// r = f - M(e) on a level.
template <typename T, int KIND, int DIM>
__global__ void __launch_bounds__(TPB) k_gf_resid(Lvl<T> L, Phys<T> P) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= L.g.N) return;
  constexpr int NU = GL<KIND>::NU;
  int i, j, k;
  coords(idx, L.g, i, j, k);
  T M[NU], fv[NU];
#pragma unroll
  for (int q = 0; q < NU; ++q) fv[q] = L.f[q][idx];
  gf_applyM<T, KIND, DIM>(L, P, make_gk<T, DIM>(P, L.h), neighbours(i, j, k, L.g), M);
#pragma unroll
  for (int q = 0; q < NU; ++q) L.r[q][idx] = fv[q] - M[q];
}

// f_C = FW(r_F), e_C = eh_C = inject(e_F) (the generic transfer of the cycle).
template <typename T, int NU, int DIM>
__global__ void __launch_bounds__(TPB) k_gf_restrict(Lvl<T> F, Lvl<T> C) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < C.g.N) restrict_point<T, NU, DIM>(F, C, idx);
}

// f_C += M_C(e_C): the coarse right-hand side of FAS (e_C = the injection).
template <typename T, int KIND, int DIM>
__global__ void __launch_bounds__(TPB) k_gf_coarse_rhs(Lvl<T> C, Phys<T> P) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= C.g.N) return;
  constexpr int NU = GL<KIND>::NU;
  int i, j, k;
  coords(idx, C.g, i, j, k);
  T M[NU], fv[NU];
#pragma unroll
  for (int q = 0; q < NU; ++q) fv[q] = C.f[q][idx];
  gf_applyM<T, KIND, DIM>(C, P, make_gk<T, DIM>(P, C.h), neighbours(i, j, k, C.g), M);
#pragma unroll
  for (int q = 0; q < NU; ++q) C.f[q][idx] = fv[q] + M[q];
}

template <typename T, int NU, int DIM>
__global__ void __launch_bounds__(TPB) k_gf_prolong(Lvl<T> F, Lvl<T> C, Phys<T> P) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < F.g.N) prolong_point<T, NU, DIM>(F, C, P, idx);
}

// ---------------------------------------------------------------------------
// float64 kernels of the finest level
// ---------------------------------------------------------------------------
struct GF64 {
  const double* rho;   // rho^k
  const double* conv;  // J * rho^k (CDFT)
  double* emu;         // CDFT: E = -(2 c_e rho^k + J * rho^k)
  double* m;           // CDFT: ln g0 + 2 c_e g0 of the current iterate (scratch)
  double* S[3];
  double* g[3];
  int* nonpos;         // CDFT: set where a density <= 0 would reach ln
};

// PFC: S = (rho^k, 2 Lap rho^k, 0), g = (rho^k, ., Lap rho^k).
// CDFT: E, g0 = rho^k.
template <int KIND, int DIM>
__global__ void __launch_bounds__(TPB) k_gf_prepare(GF64 F, Geo G, double ih2, double ce) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= G.N) return;
  const double rk = F.rho[idx];
  if constexpr (KIND == KPFC) {
    int i, j, k;
    coords(idx, G, i, j, k);
    const Nb n = neighbours(i, j, k, G);
    const double lap = (nbsum<double, DIM>(F.rho, n) - 2.0 * DIM * rk) * ih2;
    F.S[0][idx] = rk;
    F.S[1][idx] = 2.0 * lap;
    F.S[2][idx] = 0.0;
    F.g[0][idx] = rk;
    F.g[2][idx] = lap;
  } else {
    if (F.nonpos && rk <= 0.0) atomicOr(F.nonpos, 1);
    F.emu[idx] = -(2.0 * ce * rk + F.conv[idx]);
    F.g[0][idx] = rk;
  }
}

// PFC: mu^0 = psi^3/3 + alpha psi + Lap kappa^0 + S_mu.  CDFT: S0 = rho^k + s Lap E.
template <int KIND, int DIM>
__global__ void __launch_bounds__(TPB) k_gf_prepare2(GF64 F, Geo G, double ih2, double alpha, double s) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= G.N) return;
  int i, j, k;
  coords(idx, G, i, j, k);
  const Nb n = neighbours(i, j, k, G);
  if constexpr (KIND == KPFC) {
    const double psi = F.rho[idx] - 1.5;
    const double lapk = (nbsum<double, DIM>(F.g[2], n) - 2.0 * DIM * F.g[2][idx]) * ih2;
    F.g[1][idx] = psi * psi * psi * (1.0 / 3.0) + alpha * psi + lapk + F.S[1][idx];
  } else {
    const double lapE = (nbsum<double, DIM>(F.emu, n) - 2.0 * DIM * F.emu[idx]) * ih2;
    F.S[0][idx] = F.rho[idx] + s * lapE;
  }
}

// CDFT: m = ln g0 + 2 c_e g0 of the iterate (one logarithm per point).
__global__ void __launch_bounds__(TPB) k_gf_m64(GF64 F, int N, double ce) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= N) return;
  const double r = F.g[0][idx];
  F.m[idx] = log(r) + 2.0 * ce * r;
}

// r = S - N(g) in float64, the level-0 set-up of a cycle (f0 = r in T, e0 =
// 0, the coefficient density in float for the mixed path) and the block
// partial sums of r^2 (grid-stride loop, fixed order).
template <int KIND, int DIM, typename T>
__global__ void __launch_bounds__(TPB) k_gf_resid64(GF64 F, Resid64Out O, Geo G, double ih2, double s, double alpha,
                                                    double* partials) {
  constexpr int NU = GL<KIND>::NU;
  double acc[NU];
  float fa[NU];
#pragma unroll
  for (int q = 0; q < NU; ++q) {
    acc[q] = 0.0;
    fa[q] = 0.0f;
  }
  const double c = 2.0 * DIM * ih2;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < G.N; idx += gridDim.x * blockDim.x) {
    int i, j, k;
    coords(idx, G, i, j, k);
    const Nb n = neighbours(i, j, k, G);
    double r[NU];
    const double g0 = F.g[0][idx];
    if constexpr (KIND == KPFC) {
      const double g1 = F.g[1][idx], g2 = F.g[2][idx];
      const double psi = g0 - 1.5;
      const double N0 = g0 + s * c * g1 - s * ih2 * nbsum<double, DIM>(F.g[1], n);
      const double N1 = g1 - psi * (psi * psi * (1.0 / 3.0) + alpha) + c * g2 - ih2 * nbsum<double, DIM>(F.g[2], n);
      const double N2 = g2 + c * g0 - ih2 * nbsum<double, DIM>(F.g[0], n);
      r[0] = F.S[0][idx] - N0;
      r[1] = F.S[1][idx] - N1;
      r[2] = F.S[2][idx] - N2;
    } else {
      const double N0 = g0 + s * c * F.m[idx] - s * ih2 * nbsum<double, DIM>(F.m, n);
      r[0] = F.S[0][idx] - N0;
    }
#pragma unroll
    for (int q = 0; q < NU; ++q) {
      norm_add<T>(O.f0[q], r[q], acc[q], fa[q], idx);
      if (O.e0[q]) static_cast<T*>(O.e0[q])[idx] = T(0);
      if (O.r64[q]) O.r64[q][idx] = r[q];
    }
    if (O.cr32) O.cr32[idx] = narrow_rn(g0);
  }
  norm_partials<T, NU>(O.f0[0], acc, fa, partials, blockIdx.x);
}

// rho^{k+1} = rho^k + s Lap_h mu with mu = g1 (PFC) or m + E (CDFT), projected;
// skipped unless the solve succeeded.
template <int KIND, int DIM>
__global__ void __launch_bounds__(TPB) k_gf_closure(GF64 F, Geo G, double ih2, double s, double delta, double* out,
                                                    const Ctl* ctl) {
  if (ctl->status != FM_OK) return;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= G.N) return;
  int i, j, k;
  coords(idx, G, i, j, k);
  const Nb n = neighbours(i, j, k, G);
  double lap;
  if constexpr (KIND == KPFC) {
    lap = (nbsum<double, DIM>(F.g[1], n) - 2.0 * DIM * F.g[1][idx]) * ih2;
  } else {
    const double mc = F.m[idx] + F.emu[idx];
    double nb = 0.0;
#pragma unroll
    for (int d = 0; d < DIM; ++d) nb += F.m[n.m[d]] + F.emu[n.m[d]] + F.m[n.p[d]] + F.emu[n.p[d]];
    lap = (nb - 2.0 * DIM * mc) * ih2;
  }
  const double r = F.rho[idx] + s * lap;
  out[idx] = (delta > 0.0) ? sqrt(r * r + delta * delta) : fabs(r);
}

__global__ void __launch_bounds__(TPB) k_gf_commit(double* rho, const double* rnew, int N, const Ctl* ctl) {
  if (ctl->status != FM_OK) return;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < N) rho[idx] = rnew[idx];
}

// ---------------------------------------------------------------------------
// Host driver
// ---------------------------------------------------------------------------
template <typename T, int KIND, int DIM>
struct GFSolver {
  static constexpr int NU = GL<KIND>::NU;
  static constexpr int NVEL = 0;

  static GF64 fields(fm_state* st) {
    GF64 F;
    F.rho = st->rho;
    F.conv = st->conv;
    F.emu = st->emu;
    F.m = st->tmp;
    for (int q = 0; q < 3; ++q) {
      F.S[q] = q < NU ? st->S[q] : nullptr;
      F.g[q] = q < NU ? st->g[q] : nullptr;
    }
    F.nonpos = KIND == KCDFT ? &static_cast<Ctl*>(st->ctl)->nonpos : nullptr;
    return F;
  }

  static Resid64Out out0(fm_state* st, bool cycle, double* const* r64) {
    Resid64Out O;
    memset(&O, 0, sizeof(O));
    for (int q = 0; q < NU; ++q) {
      O.f0[q] = cycle ? st->lv[0].f[q] : nullptr;
      O.e0[q] = cycle ? st->lv[0].e[q] : nullptr;
      O.r64[q] = r64 ? r64[q] : nullptr;
    }
    if (cycle && st->prm.precision == FM_MIXED) O.cr32 = (float*)st->lv[0].cr;
    return O;
  }

  static double ih2(const fm_state* st) { return 1.0 / (st->lv[0].h * st->lv[0].h); }

  static int enqueue_prepare(fm_state* st) {
    const Geo G = st->lv[0].g;
    cudaStream_t s = st->stream;
    if (KIND == KCDFT) {
      FM_CUDA(cudaMemsetAsync(&static_cast<Ctl*>(st->ctl)->nonpos, 0, sizeof(int), s));
      const int rc = fft_convolve(st, st->rho, st->conv);
      if (rc) return rc;
    }
    const GF64 F = fields(st);
    k_gf_prepare<KIND, DIM><<<nblocks(G.N), TPB, 0, s>>>(F, G, ih2(st), st->ce);
    FM_LAUNCHED();
    k_gf_prepare2<KIND, DIM><<<nblocks(G.N), TPB, 0, s>>>(F, G, ih2(st), st->fn.alpha, st->dt);
    FM_LAUNCHED();
    return FM_OK;
  }

  static int launch_resid64(fm_state* st, const Resid64Out& O) {
    const Geo G = st->lv[0].g;
    cudaStream_t s = st->stream;
    const GF64 F = fields(st);
    if (KIND == KCDFT) {
      k_gf_m64<<<nblocks(G.N), TPB, 0, s>>>(F, G.N, st->ce);
      FM_LAUNCHED();
    }
    k_gf_resid64<KIND, DIM, T><<<st->nblk, TPB, 0, s>>>(F, O, G, ih2(st), st->dt, st->fn.alpha, st->partials);
    FM_LAUNCHED();
    return FM_OK;
  }

  static int enqueue_resid_norm(fm_state* st, int in_body, cudaGraphConditionalHandle hdl, int use_handle) {
    int rc = launch_resid64(st, out0(st, true, nullptr));
    if (rc) return rc;
    const double h = st->lv[0].h;
    const double w = DIM == 3 ? h * h * h : h * h;
    k_norm_ctl<NU><<<1, TPB, 0, st->stream>>>(st->partials, st->nblk, w, (Ctl*)st->ctl, st->prm.tol,
                                              st->prm.max_cycles, in_body, hdl, use_handle);
    FM_LAUNCHED();
    return FM_OK;
  }

  static int smooth(fm_state* st, const Lvl<T>& L, const Phys<T>& P, int iters) {
    for (int it = 0; it < iters; ++it)
      for (int color = 0; color < 2; ++color) {
        k_gf_smooth<T, KIND, DIM><<<nblocks(L.g.N / 2), TPB, 0, st->stream>>>(L, P, color);
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
    k_gf_resid<T, KIND, DIM><<<nblocks(F.g.N), TPB, 0, s>>>(F, P);
    FM_LAUNCHED();
    k_gf_restrict<T, NU, DIM><<<nblocks(C.g.N), TPB, 0, s>>>(F, C);
    FM_LAUNCHED();
    k_gf_coarse_rhs<T, KIND, DIM><<<nblocks(C.g.N), TPB, 0, s>>>(C, P);
    FM_LAUNCHED();
    rc = vcycle(st, l + 1, P);
    if (rc) return rc;
    k_gf_prolong<T, NU, DIM><<<nblocks(F.g.N), TPB, 0, s>>>(F, C, P);
    FM_LAUNCHED();
    return smooth(st, F, P, st->prm.nu2);
  }

  // The coefficient density of level 0 (precision T) down the hierarchy.
  static int inject_coefficient(fm_state* st) {
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
    A.src[0] = (const T*)st->lv[0].cr;
    for (int l = 1; l < st->nlev; ++l) A.dst[l][0] = (T*)st->lv[l].cr;
    A.nsrc = 1;
    k_inject_all<T><<<nblocks(A.off[st->nlev]), TPB, 0, st->stream>>>(A);
    FM_LAUNCHED();
    return FM_OK;
  }

  static int enqueue_body(fm_state* st, cudaGraphConditionalHandle hdl, int use_handle) {
    int rc = inject_coefficient(st);
    if (rc) return rc;
    rc = vcycle(st, 0, make_phys<T>(st));
    if (rc) return rc;
    const Geo G = st->lv[0].g;
    Fields64 F;
    memset(&F, 0, sizeof(F));
    for (int q = 0; q < NU; ++q) F.g[q] = st->g[q];
    F.nonpos = KIND == KCDFT ? &static_cast<Ctl*>(st->ctl)->nonpos : nullptr;
    k_update64<NU, T><<<nblocks(G.N), TPB, 0, st->stream>>>(F, out0(st, true, nullptr), G.N, st->prm.delta);
    FM_LAUNCHED();
    return enqueue_resid_norm(st, 1, hdl, use_handle);
  }

  static int enqueue_post(fm_state* st) {
    const Geo G = st->lv[0].g;
    const GF64 F = fields(st);
    const Ctl* ctl = (const Ctl*)st->ctl;
    k_gf_closure<KIND, DIM><<<nblocks(G.N), TPB, 0, st->stream>>>(F, G, ih2(st), st->dt, st->prm.delta,
                                                                   st->r64[0], ctl);
    FM_LAUNCHED();
    k_gf_commit<<<nblocks(G.N), TPB, 0, st->stream>>>(st->rho, st->r64[0], G.N, ctl);
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

  // fm_residual: r = S - N(g) of the caller's iterate (already in st->g).
  static int residual64(fm_state* st, double* const* r64, double* norm_host) {
    int rc = launch_resid64(st, out0(st, false, r64));
    if (rc) return rc;
    const double h = st->lv[0].h;
    const double w = DIM == 3 ? h * h * h : h * h;
    k_norm_final<NU><<<1, TPB, 0, st->stream>>>(st->partials, st->nblk, w, st->dscal);
    FM_LAUNCHED();
    FM_CUDA(cudaMemcpyAsync(st->hscal, st->dscal, sizeof(double), cudaMemcpyDeviceToHost, st->stream));
    FM_CUDA(cudaStreamSynchronize(st->stream));
    *norm_host = st->hscal[0];
    return FM_OK;
  }
};

template <typename T, int KIND>
static int dispatch(fm_state* st, int what, fm_step_info* info, const double* ri, double* ro, double* const* r64,
                    double* nrm) {
  switch (what) {
    case 0: return st->dim == 2 ? Stepper<GFSolver<T, KIND, 2>>::step(st, info)
                                : Stepper<GFSolver<T, KIND, 3>>::step(st, info);
    case 1: return st->dim == 2 ? Stepper<GFSolver<T, KIND, 2>>::step_host(st, ri, nullptr, ro, nullptr, info)
                                : Stepper<GFSolver<T, KIND, 3>>::step_host(st, ri, nullptr, ro, nullptr, info);
    case 2: return st->dim == 2 ? GFSolver<T, KIND, 2>::prepare(st) : GFSolver<T, KIND, 3>::prepare(st);
    default: return st->dim == 2 ? GFSolver<T, KIND, 2>::residual64(st, r64, nrm)
                                 : GFSolver<T, KIND, 3>::residual64(st, r64, nrm);
  }
}

static int run(fm_state* st, int what, fm_step_info* info, const double* ri, double* ro, double* const* r64,
               double* nrm) {
  if (st->prm.precision == FM_MIXED)
    return st->kind == FM_PFC ? dispatch<float, KPFC>(st, what, info, ri, ro, r64, nrm)
                              : dispatch<float, KCDFT>(st, what, info, ri, ro, r64, nrm);
  return st->kind == FM_PFC ? dispatch<double, KPFC>(st, what, info, ri, ro, r64, nrm)
                            : dispatch<double, KCDFT>(st, what, info, ri, ro, r64, nrm);
}

}  // namespace gf

int gf_step(fm_state* st, fm_step_info* info) { return gf::run(st, 0, info, nullptr, nullptr, nullptr, nullptr); }
int gf_step_host(fm_state* st, const double* rho_in, double* rho_out, fm_step_info* info) {
  return gf::run(st, 1, info, rho_in, rho_out, nullptr, nullptr);
}
int gf_prepare(fm_state* st) { return gf::run(st, 2, nullptr, nullptr, nullptr, nullptr, nullptr); }
int gf_residual(fm_state* st, double* const* r64, double* norm) {
  return gf::run(st, 3, nullptr, nullptr, nullptr, r64, norm);
}

}  // namespace fm
