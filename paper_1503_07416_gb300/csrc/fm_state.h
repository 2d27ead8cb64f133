// Host-side state of one solver instance (shared by the libfm translation
// units).  All device buffers live in one arena allocated at fm_create.
#pragma once

#include <cuda_runtime.h>
#include "../../include/fm.h"
#include "fm_internal.cuh"

namespace fm {

constexpr int MAXLEV = 16;
constexpr int MAXEV = 64;     // profiling events (pairs) per outer iteration

struct LevelBufs {
  Geo g;
  double h;
  void* e[MAXU];
  void* f[MAXU];
  void* r[MAXU];
  void* eh[MAXU];
  void* rk;        // precision-T rho^k (level 0 of the FP64 path: aliases st.rho)
  void* om[3];
  void* cr;        // precision-T coefficient iterate (level 0 FP64: aliases st.g)
  void* cv[3];
};

struct FFTBufs {
  double2* Jhat;       // transform of h^d J / N (scaled so that the inverse needs no scale)
  double* Jr;          // its real part at kx = 0 .. nx/2 (the real-input convolution; rows of nx/2 + 1)
  double2* work;       // complex work array, N values
  double2* tw[3];      // twiddles exp(-2 pi i k / n_d), k < n_d / 2
};

}  // namespace fm

struct fm_state {
  fm_grid grid;
  fm_params prm;
  fm_functional fn;
  int model;                      // FM_HYDRO or FM_GRADFLOW
  int kind, dim, nu, nom, nlev;
  int elem;                       // sizeof(T) of the hierarchy
  fm::LevelBufs lv[fm::MAXLEV];
  fm::LevelBufs lv64[fm::MAXLEV];  // mixed path, coarse_precision FM_FP64: float64 copies of the coarse levels
  bool coarse64;                   // the coarsest-grid solve runs on lv64 (levels small_from .. nlev - 1)
  // float64 finest-level fields
  double* rho;
  double* vel[3];
  double* g[fm::MAXU];
  double* gp[fm::MAXU];           // FM_INIT_EXTRAPOLATE: converged iterate of the step before
  double* S[fm::MAXU];
  double* om[3];
  double* conv;                   // J * rho^k (CDFT)
  double* emu;                    // gradient flow, CDFT: -(2 c_e rho^k + J * rho^k)
  double* tmp;                    // float64 scratch of N values
  double* r64[fm::MAXU];          // float64 residual scratch (row-level entry points)
  double* x64[5];                 // 3-D: per-point quantities shared by the residual
  double* partials;               // per-block partial sums (deterministic reductions)
  int nblk;                       // blocks of the reduction kernels
  int sms;                        // multiprocessors of the device
  int smem_optin;                 // shared memory per block (opt-in maximum)
  double* dscal;                  // device scalars
  double* hscal;                  // pinned host mirror of dscal
  double ce;                      // (J_e * 1) (CDFT)
  fm::FFTBufs fft;
  double dt;                      // step of the last fm_prepare
  double hist_dt;                 // step size the kept converged iterates belong to
  bool prepared;
  cudaStream_t stream;
  cudaStream_t cap[2];            // private streams used to capture the step graph
  bool capturing;
  bool use_graph;                 // run fm_step as one CUDA graph launch
  bool fused_rb;                  // 2-D: one tiled launch per red-black sweep
  bool coarse_fused;              // the coarsest level alone exceeds one block's share: multi-block sweeps
  int rbv[fm::MAXLEV];            // chosen variant of the fused sweep per level
  float rbt[fm::MAXLEV][FM_SWEEP_VARIANTS];  // autotuner timings (ms per sweep)
  int small_from;                 // first level handled by the single-block V-cycle
  void* ctl;                      // device control block of the step
  cudaGraph_t graph;
  cudaGraphExec_t gexec;
  double graph_dt;                // step size the graph was captured with
  long long cnt_pre, cnt_body, cnt_post;  // kernels per graph part (launch accounting)
  long long launches;             // kernels launched by this state
  bool prof;                      // time the finest-level smoother launches
  bool pev_ready;
  cudaEvent_t pev[fm::MAXEV];
  int npev;
  double prof_ms;
  long long prof_count;
  void* arena;
  size_t arena_bytes;
};

namespace fm {
// fm_gradflow.cu: the gradient-flow model (fm_params.model = FM_GRADFLOW)
int gf_step(fm_state* st, fm_step_info* info);
int gf_step_host(fm_state* st, const double* rho_in, double* rho_out, fm_step_info* info);
int gf_prepare(fm_state* st);
int gf_residual(fm_state* st, double* const* r64, double* norm);
// fm_channel.cu: the 2-D PFC channel (fm_params.walls = FM_WALLS_Y)
int ch_step(fm_state* st, fm_step_info* info);
int ch_step_host(fm_state* st, const double* rho_in, const double* const* vel_in, double* rho_out,
                 double* const* vel_out, fm_step_info* info);
int ch_prepare(fm_state* st);
int ch_residual(fm_state* st, double* const* r64, double* norm);
int ch_energy_launch(fm_state* st);  // energy partial sums (Neumann Laplacian) into st->partials
// fm_fft.cu
int fft_init(fm_state* st);                                    // twiddles, J, c_e, Jhat
int fft_convolve(fm_state* st, const double* rho, double* out);  // out = J * rho
}  // namespace fm
